// fea_assemble: element kernel (local matrices and loads into per-element
// scratch) followed by the deterministic row-gather scatter into CSR.
#include <cuda_runtime.h>

#include <algorithm>

#include "elem_kernels.cuh"
#include "gather.cuh"
#include "gather_tiled.cuh"

namespace fea {

namespace {

template <int NB, int NDPN, typename LT>
fea_status gather_one(const GatherArgs& G, int rows, int64_t max_tile_nnz, cudaStream_t s, const int32_t* tiles,
                      int64_t ntiles, bool deep) {
  const size_t smem = (size_t)max_tile_nnz * sizeof(double);
  static size_t configured = 0;  // opt-in above the 48 KB default, once per instance
  if (smem > 48 * 1024 && smem > configured) {
    FEA_CUDA(cudaFuncSetAttribute(k_gather<NB, NDPN, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FEA_CUDA(cudaFuncSetAttribute(k_gather_list<NB, NDPN, LT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    FEA_CUDA(cudaFuncSetAttribute(k_gather_list<NB, NDPN, LT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    configured = smem;
  }
  if (tiles) {
    if (ntiles > 0) {
      if (deep) k_gather_list<NB, NDPN, LT, true><<<(unsigned)ntiles, rows, smem, s>>>(G, tiles);
      else k_gather_list<NB, NDPN, LT, false><<<(unsigned)ntiles, rows, smem, s>>>(G, tiles);
    }
  } else {
    const int64_t n = (G.ndof + rows - 1) / rows;
    if (n > 0) k_gather<NB, NDPN, LT><<<(unsigned)n, rows, smem, s>>>(G);
  }
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

}  // namespace

fea_status launch_gather(int nb, int ndpn, bool mixed, const GatherArgs& G, int rows, int64_t max_tile_nnz,
                         cudaStream_t s, const int32_t* tiles, int64_t ntiles, bool deep) {
  if (nb == 3 && ndpn == 1 && !mixed) return gather_one<3, 1, double>(G, rows, max_tile_nnz, s, tiles, ntiles, deep);
  if (nb == 4 && ndpn == 1)
    return mixed ? gather_one<4, 1, float>(G, rows, max_tile_nnz, s, tiles, ntiles, deep)
                 : gather_one<4, 1, double>(G, rows, max_tile_nnz, s, tiles, ntiles, deep);
  if (nb == 10 && ndpn == 1)
    return mixed ? gather_one<10, 1, float>(G, rows, max_tile_nnz, s, tiles, ntiles, deep)
                 : gather_one<10, 1, double>(G, rows, max_tile_nnz, s, tiles, ntiles, deep);
  if (nb == 4 && ndpn == 3)
    return mixed ? gather_one<4, 3, float>(G, rows, max_tile_nnz, s, tiles, ntiles, deep)
                 : gather_one<4, 3, double>(G, rows, max_tile_nnz, s, tiles, ntiles, deep);
  return fail(FEA_ERR_ARG, "no scatter for this element / dof layout");
}

namespace {

// The rows of more than 255 entries (whose column slots do not fit a byte),
// one block per row, after the row-gather scatter: every local row of the
// row's incidences, in ascending element order, added into a shared-memory
// copy of the row at the columns found by binary search; between two
// incidences a barrier, so each entry sums its contributions in element
// order (deterministic, no atomics).  Overwrites what the row-gather wrote
// for these rows; their loads are the row-gather's.
template <typename LT>
__global__ void __launch_bounds__(256) k_long_rows(const int32_t* __restrict__ rows, const int32_t* __restrict__ rp,
                                                   const int32_t* __restrict__ ci, const int32_t* __restrict__ inc_ptr,
                                                   const int32_t* __restrict__ inc, const int32_t* __restrict__ edof,
                                                   int64_t E, int nb, const int32_t* __restrict__ pos,
                                                   const LT* __restrict__ Lm, int ls, double* __restrict__ values) {
  extern __shared__ double lacc[];
  const int32_t row = rows[blockIdx.x];
  const int32_t r0 = rp[row], len = rp[row + 1] - r0;
  for (int j = threadIdx.x; j < len; j += blockDim.x) lacc[j] = 0.0;
  __syncthreads();
  for (int32_t t = inc_ptr[row]; t < inc_ptr[row + 1]; ++t) {
    const int32_t v = inc[t];
    const int64_t e = v / nb;
    const int a = v - (int)e * nb;
    if ((int)threadIdx.x < nb) {
      const int32_t d = edof[threadIdx.x * E + e];
      int32_t lo = 0, hi = len;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (ci[r0 + mid] < d) lo = mid + 1;
        else hi = mid;
      }
      lacc[lo] += static_cast<double>(Lm[(int64_t)pos[(int64_t)a * E + e] * ls + threadIdx.x]);
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < len; j += blockDim.x) values[r0 + j] = lacc[j];
}

fea_status long_rows(const Base* B, const Pattern* P, int64_t E, bool mixed, const int32_t* pos, const void* Lm,
                     double* values, cudaStream_t s) {
  if (B->nlong == 0) return FEA_OK;
  const size_t smem = (size_t)B->max_row * sizeof(double);
  if (mixed) {
    FEA_CUDA(cudaFuncSetAttribute(k_long_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_long_rows<float><<<(unsigned)B->nlong, 256, smem, s>>>(B->long_rows, P->row_ptr, P->col_idx, B->inc_ptr, B->inc,
                                                             B->edof, E, B->nb, pos, static_cast<const float*>(Lm),
                                                             lstride(B->nb, sizeof(float)), values);
  } else {
    FEA_CUDA(cudaFuncSetAttribute(k_long_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_long_rows<double><<<(unsigned)B->nlong, 256, smem, s>>>(B->long_rows, P->row_ptr, P->col_idx, B->inc_ptr,
                                                              B->inc, B->edof, E, B->nb, pos,
                                                              static_cast<const double*>(Lm),
                                                              lstride(B->nb, sizeof(double)), values);
  }
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

fea_status launch_elements(const fea_form* form, const ElemArgs& A, int load, int npts, int prec, cudaStream_t s) {
  if (form->kind == FEA_ELASTICITY) return launch_elem_elast(A, load, npts, prec, s);
  const bool mass = form->kind == FEA_DIFFUSION_MASS && form->mass_coef != 0.0;
  return form->order == 1 ? launch_elem_p1(A, mass, load, npts, prec, s) : launch_elem_p2(A, mass, load, npts, prec, s);
}

}  // namespace

fea_status assemble(fea_mesh* m, const fea_form* form, const fea_coeffs* co, const fea_quadrature* q,
                    double* values, double* rhs, cudaStream_t s) {
  if (m->nvert != 4) return fail(FEA_ERR_ARG, "fea_assemble takes tetrahedral meshes (use fea_assemble_2d)");
  const int order = form->order;
  const int ndpn = form->kind == FEA_ELASTICITY ? 3 : 1;
  Pattern* P = m->pat[order][ndpn];
  Base* B = m->base[order];
  if (!P || !B) return fail(FEA_ERR_STATE, "fea_assemble: build the pattern with fea_pattern first");
  // the chunked fixed-point scatter: requested, or automatic (elasticity)
  // when its chunks can be built for this mesh
  const bool chunked = m->scatter == FEA_SCATTER_CHUNKED ||
                       (m->scatter == FEA_SCATTER_AUTO && form->kind == FEA_ELASTICITY && !P->chunks_failed);
  if (chunked) {
    const int ld = rhs ? co->f_kind : FEA_LOAD_NONE;
    const fea_status st = form->kind == FEA_ELASTICITY ? assemble_chunked(m, P, co, q, ld, values, rhs, s)
                                                       : assemble_chunked_scalar(m, P, form, co, q, ld, values, rhs, s);
    if (st == FEA_OK || m->scatter == FEA_SCATTER_CHUNKED || !P->chunks_failed) return st;
    set_error("");  // automatic mode: the chunks cannot be built, take the local rows
  }
  if (B->nlong > 0 && ndpn != 1)
    return fail(FEA_ERR_OVERFLOW, "rows of more than 255 scalar entries: the local-row scatter takes them for scalar "
                                  "forms (elasticity: the chunked scatter)");
  const int nb = B->nb, nl = nb * ndpn;
  const bool mixed = q->prec == FEA_MIXED;
  const size_t rb = mixed ? sizeof(float) : sizeof(double);
  const int64_t E = m->n_elems;
  const int load = rhs ? co->f_kind : FEA_LOAD_NONE;
  const int stages = std::min(std::max(m->stages, 1), 16);
  const bool sequential = stages == 1 || E < (int64_t)stages * ELEM_T;
  // local rows in the tiled layout (bulk-copy scatter, scalar forms) or in
  // incidence order (E * nb incidences x ndpn rows), lstride values apart
  const bool tiled = use_tiled(m, P);
  const size_t nrows_local = tiled ? (size_t)P->npos : (size_t)E * nb * ndpn;
  FEA_TRY(ensure_scratch(m->lm, nrows_local * lstride(nl, (int)rb) * rb));
  if (load != FEA_LOAD_NONE) FEA_TRY(ensure_scratch(m->fl, nrows_local * rb));

  ElemArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.N = m->n_nodes;
  A.E = E;
  A.kappa = co->kappa;
  A.kappa_const = co->kappa_const;
  A.lam = co->lame_lambda;
  A.lam_const = co->lambda_const;
  A.mu = co->lame_mu;
  A.mu_const = co->mu_const;
  A.mass = form->mass_coef;
  for (int i = 0; i < 4; ++i) A.fp[i] = co->f_param[i];
  A.ipos = tiled ? P->tpos : B->ipos;
  A.Lm = m->lm.ptr;
  A.Fl = load != FEA_LOAD_NONE ? m->fl.ptr : nullptr;
  A.err = m->err;
  const int prec = mixed ? FEA_MIXED : FEA_FP64;

  GatherArgs G{};
  G.ndof = P->ndof;
  G.row_ptr = P->row_ptr;
  G.inc_ptr = B->inc_ptr;
  G.slot = B->slot;
  G.Lm = m->lm.ptr;
  G.Fl = A.Fl;
  G.values = values;
  G.rhs = rhs;
  G.err = m->err;

  // automatic: matrix warps and load warps in one kernel for the FP64 P2 sine
  // load (its sines run on the integer pipes beside the matrix's FP64 work:
  // 0.80 against 0.85 ms fused at 64^3); the fused kernel elsewhere (P1: 0.95
  // against 1.09 ms at 96^3)
  const int split_mode = m->load_split >= 0 ? m->load_split
                         : (order == 2 && load == FEA_LOAD_SINPROD && !mixed) ? 3
                                                                                : 0;
  const bool split = split_mode > 0 && load != FEA_LOAD_NONE && form->kind != FEA_ELASTICITY &&
                     !(split_mode == 3 && mixed);
  const bool mass = form->kind == FEA_DIFFUSION_MASS && form->mass_coef != 0.0;

  if (sequential) {
    // one element launch, then one scatter launch
    A.e0 = 0;
    A.e1 = E;
    if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[0], s));
    if (!split) {
      FEA_TRY(launch_elements(form, A, load, q->npts, prec, s));
    } else if (split_mode == 3) {
      FEA_TRY(launch_elem_roles(order, mass, A, load, q->npts, s));
    } else if (split_mode == 1) {
      FEA_TRY(launch_elements(form, A, FEA_LOAD_NONE, q->npts, prec, s));
      FEA_TRY(launch_elem_load(order, A, load, q->npts, prec, s));
    } else {
      // the load kernel on the side stream, concurrent with the matrix kernel
      if (!m->side) FEA_CUDA(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
      for (int k : {15, 16})
        if (!m->chunk_ev[k]) FEA_CUDA(cudaEventCreateWithFlags(&m->chunk_ev[k], cudaEventDisableTiming));
      FEA_CUDA(cudaEventRecord(m->chunk_ev[16], s));
      FEA_CUDA(cudaStreamWaitEvent(m->side, m->chunk_ev[16], 0));
      FEA_TRY(launch_elem_load(order, A, load, q->npts, prec, m->side));
      FEA_TRY(launch_elements(form, A, FEA_LOAD_NONE, q->npts, prec, s));
      FEA_CUDA(cudaEventRecord(m->chunk_ev[15], m->side));
      FEA_CUDA(cudaStreamWaitEvent(s, m->chunk_ev[15], 0));
    }
    if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[1], s));
    int mode = m->tile_classes;
    if (tiled) mode = 3;
    // no tiled layout (vector dofs): mode 3 means the automatic incidence-order choice
    if (mode < 0 || (mode == 3 && !tiled)) mode = (P->n_heavy > 0 && P->n_light > 0) ? 2 : 0;
    if (mode == 3) {
      FEA_TRY(scatter_tiled(m, P, B, mixed, A.Lm, A.Fl, values, rhs, s));
    } else if (mode == 2) {
      FEA_TRY(launch_gather(nb, ndpn, mixed, G, P->rows_per_tile, P->max_tile_nnz, s, P->class_list,
                            P->n_heavy + P->n_light, false));
    } else if (mode == 1 && P->class_list) {
      // heavy tiles (long rows) with the deep pipeline, then light tiles with
      // their own smaller shared-memory size and the lighter kernel
      FEA_TRY(launch_gather(nb, ndpn, mixed, G, P->rows_per_tile, P->heavy_span, s, P->class_list, P->n_heavy, true));
      FEA_TRY(launch_gather(nb, ndpn, mixed, G, P->rows_per_tile, P->light_span, s, P->class_list + P->n_heavy,
                            P->n_light, false));
    } else {
      FEA_TRY(launch_gather(nb, ndpn, mixed, G, P->rows_per_tile, P->max_tile_nnz, s));
    }
  } else {
    // Overlapped: element chunk k runs on `s`; the row tiles that chunk k
    // completes are scattered on the side stream while chunk k + 1 computes.
    FEA_TRY(build_stages(m, P, stages, s));
    if (!m->side) FEA_CUDA(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
    for (int k = 0; k <= 16; ++k)
      if (!m->chunk_ev[k]) FEA_CUDA(cudaEventCreateWithFlags(&m->chunk_ev[k], cudaEventDisableTiming));
    if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[0], s));
    // the side stream must not start before the work already queued on s
    FEA_CUDA(cudaEventRecord(m->chunk_ev[16], s));
    FEA_CUDA(cudaStreamWaitEvent(m->side, m->chunk_ev[16], 0));
    for (int k = 0; k < stages; ++k) {
      A.e0 = std::min<int64_t>(E, (int64_t)k * P->chunk);
      A.e1 = std::min<int64_t>(E, (int64_t)(k + 1) * P->chunk);
      // the chunks take the fused kernel, or the matrix/load-warp kernel when
      // that is the launch mode (the other split modes apply to one launch)
      if (split && split_mode == 3) FEA_TRY(launch_elem_roles(order, mass, A, load, q->npts, s));
      else FEA_TRY(launch_elements(form, A, load, q->npts, prec, s));
      FEA_CUDA(cudaEventRecord(m->chunk_ev[k], s));
      FEA_CUDA(cudaStreamWaitEvent(m->side, m->chunk_ev[k], 0));
      const int64_t t0 = P->stage_ptr[k], t1 = P->stage_ptr[k + 1];
      if (tiled)
        FEA_TRY(scatter_tiled_list(m, P, B, mixed, A.Lm, A.Fl, values, rhs, P->tile_list + t0, t1 - t0, m->side));
      else
        FEA_TRY(launch_gather(nb, ndpn, mixed, G, P->rows_per_tile, P->max_tile_nnz, m->side, P->tile_list + t0,
                              t1 - t0));
    }
    if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[1], s));
    FEA_CUDA(cudaEventRecord(m->chunk_ev[16], m->side));
    FEA_CUDA(cudaStreamWaitEvent(s, m->chunk_ev[16], 0));
  }
  FEA_TRY(long_rows(B, P, E, mixed, A.ipos, A.Lm, values, s));
  if (m->profile) {
    FEA_CUDA(cudaEventRecord(m->ev[2], s));
    m->profiled = true;
  }
  return FEA_OK;
}

}  // namespace fea
