// fea_assemble with the chunked scatter for the scalar forms: the chunk
// kernel of the element order (scalar_chunk_p1.cu, scalar_chunk_p2.cu), then
// the chunk-ordered sums of the shared couplings and shared loads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "scalar_chunk.cuh"

namespace fea {
namespace {

using namespace chunkfx;

// The couplings shared by several chunks: their partial sums, contiguous and
// in chunk order; the sum goes to entry (i, j) and to (j, i).
__global__ void k_chunk_reduce_scalar(const int32_t* __restrict__ gptr, const int4* __restrict__ grec, int64_t ngroup,
                                      const double* __restrict__ part, double* __restrict__ values) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroup) return;
  const int32_t p0 = gptr[g], p1 = gptr[g + 1];
  double v = part[p0];
  for (int32_t p = p0 + 1; p < p1; ++p) v += part[p];
  const int4 rec = grec[g];
  values[rec.x] = v;
  if (rec.y != rec.x) values[rec.y] = v;
}

// The loads of dofs shared by several chunks.
__global__ void k_chunk_reduce_dofs(const int32_t* __restrict__ gptr, const int32_t* __restrict__ gdof, int64_t ngroup,
                                    const double* __restrict__ npart, double* __restrict__ rhs) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroup) return;
  const int32_t p0 = gptr[g], p1 = gptr[g + 1];
  double f = npart[p0];
  for (int32_t p = p0 + 1; p < p1; ++p) f += npart[p];
  rhs[gdof[g]] = f;
}

__global__ void k_zero_dofs(const int32_t* __restrict__ dofs, int64_t n, double* __restrict__ rhs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rhs[dofs[i]] = 0.0;
}

}  // namespace

fea_status assemble_chunked_scalar(fea_mesh* m, Pattern* P, const fea_form* form, const fea_coeffs* co,
                                   const fea_quadrature* q, int load, double* values, double* rhs, cudaStream_t s) {
  FEA_TRY(build_chunks(m, P, s));
  const Chunks* K = P->chunks;
  FEA_TRY(ensure_scratch(m->part, (size_t)std::max<int64_t>(K->npart, 1) * sizeof(double)));
  if (rhs) FEA_TRY(ensure_scratch(m->npart, (size_t)std::max<int64_t>(K->nnpart, 1) * sizeof(double)));
  ElemArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.N = m->n_nodes;
  A.E = m->n_elems;
  A.kappa = co->kappa;
  A.kappa_const = co->kappa_const;
  A.mass = form->mass_coef;
  for (int i = 0; i < 4; ++i) A.fp[i] = co->f_param[i];
  A.err = m->err;
  ChunkArgs Cg{};
  Cg.cptr = K->cptr;
  Cg.celem = K->celem;
  Cg.eslot = K->eslot;
  Cg.es = K->estride;
  Cg.sptr = K->sptr;
  Cg.nptr = K->nptr;
  Cg.srec = K->srec;
  Cg.nrec = K->nrec;
  Cg.H = 63 - 2 * K->hbits;
  Cg.K = 32 - K->hbits;
  const int ld = rhs ? load : LOAD_NONE;
  // |f| < 2^ef: the amplitude of the scalar load
  Cg.ef = EXP_ZERO;
  if (ld != LOAD_NONE) {
    const double a = std::fabs(co->f_param[0]);
    if (!std::isfinite(a)) Cg.ef = EXP_POISON;
    else if (a > 0.0) std::frexp(a, &Cg.ef);
  }
  Cg.max_slots = K->max_slots;
  Cg.max_nodes = K->max_nodes;
  Cg.values = values;
  Cg.rhs = rhs;
  Cg.part = static_cast<double*>(m->part.ptr);
  Cg.npart = rhs ? static_cast<double*>(m->npart.ptr) : nullptr;
  const size_t smem = (size_t)K->max_slots * 3 * sizeof(int) + (size_t)K->max_nodes * 3 * sizeof(int);
  const bool mass = form->kind == FEA_DIFFUSION_MASS && form->mass_coef != 0.0;
  const bool mixed = q->prec == FEA_MIXED;
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[0], s));
  if (K->nchunk > 0) {
    if (form->order == 1) FEA_TRY(launch_scalar_chunk_p1(mass, ld, q->npts, mixed, A, Cg, K->nchunk, smem, s));
    else FEA_TRY(launch_scalar_chunk_p2(mass, ld, q->npts, mixed, A, Cg, K->nchunk, smem, s));
  }
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[1], s));
  if (K->ngroup > 0)
    k_chunk_reduce_scalar<<<(unsigned)((K->ngroup + 255) / 256), 256, 0, s>>>(K->gptr, K->grec, K->ngroup, Cg.part,
                                                                               values);
  if (rhs && K->niso > 0) k_zero_dofs<<<(unsigned)((K->niso + 255) / 256), 256, 0, s>>>(K->iso, K->niso, rhs);
  if (rhs && K->nngroup > 0)
    k_chunk_reduce_dofs<<<(unsigned)((K->nngroup + 255) / 256), 256, 0, s>>>(K->ngptr, K->ngnode, K->nngroup,
                                                                              Cg.npart, rhs);
  FEA_CUDA(cudaGetLastError());
  if (m->profile) {
    FEA_CUDA(cudaEventRecord(m->ev[2], s));
    m->profiled = true;
  }
  return FEA_OK;
}

}  // namespace fea
