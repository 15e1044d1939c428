// Chunked scatter of P1 linear elasticity (one CTA per chunk of elements,
// chunks.cu): the local entries of the chunk's elements are accumulated in
// shared memory as fixed-point integers, then each coupling the chunk
// completes is written to the CSR values once, and each coupling it shares
// with other chunks as one FP64 partial sum, which k_chunk_reduce adds in
// chunk order.
//
// Why fixed point.  Eq. 3 sums, per matrix entry, the contributions of every
// element that holds both dofs.  The paper's Algorithm 1 adds them with
// floating-point atomicAdd, whose order (and result) changes from run to run.
// Integer addition is associative, so integer atomics give the same sum in
// any order: the scatter is bitwise reproducible without sorting the
// contributions, and it runs on the integer pipes and the shared-memory
// atomic units, leaving the FP64 pipe (2 DFMA per SM and clock on this part)
// to the element arithmetic.  Each slot (a node pair of the chunk) has its own
// scale 2^(H - Es): Es is the largest exponent bound of the contributing
// elements, computed before any entry is added (phase A), and H = 63 - 2 hbits
// (2^hbits: the most contributions one slot receives) leaves room for the
// contributions to add up without overflow in two 32-bit words (acc_add).  A
// contribution below the slot's resolution 2^(Es - H) is rounded to it; the
// bound is within a factor of a few hundred of the largest entry, so with
// hbits = 5 (24 tets around a vertex) that resolution is about 2^-47 of the
// largest contribution.  The sum is rounded to FP64 once.
//
// Phases of k_elast_chunk (one CTA, CHUNK_T threads, elements strided over
// the threads), after the chunk's vertex coordinates are staged in shared
// memory (and, in the FP32 instance, its element ids and dof-pair slots,
// brought in by bulk copies on the TMA engine):
//   A. per element: an upper bound on |K entry| from the Lame parameters, the
//      cofactors of J (in FP32 on edges normalised by their largest exponent,
//      the edges formed in FP32 from the staged coordinates split into two
//      floats: element_bounds_split) and det J; its exponent is max-reduced
//      into the element's ten slots (and the load bound into its four node
//      slots);
//   B. per element: the local matrix (the FP64 or FP32 arithmetic of the
//      local-row path, elast_upper), each of its 78 upper entries converted
//      at its slot's scale and atomically added into the slot's 3 x 3 block;
//      the 12 load entries likewise into the node slots;
//   C. per slot: the sums converted to FP64 (correctly rounded) and written,
//      to the CSR values (owned slots: both blocks (i, j) and (j, i), the
//      transpose of each other, so the matrix stays bitwise symmetric) or to
//      the partial-sum buffer (shared slots).
// An element with non-finite inputs, det J = 0, or a bound beyond the FP64
// range poisons its slots: their values come out NaN.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "bulkcopy.cuh"
#include "chunk_common.cuh"

namespace fea {
namespace {

using namespace chunkfx;

// Three CTAs of 128 threads per SM: at 168 registers a thread (FP64) the
// register file and the shared memory both hold three.  Sixteen warps per SM
// (two CTAs of 256 threads, registers capped at 128) measured the same for
// both precisions.
constexpr int CHUNK_T = 128;
constexpr int CHUNK_MIN_BLOCKS = 3;
// A partial sum of a shared 3 x 3 block takes 12 doubles (three whole 32-byte
// sectors, so its stores never leave a sector partly written), a partial load
// 4 (one sector).
constexpr int PART_STRIDE = 12;

// The chunk's element ids and dof-pair slots staged in shared memory by bulk
// copies (STAGE): rows of STAGE_E entries, wide enough for the largest chunk
// plus the elements before the chunk's first one that round its copies down
// to a 16-byte boundary; then the mbarrier the copies complete.
constexpr int STAGE_E = CHUNK_STAGE_E;
constexpr int STAGE_BYTES = CHUNK_STAGE_BYTES;
static_assert((STAGE_E * 4) % 16 == 0 && (STAGE_E * 2) % 16 == 0, "staged rows must start on 16-byte boundaries");

// Vertex coordinates of an element from the chunk's staged vertices.
__device__ __forceinline__ void staged_vertices(const double* sxyz, const int* slot, double X[4][3]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) X[a][d] = sxyz[3 * slot[a] + d];
}

// Phase-A bounds from the FP64 staged coordinates: the path of elements whose
// split coordinates do not serve (out of the split's range, or edges far
// below the coordinates) and of very flat elements.
static __device__ __noinline__ int2 staged_bounds_fp64(const double* sxyz, int s0, int s1, int s2, int s3, double C1,
                                                       int ef) {
  const int slot[4] = {s0, s1, s2, s3};
  double X[4][3];
  staged_vertices(sxyz, slot, X);
  return element_bounds(X, C1, 0.0, ef);
}

template <int LOAD, int NPTS, typename R, bool STAGE>
__global__ void __launch_bounds__(CHUNK_T, CHUNK_MIN_BLOCKS) k_elast_chunk(ElemArgs A, ChunkArgs C) {
  extern __shared__ __align__(16) double smem_chunk[];
  int32_t* s_ce = reinterpret_cast<int32_t*>(smem_chunk);      // STAGE: [STAGE_E] element ids
  uint16_t* s_es = reinterpret_cast<uint16_t*>(s_ce + STAGE_E); // STAGE: [10][STAGE_E] dof-pair slots
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_es + 10 * STAGE_E);
  double* sxyz = smem_chunk + (STAGE ? STAGE_BYTES / 8 : 0);   // [max_nodes][3] vertex coordinates
  unsigned* alo = reinterpret_cast<unsigned*>(sxyz + 3 * C.max_nodes);  // [max_slots][9] low words
  int* ahi = reinterpret_cast<int*>(alo + 9 * C.max_slots);     // [max_slots][9] high words
  unsigned* rlo = reinterpret_cast<unsigned*>(ahi + 9 * C.max_slots);  // [max_nodes][3]
  int* rhi = reinterpret_cast<int*>(rlo + 3 * C.max_nodes);     // [max_nodes][3]
  int* sexp = rhi + 3 * C.max_nodes;                            // [max_slots]
  int* rexp = sexp + C.max_slots;                               // [max_nodes]
  float* sxh = reinterpret_cast<float*>(rexp + C.max_nodes);    // [max_nodes][3] coordinates split into
  float* sxl = sxh + 3 * C.max_nodes;                           //   h + l (split_coord)
  uint8_t* sxok = reinterpret_cast<uint8_t*>(sxl + 3 * C.max_nodes);  // [max_nodes] the split serves
  const int c = blockIdx.x, tid = threadIdx.x;
  const int e0 = C.cptr[c], ne = C.cptr[c + 1] - e0;
  const int s0 = C.sptr[c], ns = C.sptr[c + 1] - s0;
  const int n0 = C.nptr[c], nn = C.nptr[c + 1] - n0;
  constexpr bool HAS_LOAD = LOAD != LOAD_NONE;
  // STAGE: the chunk's element ids and its ten rows of slots are copied to
  // shared memory with bulk copies (the TMA engine), each rounded out to 16-byte
  // boundaries (ca, ea: the entries before the chunk's first one)
  const int ca = e0 & 3, ea = e0 & 7;
  if constexpr (STAGE) {
    if (ne > CHUNK_MAX_ELEMS) {  // cannot happen with chunks from chunks.cu
      if (tid == 0) atomicOr(A.err, DEV_ERR_INDEX);
      return;
    }
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_init_fence();
      const uint32_t cb = (uint32_t)(((ca + ne) * 4 + 15) & ~15), eb = (uint32_t)(((ea + ne) * 2 + 15) & ~15);
      mbar_expect_tx(bar, cb + 10u * eb);
      if (cb) bulk_load(s_ce, C.celem + (e0 - ca), cb, bar);
      if (eb) {
#pragma unroll
        for (int k = 0; k < 10; ++k) bulk_load(s_es + k * STAGE_E, C.eslot + k * C.es + (e0 - ea), eb, bar);
      }
    }
  }
  auto elem_id = [&](int t) -> int64_t { return STAGE ? s_ce[ca + t] : C.celem[e0 + t]; };
  auto pair_slot = [&](int k, int t) -> int { return STAGE ? s_es[k * STAGE_E + ea + t] : C.eslot[k * C.es + e0 + t]; };
  const int K = C.K;
  // f_c |T| = f_c |det J| / 6: the amplitudes over 6, once per thread
  [[maybe_unused]] const double fp6[3] = {A.fp[0] * (1.0 / 6.0), A.fp[1] * (1.0 / 6.0), A.fp[2] * (1.0 / 6.0)};
  for (int i = tid; i < 9 * ns; i += CHUNK_T) {
    alo[i] = 0u;
    ahi[i] = 0;
  }
  for (int i = tid; i < 3 * nn; i += CHUNK_T) {
    rlo[i] = 0u;
    rhi[i] = 0;
  }
  for (int i = tid; i < ns; i += CHUNK_T) sexp[i] = EXP_EMPTY;
  for (int i = tid; i < nn; i += CHUNK_T) rexp[i] = EXP_EMPTY;
  // the chunk's vertices, staged once: an element's vertex a is node slot
  // eslot[a] (the diagonal pairs come first), so the elements read their
  // coordinates from shared memory instead of gathering them twice from HBM
  for (int k = tid; k < nn; k += CHUNK_T) {
    int64_t v = C.nrec[n0 + k].x;
    if (!index_ok(v, C.n_nodes, A.err)) v = 0;
    const double xv[3] = {__ldg(A.x + v), __ldg(A.y + v), __ldg(A.z + v)};
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      sxyz[3 * k + d] = xv[d];
      float h, l;
      ok = split_coord(xv[d], h, l) && ok;
      sxh[3 * k + d] = h;
      sxl[3 * k + d] = l;
    }
    sxok[k] = ok;
  }
  __syncthreads();
  if constexpr (STAGE) {
    // every thread waits (bounded) for the staged rows; if they never land the
    // chunk raises DEV_ERR_TIMEOUT and writes nothing, after thread 0 has
    // waited (bounded) once more for the copies still in flight
    const bool ok = mbar_wait(bar, 0);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(A.err, DEV_ERR_TIMEOUT);
        mbar_wait(bar, 0);
      }
      return;
    }
  }
  // Elements are dealt to the lanes across 64 segments of the chunk (lane i
  // takes position i / 64 of segment i % 64): neighbouring elements, which
  // share node pairs, go to different warp instructions, so the atomics of
  // one instruction seldom hit the same accumulator.
  const int L = (ne + 63) >> 6;
  // A: exponent bounds of every slot
  for (int i = tid; i < 64 * L; i += CHUNK_T) {
    const int t = (i & 63) * L + (i >> 6);
    if (t >= ne) continue;
    const int64_t e = elem_id(t);
    int slot[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      slot[k] = pair_slot(k, t) & 0x7FFF;
      if (!index_ok(slot[k], k < 4 ? nn : ns, A.err)) slot[k] = 0;
    }
    // the edges in FP32 from the split coordinates (no FP64 work), or from
    // the FP64 ones where the split does not serve
    const double lam = A.lam ? __ldg(A.lam + e) : A.lam_const;
    const double mu = A.mu ? __ldg(A.mu + e) : A.mu_const;
    const double C1 = fma(2.0, fabs(mu), fabs(lam));
    auto fb = [&]() { return staged_bounds_fp64(sxyz, slot[0], slot[1], slot[2], slot[3], C1, C.ef); };
    bool split = true;
    float Hh[4][3], Ll[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      split = split && sxok[slot[a]];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Hh[a][d] = sxh[3 * slot[a] + d];
        Ll[a][d] = sxl[3 * slot[a] + d];
      }
    }
    const int2 eb = split ? element_bounds_split(Hh, Ll, C1, 0.0, C.ef, fb) : fb();
#pragma unroll
    for (int k = 0; k < 10; ++k) atomicMax(sexp + slot[k], eb.x);
    if constexpr (HAS_LOAD) {
#pragma unroll
      for (int k = 0; k < 4; ++k) atomicMax(rexp + slot[k], eb.y);
    }
  }
  __syncthreads();
  // B: the entries, added in fixed point
  for (int i = tid; i < 64 * L; i += CHUNK_T) {
    const int t = (i & 63) * L + (i >> 6);
    if (t >= ne) continue;
    const int64_t e = elem_id(t);
    int slot[10], sh[10];
    bool tr[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const int v = pair_slot(k, t);
      slot[k] = v & 0x7FFF;
      if (!index_ok(slot[k], k < 4 ? nn : ns, A.err)) slot[k] = 0;
      tr[k] = (v & 0x8000) != 0;
      sh[k] = C.H - sexp[slot[k]];
    }
    double X[4][3];
    staged_vertices(sxyz, slot, X);
    Geo g;
    geometry(X, g);
    if (!(g.det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
    const double adet = fabs(g.det);
    const double lam = A.lam ? __ldg(A.lam + e) : A.lam_const;
    const double mu = A.mu ? __ldg(A.mu + e) : A.mu_const;
    elast_upper<R>(g, adet, lam, mu, [&](auto KK, R v) {
      constexpr int r = upper_a(12, KK), cc = upper_b(12, KK);
      constexpr int a = r / 3, i3 = r % 3, b = cc / 3, j3 = cc % 3;
      constexpr int k = pair_index(4, a, b);
      const int idx = 9 * slot[k] + ((a != b && tr[k]) ? 3 * j3 + i3 : 3 * i3 + j3);
      acc_add(alo + idx, ahi + idx, fx_of(v, sh[k]), K);
    });
    if constexpr (HAS_LOAD) {
      int shf[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) shf[a] = C.H - rexp[slot[a]];
      if constexpr (LOAD == LOAD_CONST) {
        // a constant f: every rule integrates f lambda_a exactly, f |T| / 4 at
        // each vertex; the factor 1/4 is taken by the fixed-point shift
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (A.fp[q] == 0.0) continue;  // same for every thread
          const R fq = R(fp6[q] * adet);
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int idx = 3 * slot[a] + q;
            acc_add(rlo + idx, rhi + idx, fx_of(fq, shf[a] - 2), K);
          }
        }
      } else {
        R Xr[4][3];
        vertices_r<R>(X, Xr);
        R Fs[4];
        shape_load<1, NPTS, LOAD, R>(Xr, Fs);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (A.fp[q] == 0.0) continue;  // same for every thread
          const R fq = R(fp6[q] * adet);
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int idx = 3 * slot[a] + q;
            acc_add(rlo + idx, rhi + idx, fx_of(R(fq * Fs[a]), shf[a]), K);
          }
        }
      }
    }
  }
  __syncthreads();
  // C: sums to FP64; owned slots to the CSR values, shared ones to partials
  for (int k = tid; k < ns; k += CHUNK_T) {
    const int4 rec = C.srec[s0 + k];
    const int es = sexp[k];
    double v[9];
    if (es >= EXP_POISON) {
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = __longlong_as_double(0x7FF8000000000000LL);
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = f64_of(acc_sum(alo + 9 * k + q, ahi + 9 * k + q, K), es - C.H);
    }
    if (k < nn) {  // node slot: the upper triangle was accumulated; mirror it
      v[3] = v[1];
      v[6] = v[2];
      v[7] = v[5];
    }
    if (rec.w < 0) {
      const int Li = rec.z & 0xFFFF, Lj = rec.z >> 16;
      if (block_ok(rec.x, Li, C.nnz, A.err)) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) C.values[(int64_t)rec.x + i * Li + j] = v[3 * i + j];
      }
      if (k >= nn && block_ok(rec.y, Lj, C.nnz, A.err)) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int i = 0; i < 3; ++i) C.values[(int64_t)rec.y + j * Lj + i] = v[3 * i + j];
      }
    } else if (index_ok(rec.w, C.n_part, A.err)) {
      double* p = C.part + PART_STRIDE * (int64_t)rec.w;
      st_v4(p, v[0], v[1], v[2], v[3]);
      st_v4(p + 4, v[4], v[5], v[6], v[7]);
      st_v4(p + 8, v[8], 0.0, 0.0, 0.0);
    }
  }
  if (C.rhs) {
    for (int k = tid; k < nn; k += CHUNK_T) {
      const int2 nr = C.nrec[n0 + k];
      const int es = rexp[k];
      double f[3];
#pragma unroll
      for (int q = 0; q < 3; ++q)
        f[q] = es >= EXP_POISON ? __longlong_as_double(0x7FF8000000000000LL)
                                : f64_of(acc_sum(rlo + 3 * k + q, rhi + 3 * k + q, K), es - C.H);
      if (nr.y < 0) {
        if (index_ok(nr.x, C.n_nodes, A.err)) {
#pragma unroll
          for (int q = 0; q < 3; ++q) C.rhs[3 * (int64_t)nr.x + q] = f[q];
        }
      } else if (index_ok(nr.y, C.n_npart, A.err)) {
        st_v4(C.npart + 4 * (int64_t)nr.y, f[0], f[1], f[2], 0.0);
      }
    }
  }
}

// The couplings shared by several chunks: their partial sums (contiguous,
// in chunk order) added and written as both 3 x 3 blocks.  One thread per
// entry of a group: the nine threads of a group read its partial sums as
// whole sectors and write each row of a block as one 24-byte run, so a warp
// instruction touches about a dozen sectors instead of 32 scattered ones.
__global__ void k_chunk_reduce(const int32_t* __restrict__ gptr, const int4* __restrict__ grec, int64_t ngroup,
                               const double* __restrict__ part, double* __restrict__ values, int64_t n_part,
                               int64_t nnz, int* err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 9 * ngroup) return;
  const int64_t g = t / 9;
  const int q = (int)(t - 9 * g), i = q / 3, j = q - 3 * i;
  const int32_t p0 = gptr[g], p1 = gptr[g + 1];
  const int4 rec = grec[g];
  if (!index_ok(p0, n_part, err) || !index_ok(p1 - 1, n_part, err)) return;
  double v = __ldg(part + PART_STRIDE * (int64_t)p0 + q);
#pragma unroll 4
  for (int32_t p = p0 + 1; p < p1; ++p) v += __ldg(part + PART_STRIDE * (int64_t)p + q);
  const int Li = rec.z & 0xFFFF, Lj = rec.z >> 16;
  if (block_ok(rec.x, Li, nnz, err)) values[(int64_t)rec.x + i * Li + j] = v;
  if (rec.x != rec.y && block_ok(rec.y, Lj, nnz, err)) values[(int64_t)rec.y + j * Lj + i] = v;
}

__global__ void k_chunk_reduce_nodes(const int32_t* __restrict__ gptr, const int32_t* __restrict__ gnode,
                                     int64_t ngroup, const double* __restrict__ npart, double* __restrict__ rhs,
                                     int64_t n_npart, int64_t n_nodes, int* err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroup) return;
  const int32_t p0 = gptr[g], p1 = gptr[g + 1];
  if (!index_ok(p0, n_npart, err) || !index_ok(p1 - 1, n_npart, err) || !index_ok(gnode[g], n_nodes, err)) return;
  double f[4];
  ld_v4(npart + 4 * (int64_t)p0, f[0], f[1], f[2], f[3]);
  for (int32_t p = p0 + 1; p < p1; ++p) {
    double w[4];
    ld_v4(npart + 4 * (int64_t)p, w[0], w[1], w[2], w[3]);
#pragma unroll
    for (int q = 0; q < 3; ++q) f[q] += w[q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) rhs[3 * (int64_t)gnode[g] + q] = f[q];
}

__global__ void k_zero_nodes(const int32_t* __restrict__ nodes, int64_t n, double* __restrict__ rhs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) rhs[3 * (int64_t)nodes[i / 3] + i % 3] = 0.0;
}

template <int LOAD, int NPTS, typename R, bool STAGE>
fea_status launch_stage(const ElemArgs& A, const ChunkArgs& Cg, int64_t nchunk, size_t smem, cudaStream_t s) {
  static size_t configured = 0;  // opt-in above the 48 KB default, once per instance
  if (smem > 48 * 1024 && smem > configured) {
    FEA_CUDA(cudaFuncSetAttribute(k_elast_chunk<LOAD, NPTS, R, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    configured = smem;
  }
  k_elast_chunk<LOAD, NPTS, R, STAGE><<<(unsigned)nchunk, CHUNK_T, smem, s>>>(A, Cg);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

// The FP32 (mixed) kernel stages the chunk's connectivity with bulk copies:
// 3.79 -> 3.69 ms at 128^3.  The FP64 kernel, bound by its FP64 pipe, reads
// it from global memory: staged it measured 6.31 -> 6.33 ms.
template <int LOAD, int NPTS, typename R>
fea_status launch_one(const ElemArgs& A, const ChunkArgs& Cg, int64_t nchunk, size_t smem, cudaStream_t s) {
  constexpr bool STAGE = !IsDouble<R>::value;
  return launch_stage<LOAD, NPTS, R, STAGE>(A, Cg, nchunk, smem + (STAGE ? STAGE_BYTES : 0), s);
}

template <typename R>
fea_status launch_prec(const ElemArgs& A, const ChunkArgs& Cg, int64_t nchunk, size_t smem, int load, int npts,
                       cudaStream_t s) {
  if (load == LOAD_NONE) return launch_one<LOAD_NONE, 1, R>(A, Cg, nchunk, smem, s);
  if (load == LOAD_CONST) {
    if (npts == 1) return launch_one<LOAD_CONST, 1, R>(A, Cg, nchunk, smem, s);
    if (npts == 4) return launch_one<LOAD_CONST, 4, R>(A, Cg, nchunk, smem, s);
    return launch_one<LOAD_CONST, 11, R>(A, Cg, nchunk, smem, s);
  }
  if (npts == 1) return launch_one<LOAD_SIN, 1, R>(A, Cg, nchunk, smem, s);
  if (npts == 4) return launch_one<LOAD_SIN, 4, R>(A, Cg, nchunk, smem, s);
  return launch_one<LOAD_SIN, 11, R>(A, Cg, nchunk, smem, s);
}

// |f_c| < 2^result over the three load amplitudes.
int load_exponent(const fea_coeffs* co, int load) {
  if (load == LOAD_NONE) return EXP_ZERO;
  double m = 0.0;
  for (int q = 0; q < 3; ++q) {
    const double a = std::fabs(co->f_param[q]);
    if (!std::isfinite(a)) return EXP_POISON;
    m = std::max(m, a);
  }
  if (m == 0.0) return EXP_ZERO;
  int e = 0;
  std::frexp(m, &e);
  return e;
}

}  // namespace

fea_status assemble_chunked(fea_mesh* m, Pattern* P, const fea_coeffs* co, const fea_quadrature* q, int load,
                            double* values, double* rhs, cudaStream_t s) {
  FEA_TRY(build_chunks(m, P, s));
  const Chunks* K = P->chunks;
  FEA_TRY(ensure_scratch(m->part, (size_t)std::max<int64_t>(K->npart, 1) * PART_STRIDE * sizeof(double)));
  if (rhs) FEA_TRY(ensure_scratch(m->npart, (size_t)std::max<int64_t>(K->nnpart, 1) * 4 * sizeof(double)));
  ElemArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.N = m->n_nodes;
  A.E = m->n_elems;
  A.lam = co->lame_lambda;
  A.lam_const = co->lambda_const;
  A.mu = co->lame_mu;
  A.mu_const = co->mu_const;
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
  Cg.ef = load_exponent(co, ld);
  Cg.max_slots = K->max_slots;
  Cg.max_nodes = K->max_nodes;
  Cg.values = values;
  Cg.rhs = rhs;
  Cg.part = static_cast<double*>(m->part.ptr);
  Cg.npart = rhs ? static_cast<double*>(m->npart.ptr) : nullptr;
  Cg.n_nodes = m->n_nodes;
  Cg.nnz = P->nnz;
  Cg.n_part = K->npart;
  Cg.n_npart = K->nnpart;
  const size_t smem = (size_t)K->max_slots * (9 * 2 * sizeof(int) + sizeof(int)) +
                      (size_t)K->max_nodes * (3 * sizeof(double) + 3 * 2 * sizeof(int) + sizeof(int) +
                                              6 * sizeof(float) + 1);
  if (smem + STAGE_BYTES > 227 * 1024)
    return fail(FEA_ERR_OVERFLOW, "chunked scatter: chunk too large for shared memory");
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[0], s));
  if (K->nchunk > 0) {
    if (q->prec == FEA_MIXED) FEA_TRY(launch_prec<float>(A, Cg, K->nchunk, smem, ld, q->npts, s));
    else FEA_TRY(launch_prec<double>(A, Cg, K->nchunk, smem, ld, q->npts, s));
  }
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[1], s));
  if (K->ngroup > 0)
    k_chunk_reduce<<<(unsigned)((9 * K->ngroup + 255) / 256), 256, 0, s>>>(K->gptr, K->grec, K->ngroup, Cg.part,
                                                                           values, Cg.n_part, Cg.nnz, m->err);
  if (rhs && K->niso > 0)
    k_zero_nodes<<<(unsigned)((3 * K->niso + 255) / 256), 256, 0, s>>>(K->iso, K->niso, rhs);
  if (rhs && K->nngroup > 0)
    k_chunk_reduce_nodes<<<(unsigned)((K->nngroup + 127) / 128), 128, 0, s>>>(K->ngptr, K->ngnode, K->nngroup,
                                                                             Cg.npart, rhs, Cg.n_npart, Cg.n_nodes,
                                                                             m->err);
  FEA_CUDA(cudaGetLastError());
  if (m->profile) {
    FEA_CUDA(cudaEventRecord(m->ev[2], s));
    m->profiled = true;
  }
  return FEA_OK;
}

}  // namespace fea
