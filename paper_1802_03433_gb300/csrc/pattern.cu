// Global CSR sparsity pattern and the structures of the deterministic scatter.
//
// The paper's sparse kernel (Sec. 5, sparse variant of Algorithm 1) receives
// the row structure as input: the nonzero count of each row (gNbrNodeLen) and
// the column indices of each row (gNbrNodeIdx), padded to a row width MAX_NZ
// derived from the mesh and the element type.  Here that structure is built
// on the GPU from the connectivity alone:
//
//  1. dof -> element incidences: histogram, scan, fill, then each dof's list
//     sorted by element id (so every later step is deterministic);
//  2. CSR rows: one warp per row gathers the dofs of the row's incident
//     elements into shared memory, drops repeats and ranks the survivors
//     (count pass, scan to row_ptr, fill pass);
//  3. slots: for every incidence (row, element, local a) the position of
//     each of the element's dofs inside the row, 1 byte each; the scatter
//     then needs no search;
//  4. P2: the edge dofs come straight from the P1 pattern - the upper
//     triangle of row a lists exactly the edges (a, b), b > a, in
//     lexicographic order, so the rank of an edge is a scan offset plus a
//     position in a row;
//  5. vector (3 dofs per node) patterns expand each scalar coupling into a
//     3 x 3 block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "buildutil.cuh"
#include "internal.cuh"

namespace fea {

namespace {

constexpr int ROW_CAP = 1024;     // candidate couplings per scalar row sorted by one warp
constexpr int LONG_CAP = 16384;   // candidate couplings per scalar row sorted by one block (longer: refused)
constexpr int UNIQ_WARPS = 4;   // warps per block of the row kernels

// ------------------------------------------------------------------ validation
template <int NV>
__global__ void k_validate(const int32_t* __restrict__ tets, int64_t E, int64_t N, int* err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int32_t v[NV];
  bool bad = false;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    v[a] = tets[a * E + e];
    bad |= v[a] < 0 || (int64_t)v[a] >= N;
  }
#pragma unroll
  for (int a = 0; a < NV; ++a)
#pragma unroll
    for (int b = a + 1; b < NV; ++b) bad |= v[a] == v[b];
  if (bad) atomicOr(err, DEV_ERR_INDEX);
}

// ------------------------------------------------------------------ incidences
__global__ void k_inc_count(const int32_t* __restrict__ edof, int64_t n, int32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(cnt + edof[i], 1);
}

// edof is SoA [nb][E]: entry i is local dof a = i / E of element e = i % E.
__global__ void k_inc_fill(const int32_t* __restrict__ edof, int64_t E, int nb,
                           const int32_t* __restrict__ ptr, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ inc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E * nb) return;
  const int64_t a = i / E, e = i - a * E;
  const int32_t d = edof[i];
  const int32_t pos = ptr[d] + atomicAdd(cursor + d, 1);
  inc[pos] = (int32_t)(e * nb + a);
}

// ------------------------------------------------------------------ rows
// One warp per scalar row, one pass: the row's candidate columns (the nb dofs
// of each incident element, in incidence order t = incidence * NB + local
// dof) are sorted as 64-bit keys (column << 32 | t) by a bitonic network.
// The first key of each run of equal columns is a distinct column, in
// ascending order, and the rank of its run is the slot of every candidate in
// the run.  Writes the distinct columns to cols[inc_ptr[row] * NB ...]
// (scratch with room for every candidate), their count, and each
// candidate's slot.

// Candidate t of a row as its sort key (t < k), or a key that sorts last.
template <int NB>
__device__ __forceinline__ unsigned long long row_key(int t, int k, int32_t i0, const int32_t* __restrict__ inc,
                                                      const int32_t* __restrict__ edof, int64_t E) {
  if (t >= k) return ~0ull;
  const int64_t e = inc[i0 + t / NB] / NB;
  const uint32_t d = (uint32_t)edof[(int64_t)(t % NB) * E + e];
  return ((unsigned long long)d << 32) | (uint32_t)t;
}

// Outputs of one sorted key: the distinct column (first of its run) and the
// candidate's slot (its run's rank).  Rows of more than 255 entries are long
// rows: their slot bytes (a byte holds ranks below 255) are not used, a
// separate kernel adds them (k_long_rows).
template <int NB, int SW>
__device__ __forceinline__ void row_emit(unsigned long long key, bool keep, int rank, int32_t i0, int32_t* cols,
                                         int64_t cbase, uint8_t* slot, int* err) {
  (void)err;
  if (keep) cols[cbase + rank] = (int32_t)(key >> 32);
  if (rank < 255) {
    const uint32_t o = (uint32_t)key;
    slot[((int64_t)i0 + o / NB) * SW + o % NB] = (uint8_t)rank;
  }
}

// Rows of up to 32 * R candidates, in registers (warp_sort_reg).  Returns the
// count of distinct columns.
template <int NB, int SW, int R>
__device__ __forceinline__ int row_build_reg(int k, int32_t i0, const int32_t* __restrict__ inc,
                                             const int32_t* __restrict__ edof, int64_t E, int32_t* cols,
                                             uint8_t* slot, int* err) {
  const int lane = threadIdx.x & 31;
  unsigned long long key[R];
#pragma unroll
  for (int r = 0; r < R; ++r) key[r] = row_key<NB>(lane * R + r, k, i0, inc, edof, E);
  warp_sort_reg<unsigned long long, R>(key);
  // run starts: the previous position is in this lane, or the last of the
  // lane before
  const unsigned long long before = __shfl_up_sync(0xffffffffu, key[R - 1], 1);
  bool keep[R];
  int pre[R], nkeep = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = lane * R + r;
    const uint32_t prev = (uint32_t)((r == 0 ? before : key[r - 1]) >> 32);
    keep[r] = i < k && (i == 0 || prev != (uint32_t)(key[r] >> 32));
    nkeep += keep[r];
    pre[r] = nkeep;
  }
  int incl = nkeep;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int64_t cbase = (int64_t)i0 * NB;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (lane * R + r < k) row_emit<NB, SW>(key[r], keep[r], incl - nkeep + pre[r] - 1, i0, cols, cbase, slot, err);
  return __shfl_sync(0xffffffffu, incl, 31);
}

// Rows of up to `cap` candidates (a power of two <= ROW_CAP) in the warp's
// shared-memory buffer, the same network with the lanes striding over each
// stage's compare-exchanges.
template <int NB, int SW>
__device__ __forceinline__ int row_build_smem(int k, int32_t i0, const int32_t* __restrict__ inc,
                                              const int32_t* __restrict__ edof, int64_t E, int32_t* cols,
                                              uint8_t* slot, int* err, unsigned long long* buf) {
  const int lane = threadIdx.x & 31;
  int n2 = 32;
  while (n2 < k) n2 <<= 1;
  for (int t = lane; t < n2; t += 32) buf[t] = row_key<NB>(t, k, i0, inc, edof, E);
  __syncwarp();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane; t < (n2 >> 1); t += 32) {
        const int i = 2 * stride * (t / stride) + (t % stride), j = i + stride;
        const unsigned long long a = buf[i], b = buf[j];
        if ((a > b) == ((i & size) == 0)) {
          buf[i] = b;
          buf[j] = a;
        }
      }
      __syncwarp();
    }
  const int64_t cbase = (int64_t)i0 * NB;
  int c = 0;
  for (int t0 = 0; t0 < k; t0 += 32) {
    const int t = t0 + lane;
    const unsigned long long key = t < k ? buf[t] : 0ull;
    const bool keep = t < k && (t == 0 || (uint32_t)(buf[t - 1] >> 32) != (uint32_t)(key >> 32));
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (t < k) row_emit<NB, SW>(key, keep, c + __popc(mask & (0xffffffffu >> (31 - lane))) - 1, i0, cols, cbase, slot, err);
    c += __popc(mask);
  }
  __syncwarp();
  return c;
}

// cap: the mesh's longest candidate list rounded up to a power of two >= 32
// (<= ROW_CAP).  Rows of up to 256 candidates sort in registers; above that
// in the warp's buffer of the dynamic shared memory (UNIQ_WARPS * cap keys,
// present only when cap > 256).
template <int NB, int SW>
__global__ void __launch_bounds__(32 * UNIQ_WARPS) k_row_build(int64_t nrows, const int32_t* __restrict__ inc_ptr,
                                                               const int32_t* __restrict__ inc,
                                                               const int32_t* __restrict__ edof, int64_t E,
                                                               int cap, int32_t* __restrict__ counts,
                                                               int32_t* __restrict__ cols,
                                                               uint8_t* __restrict__ slot, int* err) {
  extern __shared__ unsigned long long sbuf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * UNIQ_WARPS;
  for (int64_t row = (int64_t)blockIdx.x * UNIQ_WARPS + w; row < nrows; row += nwarps) {
    const int32_t i0 = inc_ptr[row], i1 = inc_ptr[row + 1];
    const int k = (i1 - i0) * NB;
    int c;
    if (k > cap) {
      c = 0;  // a long candidate list: k_row_build_long
    } else if (k <= 32) {
      c = row_build_reg<NB, SW, 1>(k, i0, inc, edof, E, cols, slot, err);
    } else if (k <= 64) {
      c = row_build_reg<NB, SW, 2>(k, i0, inc, edof, E, cols, slot, err);
    } else if (k <= 128) {
      c = row_build_reg<NB, SW, 4>(k, i0, inc, edof, E, cols, slot, err);
    } else if (k <= 256) {
      c = row_build_reg<NB, SW, 8>(k, i0, inc, edof, E, cols, slot, err);
    } else {
      c = row_build_smem<NB, SW>(k, i0, inc, edof, E, cols, slot, err, sbuf + (size_t)w * cap);
    }
    if (lane == 0) counts[row] = c;
  }
}

// Rows whose candidate list exceeds the warp kernel's cap.
__global__ void k_long_list(const int32_t* __restrict__ inc_ptr, int64_t n, int nb, int cap, int32_t* __restrict__ cursor,
                            int32_t* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n && (int64_t)(inc_ptr[r + 1] - inc_ptr[r]) * nb > cap) out[atomicAdd(cursor, 1)] = (int32_t)r;
}

// Rows of more than ROW_CAP (up to LONG_CAP) candidates, one block each: the
// warp kernel's sort and runs with the block striding over the network in
// shared memory.
template <int NB, int SW>
__global__ void __launch_bounds__(256) k_row_build_long(const int32_t* __restrict__ rows,
                                                        const int32_t* __restrict__ inc_ptr,
                                                        const int32_t* __restrict__ inc,
                                                        const int32_t* __restrict__ edof, int64_t E,
                                                        int32_t* __restrict__ counts, int32_t* __restrict__ cols,
                                                        uint8_t* __restrict__ slot, int* err) {
  extern __shared__ unsigned long long lbuf[];
  const int32_t row = rows[blockIdx.x];
  const int32_t i0 = inc_ptr[row];
  const int k = (inc_ptr[row + 1] - i0) * NB;
  int n2 = 32;
  while (n2 < k) n2 <<= 1;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) lbuf[t] = row_key<NB>(t, k, i0, inc, edof, E);
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (n2 >> 1); t += blockDim.x) {
        const int i = 2 * stride * (t / stride) + (t % stride), j = i + stride;
        const unsigned long long a = lbuf[i], b = lbuf[j];
        if ((a > b) == ((i & size) == 0)) {
          lbuf[i] = b;
          lbuf[j] = a;
        }
      }
      __syncthreads();
    }
  // runs: each thread a contiguous range of sorted positions
  const int per = (k + blockDim.x - 1) / blockDim.x;
  const int p0 = min(k, (int)threadIdx.x * per), p1 = min(k, p0 + per);
  int nk = 0;
  for (int p = p0; p < p1; ++p) nk += (p == 0 || (uint32_t)(lbuf[p - 1] >> 32) != (uint32_t)(lbuf[p] >> 32));
  int64_t total;
  int rank = (int)block_excl_scan(nk, &total) - 1;
  const int64_t cbase = (int64_t)i0 * NB;
  for (int p = p0; p < p1; ++p) {
    const bool keep = p == 0 || (uint32_t)(lbuf[p - 1] >> 32) != (uint32_t)(lbuf[p] >> 32);
    rank += keep;
    row_emit<NB, SW>(lbuf[p], keep, rank, i0, cols, cbase, slot, err);
  }
  if (threadIdx.x == 0) counts[row] = (int32_t)total;
}

// Rows of more than 255 entries (the long rows of the local-row scatter).
__global__ void k_wide_list(const int32_t* __restrict__ rp, int64_t n, int32_t* __restrict__ cursor,
                            int32_t* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n && rp[r + 1] - rp[r] > 255) out[atomicAdd(cursor, 1)] = (int32_t)r;
}

// col_idx of each row from the row's distinct columns in the scratch of
// k_row_build; one warp per row.
__global__ void k_cols_compact(int64_t nrows, const int32_t* __restrict__ inc_ptr, int nb,
                               const int32_t* __restrict__ cols, const int32_t* __restrict__ rp,
                               int32_t* __restrict__ ci) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < nrows; row += nwarps) {
    const int32_t* src = cols + (int64_t)inc_ptr[row] * nb;
    const int32_t lo = rp[row], len = rp[row + 1] - lo;
    for (int32_t j = lane; j < len; j += 32) ci[lo + j] = src[j];
  }
}

__global__ void k_max_row(const int32_t* __restrict__ rp, int64_t n, int* out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) atomicMax(out, rp[r + 1] - rp[r]);
}

__global__ void k_tile_max(const int32_t* __restrict__ rp, int64_t n, int rows, int* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r0 = t * rows;
  if (r0 >= n) return;
  const int64_t r1 = std::min<int64_t>(r0 + rows, n);
  atomicMax(out, rp[r1] - rp[r0]);
}

__global__ void k_tile_span(const int32_t* __restrict__ rp, int64_t n, int rows, int32_t* __restrict__ span) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r0 = t * rows;
  if (r0 >= n) return;
  const int64_t r1 = std::min<int64_t>(r0 + rows, n);
  span[t] = rp[r1] - rp[r0];
}

// ------------------------------------------------------------------ P2 edges
// Number of columns above the diagonal in each P1 row = edges (a, b), b > a.
__global__ void k_upper_count(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t N,
                              int32_t* __restrict__ cnt) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= N) return;
  int32_t c = 0;
  for (int32_t p = rp[a]; p < rp[a + 1]; ++p) c += ci[p] > a;
  cnt[a] = c;
}

__device__ __forceinline__ int32_t lower_bound(const int32_t* __restrict__ c, int32_t lo, int32_t hi, int32_t v) {
  while (lo < hi) {
    const int32_t m = (lo + hi) >> 1;
    if (c[m] < v) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// edof2 [10][E]: vertices, then edge k = (p, q): N + ebase[a] + index of b
// among the columns of row a above the diagonal, a = min, b = max.
__global__ void k_p2_edof(const int32_t* __restrict__ tets, int64_t E, int64_t N, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int64_t* __restrict__ ebase,
                          int32_t* __restrict__ edof2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 10 * E) return;
  const int64_t k = i / E, e = i - k * E;
  if (k < 4) {
    edof2[i] = tets[i];
    return;
  }
  const int kk = (int)k - 4;
  const int p = kk < 3 ? 0 : (kk < 5 ? 1 : 2);
  const int q = kk < 3 ? kk + 1 : (kk < 5 ? kk - 1 : 3);
  int32_t a = tets[(int64_t)p * E + e], b = tets[(int64_t)q * E + e];
  if (a > b) {
    const int32_t t = a;
    a = b;
    b = t;
  }
  const int32_t lo = rp[a], hi = rp[a + 1];
  const int32_t first_up = lower_bound(ci, lo, hi, a + 1);
  const int32_t pos = lower_bound(ci, lo, hi, b);
  edof2[i] = (int32_t)(N + ebase[a] + (pos - first_up));
}

// ------------------------------------------------------------------ vector expansion
__global__ void k_expand_rowptr(const int32_t* __restrict__ rp, int64_t N, int ndpn, int32_t* __restrict__ rp3) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > N * ndpn) return;
  if (r == N * ndpn) {
    rp3[r] = (int32_t)((int64_t)ndpn * ndpn * rp[N]);
    return;
  }
  const int64_t a = r / ndpn, c = r - a * ndpn;
  rp3[r] = (int32_t)((int64_t)ndpn * ndpn * rp[a] + ndpn * c * (int64_t)(rp[a + 1] - rp[a]));
}

// Columns of the NDPN x NDPN block expansion, one warp per expanded row
// (coalesced stores).
template <int NDPN>
__global__ void k_expand_cols(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t N,
                              const int32_t* __restrict__ rp3, int32_t* __restrict__ ci3) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N * NDPN; r += nwarps) {
    const int64_t a = r / NDPN;
    const int32_t p0 = rp[a], len = (rp[a + 1] - p0) * NDPN;
    int32_t* out = ci3 + rp3[r];
    for (int32_t j = lane; j < len; j += 32) out[j] = NDPN * ci[p0 + j / NDPN] + j % NDPN;
  }
}

// ------------------------------------------------------------------ ipos
// Inverse of the incidence list: ipos[a][e] = i such that inc[i] = e * nb + a.
__global__ void k_ipos(int64_t nI, int nb, int64_t E, const int32_t* __restrict__ inc, int32_t* __restrict__ ipos) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nI) return;
  const int64_t p = inc[i];
  const int64_t e = p / nb, a = p - e * nb;
  ipos[a * E + e] = (int32_t)i;
}

// ------------------------------------------------------------------ tiled layout
// Steps of row tile t (the most contributions any of its rows has) and its
// position count steps * S_t.
__global__ void k_tile_steps(int64_t nrows, int rows, const int32_t* __restrict__ inc_ptr,
                             int32_t* __restrict__ steps, int64_t* __restrict__ cnt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r0 = t * rows;
  if (r0 >= nrows) return;
  const int64_t r1 = r0 + rows < nrows ? r0 + rows : nrows;
  int32_t K = 0;
  for (int64_t r = r0; r < r1; ++r) K = max(K, inc_ptr[r + 1] - inc_ptr[r]);
  steps[t] = K;
  cnt[t] = (int64_t)K * (((r1 - r0) + 3) & ~int64_t(3));
}

// Position of every incidence in the tiled layout; its slots copied there.
template <int SW>
__global__ void k_tpos(int64_t nrows, int rows, int nb, int64_t E, const int32_t* __restrict__ inc_ptr,
                       const int32_t* __restrict__ inc, const uint8_t* __restrict__ slot,
                       const int64_t* __restrict__ tile_base, int32_t* __restrict__ tpos,
                       uint8_t* __restrict__ tslot) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int64_t t = r / rows, j = r - t * rows;
  const int64_t r1 = (t + 1) * rows < nrows ? (t + 1) * rows : nrows;
  const int64_t S = ((r1 - t * rows) + 3) & ~int64_t(3);
  const int64_t base = tile_base[t];
  const int32_t i0 = inc_ptr[r];
  for (int32_t i = i0; i < inc_ptr[r + 1]; ++i) {
    const int64_t pos = base + (int64_t)(i - i0) * S + j;
    const int64_t p = inc[i];
    const int64_t e = p / nb, a = p - e * nb;
    tpos[a * E + e] = (int32_t)pos;
    const uint4* src = reinterpret_cast<const uint4*>(slot + (int64_t)i * SW);
    if constexpr (SW == 16) {
      *reinterpret_cast<uint4*>(tslot + pos * 16) = *src;
    } else {
      *reinterpret_cast<uint32_t*>(tslot + pos * 4) = *reinterpret_cast<const uint32_t*>(slot + (int64_t)i * 4);
    }
  }
}

fea_status build_tiled(fea_mesh* m, Pattern* P, const Base* B, cudaStream_t s) {
  const int64_t nrows = P->ndof;
  const int rows = P->rows_per_tile;
  const int64_t ntiles = (nrows + rows - 1) / rows;
  if (ntiles == 0) return FEA_OK;
  FEA_TRY(dalloc(&P->tile_steps, ntiles));
  FEA_TRY(dalloc(&P->tile_base, ntiles + 1));
  Tmp<int64_t> cnt;
  FEA_TRY(cnt.alloc(ntiles));
  k_tile_steps<<<blocks_for(ntiles, 256), 256, 0, s>>>(nrows, rows, B->inc_ptr, P->tile_steps, cnt.p);
  FEA_CUDA(cudaGetLastError());
  FEA_TRY(scan(cnt.p, ntiles, P->tile_base, s));
  int64_t npos = 0;
  FEA_TRY(read_i64(P->tile_base + ntiles, &npos, s));
  if (npos > (int64_t)INT32_MAX) return FEA_OK;  // positions must fit int32: keep the incidence layout
  const int sw = B->slot_width;
  FEA_TRY(dalloc(&P->tpos, (size_t)m->n_elems * B->nb));
  FEA_TRY(dalloc(&P->tslot, (size_t)std::max<int64_t>(npos, 1) * sw));
  if (sw == 16)
    k_tpos<16><<<blocks_for(nrows, 128), 128, 0, s>>>(nrows, rows, B->nb, m->n_elems, B->inc_ptr, B->inc, B->slot,
                                                      P->tile_base, P->tpos, P->tslot);
  else
    k_tpos<4><<<blocks_for(nrows, 128), 128, 0, s>>>(nrows, rows, B->nb, m->n_elems, B->inc_ptr, B->inc, B->slot,
                                                     P->tile_base, P->tpos, P->tslot);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaStreamSynchronize(s));
  P->npos = npos;
  return FEA_OK;
}

// ------------------------------------------------------------------ stages
// Stage of a row tile = chunk of the largest element id among its rows'
// incidences (each incidence list is sorted, so its last entry).
__global__ void k_tile_stage(int64_t ndof, int ndpn, int rows, int nb, const int32_t* __restrict__ inc_ptr,
                             const int32_t* __restrict__ inc, int64_t chunk, int32_t* __restrict__ stage) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r0 = t * rows;
  if (r0 >= ndof) return;
  const int64_t r1 = r0 + rows < ndof ? r0 + rows : ndof;
  int64_t emax = -1;
  for (int64_t node = r0 / ndpn; node <= (r1 - 1) / ndpn; ++node) {
    const int32_t i0 = inc_ptr[node], i1 = inc_ptr[node + 1];
    if (i1 > i0) emax = max(emax, (int64_t)(inc[i1 - 1] / nb));
  }
  stage[t] = emax < 0 ? 0 : (int32_t)(emax / chunk);
}

// ------------------------------------------------------------------ emap
__global__ void k_emap(int64_t nrows, int nb, int sw, const int32_t* __restrict__ inc_ptr,
                       const int32_t* __restrict__ inc, const uint8_t* __restrict__ slot,
                       const int32_t* __restrict__ rp, int32_t* __restrict__ emap) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  for (int32_t i = inc_ptr[r]; i < inc_ptr[r + 1]; ++i) {
    const int64_t p = inc[i];  // e * nb + a
    for (int b = 0; b < nb; ++b) emap[p * nb + b] = rp[r] + slot[(int64_t)i * sw + b];
  }
}

fea_status check_err(fea_mesh* m, cudaStream_t s, const char* what) {
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaStreamSynchronize(s));
  int h = 0;
  FEA_CUDA(cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h & DEV_ERR_OVERFLOW) {
    FEA_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    return fail(FEA_ERR_OVERFLOW, std::string(what) +
                                      ": a row exceeds the scatter limits (more than 1024 candidate "
                                      "couplings or more than 255 entries in a scalar row)");
  }
  if (h & DEV_ERR_INDEX) {
    FEA_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    return fail(FEA_ERR_INDEX, std::string(what) + ": connectivity index out of range or repeated");
  }
  return FEA_OK;
}

template <int NB>
fea_status rows_and_slots(fea_mesh* m, Base* B, cudaStream_t s) {
  const int64_t n = B->nsd, E = m->n_elems;
  const int uniq_blocks = (int)std::min<int64_t>(std::max<int64_t>(1, (n + UNIQ_WARPS - 1) / UNIQ_WARPS), 152 * 64);
  constexpr int SW = NB <= 4 ? 4 : 16;
  B->slot_width = SW;
  FEA_TRY(dalloc(&B->slot, (size_t)E * NB * SW));
  // the slot bytes of long rows stay 0 (never used)
  FEA_CUDA(cudaMemsetAsync(B->slot, 0, (size_t)E * NB * SW, s));
  Tmp<int32_t> cnt, cols;
  Tmp<int> mx;
  FEA_TRY(cnt.alloc(n));
  FEA_TRY(cols.alloc(std::max<size_t>((size_t)E * NB * NB, 1)));
  FEA_TRY(mx.alloc(1));
  // the sort buffers hold the longest candidate list (most incidences x NB)
  FEA_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(int), s));
  k_max_row<<<blocks_for(n, 256), 256, 0, s>>>(B->inc_ptr, n, mx.p);
  int max_inc = 0;
  FEA_CUDA(cudaMemcpyAsync(&max_inc, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  if ((int64_t)max_inc * NB > LONG_CAP)
    return fail(FEA_ERR_OVERFLOW, "pattern: a row has more than 16384 candidate couplings (elements x local dofs)");
  int cap = 32;
  while (cap < max_inc * NB && cap < ROW_CAP) cap <<= 1;
  const size_t smem = cap > 256 ? (size_t)UNIQ_WARPS * cap * sizeof(unsigned long long) : 0;
  k_row_build<NB, SW><<<uniq_blocks, 32 * UNIQ_WARPS, smem, s>>>(n, B->inc_ptr, B->inc, B->edof, E, cap, cnt.p,
                                                                 cols.p, B->slot, m->err);
  if ((int64_t)max_inc * NB > ROW_CAP) {
    // candidate lists above the warp's cap: one block per row
    Tmp<int32_t> nl, list;
    FEA_TRY(nl.alloc(1));
    FEA_TRY(list.alloc(n));
    FEA_CUDA(cudaMemsetAsync(nl.p, 0, sizeof(int32_t), s));
    k_long_list<<<blocks_for(n, 256), 256, 0, s>>>(B->inc_ptr, n, NB, cap, nl.p, list.p);
    int32_t hn = 0;
    FEA_CUDA(cudaMemcpyAsync(&hn, nl.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FEA_CUDA(cudaStreamSynchronize(s));
    int n2 = 32;
    while (n2 < max_inc * NB) n2 <<= 1;
    const size_t lsmem = (size_t)n2 * sizeof(unsigned long long);
    FEA_CUDA(cudaFuncSetAttribute(k_row_build_long<NB, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
    if (hn > 0)
      k_row_build_long<NB, SW><<<hn, 256, lsmem, s>>>(list.p, B->inc_ptr, B->inc, B->edof, E, cnt.p, cols.p, B->slot,
                                                      m->err);
  }
  FEA_TRY(check_err(m, s, "pattern"));
  FEA_TRY(dalloc(&B->rp, n + 1));
  FEA_TRY(scan_to_ptr32(cnt.p, n, B->rp, &B->nnz, s, "nonzero"));
  FEA_TRY(dalloc(&B->ci, B->nnz));
  k_cols_compact<<<uniq_blocks, 32 * UNIQ_WARPS, 0, s>>>(n, B->inc_ptr, NB, cols.p, B->rp, B->ci);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(int), s));
  k_max_row<<<blocks_for(n, 256), 256, 0, s>>>(B->rp, n, mx.p);
  FEA_CUDA(cudaMemcpyAsync(&B->max_row, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  if (B->max_row > 255) {
    // rows past the slot bytes: listed (ascending) for k_long_rows
    Tmp<int32_t> nw;
    FEA_TRY(nw.alloc(1));
    FEA_TRY(dalloc(&B->long_rows, n));
    FEA_CUDA(cudaMemsetAsync(nw.p, 0, sizeof(int32_t), s));
    k_wide_list<<<blocks_for(n, 256), 256, 0, s>>>(B->rp, n, nw.p, B->long_rows);
    int32_t hw = 0;
    FEA_CUDA(cudaMemcpyAsync(&hw, nw.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FEA_CUDA(cudaStreamSynchronize(s));
    B->nlong = hw;
  }
  return FEA_OK;
}

fea_status incidences(fea_mesh* m, Base* B, cudaStream_t s) {
  const int64_t E = m->n_elems, n = B->nsd, nI = E * B->nb;
  if (nI > (int64_t)INT32_MAX) return fail(FEA_ERR_OVERFLOW, "elements x local dofs exceeds INT32_MAX");
  Tmp<int32_t> cnt, cur;
  FEA_TRY(cnt.alloc(n));
  FEA_TRY(cur.alloc(n));
  FEA_CUDA(cudaMemsetAsync(cnt.p, 0, n * sizeof(int32_t), s));
  FEA_CUDA(cudaMemsetAsync(cur.p, 0, n * sizeof(int32_t), s));
  k_inc_count<<<blocks_for(nI, 256), 256, 0, s>>>(B->edof, nI, cnt.p);
  FEA_TRY(dalloc(&B->inc_ptr, n + 1));
  int64_t tot = 0;
  FEA_TRY(scan_to_ptr32(cnt.p, n, B->inc_ptr, &tot, s, "incidence"));
  FEA_TRY(dalloc(&B->inc, nI));
  k_inc_fill<<<blocks_for(nI, 256), 256, 0, s>>>(B->edof, E, B->nb, B->inc_ptr, cur.p, B->inc);
  k_sort_lists<<<(int)std::min<int64_t>(blocks_for(n, 4), 152 * 64), 128, 0, s>>>(B->inc_ptr, n, B->inc);
  FEA_TRY(dalloc(&B->ipos, nI));
  k_ipos<<<blocks_for(nI, 256), 256, 0, s>>>(nI, B->nb, E, B->inc, B->ipos);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaStreamSynchronize(s));
  return FEA_OK;
}

}  // namespace

void free_base(Base* b) {
  if (!b) return;
  if (b->own_edof) dfree(b->edof);
  dfree(b->rp);
  dfree(b->ci);
  dfree(b->inc_ptr);
  dfree(b->inc);
  dfree(b->slot);
  dfree(b->ipos);
  dfree(b->emap);
  dfree(b->long_rows);
  delete b;
}

void free_pattern(Pattern* p) {
  if (!p) return;
  free_chunks(p->chunks);
  dfree(p->tile_list);
  dfree(p->class_list);
  dfree(p->tpos);
  dfree(p->tslot);
  dfree(p->tile_base);
  dfree(p->tile_steps);
  if (p->own) {
    dfree(p->row_ptr);
    dfree(p->col_idx);
  }
  delete p;
}

fea_status validate_connectivity(fea_mesh* m, cudaStream_t s) {
  if (m->n_elems > 0) {
    if (m->nvert == 3) k_validate<3><<<blocks_for(m->n_elems, 256), 256, 0, s>>>(m->tets, m->n_elems, m->n_nodes, m->err);
    else k_validate<4><<<blocks_for(m->n_elems, 256), 256, 0, s>>>(m->tets, m->n_elems, m->n_nodes, m->err);
  }
  return check_err(m, s, "mesh");
}

fea_status build_base(fea_mesh* m, int order, cudaStream_t s) {
  if (m->base[order]) return FEA_OK;
  if (order == 2) FEA_TRY(build_base(m, 1, s));
  Base* B = new Base();
  B->nb = order == 1 ? m->nvert : 10;
  const int64_t E = m->n_elems, N = m->n_nodes;
  fea_status st = FEA_OK;
  do {
    if (order == 1) {
      B->edof = m->tets;
      B->nsd = N;
    } else {
      const Base* P1 = m->base[1];
      Tmp<int32_t> up;
      Tmp<int64_t> ebase;
      if ((st = up.alloc(N)) != FEA_OK) break;
      if ((st = ebase.alloc(N + 1)) != FEA_OK) break;
      k_upper_count<<<blocks_for(N, 256), 256, 0, s>>>(P1->rp, P1->ci, N, up.p);
      if ((st = scan(up.p, N, ebase.p, s)) != FEA_OK) break;
      int64_t nedges = 0;
      if ((st = read_i64(ebase.p + N, &nedges, s)) != FEA_OK) break;
      if (N + nedges > (int64_t)INT32_MAX) {
        st = fail(FEA_ERR_OVERFLOW, "P2 dof count exceeds INT32_MAX");
        break;
      }
      B->nsd = N + nedges;
      if ((st = dalloc(&B->edof, (size_t)10 * E)) != FEA_OK) break;
      B->own_edof = true;
      if (E > 0)
        k_p2_edof<<<blocks_for(10 * E, 256), 256, 0, s>>>(m->tets, E, N, P1->rp, P1->ci, ebase.p, B->edof);
      cudaError_t ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) {
        st = cuda_fail(ce, "p2 edof");
        break;
      }
    }
    if ((st = incidences(m, B, s)) != FEA_OK) break;
    st = B->nb == 3 ? rows_and_slots<3>(m, B, s) : B->nb == 4 ? rows_and_slots<4>(m, B, s) : rows_and_slots<10>(m, B, s);
  } while (0);
  if (st != FEA_OK) {
    free_base(B);
    return st;
  }
  m->base[order] = B;
  return FEA_OK;
}

fea_status build_pattern(fea_mesh* m, int order, int ndpn, cudaStream_t s) {
  if (m->pat[order][ndpn]) return FEA_OK;
  FEA_TRY(build_base(m, order, s));
  Base* B = m->base[order];
  Pattern* P = new Pattern();
  P->order = order;
  P->ndpn = ndpn;
  P->ndof = B->nsd * ndpn;
  fea_status st = FEA_OK;
  do {
    if (ndpn == 1) {
      P->row_ptr = B->rp;
      P->col_idx = B->ci;
      P->nnz = B->nnz;
      P->own = false;
    } else {
      const int64_t nnz = B->nnz * ndpn * ndpn;
      if (nnz > (int64_t)INT32_MAX) {
        st = fail(FEA_ERR_OVERFLOW, "vector pattern nnz " + std::to_string(nnz) + " exceeds INT32_MAX");
        break;
      }
      P->nnz = nnz;
      P->own = true;
      if ((st = dalloc(&P->row_ptr, P->ndof + 1)) != FEA_OK) break;
      if ((st = dalloc(&P->col_idx, nnz)) != FEA_OK) break;
      k_expand_rowptr<<<blocks_for(P->ndof + 1, 256), 256, 0, s>>>(B->rp, B->nsd, ndpn, P->row_ptr);
      k_expand_cols<3><<<(int)std::min<int64_t>(blocks_for(P->ndof, 4), 152 * 64), 128, 0, s>>>(B->rp, B->ci, B->nsd,
                                                                                              P->row_ptr, P->col_idx);
    }
    // gather tiles: as many rows per CTA (<= 128) as keep the tile's CSR span
    // within the shared-memory budget
    Tmp<int> mx;
    if ((st = mx.alloc(1)) != FEA_OK) break;
    int rows = 128;
    for (;;) {
      cudaMemsetAsync(mx.p, 0, sizeof(int), s);
      k_tile_max<<<blocks_for((P->ndof + rows - 1) / rows + 1, 256), 256, 0, s>>>(P->row_ptr, P->ndof, rows, mx.p);
      int h = 0;
      cudaMemcpyAsync(&h, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaError_t ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) {
        st = cuda_fail(ce, "tile sizing");
        break;
      }
      if ((int64_t)h * 8 <= 160 * 1024 || rows == 1) {
        P->rows_per_tile = rows;
        P->max_tile_nnz = h;
        break;
      }
      rows /= 2;
    }
  } while (0);
  if (st == FEA_OK && (int64_t)P->max_tile_nnz * 8 > 220 * 1024)
    st = fail(FEA_ERR_OVERFLOW, "a single row is too long for the shared-memory scatter");
  if (st == FEA_OK) {
    // two tile classes: spans up to half the widest go to the light launch
    // (for P2 that separates the vertex-dof tiles from the edge-dof tiles,
    // whose accumulator then leaves room for three CTAs per SM)
    const int64_t ntiles = (P->ndof + P->rows_per_tile - 1) / P->rows_per_tile;
    std::vector<int32_t> span(std::max<int64_t>(ntiles, 1));
    if (ntiles > 0) {
      Tmp<int32_t> d;
      if ((st = d.alloc(ntiles)) == FEA_OK) {
        k_tile_span<<<blocks_for(ntiles, 256), 256, 0, s>>>(P->row_ptr, P->ndof, P->rows_per_tile, d.p);
        cudaMemcpyAsync(span.data(), d.p, ntiles * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        cudaError_t ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) st = cuda_fail(ce, "tile spans");
      }
    }
    if (st == FEA_OK) {
      const int64_t cut = P->max_tile_nnz / 2;
      std::vector<int32_t> list;
      list.reserve(ntiles);
      for (int64_t t = 0; t < ntiles; ++t)
        if (span[t] > cut) {
          list.push_back((int32_t)t);
          P->heavy_span = std::max<int64_t>(P->heavy_span, span[t]);
        }
      P->n_heavy = (int64_t)list.size();
      for (int64_t t = 0; t < ntiles; ++t)
        if (span[t] <= cut) {
          list.push_back((int32_t)t);
          P->light_span = std::max<int64_t>(P->light_span, span[t]);
        }
      P->n_light = ntiles - P->n_heavy;
      if ((st = dalloc(&P->class_list, std::max<size_t>(list.size(), 1))) == FEA_OK && !list.empty()) {
        cudaError_t ce = cudaMemcpy(P->class_list, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) st = cuda_fail(ce, "tile classes");
      }
    }
  }
  // the tiled local-row layout of the bulk-copy scatter (scalar patterns)
  if (st == FEA_OK && ndpn == 1) st = build_tiled(m, P, B, s);
  if (st != FEA_OK) {
    free_pattern(P);
    return st;
  }
  m->pat[order][ndpn] = P;
  return FEA_OK;
}

fea_status build_stages(fea_mesh* m, Pattern* P, int stages, cudaStream_t s) {
  if (P->stages == stages) return FEA_OK;
  dfree(P->tile_list);
  P->stage_ptr.clear();
  P->stages = 0;
  const Base* B = m->base[P->order];
  const int64_t ntiles = (P->ndof + P->rows_per_tile - 1) / P->rows_per_tile;
  const int64_t E = m->n_elems;
  P->chunk = std::max<int64_t>(1, (E + stages - 1) / stages);
  std::vector<int32_t> st(ntiles > 0 ? ntiles : 1), list(ntiles > 0 ? ntiles : 1);
  if (ntiles > 0) {
    Tmp<int32_t> d;
    FEA_TRY(d.alloc(ntiles));
    k_tile_stage<<<blocks_for(ntiles, 128), 128, 0, s>>>(P->ndof, P->ndpn, P->rows_per_tile, B->nb, B->inc_ptr, B->inc,
                                                          P->chunk, d.p);
    FEA_CUDA(cudaGetLastError());
    FEA_CUDA(cudaMemcpyAsync(st.data(), d.p, ntiles * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FEA_CUDA(cudaStreamSynchronize(s));
  }
  // counting sort of the tiles by stage (ascending tile id inside a stage)
  P->stage_ptr.assign(stages + 1, 0);
  for (int64_t t = 0; t < ntiles; ++t) P->stage_ptr[std::min(st[t], stages - 1) + 1] += 1;
  for (int k = 0; k < stages; ++k) P->stage_ptr[k + 1] += P->stage_ptr[k];
  std::vector<int64_t> cur(P->stage_ptr.begin(), P->stage_ptr.end() - 1);
  for (int64_t t = 0; t < ntiles; ++t) list[cur[std::min(st[t], stages - 1)]++] = (int32_t)t;
  FEA_TRY(dalloc(&P->tile_list, ntiles));
  if (ntiles > 0)
    FEA_CUDA(cudaMemcpy(P->tile_list, list.data(), ntiles * sizeof(int32_t), cudaMemcpyHostToDevice));
  P->stages = stages;
  return FEA_OK;
}

fea_status build_emap(fea_mesh* m, int order, cudaStream_t s) {
  FEA_TRY(build_pattern(m, order, 1, s));
  Base* B = m->base[order];
  if (B->emap) return FEA_OK;
  FEA_TRY(dalloc(&B->emap, (size_t)m->n_elems * B->nb * B->nb));
  k_emap<<<blocks_for(B->nsd, 128), 128, 0, s>>>(B->nsd, B->nb, B->slot_width, B->inc_ptr, B->inc, B->slot, B->rp,
                                                 B->emap);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

}  // namespace fea
