// Chunks of the chunked scatter, built once per (mesh, pattern) on the first
// chunked assembly: the P1 vector (elasticity) pattern and the scalar P1 and
// P2 patterns (the structures are described with struct Chunks in
// internal.cuh; the assembly kernels are in elast_chunk.cu and
// scalar_chunk.cu).
//
// The paper's Algorithm 1 (Sec. 5) first accumulates a batch of elements in
// shared memory and only then adds the batch into the global matrix.  The
// chunks are those batches, chosen for locality so that most of a batch's
// couplings are complete inside it:
//  1. every element goes to a cell of a G x G x G grid over the bounding box
//     of the nodes (by its centroid), G^3 about E / CHUNK_MAX_ELEMS;
//  2. the cells are visited in Morton order and cut into chunks of at most
//     CHUNK_MAX_ELEMS elements (whole cells; a larger cell is split), the
//     elements of a cell in ascending id;
//  3. per chunk (one CTA): the pairs of local dofs (vertices for P1, the
//     ten P2 dofs for P2) of its elements are sorted and de-duplicated into
//     slots (scalar dof pairs i <= j, the dof slots i == i first;
//     k_chunk_slots, which also counts them), then, once the slot offsets
//     are known, each slot's record is written from its first candidate
//     (k_chunk_records, no second sort); a slot is
//     owned when the chunk holds every element that contains both dofs (the
//     incidence lists say how many do); each slot gets the CSR positions of
//     its two blocks ((i, j) and (j, i), 3 x 3 for elasticity, single
//     entries otherwise) and, when it is shared, the index of its partial
//     sum;
//  4. the partial sums of every shared coupling (and every shared node's
//     load) get consecutive places, in chunk order, for the second kernel.
// Every step is deterministic: atomics only count or take a minimum, and
// every list filled through an atomic cursor is sorted afterwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "buildutil.cuh"
#include "internal.cuh"

namespace fea {
namespace {

constexpr int BUILD_T = 256;
constexpr int MAX_CELL_LIST = 1024;  // longest cell whose elements sort in registers

// Candidate dof pairs of one chunk (its elements x their NB (NB + 1) / 2
// pairs) that the slot kernel sorts in shared memory.
template <int NB>
constexpr int sort_cap() {
  return NB == 4 ? 4096 : 8192;
}
static_assert(CHUNK_MAX_ELEMS * 10 <= sort_cap<4>(), "P1 chunk too large for the slot sort");
static_assert(CHUNK_MAX_ELEMS_P2 * 55 <= sort_cap<10>(), "P2 chunk too large for the slot sort");

// local dof pair k of an element (pair_index in internal.cuh, inverted)
__device__ __forceinline__ void pair_of(int nb, int k, int& a, int& b) {
  if (k < nb) {
    a = b = k;
    return;
  }
  int q = k - nb;
  a = 0;
  while (q >= nb - 1 - a) {
    q -= nb - 1 - a;
    ++a;
  }
  b = a + 1 + q;
}

// ------------------------------------------------------------------ cells
__global__ void __launch_bounds__(BUILD_T) k_bbox(const double* __restrict__ x, const double* __restrict__ y,
                                                  const double* __restrict__ z, int64_t n, double* __restrict__ out) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v[3] = {x[i], y[i], z[i]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo[k] = fmin(lo[k], v[k]);  // NaN coordinates are ignored
      hi[k] = fmax(hi[k], v[k]);
    }
  }
  __shared__ double sh[6][BUILD_T];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sh[k][threadIdx.x] = lo[k];
    sh[3 + k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    double r = sh[k][0];
    for (int t = 1; t < BUILD_T; ++t) r = k < 3 ? fmin(r, sh[k][t]) : fmax(r, sh[k][t]);
    out[blockIdx.x * 6 + k] = r;
  }
}

struct Grid {
  double lo[3], scale[3];  // cell coordinate = (c - lo) * scale
  int g;
};

__device__ __forceinline__ int cell_coord(double c, double lo, double scale, int g) {
  const double t = (c - lo) * scale;
  if (!(t > 0.0)) return 0;  // also NaN
  return t >= (double)(g - 1) ? g - 1 : (int)t;
}

__global__ void k_cells(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                        const int32_t* __restrict__ tets, int64_t E, Grid G, int32_t* __restrict__ cell,
                        int32_t* __restrict__ cnt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double c[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int32_t v = tets[a * E + e];
    c[0] += x[v];
    c[1] += y[v];
    c[2] += z[v];
  }
  int ix[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) ix[k] = cell_coord(0.25 * c[k], G.lo[k], G.scale[k], G.g);
  const int32_t id = ix[0] + G.g * (ix[1] + G.g * ix[2]);
  cell[e] = id;
  atomicAdd(cnt + id, 1);
}

__global__ void k_cell_fill(const int32_t* __restrict__ cell, int64_t E, const int32_t* __restrict__ cell_off,
                            int32_t* __restrict__ cursor, int32_t* __restrict__ celem) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t c = cell[e];
  celem[cell_off[c] + atomicAdd(cursor + c, 1)] = (int32_t)e;
}

// ------------------------------------------------------------------ slots
struct SlotArgs {
  const int32_t* edof;     // [nb][E] element -> scalar dof
  int64_t E;
  int ndpn;                // dofs per scalar dof of the pattern (3 for elasticity)
  const int32_t* cptr;
  const int32_t* celem;
  const int32_t* rp;       // scalar CSR of the element order
  const int32_t* ci;
  const int32_t* inc_ptr;  // scalar incidences (e * nb + a, ascending e)
  const int32_t* mult;     // [scalar nnz] elements holding both dofs of a coupling (upper positions)
  const int32_t* rp3;      // row pointer of the pattern (vector or scalar)
  // pass 0
  int32_t* cnt_slot;
  int32_t* cnt_node;
  int32_t* cnt_shared;
  int32_t* cnt_shnode;
  int32_t* cnt_max;
  // pass 1
  const int32_t* sptr;
  const int32_t* nptr;
  const int64_t* pbase;
  const int64_t* npbase;
  int4* srec;
  int2* nrec;
  int32_t* pkey;
  uint16_t* eslot;
  int64_t es;              // row stride of eslot
};

__device__ __forceinline__ int32_t col_offset(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t i,
                                              int32_t j) {
  int32_t lo = rp[i], hi = rp[i + 1];
  const int32_t base = lo;
  while (lo < hi) {
    const int32_t m = (lo + hi) >> 1;
    if (ci[m] < j) lo = m + 1;
    else hi = m;
  }
  return lo - base;
}

// Multiplicity of every coupling: for each element and each pair of its
// distinct dofs lo < hi, one count at the scalar CSR position (lo, hi).  A
// chunk owns a coupling when it holds all of the elements counted there.
template <int NB>
__global__ void k_pair_mult(const int32_t* __restrict__ edof, int64_t E, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, int32_t* __restrict__ mult) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int32_t v[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) v[a] = edof[a * E + e];
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int b = a + 1; b < NB; ++b) {
      const int32_t lo = min(v[a], v[b]), hi = max(v[a], v[b]);
      atomicAdd(mult + rp[lo] + col_offset(rp, ci, lo, hi), 1);
    }
}

// Exclusive scan over the block of one int per thread (a thread's count of a
// contiguous range); *total receives the sum.
__device__ __forceinline__ int block_scan_int(int v, int* total) {
  int64_t t64;
  const int64_t ex = block_excl_scan((int64_t)v, &t64);
  *total = (int)t64;
  return (int)ex;
}

// Bits of a slot-sort key (key_bits<NB>): the candidate's index in the
// chunk (below sort_cap) and its transposed bit in the low PB bits, the two
// scalar dofs lo <= hi (DB bits each) above, and the pair flag (a pair of two
// local dofs, not a dof with itself) on top, so that sorting the keys sorts
// the candidates by (pair flag, lo, hi) with no payload beside them.
template <int NB>
struct KeyBits {
  static constexpr int PBITS = NB == 4 ? 12 : 13;  // log2(sort_cap<NB>())
  static constexpr int PB = PBITS + 1;
  static constexpr int DB = (63 - PB) / 2;        // dof bits: 25 (P1), 24 (P2)
};
static_assert((1 << KeyBits<4>::PBITS) == sort_cap<4>() && (1 << KeyBits<10>::PBITS) == sort_cap<10>(),
              "candidate index bits");

__device__ __forceinline__ void block_bitonic_keys(unsigned long long* key, int np) {
  for (int size = 2; size <= np; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (np >> 1); i += blockDim.x) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const unsigned long long a = key[lo], b = key[hi];
        if ((a > b) == asc) {
          key[lo] = b;
          key[hi] = a;
        }
      }
      __syncthreads();
    }
}

template <int NB>
__global__ void __launch_bounds__(BUILD_T) k_chunk_slots(SlotArgs A) {
  constexpr int SORT_CAP = sort_cap<NB>();
  constexpr int NPAIR = NB * (NB + 1) / 2;
  using KB = KeyBits<NB>;
  constexpr unsigned long long DMASK = (1ull << KB::DB) - 1, PMASK = (1ull << KB::PBITS) - 1;
  extern __shared__ unsigned long long smem_u64[];
  unsigned long long* key = smem_u64;                              // [SORT_CAP]
  uint16_t* sid = reinterpret_cast<uint16_t*>(key + SORT_CAP);      // [SORT_CAP] slot of each sorted position
  uint16_t* start = sid + SORT_CAP;                                  // [SORT_CAP + 1] first position of each slot
  __shared__ int s_nn, s_shared, s_shnode, s_max;
  const int c = blockIdx.x, tid = threadIdx.x;
  const int e0 = A.cptr[c], ne = A.cptr[c + 1] - e0;
  const int n = ne * NPAIR;
  int np = 2;
  while (np < n) np <<= 1;
  if (tid == 0) {
    s_nn = 0;
    s_shared = 0;
    s_shnode = 0;
    s_max = 0;
  }
  for (int p = tid; p < np; p += BUILD_T) {
    if (p < n) {
      const int t = p / NPAIR, k = p - NPAIR * t;
      const int64_t e = A.celem[e0 + t];
      int a, b;
      pair_of(NB, k, a, b);
      const uint32_t va = (uint32_t)A.edof[a * A.E + e], vb = (uint32_t)A.edof[b * A.E + e];
      const unsigned long long lo = va < vb ? va : vb, hi = va < vb ? vb : va;
      key[p] = ((unsigned long long)(k >= NB) << 63) | (lo << (KB::PB + KB::DB)) | (hi << KB::PB) |
               ((unsigned long long)(va > vb) << KB::PBITS) | (unsigned long long)p;
    } else {
      key[p] = ~0ull;
    }
  }
  __syncthreads();
  block_bitonic_keys(key, np);
  // runs of equal (pair flag, lo, hi) -> slots
  const int per = (n + BUILD_T - 1) / BUILD_T;
  const int p0 = min(n, tid * per), p1 = min(n, p0 + per);
  int nf = 0;
  for (int p = p0; p < p1; ++p) nf += (p == 0 || (key[p] >> KB::PB) != (key[p - 1] >> KB::PB));
  int ns;
  int sbase = block_scan_int(nf, &ns);
  for (int p = p0; p < p1; ++p) {
    if (p == 0 || (key[p] >> KB::PB) != (key[p - 1] >> KB::PB)) {
      start[sbase] = (uint16_t)p;
      ++sbase;
    }
    sid[p] = (uint16_t)(sbase - 1);
  }
  if (tid == 0) start[ns] = (uint16_t)n;
  __syncthreads();
  // owned or shared, and counts
  int my_nn = 0, my_sh = 0, my_shn = 0, my_max = 0;
  for (int s = tid; s < ns; s += BUILD_T) {
    const unsigned long long k0 = key[start[s]];
    const bool off = (k0 >> 63) != 0;
    const int32_t i = (int32_t)((k0 >> (KB::PB + KB::DB)) & DMASK), j = (int32_t)((k0 >> KB::PB) & DMASK);
    const int cnt = start[s + 1] - start[s];
    const int g = off ? A.mult[A.rp[i] + col_offset(A.rp, A.ci, i, j)] : A.inc_ptr[i + 1] - A.inc_ptr[i];
    my_nn += !off;
    my_sh += cnt != g;
    my_shn += (cnt != g) && !off;
    my_max = max(my_max, cnt);
  }
  atomicAdd(&s_nn, my_nn);
  atomicAdd(&s_shared, my_sh);
  atomicAdd(&s_shnode, my_shn);
  atomicMax(&s_max, my_max);
  __syncthreads();
  // every candidate's slot (chunk-local, the rank of its key), with the
  // transposed bit
  for (int p = tid; p < n; p += BUILD_T) {
    const unsigned long long kp = key[p];
    const int orig = (int)(kp & PMASK);
    const int t = orig / NPAIR, k = orig - NPAIR * t;
    const bool tr = k >= NB && ((kp >> KB::PBITS) & 1ull);
    A.eslot[k * A.es + e0 + t] = (uint16_t)(sid[p] | (tr ? 0x8000 : 0));
  }
  if (tid == 0) {
    A.cnt_slot[c] = ns;
    A.cnt_node[c] = s_nn;
    A.cnt_shared[c] = s_shared;
    A.cnt_shnode[c] = s_shnode;
    A.cnt_max[c] = s_max;
  }
}

// Pass 1: the records of every slot of a chunk, once the slot offsets are
// known, from the slots pass 0 left in eslot (no second sort): a slot's key
// is that of its first candidate, its count the number of candidates that
// name it (shared-memory atomics; only the minimum and the count are taken
// from them, so the records do not depend on their order).
template <int NB>
__global__ void __launch_bounds__(BUILD_T) k_chunk_records(SlotArgs A) {
  constexpr int CAP = sort_cap<NB>();
  constexpr int NPAIR = NB * (NB + 1) / 2;
  extern __shared__ int smem_i32[];
  int* first = smem_i32;                                  // [CAP] first candidate of each slot
  int* cnt = first + CAP;                                 // [CAP] candidates of each slot
  uint8_t* own = reinterpret_cast<uint8_t*>(cnt + CAP);  // [CAP]
  const int c = blockIdx.x, tid = threadIdx.x;
  const int e0 = A.cptr[c], ne = A.cptr[c + 1] - e0;
  const int n = ne * NPAIR;
  const int64_t s_off = A.sptr[c], n_off = A.nptr[c];
  const int ns = A.sptr[c + 1] - A.sptr[c], nn = A.nptr[c + 1] - A.nptr[c];
  for (int q = tid; q < ns; q += BUILD_T) {
    first[q] = INT_MAX;
    cnt[q] = 0;
  }
  __syncthreads();
  for (int p = tid; p < n; p += BUILD_T) {
    const int t = p / NPAIR, k = p - NPAIR * t;
    const int sl = A.eslot[k * A.es + e0 + t] & 0x7FFF;
    if (sl < ns) {
      atomicMin(first + sl, p);
      atomicAdd(cnt + sl, 1);
    }
  }
  __syncthreads();
  // each slot's dof pair i <= j (off_pair: a pair of two local dofs, not a
  // dof with itself) and whether the chunk holds all its elements
  bool off_pair = false;
  auto pair_of_slot = [&](int q, int32_t& i, int32_t& j) {
    const int p = min(first[q], n - 1);  // every slot has a candidate (pass 0 made them from the candidates)
    const int t = p / NPAIR, k = p - NPAIR * t;
    off_pair = k >= NB;
    const int64_t e = A.celem[e0 + t];
    int a, b;
    pair_of(NB, k, a, b);
    const int32_t va = A.edof[a * A.E + e], vb = A.edof[b * A.E + e];
    i = va < vb ? va : vb;
    j = va < vb ? vb : va;
  };
  for (int q = tid; q < ns; q += BUILD_T) {
    int32_t i, j;
    pair_of_slot(q, i, j);
    const int g = off_pair ? A.mult[A.rp[i] + col_offset(A.rp, A.ci, i, j)] : A.inc_ptr[i + 1] - A.inc_ptr[i];
    own[q] = cnt[q] == g;
  }
  __syncthreads();
  // ranks of the shared slots and shared node slots, in slot order
  const int sper = (ns + BUILD_T - 1) / BUILD_T;
  const int q0 = min(ns, tid * sper), q1 = min(ns, q0 + sper);
  int a_sh = 0, a_shn = 0;
  for (int q = q0; q < q1; ++q) {
    a_sh += !own[q];
    a_shn += !own[q] && q < nn;
  }
  int tot;
  int r_sh = block_scan_int(a_sh, &tot);
  int r_shn = block_scan_int(a_shn, &tot);
  for (int q = q0; q < q1; ++q) {
    int32_t i, j;
    pair_of_slot(q, i, j);
    const int32_t oij = col_offset(A.rp, A.ci, i, j), oji = i == j ? oij : col_offset(A.rp, A.ci, j, i);
    const int d = A.ndpn;
    const int32_t Li = A.rp3[d * i + 1] - A.rp3[d * i], Lj = A.rp3[d * j + 1] - A.rp3[d * j];
    const int32_t part = own[q] ? -1 : (int32_t)(A.pbase[c] + r_sh);
    r_sh += !own[q];
    A.srec[s_off + q] = make_int4(A.rp3[d * i] + d * oij, A.rp3[d * j] + d * oji, Li | (Lj << 16), part);
    A.pkey[s_off + q] = A.rp[i] + oij;
    if (q < nn) {
      A.nrec[n_off + q] = make_int2(i, own[q] ? -1 : (int32_t)(A.npbase[c] + r_shn));
      r_shn += !own[q];
    }
  }
}

// ------------------------------------------------------------------ shared couplings
__global__ void k_count_keys(const int32_t* __restrict__ keyv, int kstride, const int32_t* __restrict__ sel,
                             int pstride, int64_t n, int32_t* __restrict__ cnt) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && sel[s * pstride] >= 0) atomicAdd(cnt + keyv[s * kstride], 1);
}

__global__ void k_flags(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = cnt[i] > 0;
}

// One entry per shared visit: its chunk-major partial index goes to the list
// of its key (inv maps it back to the visit); the group's first list
// position and its record are written by every visit (identical values).
__global__ void k_fill_groups(const int32_t* __restrict__ keyv, int kstride, const int32_t* __restrict__ part,
                              int pstride, int64_t n, const int64_t* __restrict__ goff, const int64_t* __restrict__ gid,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ list, int32_t* __restrict__ inv,
                              int32_t* __restrict__ gptr, const int4* __restrict__ srec, int4* __restrict__ grec,
                              int32_t* __restrict__ gnode) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int32_t pi = part[s * pstride];
  if (pi < 0) return;
  const int32_t k = keyv[s * kstride];
  list[goff[k] + atomicAdd(cursor + k, 1)] = pi;
  inv[pi] = (int32_t)s;
  const int64_t g = gid[k];
  gptr[g] = (int32_t)goff[k];
  if (grec) {
    const int4 r = srec[s];
    grec[g] = make_int4(r.x, r.y, r.z, 0);
  }
  if (gnode) gnode[g] = k;
}

// After each group's list is sorted (chunk order), every shared visit gets
// its list position as its partial index: a group's partial sums are then
// contiguous, in chunk order.
__global__ void k_relink(const int32_t* __restrict__ list, int64_t n, const int32_t* __restrict__ inv,
                         int32_t* __restrict__ part, int pstride) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) part[(int64_t)inv[list[p]] * pstride] = (int32_t)p;
}

// Build the partial-sum groups per key (scalar CSR position of a coupling,
// or node id): visits s = 0 .. n-1 with key keyv[s * kstride] and
// chunk-major partial index part[s * pstride] (< 0: not shared), which is
// replaced by the visit's position in its group.
fea_status build_groups(const int32_t* keyv, int kstride, int32_t* part, int pstride, int64_t n, int64_t nkeys,
                        int64_t npart_in, const int4* srec, int64_t* ngroup, int64_t* nlist, int32_t** gptr,
                        int4** grec, int32_t** gnode, cudaStream_t s) {
  Tmp<int32_t> cnt, flag, cur, list, inv;
  Tmp<int64_t> goff, gid;
  FEA_TRY(cnt.alloc(nkeys));
  FEA_TRY(flag.alloc(nkeys));
  FEA_TRY(cur.alloc(nkeys));
  FEA_TRY(goff.alloc(nkeys + 1));
  FEA_TRY(gid.alloc(nkeys + 1));
  FEA_TRY(inv.alloc(npart_in));
  FEA_CUDA(cudaMemsetAsync(cnt.p, 0, nkeys * sizeof(int32_t), s));
  FEA_CUDA(cudaMemsetAsync(cur.p, 0, nkeys * sizeof(int32_t), s));
  if (n > 0) k_count_keys<<<blocks_for(n, 256), 256, 0, s>>>(keyv, kstride, part, pstride, n, cnt.p);
  k_flags<<<blocks_for(nkeys, 256), 256, 0, s>>>(cnt.p, nkeys, flag.p);
  FEA_CUDA(cudaGetLastError());
  FEA_TRY(scan(cnt.p, nkeys, goff.p, s));
  FEA_TRY(scan(flag.p, nkeys, gid.p, s));
  FEA_TRY(read_i64(goff.p + nkeys, nlist, s));
  FEA_TRY(read_i64(gid.p + nkeys, ngroup, s));
  if (*nlist != npart_in) return fail(FEA_ERR_STATE, "chunked scatter: inconsistent partial-sum count");
  FEA_TRY(dalloc(gptr, *ngroup + 1));
  FEA_TRY(list.alloc(*nlist));
  if (grec) FEA_TRY(dalloc(grec, *ngroup));
  if (gnode) FEA_TRY(dalloc(gnode, *ngroup));
  if (n > 0)
    k_fill_groups<<<blocks_for(n, 256), 256, 0, s>>>(keyv, kstride, part, pstride, n, goff.p, gid.p, cur.p, list.p,
                                                      inv.p, *gptr, srec, grec ? *grec : nullptr,
                                                      gnode ? *gnode : nullptr);
  const int32_t tot = (int32_t)*nlist;
  FEA_CUDA(cudaMemcpyAsync(*gptr + *ngroup, &tot, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (*ngroup > 0)
    k_sort_lists<<<(int)std::min<int64_t>(blocks_for(*ngroup, 4), 152 * 64), 128, 0, s>>>(*gptr, *ngroup, list.p);
  if (*nlist > 0) k_relink<<<blocks_for(*nlist, 256), 256, 0, s>>>(list.p, *nlist, inv.p, part, pstride);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaStreamSynchronize(s));
  return FEA_OK;
}

__global__ void k_isolated(const int32_t* __restrict__ inc_ptr, int64_t n, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && inc_ptr[i + 1] == inc_ptr[i]) out[atomicAdd(cursor, 1)] = (int32_t)i;
}

uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t m = 0;
  for (int b = 0; b < 11; ++b)
    m |= ((uint64_t)((x >> b) & 1) << (3 * b)) | ((uint64_t)((y >> b) & 1) << (3 * b + 1)) |
         ((uint64_t)((z >> b) & 1) << (3 * b + 2));
  return m;
}

fea_status build(fea_mesh* m, Pattern* P, Chunks* C, cudaStream_t s) {
  const int64_t E = m->n_elems, N = m->n_nodes;
  const Base* B = m->base[P->order];
  const int NB = B->nb, NPAIR = NB * (NB + 1) / 2;
  const int64_t nsd = B->nsd;  // scalar dofs (the node-slot keys)
  const int CE = NB == 4 ? CHUNK_MAX_ELEMS : CHUNK_MAX_ELEMS_P2;
  C->nb = NB;
  C->npair = NPAIR;
  C->ndpn = P->ndpn;
  // 1. cells
  // the smallest G with G^3 cells of CE elements holding E
  int G = std::max(1, (int)std::cbrt((double)E / CE));
  while ((int64_t)G * G * G * CE < E) ++G;
  const int nbb = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (N + BUILD_T - 1) / BUILD_T));
  Tmp<double> bb;
  FEA_TRY(bb.alloc((size_t)nbb * 6));
  k_bbox<<<nbb, BUILD_T, 0, s>>>(m->x, m->y, m->z, N, bb.p);
  std::vector<double> hb((size_t)nbb * 6);
  FEA_CUDA(cudaMemcpyAsync(hb.data(), bb.p, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  Grid grid{};
  grid.g = G;
  for (int k = 0; k < 3; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int b = 0; b < nbb; ++b) {
      lo = std::fmin(lo, hb[b * 6 + k]);
      hi = std::fmax(hi, hb[b * 6 + 3 + k]);
    }
    const double w = hi - lo;
    grid.lo[k] = std::isfinite(lo) ? lo : 0.0;
    grid.scale[k] = (std::isfinite(w) && w > 0.0) ? G / w : 0.0;
  }
  const int64_t ncell = (int64_t)G * G * G;
  Tmp<int32_t> cell, ccnt, cur, coff;
  FEA_TRY(cell.alloc(E));
  FEA_TRY(ccnt.alloc(ncell));
  FEA_TRY(cur.alloc(ncell));
  FEA_TRY(coff.alloc(ncell));
  FEA_CUDA(cudaMemsetAsync(ccnt.p, 0, ncell * sizeof(int32_t), s));
  FEA_CUDA(cudaMemsetAsync(cur.p, 0, ncell * sizeof(int32_t), s));
  k_cells<<<blocks_for(E, 256), 256, 0, s>>>(m->x, m->y, m->z, m->tets, E, grid, cell.p, ccnt.p);
  std::vector<int32_t> hc(ncell);
  FEA_CUDA(cudaMemcpyAsync(hc.data(), ccnt.p, ncell * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  // 2. cells in Morton order, cut into chunks
  std::vector<std::pair<uint64_t, int32_t>> order;
  order.reserve(ncell);
  for (int64_t c = 0; c < ncell; ++c)
    if (hc[c] > 0) {
      const int ix = (int)(c % G), iy = (int)((c / G) % G), iz = (int)(c / ((int64_t)G * G));
      order.push_back({morton3(ix, iy, iz), (int32_t)c});
    }
  std::sort(order.begin(), order.end());
  std::vector<int32_t> off(ncell, 0), lists, cptr{0};
  int64_t pos = 0, open = 0;
  for (const auto& oc : order) {
    const int32_t k = hc[oc.second];
    if (k > MAX_CELL_LIST) return fail(FEA_ERR_OVERFLOW, "chunked scatter: a cell holds too many elements");
    off[oc.second] = (int32_t)pos;
    lists.push_back((int32_t)pos);
    if (k > CE) {
      if (open) cptr.push_back((int32_t)pos);
      const int parts = (k + CE - 1) / CE;
      for (int q = 1; q < parts; ++q) cptr.push_back((int32_t)(pos + (int64_t)k * q / parts));
      pos += k;
      cptr.push_back((int32_t)pos);
      open = 0;
    } else {
      if (open + k > CE) {
        cptr.push_back((int32_t)pos);
        open = 0;
      }
      pos += k;
      open += k;
    }
  }
  if (open) cptr.push_back((int32_t)pos);
  lists.push_back((int32_t)pos);
  C->nchunk = (int64_t)cptr.size() - 1;
  FEA_TRY(dalloc(&C->cptr, cptr.size()));
  FEA_TRY(dalloc(&C->celem, E + 4));  // padded: bulk copies of a chunk round up to 16 bytes
  Tmp<int32_t> lptr;
  FEA_TRY(lptr.alloc(lists.size()));
  FEA_CUDA(cudaMemcpy(C->cptr, cptr.data(), cptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  FEA_CUDA(cudaMemcpy(coff.p, off.data(), ncell * sizeof(int32_t), cudaMemcpyHostToDevice));
  FEA_CUDA(cudaMemcpy(lptr.p, lists.data(), lists.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  k_cell_fill<<<blocks_for(E, 256), 256, 0, s>>>(cell.p, E, coff.p, cur.p, C->celem);
  const int64_t nl = (int64_t)lists.size() - 1;
  if (nl > 0) k_sort_lists<<<(int)std::min<int64_t>(blocks_for(nl, 4), 152 * 64), 128, 0, s>>>(lptr.p, nl, C->celem);
  FEA_CUDA(cudaGetLastError());
  // 3. slots: counts, then records
  const int64_t nc = C->nchunk;
  Tmp<int32_t> cs, cn, csh, cshn, cmax;
  FEA_TRY(cs.alloc(nc));
  FEA_TRY(cn.alloc(nc));
  FEA_TRY(csh.alloc(nc));
  FEA_TRY(cshn.alloc(nc));
  FEA_TRY(cmax.alloc(nc));
  SlotArgs A{};
  A.edof = B->edof;
  A.E = E;
  A.ndpn = P->ndpn;
  A.cptr = C->cptr;
  A.celem = C->celem;
  A.rp = B->rp;
  A.ci = B->ci;
  A.inc_ptr = B->inc_ptr;
  Tmp<int32_t> mult;
  FEA_TRY(mult.alloc(std::max<int64_t>(B->nnz, 1)));
  FEA_CUDA(cudaMemsetAsync(mult.p, 0, std::max<int64_t>(B->nnz, 1) * sizeof(int32_t), s));
  if (E > 0) {
    if (NB == 4) k_pair_mult<4><<<blocks_for(E, 256), 256, 0, s>>>(B->edof, E, B->rp, B->ci, mult.p);
    else k_pair_mult<10><<<blocks_for(E, 256), 256, 0, s>>>(B->edof, E, B->rp, B->ci, mult.p);
  }
  A.mult = mult.p;
  A.rp3 = P->row_ptr;
  A.cnt_slot = cs.p;
  A.cnt_node = cn.p;
  A.cnt_shared = csh.p;
  A.cnt_shnode = cshn.p;
  A.cnt_max = cmax.p;
  const int cap = NB == 4 ? sort_cap<4>() : sort_cap<10>();
  // pass 0 (sort): every candidate's slot into eslot, and the counts
  C->estride = (E + 7) & ~(int64_t)7;
  FEA_TRY(dalloc(&C->eslot, (size_t)NPAIR * C->estride + 8));
  A.eslot = C->eslot;
  A.es = C->estride;
  if (nsd >= (int64_t(1) << (NB == 4 ? KeyBits<4>::DB : KeyBits<10>::DB)))
    return fail(FEA_ERR_OVERFLOW, "chunked scatter: more scalar dofs than the slot sort's keys hold");
  const size_t smem = (size_t)cap * (8 + 2) + (cap + 1) * 2;
  FEA_CUDA(cudaFuncSetAttribute(NB == 4 ? k_chunk_slots<4> : k_chunk_slots<10>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (nc > 0) {
    if (NB == 4) k_chunk_slots<4><<<(unsigned)nc, BUILD_T, smem, s>>>(A);
    else k_chunk_slots<10><<<(unsigned)nc, BUILD_T, smem, s>>>(A);
  }
  FEA_CUDA(cudaGetLastError());
  std::vector<int32_t> hs(nc), hn(nc), hsh(nc), hshn(nc), hmax(nc);
  FEA_CUDA(cudaMemcpyAsync(hs.data(), cs.p, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(hn.data(), cn.p, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(hsh.data(), csh.p, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(hshn.data(), cshn.p, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(hmax.data(), cmax.p, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> sptr(nc + 1, 0), nptr(nc + 1, 0);
  std::vector<int64_t> pbase(nc + 1, 0), npbase(nc + 1, 0);
  int maxcnt = 1;
  for (int64_t c = 0; c < nc; ++c) {
    if ((int64_t)sptr[c] + hs[c] > INT32_MAX) return fail(FEA_ERR_OVERFLOW, "chunked scatter: too many slots");
    sptr[c + 1] = sptr[c] + hs[c];
    nptr[c + 1] = nptr[c] + hn[c];
    pbase[c + 1] = pbase[c] + hsh[c];
    npbase[c + 1] = npbase[c] + hshn[c];
    C->max_slots = std::max(C->max_slots, hs[c]);
    C->max_nodes = std::max(C->max_nodes, hn[c]);
    maxcnt = std::max(maxcnt, hmax[c]);
  }
  if (pbase[nc] > INT32_MAX) return fail(FEA_ERR_OVERFLOW, "chunked scatter: too many partial sums");
  C->hbits = 0;
  while ((1 << C->hbits) < maxcnt) ++C->hbits;
  // the accumulators of the largest chunk must fit one CTA's shared memory
  // (ndpn^2 sums of two words and an exponent per slot, ndpn sums and an
  // exponent per node slot, and for elasticity the node's staged
  // coordinates, FP64 and split into floats), and a slot may take at most
  // 128 contributions (the
  // fixed-point scale 2^(63 - 2 hbits) keeps 49 bits or more)
  const size_t d = P->ndpn;
  if ((size_t)C->max_slots * (d * d * 8 + 4) + (size_t)C->max_nodes * (d * 8 + 4 + (d == 3 ? 24 + 25 : 0)) +
              (d == 3 ? CHUNK_STAGE_BYTES : 0) > 227 * 1024 ||
      C->hbits > 7)
    return fail(FEA_ERR_OVERFLOW, "chunked scatter: a chunk couples too many node pairs for shared memory");
  C->nslot = sptr[nc];
  C->nnode_slot = nptr[nc];
  C->npart = pbase[nc];
  C->nnpart = npbase[nc];
  FEA_TRY(dalloc(&C->sptr, nc + 1));
  FEA_TRY(dalloc(&C->nptr, nc + 1));
  FEA_TRY(dalloc(&C->srec, C->nslot));
  FEA_TRY(dalloc(&C->nrec, C->nnode_slot));
  Tmp<int64_t> dpb, dnpb;
  Tmp<int32_t> pkey;
  FEA_TRY(dpb.alloc(nc + 1));
  FEA_TRY(dnpb.alloc(nc + 1));
  FEA_TRY(pkey.alloc(C->nslot));
  FEA_CUDA(cudaMemcpy(C->sptr, sptr.data(), (nc + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  FEA_CUDA(cudaMemcpy(C->nptr, nptr.data(), (nc + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
  FEA_CUDA(cudaMemcpy(dpb.p, pbase.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  FEA_CUDA(cudaMemcpy(dnpb.p, npbase.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
  // pass 1 (no sort): the slot records
  A.sptr = C->sptr;
  A.nptr = C->nptr;
  A.pbase = dpb.p;
  A.npbase = dnpb.p;
  A.srec = C->srec;
  A.nrec = C->nrec;
  A.pkey = pkey.p;
  const size_t rsmem = (size_t)cap * (4 + 4 + 1);
  FEA_CUDA(cudaFuncSetAttribute(NB == 4 ? k_chunk_records<4> : k_chunk_records<10>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem));
  if (nc > 0) {
    if (NB == 4) k_chunk_records<4><<<(unsigned)nc, BUILD_T, rsmem, s>>>(A);
    else k_chunk_records<10><<<(unsigned)nc, BUILD_T, rsmem, s>>>(A);
  }
  FEA_CUDA(cudaGetLastError());
  // 4. partial-sum lists of the shared couplings (key: the scalar CSR position
  // of the coupling's upper entry) and of the shared nodes (key: node id)
  int32_t* partcol = reinterpret_cast<int32_t*>(C->srec) + 3;  // .w of every record
  FEA_TRY(build_groups(pkey.p, 1, partcol, 4, C->nslot, B->nnz, C->npart, C->srec, &C->ngroup, &C->npart, &C->gptr,
                       &C->grec, nullptr, s));
  int32_t* nodecol = reinterpret_cast<int32_t*>(C->nrec);
  FEA_TRY(build_groups(nodecol, 2, nodecol + 1, 2, C->nnode_slot, nsd, C->nnpart, nullptr, &C->nngroup, &C->nnpart,
                       &C->ngptr, nullptr, &C->ngnode, s));
  // nodes of no element: no chunk writes their load entries (the set, not
  // its order, matters: they are written with zeros)
  Tmp<int32_t> niso;
  FEA_TRY(niso.alloc(1));
  FEA_TRY(dalloc(&C->iso, nsd));
  FEA_CUDA(cudaMemsetAsync(niso.p, 0, sizeof(int32_t), s));
  k_isolated<<<blocks_for(nsd, 256), 256, 0, s>>>(B->inc_ptr, nsd, niso.p, C->iso);
  int32_t hiso = 0;
  FEA_CUDA(cudaMemcpyAsync(&hiso, niso.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  C->niso = hiso;
  return FEA_OK;
}

}  // namespace

void free_chunks(Chunks* c) {
  if (!c) return;
  dfree(c->cptr);
  dfree(c->celem);
  dfree(c->eslot);
  dfree(c->sptr);
  dfree(c->nptr);
  dfree(c->srec);
  dfree(c->nrec);
  dfree(c->gptr);
  dfree(c->grec);
  dfree(c->ngptr);
  dfree(c->ngnode);
  dfree(c->iso);
  delete c;
}

fea_status build_chunks(fea_mesh* m, Pattern* P, cudaStream_t s) {
  if (P->chunks) return FEA_OK;
  if (P->chunks_failed) return fail(FEA_ERR_OVERFLOW, "chunked scatter: not available for this mesh");
  if (!m->base[P->order] || !(P->ndpn == 1 || (P->order == 1 && P->ndpn == 3)) || m->nvert != 4)
    return fail(FEA_ERR_STATE, "chunked scatter: tetrahedral scalar P1/P2 or P1 vector patterns only");
  NvtxRange range("chunk build");
  Chunks* C = new Chunks();
  fea_status st = build(m, P, C, s);
  if (st == FEA_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "chunk build");
  }
  if (st != FEA_OK) {
    free_chunks(C);
    if (st == FEA_ERR_OVERFLOW) P->chunks_failed = true;
    return st;
  }
  P->chunks = C;
  return FEA_OK;
}

}  // namespace fea
