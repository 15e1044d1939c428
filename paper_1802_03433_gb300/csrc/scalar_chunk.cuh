// Chunked scatter of the scalar forms (P1 and P2 -div(kappa grad u) [+ mass
// u]): one CTA per chunk of elements (chunks.cu) adds the entries of its
// elements into shared memory as fixed-point integers, one accumulator per
// pair of scalar dofs the chunk couples, then writes each coupling the chunk
// completes to the CSR values (entries (i, j) and (j, i), the same value) and
// each coupling it shares as one FP64 partial sum, added in chunk order by
// k_chunk_reduce_scalar.  The fixed-point scheme, its bounds and its
// determinism are those of the elasticity kernel (elast_chunk.cu,
// chunk_common.cuh).  The element arithmetic is that of the local-row
// kernels (elem_scalar_body); the FP64 P2 entries, which those kernels form
// as exact integer sums on a per-element scale, are moved onto the slot's
// scale by an integer shift, without an FP64 conversion.
#pragma once

#include <cuda_runtime.h>

#include "chunk_common.cuh"

namespace fea {
namespace chunkfx {

constexpr int SC_T = 128;  // element threads per CTA (the load role, when split off, adds as many)

// The FP64 P2 entries by FMA chains for inputs outside the fixed-point range
// (out of line: the rare path).  Gu: the ten upper Gram entries row by row,
// then the mass scale t; out: the 55 upper entries.
template <bool MASS>
static __device__ __noinline__ void p2_entries_fp64(const double* __restrict__ Gu, double* __restrict__ out) {
  double G[4][4];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = i; j < 4; ++j) G[i][j] = Gu[k++];
  const double t = Gu[10];
  double tm[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) tm[c] = MASS ? (c == 1 ? t : p2_mass_value(c) * t) : 0.0;
  static_for<55>([&](auto K) {
    constexpr int a = upper_a(10, K), b = upper_b(10, K);
    out[K] = MASS ? p2_stiff<K, double>(G, tm[p2_mass_class(a, b)]) : p2_stiff<K, double>(G);
  });
}

// The upper entries of element e's matrix (K in upper-triangle order), by the
// arithmetic of elem_scalar_body: put(K, value) for FP64 or FP32 values,
// put_fx(K, F, p) for FP64 P2 entries held exactly as the integer F of
// F 2^-p.  Returns |det J|.
template <int ORDER, bool MASS, typename R, typename Put, typename PutFx>
__device__ __forceinline__ double scalar_upper(const ElemArgs& A, int64_t e, const double X[4][3], Put&& put,
                                               PutFx&& put_fx) {
  Geo g;
  geometry(X, g);
  if (!(g.det > 0.0)) atomicOr(A.err, DEV_ERR_DEGENERATE);
  const double adet = fabs(g.det);
  const double kap = A.kappa ? __ldg(A.kappa + e) : A.kappa_const;
  R Gr[4][3];
  grads<R>(g, Gr);
  const R s = R(kap * grad_scale<R>(adet) * (ORDER == 2 ? 1.0 / 20.0 : 1.0));
  constexpr bool SCALE_IN_FMA = ORDER == 1 && MASS && IsDouble<R>::value;
  R G[4][4];
  gram<R>(Gr, SCALE_IN_FMA ? R(1) : s, G);
  if constexpr (ORDER == 1) {
    [[maybe_unused]] R t1 = R(0), t2 = R(0);
    if constexpr (MASS) {
      t1 = R(A.mass * adet * (1.0 / 120.0));
      t2 = t1 + t1;
    }
    static_for<10>([&](auto K) {
      constexpr int a = upper_a(4, K), b = upper_b(4, K);
      R v;
      if constexpr (SCALE_IN_FMA) v = fma(s, G[a][b], a == b ? t2 : t1);
      else if constexpr (MASS) v = G[a][b] + (a == b ? t2 : t1);
      else v = G[a][b];
      put(K, v);
    });
  } else {
    [[maybe_unused]] R t = R(0);
    if constexpr (MASS) t = R(A.mass * adet * (1.0 / 2520.0));
    if constexpr (IsDouble<R>::value) {
      int E = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) E = max(E, exp_bits(G[i][j]) + 2);
      if constexpr (MASS) E = max(E, exp_bits(t) + 5);
      if (E >= P2FX_EMIN && E <= P2FX_EMAX) {
        long long Gf[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = i; j < 4; ++j) Gf[i][j] = to_fx(G[i][j], E - 1019);
        [[maybe_unused]] long long tf = 0;
        if constexpr (MASS) tf = to_fx(t, E - 1017);
        const int p = 1078 - E;
        static_for<55>([&](auto K) {
          constexpr int a = upper_a(10, K), b = upper_b(10, K);
          long long m = 0;
          if constexpr (MASS) m = static_cast<long long>(p2_mass420(a, b)) * tf;
          put_fx(K, p2_stiff_fx<K>(Gf, m), p);
        });
      } else {
        double Gu[11], out[55];
        int k = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = i; j < 4; ++j) Gu[k++] = G[i][j];
        Gu[10] = t;
        p2_entries_fp64<MASS>(Gu, out);
        static_for<55>([&](auto K) { put(K, out[K]); });
      }
    } else {
      static_for<55>([&](auto K) {
        constexpr int a = upper_a(10, K), b = upper_b(10, K);
        R v = p2_stiff<K, R>(G);
        if constexpr (MASS) v = fma(t, R(p2_mass420(a, b)), v);
        put(K, v);
      });
    }
  }
  return adet;
}

// Chunk kernel of the scalar forms.  ROLES (FP64 P2 with a load): the first
// SC_T threads compute the local matrices, the other SC_T the local loads of
// the same elements (the split of the local-row path's k_elem_roles: the
// loads' fixed-point sines run on the integer pipes beside the matrices'
// FP64 work).
template <int ORDER, bool MASS, int LOAD, int NPTS, typename R, bool ROLES>
__global__ void __launch_bounds__(ROLES ? 2 * SC_T : SC_T, ROLES ? 3 : 4) k_scalar_chunk(ElemArgs A, ChunkArgs C) {
  constexpr int NB = ORDER == 1 ? 4 : 10;
  constexpr int NT = ROLES ? 2 * SC_T : SC_T;
  constexpr bool HAS_LOAD = LOAD != LOAD_NONE;
  extern __shared__ unsigned smem_sc[];
  unsigned* alo = smem_sc;                                     // [max_slots]
  int* ahi = reinterpret_cast<int*>(alo + C.max_slots);        // [max_slots]
  unsigned* rlo = reinterpret_cast<unsigned*>(ahi + C.max_slots);  // [max_nodes]
  int* rhi = reinterpret_cast<int*>(rlo + C.max_nodes);        // [max_nodes]
  int* sexp = rhi + C.max_nodes;                               // [max_slots]
  int* rexp = sexp + C.max_slots;                              // [max_nodes]
  const int c = blockIdx.x, tid = threadIdx.x;
  const int e0 = C.cptr[c], ne = C.cptr[c + 1] - e0;
  const int s0 = C.sptr[c], ns = C.sptr[c + 1] - s0;
  const int n0 = C.nptr[c], nn = C.nptr[c + 1] - n0;
  const int KS = C.K;
  for (int i = tid; i < ns; i += NT) {
    alo[i] = 0u;
    ahi[i] = 0;
    sexp[i] = EXP_EMPTY;
  }
  for (int i = tid; i < nn; i += NT) {
    rlo[i] = 0u;
    rhi[i] = 0;
    rexp[i] = EXP_EMPTY;
  }
  __syncthreads();
  // elements dealt to the lanes across 64 segments of the chunk (as in the
  // elasticity kernel), so one warp instruction's atomics seldom collide
  const int L = (ne + 63) >> 6;
  // A: exponent bounds of every slot.  |grad phi| <= max |grad lambda| for P1
  // and <= 4 max |grad lambda| for P2; |phi| <= 1; the mass entries are below
  // |mass| |T|
  for (int i = tid; i < 64 * L; i += NT) {
    const int t = (i & 63) * L + (i >> 6);
    if (t >= ne) continue;
    const int64_t e = C.celem[e0 + t];
    double X[4][3];
    load_element(A, e, X);
    const double kap = A.kappa ? __ldg(A.kappa + e) : A.kappa_const;
    const int2 eb = element_bounds(X, (ORDER == 2 ? 16.0 : 1.0) * fabs(kap), MASS ? fabs(A.mass) : 0.0, C.ef);
    constexpr int NP = NB * (NB + 1) / 2;
    for (int k = 0; k < NP; ++k) atomicMax(sexp + (C.eslot[k * C.es + e0 + t] & 0x7FFF), eb.x);
    if constexpr (HAS_LOAD) {
#pragma unroll
      for (int k = 0; k < NB; ++k) atomicMax(rexp + C.eslot[k * C.es + e0 + t], eb.y);
    }
  }
  __syncthreads();
  // B: the entries (and loads), added in fixed point
  const bool mat = !ROLES || tid < SC_T;
  const int rt = ROLES ? tid % SC_T : tid;
  for (int i = rt; i < 64 * L; i += SC_T) {
    const int t = (i & 63) * L + (i >> 6);
    if (t >= ne) continue;
    const int64_t e = C.celem[e0 + t];
    const uint16_t* es = C.eslot + e0 + t;
    double X[4][3];
    load_element(A, e, X);
    double adet = 0.0;
    if (mat) {
      auto slot_of = [&](int a, int b) { return es[pair_index(NB, a, b) * C.es] & 0x7FFF; };
      adet = scalar_upper<ORDER, MASS, R>(
          A, e, X,
          [&](auto K, R v) {
            const int sl = slot_of(upper_a(NB, K), upper_b(NB, K));
            acc_add(alo + sl, ahi + sl, fx_of(v, C.H - sexp[sl]), KS);
          },
          [&](auto K, long long F, int p) {
            const int sl = slot_of(upper_a(NB, K), upper_b(NB, K));
            acc_add(alo + sl, ahi + sl, fx_shift(F, C.H - sexp[sl] - p), KS);
          });
    }
    if constexpr (HAS_LOAD) {
      if (!ROLES || !mat) {
        if (ROLES) adet = fabs(det_only(X));
        R Xr[4][3];
        vertices_r<R>(X, Xr);
        R Fs[NB];
        shape_load<ORDER, NPTS, LOAD, R>(Xr, Fs);
        const R amp = R(A.fp[0] * adet * (1.0 / 6.0));
#pragma unroll
        for (int a = 0; a < NB; ++a) {
          const int sl = es[a * C.es];
          acc_add(rlo + sl, rhi + sl, fx_of(R(amp * Fs[a]), C.H - rexp[sl]), KS);
        }
      }
    }
  }
  __syncthreads();
  // C: sums to FP64; owned couplings to both CSR entries, shared ones to partials
  for (int k = tid; k < ns; k += NT) {
    const int4 rec = C.srec[s0 + k];
    const int es = sexp[k];
    const double v = es >= EXP_POISON ? __longlong_as_double(0x7FF8000000000000LL)
                                      : f64_of(acc_sum(alo + k, ahi + k, KS), es - C.H);
    if (rec.w < 0) {
      C.values[rec.x] = v;
      if (k >= nn) C.values[rec.y] = v;
    } else {
      C.part[rec.w] = v;
    }
  }
  if (C.rhs) {
    for (int k = tid; k < nn; k += NT) {
      const int2 nr = C.nrec[n0 + k];
      const int es = rexp[k];
      const double f = es >= EXP_POISON ? __longlong_as_double(0x7FF8000000000000LL)
                                        : f64_of(acc_sum(rlo + k, rhi + k, KS), es - C.H);
      if (nr.y < 0) C.rhs[nr.x] = f;
      else C.npart[nr.y] = f;
    }
  }
}

// Launches of one order's chunk kernel (scalar_chunk_p1.cu, scalar_chunk_p2.cu).
fea_status launch_scalar_chunk_p1(bool mass, int load, int npts, bool mixed, const ElemArgs& A, const ChunkArgs& Cg,
                                  int64_t nchunk, size_t smem, cudaStream_t s);
fea_status launch_scalar_chunk_p2(bool mass, int load, int npts, bool mixed, const ElemArgs& A, const ChunkArgs& Cg,
                                  int64_t nchunk, size_t smem, cudaStream_t s);

}  // namespace chunkfx
}  // namespace fea
