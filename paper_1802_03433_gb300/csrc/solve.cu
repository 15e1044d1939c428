// Dirichlet conditions and a conjugate-gradient solve on the assembled CSR
// system, closing the loop from assembly to a solution.  The paper assembles
// the pure Neumann operator and leaves the solve out (Sec. 2, Sec. 4.1); this
// file is the step after it.
//
// fea_dirichlet: symmetric elimination.  For a fixed dof d, row d becomes the
// identity row with rhs_d = g_d; every other row i moves A_id g_d to the right
// side and zeroes A_id.  One thread per row, columns in CSR order.
//
// fea_cg: conjugate gradients with the Jacobi (diagonal) preconditioner.
// Every dot product is a fixed-shape reduction (RED_BLOCKS block partials,
// each a fixed tree, then one fixed tree over the partials), so a solve is
// bitwise reproducible.  The scalars (alpha, beta, the residual) never leave
// the device inside the iteration: each iteration is five kernels
// (SpMV + p.q, alpha, x/r/z update + r.z and r.r, beta, p update), a batch of
// CG_BATCH iterations is captured once into a CUDA graph and replayed, and
// the host reads the iteration state between batches.  Once converged (or at
// max_iter, or on a breakdown) the device marks the state done and the
// remaining iterations of the batch change nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace fea {
namespace {

constexpr int SOLVE_T = 256;
constexpr int RED_BLOCKS = 1024;
constexpr int VL = 4;  // threads per row in the SpMV
constexpr int CG_BATCH = 16;

// ------------------------------------------------------------------ Dirichlet
__global__ void k_mark(const int32_t* __restrict__ dofs, int64_t n, const double* __restrict__ g, int64_t ndof,
                       uint8_t* __restrict__ fixed, double* __restrict__ gv, int* err) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = dofs[k];
    if (d < 0 || d >= ndof) {
      atomicOr(err, DEV_ERR_INDEX);
      continue;
    }
    fixed[d] = 1;
    gv[d] = g ? g[k] : 0.0;
  }
}

__global__ void k_dirichlet_rows(int64_t ndof, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const uint8_t* __restrict__ fixed, const double* __restrict__ gv,
                                 double* __restrict__ values, double* __restrict__ rhs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p0 = rp[i], p1 = rp[i + 1];
    if (fixed[i]) {
      for (int32_t p = p0; p < p1; ++p) values[p] = ci[p] == i ? 1.0 : 0.0;
      if (rhs) rhs[i] = gv[i];
    } else {
      double acc = rhs ? rhs[i] : 0.0;
      for (int32_t p = p0; p < p1; ++p) {
        const int32_t c = ci[p];
        if (fixed[c]) {
          acc -= values[p] * gv[c];
          values[p] = 0.0;
        }
      }
      if (rhs) rhs[i] = acc;
    }
  }
}

// ------------------------------------------------------------------ reductions
// Block sum of v in a fixed tree order; thread 0 writes it to out.
__device__ __forceinline__ void block_sum_to(double v, double* out) {
  __shared__ double sh[SOLVE_T / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < SOLVE_T / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) *out = w;
  }
  __syncthreads();
}

// Sum of partials[0 .. RED_BLOCKS) in a fixed order (one block of 1024).
__device__ __forceinline__ double sum_partials(const double* __restrict__ partials) {
  __shared__ double sh[32];
  double v = partials[threadIdx.x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double w = 0.0;
  if (threadIdx.x < 32) {
    w = sh[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
  }
  __syncthreads();  // sh is reused by the next call
  return w;         // valid in thread 0
}

// ------------------------------------------------------------------ CG state
struct CGState {
  double rz;       // r . z of the current iterate
  double pq;       // p . A p
  double alpha, beta;
  double rr;       // r . r
  double bb;       // b . b
  double target;   // rtol^2 * (b . b) (or rtol^2 when b = 0)
  int32_t it;      // iterations done
  int32_t max_it;
  int32_t done;    // 0 running, 1 converged, 2 max_iter, 3 breakdown (p . A p <= 0)
  int32_t pad;
};

struct CGArgs {
  int64_t n;
  const int32_t* rp;
  const int32_t* ci;
  const double* A;
  const double* b;
  double* x;
  double* r;
  double* z;
  double* p;
  double* q;
  double* dinv;
  double* part;  // [3][RED_BLOCKS]
  CGState* st;
};

// y = A v and the block partial of v . y (VL threads per row, fixed order).
__global__ void __launch_bounds__(SOLVE_T) k_spmv_dot(CGArgs C, const double* __restrict__ v, double* __restrict__ y,
                                                        double* __restrict__ part) {
  const int lane = threadIdx.x % VL;
  double local = 0.0;
  const int64_t rows_per_pass = (int64_t)gridDim.x * (SOLVE_T / VL);
  for (int64_t i = (int64_t)blockIdx.x * (SOLVE_T / VL) + threadIdx.x / VL; i - threadIdx.x / VL < C.n;
       i += rows_per_pass) {
    double s = 0.0;
    if (i < C.n) {
      const int32_t p0 = C.rp[i], p1 = C.rp[i + 1];
      for (int32_t k = p0 + lane; k < p1; k += VL) s = fma(C.A[k], v[C.ci[k]], s);
    }
#pragma unroll
    for (int o = VL / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, VL);
    if (i < C.n && lane == 0) {
      y[i] = s;
      local = fma(v[i], s, local);
    }
  }
  block_sum_to(local, part + blockIdx.x);
}

// Diagonal inverse, r = b - q (q = A x), z = dinv r, p = z; partials r.z, r.r, b.b.
__global__ void __launch_bounds__(SOLVE_T) k_cg_init(CGArgs C) {
  double rz = 0.0, rr = 0.0, bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * SOLVE_T + threadIdx.x; i < C.n; i += (int64_t)gridDim.x * SOLVE_T) {
    double d = 0.0;
    for (int32_t k = C.rp[i]; k < C.rp[i + 1]; ++k)
      if (C.ci[k] == i) d = C.A[k];
    const double di = d != 0.0 ? 1.0 / d : 1.0;
    C.dinv[i] = di;
    const double bi = C.b[i];
    const double ri = bi - C.q[i];
    const double zi = di * ri;
    C.r[i] = ri;
    C.z[i] = zi;
    C.p[i] = zi;
    rz = fma(ri, zi, rz);
    rr = fma(ri, ri, rr);
    bb = fma(bi, bi, bb);
  }
  block_sum_to(rz, C.part + blockIdx.x);
  block_sum_to(rr, C.part + RED_BLOCKS + blockIdx.x);
  block_sum_to(bb, C.part + 2 * RED_BLOCKS + blockIdx.x);
}

__global__ void __launch_bounds__(RED_BLOCKS) k_cg_init_finish(CGArgs C, double rtol2) {
  const double rz = sum_partials(C.part);
  const double rr = sum_partials(C.part + RED_BLOCKS);
  const double bb = sum_partials(C.part + 2 * RED_BLOCKS);
  if (threadIdx.x == 0) {
    CGState& s = *C.st;
    s.rz = rz;
    s.rr = rr;
    s.bb = bb;
    s.target = rtol2 * (bb > 0.0 ? bb : 1.0);
    s.it = 0;
    s.done = rr <= s.target ? 1 : (s.max_it <= 0 ? 2 : 0);
    s.alpha = s.beta = 0.0;
  }
}

__global__ void __launch_bounds__(RED_BLOCKS) k_cg_alpha(CGArgs C) {
  const double pq = sum_partials(C.part);
  if (threadIdx.x == 0) {
    CGState& s = *C.st;
    s.pq = pq;
    if (s.done) {
      s.alpha = 0.0;
    } else if (!(pq > 0.0)) {
      s.alpha = 0.0;
      s.done = 3;
    } else {
      s.alpha = s.rz / pq;
    }
  }
}

// x += alpha p, r -= alpha q, z = dinv r; partials r.z and r.r.
__global__ void __launch_bounds__(SOLVE_T) k_cg_update(CGArgs C) {
  const CGState& s = *C.st;
  const double a = s.alpha;
  const bool live = s.done == 0;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * SOLVE_T + threadIdx.x; i < C.n; i += (int64_t)gridDim.x * SOLVE_T) {
    double ri = C.r[i];
    if (live) {
      C.x[i] = fma(a, C.p[i], C.x[i]);
      ri = fma(-a, C.q[i], ri);
      C.r[i] = ri;
    }
    const double zi = C.dinv[i] * ri;
    C.z[i] = zi;
    rz = fma(ri, zi, rz);
    rr = fma(ri, ri, rr);
  }
  block_sum_to(rz, C.part + RED_BLOCKS + blockIdx.x);
  block_sum_to(rr, C.part + 2 * RED_BLOCKS + blockIdx.x);
}

__global__ void __launch_bounds__(RED_BLOCKS) k_cg_beta(CGArgs C) {
  const double rz = sum_partials(C.part + RED_BLOCKS);
  const double rr = sum_partials(C.part + 2 * RED_BLOCKS);
  if (threadIdx.x == 0) {
    CGState& s = *C.st;
    if (s.done) {
      s.beta = 0.0;
    } else {
      s.it += 1;
      s.rr = rr;
      s.beta = s.rz != 0.0 ? rz / s.rz : 0.0;
      s.rz = rz;
      if (rr <= s.target) s.done = 1;
      else if (s.it >= s.max_it) s.done = 2;
    }
  }
}

// p = z + beta p (the next direction; unchanged once done).
__global__ void __launch_bounds__(SOLVE_T) k_cg_dir(CGArgs C) {
  const CGState& s = *C.st;
  if (s.done) return;
  const double b = s.beta;
  for (int64_t i = (int64_t)blockIdx.x * SOLVE_T + threadIdx.x; i < C.n; i += (int64_t)gridDim.x * SOLVE_T)
    C.p[i] = fma(b, C.p[i], C.z[i]);
}

void cg_iteration(const CGArgs& C, cudaStream_t s) {
  k_spmv_dot<<<RED_BLOCKS, SOLVE_T, 0, s>>>(C, C.p, C.q, C.part);
  k_cg_alpha<<<1, RED_BLOCKS, 0, s>>>(C);
  k_cg_update<<<RED_BLOCKS, SOLVE_T, 0, s>>>(C);
  k_cg_beta<<<1, RED_BLOCKS, 0, s>>>(C);
  k_cg_dir<<<RED_BLOCKS, SOLVE_T, 0, s>>>(C);
}

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" {

fea_status fea_dirichlet(fea_mesh* m, int32_t order, int32_t ndpn, const int32_t* dofs, int64_t n, const double* g,
                         double* values, double* rhs, void* stream) {
  if (!m || !values) return fail(FEA_ERR_ARG, "NULL mesh or values");
  if (n < 0 || (n > 0 && !dofs)) return fail(FEA_ERR_ARG, "bad dof list");
  if (order < 1 || order > 2 || (ndpn != 1 && ndpn != 3)) return fail(FEA_ERR_ARG, "bad order or dofs_per_node");
  Pattern* P = m->pat[order][ndpn];
  if (!P) return fail(FEA_ERR_STATE, "fea_dirichlet: build the pattern of (order, dofs_per_node) first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N = P->ndof;
  const size_t gv_bytes = (size_t)N * sizeof(double);
  FEA_TRY(ensure_scratch(m->bc, gv_bytes + (size_t)N + 16));
  double* gv = static_cast<double*>(m->bc.ptr);
  uint8_t* fixed = reinterpret_cast<uint8_t*>(gv + N);
  FEA_CUDA(cudaMemsetAsync(fixed, 0, (size_t)N, s));
  if (n > 0) {
    const unsigned gb = (unsigned)std::min<int64_t>((n + SOLVE_T - 1) / SOLVE_T, 4096);
    k_mark<<<gb, SOLVE_T, 0, s>>>(dofs, n, g, N, fixed, gv, m->err);
    FEA_CUDA(cudaGetLastError());
  }
  if (N > 0) {
    const unsigned gb = (unsigned)std::min<int64_t>((N + SOLVE_T - 1) / SOLVE_T, 65535);
    k_dirichlet_rows<<<gb, SOLVE_T, 0, s>>>(N, P->row_ptr, P->col_idx, fixed, gv, values, rhs);
    FEA_CUDA(cudaGetLastError());
  }
  return FEA_OK;
}

fea_status fea_cg(fea_mesh* m, int32_t order, int32_t ndpn, const double* values, const double* b, double* x,
                  double rtol, int32_t max_iter, int32_t* iters, double* rel_res, void* stream) {
  if (!m || !values || !b || !x) return fail(FEA_ERR_ARG, "NULL mesh, values, b or x");
  if (order < 1 || order > 2 || (ndpn != 1 && ndpn != 3)) return fail(FEA_ERR_ARG, "bad order or dofs_per_node");
  if (!(rtol >= 0.0) || max_iter < 0) return fail(FEA_ERR_ARG, "rtol must be >= 0 and max_iter >= 0");
  Pattern* P = m->pat[order][ndpn];
  if (!P) return fail(FEA_ERR_STATE, "fea_cg: build the pattern of (order, dofs_per_node) first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N = P->ndof;
  const size_t vec = ((size_t)N * sizeof(double) + 255) / 256 * 256;
  FEA_TRY(ensure_scratch(m->cg, 5 * vec + 3 * RED_BLOCKS * sizeof(double) + sizeof(CGState)));
  char* base = static_cast<char*>(m->cg.ptr);
  CGArgs C{};
  C.n = N;
  C.rp = P->row_ptr;
  C.ci = P->col_idx;
  C.A = values;
  C.b = b;
  C.x = x;
  C.r = reinterpret_cast<double*>(base);
  C.z = reinterpret_cast<double*>(base + vec);
  C.p = reinterpret_cast<double*>(base + 2 * vec);
  C.q = reinterpret_cast<double*>(base + 3 * vec);
  C.dinv = reinterpret_cast<double*>(base + 4 * vec);
  C.part = reinterpret_cast<double*>(base + 5 * vec);
  C.st = reinterpret_cast<CGState*>(base + 5 * vec + 3 * RED_BLOCKS * sizeof(double));

  // The iteration graph is captured on the mesh's own stream (capture is not
  // allowed on the legacy default stream), ordered after the caller's work.
  if (!m->solve_stream) FEA_CUDA(cudaStreamCreateWithFlags(&m->solve_stream, cudaStreamNonBlocking));
  if (!m->solve_ev) FEA_CUDA(cudaEventCreateWithFlags(&m->solve_ev, cudaEventDisableTiming));
  FEA_CUDA(cudaEventRecord(m->solve_ev, s));
  s = m->solve_stream;
  FEA_CUDA(cudaStreamWaitEvent(s, m->solve_ev, 0));
  CGState h{};
  h.max_it = max_iter;
  FEA_CUDA(cudaMemcpyAsync(C.st, &h, sizeof(CGState), cudaMemcpyHostToDevice, s));
  // r = b - A x
  k_spmv_dot<<<RED_BLOCKS, SOLVE_T, 0, s>>>(C, x, C.q, C.part);
  k_cg_init<<<RED_BLOCKS, SOLVE_T, 0, s>>>(C);
  k_cg_init_finish<<<1, RED_BLOCKS, 0, s>>>(C, rtol * rtol);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaMemcpyAsync(&h, C.st, sizeof(CGState), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));

  if (!h.done) {
    // one batch of iterations as a CUDA graph, replayed until done
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    FEA_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < CG_BATCH; ++k) cg_iteration(C, s);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    while (e == cudaSuccess && !h.done) {
      e = cudaGraphLaunch(exec, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&h, C.st, sizeof(CGState), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "fea_cg iteration graph");
  }
  if (iters) *iters = h.it;
  if (rel_res) *rel_res = std::sqrt(h.rr / (h.bb > 0.0 ? h.bb : 1.0));
  if (h.done == 3) return fail(FEA_ERR_ARG, "fea_cg: p . A p <= 0 (the matrix is not positive definite)");
  return FEA_OK;
}

}  // extern "C"
