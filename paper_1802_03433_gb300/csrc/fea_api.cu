// C-ABI entry points of libfea (declared in include/fea.h): argument checks,
// handle lifetime, error reporting.  Compute happens in the kernels of
// pattern.cu, assemble.cu and adjoint.cu.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "internal.cuh"

namespace fea {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

fea_status fail(fea_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

fea_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? FEA_ERR_NOMEM : FEA_ERR_CUDA;
}

fea_status ensure_scratch(Scratch& sc, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (sc.bytes >= bytes) return FEA_OK;
  if (sc.ptr) cudaFree(sc.ptr);
  sc.ptr = nullptr;
  sc.bytes = 0;
  cudaError_t e = cudaMalloc(&sc.ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sc.ptr = nullptr;
    return fail(FEA_ERR_NOMEM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
  }
  sc.bytes = bytes;
  return FEA_OK;
}

fea_status read_and_clear_err(fea_mesh* m, cudaStream_t s) {
  FEA_CUDA(cudaStreamSynchronize(s));
  int h = 0;
  FEA_CUDA(cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) FEA_CUDA(cudaMemset(m->err, 0, sizeof(int)));
  if (h & DEV_ERR_INDEX) return fail(FEA_ERR_INDEX, "connectivity index out of range or repeated");
  if (h & DEV_ERR_OVERFLOW) return fail(FEA_ERR_OVERFLOW, "a row exceeds the scatter limits");
  if (h & DEV_ERR_TIMEOUT) return fail(FEA_ERR_TIMEOUT, "a bounded device wait gave up");
  if (h & DEV_ERR_DEGENERATE) return fail(FEA_ERR_DEGENERATE, "an element has det J <= 0");
  return FEA_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

fea_status check_form(const fea_mesh* m, const fea_form* f, const fea_coeffs* c, const fea_quadrature* q) {
  if (!m || !f || !c || !q) return fail(FEA_ERR_ARG, "NULL mesh, form, coeffs or quadrature");
  if (f->order != FEA_P1 && f->order != FEA_P2) return fail(FEA_ERR_ARG, "order must be FEA_P1 or FEA_P2");
  if (f->kind != FEA_POISSON && f->kind != FEA_DIFFUSION_MASS && f->kind != FEA_ELASTICITY)
    return fail(FEA_ERR_ARG, "unknown form kind");
  if (f->kind == FEA_ELASTICITY && f->order != FEA_P1) return fail(FEA_ERR_ARG, "elasticity is P1 only");
  if (q->npts != 1 && q->npts != 4 && q->npts != 11) return fail(FEA_ERR_ARG, "npts must be 1, 4 or 11");
  if (q->prec != FEA_FP64 && q->prec != FEA_MIXED) return fail(FEA_ERR_ARG, "prec must be FEA_FP64 or FEA_MIXED");
  if (c->f_kind < FEA_LOAD_NONE || c->f_kind > FEA_LOAD_SINPROD) return fail(FEA_ERR_ARG, "unknown load kind");
  if ((c->kappa && !aligned(c->kappa, 8)) || (c->lame_lambda && !aligned(c->lame_lambda, 8)) ||
      (c->lame_mu && !aligned(c->lame_mu, 8)))
    return fail(FEA_ERR_ARG, "coefficient arrays must be 8-byte aligned");
  return FEA_OK;
}

}  // namespace fea

using namespace fea;

extern "C" {

const char* fea_last_error(void) { return g_last_error.c_str(); }

const char* fea_status_string(fea_status s) {
  switch (s) {
    case FEA_OK: return "FEA_OK";
    case FEA_ERR_ARG: return "FEA_ERR_ARG";
    case FEA_ERR_INDEX: return "FEA_ERR_INDEX";
    case FEA_ERR_DEGENERATE: return "FEA_ERR_DEGENERATE";
    case FEA_ERR_OVERFLOW: return "FEA_ERR_OVERFLOW";
    case FEA_ERR_NOMEM: return "FEA_ERR_NOMEM";
    case FEA_ERR_CUDA: return "FEA_ERR_CUDA";
    case FEA_ERR_TIMEOUT: return "FEA_ERR_TIMEOUT";
    case FEA_ERR_STATE: return "FEA_ERR_STATE";
  }
  return "FEA_ERR_UNKNOWN";
}

fea_status fea_mesh_create(const double* x, const double* y, const double* z, int64_t n_nodes,
                           const int32_t* tets, int64_t n_elems, void* stream, fea_mesh** out) {
  g_last_error.clear();
  if (!out) return fail(FEA_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!x || !y || !z) return fail(FEA_ERR_ARG, "coordinate array is NULL");
  if (n_nodes <= 0 || n_nodes > (int64_t)INT32_MAX) return fail(FEA_ERR_ARG, "n_nodes must be in [1, INT32_MAX]");
  if (n_elems < 0 || n_elems > (int64_t)INT32_MAX / 10) return fail(FEA_ERR_ARG, "n_elems out of range");
  if (n_elems > 0 && !tets) return fail(FEA_ERR_ARG, "tets is NULL");
  if (!aligned(x, 8) || !aligned(y, 8) || !aligned(z, 8) || (tets && !aligned(tets, 4)))
    return fail(FEA_ERR_ARG, "misaligned array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fea_mesh* m = new fea_mesh();
  m->x = x;
  m->y = y;
  m->z = z;
  m->n_nodes = n_nodes;
  m->n_elems = n_elems;
  cudaError_t e = cudaMalloc(&m->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->tets, 4 * (size_t)(n_elems > 0 ? n_elems : 1) * sizeof(int32_t));
  if (e != cudaSuccess) {
    fea_status st = cuda_fail(e, "fea_mesh_create allocation");
    fea_mesh_destroy(m);
    return st;
  }
  e = cudaMemsetAsync(m->err, 0, sizeof(int), s);
  if (e == cudaSuccess && n_elems > 0)
    e = cudaMemcpyAsync(m->tets, tets, 4 * (size_t)n_elems * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    fea_status st = cuda_fail(e, "fea_mesh_create copy");
    fea_mesh_destroy(m);
    return st;
  }
  fea_status st = validate_connectivity(m, s);
  if (st != FEA_OK) {
    fea_mesh_destroy(m);
    return st;
  }
  *out = m;
  return FEA_OK;
}

fea_status fea_mesh_create_tri(const double* x, const double* y, int64_t n_nodes, const int32_t* tris,
                               int64_t n_elems, void* stream, fea_mesh** out) {
  g_last_error.clear();
  if (!out) return fail(FEA_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!x || !y) return fail(FEA_ERR_ARG, "coordinate array is NULL");
  if (n_nodes <= 0 || n_nodes > (int64_t)INT32_MAX) return fail(FEA_ERR_ARG, "n_nodes must be in [1, INT32_MAX]");
  if (n_elems < 0 || n_elems > (int64_t)INT32_MAX / 10) return fail(FEA_ERR_ARG, "n_elems out of range");
  if (n_elems > 0 && !tris) return fail(FEA_ERR_ARG, "tris is NULL");
  if (!aligned(x, 8) || !aligned(y, 8) || (tris && !aligned(tris, 4))) return fail(FEA_ERR_ARG, "misaligned array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  fea_mesh* m = new fea_mesh();
  m->x = x;
  m->y = y;
  m->z = nullptr;
  m->nvert = 3;
  m->n_nodes = n_nodes;
  m->n_elems = n_elems;
  cudaError_t e = cudaMalloc(&m->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->tets, 3 * (size_t)(n_elems > 0 ? n_elems : 1) * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int), s);
  if (e == cudaSuccess && n_elems > 0)
    e = cudaMemcpyAsync(m->tets, tris, 3 * (size_t)n_elems * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    fea_status st = cuda_fail(e, "fea_mesh_create_tri");
    fea_mesh_destroy(m);
    return st;
  }
  fea_status st = validate_connectivity(m, s);
  if (st != FEA_OK) {
    fea_mesh_destroy(m);
    return st;
  }
  *out = m;
  return FEA_OK;
}

fea_status fea_mesh_set_coords(fea_mesh* m, const double* x, const double* y, const double* z) {
  if (!m || !x || !y || (!z && m->nvert == 4)) return fail(FEA_ERR_ARG, "NULL argument");
  if (!aligned(x, 8) || !aligned(y, 8) || (z && !aligned(z, 8))) return fail(FEA_ERR_ARG, "misaligned array");
  m->x = x;
  m->y = y;
  m->z = z;
  return FEA_OK;
}

fea_status fea_mesh_set_stages(fea_mesh* m, int32_t stages) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (stages < 1 || stages > 16) return fail(FEA_ERR_ARG, "stages must be in [1, 16]");
  m->stages = stages;
  return FEA_OK;
}

fea_status fea_mesh_set_load_split(fea_mesh* m, int32_t mode) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (mode < -1 || mode > 3) return fail(FEA_ERR_ARG, "mode must be -1, 0, 1, 2 or 3");
  m->load_split = mode;
  return FEA_OK;
}

fea_status fea_mesh_set_scatter_classes(fea_mesh* m, int32_t mode) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (mode < -1 || mode > 3) return fail(FEA_ERR_ARG, "mode must be -1, 0, 1, 2 or 3");
  m->tile_classes = mode;
  return FEA_OK;
}

fea_status fea_mesh_set_scatter(fea_mesh* m, int32_t mode) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (mode < FEA_SCATTER_AUTO || mode > FEA_SCATTER_CHUNKED) return fail(FEA_ERR_ARG, "mode must be 0, 1 or 2");
  m->scatter = mode;
  return FEA_OK;
}

fea_status fea_mesh_set_scatter_stages(fea_mesh* m, int32_t stages) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (stages != 0 && (stages < 2 || stages > 4)) return fail(FEA_ERR_ARG, "stages must be 0, 2, 3 or 4");
  m->tiled_stages = stages;
  return FEA_OK;
}

fea_status fea_mesh_destroy(fea_mesh* m) {
  if (!m) return FEA_OK;
  cudaDeviceSynchronize();
  for (int k = 0; k <= 16; ++k)
    if (m->chunk_ev[k]) cudaEventDestroy(m->chunk_ev[k]);
  if (m->side) cudaStreamDestroy(m->side);
  for (int o = 0; o < 3; ++o)
    for (int d = 0; d < 4; ++d) free_pattern(m->pat[o][d]);
  for (int o = 2; o >= 1; --o) free_base(m->base[o]);
  for (int i = 0; i < 3; ++i)
    if (m->ev[i]) cudaEventDestroy(m->ev[i]);
  if (m->lm.ptr) cudaFree(m->lm.ptr);
  if (m->fl.ptr) cudaFree(m->fl.ptr);
  if (m->part.ptr) cudaFree(m->part.ptr);
  if (m->npart.ptr) cudaFree(m->npart.ptr);
  if (m->gxs.ptr) cudaFree(m->gxs.ptr);
  if (m->bc.ptr) cudaFree(m->bc.ptr);
  if (m->cg.ptr) cudaFree(m->cg.ptr);
  if (m->solve_ev) cudaEventDestroy(m->solve_ev);
  if (m->solve_stream) cudaStreamDestroy(m->solve_stream);
  if (m->tets) cudaFree(m->tets);
  if (m->err) cudaFree(m->err);
  delete m;
  return FEA_OK;
}

fea_status fea_mesh_check(fea_mesh* m, void* stream) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  return read_and_clear_err(m, static_cast<cudaStream_t>(stream));
}

fea_status fea_pattern(fea_mesh* m, int32_t order, int32_t dofs_per_node, int64_t* ndof, int64_t* nnz, void* stream) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (order != FEA_P1 && order != FEA_P2) return fail(FEA_ERR_ARG, "order must be FEA_P1 or FEA_P2");
  if (dofs_per_node != 1 && dofs_per_node != 3) return fail(FEA_ERR_ARG, "dofs_per_node must be 1 or 3");
  if (order == FEA_P2 && dofs_per_node != 1) return fail(FEA_ERR_ARG, "vector dofs are P1 only");
  if (m->nvert == 3 && (order != FEA_P1 || dofs_per_node != 1))
    return fail(FEA_ERR_ARG, "triangle meshes have the scalar P1 pattern only");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NvtxRange range("fea_pattern");
  FEA_TRY(build_pattern(m, order, dofs_per_node, s));
  FEA_TRY(read_and_clear_err(m, s));
  const Pattern* P = m->pat[order][dofs_per_node];
  if (ndof) *ndof = P->ndof;
  if (nnz) *nnz = P->nnz;
  return FEA_OK;
}

fea_status fea_pattern_copy(fea_mesh* m, int32_t order, int32_t dofs_per_node, int32_t* row_ptr, int32_t* col_idx,
                            void* stream) {
  if (!m || order < 1 || order > 2 || dofs_per_node < 1 || dofs_per_node > 3)
    return fail(FEA_ERR_ARG, "bad mesh, order or dofs_per_node");
  const Pattern* P = m->pat[order][dofs_per_node];
  if (!P) return fail(FEA_ERR_STATE, "pattern not built");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (row_ptr)
    FEA_CUDA(cudaMemcpyAsync(row_ptr, P->row_ptr, (P->ndof + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (col_idx && P->nnz > 0)
    FEA_CUDA(cudaMemcpyAsync(col_idx, P->col_idx, P->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return FEA_OK;
}

fea_status fea_dof_table_copy(fea_mesh* m, int32_t order, int32_t* edof, void* stream) {
  if (!m || !edof || order < 1 || order > 2) return fail(FEA_ERR_ARG, "bad argument");
  const Base* B = m->base[order];
  if (!B) return fail(FEA_ERR_STATE, "pattern of this order not built");
  if (m->n_elems > 0)
    FEA_CUDA(cudaMemcpyAsync(edof, B->edof, (size_t)B->nb * m->n_elems * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                             static_cast<cudaStream_t>(stream)));
  return FEA_OK;
}

fea_status fea_assemble(fea_mesh* m, const fea_form* form, const fea_coeffs* coeffs, const fea_quadrature* quad,
                        double* values, double* rhs, void* stream) {
  FEA_TRY(check_form(m, form, coeffs, quad));
  if (!values) return fail(FEA_ERR_ARG, "values is NULL");
  if (!aligned(values, 8) || (rhs && !aligned(rhs, 8))) return fail(FEA_ERR_ARG, "misaligned output");
  NvtxRange range("fea_assemble");
  return assemble(m, form, coeffs, quad, values, rhs, static_cast<cudaStream_t>(stream));
}

fea_status fea_assemble_backward(fea_mesh* m, const fea_form* form, const fea_coeffs* coeffs,
                                 const fea_quadrature* quad, const double* grad_values, const double* grad_rhs,
                                 double* grad_kappa, double* grad_x, void* stream) {
  FEA_TRY(check_form(m, form, coeffs, quad));
  if (form->kind == FEA_ELASTICITY) return fail(FEA_ERR_ARG, "backward is implemented for the scalar forms");
  if (m->nvert != 4) return fail(FEA_ERR_ARG, "backward takes tetrahedral meshes");
  if (quad->prec != FEA_FP64) return fail(FEA_ERR_ARG, "backward runs in FP64");
  NvtxRange range("fea_assemble_backward");
  return assemble_backward(m, form, coeffs, quad, grad_values, grad_rhs, grad_kappa, grad_x,
                           static_cast<cudaStream_t>(stream));
}

fea_status fea_profile_enable(fea_mesh* m, int32_t enable) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (enable && !m->ev[0])
    for (int i = 0; i < 3; ++i) FEA_CUDA(cudaEventCreate(&m->ev[i]));
  m->profile = enable != 0;
  return FEA_OK;
}

fea_status fea_profile_last(fea_mesh* m, float* elem_ms, float* scatter_ms) {
  if (!m) return fail(FEA_ERR_ARG, "mesh is NULL");
  if (!m->profiled) return fail(FEA_ERR_STATE, "no profiled fea_assemble call");
  FEA_CUDA(cudaEventSynchronize(m->ev[2]));
  float a = 0.f, b = 0.f;
  FEA_CUDA(cudaEventElapsedTime(&a, m->ev[0], m->ev[1]));
  FEA_CUDA(cudaEventElapsedTime(&b, m->ev[1], m->ev[2]));
  if (elem_ms) *elem_ms = a;
  if (scatter_ms) *scatter_ms = b;
  return FEA_OK;
}

}  // extern "C"
