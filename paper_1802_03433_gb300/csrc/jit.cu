// Runtime specialisation of the element kernel (NVRTC) for user expressions.
//
// The paper's pipeline builds the integrand of the user's weak form
// symbolically, substitutes it into a CUDA kernel template and compiles that
// source with NVRTC while the program runs, then loads and launches it
// (Sec. 5, runtime compilation).  Here the kernel template is elem_user.cuh
// and the user's part is two CUDA C++ expressions: the coefficient k(x, y, z)
// inside the stiffness integral and the load f(x, y, z).  fea_jit_compile
// pastes them into a Spec struct, compiles the template for the requested
// (order, mass term, rule, precision) to an sm_103a cubin, and keeps the cubin
// in the handle (and in a process-wide cache keyed by the full source, so the
// same specialisation is compiled once per process).  NVRTC runs on the host
// only, so compiling needs no GPU.  fea_jit_assemble loads the cubin once
// (cudaLibraryLoadData, context independent), launches it over the mesh and
// finishes with the same deterministic scatter as fea_assemble.
//
// The headers the template needs are embedded at build time
// (jit_headers.inc, generated by build_lib.py from csrc/*.cuh).
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "elem_user.cuh"
#include "gather.cuh"
#include "gather_tiled.cuh"
#include "jit_headers.inc"

struct fea_jit {
  int order = 1;
  bool mass = false;
  double mass_coef = 0.0;
  int npts = 4;
  int prec = FEA_FP64;
  bool has_k = false, has_f = false;
  std::string source;
  std::string log;
  std::vector<char> cubin;
  double compile_ms = 0.0;
  bool cache_hit = false;
  std::mutex mu;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
};

namespace fea {
namespace {

constexpr size_t MAX_EXPR = 4096;

// An expression must stay an expression: no statement or block punctuation,
// no preprocessor, no string or character literals, no comments.
bool expr_ok(const char* e, std::string& why) {
  const std::string s(e);
  if (s.empty()) {
    why = "empty expression";
    return false;
  }
  if (s.size() > MAX_EXPR) {
    why = "expression longer than 4096 characters";
    return false;
  }
  for (char c : s) {
    const unsigned char u = static_cast<unsigned char>(c);
    if (u < 32 || u > 126 || c == ';' || c == '{' || c == '}' || c == '#' || c == '"' || c == '\'' || c == '\\' ||
        c == '`' || c == '@' || c == '$') {
      why = std::string("character '") + (u >= 32 && u <= 126 ? std::string(1, c) : std::string("\\x")) +
            "' is not allowed in an expression";
      return false;
    }
  }
  if (s.find("//") != std::string::npos || s.find("/*") != std::string::npos) {
    why = "comments are not allowed in an expression";
    return false;
  }
  int depth = 0;
  for (char c : s) {
    depth += (c == '(') - (c == ')');
    if (depth < 0) break;
  }
  if (depth != 0) {
    why = "unbalanced parentheses";
    return false;
  }
  return true;
}

std::string point_fn(const char* name, const char* expr) {
  std::string b = "  template <typename R>\n  static __device__ __forceinline__ R " + std::string(name) +
                  "(R x, R y, R z, double p0, double p1, double p2, double p3) {\n";
  b += "    constexpr double pi = 3.141592653589793238462643383279502884;\n";
  b += "    auto sinpi_fx = [](double v) { return fea::sinpi_fx_call(v); };\n";
  b += "    (void)x; (void)y; (void)z; (void)p0; (void)p1; (void)p2; (void)p3; (void)pi; (void)sinpi_fx;\n";
  b += "    return R(" + std::string(expr ? expr : "1") + ");\n  }\n";
  return b;
}

std::string make_source(const fea_jit& j, const char* k_expr, const char* f_expr) {
  std::string s = "#include \"elem_user.cuh\"\nnamespace fea {\nstruct UserSpec {\n";
  s += std::string("  static constexpr bool HAS_K = ") + (j.has_k ? "true" : "false") + ";\n";
  s += std::string("  static constexpr bool HAS_F = ") + (j.has_f ? "true" : "false") + ";\n";
  s += point_fn("k", k_expr);
  s += point_fn("f", f_expr);
  s += "};\n}  // namespace fea\n";
  s += "extern \"C\" __global__ void __launch_bounds__(fea::USER_T) fea_user_elem(fea::UserArgs A) {\n";
  s += "  const int64_t e = (int64_t)blockIdx.x * fea::USER_T + threadIdx.x;\n";
  s += "  if (e < A.E) fea::elem_user_body<" + std::to_string(j.order) + ", " + (j.mass ? "true" : "false") + ", " +
       std::to_string(j.npts) + ", " + (j.prec == FEA_FP64 ? "double" : "float") + ", fea::UserSpec>(A, e);\n}\n";
  return s;
}

#ifdef FEA_CHECKED
const char* const NVRTC_OPTS[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "-DFEA_CHECKED"};
#else
const char* const NVRTC_OPTS[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
#endif

std::mutex g_cache_mu;
std::map<std::string, std::vector<char>>& cubin_cache() {
  static std::map<std::string, std::vector<char>> c;
  return c;
}

fea_status nvrtc_compile(const std::string& src, std::vector<char>& cubin, std::string& log) {
  nvrtcProgram prog = nullptr;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "fea_user_elem.cu", JIT_HEADER_COUNT, JIT_HEADER_SOURCES,
                                     JIT_HEADER_NAMES);
  if (r != NVRTC_SUCCESS) return fail(FEA_ERR_CUDA, std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r));
  r = nvrtcCompileProgram(prog, (int)(sizeof(NVRTC_OPTS) / sizeof(NVRTC_OPTS[0])), NVRTC_OPTS);
  size_t n = 0;
  if (nvrtcGetProgramLogSize(prog, &n) == NVRTC_SUCCESS && n > 1) {
    log.assign(n, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    log.resize(n - 1);
  }
  if (r != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return fail(FEA_ERR_ARG, "NVRTC could not compile the expressions: " + log);
  }
  size_t nc = 0;
  r = nvrtcGetCUBINSize(prog, &nc);
  if (r == NVRTC_SUCCESS && nc > 0) {
    cubin.resize(nc);
    r = nvrtcGetCUBIN(prog, cubin.data());
  }
  nvrtcDestroyProgram(&prog);
  if (r != NVRTC_SUCCESS || nc == 0) return fail(FEA_ERR_CUDA, "NVRTC produced no cubin");
  return FEA_OK;
}

fea_status ensure_loaded(fea_jit* j) {
  std::lock_guard<std::mutex> lock(j->mu);
  if (j->kern) return FEA_OK;
  cudaLibrary_t lib = nullptr;
  cudaError_t e = cudaLibraryLoadData(&lib, j->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLibraryLoadData(runtime-compiled element kernel)");
  cudaKernel_t k = nullptr;
  e = cudaLibraryGetKernel(&k, lib, "fea_user_elem");
  if (e != cudaSuccess) {
    cudaLibraryUnload(lib);
    return cuda_fail(e, "cudaLibraryGetKernel(fea_user_elem)");
  }
  j->lib = lib;
  j->kern = k;
  return FEA_OK;
}

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" {

fea_status fea_jit_compile(const fea_form* form, const fea_quadrature* q, const char* kappa_expr, const char* f_expr,
                           fea_jit** out) {
  if (!form || !q || !out) return fail(FEA_ERR_ARG, "NULL form, quadrature or output");
  *out = nullptr;
  if (form->order != FEA_P1 && form->order != FEA_P2) return fail(FEA_ERR_ARG, "order must be FEA_P1 or FEA_P2");
  if (form->kind != FEA_POISSON && form->kind != FEA_DIFFUSION_MASS)
    return fail(FEA_ERR_ARG, "runtime-compiled kernels take the scalar forms (FEA_POISSON, FEA_DIFFUSION_MASS)");
  if (q->npts != 1 && q->npts != 4 && q->npts != 11) return fail(FEA_ERR_ARG, "npts must be 1, 4 or 11");
  if (q->prec != FEA_FP64 && q->prec != FEA_MIXED) return fail(FEA_ERR_ARG, "prec must be FEA_FP64 or FEA_MIXED");
  std::string why;
  if (kappa_expr && !expr_ok(kappa_expr, why)) return fail(FEA_ERR_ARG, "kappa expression: " + why);
  if (f_expr && !expr_ok(f_expr, why)) return fail(FEA_ERR_ARG, "f expression: " + why);
  const auto t0 = std::chrono::steady_clock::now();
  fea_jit* j = new (std::nothrow) fea_jit();
  if (!j) return fail(FEA_ERR_NOMEM, "out of host memory");
  j->order = form->order;
  j->mass = form->kind == FEA_DIFFUSION_MASS && form->mass_coef != 0.0;
  j->mass_coef = j->mass ? form->mass_coef : 0.0;
  j->npts = q->npts;
  j->prec = q->prec;
  j->has_k = kappa_expr != nullptr;
  j->has_f = f_expr != nullptr;
  j->source = make_source(*j, kappa_expr, f_expr);
  {
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto it = cubin_cache().find(j->source);
    if (it != cubin_cache().end()) {
      j->cubin = it->second;
      j->cache_hit = true;
    }
  }
  if (!j->cache_hit) {
    const fea_status st = nvrtc_compile(j->source, j->cubin, j->log);
    if (st != FEA_OK) {
      delete j;
      return st;
    }
    std::lock_guard<std::mutex> lock(g_cache_mu);
    cubin_cache()[j->source] = j->cubin;
  }
  j->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = j;
  return FEA_OK;
}

fea_status fea_jit_info(const fea_jit* j, double* compile_ms, int64_t* cubin_bytes, int32_t* cache_hit) {
  if (!j) return fail(FEA_ERR_ARG, "NULL handle");
  if (compile_ms) *compile_ms = j->compile_ms;
  if (cubin_bytes) *cubin_bytes = (int64_t)j->cubin.size();
  if (cache_hit) *cache_hit = j->cache_hit ? 1 : 0;
  return FEA_OK;
}

const char* fea_jit_source(const fea_jit* j) { return j ? j->source.c_str() : ""; }
const char* fea_jit_log(const fea_jit* j) { return j ? j->log.c_str() : ""; }

fea_status fea_jit_assemble(fea_mesh* m, fea_jit* j, const fea_coeffs* co, double* values, double* rhs,
                            void* stream) {
  if (!m || !j || !co || !values) return fail(FEA_ERR_ARG, "NULL mesh, handle, coeffs or values");
  if (m->nvert != 4) return fail(FEA_ERR_ARG, "fea_jit_assemble takes tetrahedral meshes");
  if (rhs && !j->has_f) return fail(FEA_ERR_ARG, "rhs given but the kernel was compiled without an f expression");
  if (!rhs && j->has_f) return fail(FEA_ERR_ARG, "the kernel computes a load: pass rhs");
  if ((reinterpret_cast<uintptr_t>(values) & 7) || (reinterpret_cast<uintptr_t>(rhs) & 7))
    return fail(FEA_ERR_ARG, "misaligned output");
  Pattern* P = m->pat[j->order][1];
  Base* B = m->base[j->order];
  if (!P || !B) return fail(FEA_ERR_STATE, "fea_jit_assemble: build the pattern with fea_pattern(mesh, order, 1)");
  FEA_TRY(refuse_long_rows(B, "fea_jit_assemble"));
  FEA_TRY(ensure_loaded(j));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = B->nb;
  const bool mixed = j->prec == FEA_MIXED;
  const size_t rb = mixed ? sizeof(float) : sizeof(double);
  const int64_t E = m->n_elems;
  const bool tiled = use_tiled(m, P);
  const size_t npos = tiled ? (size_t)P->npos : (size_t)E * nb;
  FEA_TRY(ensure_scratch(m->lm, npos * lstride(nb, (int)rb) * rb));
  if (rhs) FEA_TRY(ensure_scratch(m->fl, npos * rb));
  UserArgs A{};
  A.x = m->x;
  A.y = m->y;
  A.z = m->z;
  A.tets = m->tets;
  A.E = E;
  A.N = m->n_nodes;
  A.kappa = co->kappa;
  A.kappa_const = co->kappa_const;
  A.mass = j->mass_coef;
  for (int k = 0; k < 4; ++k) A.p[k] = co->f_param[k];
  A.ipos = tiled ? P->tpos : B->ipos;
  A.Lm = m->lm.ptr;
  A.Fl = rhs ? m->fl.ptr : nullptr;
  A.err = m->err;
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[0], s));
  if (E > 0) {
    void* args[] = {&A};
    FEA_CUDA(cudaLaunchKernel(reinterpret_cast<const void*>(j->kern), dim3((unsigned)((E + USER_T - 1) / USER_T)),
                              dim3(USER_T), args, 0, s));
  }
  if (m->profile) FEA_CUDA(cudaEventRecord(m->ev[1], s));
  if (tiled) {
    FEA_TRY(scatter_tiled(m, P, B, mixed, A.Lm, A.Fl, values, rhs, s));
  } else {
    GatherArgs G{};
    G.ndof = P->ndof;
    G.row_ptr = P->row_ptr;
    G.inc_ptr = B->inc_ptr;
    G.slot = B->slot;
    G.Lm = A.Lm;
    G.Fl = A.Fl;
    G.values = values;
    G.rhs = rhs;
  G.err = m->err;
    FEA_TRY(launch_gather(nb, 1, mixed, G, P->rows_per_tile, P->max_tile_nnz, s));
  }
  if (m->profile) {
    FEA_CUDA(cudaEventRecord(m->ev[2], s));
    m->profiled = true;
  }
  return FEA_OK;
}

fea_status fea_jit_destroy(fea_jit* j) {
  if (!j) return FEA_OK;
  if (j->lib) cudaLibraryUnload(j->lib);
  delete j;
  return FEA_OK;
}

}  // extern "C"
