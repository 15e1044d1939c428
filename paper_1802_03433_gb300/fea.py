"""Thin Python binding of libfea (include/fea.h): argument marshalling only.

Every function here forwards torch tensors' device pointers and the current
CUDA stream to the C entry point of the same name; all assembly work runs in
the library's CUDA kernels.  There is no CPU fallback: if libfea.so is
missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# FEA_CHECKED=1 selects the bounds-checked build (build_lib.build(checked=True))
LIB_PATH = os.path.join(_HERE, "libfea_checked.so" if os.environ.get("FEA_CHECKED") == "1" else "libfea.so")

FEA_OK = 0
STATUS = {0: "FEA_OK", 1: "FEA_ERR_ARG", 2: "FEA_ERR_INDEX", 3: "FEA_ERR_DEGENERATE",
          4: "FEA_ERR_OVERFLOW", 5: "FEA_ERR_NOMEM", 6: "FEA_ERR_CUDA", 7: "FEA_ERR_TIMEOUT",
          8: "FEA_ERR_STATE"}
FEA_P1, FEA_P2 = 1, 2
FEA_POISSON, FEA_DIFFUSION_MASS, FEA_ELASTICITY = 0, 1, 2
FEA_FP64, FEA_MIXED = 0, 1
FEA_LOAD_NONE, FEA_LOAD_CONST, FEA_LOAD_SINPROD = 0, 1, 2
FEA_SCATTER_AUTO, FEA_SCATTER_LOCAL_ROWS, FEA_SCATTER_CHUNKED = 0, 1, 2


class FeaError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class fea_form(C.Structure):
    _fields_ = [("kind", C.c_int32), ("order", C.c_int32), ("mass_coef", C.c_double)]


class fea_coeffs(C.Structure):
    _fields_ = [("kappa", C.c_void_p), ("kappa_const", C.c_double),
                ("lame_lambda", C.c_void_p), ("lambda_const", C.c_double),
                ("lame_mu", C.c_void_p), ("mu_const", C.c_double),
                ("f_kind", C.c_int32), ("f_param", C.c_double * 4)]


class fea_quadrature(C.Structure):
    _fields_ = [("npts", C.c_int32), ("prec", C.c_int32)]


class fea_form2d(C.Structure):
    _fields_ = [("sigma0", C.c_double * 4), ("sigma_x", C.c_double * 4), ("sigma_y", C.c_double * 4),
                ("lambda_", C.c_double), ("f", C.c_double * 6), ("npts", C.c_int32)]


def make_form2d(sigma0=(1.0, 0.0, 0.0, 1.0), sigma_x=(0.0, -1.0, 1.0, 0.0), sigma_y=(0.0, -1.0, 1.0, 0.0),
                lam=1.0, f=(36.0, 0.0, 0.0, -2.0, 0.0, -2.0), npts=6):
    """Defaults: the paper's example (Sec. 4.2), sigma = [[1, -x-y], [x+y, 1]],
    lambda = 1, f = -2 (x^2 + y^2) + 36."""
    D4, D6 = C.c_double * 4, C.c_double * 6
    return fea_form2d(D4(*sigma0), D4(*sigma_x), D4(*sigma_y), lam, D6(*f), npts)


_lib = None
_vp = C.c_void_p


def lib() -> C.CDLL:
    """Load libfea.so (built by build_lib.build()); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FeaError(-1, "lib", f"{LIB_PATH} not built: run build_lib.build() (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    i64p = C.POINTER(C.c_int64)
    sig = {
        "fea_mesh_create": [_vp, _vp, _vp, C.c_int64, _vp, C.c_int64, _vp, C.POINTER(_vp)],
        "fea_mesh_set_coords": [_vp, _vp, _vp, _vp],
        "fea_mesh_create_tri": [_vp, _vp, C.c_int64, _vp, C.c_int64, _vp, C.POINTER(_vp)],
        "fea_assemble_2d": [_vp, C.POINTER(fea_form2d), _vp, _vp, _vp],
        "fea_mesh_destroy": [_vp],
        "fea_mesh_set_stages": [_vp, C.c_int32],
        "fea_mesh_set_scatter_classes": [_vp, C.c_int32],
        "fea_mesh_set_load_split": [_vp, C.c_int32],
        "fea_mesh_set_scatter_stages": [_vp, C.c_int32],
        "fea_mesh_set_scatter": [_vp, C.c_int32],
        "fea_mesh_check": [_vp, _vp],
        "fea_pattern": [_vp, C.c_int32, C.c_int32, i64p, i64p, _vp],
        "fea_pattern_copy": [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp],
        "fea_dof_table_copy": [_vp, C.c_int32, _vp, _vp],
        "fea_assemble": [_vp, C.POINTER(fea_form), C.POINTER(fea_coeffs), C.POINTER(fea_quadrature),
                         _vp, _vp, _vp],
        "fea_assemble_noalloc": [_vp, C.POINTER(fea_form), C.POINTER(fea_coeffs), C.POINTER(fea_quadrature),
                                 _vp, _vp, _vp],
        "fea_assemble_atomic": [_vp, C.POINTER(fea_form), C.POINTER(fea_coeffs), C.POINTER(fea_quadrature),
                                _vp, _vp, _vp],
        "fea_assemble_backward": [_vp, C.POINTER(fea_form), C.POINTER(fea_coeffs),
                                  C.POINTER(fea_quadrature), _vp, _vp, _vp, _vp, _vp],
        "fea_profile_enable": [_vp, C.c_int32],
        "fea_profile_last": [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float)],
        "fea_diag_sinpi": [_vp, C.c_int64, C.c_int32, _vp, _vp, _vp],
        "fea_diag_rcp": [_vp, C.c_int64, _vp, _vp, _vp],
        "fea_diag_wait_timeout": [_vp, C.c_int32, _vp],
        "fea_diag_checked_gather": [_vp, _vp, C.c_int64, C.c_int64, _vp, C.POINTER(C.c_int32), _vp],
        "fea_diag_fp64_rate": [C.POINTER(C.c_double), _vp],
        "fea_batch_create": [C.POINTER(_vp), C.c_int32, C.POINTER(fea_form), C.POINTER(fea_quadrature),
                             C.c_int32, _vp, C.POINTER(_vp)],
        "fea_batch_bind": [_vp, C.POINTER(fea_coeffs), C.POINTER(_vp), C.POINTER(_vp)],
        "fea_batch_assemble": [_vp, _vp],
        "fea_batch_tune": [_vp, _vp, C.POINTER(C.c_int32)],
        "fea_batch_destroy": [_vp],
        "fea_jit_compile": [C.POINTER(fea_form), C.POINTER(fea_quadrature), C.c_char_p, C.c_char_p,
                            C.POINTER(_vp)],
        "fea_jit_info": [_vp, C.POINTER(C.c_double), i64p, C.POINTER(C.c_int32)],
        "fea_jit_assemble": [_vp, _vp, C.POINTER(fea_coeffs), _vp, _vp, _vp],
        "fea_jit_destroy": [_vp],
        "fea_dirichlet": [_vp, C.c_int32, C.c_int32, _vp, C.c_int64, _vp, _vp, _vp, _vp],
        "fea_cg": [_vp, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                   C.POINTER(C.c_double), _vp],
        "fea_partition": [_vp, C.c_int64, C.c_int64, C.c_int32, C.c_int32, i64p, i64p, i64p, i64p, _vp, _vp, _vp],
        "fea_partition_batch": [_vp, C.c_int32, C.c_int32, _vp, _vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.fea_last_error.restype = C.c_char_p
    L.fea_last_error.argtypes = []
    for name in ("fea_jit_source", "fea_jit_log"):
        getattr(L, name).restype = C.c_char_p
        getattr(L, name).argtypes = [_vp]
    L.fea_status_string.restype = C.c_char_p
    L.fea_status_string.argtypes = [C.c_int]
    _lib = L
    return L


def _check(st: int, where: str):
    if st != FEA_OK:
        raise FeaError(st, where, lib().fea_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise FeaError(1, name, f"expected a contiguous CUDA {dtype} tensor")
    return t


# ---------------------------------------------------------------- same-name calls
def fea_mesh_create(x, y, z, tets, stream=None):
    """Handle (c_void_p) for coordinates x, y, z [N] float64 and tets [4, E] int32."""
    for t, n in ((x, "x"), (y, "y"), (z, "z")):
        _dev(t, torch.float64, n)
    _dev(tets, torch.int32, "tets")
    h = C.c_void_p()
    _check(lib().fea_mesh_create(_ptr(x), _ptr(y), _ptr(z), x.numel(), _ptr(tets), tets.shape[1],
                                 _stream(stream), C.byref(h)), "fea_mesh_create")
    return h


def fea_mesh_create_tri(x, y, tris, stream=None):
    """Handle of a 2-D triangle mesh: x, y [N] float64, tris [3, E] int32 (CUDA)."""
    for t, n in ((x, "x"), (y, "y")):
        _dev(t, torch.float64, n)
    _dev(tris, torch.int32, "tris")
    h = C.c_void_p()
    _check(lib().fea_mesh_create_tri(_ptr(x), _ptr(y), x.numel(), _ptr(tris), tris.shape[1], _stream(stream),
                                     C.byref(h)), "fea_mesh_create_tri")
    return h


def fea_assemble_2d(h, form2d, values, rhs=None, stream=None):
    _check(lib().fea_assemble_2d(h, C.byref(form2d), _ptr(values), _ptr(rhs), _stream(stream)), "fea_assemble_2d")


def fea_jit_compile(form, quad, kappa_expr=None, f_expr=None):
    """Compile (NVRTC, host side) the element kernel for the expressions;
    returns the handle."""
    out = C.c_void_p()
    enc = lambda e: None if e is None else e.encode()  # noqa: E731
    _check(lib().fea_jit_compile(C.byref(form), C.byref(quad), enc(kappa_expr), enc(f_expr), C.byref(out)),
           "fea_jit_compile")
    return out


def fea_jit_info(jh):
    """(compile_ms, cubin_bytes, cache_hit)."""
    ms, nb, hit = C.c_double(), C.c_int64(), C.c_int32()
    _check(lib().fea_jit_info(jh, C.byref(ms), C.byref(nb), C.byref(hit)), "fea_jit_info")
    return ms.value, nb.value, bool(hit.value)


def fea_jit_source(jh):
    return lib().fea_jit_source(jh).decode()


def fea_jit_log(jh):
    return lib().fea_jit_log(jh).decode()


def fea_jit_assemble(h, jh, coeffs, values, rhs=None, stream=None):
    _check(lib().fea_jit_assemble(h, jh, C.byref(coeffs), _ptr(values), _ptr(rhs), _stream(stream)),
           "fea_jit_assemble")


def fea_jit_destroy(jh):
    _check(lib().fea_jit_destroy(jh), "fea_jit_destroy")


def fea_dirichlet(h, order, dofs_per_node, dofs, g, values, rhs=None, stream=None):
    """Impose u = g at dofs (int32 CUDA tensor; g FP64 CUDA tensor or None)."""
    n = 0 if dofs is None else dofs.numel()
    _check(lib().fea_dirichlet(h, order, dofs_per_node, _ptr(dofs), n, _ptr(g), _ptr(values), _ptr(rhs),
                               _stream(stream)), "fea_dirichlet")


def fea_cg(h, order, dofs_per_node, values, b, x, rtol=1e-10, max_iter=10000, stream=None):
    """Jacobi-preconditioned CG in place on x; returns (iterations, ||r|| / ||b||)."""
    it, rr = C.c_int32(), C.c_double()
    _check(lib().fea_cg(h, order, dofs_per_node, _ptr(values), _ptr(b), _ptr(x), rtol, max_iter, C.byref(it),
                        C.byref(rr), _stream(stream)), "fea_cg")
    return it.value, rr.value


def fea_mesh_set_coords(h, x, y, z):
    _check(lib().fea_mesh_set_coords(h, _ptr(x), _ptr(y), _ptr(z)), "fea_mesh_set_coords")


def fea_mesh_set_stages(h, stages):
    _check(lib().fea_mesh_set_stages(h, stages), "fea_mesh_set_stages")


def fea_mesh_set_load_split(h, mode):
    _check(lib().fea_mesh_set_load_split(h, mode), "fea_mesh_set_load_split")


def fea_mesh_set_scatter_classes(h, mode):
    _check(lib().fea_mesh_set_scatter_classes(h, mode), "fea_mesh_set_scatter_classes")


def fea_mesh_set_scatter(h, mode):
    """FEA_SCATTER_AUTO, FEA_SCATTER_LOCAL_ROWS or FEA_SCATTER_CHUNKED (P1
    elasticity: fixed-point accumulation per chunk of elements)."""
    _check(lib().fea_mesh_set_scatter(h, mode), "fea_mesh_set_scatter")


def fea_mesh_set_scatter_stages(h, stages):
    _check(lib().fea_mesh_set_scatter_stages(h, stages), "fea_mesh_set_scatter_stages")


def fea_mesh_destroy(h):
    _check(lib().fea_mesh_destroy(h), "fea_mesh_destroy")


def fea_mesh_check(h, stream=None):
    _check(lib().fea_mesh_check(h, _stream(stream)), "fea_mesh_check")


def fea_pattern(h, order, dofs_per_node=1, stream=None):
    ndof, nnz = C.c_int64(), C.c_int64()
    _check(lib().fea_pattern(h, order, dofs_per_node, C.byref(ndof), C.byref(nnz), _stream(stream)),
           "fea_pattern")
    return ndof.value, nnz.value


def fea_pattern_copy(h, order, dofs_per_node, row_ptr, col_idx, stream=None):
    _check(lib().fea_pattern_copy(h, order, dofs_per_node, _ptr(row_ptr), _ptr(col_idx), _stream(stream)),
           "fea_pattern_copy")


def fea_dof_table_copy(h, order, edof, stream=None):
    _check(lib().fea_dof_table_copy(h, order, _ptr(edof), _stream(stream)), "fea_dof_table_copy")


def make_form(kind, order, mass_coef=0.0):
    return fea_form(kind, order, mass_coef)


def make_coeffs(kappa=None, kappa_const=1.0, lam=None, lam_const=1.0, mu=None, mu_const=1.0,
                f_kind=FEA_LOAD_NONE, f_param=(0.0, 0.0, 0.0, 0.0)):
    fp = (C.c_double * 4)(*(list(f_param) + [0.0] * 4)[:4])
    return fea_coeffs(_ptr(kappa), kappa_const, _ptr(lam), lam_const, _ptr(mu), mu_const, f_kind, fp)


def make_quadrature(npts=4, prec=FEA_FP64):
    return fea_quadrature(npts, prec)


def fea_assemble(h, form, coeffs, quad, values, rhs=None, stream=None):
    _check(lib().fea_assemble(h, C.byref(form), C.byref(coeffs), C.byref(quad), _ptr(values), _ptr(rhs),
                              _stream(stream)), "fea_assemble")


def fea_assemble_noalloc(h, form, coeffs, quad, values, rhs=None, stream=None):
    """fea_assemble with the scratch in the library's fixed device array (the
    call allocates nothing; meshes above the array's 32 MiB are rejected)."""
    _check(lib().fea_assemble_noalloc(h, C.byref(form), C.byref(coeffs), C.byref(quad), _ptr(values), _ptr(rhs),
                                      _stream(stream)), "fea_assemble_noalloc")


def fea_assemble_atomic(h, form, coeffs, quad, values, rhs=None, stream=None):
    """The paper's sparse Algorithm 1: global FP64 atomicAdd after a row search
    (not reproducible bit for bit; a comparison point)."""
    _check(lib().fea_assemble_atomic(h, C.byref(form), C.byref(coeffs), C.byref(quad), _ptr(values), _ptr(rhs),
                                     _stream(stream)), "fea_assemble_atomic")


def fea_assemble_backward(h, form, coeffs, quad, grad_values, grad_rhs, grad_kappa, grad_x, stream=None):
    _check(lib().fea_assemble_backward(h, C.byref(form), C.byref(coeffs), C.byref(quad), _ptr(grad_values),
                                       _ptr(grad_rhs), _ptr(grad_kappa), _ptr(grad_x), _stream(stream)),
           "fea_assemble_backward")


def fea_profile_enable(h, enable=True):
    _check(lib().fea_profile_enable(h, 1 if enable else 0), "fea_profile_enable")


def fea_profile_last(h):
    """(element-kernel ms, scatter-kernel ms) of the last profiled fea_assemble."""
    a, b = C.c_float(), C.c_float()
    _check(lib().fea_profile_last(h, C.byref(a), C.byref(b)), "fea_profile_last")
    return a.value, b.value


def fea_diag_wait_timeout(h, polls=1024, stream=None):
    _check(lib().fea_diag_wait_timeout(h, polls, _stream(stream)), "fea_diag_wait_timeout")


def fea_diag_checked_gather(h, src, n, idx, out, stream=None):
    """Read src[idx] into out[0] through the checked build's bounds check;
    returns True for the checked build (False: nothing was launched)."""
    chk = C.c_int32()
    _check(lib().fea_diag_checked_gather(h, _ptr(src), n, idx, _ptr(out), C.byref(chk), _stream(stream)),
           "fea_diag_checked_gather")
    return bool(chk.value)


def fea_diag_sinpi(x, variant=0, stream=None):
    """(helper sin(pi x), CUDA sinpi(x)) for a CUDA float64 tensor x; variant 0
    = the element kernels' fixed-point evaluation, 1 = the FP64 polynomial."""
    _dev(x, torch.float64, "x")
    mine, ref = torch.empty_like(x), torch.empty_like(x)
    _check(lib().fea_diag_sinpi(_ptr(x), x.numel(), variant, _ptr(mine), _ptr(ref), _stream(stream)),
           "fea_diag_sinpi")
    return mine, ref


def fea_diag_rcp(x, stream=None):
    """(helper 1 / x, CUDA's 1.0 / x) for a CUDA float64 tensor x."""
    _dev(x, torch.float64, "x")
    mine, ref = torch.empty_like(x), torch.empty_like(x)
    _check(lib().fea_diag_rcp(_ptr(x), x.numel(), _ptr(mine), _ptr(ref), _stream(stream)), "fea_diag_rcp")
    return mine, ref


def fea_diag_fp64_rate(stream=None):
    """Sustained FP64 FMA throughput of the current device (flop/s)."""
    r = C.c_double()
    _check(lib().fea_diag_fp64_rate(C.byref(r), _stream(stream)), "fea_diag_fp64_rate")
    return r.value


def fea_batch_create(meshes, forms, quads, f_kind, stream=None):
    n = len(meshes)
    hs = (_vp * n)(*[m.h.value if hasattr(m, "h") else m.value for m in meshes])
    fs = (fea_form * n)(*forms)
    qs = (fea_quadrature * n)(*quads)
    out = _vp()
    _check(lib().fea_batch_create(hs, n, fs, qs, f_kind, _stream(stream), C.byref(out)), "fea_batch_create")
    return out


def fea_batch_bind(b, coeffs, values, rhs=None):
    n = len(values)
    cs = (fea_coeffs * n)(*coeffs)
    vs = (_vp * n)(*[v.data_ptr() for v in values])
    rs = None if rhs is None else (_vp * n)(*[0 if r is None else r.data_ptr() for r in rhs])
    _check(lib().fea_batch_bind(b, cs, vs, rs), "fea_batch_bind")


def fea_batch_assemble(b, stream=None):
    _check(lib().fea_batch_assemble(b, _stream(stream)), "fea_batch_assemble")


def fea_batch_tune(b, stream=None):
    p = (C.c_int32 * 6)()
    _check(lib().fea_batch_tune(b, _stream(stream), p), "fea_batch_tune")
    return tuple(p)


def fea_batch_destroy(b):
    _check(lib().fea_batch_destroy(b), "fea_batch_destroy")


class Batch:
    """Many meshes assembled by one CUDA-graph launch (fea_batch_*).

    meshes: list of Mesh; forms/quads: per mesh; coeffs: per-mesh fea_coeffs.
    Owns the output tensors values[k], rhs[k]."""

    def __init__(self, meshes, forms, quads, coeffs, f_kind, with_rhs=True, stream=None):
        self.meshes = meshes
        self.h = fea_batch_create(meshes, forms, quads, f_kind, stream)
        self.values, self.rhs = [], []
        for m, f in zip(meshes, forms):
            ndof, nnz = m.pattern(f.order, 1)
            self.values.append(torch.empty(max(nnz, 1), dtype=torch.float64, device=m.x.device))
            self.rhs.append(torch.empty(ndof, dtype=torch.float64, device=m.x.device) if with_rhs else None)
        self.coeffs = coeffs
        fea_batch_bind(self.h, coeffs, self.values, self.rhs if with_rhs else None)

    def tune(self, stream=None):
        """Time the launch parameters on these meshes, keep the fastest and
        return them: (elements per item, P2 element CTAs, P1 element CTAs,
        scatter CTAs, P2 register variant, P1 register variant)."""
        return fea_batch_tune(self.h, stream)

    def assemble(self, stream=None):
        """Assemble every mesh into values[k] / rhs[k] with one graph launch
        (asynchronous on `stream`)."""
        fea_batch_assemble(self.h, stream)

    def close(self):
        if self.h is not None:
            fea_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fea_partition(tets, n_nodes, nparts, part):
    """Row partition of a P1 mesh (host arrays; no GPU needed): part `part` of
    `nparts` owns nodes [lo, hi) and takes every element with a vertex there.
    tets: int32 (4, E) numpy array.  Returns dict(lo, hi, elems, nodes,
    sub_tets) with numpy arrays: the global ids of the part's elements and
    nodes (ascending) and its connectivity in local node numbers."""
    import numpy as np
    t = np.ascontiguousarray(tets, dtype=np.int32)
    E = t.shape[1]
    lo, hi, ne, nn = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    tp = C.c_void_p(t.ctypes.data) if E else None
    _check(lib().fea_partition(tp, E, n_nodes, nparts, part, C.byref(lo), C.byref(hi), C.byref(ne), C.byref(nn),
                               None, None, None), "fea_partition")
    elems = np.empty(max(ne.value, 1), dtype=np.int32)
    nodes = np.empty(max(nn.value, 1), dtype=np.int32)
    sub = np.empty((4, max(ne.value, 1)), dtype=np.int32)
    _check(lib().fea_partition(tp, E, n_nodes, nparts, part, C.byref(lo), C.byref(hi), C.byref(ne), C.byref(nn),
                               C.c_void_p(elems.ctypes.data), C.c_void_p(nodes.ctypes.data),
                               C.c_void_p(sub.ctypes.data)), "fea_partition")
    return dict(lo=lo.value, hi=hi.value, elems=elems[:ne.value], nodes=nodes[:nn.value],
                sub_tets=np.ascontiguousarray(sub[:, :ne.value]))


def fea_partition_batch(cost, nparts):
    """Meshes of a batch over `nparts` GPUs by longest processing time first
    (host only): cost is one non-negative number per mesh.  Returns
    (part_of, load) numpy arrays: the part of each mesh and each part's
    total cost."""
    import numpy as np
    c = np.ascontiguousarray(cost, dtype=np.float64)
    part_of = np.empty(max(c.size, 1), dtype=np.int32)
    load = np.empty(nparts, dtype=np.float64) if nparts > 0 else np.empty(1, dtype=np.float64)
    _check(lib().fea_partition_batch(C.c_void_p(c.ctypes.data), c.size, nparts, C.c_void_p(part_of.ctypes.data),
                                     C.c_void_p(load.ctypes.data)), "fea_partition_batch")
    return part_of[:c.size], load[:max(nparts, 0)]


def owned_rows(part, row_ptr, col_idx, values, dofs_per_node=1):
    """The owned rows of a part's assembled sub-mesh in global numbering:
    (first global row, row lengths, global columns, values) as numpy arrays
    (row_ptr, col_idx, values of the sub-mesh's CSR, host or device)."""
    import numpy as np
    rp = np.asarray(row_ptr.cpu() if hasattr(row_ptr, "cpu") else row_ptr).astype(np.int64)
    ci = np.asarray(col_idx.cpu() if hasattr(col_idx, "cpu") else col_idx).astype(np.int64)
    v = np.asarray(values.cpu() if hasattr(values, "cpu") else values)
    nodes = part["nodes"].astype(np.int64)
    a = int(np.searchsorted(nodes, part["lo"]))
    b = int(np.searchsorted(nodes, part["hi"]))
    r0, r1 = dofs_per_node * a, dofs_per_node * b
    s0, s1 = int(rp[r0]), int(rp[r1])
    cols = dofs_per_node * nodes[ci[s0:s1] // dofs_per_node] + ci[s0:s1] % dofs_per_node
    return dofs_per_node * part["lo"], np.diff(rp[r0:r1 + 1]), cols, v[s0:s1]


def sub_positions(part, sub_row_ptr, sub_col_idx, row_ptr, col_idx, dofs_per_node=1):
    """Global CSR position of every entry of a part's sub-mesh pattern (int64
    numpy array, host logic): with it, a gradient with respect to the whole
    mesh's CSR values gives the sub-mesh's (grad_values[positions]), so the
    adjoint of a partitioned mesh runs part by part - each part's backward
    gives complete dL/dx for its owned nodes and dL/dkappa for all its
    elements, with no exchange."""
    import numpy as np

    def host(a):
        return np.asarray(a.cpu() if hasattr(a, "cpu") else a).astype(np.int64)
    srp, sci, rp, ci = host(sub_row_ptr), host(sub_col_idx), host(row_ptr), host(col_idx)
    d = dofs_per_node
    nodes = part["nodes"].astype(np.int64)
    rows = np.repeat(np.arange(srp.size - 1, dtype=np.int64), np.diff(srp))
    grow = d * nodes[rows // d] + rows % d
    gcol = d * nodes[sci[:srp[-1]] // d] + sci[:srp[-1]] % d
    nd = rp.size - 1
    gkeys = np.repeat(np.arange(nd, dtype=np.int64), np.diff(rp)) * nd + ci[:rp[-1]]
    pos = np.searchsorted(gkeys, grow * nd + gcol)
    if pos.size and (pos.max() >= gkeys.size or not np.array_equal(gkeys[pos], grow * nd + gcol)):
        raise ValueError("sub_positions: a sub-mesh entry is not in the global pattern")
    return pos


# ---------------------------------------------------------------- convenience wrapper
class Mesh:
    """Owns an fea_mesh handle plus the device tensors it references.
    coords (3, N) with tets (4, E), or coords (2, N) with triangles (3, E)."""

    def __init__(self, coords, tets, device="cuda", stream=None):
        c = torch.as_tensor(coords, dtype=torch.float64).to(device).contiguous()
        self.tets = torch.as_tensor(tets, dtype=torch.int32).to(device).contiguous()
        self.n_elems = self.tets.shape[1]
        if c.shape[0] == 2:
            self.x, self.y, self.z = c[0].contiguous(), c[1].contiguous(), None
            self.h = fea_mesh_create_tri(self.x, self.y, self.tets, stream)
        else:
            self.x, self.y, self.z = c[0].contiguous(), c[1].contiguous(), c[2].contiguous()
            self.h = fea_mesh_create(self.x, self.y, self.z, self.tets, stream)
        self.n_nodes = self.x.numel()
        self._pat = {}

    def set_coords(self, x, y, z):
        """Point the handle at new device coordinates (same node count); the
        pattern and scatter structures are kept."""
        self.x, self.y, self.z = x, y, z
        fea_mesh_set_coords(self.h, x, y, z)

    def pattern(self, order=1, dofs_per_node=1):
        """Build (once, cached) the CSR pattern of this order; returns
        (ndof, nnz)."""
        key = (order, dofs_per_node)
        if key not in self._pat:
            self._pat[key] = fea_pattern(self.h, order, dofs_per_node)
        return self._pat[key]

    def pattern_tensors(self, order=1, dofs_per_node=1):
        """(row_ptr, col_idx) of the pattern as int32 device tensors."""
        ndof, nnz = self.pattern(order, dofs_per_node)
        rp = torch.empty(ndof + 1, dtype=torch.int32, device=self.x.device)
        ci = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.x.device)
        fea_pattern_copy(self.h, order, dofs_per_node, rp, ci)
        return rp, ci[:nnz]

    def dof_table(self, order=1):
        """Element -> scalar dof table, int32 (nb, E) on the device (P2: the
        four vertex dofs, then the six edge dofs)."""
        self.pattern(order, 1)
        nb = self.tets.shape[0] if order == 1 else 10
        ed = torch.empty((nb, self.n_elems), dtype=torch.int32, device=self.x.device)
        if self.n_elems:
            fea_dof_table_copy(self.h, order, ed)
        return ed

    def assemble(self, form, coeffs, quad, values=None, rhs=None, with_rhs=True, stream=None):
        """Assemble the CSR values and the load vector of `form`; returns
        (values[:nnz], rhs) as FP64 device tensors (allocated unless given).
        Asynchronous on `stream`; device-side faults surface at check()."""
        ndpn = 3 if form.kind == FEA_ELASTICITY else 1
        ndof, nnz = self.pattern(form.order, ndpn)
        dev = self.x.device
        if values is None:
            values = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
        if rhs is None and with_rhs:
            rhs = torch.empty(ndof, dtype=torch.float64, device=dev)
        fea_assemble(self.h, form, coeffs, quad, values, rhs, stream)
        return values[:nnz], rhs

    def assemble_2d(self, form2d, values=None, rhs=None, with_rhs=True, stream=None):
        """The paper's 2-D form on a triangle mesh (make_form2d); returns
        (values[:nnz], rhs)."""
        ndof, nnz = self.pattern(1, 1)
        if values is None:
            values = torch.empty(max(nnz, 1), dtype=torch.float64, device=self.x.device)
        if rhs is None and with_rhs:
            rhs = torch.empty(ndof, dtype=torch.float64, device=self.x.device)
        fea_assemble_2d(self.h, form2d, values, rhs, stream)
        return values[:nnz], rhs

    def check(self, stream=None):
        """Synchronise and raise FeaError for a fault latched by earlier
        calls (bad index, det J <= 0, timeout)."""
        fea_mesh_check(self.h, stream)

    def close(self):
        if self.h is not None:
            fea_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
