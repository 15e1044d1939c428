"""CPU oracle for finite element assembly (test infrastructure only).

Plain FP64 C++ (oracle.cpp) behind ctypes.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg use it; the product package never
imports it.  See oracle.cpp for what each routine computes and which passage
of the paper (Sec. 4.1 Eq. 1-3, Sec. 5 Algorithm 1) it follows.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _lib.orc_rule.restype = C.c_int
        _lib.orc_p2_dofs.restype = C.c_int64
        _lib.orc_pattern.restype = C.c_int64
        _lib.orc_assemble.restype = C.c_int64
        _lib.orc_rows.restype = C.c_int64
        _lib.orc_assemble_grad.restype = C.c_int64
        _lib.orc_tri_rule.restype = C.c_int
        _lib.orc_assemble_tri.restype = C.c_int64
        _lib.orc_assemble_user.restype = C.c_int64
        _lib.orc_free.argtypes = [C.c_void_p]
        _lib.orc_assemble_par.restype = C.c_int64
    return _lib


def _d(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(_dp)


def _keep(*arrs):
    return [None if a is None else np.ascontiguousarray(a) for a in arrs]


def rule(npts: int):
    """Quadrature rule: (bary (npts, 4), weights summing to 1)."""
    b = np.zeros((11, 4))
    w = np.zeros(11)
    n = lib().orc_rule(npts, b.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    if n == 0:
        raise ValueError(f"no {npts}-point rule")
    return b[:n].copy(), w[:n].copy()


def p2_dofs(n_nodes: int, tets: np.ndarray):
    """(edof int32 (10, E), n_edges)."""
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    E = tets.shape[1]
    edof = np.empty((10, E), dtype=np.int32)
    ne = lib().orc_p2_dofs(C.c_int64(n_nodes), C.c_int64(E), tets.ctypes.data_as(_ip),
                           edof.ctypes.data_as(_ip))
    return edof, int(ne)


def dof_table(order: int, n_nodes: int, tets: np.ndarray):
    """(edof (nb, E), n_scalar_dofs)."""
    if order == 1:
        return np.ascontiguousarray(tets, dtype=np.int32), n_nodes
    edof, ne = p2_dofs(n_nodes, tets)
    return edof, n_nodes + ne


def pattern(ndof_scalar: int, edof: np.ndarray, ndpn: int = 1):
    """CSR pattern (row_ptr int32, col_idx int32) of the assembled matrix."""
    edof = np.ascontiguousarray(edof, dtype=np.int32)
    nb, E = edof.shape
    rp = C.POINTER(C.c_int32)()
    ci = C.POINTER(C.c_int32)()
    nnz = lib().orc_pattern(C.c_int64(ndof_scalar), C.c_int64(E), C.c_int(nb),
                            edof.ctypes.data_as(_ip), C.c_int(ndpn), C.byref(rp), C.byref(ci))
    ndof = ndof_scalar * ndpn
    row_ptr = np.ctypeslib.as_array(rp, shape=(ndof + 1,)).copy()
    col_idx = np.ctypeslib.as_array(ci, shape=(max(nnz, 1),))[:nnz].copy()
    lib().orc_free(C.cast(rp, C.c_void_p))
    lib().orc_free(C.cast(ci, C.c_void_p))
    return row_ptr, col_idx


KIND = {"diffusion": 0, "elasticity": 1}
FKIND = {None: 0, "zero": 0, "const": 1, "sinprod": 2}


def _fparam(f_param):
    fp = np.zeros(4)
    if f_param is not None:
        f_param = np.atleast_1d(np.asarray(f_param, dtype=np.float64))
        fp[: f_param.size] = f_param
    return fp


def assemble(coords, tets, order, edof, row_ptr, col_idx, kind="diffusion", mass=0.0,
             kappa=None, kappa_const=1.0, lam=None, lam_const=1.0, mu=None, mu_const=1.0,
             f_kind="sinprod", f_param=(3 * np.pi ** 2,), npts=4):
    """Assembled CSR values and load vector (the definition of Eq. 3)."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    edof = np.ascontiguousarray(edof, dtype=np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    kappa, lam, mu = _keep(kappa, lam, mu)
    ndof = row_ptr.size - 1
    values = np.empty(int(row_ptr[-1]))
    rhs = np.empty(ndof)
    fp = _fparam(f_param)
    bad = lib().orc_assemble(
        C.c_int64(coords.shape[1]), _d(coords[0]), _d(coords[1]), _d(coords[2]),
        C.c_int64(tets.shape[1]), tets.ctypes.data_as(_ip), C.c_int(order),
        edof.ctypes.data_as(_ip), C.c_int(KIND[kind]), C.c_double(mass),
        _d(kappa), C.c_double(kappa_const), _d(lam), C.c_double(lam_const), _d(mu),
        C.c_double(mu_const), C.c_int(FKIND[f_kind]), fp.ctypes.data_as(_dp), C.c_int(npts),
        C.c_int64(ndof), row_ptr.ctypes.data_as(_ip), col_idx.ctypes.data_as(_ip),
        values.ctypes.data_as(_dp), rhs.ctypes.data_as(_dp))
    if bad < 0:
        raise RuntimeError("local entry without a slot in the pattern")
    return values, rhs, int(bad)


def assemble_par(coords, tets, order, edof, row_ptr, col_idx, kind="diffusion", mass=0.0,
                 kappa=None, kappa_const=1.0, lam=None, lam_const=1.0, mu=None, mu_const=1.0,
                 f_kind="sinprod", f_param=(3 * np.pi ** 2,), npts=4, threads=0):
    """Timing baseline, not a checker: assemble() with the elements split over
    OpenMP threads (per-thread copies of the outputs, summed at the end).
    Returns (values, rhs, bad, threads used)."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    edof = np.ascontiguousarray(edof, dtype=np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    kappa, lam, mu = _keep(kappa, lam, mu)
    ndof = row_ptr.size - 1
    values = np.empty(int(row_ptr[-1]))
    rhs = np.empty(ndof)
    fp = _fparam(f_param)
    used = C.c_int(0)
    bad = lib().orc_assemble_par(
        _d(coords[0]), _d(coords[1]), _d(coords[2]), C.c_int64(tets.shape[1]), tets.ctypes.data_as(_ip),
        C.c_int(order), edof.ctypes.data_as(_ip), C.c_int(KIND[kind]), C.c_double(mass), _d(kappa),
        C.c_double(kappa_const), _d(lam), C.c_double(lam_const), _d(mu), C.c_double(mu_const),
        C.c_int(FKIND[f_kind]), fp.ctypes.data_as(_dp), C.c_int(npts), C.c_int64(ndof),
        row_ptr.ctypes.data_as(_ip), col_idx.ctypes.data_as(_ip), values.ctypes.data_as(_dp),
        rhs.ctypes.data_as(_dp), C.c_int(threads), C.byref(used))
    if bad < 0:
        raise RuntimeError("local entry without a slot in the pattern")
    return values, rhs, int(bad), used.value


def local(X, order=1, kind="diffusion", mass=0.0, kappa=None, lam=None, mu=None,
          f_kind="zero", f_param=None, npts=4):
    """Local matrices (n, nl, nl), load vectors (n, nl), det J (n) for vertex
    coordinates X of shape (n, 4, 3)."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 4, 3)
    n = X.shape[0]
    nl = (4 if order == 1 else 10) * (3 if kind == "elasticity" else 1)
    Ke = np.empty((n, nl, nl))
    Fe = np.empty((n, nl))
    det = np.empty(n)
    kappa, lam, mu = _keep(kappa, lam, mu)
    fp = _fparam(f_param)
    lib().orc_local(X.ctypes.data_as(_dp), C.c_int64(n), C.c_int(order), C.c_int(KIND[kind]),
                    C.c_double(mass), _d(kappa), _d(lam), _d(mu), C.c_int(FKIND[f_kind]),
                    fp.ctypes.data_as(_dp), C.c_int(npts), Ke.ctypes.data_as(_dp),
                    Fe.ctypes.data_as(_dp), det.ctypes.data_as(_dp))
    return Ke, Fe, det


def rows_arrays(coords, tets, order, edof, rows_, kind="diffusion", mass=0.0, kappa=None,
                kappa_const=1.0, lam=None, lam_const=1.0, mu=None, mu_const=1.0, f_kind="sinprod",
                f_param=(3 * np.pi ** 2,), npts=4):
    """Selected assembled rows by brute force (no pattern needed), as flat
    arrays: (rows int64, cols int64, vals) sorted by (row, col), the rows
    asked for (ascending, unique), and their load entries."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    edof = np.ascontiguousarray(edof, dtype=np.int32)
    rr = np.unique(np.asarray(rows_, dtype=np.int64))
    kappa, lam, mu = _keep(kappa, lam, mu)
    fp = _fparam(f_param)
    R = C.POINTER(C.c_int64)()
    Cc = C.POINTER(C.c_int64)()
    V = C.POINTER(C.c_double)()
    rhs = np.empty(rr.size)
    n = lib().orc_rows(
        _d(coords[0]), _d(coords[1]), _d(coords[2]), C.c_int64(tets.shape[1]),
        tets.ctypes.data_as(_ip), C.c_int(order), edof.ctypes.data_as(_ip), C.c_int(KIND[kind]),
        C.c_double(mass), _d(kappa), C.c_double(kappa_const), _d(lam), C.c_double(lam_const),
        _d(mu), C.c_double(mu_const), C.c_int(FKIND[f_kind]), fp.ctypes.data_as(_dp),
        C.c_int(npts), rr.ctypes.data_as(_lp), C.c_int64(rr.size), C.byref(R), C.byref(Cc),
        C.byref(V), rhs.ctypes.data_as(_dp))
    r = np.ctypeslib.as_array(R, shape=(max(n, 1),))[:n].copy()
    c = np.ctypeslib.as_array(Cc, shape=(max(n, 1),))[:n].copy()
    v = np.ctypeslib.as_array(V, shape=(max(n, 1),))[:n].copy()
    for p in (R, Cc, V):
        lib().orc_free(C.cast(p, C.c_void_p))
    return r, c, v, rr, rhs


def rows(coords, tets, order, edof, rows_, **kw):
    """Selected assembled rows by brute force (no pattern needed).

    Returns dict row -> (cols int64 ascending, vals), and rhs per row."""
    r, c, v, rr, rhs = rows_arrays(coords, tets, order, edof, rows_, **kw)
    lo = np.searchsorted(r, rr, side="left")
    hi = np.searchsorted(r, rr, side="right")
    out = {int(row): (c[a:b], v[a:b]) for row, a, b in zip(rr, lo, hi)}
    return out, dict(zip(rr.tolist(), rhs.tolist()))


def assemble_grad(coords, tets, order, edof, row_ptr, col_idx, grad_values, grad_rhs,
                  mass=0.0, kappa=None, kappa_const=1.0, f_kind="sinprod",
                  f_param=(3 * np.pi ** 2,), npts=4):
    """(dL/dkappa per element, dL/dx (3, N)) for L = <grad_values, values> +
    <grad_rhs, rhs>, by forward-mode dual numbers through the element routine."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    edof = np.ascontiguousarray(edof, dtype=np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    kappa, grad_values, grad_rhs = _keep(kappa, grad_values, grad_rhs)
    N = coords.shape[1]
    E = tets.shape[1]
    gk = np.empty(E)
    gx = np.empty((3, N))
    fp = _fparam(f_param)
    rc = lib().orc_assemble_grad(
        C.c_int64(N), _d(coords[0]), _d(coords[1]), _d(coords[2]), C.c_int64(E),
        tets.ctypes.data_as(_ip), C.c_int(order), edof.ctypes.data_as(_ip), C.c_double(mass),
        _d(kappa), C.c_double(kappa_const), C.c_int(FKIND[f_kind]), fp.ctypes.data_as(_dp),
        C.c_int(npts), C.c_int64(row_ptr.size - 1), row_ptr.ctypes.data_as(_ip),
        col_idx.ctypes.data_as(_ip), _d(grad_values), _d(grad_rhs), gk.ctypes.data_as(_dp),
        gx.ctypes.data_as(_dp))
    if rc < 0:
        raise RuntimeError("local entry without a slot in the pattern")
    return gk, gx


# ---------------------------------------------------------------- 2-D triangles
PAPER_2D = dict(S0=(1.0, 0.0, 0.0, 1.0), Sx=(0.0, -1.0, 1.0, 0.0), Sy=(0.0, -1.0, 1.0, 0.0), lam=1.0,
                f=(36.0, 0.0, 0.0, -2.0, 0.0, -2.0))
"""The paper's example (Sec. 4.2): sigma = [[1, -x-y], [x+y, 1]], lambda = 1,
f = -2 (x^2 + y^2) + 36."""


def _v(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(n))
    return a


def tri_rule(npts: int):
    b = np.zeros((6, 3))
    w = np.zeros(6)
    n = lib().orc_tri_rule(npts, b.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    if n == 0:
        raise ValueError(f"no {npts}-point triangle rule")
    return b[:n].copy(), w[:n].copy()


def local_tri(X, S0=PAPER_2D["S0"], Sx=PAPER_2D["Sx"], Sy=PAPER_2D["Sy"], lam=PAPER_2D["lam"],
              f=PAPER_2D["f"], npts=6):
    """Local 3x3 matrices (row = test function), loads and det J of triangles X (n, 3, 2)."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3, 2)
    n = X.shape[0]
    Ke, Fe, det = np.empty((n, 3, 3)), np.empty((n, 3)), np.empty(n)
    keep = [_v(S0, 4), _v(Sx, 4), _v(Sy, 4), _v(f, 6)]
    lib().orc_local_tri(X.ctypes.data_as(_dp), C.c_int64(n), keep[0].ctypes.data_as(_dp),
                        keep[1].ctypes.data_as(_dp), keep[2].ctypes.data_as(_dp), C.c_double(lam),
                        keep[3].ctypes.data_as(_dp), C.c_int(npts), Ke.ctypes.data_as(_dp),
                        Fe.ctypes.data_as(_dp), det.ctypes.data_as(_dp))
    return Ke, Fe, det


def assemble_tri(coords2, tris, row_ptr, col_idx, S0=PAPER_2D["S0"], Sx=PAPER_2D["Sx"], Sy=PAPER_2D["Sy"],
                 lam=PAPER_2D["lam"], f=PAPER_2D["f"], npts=6):
    """Assembled CSR values and load of the 2-D P1 problem (coords2: (2, N))."""
    coords2 = np.ascontiguousarray(coords2, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    N = coords2.shape[1]
    values, rhs = np.empty(int(row_ptr[-1])), np.empty(N)
    keep = [_v(S0, 4), _v(Sx, 4), _v(Sy, 4), _v(f, 6)]
    bad = lib().orc_assemble_tri(
        C.c_int64(N), _d(coords2[0]), _d(coords2[1]), C.c_int64(tris.shape[1]), tris.ctypes.data_as(_ip),
        keep[0].ctypes.data_as(_dp), keep[1].ctypes.data_as(_dp), keep[2].ctypes.data_as(_dp), C.c_double(lam),
        keep[3].ctypes.data_as(_dp), C.c_int(npts), row_ptr.ctypes.data_as(_ip), col_idx.ctypes.data_as(_ip),
        values.ctypes.data_as(_dp), rhs.ctypes.data_as(_dp))
    if bad < 0:
        raise RuntimeError("local entry without a slot in the pattern")
    return values, rhs, int(bad)


# ---------------------------------------------------------------- user coefficients
POINT_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_double, C.c_double)


def _point_fn(fn):
    if fn is None:
        return None, C.cast(None, POINT_FN)
    cb = POINT_FN(lambda x, y, z: float(fn(x, y, z)))
    return cb, cb


def assemble_user(coords, tets, order, edof, row_ptr, col_idx, kfn=None, ffn=None, kappa=None,
                  kappa_const=1.0, mass=0.0, npts=11):
    """CSR values and load of -div(kappa_T k(x) grad u) + mass u = f(x) with
    Python point functions k(x, y, z) and f(x, y, z) (None: k = 1, f = 0);
    stiffness and load by the npts rule (stiffness by the exact 11-point rule
    when k is None), mass exact."""
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    edof = np.ascontiguousarray(edof, dtype=np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    (kappa,) = _keep(kappa)
    ndof = row_ptr.size - 1
    values, rhs = np.empty(int(row_ptr[-1])), np.empty(ndof)
    kkeep, kcb = _point_fn(kfn)
    fkeep, fcb = _point_fn(ffn)
    bad = lib().orc_assemble_user(
        C.c_int64(coords.shape[1]), _d(coords[0]), _d(coords[1]), _d(coords[2]), C.c_int64(tets.shape[1]),
        tets.ctypes.data_as(_ip), C.c_int(order), edof.ctypes.data_as(_ip), C.c_double(mass), _d(kappa),
        C.c_double(kappa_const), kcb, fcb, C.c_int(npts), C.c_int64(ndof), row_ptr.ctypes.data_as(_ip),
        col_idx.ctypes.data_as(_ip), values.ctypes.data_as(_dp), rhs.ctypes.data_as(_dp))
    del kkeep, fkeep
    if bad < 0:
        raise RuntimeError("local entry without a slot in the pattern")
    return values, rhs, int(bad)


def local_user(X, order=1, mass=0.0, kfn=None, ffn=None, npts=11):
    """Local matrices (n, nb, nb) and loads (n, nb) of the user-coefficient form, kappa_T = 1."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 4, 3)
    n = X.shape[0]
    nb = 4 if order == 1 else 10
    Ke, Fe = np.empty((n, nb, nb)), np.empty((n, nb))
    kkeep, kcb = _point_fn(kfn)
    fkeep, fcb = _point_fn(ffn)
    lib().orc_local_user(X.ctypes.data_as(_dp), C.c_int64(n), C.c_int(order), C.c_double(mass), kcb, fcb,
                         C.c_int(npts), Ke.ctypes.data_as(_dp), Fe.ctypes.data_as(_dp))
    del kkeep, fkeep
    return Ke, Fe


# ---------------------------------------------------------------- Dirichlet conditions
def dirichlet(row_ptr, col_idx, values, rhs, dofs, g=None):
    """Copies of (values, rhs) with u = g imposed at dofs by symmetric elimination."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    v = np.array(values, dtype=np.float64, copy=True)
    r = np.array(rhs, dtype=np.float64, copy=True)
    dofs = np.ascontiguousarray(dofs, dtype=np.int32)
    (g,) = _keep(None if g is None else np.asarray(g, dtype=np.float64))
    lib().orc_dirichlet(C.c_int64(row_ptr.size - 1), row_ptr.ctypes.data_as(_ip), col_idx.ctypes.data_as(_ip),
                        v.ctypes.data_as(_dp), r.ctypes.data_as(_dp), C.c_int64(dofs.size),
                        dofs.ctypes.data_as(_ip), _d(g))
    return v, r
