"""Runtime-compiled element kernels (fea_jit_compile / fea_jit_assemble)
against the oracle's user-coefficient form: k(x) inside the stiffness
integral and f(x) as the load, given to the GPU as CUDA C++ expressions and
to the oracle as Python point functions with the same mathematics."""
import math

import numpy as np
import pytest

import oracle
from common import TOL_FP64, TOL_MIXED, row_scaled_error, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

P = (3 * math.pi ** 2, 0.5, -0.25, 2.0)  # p0..p3
CASES = {
    # name: (CUDA expression, Python function of (x, y, z))
    "smooth_k": ("1 + 0.5*sin(3*x)*cos(2*y) + z*z",
                 lambda x, y, z: 1 + 0.5 * math.sin(3 * x) * math.cos(2 * y) + z * z),
    "param_k": ("p3 + x*y - p2*z", lambda x, y, z: P[3] + x * y - P[2] * z),
    "sin_f": ("p0*sinpi_fp64(x)*sinpi_fp64(y)*sinpi_fp64(z)",
              lambda x, y, z: P[0] * math.sin(math.pi * x) * math.sin(math.pi * y) * math.sin(math.pi * z)),
    "exp_f": ("exp(-x)*(1 + y*z) + p1", lambda x, y, z: math.exp(-x) * (1 + y * z) + P[1]),
    "sinx_f": ("p0*sinpi_fx(x)*sinpi_fx(y)*sinpi_fx(z)",
               lambda x, y, z: P[0] * math.sin(math.pi * x) * math.sin(math.pi * y) * math.sin(math.pi * z)),
}


def _run(order, n, npts, prec, k, f, mass, seed=0, kappa_per_elem=True):
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, rng = mg.make_cube(n, 0.2, seed)
    E = tets.shape[1]
    kap = mg.lognormal(rng, E) if kappa_per_elem else None
    m = fea.Mesh(coords, tets)
    ndof, nnz = m.pattern(order, 1)
    kind = fea.FEA_DIFFUSION_MASS if mass else fea.FEA_POISSON
    j = fea.fea_jit_compile(fea.make_form(kind, order, mass), fea.make_quadrature(npts, prec),
                            None if k is None else CASES[k][0], None if f is None else CASES[f][0])
    kt = None if kap is None else torch.as_tensor(kap, device="cuda")
    co = fea.make_coeffs(kappa=kt, kappa_const=1.0, f_param=P)
    vals = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
    rhs = torch.empty(ndof, dtype=torch.float64, device="cuda") if f else None
    fea.fea_jit_assemble(m.h, j, co, vals, rhs)
    torch.cuda.synchronize()
    m.check()
    rp, ci = m.pattern_tensors(order, 1)
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    edof, _ = oracle.dof_table(order, coords.shape[1], tets)
    ov, orr, bad = oracle.assemble_user(coords, tets, order, edof, rp, ci, kfn=None if k is None else CASES[k][1],
                                        ffn=None if f is None else CASES[f][1], kappa=kap, mass=mass, npts=npts)
    assert bad == 0
    got_r = rhs.cpu().numpy() if f else None
    fea.fea_jit_destroy(j)
    m.close()
    return rp, vals[:nnz].cpu().numpy(), ov, got_r, orr


@pytest.mark.parametrize("order,npts,mass", [(1, 1, 0.0), (1, 4, 0.0), (1, 11, 1.0), (2, 4, 0.0), (2, 11, 1.0)])
@pytest.mark.parametrize("k,f", [("smooth_k", "sin_f"), ("param_k", "exp_f"), (None, "exp_f"), ("smooth_k", None),
                                 (None, "sinx_f")])
def test_fp64_matches_oracle(order, npts, mass, k, f):
    rp, v, ov, r, orr = _run(order, 6, npts, 0, k, f, mass)
    assert row_scaled_error(rp, ov, v) <= TOL_FP64
    if f:
        assert vec_scaled_error(orr, r) <= TOL_FP64


@pytest.mark.parametrize("order,npts", [(1, 4), (2, 11)])
def test_mixed_matches_oracle(order, npts):
    rp, v, ov, r, orr = _run(order, 6, npts, 1, "smooth_k", "sin_f", 1.0)
    assert row_scaled_error(rp, ov, v) <= TOL_MIXED
    assert vec_scaled_error(orr, r) <= TOL_MIXED


def test_several_tiles_and_a_ragged_tail():
    # 14^3 cubes: 16,464 tets (129 element CTAs, the last one partial), P2
    rp, v, ov, r, orr = _run(2, 14, 11, 0, "smooth_k", "exp_f", 1.0, seed=3)
    assert row_scaled_error(rp, ov, v) <= TOL_FP64
    assert vec_scaled_error(orr, r) <= TOL_FP64


def test_constant_kappa_constant_expression_and_builtin_path_agree():
    """k = "1" (quadrature of a constant, 11 points, exact) vs no k (exact
    moments) vs the precompiled kernel (closed form): the same matrix up to
    rounding; the sin load through sinpi_fp64 vs the precompiled sin load."""
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, rng = mg.make_cube(8, 0.2, 11)
    kap = torch.as_tensor(mg.lognormal(rng, tets.shape[1]), device="cuda")
    m = fea.Mesh(coords, tets)
    ndof, nnz = m.pattern(2, 1)
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0)
    q = fea.make_quadrature(11)
    co = fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=P)
    base_v, base_r = m.assemble(form, co, q)
    rp = m.pattern_tensors(2, 1)[0].cpu().numpy()
    outs = []
    for kexpr in ("1", None):
        j = fea.fea_jit_compile(form, q, kexpr, CASES["sin_f"][0])
        v = torch.empty(nnz, dtype=torch.float64, device="cuda")
        r = torch.empty(ndof, dtype=torch.float64, device="cuda")
        fea.fea_jit_assemble(m.h, j, co, v, r)
        outs.append((v.cpu().numpy(), r.cpu().numpy()))
        fea.fea_jit_destroy(j)
    torch.cuda.synchronize()
    bv, br = base_v.cpu().numpy(), base_r.cpu().numpy()
    for v, r in outs:
        assert row_scaled_error(rp, bv, v) <= 1e-13
        assert vec_scaled_error(br, r) <= 1e-14
    m.close()


def test_deterministic_and_symmetric():
    import torch
    from paper_1802_03433_gb300 import fea
    import scipy.sparse as sps
    coords, tets, _ = mg.make_cube(7, 0.2, 2)
    m = fea.Mesh(coords, tets)
    ndof, nnz = m.pattern(2, 1)
    j = fea.fea_jit_compile(fea.make_form(fea.FEA_POISSON, 2), fea.make_quadrature(11), CASES["smooth_k"][0], None)
    co = fea.make_coeffs()
    runs = []
    for _ in range(2):
        v = torch.empty(nnz, dtype=torch.float64, device="cuda")
        fea.fea_jit_assemble(m.h, j, co, v, None)
        runs.append(v)
    torch.cuda.synchronize()
    assert torch.equal(runs[0].view(torch.int64), runs[1].view(torch.int64))
    rp, ci = (t.cpu().numpy() for t in m.pattern_tensors(2, 1))
    A = sps.csr_matrix((runs[0].cpu().numpy(), ci, rp), shape=(ndof, ndof))
    assert (A != A.T).nnz == 0
    fea.fea_jit_destroy(j)
    m.close()


def test_argument_errors():
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(2, 0.2, 0)
    m = fea.Mesh(coords, tets)
    j = fea.fea_jit_compile(fea.make_form(fea.FEA_POISSON, 2), fea.make_quadrature(4), "1+x", "x")
    co = fea.make_coeffs()
    v = torch.empty(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(fea.FeaError, match="pattern"):
        fea.fea_jit_assemble(m.h, j, co, v, torch.empty(100, dtype=torch.float64, device="cuda"))
    m.pattern(2, 1)
    with pytest.raises(fea.FeaError, match="pass rhs"):
        fea.fea_jit_assemble(m.h, j, co, v, None)
    fea.fea_jit_destroy(j)
    m.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_scatter_modes_bitwise_identical(prec):
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(9, 0.2, 8)
    m = fea.Mesh(coords, tets)
    ndof, nnz = m.pattern(2, 1)
    j = fea.fea_jit_compile(fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0), fea.make_quadrature(11, prec),
                            CASES["smooth_k"][0], CASES["exp_f"][0])
    co = fea.make_coeffs(f_param=P)
    outs = []
    for mode in (2, 3):
        fea.fea_mesh_set_scatter_classes(m.h, mode)
        v = torch.empty(nnz, dtype=torch.float64, device="cuda")
        r = torch.empty(ndof, dtype=torch.float64, device="cuda")
        fea.fea_jit_assemble(m.h, j, co, v, r)
        torch.cuda.synchronize()
        outs.append((v.cpu().numpy().view(np.uint64), r.cpu().numpy().view(np.uint64)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    fea.fea_jit_destroy(j)
    m.close()
