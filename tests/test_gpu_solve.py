"""Dirichlet elimination and the CG solve on the GPU (fea_dirichlet,
fea_cg) against the oracle's elimination, a library direct solve of the
oracle's system, and the exact solution of the PDE."""
import math

import numpy as np
import pytest

import oracle
from common import row_scaled_error, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
sps = pytest.importorskip("scipy.sparse")
spla = pytest.importorskip("scipy.sparse.linalg")

AMP = 3 * math.pi ** 2


def _gpu_problem(n, order, kappa=False, g_fn=None, seed=0, npts=11):
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, rng = mg.make_cube(n, 0.2, seed)
    kap = mg.lognormal(rng, tets.shape[1]) if kappa else None
    m = fea.Mesh(coords, tets)
    ndof, nnz = m.pattern(order, 1)
    kt = None if kap is None else torch.as_tensor(kap, device="cuda")
    form = fea.make_form(fea.FEA_POISSON, order)
    co = fea.make_coeffs(kappa=kt, f_kind=fea.FEA_LOAD_SINPROD if g_fn is None else fea.FEA_LOAD_NONE,
                         f_param=(AMP,))
    vals, rhs = m.assemble(form, co, fea.make_quadrature(npts))
    if g_fn is not None:
        rhs.zero_()
    ed = m.dof_table(order).cpu().numpy()
    bd, pos = mg.cube_boundary_dofs(coords, ed, ndof)
    g = None if g_fn is None else torch.as_tensor(g_fn(*pos[:, bd]), device="cuda")
    fea.fea_dirichlet(m.h, order, 1, torch.as_tensor(bd, device="cuda"), g, vals, rhs)
    rp, ci = m.pattern_tensors(order, 1)
    return dict(m=m, coords=coords, tets=tets, kap=kap, vals=vals, rhs=rhs, rp=rp.cpu().numpy(),
                ci=ci.cpu().numpy(), bd=bd, pos=pos, ed=ed, ndof=ndof, keep=(kt, g))


@pytest.mark.parametrize("order", [1, 2])
def test_dirichlet_matches_oracle(order):
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, rng = mg.make_cube(5, 0.2, 3)
    m = fea.Mesh(coords, tets)
    ndof, _ = m.pattern(order, 1)
    rp, ci = (t.cpu().numpy() for t in m.pattern_tensors(order, 1))
    ed, _ = oracle.dof_table(order, coords.shape[1], tets)
    v, r, _ = oracle.assemble(coords, tets, order, ed, rp, ci, kappa=mg.lognormal(rng, tets.shape[1]), npts=11)
    bd, pos = mg.cube_boundary_dofs(coords, ed, ndof)
    g = np.cos(pos[0, bd]) + pos[1, bd] * pos[2, bd]
    # a shuffled list with repeats
    lst = np.concatenate([bd, bd[:7]])
    gl = np.concatenate([g, g[:7]])
    order_idx = np.random.default_rng(0).permutation(lst.size)
    lst, gl = lst[order_idx], gl[order_idx]
    vt = torch.as_tensor(v, device="cuda")
    rt = torch.as_tensor(r, device="cuda")
    fea.fea_dirichlet(m.h, order, 1, torch.as_tensor(lst.astype(np.int32), device="cuda"),
                      torch.as_tensor(gl, device="cuda"), vt, rt)
    torch.cuda.synchronize()
    m.check()
    ov, orr = oracle.dirichlet(rp, ci, v, r, bd, g)
    assert row_scaled_error(rp, ov, vt.cpu().numpy()) <= 1e-15
    assert vec_scaled_error(orr, rt.cpu().numpy()) <= 1e-14
    m.close()


def test_dirichlet_rejects_bad_ids():
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(2, 0.2, 0)
    m = fea.Mesh(coords, tets)
    ndof, nnz = m.pattern(1, 1)
    v = torch.ones(nnz, dtype=torch.float64, device="cuda")
    fea.fea_dirichlet(m.h, 1, 1, torch.tensor([0, ndof], dtype=torch.int32, device="cuda"), None, v, None)
    with pytest.raises(fea.FeaError, match="INDEX"):
        m.check()
    m.close()


@pytest.mark.parametrize("order,n,kappa", [(1, 8, False), (1, 10, True), (2, 5, True)])
def test_cg_matches_direct_solve(order, n, kappa):
    import torch
    from paper_1802_03433_gb300 import fea
    P = _gpu_problem(n, order, kappa=kappa)
    x = torch.zeros(P["ndof"], dtype=torch.float64, device="cuda")
    it, rel = fea.fea_cg(P["m"].h, order, 1, P["vals"], P["rhs"], x, rtol=1e-13, max_iter=5000)
    assert rel <= 1e-13 and 0 < it < 5000
    # reference: the oracle's own system, eliminated by the oracle, direct solve
    v, r, _ = oracle.assemble(P["coords"], P["tets"], order, P["ed"], P["rp"], P["ci"], kappa=P["kap"],
                              f_param=(AMP,), npts=11)
    v2, r2 = oracle.dirichlet(P["rp"], P["ci"], v, r, P["bd"])
    A = sps.csr_matrix((v2, P["ci"], P["rp"]), shape=(P["ndof"],) * 2)
    u = spla.spsolve(A.tocsc(), r2)
    assert vec_scaled_error(u, x.cpu().numpy()) <= 1e-10
    P["m"].close()


def test_manufactured_solution_p2():
    import torch
    from paper_1802_03433_gb300 import fea
    P = _gpu_problem(8, 2)
    x = torch.zeros(P["ndof"], dtype=torch.float64, device="cuda")
    fea.fea_cg(P["m"].h, 2, 1, P["vals"], P["rhs"], x, rtol=1e-12)
    pos = P["pos"]
    exact = np.sin(math.pi * pos[0]) * np.sin(math.pi * pos[1]) * np.sin(math.pi * pos[2])
    assert np.abs(x.cpu().numpy() - exact).max() < 2e-3
    P["m"].close()


def test_linear_field_with_boundary_data():
    import torch
    from paper_1802_03433_gb300 import fea
    gfn = lambda x, y, z: 1 + x + 2 * y - 3 * z  # noqa: E731
    P = _gpu_problem(6, 2, g_fn=gfn)
    x = torch.zeros(P["ndof"], dtype=torch.float64, device="cuda")
    fea.fea_cg(P["m"].h, 2, 1, P["vals"], P["rhs"], x, rtol=1e-14, max_iter=4000)
    np.testing.assert_allclose(x.cpu().numpy(), gfn(*P["pos"]), rtol=0, atol=1e-11)
    P["m"].close()


def test_cg_is_bitwise_reproducible_and_respects_max_iter():
    import torch
    from paper_1802_03433_gb300 import fea
    P = _gpu_problem(9, 1, kappa=True)
    xs = []
    for _ in range(2):
        x = torch.zeros(P["ndof"], dtype=torch.float64, device="cuda")
        fea.fea_cg(P["m"].h, 1, 1, P["vals"], P["rhs"], x, rtol=1e-12)
        xs.append(x)
    assert torch.equal(xs[0].view(torch.int64), xs[1].view(torch.int64))
    x = torch.zeros(P["ndof"], dtype=torch.float64, device="cuda")
    it, rel = fea.fea_cg(P["m"].h, 1, 1, P["vals"], P["rhs"], x, rtol=1e-14, max_iter=5)
    assert it == 5 and rel > 1e-6
    it0, _ = fea.fea_cg(P["m"].h, 1, 1, P["vals"], P["rhs"], xs[0], rtol=1e-6)
    assert it0 == 0  # already converged from that initial guess
    P["m"].close()


def test_cg_reports_an_indefinite_matrix():
    import torch
    from paper_1802_03433_gb300 import fea
    P = _gpu_problem(4, 1)
    neg = -P["vals"]
    x = torch.zeros(P["ndof"], dtype=torch.float64, device="cuda")
    with pytest.raises(fea.FeaError, match="positive definite"):
        fea.fea_cg(P["m"].h, 1, 1, neg, P["rhs"], x, rtol=1e-10)
    P["m"].close()
