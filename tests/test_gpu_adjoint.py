"""The hand-written adjoint (fea_assemble_backward, FeaAssemble) against the
oracle's dual-number gradient and against central differences (GPU)."""
import numpy as np
import pytest

import oracle
from common import case, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-12


def _loss_weights(nd, rp, ci, seed):
    rng = np.random.default_rng(seed)
    v, w, g = rng.standard_normal(nd), rng.standard_normal(nd), rng.standard_normal(nd)
    rows = np.repeat(np.arange(nd), np.diff(rp))
    return v, w, g, v[rows] * w[ci]


def _gpu_backward(m, c, gV, g, kappa):
    import torch
    from paper_1802_03433_gb300 import fea
    dev = "cuda"
    kind = fea.FEA_DIFFUSION_MASS if c["mass"] else fea.FEA_POISSON
    form = fea.make_form(kind, c["order"], c["mass"])
    kap = torch.as_tensor(kappa, device=dev)
    co = fea.make_coeffs(kappa=kap, f_kind={"const": 1, "sinprod": 2}[c["f_kind"]], f_param=c["f_param"])
    q = fea.make_quadrature(c["npts"], fea.FEA_FP64)
    m.pattern(c["order"])
    gk = torch.empty(c["tets"].shape[1], dtype=torch.float64, device=dev)
    gx = torch.empty((3, c["coords"].shape[1]), dtype=torch.float64, device=dev)
    fea.fea_assemble_backward(m.h, form, co, q, torch.as_tensor(gV, device=dev), torch.as_tensor(g, device=dev),
                              gk, gx)
    torch.cuda.synchronize()
    m.check()
    return gk.cpu().numpy(), gx.cpu().numpy()


@pytest.mark.parametrize("kind,n", [("p1_kappa", 5), ("p2_diffmass", 4), ("p2_poisson", 3)])
def test_backward_matches_oracle_dual_numbers(kind, n):
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=5)
    edof, nsd = oracle.dof_table(c["order"], c["coords"].shape[1], c["tets"])
    rp, ci = oracle.pattern(nsd, edof)
    v, w, g, gV = _loss_weights(nsd, rp, ci, seed=n)
    gk_o, gx_o = oracle.assemble_grad(c["coords"], c["tets"], c["order"], edof, rp, ci, gV, g, mass=c["mass"],
                                      kappa=c["kappa"], f_kind=c["f_kind"], f_param=c["f_param"], npts=c["npts"])
    m = fea.Mesh(c["coords"], c["tets"])
    gk, gx = _gpu_backward(m, c, gV, g, c["kappa"])
    assert vec_scaled_error(gk_o, gk) <= TOL_GRAD
    assert vec_scaled_error(gx_o, gx) <= TOL_GRAD


def test_backward_partial_inputs():
    # NULL grad_values or grad_rhs are zero; outputs are linear in them
    import torch
    from paper_1802_03433_gb300 import fea
    c = case("p2_diffmass", 3, seed=2)
    edof, nsd = oracle.dof_table(2, c["coords"].shape[1], c["tets"])
    rp, ci = oracle.pattern(nsd, edof)
    _, _, g, gV = _loss_weights(nsd, rp, ci, seed=1)
    m = fea.Mesh(c["coords"], c["tets"])
    gk_all, gx_all = _gpu_backward(m, c, gV, g, c["kappa"])
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0)
    kap = torch.as_tensor(c["kappa"], device="cuda")
    co = fea.make_coeffs(kappa=kap, f_kind=2, f_param=c["f_param"])
    q = fea.make_quadrature(11)
    parts = []
    for a, b in ((gV, None), (None, g)):
        gk = torch.empty(c["tets"].shape[1], dtype=torch.float64, device="cuda")
        gx = torch.empty((3, c["coords"].shape[1]), dtype=torch.float64, device="cuda")
        fea.fea_assemble_backward(m.h, form, co, q, None if a is None else torch.as_tensor(a, device="cuda"),
                                  None if b is None else torch.as_tensor(b, device="cuda"), gk, gx)
        parts.append((gk.cpu().numpy(), gx.cpu().numpy()))
    assert np.abs(parts[1][0]).max() == 0.0  # the load does not depend on kappa
    np.testing.assert_allclose(parts[0][0] + parts[1][0], gk_all, rtol=0, atol=1e-13 * np.abs(gk_all).max())
    np.testing.assert_allclose(parts[0][1] + parts[1][1], gx_all, rtol=0, atol=1e-13 * np.abs(gx_all).max())


def test_autograd_function_gradcheck():
    import torch
    from paper_1802_03433_gb300 import fea
    from paper_1802_03433_gb300.autograd import FeaAssemble
    c = case("p1_kappa", 2, seed=3)
    m = fea.Mesh(c["coords"], c["tets"])
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 1, 0.5)
    kap = torch.as_tensor(c["kappa"], device="cuda").requires_grad_()
    xyz = [torch.as_tensor(c["coords"][k].copy(), device="cuda").requires_grad_() for k in range(3)]

    def f(k, x, y, z):
        return FeaAssemble.apply(k, x, y, z, m, form, 4, fea.FEA_LOAD_SINPROD, (mg.SIN_AMP,))

    assert torch.autograd.gradcheck(f, (kap, *xyz), eps=1e-6, atol=1e-6, rtol=1e-5)


def test_autograd_loss_matches_oracle():
    import torch
    from paper_1802_03433_gb300 import fea
    from paper_1802_03433_gb300.autograd import FeaAssemble
    c = case("p2_diffmass", 3, seed=8)
    m = fea.Mesh(c["coords"], c["tets"])
    rp_t, ci_t = m.pattern_tensors(2)
    rp, ci = rp_t.cpu().numpy(), ci_t.cpu().numpy()
    nd = rp.size - 1
    v, w, g, gV = _loss_weights(nd, rp, ci, seed=4)
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0)
    kap = torch.as_tensor(c["kappa"], device="cuda").requires_grad_()
    xyz = [torch.as_tensor(c["coords"][k].copy(), device="cuda").requires_grad_() for k in range(3)]
    vals, rhs = FeaAssemble.apply(kap, *xyz, m, form, 11, fea.FEA_LOAD_SINPROD, (mg.SIN_AMP,))
    rows = torch.repeat_interleave(torch.arange(nd, device="cuda"), torch.diff(rp_t.long()))
    vt, wt, gt = (torch.as_tensor(a, device="cuda") for a in (v, w, g))
    L = (vals * vt[rows] * wt[ci_t.long()]).sum() + (gt * rhs).sum()
    L.backward()
    edof, _ = oracle.dof_table(2, c["coords"].shape[1], c["tets"])
    gk_o, gx_o = oracle.assemble_grad(c["coords"], c["tets"], 2, edof, rp, ci, gV, g, mass=1.0, kappa=c["kappa"],
                                      f_kind="sinprod", f_param=c["f_param"], npts=11)
    assert vec_scaled_error(gk_o, kap.grad.cpu().numpy()) <= TOL_GRAD
    gx = np.stack([t.grad.cpu().numpy() for t in xyz])
    assert vec_scaled_error(gx_o, gx) <= TOL_GRAD


def test_adjoint_96_cube_central_differences():
    """Adjoint of P1 kappa-diffusion on the 96^3 mesh (5,308,416 tets):
    L = v^T K w + g^T f; dL/dkappa and dL/dx at 64 random entries (32 + 32)
    against central differences with h = 1e-6, evaluated element-locally
    (the difference of two deterministic assemblies is nonzero only on the
    perturbed element's entries)."""
    import torch
    from paper_1802_03433_gb300 import fea
    d = mg.adjoint_p1(96)
    m = fea.Mesh(d["coords"], d["tets"])
    rp, ci = m.pattern_tensors(1)
    nd = rp.numel() - 1
    rows = torch.repeat_interleave(torch.arange(nd, device="cuda"), torch.diff(rp.long()))
    v, w, g = (torch.as_tensor(d[k], device="cuda") for k in ("v", "w", "g"))
    gV = v[rows] * w[ci.long()]
    kap = torch.as_tensor(d["kappa"], device="cuda")
    form = fea.make_form(fea.FEA_POISSON, 1)
    q = fea.make_quadrature(4)

    def assemble(k):
        co = fea.make_coeffs(kappa=k, f_kind=2, f_param=(mg.SIN_AMP,))
        vals, rhs = m.assemble(form, co, q)
        return vals.clone(), rhs.clone()

    E, N = d["tets"].shape[1], d["coords"].shape[1]
    gk = torch.empty(E, dtype=torch.float64, device="cuda")
    gx = torch.empty((3, N), dtype=torch.float64, device="cuda")
    fea.fea_assemble_backward(m.h, form, fea.make_coeffs(kappa=kap, f_kind=2, f_param=(mg.SIN_AMP,)), q, gV, g, gk, gx)
    torch.cuda.synchronize()
    gk, gx = gk.cpu().numpy(), gx.cpu().numpy()
    med = np.median(np.abs(np.concatenate([gk, gx.ravel()])))
    h = 1e-6
    rng = np.random.default_rng(1)

    def dL(p, mm):
        return float((gV * (p[0] - mm[0])).sum() + (g * (p[1] - mm[1])).sum()) / (2 * h)

    for e in rng.choice(E, 32, replace=False):
        kp, km = kap.clone(), kap.clone()
        kp[e] += h
        km[e] -= h
        fd = dL(assemble(kp), assemble(km))
        assert abs(fd - gk[e]) <= 1e-6 * max(abs(gk[e]), med), (e, fd, gk[e])
    coords = [m.x, m.y, m.z]
    for node in rng.choice(N, 32, replace=False):
        comp = int(rng.integers(3))
        orig = coords[comp][node].item()
        coords[comp][node] = orig + h
        p = assemble(kap)
        coords[comp][node] = orig - h
        mm = assemble(kap)
        coords[comp][node] = orig
        fd = dL(p, mm)
        assert abs(fd - gx[comp, node]) <= 1e-6 * max(abs(gx[comp, node]), med), (node, comp, fd, gx[comp, node])
    m.close()
