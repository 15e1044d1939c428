"""Parity at the workloads' full sizes (GPU against the CPU oracle, Eq. 3).

- P2 diffusion + mass on 64^3 (1,572,864 tets) and P1 kappa-diffusion on 96^3
  (5,308,416 tets): the complete CSR pattern bit for bit, every value within
  1e-12 row-scaled, every load entry within 1e-12 of the largest.
- P1 elasticity on 128^3 (12,582,912 tets): the complete scalar P1 pattern
  bit for bit against the oracle, the 3-dof pattern as exactly the 3 x 3
  block expansion of it, and every value and load entry of the rows of 1% of
  the nodes (all three components) against the oracle's brute-force rows.
- The adjoint on 96^3: the whole dL/dkappa and dL/dx against the oracle's
  dual-number gradient, 1e-12 of the largest entry.
- The 256-mesh batch: every mesh, pattern and values, against the oracle.

The oracle is single-threaded; the slow parts (the dual-number gradient, the
256 meshes) run as several oracle calls on host threads (ctypes releases the
GIL), each on a part of the elements or on its own meshes."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
from common import TOL_FP64, row_scaled_error, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = max(1, min(16, os.cpu_count() or 1))


def _gpu_scalar(d):
    import torch
    from paper_1802_03433_gb300 import fea
    m = fea.Mesh(d["coords"], d["tets"])
    kap = None if d["kappa"] is None else torch.as_tensor(d["kappa"], device="cuda")
    kind = fea.FEA_DIFFUSION_MASS if d["mass"] else fea.FEA_POISSON
    form = fea.make_form(kind, d["order"], d["mass"])
    co = fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=(d["f_amp"],))
    vals, rhs = m.assemble(form, co, fea.make_quadrature(d["npts"]))
    torch.cuda.synchronize()
    m.check()
    rp, ci = m.pattern_tensors(d["order"])
    out = dict(rp=rp.cpu().numpy(), ci=ci.cpu().numpy(), vals=vals.cpu().numpy(), rhs=rhs.cpu().numpy(),
               edof=m.dof_table(d["order"]).cpu().numpy())
    m.close()
    return out


def _oracle_scalar(d, edof=None):
    if edof is None:
        edof, nsd = oracle.dof_table(d["order"], d["coords"].shape[1], d["tets"])
    else:
        nsd = int(edof.max()) + 1 if edof.size else d["coords"].shape[1]
    rp, ci = oracle.pattern(nsd, edof)
    vals, rhs, bad = oracle.assemble(d["coords"], d["tets"], d["order"], edof, rp, ci, mass=d["mass"],
                                     kappa=d["kappa"], f_kind="sinprod", f_param=(d["f_amp"],), npts=d["npts"])
    assert bad == 0
    return dict(edof=edof, rp=rp, ci=ci, vals=vals, rhs=rhs)


@pytest.mark.parametrize("workload", ["p2_diffmass_64", "p1_kappa_96"])
def test_full_pattern_and_every_value(workload):
    if workload == "p2_diffmass_64":
        d = mg.diffusion_mass_p2(64)
    else:
        d = mg.adjoint_p1(96)
    g = _gpu_scalar(d)
    o = _oracle_scalar(d)
    if d["order"] == 2:
        np.testing.assert_array_equal(g["edof"], o["edof"])
    np.testing.assert_array_equal(g["rp"], o["rp"])
    np.testing.assert_array_equal(g["ci"], o["ci"])
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64


def test_elasticity_128_full_pattern_and_one_percent_of_rows():
    import torch
    from paper_1802_03433_gb300 import fea
    d = mg.elasticity_p1(128)
    m = fea.Mesh(d["coords"], d["tets"])
    lam, mu = torch.as_tensor(d["lam"], device="cuda"), torch.as_tensor(d["mu"], device="cuda")
    co = fea.make_coeffs(lam=lam, mu=mu, f_kind=fea.FEA_LOAD_CONST, f_param=d["body"])
    vals, rhs = m.assemble(fea.make_form(fea.FEA_ELASTICITY, 1), co, fea.make_quadrature(d["npts"]))
    torch.cuda.synchronize()
    m.check()
    # the scalar P1 pattern, bit for bit
    rp1, ci1 = m.pattern_tensors(1, 1)
    N = d["coords"].shape[1]
    orp, oci = oracle.pattern(N, d["tets"])
    np.testing.assert_array_equal(rp1.cpu().numpy(), orp)
    np.testing.assert_array_equal(ci1.cpu().numpy(), oci)
    del orp, oci
    # the 3-dof pattern is its 3 x 3 block expansion: row 3i + c holds, for
    # each column j of scalar row i in order, the columns 3j, 3j + 1, 3j + 2
    rp3, ci3 = m.pattern_tensors(1, 3)
    rp1l, ci1l, rp3l = rp1.long(), ci1.long(), rp3.long()
    lens = torch.diff(rp1l)
    want_rp3 = torch.zeros(3 * N + 1, dtype=torch.int64, device="cuda")
    want_rp3[1:] = torch.cumsum(torch.repeat_interleave(3 * lens, 3), 0)
    assert torch.equal(rp3l, want_rp3)
    t = (3 * ci1l[:, None] + torch.arange(3, device="cuda")[None, :]).reshape(-1)
    rows3 = torch.repeat_interleave(torch.arange(3 * N, device="cuda"), torch.diff(rp3l))
    q = torch.arange(ci3.numel(), device="cuda") - rp3l[rows3]
    assert torch.equal(ci3.long(), t[3 * rp1l[rows3 // 3] + q])
    del t, rows3, q
    # every value and load entry of the rows of 1% of the nodes
    rng = np.random.default_rng(128)
    nodes = np.unique(np.concatenate([[0, N - 1], rng.choice(N, N // 100, replace=False)]))
    rows = (3 * nodes[:, None] + np.arange(3)[None, :]).reshape(-1)
    r, c, v, rr, orhs = oracle.rows_arrays(d["coords"], d["tets"], 1, d["tets"], rows, kind="elasticity",
                                           lam=d["lam"], mu=d["mu"], f_kind="const", f_param=d["body"],
                                           npts=d["npts"])
    rp = rp3.cpu().numpy().astype(np.int64)
    lens3 = rp[rr + 1] - rp[rr]
    idx = np.repeat(rp[rr] - np.concatenate([[0], np.cumsum(lens3)[:-1]]), lens3) + np.arange(lens3.sum())
    assert np.array_equal(np.repeat(rr, lens3), r)
    np.testing.assert_array_equal(ci3.cpu().numpy()[idx], c)
    got = vals.cpu().numpy()[idx]
    scale = np.maximum.reduceat(np.abs(v), np.concatenate([[0], np.cumsum(lens3)[:-1]]))
    assert float(np.max(np.abs(got - v) / np.repeat(scale, lens3))) <= TOL_FP64
    grhs = rhs.cpu().numpy()
    assert np.abs(grhs[rr] - orhs).max() <= TOL_FP64 * np.abs(grhs).max()
    assert rr.size >= 3 * (N // 100)
    m.close()


def test_adjoint_96_whole_gradient_against_dual_numbers():
    import torch
    from paper_1802_03433_gb300 import fea
    d = mg.adjoint_p1(96)
    m = fea.Mesh(d["coords"], d["tets"])
    rp, ci = m.pattern_tensors(1)
    nd = rp.numel() - 1
    rows = torch.repeat_interleave(torch.arange(nd, device="cuda"), torch.diff(rp.long()))
    v, w, g = (torch.as_tensor(d[k], device="cuda") for k in ("v", "w", "g"))
    gV = (v[rows] * w[ci.long()]).contiguous()
    kap = torch.as_tensor(d["kappa"], device="cuda")
    co = fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=(d["f_amp"],))
    E, N = d["tets"].shape[1], d["coords"].shape[1]
    gk = torch.empty(E, dtype=torch.float64, device="cuda")
    gx = torch.empty((3, N), dtype=torch.float64, device="cuda")
    fea.fea_assemble_backward(m.h, fea.make_form(fea.FEA_POISSON, 1), co, fea.make_quadrature(4), gV, g, gk, gx)
    torch.cuda.synchronize()
    m.check()
    gk, gx = gk.cpu().numpy(), gx.cpu().numpy()
    rp_h, ci_h, gV_h = rp.cpu().numpy(), ci.cpu().numpy(), gV.cpu().numpy()
    m.close()
    # the oracle's gradient, element ranges on host threads; the node
    # gradients of the ranges are summed
    cuts = np.linspace(0, E, THREADS + 1).astype(np.int64)

    def part(k):
        lo, hi = cuts[k], cuts[k + 1]
        t = np.ascontiguousarray(d["tets"][:, lo:hi])
        return oracle.assemble_grad(d["coords"], t, 1, t, rp_h, ci_h, gV_h, d["g"], kappa=d["kappa"][lo:hi],
                                    f_kind="sinprod", f_param=(d["f_amp"],), npts=4)

    with cf.ThreadPoolExecutor(THREADS) as ex:
        parts = list(ex.map(part, range(THREADS)))
    gk_o = np.concatenate([p[0] for p in parts])
    gx_o = np.sum([p[1] for p in parts], axis=0)
    assert vec_scaled_error(gk_o, gk) <= 1e-12
    assert vec_scaled_error(gx_o, gx) <= 1e-12


def test_batch_256_every_mesh_against_oracle():
    import torch
    from paper_1802_03433_gb300 import fea
    specs = mg.batch()
    meshes, forms, quads, coeffs, keep = [], [], [], [], []
    for d in specs:
        m = fea.Mesh(d["coords"], d["tets"])
        kap = torch.as_tensor(d["kappa"], device="cuda")
        keep.append(kap)
        meshes.append(m)
        forms.append(fea.make_form(fea.FEA_POISSON, d["order"]))
        quads.append(fea.make_quadrature(d["npts"]))
        coeffs.append(fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=(d["f_amp"],)))
    b = fea.Batch(meshes, forms, quads, coeffs, fea.FEA_LOAD_SINPROD)
    b.tune()
    b.assemble()
    torch.cuda.synchronize()
    got = []
    for k, m in enumerate(meshes):
        m.check()
        nnz = m.pattern(forms[k].order)[1]
        rp, ci = m.pattern_tensors(forms[k].order)
        got.append((rp.cpu().numpy(), ci.cpu().numpy(), b.values[k][:nnz].cpu().numpy(), b.rhs[k].cpu().numpy()))
    b.close()

    def check(k):
        d = specs[k]
        o = _oracle_scalar(d)
        rp, ci, v, r = got[k]
        ok = np.array_equal(rp, o["rp"]) and np.array_equal(ci, o["ci"])
        return (k, ok, row_scaled_error(o["rp"], o["vals"], v) if ok else np.inf, vec_scaled_error(o["rhs"], r))

    with cf.ThreadPoolExecutor(THREADS) as ex:
        res = list(ex.map(check, range(len(specs))))
    assert len(res) == 256
    for k, ok, ev, er in res:
        assert ok, f"mesh {k}: pattern differs"
        assert ev <= TOL_FP64 and er <= TOL_FP64, (k, ev, er)
