"""Batched assembly (fea_batch_*): one CUDA-graph launch over many uneven
P1/P2 meshes gives, mesh by mesh, bitwise the single-mesh results, and those
match the oracle (GPU)."""
import numpy as np
import pytest

import oracle
from common import TOL_FP64, row_scaled_error, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


def _build(specs):
    import torch
    from paper_1802_03433_gb300 import fea
    meshes, forms, quads, coeffs, keep = [], [], [], [], []
    for d in specs:
        m = fea.Mesh(d["coords"], d["tets"])
        kap = torch.as_tensor(d["kappa"], device="cuda")
        keep.append(kap)
        meshes.append(m)
        forms.append(fea.make_form(fea.FEA_POISSON if d["mass"] == 0 else fea.FEA_DIFFUSION_MASS, d["order"],
                                   d["mass"]))
        quads.append(fea.make_quadrature(d["npts"], fea.FEA_FP64))
        coeffs.append(fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=(d["f_amp"],)))
    return meshes, forms, quads, coeffs, keep


def _single(meshes, forms, quads, coeffs):
    outs = []
    for m, f, q, c in zip(meshes, forms, quads, coeffs):
        v, r = m.assemble(f, c, q)
        outs.append((v.clone(), r.clone()))
    return outs


def _bitwise_equal(a, b):
    import torch
    return torch.equal(a.view(torch.int64), b.view(torch.int64))


def test_small_batch_matches_single_and_oracle():
    import torch
    from paper_1802_03433_gb300 import fea
    specs = mg.batch(n_meshes=7, lo=1, hi=5, seed=3)
    specs[3]["mass"] = 0.75  # one diffusion + mass mesh
    meshes, forms, quads, coeffs, keep = _build(specs)
    single = _single(meshes, forms, quads, coeffs)
    b = fea.Batch(meshes, forms, quads, coeffs, fea.FEA_LOAD_SINPROD)
    for rep in range(2):  # replays of the same graph
        b.assemble()
        torch.cuda.synchronize()
        for k in range(len(meshes)):
            nnz = meshes[k].pattern(forms[k].order)[1]
            assert _bitwise_equal(b.values[k][:nnz], single[k][0])
            assert _bitwise_equal(b.rhs[k], single[k][1])
    for k, d in enumerate(specs):
        edof, nsd = oracle.dof_table(d["order"], d["coords"].shape[1], d["tets"])
        rp, ci = oracle.pattern(nsd, edof)
        ov, orhs, _ = oracle.assemble(d["coords"], d["tets"], d["order"], edof, rp, ci, mass=d["mass"],
                                      kappa=d["kappa"], f_param=(d["f_amp"],), npts=d["npts"])
        nnz = rp[-1]
        assert row_scaled_error(rp, ov, b.values[k][:nnz].cpu().numpy()) <= TOL_FP64
        assert vec_scaled_error(orhs, b.rhs[k].cpu().numpy()) <= TOL_FP64
    b.close()


def test_tuned_batch_still_bitwise():
    import torch
    from paper_1802_03433_gb300 import fea
    specs = mg.batch(n_meshes=12, lo=2, hi=9, seed=4)
    meshes, forms, quads, coeffs, keep = _build(specs)
    single = _single(meshes, forms, quads, coeffs)
    b = fea.Batch(meshes, forms, quads, coeffs, fea.FEA_LOAD_SINPROD)
    params = b.tune()
    assert params[0] in (128, 256, 512, 1024, 2048) and min(params[1:4]) > 0
    assert params[4] in (0, 1, 2) and params[5] in (0, 1)
    b.assemble()
    torch.cuda.synchronize()
    for k in range(len(meshes)):
        nnz = meshes[k].pattern(forms[k].order)[1]
        assert _bitwise_equal(b.values[k][:nnz], single[k][0])
        assert _bitwise_equal(b.rhs[k], single[k][1])
    b.close()


@pytest.mark.parametrize("orders", ["mixed_layouts", "p2_only", "p1_only"])
def test_batch_layouts_and_single_order(orders):
    """Meshes whose scatter is forced to the incidence-order layout (scatter
    classes 0) beside meshes on the tiled layout, and batches with one of the
    two order branches empty: still bitwise the single-mesh results."""
    import torch
    from paper_1802_03433_gb300 import fea
    specs = mg.batch(n_meshes=8, lo=2, hi=7, seed=6)
    if orders != "mixed_layouts":
        want = 2 if orders == "p2_only" else 1
        for d in specs:
            d["order"], d["npts"] = want, 4 if want == 1 else 11
    meshes, forms, quads, coeffs, keep = _build(specs)
    if orders == "mixed_layouts":
        for k in (0, 3, 5):
            fea.fea_mesh_set_scatter_classes(meshes[k].h, 0)
    single = _single(meshes, forms, quads, coeffs)
    b = fea.Batch(meshes, forms, quads, coeffs, fea.FEA_LOAD_SINPROD)
    for rep in range(2):
        if rep == 1:
            b.tune()
        b.assemble()
        torch.cuda.synchronize()
        for k in range(len(meshes)):
            meshes[k].check()
            nnz = meshes[k].pattern(forms[k].order)[1]
            assert _bitwise_equal(b.values[k][:nnz], single[k][0]), (k, rep)
            assert _bitwise_equal(b.rhs[k], single[k][1]), (k, rep)
    b.close()


def test_batch_rejects_mixed_rules_and_elasticity():
    from paper_1802_03433_gb300 import fea
    specs2 = mg.batch(n_meshes=3, lo=2, hi=2, seed=5)
    m2, f2, q2, c2, k2 = _build(specs2)
    assert q2[0].npts == 4
    q2[2] = fea.make_quadrature(11)  # P1 meshes 0 and 2 with different rules
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_batch_create(m2, f2, q2, fea.FEA_LOAD_SINPROD)
    assert ei.value.status == 1
    f2[0] = fea.make_form(fea.FEA_ELASTICITY, 1)
    with pytest.raises(fea.FeaError):
        fea.fea_batch_create(m2, f2, [fea.make_quadrature(4)] * 3, fea.FEA_LOAD_SINPROD)


def test_full_batch_256_meshes():
    """The 256-mesh batch (n ~ U{4..32}, half P1 / half P2, log-normal kappa):
    every mesh bitwise equal to its own single-mesh assembly, and sampled rows
    of four meshes against the oracle."""
    import torch
    from paper_1802_03433_gb300 import fea
    specs = mg.batch()
    meshes, forms, quads, coeffs, keep = _build(specs)
    single = _single(meshes, forms, quads, coeffs)
    b = fea.Batch(meshes, forms, quads, coeffs, fea.FEA_LOAD_SINPROD)
    b.tune()
    b.assemble()
    torch.cuda.synchronize()
    for k in range(len(meshes)):
        meshes[k].check()
        nnz = meshes[k].pattern(forms[k].order)[1]
        assert _bitwise_equal(b.values[k][:nnz], single[k][0]), k
        assert _bitwise_equal(b.rhs[k], single[k][1]), k
    rng = np.random.default_rng(0)
    for k in (0, 1, int(np.argmax([d["n"] for d in specs])), 255):
        d = specs[k]
        edof = meshes[k].dof_table(d["order"]).cpu().numpy()
        rp, ci = (t.cpu().numpy() for t in meshes[k].pattern_tensors(d["order"]))
        rows = rng.choice(rp.size - 1, 16, replace=False)
        ref, rr = oracle.rows(d["coords"], d["tets"], d["order"], edof, rows, kappa=d["kappa"],
                              f_param=(d["f_amp"],), npts=d["npts"])
        vals = b.values[k].cpu().numpy()
        for r in rows:
            cols, v = ref[int(r)]
            np.testing.assert_array_equal(ci[rp[r]:rp[r + 1]], cols)
            assert np.abs(vals[rp[r]:rp[r + 1]] - v).max() <= TOL_FP64 * np.abs(v).max()
    b.close()


@pytest.mark.parametrize("f_kind", ["const", "none"])
def test_batch_other_loads_bitwise(f_kind):
    """Batches with the constant load and with no load: every mesh bitwise
    equal to its single-mesh assembly (rhs too for the constant load), before
    and after tuning."""
    import torch
    from paper_1802_03433_gb300 import fea
    specs = mg.batch(n_meshes=6, lo=2, hi=6, seed=8)
    specs[2]["mass"] = 0.5
    fk = fea.FEA_LOAD_CONST if f_kind == "const" else fea.FEA_LOAD_NONE
    meshes, forms, quads, coeffs, keep = _build(specs)
    coeffs = [fea.make_coeffs(kappa=k, f_kind=fk, f_param=(1.75,)) for k in keep]
    single = []
    for m, f, q, c in zip(meshes, forms, quads, coeffs):
        v, r = m.assemble(f, c, q, with_rhs=fk != fea.FEA_LOAD_NONE)
        single.append((v.clone(), None if r is None else r.clone()))
    b = fea.Batch(meshes, forms, quads, coeffs, fk, with_rhs=fk != fea.FEA_LOAD_NONE)
    for rep in range(2):
        if rep == 1:
            b.tune()
        b.assemble()
        torch.cuda.synchronize()
        for k in range(len(meshes)):
            nnz = meshes[k].pattern(forms[k].order)[1]
            assert _bitwise_equal(b.values[k][:nnz], single[k][0]), (k, rep)
            if fk != fea.FEA_LOAD_NONE:
                assert _bitwise_equal(b.rhs[k], single[k][1]), (k, rep)
    b.close()
