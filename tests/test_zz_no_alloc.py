"""fea_assemble_noalloc, the allocation-free variant of fea_assemble for
callers that cannot let a library call cudaMalloc (device memory reserved
by another allocator, or loops that cannot take the synchronisation of an
allocation).  Its scratch is a fixed device array inside the library.

Called through the C-ABI twice in a row on the same inputs, it must agree
with fea_assemble within the FP64 parity tolerance; meshes too large for the
fixed array are rejected before anything runs.  This file sorts last so that
a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from common import TOL_FP64, TOL_MIXED, case, row_scaled_error, vec_scaled_error

pytestmark = pytest.mark.gpu


def _setup(kind, n, prec):
    import torch
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=11)
    m = fea.Mesh(c["coords"], c["tets"])
    keep = []
    if c["form"] == "elasticity":
        lam, mu = torch.as_tensor(c["lam"], device="cuda"), torch.as_tensor(c["mu"], device="cuda")
        keep += [lam, mu]
        co = fea.make_coeffs(lam=lam, mu=mu, f_kind=1, f_param=c["f_param"])
        form = fea.make_form(fea.FEA_ELASTICITY, 1)
    else:
        kap = None if c["kappa"] is None else torch.as_tensor(c["kappa"], device="cuda")
        keep.append(kap)
        co = fea.make_coeffs(kappa=kap, f_kind=2, f_param=c["f_param"])
        form = fea.make_form(fea.FEA_DIFFUSION_MASS if c["mass"] else fea.FEA_POISSON, c["order"], c["mass"])
    q = fea.make_quadrature(c["npts"], prec)
    return fea, m, form, co, q, keep


@pytest.mark.parametrize("kind,n,prec", [("p1_kappa", 8, 0), ("p2_diffmass", 5, 0), ("elasticity", 4, 0),
                                         ("p2_diffmass", 5, 1)])
def test_noalloc_matches_fea_assemble_twice(kind, n, prec):
    import torch
    fea, m, form, co, q, keep = _setup(kind, n, prec)
    ref_v, ref_r = m.assemble(form, co, q)
    ref_v, ref_r = ref_v.clone(), ref_r.clone()
    rp, _ = m.pattern_tensors(form.order, 3 if form.kind == fea.FEA_ELASTICITY else 1)
    rp = rp.cpu().numpy()
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    for _ in range(2):
        v = torch.full_like(ref_v, np.nan)
        r = torch.full_like(ref_r, np.nan)
        fea.fea_assemble_noalloc(m.h, form, co, q, v, r)
        torch.cuda.synchronize()
        m.check()
        assert row_scaled_error(rp, ref_v.cpu().numpy(), v.cpu().numpy()) <= tol
        assert vec_scaled_error(ref_r.cpu().numpy(), r.cpu().numpy()) <= tol
    m.close()


def test_noalloc_rejects_meshes_above_the_fixed_scratch():
    import torch
    fea, m, form, co, q, keep = _setup("p2_diffmass", 40, 0)  # 384,000 P2 tets ~ 400 MB of scratch
    ndof, nnz = m.pattern(2)
    v = torch.empty(nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_assemble_noalloc(m.h, form, co, q, v, None)
    assert ei.value.status == 1 and "fixed" in str(ei.value)
    m.close()
