"""The usage shown in the README (mesh, pattern, assemble, check) runs as
written, on a small mesh, and agrees with the oracle (GPU)."""
import numpy as np
import pytest

import oracle
from common import TOL_FP64, row_scaled_error, vec_scaled_error

pytestmark = pytest.mark.gpu


def test_readme_usage_small_mesh():
    import torch
    from paper_1802_03433_gb300 import fea, meshgen as mg

    coords, tets, rng = mg.make_cube(6, 0.2, seed=0)
    kappa_np = mg.lognormal(rng, tets.shape[1])
    kappa = torch.as_tensor(kappa_np, device="cuda")
    m = fea.Mesh(coords, tets)
    ndof, nnz = m.pattern(2)
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0)
    co = fea.make_coeffs(kappa=kappa, f_kind=fea.FEA_LOAD_SINPROD, f_param=(mg.SIN_AMP,))
    values, rhs = m.assemble(form, co, fea.make_quadrature(11, fea.FEA_FP64))
    row_ptr, col_idx = m.pattern_tensors(2)
    m.check()
    assert values.shape[0] >= nnz and rhs.shape[0] == ndof
    assert int(row_ptr[-1]) == nnz and col_idx.shape[0] == nnz

    edof, nsd = oracle.dof_table(2, coords.shape[1], tets)
    rp, ci = oracle.pattern(nsd, edof)
    np.testing.assert_array_equal(row_ptr.cpu().numpy(), rp)
    np.testing.assert_array_equal(col_idx.cpu().numpy(), ci)
    ov, orhs, _ = oracle.assemble(coords, tets, 2, edof, rp, ci, mass=1.0, kappa=kappa_np,
                                  f_param=(mg.SIN_AMP,), npts=11)
    assert row_scaled_error(rp, ov, values[:nnz].cpu().numpy()) <= TOL_FP64
    assert vec_scaled_error(orhs, rhs.cpu().numpy()) <= TOL_FP64
    m.close()
