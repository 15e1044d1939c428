"""The largest meshes the CSR layout takes: row_ptr and col_idx are int32, so
a pattern holds at most INT32_MAX nonzeros.  For P1 elasticity on the n^3
Kuhn cube, nnz = 9 (15 n^3 + 21 n^2 + 9 n + 1): n = 251 gives 2,146,716,414
(94,879,506 tets, 48,009,024 dofs, 17.2 GB of values), the largest that
fits; n = 252 gives 2,172,428,757, above INT32_MAX, and is refused with
FEA_ERR_OVERFLOW when its pattern is asked for, before anything of that size
is allocated.

At n = 251 the system is assembled through the automatic path (chunked
fixed-point scatter) and the rows of 200 sampled nodes, all three
components, are checked against the oracle's brute-force rows (Eq. 3):
columns bit for bit, values within 1e-12 row-scaled, loads within 1e-12 of
the largest.  The values stay on the device; only the sampled rows are read
back."""
import numpy as np
import pytest

import oracle
from common import TOL_FP64
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

INT32_MAX = 2 ** 31 - 1


def elasticity_nnz(n):
    return 9 * (15 * n ** 3 + 21 * n ** 2 + 9 * n + 1)


def test_the_size_limit_is_where_the_closed_form_puts_it():
    assert elasticity_nnz(251) <= INT32_MAX < elasticity_nnz(252)


def test_elasticity_252_pattern_is_refused():
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(252, 0.0, 0)
    m = fea.Mesh(coords, tets)
    assert m.pattern(1, 1)[1] == elasticity_nnz(252) // 9  # the scalar pattern fits
    with pytest.raises(fea.FeaError) as ei:
        m.pattern(1, 3)
    assert ei.value.status == 4  # FEA_ERR_OVERFLOW
    assert "INT32_MAX" in str(ei.value)
    m.close()


def test_elasticity_251_sampled_rows_against_oracle():
    import torch
    from paper_1802_03433_gb300 import fea
    n = 251
    d = mg.elasticity_p1(n, seed=5)
    N = d["coords"].shape[1]
    m = fea.Mesh(d["coords"], d["tets"])
    ndof, nnz = m.pattern(1, 3)
    assert ndof == 3 * N and nnz == elasticity_nnz(n)
    lam, mu = torch.as_tensor(d["lam"], device="cuda"), torch.as_tensor(d["mu"], device="cuda")
    co = fea.make_coeffs(lam=lam, mu=mu, f_kind=fea.FEA_LOAD_CONST, f_param=d["body"])
    vals, rhs = m.assemble(fea.make_form(fea.FEA_ELASTICITY, 1), co, fea.make_quadrature(d["npts"]))
    torch.cuda.synchronize()
    m.check()
    rp3, ci3 = m.pattern_tensors(1, 3)
    assert int(rp3[-1]) == nnz
    rng = np.random.default_rng(251)
    nodes = np.unique(np.concatenate([[0, N - 1, N // 2], rng.choice(N, 200, replace=False)]))
    rows = (3 * nodes[:, None] + np.arange(3)[None, :]).reshape(-1)
    r, c, v, rr, orhs = oracle.rows_arrays(d["coords"], d["tets"], 1, d["tets"], rows, kind="elasticity",
                                           lam=d["lam"], mu=d["mu"], f_kind="const", f_param=d["body"],
                                           npts=d["npts"])
    rp = rp3[torch.as_tensor(np.stack([rr, rr + 1]), device="cuda").long()].cpu().numpy().astype(np.int64)
    lens = rp[1] - rp[0]
    assert np.array_equal(np.repeat(rr, lens), r)
    idx = np.repeat(rp[0] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + np.arange(lens.sum())
    didx = torch.as_tensor(idx, device="cuda")
    np.testing.assert_array_equal(ci3[didx].cpu().numpy(), c)
    got = vals[didx].cpu().numpy()
    scale = np.maximum.reduceat(np.abs(v), np.concatenate([[0], np.cumsum(lens)[:-1]]))
    assert float(np.max(np.abs(got - v) / np.repeat(scale, lens))) <= TOL_FP64
    grhs = rhs[torch.as_tensor(rr, device="cuda")].cpu().numpy()
    assert np.abs(grhs - orhs).max() <= TOL_FP64 * float(rhs.abs().max())
    m.close()
