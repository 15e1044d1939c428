"""Row partition on the GPU: each part's sub-mesh (fea_partition) assembled
with the library; the parts' owned rows put together are the whole mesh's
system.  With the local-row scatter (contributions added in element order,
which the partition keeps) they are bitwise equal; the chunked scatter groups
the elements differently on a sub-mesh and agrees to rounding.  The parts
run one after the other on one GPU (no kernel waits on another)."""
import numpy as np
import pytest

from common import TOL_FP64, case, gpu_system, row_scaled_error, vec_scaled_error

pytestmark = pytest.mark.gpu


def _parts(c, nparts, mode):
    from paper_1802_03433_gb300 import fea
    ndpn = c["ndpn"]
    N = c["coords"].shape[1]
    lens, cols, vals, rhs = [], [], [], []
    for part in range(nparts):
        p = fea.fea_partition(c["tets"], N, nparts, part)
        sub = dict(c, coords=np.ascontiguousarray(c["coords"][:, p["nodes"]]), tets=p["sub_tets"])
        for key in ("kappa", "lam", "mu"):
            if sub.get(key) is not None:
                sub[key] = np.ascontiguousarray(c[key][p["elems"]])
        m = fea.Mesh(sub["coords"], sub["tets"])
        fea.fea_mesh_set_scatter(m.h, mode)
        g = gpu_system(sub, mesh=m)
        r0, ln, cc, vv = fea.owned_rows(p, g["rp"], g["ci"], g["vals"], ndpn)
        a = int(np.searchsorted(p["nodes"], p["lo"]))
        lens.append(ln)
        cols.append(cc)
        vals.append(vv)
        rhs.append(g["rhs"][ndpn * a: ndpn * a + ndpn * (p["hi"] - p["lo"])])
        m.close()
    return np.concatenate(lens), np.concatenate(cols), np.concatenate(vals), np.concatenate(rhs)


@pytest.mark.parametrize("kind,n,nparts", [("p1_kappa", 12, 2), ("p1_kappa", 9, 3), ("elasticity", 10, 2),
                                           ("elasticity", 8, 4)])
def test_owned_rows_bitwise_the_single_mesh_with_local_rows(kind, n, nparts):
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=33)
    m = fea.Mesh(c["coords"], c["tets"])
    fea.fea_mesh_set_scatter(m.h, fea.FEA_SCATTER_LOCAL_ROWS)
    whole = gpu_system(c, mesh=m)
    lens, cols, vals, rhs = _parts(c, nparts, fea.FEA_SCATTER_LOCAL_ROWS)
    np.testing.assert_array_equal(lens, np.diff(whole["rp"]))
    np.testing.assert_array_equal(cols, whole["ci"])
    assert np.array_equal(vals.view(np.uint64), whole["vals"].view(np.uint64))
    assert np.array_equal(rhs.view(np.uint64), whole["rhs"].view(np.uint64))
    m.close()


@pytest.mark.parametrize("n,nparts", [(10, 2), (12, 3)])
def test_owned_rows_with_the_chunked_scatter(n, nparts):
    from paper_1802_03433_gb300 import fea
    c = case("elasticity", n, seed=35)
    whole = gpu_system(c)  # automatic: chunked
    lens, cols, vals, rhs = _parts(c, nparts, fea.FEA_SCATTER_CHUNKED)
    np.testing.assert_array_equal(lens, np.diff(whole["rp"]))
    np.testing.assert_array_equal(cols, whole["ci"])
    assert row_scaled_error(whole["rp"], whole["vals"], vals) <= TOL_FP64
    assert vec_scaled_error(whole["rhs"], rhs) <= TOL_FP64
    whole["mesh"].close()


def _backward(fea, coords, tets, kappa, gV, g, c):
    import torch
    m = fea.Mesh(coords, tets)
    m.pattern(1)
    kap = torch.as_tensor(kappa, device="cuda")
    form = fea.make_form(fea.FEA_POISSON, 1)
    co = fea.make_coeffs(kappa=kap, f_kind=fea.FEA_LOAD_SINPROD, f_param=c["f_param"])
    q = fea.make_quadrature(c["npts"], fea.FEA_FP64)
    gk = torch.empty(tets.shape[1], dtype=torch.float64, device="cuda")
    gx = torch.empty((3, coords.shape[1]), dtype=torch.float64, device="cuda")
    fea.fea_assemble_backward(m.h, form, co, q, torch.as_tensor(gV, device="cuda"),
                              torch.as_tensor(g, device="cuda"), gk, gx)
    torch.cuda.synchronize()
    m.check()
    rp, ci = m.pattern_tensors(1)
    out = gk.cpu().numpy(), gx.cpu().numpy(), rp.cpu().numpy(), ci.cpu().numpy()
    m.close()
    return out


@pytest.mark.parametrize("n,nparts", [(10, 2), (9, 3)])
def test_adjoint_by_parts_matches_the_whole_mesh(n, nparts):
    """The backward kernel on each part's sub-mesh, given the whole mesh's
    dL/dvalues at the sub-mesh's entries (sub_positions): dL/dx of the owned
    nodes and dL/dkappa of the part's elements are bitwise those of the whole
    mesh (L = v^T K w + g^T f); the parts run one after the other on one GPU."""
    from paper_1802_03433_gb300 import fea
    c = case("p1_kappa", n, seed=37)
    N = c["coords"].shape[1]
    rng = np.random.default_rng(38)
    v, w, g = rng.standard_normal(N), rng.standard_normal(N), rng.standard_normal(N)
    m = fea.Mesh(c["coords"], c["tets"])
    rp, ci = (t.cpu().numpy() for t in m.pattern_tensors(1))
    m.close()
    rows = np.repeat(np.arange(N), np.diff(rp))
    gV = v[rows] * w[ci]
    gk, gx, _, _ = _backward(fea, c["coords"], c["tets"], c["kappa"], gV, g, c)
    for part in range(nparts):
        p = fea.fea_partition(c["tets"], N, nparts, part)
        sc = np.ascontiguousarray(c["coords"][:, p["nodes"]])
        # the sub-mesh's pattern, then the gradient at its entries
        sm = fea.Mesh(sc, p["sub_tets"])
        srp, sci = (t.cpu().numpy() for t in sm.pattern_tensors(1))
        sm.close()
        pos = fea.sub_positions(p, srp, sci, rp, ci)
        sgk, sgx, _, _ = _backward(fea, sc, p["sub_tets"], np.ascontiguousarray(c["kappa"][p["elems"]]), gV[pos],
                                   g[p["nodes"]], c)
        a, b = np.searchsorted(p["nodes"], [p["lo"], p["hi"]])
        # same elements in the same order, each node's contributions added
        # in element order: bit for bit
        assert np.array_equal(gk[p["elems"]].view(np.uint64), sgk.view(np.uint64))
        assert np.array_equal(gx[:, p["lo"]:p["hi"]].view(np.uint64), sgx[:, a:b].view(np.uint64))
