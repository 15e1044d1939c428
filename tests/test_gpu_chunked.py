"""The chunked fixed-point scatter (FEA_SCATTER_CHUNKED; the automatic choice
for elasticity, selectable for the scalar P1 and P2 forms) against the CPU
oracle (Eq. 3), against the local-row scatter, and on the cases its
construction has to get right:
meshes smaller than one chunk, couplings shared by several chunks, vertices
in many elements, a random element and node numbering, nodes of no element,
power-of-two scaling of the coefficients, non-finite coefficients (GPU)."""
import numpy as np
import pytest

import oracle
from common import TOL_FP64, TOL_MIXED, case, gpu_system, oracle_system, row_scaled_error, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


def _mesh(c, mode):
    from paper_1802_03433_gb300 import fea
    m = fea.Mesh(c["coords"], c["tets"])
    fea.fea_mesh_set_scatter(m.h, mode)
    return m


def _chunked(c, prec=0, mesh=None):
    from paper_1802_03433_gb300 import fea
    return gpu_system(c, prec=prec, mesh=mesh or _mesh(c, fea.FEA_SCATTER_CHUNKED))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9])
@pytest.mark.parametrize("prec", [0, 1])
def test_chunked_matches_oracle(n, prec):
    c = case("elasticity", n, seed=n + 40)
    o = oracle_system(c)
    g = _chunked(c, prec)
    np.testing.assert_array_equal(g["ci"], o["ci"])
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= tol
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= tol
    g["mesh"].close()


@pytest.mark.parametrize("f_kind,f_param,npts", [("zero", (0.0,), 4), ("const", (0.5, -2.0, 3.0), 1),
                                                 ("sinprod", (1.0, 2.0, -0.5), 4), ("sinprod", (3.0, 0.0, 1.0), 11)])
@pytest.mark.parametrize("prec", [0, 1])
def test_chunked_every_load(f_kind, f_param, npts, prec):
    # FP64 and the FP32 instance (connectivity staged by bulk copies); force
    # components that are zero are skipped, a constant load's 1/4 is a shift
    c = case("elasticity", 6, seed=3)
    c["f_kind"], c["f_param"], c["npts"] = f_kind, f_param, npts
    o = oracle_system(c)
    g = _chunked(c, prec)
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= tol
    if f_kind == "zero":
        assert np.abs(g["rhs"]).max() == 0.0
    else:
        assert vec_scaled_error(o["rhs"], g["rhs"]) <= tol
    g["mesh"].close()


@pytest.mark.parametrize("prec", [0, 1])
def test_chunked_deterministic_and_bitwise_symmetric(prec):
    c = case("elasticity", 10, seed=5)
    g1 = _chunked(c, prec)
    g2 = gpu_system(c, prec=prec, mesh=g1["mesh"])
    assert np.array_equal(g1["vals"].view(np.uint64), g2["vals"].view(np.uint64))
    assert np.array_equal(g1["rhs"].view(np.uint64), g2["rhs"].view(np.uint64))
    rp, ci, v = g1["rp"], g1["ci"], g1["vals"]
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    tkey = ci.astype(np.int64) * (rp.size - 1) + rows
    assert np.array_equal(v.view(np.uint64), v[np.argsort(tkey)].view(np.uint64))
    g1["mesh"].close()


def test_chunked_agrees_with_local_rows_and_auto_picks_it():
    from paper_1802_03433_gb300 import fea
    c = case("elasticity", 12, seed=8)
    gl = gpu_system(c, mesh=_mesh(c, fea.FEA_SCATTER_LOCAL_ROWS))
    gc = _chunked(c)
    ga = gpu_system(c, mesh=_mesh(c, fea.FEA_SCATTER_AUTO))
    assert row_scaled_error(gl["rp"], gl["vals"], gc["vals"]) <= TOL_FP64
    assert vec_scaled_error(gl["rhs"], gc["rhs"]) <= TOL_FP64
    assert np.array_equal(ga["vals"].view(np.uint64), gc["vals"].view(np.uint64))
    assert not np.array_equal(gl["vals"].view(np.uint64), gc["vals"].view(np.uint64))  # really another path
    for g in (gl, gc, ga):
        g["mesh"].close()


def test_chunked_rejects_a_bad_mode():
    from paper_1802_03433_gb300 import fea
    c = case("p1_kappa", 3)
    m = _mesh(c, fea.FEA_SCATTER_CHUNKED)
    with pytest.raises(fea.FeaError):
        fea.fea_mesh_set_scatter(m.h, 3)
    m.close()


def test_chunked_unstructured_numbering():
    """A random permutation of nodes and elements: the chunks come from the
    element centroids, not from the numbering."""
    c = case("elasticity", 7, seed=9)
    rng = np.random.default_rng(2)
    N = c["coords"].shape[1]
    perm_n = rng.permutation(N)
    inv = np.empty(N, dtype=np.int64)
    inv[perm_n] = np.arange(N)
    perm_e = rng.permutation(c["tets"].shape[1])
    c["coords"] = np.ascontiguousarray(c["coords"][:, perm_n])
    c["tets"] = np.ascontiguousarray(inv[c["tets"][:, perm_e]].astype(np.int32))
    c["lam"], c["mu"] = np.ascontiguousarray(c["lam"][perm_e]), np.ascontiguousarray(c["mu"][perm_e])
    o = oracle_system(c)
    g = _chunked(c)
    np.testing.assert_array_equal(g["ci"], o["ci"])
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64
    g["mesh"].close()


def test_chunked_vertex_in_sixty_elements_and_isolated_nodes():
    """A fan of 60 tetrahedra around one vertex (60 contributions to one slot)
    plus two nodes that belong to no element (their load entries are 0)."""
    from test_gpu_parity import _fan
    coords, tets = _fan(60)
    coords = np.concatenate([coords, np.array([[50.0, 51.0], [50.0, 52.0], [50.0, 53.0]])], axis=1)
    rng = np.random.default_rng(4)
    E = tets.shape[1]
    c = dict(coords=np.ascontiguousarray(coords), tets=tets, order=1, form="elasticity",
             lam=rng.uniform(0.5, 2.0, E), mu=rng.uniform(0.5, 2.0, E), f_kind="const", f_param=(1.0, 2.0, 3.0),
             npts=4, ndpn=3)
    o = oracle_system(c)
    g = _chunked(c)
    np.testing.assert_array_equal(g["ci"], o["ci"])
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64
    assert np.all(g["rhs"][-6:] == 0.0)
    g["mesh"].close()


def test_chunked_mesh_without_elements():
    import torch
    from paper_1802_03433_gb300 import fea
    coords = np.random.default_rng(0).uniform(size=(3, 5))
    m = fea.Mesh(coords, np.zeros((4, 0), dtype=np.int32))
    fea.fea_mesh_set_scatter(m.h, fea.FEA_SCATTER_CHUNKED)
    ndof, nnz = m.pattern(1, 3)
    assert (ndof, nnz) == (15, 0)
    rhs = torch.full((ndof,), float("nan"), dtype=torch.float64, device="cuda")
    vals, rhs = m.assemble(fea.make_form(fea.FEA_ELASTICITY, 1), fea.make_coeffs(f_kind=1, f_param=(1.0, 1.0, 1.0)),
                           fea.make_quadrature(4), rhs=rhs)
    torch.cuda.synchronize()
    m.check()
    assert rhs.abs().max().item() == 0.0
    m.close()


@pytest.mark.parametrize("k", [60, -60, 1000, -900])
def test_chunked_power_of_two_scaling_is_exact(k):
    """Scaling lambda and mu by 2^k scales every element entry by 2^k exactly,
    moves every slot's exponent bound by k and leaves the fixed-point
    integers unchanged: the values scale by 2^k bit for bit, the loads do not
    change."""
    c = case("elasticity", 5, seed=12)
    g1 = _chunked(c)
    c2 = dict(c, lam=np.ldexp(c["lam"], k), mu=np.ldexp(c["mu"], k))
    g2 = _chunked(c2)
    assert np.array_equal(np.ldexp(g1["vals"], k).view(np.uint64), g2["vals"].view(np.uint64))
    assert np.array_equal(g1["rhs"].view(np.uint64), g2["rhs"].view(np.uint64))
    g1["mesh"].close()
    g2["mesh"].close()


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_chunked_non_finite_coefficient_poisons_exactly_its_entries(bad):
    c = case("elasticity", 6, seed=14)
    g0 = _chunked(c)
    e = 777
    lam = c["lam"].copy()
    lam[e] = bad
    g = _chunked(dict(c, lam=lam))
    # the entries coupling two nodes of element e are NaN, every other entry
    # is bitwise unchanged
    rp, ci = g["rp"], g["ci"]
    nodes = c["tets"][:, e]
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    hit = np.isin(rows // 3, nodes) & np.isin(ci // 3, nodes)
    assert np.all(np.isnan(g["vals"][hit]))
    assert np.array_equal(g["vals"][~hit].view(np.uint64), g0["vals"][~hit].view(np.uint64))
    assert np.array_equal(g["rhs"].view(np.uint64), g0["rhs"].view(np.uint64))
    g0["mesh"].close()
    g["mesh"].close()


def test_chunked_full_size_rows_against_oracle_at_96():
    """A mesh of many chunks (96^3 cubes, 5.3M tets, 13,824 chunks): rows of
    2,000 nodes (all three components) against the oracle's brute-force rows."""
    import torch
    from paper_1802_03433_gb300 import fea
    from paper_1802_03433_gb300 import meshgen as mg
    d = mg.elasticity_p1(96, seed=1)
    m = fea.Mesh(d["coords"], d["tets"])
    lam, mu = torch.as_tensor(d["lam"], device="cuda"), torch.as_tensor(d["mu"], device="cuda")
    co = fea.make_coeffs(lam=lam, mu=mu, f_kind=fea.FEA_LOAD_CONST, f_param=d["body"])
    vals, rhs = m.assemble(fea.make_form(fea.FEA_ELASTICITY, 1), co, fea.make_quadrature(4))
    torch.cuda.synchronize()
    m.check()
    rp3, ci3 = (t.cpu().numpy() for t in m.pattern_tensors(1, 3))
    N = d["coords"].shape[1]
    nodes = np.random.default_rng(96).choice(N, 2000, replace=False)
    rows = (3 * nodes[:, None] + np.arange(3)[None, :]).reshape(-1)
    r, cc, v, rr, orhs = oracle.rows_arrays(d["coords"], d["tets"], 1, d["tets"], rows, kind="elasticity",
                                            lam=d["lam"], mu=d["mu"], f_kind="const", f_param=d["body"], npts=4)
    rp = rp3.astype(np.int64)
    lens = rp[rr + 1] - rp[rr]
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    idx = np.repeat(rp[rr] - starts, lens) + np.arange(lens.sum())
    np.testing.assert_array_equal(ci3[idx], cc)
    got = vals.cpu().numpy()[idx]
    scale = np.maximum.reduceat(np.abs(v), starts)
    assert float(np.max(np.abs(got - v) / np.repeat(scale, lens))) <= TOL_FP64
    grhs = rhs.cpu().numpy()
    assert np.abs(grhs[rr] - orhs).max() <= TOL_FP64 * np.abs(grhs).max()
    m.close()


# ---------------------------------------------------------------- scalar forms
SCALAR = [("p1_poisson", 8), ("p1_kappa", 7), ("p2_diffmass", 6), ("p2_poisson", 5), ("p2_diffmass", 1),
          ("p1_kappa", 2)]


@pytest.mark.parametrize("kind,n", SCALAR)
@pytest.mark.parametrize("prec", [0, 1])
def test_chunked_scalar_matches_oracle(kind, n, prec):
    c = case(kind, n, seed=n + 60)
    o = oracle_system(c)
    g = _chunked(c, prec)
    np.testing.assert_array_equal(g["ci"], o["ci"])
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= tol
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= tol
    g["mesh"].close()


@pytest.mark.parametrize("npts", [1, 4, 11])
@pytest.mark.parametrize("order", [1, 2])
def test_chunked_scalar_every_rule_and_load(npts, order):
    c = case("p2_diffmass" if order == 2 else "p1_kappa", 4, seed=7)
    c["npts"] = npts
    for fk, fp in (("const", (2.5,)), ("sinprod", (mg.SIN_AMP,)), ("zero", (0.0,))):
        c["f_kind"], c["f_param"] = fk, fp
        o = oracle_system(c)
        g = _chunked(c)
        assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
        assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64 if fk != "zero" else np.abs(g["rhs"]).max() == 0.0
        g["mesh"].close()


@pytest.mark.parametrize("kind", ["p1_kappa", "p2_diffmass"])
@pytest.mark.parametrize("prec", [0, 1])
def test_chunked_scalar_deterministic_symmetric_and_close_to_local_rows(kind, prec):
    from paper_1802_03433_gb300 import fea
    c = case(kind, 9, seed=4)
    g1 = _chunked(c, prec)
    g2 = gpu_system(c, prec=prec, mesh=g1["mesh"])
    assert np.array_equal(g1["vals"].view(np.uint64), g2["vals"].view(np.uint64))
    assert np.array_equal(g1["rhs"].view(np.uint64), g2["rhs"].view(np.uint64))
    rp, ci, v = g1["rp"], g1["ci"], g1["vals"]
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    tkey = ci.astype(np.int64) * (rp.size - 1) + rows
    assert np.array_equal(v.view(np.uint64), v[np.argsort(tkey)].view(np.uint64))
    gl = gpu_system(c, prec=prec, mesh=_mesh(c, fea.FEA_SCATTER_LOCAL_ROWS))
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    assert row_scaled_error(gl["rp"], gl["vals"], v) <= tol
    assert vec_scaled_error(gl["rhs"], g1["rhs"]) <= tol
    g1["mesh"].close()
    gl["mesh"].close()


@pytest.mark.parametrize("k", [60, -60, 1000, -900])
def test_chunked_scalar_power_of_two_scaling_is_exact(k):
    c = case("p2_poisson", 4, seed=16)
    g1 = _chunked(c)
    g2 = _chunked(dict(c, kappa=np.ldexp(c["kappa"], k)))
    assert np.array_equal(np.ldexp(g1["vals"], k).view(np.uint64), g2["vals"].view(np.uint64))
    assert np.array_equal(g1["rhs"].view(np.uint64), g2["rhs"].view(np.uint64))
    g1["mesh"].close()
    g2["mesh"].close()


def test_chunked_scalar_nan_kappa_poisons_exactly_its_entries():
    c = case("p2_diffmass", 5, seed=18)
    g0 = _chunked(c)
    e = 333
    kap = c["kappa"].copy()
    kap[e] = np.nan
    g = _chunked(dict(c, kappa=kap))
    rp, ci = g["rp"], g["ci"]
    dofs = g["mesh"].dof_table(2).cpu().numpy()[:, e]
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    hit = np.isin(rows, dofs) & np.isin(ci, dofs)
    assert np.all(np.isnan(g["vals"][hit]))
    assert np.array_equal(g["vals"][~hit].view(np.uint64), g0["vals"][~hit].view(np.uint64))
    assert np.array_equal(g["rhs"].view(np.uint64), g0["rhs"].view(np.uint64))
    g0["mesh"].close()
    g["mesh"].close()


def test_chunked_scalar_unstructured_numbering():
    c = case("p2_diffmass", 5, seed=19)
    rng = np.random.default_rng(3)
    N = c["coords"].shape[1]
    perm_n = rng.permutation(N)
    inv = np.empty(N, dtype=np.int64)
    inv[perm_n] = np.arange(N)
    perm_e = rng.permutation(c["tets"].shape[1])
    c["coords"] = np.ascontiguousarray(c["coords"][:, perm_n])
    c["tets"] = np.ascontiguousarray(inv[c["tets"][:, perm_e]].astype(np.int32))
    c["kappa"] = np.ascontiguousarray(c["kappa"][perm_e])
    o = oracle_system(c)
    g = _chunked(c)
    np.testing.assert_array_equal(g["ci"], o["ci"])
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64
    g["mesh"].close()


@pytest.mark.parametrize("kind,n", [("p2_diffmass", 64), ("p1_kappa", 96)])
def test_chunked_scalar_full_size_every_value(kind, n):
    """The P2 64^3 and P1 96^3 workloads with the chunked scatter: every value
    and load entry against the oracle."""
    from paper_1802_03433_gb300 import meshgen as mgen
    d = mgen.diffusion_mass_p2(n) if kind == "p2_diffmass" else mgen.adjoint_p1(n)
    c = dict(coords=d["coords"], tets=d["tets"], order=d["order"], form="diffusion", mass=d["mass"],
             kappa=d["kappa"], f_kind="sinprod", f_param=(d["f_amp"],), npts=d["npts"], ndpn=1)
    g = _chunked(c)
    o = oracle_system(c)
    np.testing.assert_array_equal(g["rp"], o["rp"])
    np.testing.assert_array_equal(g["ci"], o["ci"])
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64
    g["mesh"].close()


@pytest.mark.parametrize("shift,scale,prec", [(1e3, 1.0, 0), (1e3, 1.0, 1), (3e6, 1.0, 0), (3e6, 1.0, 1),
                                              (0.0, 2.0 ** 40, 0), (0.0, 2.0 ** -40, 0), (0.0, 2.0 ** 100, 0),
                                              (0.0, 2.0 ** -100, 0)])
def test_chunked_translated_and_scaled_coordinates(shift, scale, prec):
    """Phase A takes each element's edges in FP32 from split coordinates when
    its coordinates lie in [2^-70, 2^70) and are not far above its edges
    (shift 1e3, scale 2^+-40), else from the FP64 coordinates (shift 3e6,
    scale 2^+-100): both agree with the oracle."""
    c = case("elasticity", 5, seed=14)
    c = dict(c, coords=np.ascontiguousarray(c["coords"] * scale + shift))
    o = oracle_system(c)
    g = _chunked(c, prec)
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= tol
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= tol
    g["mesh"].close()
