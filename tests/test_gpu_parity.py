"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

CSR patterns and P2 dof tables must be bit-exact; values and loads within the
row-scaled tolerance (1e-12 FP64, 1e-5 mixed).  Sizes are chosen so the
oracle finishes in seconds while the kernels still run several CTAs with a
ragged last tile.
"""
import numpy as np
import pytest

import oracle
from common import TOL_FP64, TOL_MIXED, case, gpu_system, oracle_system, row_scaled_error, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

CASES = [("p1_poisson", 8), ("p1_kappa", 7), ("p2_diffmass", 6), ("p2_poisson", 5), ("elasticity", 5)]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.mark.parametrize("kind,n", CASES)
def test_pattern_bit_exact(torch_cuda, kind, n):
    c = case(kind, n)
    o = oracle_system(c)
    g = gpu_system(c)
    np.testing.assert_array_equal(g["rp"], o["rp"])
    np.testing.assert_array_equal(g["ci"], o["ci"])
    if c["order"] == 2:
        np.testing.assert_array_equal(g["mesh"].dof_table(2).cpu().numpy(), o["edof"])


@pytest.mark.parametrize("kind,n", CASES)
def test_values_fp64(torch_cuda, kind, n):
    c = case(kind, n)
    o = oracle_system(c)
    g = gpu_system(c, prec=0)
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64


@pytest.mark.parametrize("kind,n", CASES)
def test_values_mixed(torch_cuda, kind, n):
    c = case(kind, n)
    o = oracle_system(c)
    g = gpu_system(c, prec=1)
    e_vals = row_scaled_error(o["rp"], o["vals"], g["vals"])
    e_rhs = vec_scaled_error(o["rhs"], g["rhs"])
    assert e_vals <= TOL_MIXED and e_rhs <= TOL_MIXED
    assert e_vals > 0.0  # it really ran in reduced precision


@pytest.mark.parametrize("kind", ["p1_kappa", "p2_diffmass", "elasticity"])
def test_deterministic_and_bitwise_symmetric(torch_cuda, kind):
    c = case(kind, 4, seed=3)
    g1 = gpu_system(c)
    g2 = gpu_system(c, mesh=g1["mesh"])
    assert np.array_equal(g1["vals"].view(np.uint64), g2["vals"].view(np.uint64))
    assert np.array_equal(g1["rhs"].view(np.uint64), g2["rhs"].view(np.uint64))
    rp, ci, v = g1["rp"], g1["ci"], g1["vals"]
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    key = rows.astype(np.int64) * (rp.size - 1) + ci
    tkey = ci.astype(np.int64) * (rp.size - 1) + rows
    order = np.argsort(tkey)
    assert np.array_equal(key, np.sort(key))
    assert np.array_equal(v.view(np.uint64), v[order].view(np.uint64))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_meshes_all_forms(torch_cuda, n):
    for kind in ("p1_kappa", "p2_diffmass", "elasticity"):
        c = case(kind, n, seed=n)
        o = oracle_system(c)
        g = gpu_system(c)
        np.testing.assert_array_equal(g["ci"], o["ci"])
        assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
        assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64


@pytest.mark.parametrize("npts", [1, 4, 11])
@pytest.mark.parametrize("order", [1, 2])
def test_every_rule_and_load(torch_cuda, npts, order):
    c = case("p2_diffmass" if order == 2 else "p1_kappa", 3, seed=7)
    c["npts"] = npts
    for fk, fp in (("const", (2.5,)), ("sinprod", (mg.SIN_AMP,))):
        c["f_kind"], c["f_param"] = fk, fp
        o = oracle_system(c)
        g = gpu_system(c)
        assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64
        assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64


def test_unstructured_element_order(torch_cuda):
    # a randomly permuted element and node numbering: nothing may rely on the
    # cube ordering
    c = case("p2_diffmass", 4, seed=9)
    rng = np.random.default_rng(1)
    N = c["coords"].shape[1]
    perm_n = rng.permutation(N)
    inv = np.empty(N, dtype=np.int64)
    inv[perm_n] = np.arange(N)
    perm_e = rng.permutation(c["tets"].shape[1])
    c["coords"] = np.ascontiguousarray(c["coords"][:, perm_n])
    c["tets"] = np.ascontiguousarray(inv[c["tets"][:, perm_e]].astype(np.int32))
    c["kappa"] = np.ascontiguousarray(c["kappa"][perm_e])
    o = oracle_system(c)
    g = gpu_system(c)
    np.testing.assert_array_equal(g["ci"], o["ci"])
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64


# ---------------------------------------------------------------- edge cases
def test_mesh_without_elements(torch_cuda):
    import torch
    from paper_1802_03433_gb300 import fea
    coords = np.random.default_rng(0).uniform(size=(3, 5))
    m = fea.Mesh(coords, np.zeros((4, 0), dtype=np.int32))
    ndof, nnz = m.pattern(1)
    assert (ndof, nnz) == (5, 0)
    vals, rhs = m.assemble(fea.make_form(0, 1), fea.make_coeffs(f_kind=2, f_param=(1.0,)), fea.make_quadrature(4))
    torch.cuda.synchronize()
    assert rhs.abs().max().item() == 0.0


def test_bad_index_rejected(torch_cuda):
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(2)
    tets = tets.copy()
    tets[2, 5] = coords.shape[1] + 3
    with pytest.raises(fea.FeaError) as ei:
        fea.Mesh(coords, tets)
    assert ei.value.status == 2
    tets[2, 5] = tets[1, 5]
    with pytest.raises(fea.FeaError) as ei:
        fea.Mesh(coords, tets)
    assert ei.value.status == 2


def _fan(ntets):
    """ntets tetrahedra sharing vertex 0 and nothing else, all positively
    oriented: tet i = (0, 3i+1, 3i+2, 3i+3), its other three vertices a unit
    corner far from vertex 0."""
    pts = [np.zeros(3)]
    tets = []
    for i in range(ntets):
        o = np.array([10 + 5 * np.cos(0.1 * i), 10 + 5 * np.sin(0.1 * i), 10 + 0.05 * i])
        pts += [o + [1, 0, 0], o + [0, 1, 0], o + [0, 0, 1]]
        tets.append([0, 3 * i + 1, 3 * i + 2, 3 * i + 3])
    coords = np.ascontiguousarray(np.array(pts).T)
    tets = np.ascontiguousarray(np.array(tets, dtype=np.int32).T)
    # orient each tet positively
    for e in range(ntets):
        x = coords[:, tets[:, e]]
        if np.linalg.det(x[:, 1:] - x[:, :1]) < 0:
            tets[[1, 2], e] = tets[[2, 1], e]
    return coords, tets


def _fan_case(ntets, order, seed=0):
    coords, tets = _fan(ntets)
    rng = np.random.default_rng(seed)
    return dict(coords=coords, tets=tets, order=order, form="diffusion", mass=1.0 if order == 2 else 0.0,
                kappa=np.exp(rng.standard_normal(ntets)), f_kind="sinprod", f_param=(mg.SIN_AMP,),
                npts=11 if order == 2 else 4, ndpn=1)


@pytest.mark.parametrize("ntets,order", [(60, 2), (110, 2), (110, 1), (300, 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_long_rows_match_the_oracle(torch_cuda, ntets, order, prec):
    """Rows past the warp sort (more than 1024 candidate couplings: 110 P2 tets
    around a vertex) and past the one-byte column slots (more than 255
    entries: 541 and 991 in P2, 301 and 901 in P1) are built by one block per
    row and assembled by the long-row kernel: the pattern equals the oracle's,
    the values agree, and two runs give the same bits, symmetric."""
    c = _fan_case(ntets, order, seed=ntets)
    o = oracle_system(c)
    g1 = gpu_system(c, prec=prec)
    g2 = gpu_system(c, prec=prec, mesh=g1["mesh"])
    np.testing.assert_array_equal(g1["rp"], o["rp"])
    np.testing.assert_array_equal(g1["ci"], o["ci"])
    assert np.diff(g1["rp"]).max() > 255
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    assert row_scaled_error(o["rp"], o["vals"], g1["vals"]) <= tol
    assert vec_scaled_error(o["rhs"], g1["rhs"]) <= tol
    assert np.array_equal(g1["vals"].view(np.uint64), g2["vals"].view(np.uint64))
    rp, ci, v = g1["rp"], g1["ci"], g1["vals"]
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    tkey = ci.astype(np.int64) * (rp.size - 1) + rows
    assert np.array_equal(v.view(np.uint64), v[np.argsort(tkey)].view(np.uint64))
    g1["mesh"].close()


def test_long_rows_refused_where_slots_are_read_and_past_the_block_sort(torch_cuda):
    """The entry points that read the one-byte column slots (backward, batch,
    runtime-compiled kernels, no-alloc) refuse meshes with rows of more than
    255 entries; a row of more than 16384 candidate couplings (1,700 P2 tets
    around a vertex) is refused by the pattern build.  The handle stays usable
    after each refusal."""
    import torch
    from paper_1802_03433_gb300 import fea
    c = _fan_case(60, 2)
    m = fea.Mesh(c["coords"], c["tets"])
    ndof, nnz = m.pattern(2)
    kap = torch.as_tensor(c["kappa"], device="cuda")
    form = fea.make_form(fea.FEA_DIFFUSION_MASS, 2, 1.0)
    co = fea.make_coeffs(kappa=kap, f_kind=2, f_param=(1.0,))
    q = fea.make_quadrature(11)
    v = torch.empty(nnz, dtype=torch.float64, device="cuda")
    r = torch.empty(ndof, dtype=torch.float64, device="cuda")
    gk = torch.empty(c["tets"].shape[1], dtype=torch.float64, device="cuda")
    gx = torch.empty((3, c["coords"].shape[1]), dtype=torch.float64, device="cuda")
    for call in (lambda: fea.fea_assemble_backward(m.h, form, co, q, v, r, gk, gx),
                 lambda: fea.fea_assemble_noalloc(m.h, form, co, q, v, r),
                 lambda: fea.Batch([m], [form], [q], [co], fea.FEA_LOAD_SINPROD)):
        with pytest.raises(fea.FeaError) as ei:
            call()
        assert ei.value.status == 4
    fea.fea_assemble(m.h, form, co, q, v, r)  # fea_assemble takes them
    torch.cuda.synchronize()
    m.check()
    m.close()
    coords, tets = _fan(1700)
    m = fea.Mesh(coords, tets)
    with pytest.raises(fea.FeaError) as ei:
        m.pattern(2)
    assert ei.value.status == 4
    m.pattern(1)  # 5,101 entries in the vertex's P1 row: built
    m.check()
    m.close()


def test_inverted_element_flagged(torch_cuda):
    import torch
    from paper_1802_03433_gb300 import fea
    c = case("p1_kappa", 3)
    tets = c["tets"].copy()
    tets[[1, 2], 4] = tets[[2, 1], 4]  # flip one element's orientation
    m = fea.Mesh(c["coords"], tets)
    vals, rhs = m.assemble(fea.make_form(0, 1), fea.make_coeffs(f_kind=2, f_param=(1.0,)), fea.make_quadrature(4))
    torch.cuda.synchronize()
    with pytest.raises(fea.FeaError) as ei:
        m.check()
    assert ei.value.status == 3
    m.check()  # cleared after being reported
    # the values still use |det J| and match the oracle on the flipped mesh
    c["tets"] = tets
    o = oracle_system(c)
    assert o["bad"] == 1


def test_assemble_before_pattern_is_state_error(torch_cuda):
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(2)
    m = fea.Mesh(coords, tets)
    v = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_assemble(m.h, fea.make_form(0, 2), fea.make_coeffs(), fea.make_quadrature(4), v, None)
    assert ei.value.status == 8
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_assemble(m.h, fea.make_form(0, 1), fea.make_coeffs(), fea.make_quadrature(5), v, None)
    assert ei.value.status == 1


# ---------------------------------------------------------------- full sizes
def _sampled_rows(c, g, nrows, seed):
    ndof = g["rp"].size - 1
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([[0, ndof - 1], rng.choice(ndof, nrows, replace=False)]))
    edof = g["mesh"].dof_table(c["order"]).cpu().numpy()
    kw = dict(f_kind=c["f_kind"], f_param=c["f_param"], npts=c["npts"])
    if c["form"] == "elasticity":
        ref, rhs = oracle.rows(c["coords"], c["tets"], 1, edof, rows, kind="elasticity", lam=c["lam"],
                               mu=c["mu"], **kw)
    else:
        ref, rhs = oracle.rows(c["coords"], c["tets"], c["order"], edof, rows, mass=c["mass"],
                               kappa=c["kappa"], **kw)
    worst = 0.0
    for r in rows:
        cols, vals = ref[int(r)]
        lo, hi = g["rp"][r], g["rp"][r + 1]
        np.testing.assert_array_equal(g["ci"][lo:hi], cols)
        s = np.abs(vals).max() if vals.size else 1.0
        worst = max(worst, np.abs(g["vals"][lo:hi] - vals).max() / s)
        assert abs(g["rhs"][r] - rhs[int(r)]) <= TOL_FP64 * max(1.0, np.abs(g["rhs"]).max())
    return worst


@pytest.mark.parametrize("kind,n", [("p1_poisson", 8), ("p2_diffmass", 64), ("elasticity", 128), ("p1_kappa", 96)])
def test_full_size_sampled_rows(torch_cuda, kind, n):
    """The workloads at their full sizes: closed-form pattern size and 64 rows
    checked entry by entry against the oracle's brute-force row assembly."""
    c = case(kind, n)
    g = gpu_system(c)
    cc = mg.cube_counts(n)
    nnz = {"p1_poisson": cc["p1_nnz"], "p1_kappa": cc["p1_nnz"], "p2_diffmass": cc["p2_nnz"],
           "elasticity": 9 * cc["p1_nnz"]}[kind]
    assert g["rp"][-1] == nnz and g["ci"].size == nnz
    assert _sampled_rows(c, g, 64, seed=n) <= TOL_FP64
    if kind == "p2_diffmass":
        # 1^T A 1 = volume = 1 (the stiffness annihilates constants)
        assert abs(g["vals"].sum() - 1.0) < 1e-9
    g["mesh"].close()


@pytest.mark.parametrize("kind,n", [("p1_kappa", 12), ("p2_diffmass", 9), ("elasticity", 8)])
@pytest.mark.parametrize("prec", [0, 1])
def test_overlapped_stages_bitwise_identical(torch_cuda, kind, n, prec):
    """Element chunks overlapped with the scatter (1..16 stages) give bitwise
    the same values and loads as the sequential element-then-scatter path,
    and those match the oracle."""
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=13)
    g1 = None
    m = fea.Mesh(c["coords"], c["tets"])
    fea.fea_mesh_set_scatter(m.h, fea.FEA_SCATTER_LOCAL_ROWS)  # the stages belong to the local-row scatter
    for stages in (1, 2, 5, 8, 16):
        fea.fea_mesh_set_stages(m.h, stages)
        g = gpu_system(c, prec=prec, mesh=m)
        if g1 is None:
            g1 = g
            continue
        assert np.array_equal(g["vals"].view(np.uint64), g1["vals"].view(np.uint64)), stages
        assert np.array_equal(g["rhs"].view(np.uint64), g1["rhs"].view(np.uint64)), stages
    o = oracle_system(c)
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    assert row_scaled_error(o["rp"], o["vals"], g1["vals"]) <= tol
    assert vec_scaled_error(o["rhs"], g1["rhs"]) <= tol


@pytest.mark.parametrize("kind,n", [("p1_kappa", 7), ("p2_diffmass", 5), ("elasticity", 5), ("p2_poisson", 9)])
def test_atomic_comparison_path_matches_oracle(torch_cuda, kind, n):
    """The paper's sparse Algorithm 1 (row search + global atomicAdd): equal to
    the oracle within the FP64 tolerance (bitwise reproducibility is not
    claimed for this path)."""
    import torch
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=17)
    o = oracle_system(c)
    m = fea.Mesh(c["coords"], c["tets"])
    dev = "cuda"
    if c["form"] == "elasticity":
        lam, mu = torch.as_tensor(c["lam"], device=dev), torch.as_tensor(c["mu"], device=dev)
        co = fea.make_coeffs(lam=lam, mu=mu, f_kind=1, f_param=c["f_param"])
        form = fea.make_form(fea.FEA_ELASTICITY, 1)
        ndpn = 3
    else:
        kap = torch.as_tensor(c["kappa"], device=dev)
        co = fea.make_coeffs(kappa=kap, f_kind=2, f_param=c["f_param"])
        form = fea.make_form(fea.FEA_DIFFUSION_MASS if c["mass"] else fea.FEA_POISSON, c["order"], c["mass"])
        ndpn = 1
    ndof, nnz = m.pattern(c["order"], ndpn)
    v = torch.full((nnz,), float("nan"), dtype=torch.float64, device=dev)
    r = torch.full((ndof,), float("nan"), dtype=torch.float64, device=dev)
    fea.fea_assemble_atomic(m.h, form, co, fea.make_quadrature(c["npts"]), v, r)
    torch.cuda.synchronize()
    m.check()
    assert row_scaled_error(o["rp"], o["vals"], v.cpu().numpy()) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], r.cpu().numpy()) <= TOL_FP64


@pytest.mark.parametrize("kind,n", [("p1_kappa", 12), ("p2_diffmass", 9), ("elasticity", 8)])
@pytest.mark.parametrize("prec", [0, 1])
def test_scatter_launch_shapes_bitwise_identical(torch_cuda, kind, n, prec):
    """One deep launch, heavy/light split, one light launch, the bulk-copy
    scatter over the tiled layout (scalar forms), automatic: same bits."""
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=23)
    m = fea.Mesh(c["coords"], c["tets"])
    fea.fea_mesh_set_scatter(m.h, fea.FEA_SCATTER_LOCAL_ROWS)  # the launch shapes of the local-row scatter
    ref = None
    for mode in (0, 1, 2, 3, -1):
        fea.fea_mesh_set_scatter_classes(m.h, mode)
        g = gpu_system(c, prec=prec, mesh=m)
        if ref is None:
            ref = g
            continue
        assert np.array_equal(g["vals"].view(np.uint64), ref["vals"].view(np.uint64)), mode
        assert np.array_equal(g["rhs"].view(np.uint64), ref["rhs"].view(np.uint64)), mode
    o = oracle_system(c)
    assert row_scaled_error(o["rp"], o["vals"], ref["vals"]) <= (TOL_FP64 if prec == 0 else TOL_MIXED)


@pytest.mark.parametrize("kind,n", [("p1_kappa", 12), ("p2_diffmass", 9)])
@pytest.mark.parametrize("prec", [0, 1])
def test_scatter_stage_counts_bitwise_identical(torch_cuda, kind, n, prec):
    """The bulk-copy scatter with 2, 3 and 4 stages per CTA and the automatic
    count: same bits."""
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=29)
    m = fea.Mesh(c["coords"], c["tets"])
    fea.fea_mesh_set_scatter_classes(m.h, 3)
    ref = None
    for st in (3, 2, 4, 0):
        fea.fea_mesh_set_scatter_stages(m.h, st)
        g = gpu_system(c, prec=prec, mesh=m)
        if ref is None:
            ref = g
            continue
        assert np.array_equal(g["vals"].view(np.uint64), ref["vals"].view(np.uint64)), st
        assert np.array_equal(g["rhs"].view(np.uint64), ref["rhs"].view(np.uint64)), st
    with pytest.raises(fea.FeaError):
        fea.fea_mesh_set_scatter_stages(m.h, 5)


@pytest.mark.parametrize("kind,n", [("p1_kappa", 10), ("p2_diffmass", 7)])
@pytest.mark.parametrize("prec", [0, 1])
def test_load_split_modes_bitwise_identical(torch_cuda, kind, n, prec):
    """Fused element kernel, matrix kernel then load kernel, load kernel on a
    concurrent stream: same bits."""
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=31)
    m = fea.Mesh(c["coords"], c["tets"])
    ref = None
    for mode in (0, 1, 2, 3, -1):
        fea.fea_mesh_set_load_split(m.h, mode)
        g = gpu_system(c, prec=prec, mesh=m)
        if ref is None:
            ref = g
            continue
        assert np.array_equal(g["vals"].view(np.uint64), ref["vals"].view(np.uint64)), mode
        assert np.array_equal(g["rhs"].view(np.uint64), ref["rhs"].view(np.uint64)), mode


@pytest.mark.parametrize("kind,n", [("p1_kappa", 6), ("p2_diffmass", 5)])
def test_sine_load_under_integer_translation(torch_cuda, kind, n):
    """The sine load's quadrature points and sines run in fixed point with a
    shift set by the coordinates' size.  Translating the mesh by integers
    changes the load exactly: sin(pi (x + 2)) = sin(pi x) and
    sin(pi (x + 1)) = -sin(pi x), so a shift by (2, -4, 6) leaves every load
    value unchanged and a shift by (1, 2, -3) flips its sign twice (odd x and
    z), i.e. leaves it unchanged too, while (1, 0, 0) and (-37, 64, 1000)
    negate it (the last with a fixed-point shift set by |z| ~ 1000).  The
    translated coordinates carry a few FP64 roundings, hence the tolerance.
    The matrix does not depend on the translation at all."""
    from common import vec_scaled_error
    c = case(kind, n, seed=41)
    ref = gpu_system(c)
    for shift, sign in (((2.0, -4.0, 6.0), 1.0), ((1.0, 2.0, -3.0), 1.0), ((1.0, 0.0, 0.0), -1.0),
                        ((-37.0, 64.0, 1000.0), -1.0)):
        ct = dict(c)
        ct["coords"] = c["coords"] + np.asarray(shift)[:, None]
        g = gpu_system(ct)
        assert vec_scaled_error(sign * ref["rhs"], g["rhs"]) <= 1e-12, shift
        assert row_scaled_error(ref["rp"], ref["vals"], g["vals"]) <= 1e-12, shift


@pytest.mark.parametrize("kind,n", [("p1_kappa", 5), ("p2_diffmass", 4)])
def test_sine_load_small_offset_mesh_matches_oracle(torch_cuda, kind, n):
    """A mesh of tiny elements away from the origin (the cube scaled by 1e-3
    and moved to x = 0.3 + ..., y = -0.7 + ..., z = 12.25 + ...), where the
    fixed-point shift of each coordinate is set by its offset (resolution
    2^-56 for z): matrix and load against the oracle."""
    c = case(kind, n, seed=43)
    c = dict(c)
    c["coords"] = c["coords"] * 1e-3 + np.array([0.3, -0.7, 12.25])[:, None]
    g = gpu_system(c)
    o = oracle_system(c)
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert vec_scaled_error(o["rhs"], g["rhs"]) <= TOL_FP64


def test_bounded_wait_times_out_and_context_survives(torch_cuda):
    """A device wait that never completes (the bulk-copy scatter's bounded
    mbarrier wait on a barrier nobody arrives at) gives up, the host reads
    FEA_ERR_TIMEOUT from the mesh's error word, the word is cleared, and the
    same context then assembles correctly."""
    from paper_1802_03433_gb300 import fea
    c = case("p2_diffmass", 4, seed=47)
    m = fea.Mesh(c["coords"], c["tets"])
    fea.fea_diag_wait_timeout(m.h, 1024)
    with pytest.raises(fea.FeaError) as ei:
        m.check()
    assert ei.value.status == 7  # FEA_ERR_TIMEOUT
    m.check()  # cleared
    g = gpu_system(c, mesh=m)
    o = oracle_system(c)
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    with pytest.raises(fea.FeaError):
        fea.fea_diag_wait_timeout(m.h, 0)


@pytest.mark.parametrize("log2_scale", [-1000, -60, 60, 1000])
@pytest.mark.parametrize("kind", ["p2_poisson", "p2_diffmass"])
def test_p2_entries_across_coefficient_scales(torch_cuda, kind, log2_scale):
    """The FP64 P2 entries are integer sums on one fixed-point scale set by
    the element's largest Gram or mass term.  kappa scaled by 2^k moves that
    scale through its range: 2^1000 puts the Gram terms near its top, 2^-1000
    (Poisson) below its bottom, where the FMA chains take over.  Against the
    oracle; without a mass term the values must also scale exactly, bitwise
    2^k times the unscaled ones (k = -1000 excepted: there the FMA chains may
    meet subnormal cancellations)."""
    c = case(kind, 4, seed=11)
    base = gpu_system(c)
    cs = dict(c)
    cs["kappa"] = np.ldexp(c["kappa"], log2_scale)
    g = gpu_system(cs)
    o = oracle_system(cs)
    assert row_scaled_error(o["rp"], o["vals"], g["vals"]) <= TOL_FP64
    assert np.array_equal(g["rhs"].view(np.uint64), base["rhs"].view(np.uint64))
    if kind == "p2_poisson" and log2_scale != -1000:
        scaled = np.ldexp(base["vals"], log2_scale)
        assert np.array_equal(g["vals"].view(np.uint64), scaled.view(np.uint64))


def test_p2_nonfinite_coefficient_propagates(torch_cuda):
    """A NaN kappa on one element (outside the fixed-point range, so its
    entries take the FMA chains) gives NaN in exactly the CSR entries that
    element touches and finite values everywhere else, as plain FP64
    arithmetic would."""
    c = dict(case("p2_poisson", 4, seed=12))
    kap = c["kappa"].copy()
    kap[7] = np.nan
    c["kappa"] = kap
    g = gpu_system(c)
    edof, _ = oracle.dof_table(2, c["coords"].shape[1], c["tets"])
    d = set(int(x) for x in edof[:, 7])
    rp, ci = g["rp"], g["ci"]
    expect = np.zeros(len(ci), dtype=bool)
    for r in d:
        for p in range(rp[r], rp[r + 1]):
            expect[p] = int(ci[p]) in d
    assert np.array_equal(np.isnan(g["vals"]), expect)
    assert np.isfinite(g["rhs"]).all()
