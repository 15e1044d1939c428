"""Pins of the CPU oracle against facts fixed by the mathematics (no GPU).

Each test checks the oracle against something other than itself: exact
rational integrals (sympy, physical-coordinate basis), the cotangent formula,
the textbook Voigt B^T D B elasticity matrix, quadrature exactness, closed-form
mesh counts, invariants (row sums, volume, symmetry), patch tests, brute force
on tiny meshes, central finite differences, and the paper's printed 2-D row
width (Sec. 5, MAX_NZ = 7).
"""
import itertools
import os
from math import factorial

import numpy as np
import pytest

import oracle
from paper_1802_03433_gb300 import meshgen as mg

sp = pytest.importorskip("sympy")
import exact  # noqa: E402  (tests/exact.py, needs sympy)

REF = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)


def rand_tets(n, seed=0):
    """Random well-shaped tets (positively oriented)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        X = REF + rng.uniform(-0.25, 0.25, size=(4, 3))
        X = X * rng.uniform(0.5, 2.0) + rng.uniform(-1, 1, size=3)
        if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1)) > 0.05:
            out.append(X)
    return np.array(out)


def volume(X):
    return abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1))) / 6.0


# ------------------------------------------------------------------ rules
@pytest.mark.parametrize("npts,degree", [(1, 1), (4, 2), (11, 4)])
def test_rule_exact_for_monomials(npts, degree):
    # int_T lambda^alpha / |T| = 3! prod(alpha_i!) / (|alpha| + 3)!
    bary, w = oracle.rule(npts)
    assert abs(w.sum() - 1.0) < 1e-15
    for alpha in itertools.product(range(degree + 1), repeat=4):
        if sum(alpha) > degree:
            continue
        exact_v = 6.0 * np.prod([factorial(a) for a in alpha]) / factorial(sum(alpha) + 3)
        q = np.sum(w * np.prod(bary ** np.array(alpha), axis=1))
        assert abs(q - exact_v) < 1e-15, (npts, alpha)


def test_rule_not_exact_beyond_degree():
    # the 4-point rule is degree 2, not 3: lambda_0^3 is off
    bary, w = oracle.rule(4)
    exact_v = 6.0 * 6 / factorial(6)
    assert abs(np.sum(w * bary[:, 0] ** 3) - exact_v) > 1e-4


# ------------------------------------------------------------------ P1
def test_p1_reference_stiffness_closed_form():
    K, _, det = oracle.local(REF[None], order=1)
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    assert abs(det[0] - 1.0) < 1e-15
    np.testing.assert_allclose(K[0], ref, atol=1e-15)


def _cot_stiffness(X):
    # K_ij = -(1/6) l_kl cot(theta_kl), kl = edge opposite to ij, theta_kl its
    # dihedral angle; the diagonal makes rows sum to zero.  No J^{-1} used.
    K = np.zeros((4, 4))
    for i, j in itertools.combinations(range(4), 2):
        k, l = [m for m in range(4) if m not in (i, j)]
        e = X[l] - X[k]
        ln = np.linalg.norm(e)
        u = e / ln

        def perp(p):
            d = X[p] - X[k]
            return d - np.dot(d, u) * u

        a, b = perp(i), perp(j)
        cos_t = np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b))
        sin_t = np.linalg.norm(np.cross(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b))
        K[i, j] = K[j, i] = -ln * (cos_t / sin_t) / 6.0
    for i in range(4):
        K[i, i] = -K[i].sum()
    return K


def test_p1_stiffness_cotangent_formula():
    X = rand_tets(20, seed=1)
    K, _, _ = oracle.local(X, order=1)
    for e in range(len(X)):
        np.testing.assert_allclose(K[e], _cot_stiffness(X[e]), rtol=1e-12, atol=1e-13)


def test_p1_mass_closed_form():
    X = rand_tets(10, seed=2)
    K, _, _ = oracle.local(X, order=1, kappa=np.zeros(10), mass=1.0)
    for e in range(len(X)):
        M = volume(X[e]) / 20.0 * (np.ones((4, 4)) + np.eye(4))
        np.testing.assert_allclose(K[e], M, rtol=1e-13)
        assert abs(K[e].sum() - volume(X[e])) < 1e-14


def test_kappa_scales_stiffness():
    X = rand_tets(4, seed=3)
    kap = np.array([0.3, 1.0, 2.5, 7.0])
    K1, _, _ = oracle.local(X, order=2, kappa=np.ones(4))
    Kk, _, _ = oracle.local(X, order=2, kappa=kap)
    np.testing.assert_allclose(Kk, K1 * kap[:, None, None], rtol=1e-13)


# ------------------------------------------------------------------ P2 (exact rationals)
def _tofloat(M):
    return np.array(M.tolist(), dtype=float)


def test_p2_reference_mass_and_stiffness_exact():
    S, M = exact.ref_matrices(2)
    # known rational structure of the P2 mass on the reference tet, x 2520
    M2520 = np.array((M * 2520).tolist(), dtype=float)
    assert M2520[0, 0] == 6 and M2520[0, 1] == 1
    assert M2520[0, 4] == -4 and M2520[0, 7] == -6        # edge (0,1) holds v0, edge (1,2) not
    assert M2520[4, 4] == 32 and M2520[4, 5] == 16 and M2520[4, 9] == 8
    S30 = np.array((S * 30).tolist(), dtype=float)
    np.testing.assert_array_equal(S30[0], [9, 1, 1, 1, -6, -6, -6, 2, 2, 2])
    Ko, _, _ = oracle.local(REF[None], order=2)
    np.testing.assert_allclose(Ko[0], _tofloat(S), atol=1e-15)
    Mo, _, _ = oracle.local(REF[None], order=2, kappa=np.zeros(1), mass=1.0)
    np.testing.assert_allclose(Mo[0], _tofloat(M), atol=1e-16)


def test_p2_general_tet_exact():
    # a rational non-reference tet; exact diffusion + mass vs the oracle
    V = ((0, 0, 0), (sp.Rational(3, 2), sp.Rational(1, 5), 0), (sp.Rational(1, 3), 2, sp.Rational(1, 7)),
         (sp.Rational(1, 2), sp.Rational(1, 4), sp.Rational(5, 4)))
    Kx = exact.local_exact(V, order=2, kappa=sp.Rational(3, 2), mass=sp.Rational(2, 3))
    X = np.array([[float(c) for c in v] for v in V])
    Ko, _, _ = oracle.local(X[None], order=2, kappa=np.array([1.5]), mass=2.0 / 3.0)
    np.testing.assert_allclose(Ko[0], _tofloat(Kx), rtol=1e-13, atol=1e-14)


def test_p1_general_tet_exact():
    V = ((0, 0, 0), (1, sp.Rational(1, 3), 0), (sp.Rational(-1, 4), 1, sp.Rational(1, 2)),
         (sp.Rational(1, 5), sp.Rational(1, 6), sp.Rational(4, 3)))
    Kx = exact.local_exact(V, order=1, kappa=2, mass=sp.Rational(1, 3))
    X = np.array([[float(c) for c in v] for v in V])
    Ko, _, _ = oracle.local(X[None], order=1, kappa=np.array([2.0]), mass=1.0 / 3.0)
    np.testing.assert_allclose(Ko[0], _tofloat(Kx), rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------ elasticity
def _voigt(X, lam, mu):
    # textbook |T| B^T D B with Voigt strain (xx, yy, zz, 2yz, 2xz, 2xy)
    A = np.hstack([np.ones((4, 1)), X])            # lambda_a = row a of inv(A)^T [1 x y z]
    G = np.linalg.inv(A)[1:, :].T                   # G[a] = grad lambda_a
    B = np.zeros((6, 12))
    for a in range(4):
        gx, gy, gz = G[a]
        B[:, 3 * a:3 * a + 3] = [[gx, 0, 0], [0, gy, 0], [0, 0, gz], [0, gz, gy], [gz, 0, gx], [gy, gx, 0]]
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return volume(X) * B.T @ D @ B


def test_elasticity_matches_voigt_btdb():
    X = rand_tets(10, seed=4)
    lam = np.linspace(0.5, 2.0, 10)
    mu = np.linspace(2.0, 0.5, 10)
    K, _, _ = oracle.local(X, order=1, kind="elasticity", lam=lam, mu=mu)
    for e in range(10):
        np.testing.assert_allclose(K[e], _voigt(X[e], lam[e], mu[e]), rtol=1e-12, atol=1e-13)


def test_elasticity_p1_exact_sympy():
    V = ((0, 0, 0), (1, 0, sp.Rational(1, 5)), (0, 1, 0), (sp.Rational(1, 3), 0, 1))
    Kx = exact.local_exact(V, order=1, kind="elasticity", lam=sp.Rational(3, 4), mu=sp.Rational(5, 4))
    X = np.array([[float(c) for c in v] for v in V])
    Ko, _, _ = oracle.local(X[None], order=1, kind="elasticity", lam=np.array([0.75]), mu=np.array([1.25]))
    np.testing.assert_allclose(Ko[0], _tofloat(Kx), rtol=1e-13, atol=1e-15)


def test_elasticity_body_force_load():
    X = rand_tets(3, seed=5)
    for npts in (1, 4, 11):
        _, F, _ = oracle.local(X, order=1, kind="elasticity", f_kind="const",
                               f_param=(0.0, 0.0, -1.0), npts=npts)
        for e in range(3):
            exp_ = np.tile([0.0, 0.0, -volume(X[e]) / 4.0], 4)
            np.testing.assert_allclose(F[e], exp_, rtol=1e-14, atol=1e-18)


# ------------------------------------------------------------------ load vectors
def test_p2_load_constant_f_integrates_basis():
    # int phi_vertex = -|T|/20, int phi_edge = |T|/5 (exact for the 4- and 11-point rules)
    X = rand_tets(3, seed=6)
    for npts in (4, 11):
        _, F, _ = oracle.local(X, order=2, f_kind="const", f_param=(1.0,), npts=npts)
        for e in range(3):
            v = volume(X[e])
            np.testing.assert_allclose(F[e], [-v / 20] * 4 + [v / 5] * 6, rtol=1e-13)


def test_sin_load_against_independent_sum():
    coords, tets, _ = mg.make_cube(3, 0.2, 7)
    bary, w = oracle.rule(4)
    X = coords.T[tets.T]                     # (E, 4, 3)
    vol = np.array([volume(Xe) for Xe in X])
    xq = np.einsum("qv,evc->eqc", bary, X)
    f = 3 * np.pi ** 2 * np.prod(np.sin(np.pi * xq), axis=2)
    want = np.sum(vol[:, None] * w[None] * f)
    rp, ci = oracle.pattern(coords.shape[1], tets)
    _, rhs, _ = oracle.assemble(coords, tets, 1, tets, rp, ci, npts=4)
    assert abs(rhs.sum() - want) < 1e-12 * abs(want)


def test_sin_load_converges_to_integral():
    # sum F -> int 3 pi^2 sin sin sin = 24/pi, error O(h^2)
    errs = []
    for n in (4, 8):
        coords, tets, _ = mg.make_cube(n, 0.0, 0)
        rp, ci = oracle.pattern(coords.shape[1], tets)
        _, rhs, _ = oracle.assemble(coords, tets, 1, tets, rp, ci, npts=4)
        errs.append(abs(rhs.sum() - 24 / np.pi))
    assert errs[1] < errs[0] / 3.0


# ------------------------------------------------------------------ assembled invariants
def _system(n, order, seed, kappa=True, mass=0.0, f_kind="sinprod", f_param=(3 * np.pi ** 2,),
            npts=None, perturb=0.2):
    coords, tets, rng = mg.make_cube(n, perturb, seed)
    E = tets.shape[1]
    kap = mg.lognormal(rng, E) if kappa else None
    edof, nd = oracle.dof_table(order, coords.shape[1], tets)
    rp, ci = oracle.pattern(nd, edof)
    npts = npts or (4 if order == 1 else 11)
    vals, rhs, bad = oracle.assemble(coords, tets, order, edof, rp, ci, mass=mass, kappa=kap,
                                     f_kind=f_kind, f_param=f_param, npts=npts)
    assert bad == 0
    return dict(coords=coords, tets=tets, edof=edof, nd=nd, rp=rp, ci=ci, vals=vals, rhs=rhs, kappa=kap)


def _dense(rp, ci, vals):
    n = rp.size - 1
    A = np.zeros((n, n))
    for r in range(n):
        A[r, ci[rp[r]:rp[r + 1]]] += vals[rp[r]:rp[r + 1]]
    return A


@pytest.mark.parametrize("order", [1, 2])
def test_stiffness_rows_sum_zero_and_symmetric(order):
    s = _system(3, order, seed=11)
    A = _dense(s["rp"], s["ci"], s["vals"])
    scale = np.abs(A).max(axis=1)
    assert np.all(np.abs(A.sum(axis=1)) <= 1e-13 * scale)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())


@pytest.mark.parametrize("order", [1, 2])
def test_diffusion_mass_total_is_volume(order):
    # 1^T A 1 = volume (=1) since the stiffness annihilates constants
    s = _system(3, order, seed=12, mass=1.0)
    assert abs(s["vals"].sum() - 1.0) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_constant_load_sums_to_volume(order):
    s = _system(2, order, seed=13, f_kind="const", f_param=(1.0,))
    assert abs(s["rhs"].sum() - 1.0) < 1e-13


def _dof_coords(s, order):
    c = s["coords"]
    if order == 1:
        return c
    N = c.shape[1]
    out = np.zeros((3, s["nd"]))
    out[:, :N] = c
    for k, (p, q) in enumerate(oracle_edges()):
        e = s["edof"][4 + k]
        out[:, e] = 0.5 * (c[:, s["tets"][p]] + c[:, s["tets"][q]])
    return out


def oracle_edges():
    return [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def _interior(s, order):
    xd = _dof_coords(s, order)
    tol = 1e-12
    return np.all((xd > tol) & (xd < 1 - tol), axis=0)


def test_p1_patch_test_linear_field():
    s = _system(4, 1, seed=14, kappa=False)
    A = _dense(s["rp"], s["ci"], s["vals"])
    c = s["coords"]
    u = 0.3 + 1.7 * c[0] - 0.4 * c[1] + 2.2 * c[2]
    r = A @ u
    inner = _interior(s, 1)
    assert inner.sum() == 27
    assert np.abs(r[inner]).max() < 1e-13


def test_p2_patch_test_quadratic_field():
    # K (x^2)_I = -2 int phi_i at interior dofs (kappa = 1); int phi_i = M 1
    s = _system(3, 2, seed=15, kappa=False)
    A = _dense(s["rp"], s["ci"], s["vals"])
    m = _system(3, 2, seed=15, kappa=False, mass=1.0)
    M = _dense(m["rp"], m["ci"], m["vals"]) - A
    xd = _dof_coords(s, 2)
    u = xd[0] ** 2
    inner = _interior(s, 2)
    r = A @ u + 2 * M.sum(axis=1)
    assert np.abs(r[inner]).max() < 1e-13


def test_elasticity_rigid_body_modes_all_rows():
    coords, tets, rng = mg.make_cube(2, 0.2, 16)
    lam, mu = mg.lame(rng, tets.shape[1])
    rp, ci = oracle.pattern(coords.shape[1], tets, ndpn=3)
    vals, _, _ = oracle.assemble(coords, tets, 1, tets, rp, ci, kind="elasticity", lam=lam, mu=mu,
                                 f_kind="const", f_param=(0, 0, -1), npts=4)
    A = _dense(rp, ci, vals)
    x, y, z = coords
    N = x.size
    modes = []
    for t in range(3):
        u = np.zeros((N, 3)); u[:, t] = 1; modes.append(u)
    for u in (np.stack([-y, x, 0 * x], 1), np.stack([0 * x, -z, y], 1), np.stack([z, 0 * x, -x], 1)):
        modes.append(u)
    for u in modes:
        assert np.abs(A @ u.reshape(-1)).max() < 1e-13 * np.abs(A).max()


def test_unperturbed_kuhn_stiffness_is_seven_point_stencil():
    n = 4
    h = 1.0 / n
    s = _system(n, 1, seed=0, kappa=False, perturb=0.0)
    m = n + 1
    A = _dense(s["rp"], s["ci"], s["vals"])
    for (i, j, k) in [(1, 1, 1), (2, 2, 2), (1, 3, 2)]:
        r = i + m * j + m * m * k
        row = A[r]
        assert abs(row[r] - 6 * h) < 1e-15
        for d in (1, m, m * m):
            assert abs(row[r + d] + h) < 1e-15 and abs(row[r - d] + h) < 1e-15
        others = np.delete(row, [r, r + 1, r - 1, r + m, r - m, r + m * m, r - m * m])
        assert np.abs(others).max() < 1e-15
        assert (np.abs(row) > 0).sum() >= 7
        assert s["rp"][r + 1] - s["rp"][r] == 15


# ------------------------------------------------------------------ pattern
@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_pattern_closed_form_counts(n):
    coords, tets, _ = mg.make_cube(n, 0.2, 0)
    cc = mg.cube_counts(n)
    rp, ci = oracle.pattern(coords.shape[1], tets)
    assert rp[-1] == cc["p1_nnz"]
    edof, ne = oracle.p2_dofs(coords.shape[1], tets)
    assert ne == cc["edges"]
    rp2, _ = oracle.pattern(coords.shape[1] + ne, edof)
    assert rp2[-1] == cc["p2_nnz"]
    rp3, _ = oracle.pattern(coords.shape[1], tets, ndpn=3)
    assert rp3[-1] == 9 * cc["p1_nnz"]
    if n >= 3:
        assert np.diff(rp).max() == 15 and np.diff(rp2).max() == 65 and np.diff(rp3).max() == 45


def test_pattern_brute_force_sets():
    coords, tets, _ = mg.make_cube(2, 0.2, 0)
    edof, ne = oracle.p2_dofs(coords.shape[1], tets)
    nd = coords.shape[1] + ne
    rp, ci = oracle.pattern(nd, edof)
    pairs = set()
    for e in range(tets.shape[1]):
        d = edof[:, e]
        pairs.update((int(a), int(b)) for a in d for b in d)
    got = {(r, int(c)) for r in range(nd) for c in ci[rp[r]:rp[r + 1]]}
    assert got == pairs
    for r in range(nd):
        assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0)


def test_p2_edge_numbering_lexicographic():
    coords, tets, _ = mg.make_cube(2, 0.2, 0)
    N = coords.shape[1]
    edof, ne = oracle.p2_dofs(N, tets)
    edges = sorted({tuple(sorted((int(tets[p, e]), int(tets[q, e])))) for e in range(tets.shape[1])
                    for p, q in oracle_edges()})
    for e in range(tets.shape[1]):
        for k, (p, q) in enumerate(oracle_edges()):
            key = tuple(sorted((int(tets[p, e]), int(tets[q, e]))))
            assert edof[4 + k, e] == N + edges.index(key)


def test_max_nz_2d_paper_example():
    # the paper's 2-D P1 example (Sec. 5): widest row = 7, on a structured
    # triangulation with every square cut along the same diagonal
    with open(os.path.join(os.path.dirname(__file__), "golden", "max_nz_2d.txt")) as f:
        want = int([l.split()[1] for l in f if l.startswith("max_nz")][0])
    n = 6
    m = n + 1
    tris = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = i + m * j, i + 1 + m * j, i + m * (j + 1), i + 1 + m * (j + 1)
            tris += [(a, b, d), (a, d, c)]
    t = np.array(tris, dtype=np.int32).T.copy()
    rp, _ = oracle.pattern(m * m, t)
    assert np.diff(rp).max() == want


# ------------------------------------------------------------------ brute force, one cube
@pytest.mark.parametrize("order", [1, 2])
def test_one_cube_exact_assembly(order):
    coords, tets, _ = mg.make_cube(1, 0.0, 0)
    edof, nd = oracle.dof_table(order, 8, tets)
    rp, ci = oracle.pattern(nd, edof)
    assert rp[-1] == (46 if order == 1 else 393)
    vals, _, _ = oracle.assemble(coords, tets, order, edof, rp, ci, mass=1.0, kappa=np.full(6, 2.0),
                                 f_kind="zero")
    A = _dense(rp, ci, vals)
    Ax = np.zeros_like(A)
    for e in range(6):
        V = [tuple(int(round(c)) for c in coords[:, tets[v, e]]) for v in range(4)]
        Ke = _tofloat(exact.local_exact(V, order, kappa=2, mass=1))
        d = edof[:, e]
        Ax[np.ix_(d, d)] += Ke
    np.testing.assert_allclose(A, Ax, atol=1e-15)


# ------------------------------------------------------------------ gradient
def test_grad_kappa_is_element_form():
    # dL/dkappa_T = v^T K_T^{(kappa=1)} w exactly (L linear in kappa)
    s = _system(2, 1, seed=21)
    rng = np.random.default_rng(5)
    N = s["coords"].shape[1]
    v, w = rng.standard_normal(N), rng.standard_normal(N)
    rp, ci = s["rp"], s["ci"]
    rows = np.repeat(np.arange(N), np.diff(rp))
    gV = v[rows] * w[ci]
    gk, _ = oracle.assemble_grad(s["coords"], s["tets"], 1, s["edof"], rp, ci, gV, None,
                                 kappa=s["kappa"])
    X = s["coords"].T[s["tets"].T]
    K1, _, _ = oracle.local(X, order=1, kappa=np.ones(len(X)))
    for e in range(len(X)):
        d = s["tets"][:, e]
        assert abs(gk[e] - v[d] @ K1[e] @ w[d]) < 1e-13 * (1 + abs(gk[e]))


@pytest.mark.parametrize("order", [1, 2])
def test_grad_matches_central_differences(order):
    s = _system(2, order, seed=22, mass=0.5)
    rng = np.random.default_rng(6)
    nd = s["nd"]
    v, w, g = rng.standard_normal(nd), rng.standard_normal(nd), rng.standard_normal(nd)
    rp, ci = s["rp"], s["ci"]
    rows = np.repeat(np.arange(nd), np.diff(rp))
    gV = v[rows] * w[ci]
    npts = 4 if order == 1 else 11
    kw = dict(mass=0.5, npts=npts)

    def L(coords, kappa):
        vals, rhs, _ = oracle.assemble(coords, s["tets"], order, s["edof"], rp, ci, kappa=kappa, **kw)
        return gV @ vals + g @ rhs

    gk, gx = oracle.assemble_grad(s["coords"], s["tets"], order, s["edof"], rp, ci, gV, g,
                                  kappa=s["kappa"], **kw)
    h = 1e-6
    for e in rng.choice(s["tets"].shape[1], 4, replace=False):
        kp, km = s["kappa"].copy(), s["kappa"].copy()
        kp[e] += h
        km[e] -= h
        fd = (L(s["coords"], kp) - L(s["coords"], km)) / (2 * h)
        assert abs(fd - gk[e]) < 1e-6 * max(1.0, abs(gk[e]))
    N = s["coords"].shape[1]
    for node in rng.choice(N, 4, replace=False):
        for c in range(3):
            cp, cm = s["coords"].copy(), s["coords"].copy()
            cp[c, node] += h
            cm[c, node] -= h
            fd = (L(cp, s["kappa"]) - L(cm, s["kappa"])) / (2 * h)
            assert abs(fd - gx[c, node]) < 1e-5 * max(1.0, abs(gx[c, node]))


@pytest.mark.parametrize("order,kind", [(1, "diffusion"), (2, "diffusion"), (1, "elasticity")])
def test_rows_routine_matches_full_assembly(order, kind):
    # the brute-force row assembly used for full-size sampled checks agrees
    # with the pinned full assembly, entry by entry, pattern included
    coords, tets, rng = mg.make_cube(3, 0.2, 31)
    E = tets.shape[1]
    edof, nsd = oracle.dof_table(order, coords.shape[1], tets)
    ndpn = 3 if kind == "elasticity" else 1
    rp, ci = oracle.pattern(nsd, edof, ndpn=ndpn)
    if kind == "elasticity":
        lam, mu = mg.lame(rng, E)
        kw = dict(kind="elasticity", lam=lam, mu=mu, f_kind="const", f_param=(0, 0, -1), npts=4)
    else:
        kw = dict(mass=0.7, kappa=mg.lognormal(rng, E), npts=11 if order == 2 else 4)
    vals, rhs, _ = oracle.assemble(coords, tets, order, edof, rp, ci, **kw)
    rows = np.arange(0, rp.size - 1, 7)
    ref, rr = oracle.rows(coords, tets, order, edof, rows, **kw)
    for r in rows:
        cols, v = ref[int(r)]
        np.testing.assert_array_equal(cols, ci[rp[r]:rp[r + 1]])
        np.testing.assert_allclose(v, vals[rp[r]:rp[r + 1]], rtol=0, atol=1e-15 * max(1, np.abs(v).max()))
        assert abs(rr[int(r)] - rhs[r]) <= 1e-15 * max(1.0, abs(rhs[r]))
