"""Pins of the oracle's 2-D P1 triangle assembly: the paper's own worked
example (Sec. 4.1-4.2: sigma = [[1, -x-y], [x+y, 1]], lambda = 1,
f = -2 (x^2 + y^2) + 36), checked against exact rational integrals, the 2-D
cotangent formula, rule exactness, invariants and the paper's MAX_NZ = 7."""
import itertools
from math import factorial

import numpy as np
import pytest

import oracle
from paper_1802_03433_gb300 import meshgen as mg

sp = pytest.importorskip("sympy")
import exact  # noqa: E402

P = oracle.PAPER_2D


def rand_tris(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        X = np.array([[0, 0], [1, 0], [0, 1]], float) + rng.uniform(-0.3, 0.3, (3, 2))
        X = X * rng.uniform(0.5, 2) + rng.uniform(-1, 1, 2)
        if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0]], 1)) > 0.05:
            out.append(X)
    return np.array(out)


@pytest.mark.parametrize("npts,degree", [(1, 1), (3, 2), (6, 4)])
def test_tri_rules_exact(npts, degree):
    # int_T lambda^alpha / |T| = 2 prod(alpha_i!) / (|alpha| + 2)!
    b, w = oracle.tri_rule(npts)
    for al in itertools.product(range(degree + 1), repeat=3):
        if sum(al) > degree:
            continue
        ex = 2.0 * np.prod([factorial(a) for a in al]) / factorial(sum(al) + 2)
        assert abs(np.sum(w * np.prod(b ** np.array(al), axis=1)) - ex) < 1e-15


def test_identity_sigma_is_2d_cotangent_formula():
    # K_ij = -cot(theta_k) / 2, k the vertex opposite edge ij; mass |T|(1+delta)/12
    X = rand_tris(12, 1)
    K, _, _ = oracle.local_tri(X, S0=(1, 0, 0, 1), Sx=(0,) * 4, Sy=(0,) * 4, lam=0.0)
    M, _, _ = oracle.local_tri(X, S0=(0,) * 4, Sx=(0,) * 4, Sy=(0,) * 4, lam=1.0)
    for e, Xe in enumerate(X):
        area = abs(np.linalg.det(np.stack([Xe[1] - Xe[0], Xe[2] - Xe[0]], 1))) / 2
        Kc = np.zeros((3, 3))
        for i, j in itertools.combinations(range(3), 2):
            k = 3 - i - j
            u, v = Xe[i] - Xe[k], Xe[j] - Xe[k]
            Kc[i, j] = Kc[j, i] = -0.5 * np.dot(u, v) / abs(u[0] * v[1] - u[1] * v[0])
        np.fill_diagonal(Kc, -Kc.sum(1))
        np.testing.assert_allclose(K[e], Kc, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(M[e], area / 12 * (np.ones((3, 3)) + np.eye(3)), rtol=1e-13)


def test_paper_form_exact_on_rational_triangle():
    V = ((sp.Rational(1, 3), 0), (2, sp.Rational(1, 4)), (sp.Rational(1, 2), sp.Rational(7, 5)))
    Kx, Fx = exact.local_exact_tri(V, P["S0"], P["Sx"], P["Sy"], P["lam"], P["f"])
    X = np.array([[float(c) for c in v] for v in V])
    K, F, _ = oracle.local_tri(X[None], npts=6)
    np.testing.assert_allclose(K[0], np.array(Kx.tolist(), float), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(F[0], np.array([float(v) for v in Fx]), rtol=1e-13)
    assert np.abs(K[0] - K[0].T).max() > 1e-3  # the paper's sigma is not symmetric


def test_paper_problem_invariants():
    coords, tris = mg.tri_square(6, 0.2, 3)
    rp, ci = oracle.pattern(coords.shape[1], tris)
    assert np.diff(rp).max() == 7  # the paper's MAX_NZ (Sec. 5)
    v, r, bad = oracle.assemble_tri(coords, tris, rp, ci, lam=0.0)
    assert bad == 0
    N = coords.shape[1]
    A = np.zeros((N, N))
    for i in range(N):
        A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    assert np.abs(A.sum(1)).max() < 1e-12 and np.abs(A.sum(0)).max() < 1e-12  # rows and columns annihilate constants
    assert abs(r.sum() - (36 - 4 / 3)) < 1e-12  # int over the unit square of f, exact for the 3- and 6-point rules
    v1, _, _ = oracle.assemble_tri(coords, tris, rp, ci, lam=1.0)
    assert abs((v1 - v).sum() - 1.0) < 1e-13  # the mass part sums to the area


def test_linear_patch_with_constant_sigma():
    coords, tris = mg.tri_square(5, 0.2, 4)
    rp, ci = oracle.pattern(coords.shape[1], tris)
    v, _, _ = oracle.assemble_tri(coords, tris, rp, ci, S0=(2.0, 0.5, -0.3, 1.5), Sx=(0,) * 4, Sy=(0,) * 4, lam=0.0)
    N = coords.shape[1]
    u = 0.4 + 1.3 * coords[0] - 0.7 * coords[1]
    Au = np.zeros(N)
    for i in range(N):
        Au[i] = v[rp[i]:rp[i + 1]] @ u[ci[rp[i]:rp[i + 1]]]
    inner = np.all((coords > 1e-12) & (coords < 1 - 1e-12), axis=0)
    assert np.abs(Au[inner]).max() < 1e-13
