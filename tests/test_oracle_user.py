"""Pins of the oracle's user-coefficient path (point functions k(x) and f(x)
inside the integrals, the target of runtime-compiled kernels) against exact
rational integrals, special cases and invariants (no GPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_1802_03433_gb300 import meshgen as mg

sp = pytest.importorskip("sympy")
import exact  # noqa: E402

x, y, z = exact.x, exact.y, exact.z

# rational non-reference tets inside the positive octant
V2 = ((0, 0, 0), (sp.Rational(3, 2), sp.Rational(1, 5), 0), (sp.Rational(1, 3), 2, sp.Rational(1, 7)),
      (sp.Rational(1, 2), sp.Rational(1, 4), sp.Rational(5, 4)))
V1 = ((0, 0, 0), (1, sp.Rational(1, 3), 0), (sp.Rational(1, 4), 1, sp.Rational(1, 2)),
      (sp.Rational(1, 5), sp.Rational(1, 6), sp.Rational(4, 3)))


def _X(V):
    return np.array([[float(c) for c in v] for v in V])


def _tofloat(M):
    return np.array(M.tolist(), dtype=float)


def _load_exact(V, order, f):
    phi = exact.basis([[sp.Rational(c) for c in v] for v in V], order)
    return np.array([float(exact.integrate(V, f * p)) for p in phi])


def test_p2_linear_kappa_11pt_is_exact():
    # degree(k) + 2 (order - 1) = 3 <= 4: the 11-point rule is exact
    kx = 1 + x + 2 * y - z
    Kx = exact.local_exact(V2, order=2, kappa=kx, mass=sp.Rational(2, 3))
    Ko, _ = oracle.local_user(_X(V2)[None], order=2, mass=2.0 / 3.0, kfn=lambda a, b, c: 1 + a + 2 * b - c,
                              npts=11)
    np.testing.assert_allclose(Ko[0], _tofloat(Kx), rtol=1e-13, atol=1e-14)


def test_p1_quadratic_kappa_4pt_is_exact():
    kx = 2 + x * x + y * z
    Kx = exact.local_exact(V1, order=1, kappa=kx)
    Ko, _ = oracle.local_user(_X(V1)[None], order=1, kfn=lambda a, b, c: 2 + a * a + b * c, npts=4)
    np.testing.assert_allclose(Ko[0], _tofloat(Kx), rtol=1e-13, atol=1e-15)


def test_p1_linear_kappa_one_point_is_exact():
    # int_T k = |T| k(centroid) for linear k
    kx = 3 - x + y + 2 * z
    Kx = exact.local_exact(V1, order=1, kappa=kx)
    Ko, _ = oracle.local_user(_X(V1)[None], order=1, kfn=lambda a, b, c: 3 - a + b + 2 * c, npts=1)
    np.testing.assert_allclose(Ko[0], _tofloat(Kx), rtol=1e-13, atol=1e-15)


def test_p2_quadratic_load_11pt_is_exact():
    fx = 1 + x * x - y * z + 3 * z
    _, Fo = oracle.local_user(_X(V2)[None], order=2, ffn=lambda a, b, c: 1 + a * a - b * c + 3 * c, npts=11)
    np.testing.assert_allclose(Fo[0], _load_exact(V2, 2, fx), rtol=1e-13, atol=1e-15)


def test_p1_quadratic_load_4pt_is_exact():
    # f phi_a has degree 3 > 2: the 4-point rule is not exact, the 11-point one is
    fx = x * y + z
    _, F4 = oracle.local_user(_X(V1)[None], order=1, ffn=lambda a, b, c: a * b + c, npts=4)
    _, F11 = oracle.local_user(_X(V1)[None], order=1, ffn=lambda a, b, c: a * b + c, npts=11)
    ex = _load_exact(V1, 1, fx)
    np.testing.assert_allclose(F11[0], ex, rtol=1e-13, atol=1e-15)
    assert np.abs(F4[0] - ex).max() > 1e-6


def test_no_functions_reduces_to_the_plain_form():
    c, t, rng = mg.make_cube(3, 0.2, 4)
    kap = mg.lognormal(rng, t.shape[1])
    for order in (1, 2):
        ed, nd = oracle.dof_table(order, c.shape[1], t)
        rp, ci = oracle.pattern(nd, ed)
        vu, ru, _ = oracle.assemble_user(c, t, order, ed, rp, ci, kappa=kap, mass=0.5)
        vp, _, _ = oracle.assemble(c, t, order, ed, rp, ci, kappa=kap, mass=0.5, f_kind=None, npts=11)
        np.testing.assert_allclose(vu, vp, rtol=0, atol=1e-14 * np.abs(vp).max())
        assert not ru.any()


def test_sin_load_reduces_to_the_builtin_load():
    c, t, _ = mg.make_cube(3, 0.2, 5)
    A = 3 * math.pi ** 2
    for order, npts in ((1, 4), (2, 11)):
        ed, nd = oracle.dof_table(order, c.shape[1], t)
        rp, ci = oracle.pattern(nd, ed)
        _, ru, _ = oracle.assemble_user(c, t, order, ed, rp, ci, npts=npts, ffn=lambda a, b, cc: A * math.sin(
            math.pi * a) * math.sin(math.pi * b) * math.sin(math.pi * cc))
        _, rb, _ = oracle.assemble(c, t, order, ed, rp, ci, f_kind="sinprod", f_param=(A,), npts=npts)
        np.testing.assert_allclose(ru, rb, rtol=0, atol=1e-14 * np.abs(rb).max())


@pytest.mark.parametrize("order", [1, 2])
def test_variable_kappa_invariants(order):
    # grad(sum phi) = 0: every stiffness row sums to zero for any k; the
    # mass sums to the domain volume; the load of f = 1 sums to the volume
    c, t, _ = mg.make_cube(3, 0.2, 6)
    ed, nd = oracle.dof_table(order, c.shape[1], t)
    rp, ci = oracle.pattern(nd, ed)
    k = lambda a, b, cc: 1.0 + 0.5 * math.sin(3 * a) * math.cos(2 * b) + cc * cc  # noqa: E731
    v, r, bad = oracle.assemble_user(c, t, order, ed, rp, ci, kfn=k, ffn=lambda a, b, cc: 1.0, npts=4)
    assert bad == 0
    rows = np.add.reduceat(v, rp[:-1]) if v.size else v
    assert np.abs(rows).max() < 1e-12 * np.abs(v).max()
    np.testing.assert_allclose(r.sum(), 1.0, rtol=1e-13)
    vm, _, _ = oracle.assemble_user(c, t, order, ed, rp, ci, kfn=k, mass=2.0, npts=4)
    np.testing.assert_allclose(vm.sum(), 2.0, rtol=1e-12)
    # symmetric for any k
    n = rp.size - 1
    import scipy.sparse as sps
    A = sps.csr_matrix((v, ci, rp), shape=(n, n))
    assert abs(A - A.T).max() <= 1e-15 * np.abs(v).max()
