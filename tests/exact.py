"""Exact rational element integrals with sympy, for pinning the oracle.

Independent of the oracle's arithmetic: the basis functions are built in
*physical* coordinates (barycentrics solved from the vertex matrix), their
gradients taken by symbolic differentiation, and every integral is done by
pulling the polynomial back to the reference tetrahedron and integrating
monomials with the closed form  int xi1^a xi2^b xi3^c = a! b! c! / (a+b+c+3)!.
No quadrature, no Jacobian inverse formula, no shared tables.
"""
from __future__ import annotations

from functools import lru_cache
from math import factorial

import sympy as sp

x, y, z = sp.symbols("x y z")
s1, s2, s3 = sp.symbols("s1 s2 s3")


def _ref_integral(poly_expr):
    p = sp.Poly(sp.expand(poly_expr), s1, s2, s3)
    tot = sp.Rational(0)
    for (a, b, c), coef in p.terms():
        tot += coef * sp.Rational(factorial(a) * factorial(b) * factorial(c), factorial(a + b + c + 3))
    return tot


def _bary(V):
    """Barycentric coordinate functions lambda_0..3 of the tet with vertices V."""
    M = sp.Matrix([[1, 1, 1, 1], [V[0][0], V[1][0], V[2][0], V[3][0]],
                   [V[0][1], V[1][1], V[2][1], V[3][1]], [V[0][2], V[1][2], V[2][2], V[3][2]]])
    lam = M.inv() * sp.Matrix([1, x, y, z])
    return [sp.expand(l) for l in lam]


EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def basis(V, order):
    L = _bary(V)
    if order == 1:
        return L
    return [sp.expand(L[a] * (2 * L[a] - 1)) for a in range(4)] + [
        sp.expand(4 * L[p] * L[q]) for p, q in EDGES]


def integrate(V, expr):
    """Exact integral of a polynomial in x, y, z over the tet with vertices V."""
    V = [[sp.Rational(c) for c in v] for v in V]
    J = sp.Matrix([[V[1][i] - V[0][i], V[2][i] - V[0][i], V[3][i] - V[0][i]] for i in range(3)])
    detJ = abs(J.det())
    sub = {x: V[0][0] + J[0, 0] * s1 + J[0, 1] * s2 + J[0, 2] * s3,
           y: V[0][1] + J[1, 0] * s1 + J[1, 1] * s2 + J[1, 2] * s3,
           z: V[0][2] + J[2, 0] * s1 + J[2, 1] * s2 + J[2, 2] * s3}
    return detJ * _ref_integral(sp.expand(expr).subs(sub))


def local_exact(V, order=1, kind="diffusion", kappa=1, mass=0, lam=1, mu=1):
    """Exact local matrix of -div(kappa grad u) + mass u, or of linear elasticity."""
    V = [[sp.Rational(c) for c in v] for v in V]
    phi = basis(V, order)
    grad = [[sp.diff(p, v) for v in (x, y, z)] for p in phi]
    nb = len(phi)
    if kind == "diffusion":
        K = sp.zeros(nb, nb)
        for a in range(nb):
            for b in range(a, nb):
                e = kappa * sum(grad[a][i] * grad[b][i] for i in range(3)) + mass * phi[a] * phi[b]
                K[a, b] = K[b, a] = integrate(V, e)
        return K
    K = sp.zeros(3 * nb, 3 * nb)
    for a in range(nb):
        for b in range(nb):
            dot = sum(grad[a][k] * grad[b][k] for k in range(3))
            for i in range(3):
                for j in range(3):
                    e = lam * grad[a][i] * grad[b][j] + mu * grad[a][j] * grad[b][i]
                    if i == j:
                        e += mu * dot
                    K[3 * a + i, 3 * b + j] = integrate(V, e)
    return K


@lru_cache(None)
def ref_matrices(order):
    """(stiffness, mass) on the reference tet (0,0,0),(1,0,0),(0,1,0),(0,0,1)."""
    V = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))
    return local_exact(V, order, kappa=1, mass=0), local_exact(V, order, kappa=0, mass=1)


# ---------------------------------------------------------------- 2-D
t1, t2 = sp.symbols("t1 t2")


def integrate_tri(V, expr):
    """Exact integral of a polynomial in x, y over the triangle V."""
    V = [[sp.Rational(c) for c in v] for v in V]
    J = sp.Matrix([[V[1][i] - V[0][i], V[2][i] - V[0][i]] for i in range(2)])
    sub = {x: V[0][0] + J[0, 0] * t1 + J[0, 1] * t2, y: V[0][1] + J[1, 0] * t1 + J[1, 1] * t2}
    p = sp.Poly(sp.expand(sp.expand(expr).subs(sub)), t1, t2)
    tot = sp.Rational(0)
    for (a, b), coef in p.terms():
        tot += coef * sp.Rational(factorial(a) * factorial(b), factorial(a + b + 2))
    return abs(J.det()) * tot


def local_exact_tri(V, S0, Sx, Sy, lam, f):
    """Exact 3x3 local matrix (row = test function) and load of
    (grad v, sigma grad u) + lam (v, u) = (v, f), sigma = S0 + x Sx + y Sy."""
    V = [[sp.Rational(c) for c in v] for v in V]
    M = sp.Matrix([[1, 1, 1], [V[0][0], V[1][0], V[2][0]], [V[0][1], V[1][1], V[2][1]]])
    L = [sp.expand(l) for l in M.inv() * sp.Matrix([1, x, y])]
    sig = sp.Matrix(2, 2, [sp.nsimplify(S0[k]) + x * sp.nsimplify(Sx[k]) + y * sp.nsimplify(Sy[k]) for k in range(4)])
    g = [sp.Matrix([sp.diff(l, x), sp.diff(l, y)]) for l in L]
    K = sp.zeros(3, 3)
    for a in range(3):
        for b in range(3):
            K[a, b] = integrate_tri(V, (g[a].T * sig * g[b])[0] + sp.nsimplify(lam) * L[a] * L[b])
    fx = sum(sp.nsimplify(c) * mono for c, mono in zip(f, [1, x, y, x * x, x * y, y * y]))
    F = [integrate_tri(V, fx * L[a]) for a in range(3)]
    return K, F
