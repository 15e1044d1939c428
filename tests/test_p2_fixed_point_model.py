"""A bit-exact host model of the FP64 P2 local entries of the element
kernels: exact 64-bit fixed-point sums (element.cuh, p2_stiff_fx).

Over an affine tet the P2 stiffness is K_ab = kappa |T| / 20 sum n^ab_ij
(grad l_i . grad l_j) with integer reference-tensor coefficients n, and the
mass is |T| / 420 m_ab with integer m.  Here n and m are derived exactly
from the quadratic basis (phi = l_i (2 l_i - 1) at vertex i, 4 l_i l_j on
edge (i, j)) and pinned to the oracle's quadrature element matrices.  The
file then checks the bounds the fixed-point scale relies on (every n a
multiple of 4, sum |n| / 4 <= 24 per entry, |m| <= 32), and runs the
kernel's integer arithmetic on random inputs across the exponent range
against exact rational sums.  That arithmetic is the rounding of 4 G and t
to the scale 2^p (p = 1078 - E, E the largest biased exponent of 4 G and
32 t), the exact sums, and one rounding back.  The error must stay within
28 * 2^-55 of the largest input plus half an ulp of the entry.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np

import oracle

EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]  # local dofs 4..9


def _dphi(a):
    """d phi_a / d l_i as linear forms in l (coefficient lists), by i."""
    if a < 4:  # l_a (2 l_a - sum_k l_k)
        return [(a, [4 * (k == a) - 1 for k in range(4)])]
    i, j = EDGES[a - 4]  # 4 l_i l_j
    return [(i, [4 * (k == j) for k in range(4)]), (j, [4 * (k == i) for k in range(4)])]


def _int20(f, g):
    """20 / |T| times the integral of two linear forms in l over the tet."""
    return sum(f[k] * g[l] * (2 if k == l else 1) for k in range(4) for l in range(4))


def stiffness_terms(a, b):
    """{(i, j), i <= j: n} with K_ab = |T| / 20 sum n (grad l_i . grad l_j)."""
    t = {}
    for i, f in _dphi(a):
        for j, g in _dphi(b):
            key = (min(i, j), max(i, j))
            t[key] = t.get(key, 0) + _int20(f, g)
    return t


def _phi_poly(a):
    """phi_a as a homogeneous quadratic in l: {exponent tuple: coefficient}."""
    p = {}
    if a < 4:
        e = [0] * 4
        e[a] = 2
        p[tuple(e)] = p.get(tuple(e), 0) + 2
        for k in range(4):
            e = [0] * 4
            e[a] += 1
            e[k] += 1
            p[tuple(e)] = p.get(tuple(e), 0) - 1
    else:
        i, j = EDGES[a - 4]
        e = [0] * 4
        e[i] += 1
        e[j] += 1
        p[tuple(e)] = 4
    return p


def mass420(a, b):
    """420 / |T| times the integral of phi_a phi_b (the integral of l^alpha
    is |T| 3! prod alpha! / (|alpha| + 3)!)."""
    s = Fraction(0)
    for ea, ca in _phi_poly(a).items():
        for eb, cb in _phi_poly(b).items():
            al = [x + y for x, y in zip(ea, eb)]
            s += Fraction(ca * cb * 6 * math.prod(math.factorial(x) for x in al), math.factorial(sum(al) + 3))
    v = 420 * s
    assert v.denominator == 1
    return int(v)


UPPER = [(a, b) for a in range(10) for b in range(a, 10)]
TERMS = {ab: stiffness_terms(*ab) for ab in UPPER}
MASS = {ab: mass420(*ab) for ab in UPPER}


def test_reference_tensors_match_the_oracle():
    """K_ab from the derived coefficients equals the oracle's 11-point
    quadrature of grad phi_a . grad phi_b + phi_a phi_b on random tets."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        X = rng.standard_normal((4, 3))
        if abs(np.linalg.det(X[1:] - X[0])) < 0.1:
            continue
        if np.linalg.det(X[1:] - X[0]) < 0:
            X[[1, 2]] = X[[2, 1]]
        grad = np.linalg.inv(np.vstack([X.T, np.ones(4)]))[:, :3]  # rows: grad l_i
        vol = abs(np.linalg.det(X[1:] - X[0])) / 6
        K = np.zeros((10, 10))
        for (a, b), t in TERMS.items():
            v = vol / 20 * sum(n * grad[i] @ grad[j] for (i, j), n in t.items()) + vol / 420 * MASS[(a, b)]
            K[a, b] = K[b, a] = v
        Ke, _, _ = oracle.local(X[None], order=2, kind="diffusion", mass=1.0, npts=11)
        assert np.abs(K - Ke[0]).max() <= 1e-13 * np.abs(Ke[0]).max()


def test_fixed_point_bounds():
    """The scale's assumptions: coefficients multiples of 4, sum |n| / 4 <=
    24 in any entry, the seven mass values, |m| <= 32."""
    assert all(n % 4 == 0 for t in TERMS.values() for n in t.values())
    assert max(sum(abs(n) // 4 for n in t.values()) for t in TERMS.values()) == 24
    assert set(MASS.values()) == {6, 1, -4, -6, 32, 16, 8}
    assert max(abs(m) for m in MASS.values()) == 32


def _bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def _exp_bits(v):
    return (_bits(v) >> 52) & 0x7FF


def _to_fx(v, s):
    """round(v 2^(61 - s)) as the kernel's to_fx: shift of the significand,
    halves rounded away from zero."""
    b = _bits(v)
    e = (b >> 52) & 0x7FF
    m = (b & ((1 << 52) - 1)) | ((1 << 52) if e else 0)
    k = e - 1014 - s
    mag = (m << min(k, 63)) if k >= 0 else (((m >> min(-k - 1, 62)) + 1) >> 1)
    return -mag if b >> 63 else mag


def _fx_to_double(F, p):
    """F 2^-p: one round-to-nearest-even conversion, then an exponent shift."""
    if F == 0:
        return 0.0
    d = float(F)
    return struct.unpack("<d", struct.pack("<Q", _bits(d) - (p << 52)))[0]


def _entries(G, t, mass):
    """The kernel's entries (upper order) and the scale's largest input M."""
    E = max(_exp_bits(G[i][j]) + 2 for i in range(4) for j in range(i, 4))
    if mass:
        E = max(E, _exp_bits(t) + 5)
    assert 64 <= E <= 2032
    Gf = {(i, j): _to_fx(G[i][j], E - 1019) for i in range(4) for j in range(i, 4)}
    tf = _to_fx(t, E - 1017) if mass else 0
    p = 1078 - E
    out = []
    for ab in UPPER:
        F = (MASS[ab] * tf if mass else 0) + sum((n // 4) * Gf[ij] for ij, n in TERMS[ab].items())
        assert abs(F) < 2 ** 61
        out.append(_fx_to_double(F, p))
    M = max(max(abs(4 * G[i][j]) for i in range(4) for j in range(i, 4)), 32 * abs(t) if mass else 0.0)
    return out, M


def test_fixed_point_entries_within_their_bound():
    random.seed(7)
    worst = 0.0
    for trial in range(400):
        sc = 2.0 ** random.randint(-900, 900)
        G = [[0.0] * 4 for _ in range(4)]
        for i in range(4):
            for j in range(i, 4):
                G[i][j] = random.choice([1, -1]) * random.random() * sc * 2.0 ** random.randint(-60, 0)
                if random.random() < 0.05:
                    G[i][j] = 0.0
        t = random.random() * sc * 2.0 ** random.randint(-40, 10)
        mass = trial % 3 != 0
        got, M = _entries(G, t, mass)
        for v, ab in zip(got, UPPER):
            exact = sum(Fraction(n) * Fraction(G[i][j]) for (i, j), n in TERMS[ab].items())
            if mass:
                exact += Fraction(MASS[ab]) * Fraction(t)
            bound = Fraction(28) * Fraction(2) ** -55 * Fraction(M) + Fraction(2) ** -53 * abs(Fraction(v))
            r = float(abs(Fraction(v) - exact) / bound)
            assert r <= 1.0, (trial, ab, r)
            worst = max(worst, r)
    assert worst > 0.0


def test_scaling_by_powers_of_two_is_exact():
    """Scaling every input by 2^k shifts E by k and leaves the integers
    unchanged, so the entries scale exactly (what the GPU test checks
    bitwise on whole meshes)."""
    random.seed(9)
    G = [[random.uniform(-1, 1) for _ in range(4)] for _ in range(4)]
    t = random.uniform(0, 1e-3)
    base, _ = _entries(G, t, True)
    for k in (-700, -61, 1, 59, 800):
        Gk = [[math.ldexp(x, k) for x in row] for row in G]
        got, _ = _entries(Gk, math.ldexp(t, k), True)
        assert got == [math.ldexp(v, k) for v in base]
