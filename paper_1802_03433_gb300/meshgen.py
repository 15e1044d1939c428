"""Seeded synthetic inputs: perturbed Kuhn cube meshes and per-element coefficients.

This module is the one piece shared by the oracle-based tests and the CUDA
path's callers.  It produces *inputs* only: node coordinates, tetrahedron
connectivity and random fields.  It holds none of the assembly arithmetic (no
Jacobians, no quadrature, no basis functions, no sparsity logic).

Mesh recipe (the paper states the generalized Helmholtz problem of Sec. 4.1
on a mesh given as coordinates plus global node indices per element, but no
3-D mesh; these conventions are ours):

* the unit cube [0,1]^3 is cut into n^3 cubes of side h = 1/n;
* node id = i + (n+1) j + (n+1)^2 k, x fastest;
* every cube is split into the 6 Kuhn (Freudenthal) tetrahedra that share
  the cube diagonal (0,0,0)->(1,1,1): for each axis permutation p of
  (x, y, z), taken in lexicographic order, v0 = the cube's low corner and
  v_m = v_{m-1} + unit step along axis p[m-1];
* the split of an odd permutation is negatively oriented, so its v1 and v2
  are swapped (orientation is decided by permutation parity alone);
* element id = 6 * (cube id) + permutation index, cube id = i + n j + n^2 k;
* interior nodes move by independent uniform draws in [-0.2h, 0.2h] per
  coordinate; boundary nodes stay put so the domain volume stays exactly 1.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64) in a
fixed draw order: perturbation (N, 3) first, then the coefficient fields,
then the adjoint probe vectors.
"""
from __future__ import annotations

import numpy as np

# Axis permutations in lexicographic order and their parity (1 = odd).
_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
_ODD = (0, 1, 1, 0, 0, 1)


def cube_counts(n: int) -> dict:
    """Closed-form sizes of the n^3 Kuhn mesh (used as test expectations)."""
    return {
        "nodes": (n + 1) ** 3,
        "elems": 6 * n ** 3,
        "edges": 7 * n ** 3 + 9 * n ** 2 + 3 * n,
        "p1_nnz": 15 * n ** 3 + 21 * n ** 2 + 9 * n + 1,
        "p2_nnz": 230 * n ** 3 + 138 * n ** 2 + 24 * n + 1,
    }


def kuhn_tets(n: int) -> np.ndarray:
    """Connectivity of the n^3 Kuhn mesh, int32 SoA of shape (4, 6 n^3)."""
    m = n + 1
    step = np.array([1, m, m * m], dtype=np.int64)
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # cube id = i + n j + n^2 k  -> order with i fastest
    corner = (i + m * j + m * m * k).transpose(2, 1, 0).reshape(-1).astype(np.int64)
    tets = np.empty((4, corner.size, 6), dtype=np.int64)
    for t, (perm, odd) in enumerate(zip(_PERMS, _ODD)):
        v0 = corner
        v1 = v0 + step[perm[0]]
        v2 = v1 + step[perm[1]]
        v3 = v2 + step[perm[2]]
        if odd:
            v1, v2 = v2, v1
        tets[0, :, t], tets[1, :, t], tets[2, :, t], tets[3, :, t] = v0, v1, v2, v3
    return np.ascontiguousarray(tets.reshape(4, -1).astype(np.int32))


def make_cube(n: int, perturb: float = 0.2, seed: int = 0):
    """Perturbed Kuhn cube mesh.

    Returns (coords, tets, rng): coords float64 (3, N) SoA, tets int32 (4, E)
    SoA, and the generator positioned after the perturbation draw so callers
    can continue the documented draw order.
    """
    m = n + 1
    h = 1.0 / n
    g = np.arange(m, dtype=np.float64) * h
    # node id = i + m j + m^2 k, x fastest
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)]).copy()
    rng = np.random.default_rng(seed)
    d = rng.uniform(-perturb * h, perturb * h, size=(m ** 3, 3))
    idx = np.arange(m)
    bi = (idx == 0) | (idx == n)
    kk, jj, ii = np.meshgrid(bi, bi, bi, indexing="ij")
    boundary = (ii | jj | kk).reshape(-1)
    if perturb != 0.0:
        coords += np.where(boundary[:, None], 0.0, d).T
    return np.ascontiguousarray(coords), kuhn_tets(n), rng


def lognormal(rng, size):
    """kappa = exp(N(0, 1)) per element."""
    return np.exp(rng.standard_normal(size))


def lame(rng, n_elems):
    """Lame parameters (lambda, mu) per element, each uniform in [0.5, 2]."""
    lm = rng.uniform(0.5, 2.0, size=(n_elems, 2))
    return np.ascontiguousarray(lm[:, 0]), np.ascontiguousarray(lm[:, 1])


# --------------------------------------------------------------------------
# The five workloads.  Each returns a dict of numpy arrays plus metadata.
# --------------------------------------------------------------------------
SIN_AMP = 3.0 * np.pi ** 2  # f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)


def poisson_p1(n: int = 8, seed: int = 0) -> dict:
    """Plain P1 Poisson -div(grad u) = f on n^3 cubes (kappa = 1), 4-pt rule."""
    coords, tets, _ = make_cube(n, 0.2, seed)
    return dict(name=f"p1_poisson_{n}", n=n, order=1, coords=coords, tets=tets,
                kappa=None, kappa_const=1.0, mass=0.0, f_kind="sinprod",
                f_amp=SIN_AMP, npts=4)


def diffusion_mass_p2(n: int = 64, seed: int = 0) -> dict:
    """P2 -div(kappa grad u) + u = f, kappa log-normal per element, 11-pt rule."""
    coords, tets, rng = make_cube(n, 0.2, seed)
    kappa = lognormal(rng, tets.shape[1])
    return dict(name=f"p2_diffmass_{n}", n=n, order=2, coords=coords, tets=tets,
                kappa=kappa, kappa_const=1.0, mass=1.0, f_kind="sinprod",
                f_amp=SIN_AMP, npts=11)


def elasticity_p1(n: int = 128, seed: int = 0) -> dict:
    """P1 linear elasticity, Lame uniform in [0.5, 2] per element, body force (0,0,-1)."""
    coords, tets, rng = make_cube(n, 0.2, seed)
    lam, mu = lame(rng, tets.shape[1])
    return dict(name=f"p1_elast_{n}", n=n, order=1, coords=coords, tets=tets,
                lam=lam, mu=mu, body=(0.0, 0.0, -1.0), npts=4)


def adjoint_p1(n: int = 96, seed: int = 0) -> dict:
    """P1 kappa-diffusion with L = v^T K w + g^T f; v, w, g ~ N(0,1) per node."""
    coords, tets, rng = make_cube(n, 0.2, seed)
    kappa = lognormal(rng, tets.shape[1])
    nn = coords.shape[1]
    v = rng.standard_normal(nn)
    w = rng.standard_normal(nn)
    g = rng.standard_normal(nn)
    return dict(name=f"p1_adjoint_{n}", n=n, order=1, coords=coords, tets=tets,
                kappa=kappa, kappa_const=1.0, mass=0.0, f_kind="sinprod",
                f_amp=SIN_AMP, npts=4, v=v, w=w, g=g)


def batch_sides(n_meshes: int = 256, lo: int = 4, hi: int = 32, seed: int = 0):
    """Sides n_m ~ U{lo..hi} and element orders (even m: 1, odd m: 2) of the
    uneven batch, without building its meshes."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=n_meshes)
    return sides, np.where(np.arange(n_meshes) % 2 == 0, 1, 2)


def batch(n_meshes: int = 256, lo: int = 4, hi: int = 32, seed: int = 0) -> list:
    """Uneven batch: side n_m ~ U{lo..hi}; even m -> P1 Poisson, odd m -> P2.

    Mesh m is drawn from its own generator seeded with 1000 * seed + m + 1
    (perturbation, then log-normal kappa).
    """
    sides, _ = batch_sides(n_meshes, lo, hi, seed)
    out = []
    for m, n in enumerate(sides):
        n = int(n)
        coords, tets, r = make_cube(n, 0.2, 1000 * seed + m + 1)
        kappa = lognormal(r, tets.shape[1])
        order = 1 if m % 2 == 0 else 2
        out.append(dict(name=f"batch{m}_n{n}_p{order}", n=n, order=order,
                        coords=coords, tets=tets, kappa=kappa, kappa_const=1.0,
                        mass=0.0, f_kind="sinprod", f_amp=SIN_AMP,
                        npts=4 if order == 1 else 11))
    return out


# --------------------------------------------------------------------------
# 2-D: the unit square cut into n^2 squares, each split along its
# (i, j) -> (i + 1, j + 1) diagonal into two counter-clockwise triangles, so an
# interior node has 6 neighbours (the paper's 2-D P1 structure, Sec. 5).
# Node id = i + (n + 1) j; element id = 2 (i + n j) + t; interior nodes move
# by U[-0.2h, 0.2h] per coordinate.
def tri_square(n: int, perturb: float = 0.2, seed: int = 0):
    """(coords (2, N) float64, tris (3, 2 n^2) int32)."""
    m = n + 1
    h = 1.0 / n
    g = np.arange(m, dtype=np.float64) * h
    y, x = np.meshgrid(g, g, indexing="ij")
    coords = np.stack([x.reshape(-1), y.reshape(-1)]).copy()
    rng = np.random.default_rng(seed)
    d = rng.uniform(-perturb * h, perturb * h, size=(m * m, 2))
    idx = np.arange(m)
    bi = (idx == 0) | (idx == n)
    jj, ii = np.meshgrid(bi, bi, indexing="ij")
    boundary = (ii | jj).reshape(-1)
    if perturb != 0.0:
        coords += np.where(boundary[:, None], 0.0, d).T
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a = (i + m * j).reshape(-1)
    b, c, dd = a + 1, a + m, a + m + 1
    tris = np.empty((3, a.size, 2), dtype=np.int64)
    tris[:, :, 0] = np.stack([a, b, dd])
    tris[:, :, 1] = np.stack([a, dd, c])
    return np.ascontiguousarray(coords), np.ascontiguousarray(tris.reshape(3, -1).astype(np.int32))


def cube_boundary_dofs(coords, edof, n_dofs):
    """Dofs of a unit-cube mesh that lie on its boundary, from geometry only.
    edof: (nb, E) element -> scalar dof table (nb = 4 P1, 10 P2 with the
    local edge order (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)); a dof's position is
    its vertex, or the midpoint of its edge.  Returns (dofs int32 ascending,
    positions (3, n_dofs))."""
    edof = np.asarray(edof)
    pos = np.zeros((3, n_dofs))
    N = coords.shape[1]
    pos[:, :N] = coords
    if edof.shape[0] == 10:
        pairs = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
        for k, (a, b) in enumerate(pairs):
            pos[:, edof[4 + k]] = 0.5 * (coords[:, edof[a]] + coords[:, edof[b]])
    on = np.any((np.abs(pos) < 1e-12) | (np.abs(pos - 1.0) < 1e-12), axis=0)
    return np.nonzero(on)[0].astype(np.int32), pos
