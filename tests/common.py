"""Shared helpers for the parity tests: run a case on the GPU through the
C-ABI binding and on the CPU oracle, and compare."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1802_03433_gb300 import meshgen as mg

TOL_FP64 = 1e-12   # row-scaled, plain FP64 path
TOL_MIXED = 1e-5   # row-scaled, FP32 quadrature products


def row_scaled_error(rp, ref, got):
    """max over rows of max_j |got_ij - ref_ij| / max_k |ref_ik| (rows with a
    zero reference use scale 1)."""
    ref = np.asarray(ref)
    got = np.asarray(got)
    if ref.size == 0:
        return 0.0
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    scale = np.zeros(rp.size - 1)
    np.maximum.at(scale, rows, np.abs(ref))
    scale[scale == 0] = 1.0
    return float(np.max(np.abs(got - ref) / scale[rows]))


def vec_scaled_error(ref, got):
    ref = np.asarray(ref)
    got = np.asarray(got)
    if ref.size == 0:
        return 0.0
    s = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (s if s > 0 else 1.0))


def case(kind, n, seed=0, perturb=0.2):
    """Synthetic inputs of one workload family at side n (scaled-down configs)."""
    coords, tets, rng = mg.make_cube(n, perturb, seed)
    E = tets.shape[1]
    if kind == "p1_poisson":
        return dict(coords=coords, tets=tets, order=1, form="diffusion", mass=0.0, kappa=None,
                    f_kind="sinprod", f_param=(mg.SIN_AMP,), npts=4, ndpn=1)
    if kind == "p1_kappa":
        return dict(coords=coords, tets=tets, order=1, form="diffusion", mass=0.0,
                    kappa=mg.lognormal(rng, E), f_kind="sinprod", f_param=(mg.SIN_AMP,), npts=4, ndpn=1)
    if kind == "p2_diffmass":
        return dict(coords=coords, tets=tets, order=2, form="diffusion", mass=1.0,
                    kappa=mg.lognormal(rng, E), f_kind="sinprod", f_param=(mg.SIN_AMP,), npts=11, ndpn=1)
    if kind == "p2_poisson":
        return dict(coords=coords, tets=tets, order=2, form="diffusion", mass=0.0,
                    kappa=mg.lognormal(rng, E), f_kind="sinprod", f_param=(mg.SIN_AMP,), npts=11, ndpn=1)
    if kind == "elasticity":
        lam, mu = mg.lame(rng, E)
        return dict(coords=coords, tets=tets, order=1, form="elasticity", lam=lam, mu=mu,
                    f_kind="const", f_param=(0.0, 0.0, -1.0), npts=4, ndpn=3)
    raise KeyError(kind)


def oracle_system(c):
    edof, nsd = oracle.dof_table(c["order"], c["coords"].shape[1], c["tets"])
    rp, ci = oracle.pattern(nsd, edof, ndpn=c["ndpn"])
    kw = dict(f_kind=c["f_kind"], f_param=c["f_param"], npts=c["npts"])
    if c["form"] == "elasticity":
        vals, rhs, bad = oracle.assemble(c["coords"], c["tets"], 1, edof, rp, ci, kind="elasticity",
                                         lam=c["lam"], mu=c["mu"], **kw)
    else:
        vals, rhs, bad = oracle.assemble(c["coords"], c["tets"], c["order"], edof, rp, ci,
                                         mass=c["mass"], kappa=c["kappa"], **kw)
    return dict(edof=edof, rp=rp, ci=ci, vals=vals, rhs=rhs, bad=bad)


def gpu_system(c, prec=0, mesh=None):
    """Assemble c on the GPU through the C-ABI; returns numpy arrays."""
    import torch
    from paper_1802_03433_gb300 import fea

    m = mesh or fea.Mesh(c["coords"], c["tets"])
    dev = torch.device("cuda")
    if c["form"] == "elasticity":
        form = fea.make_form(fea.FEA_ELASTICITY, 1)
        lam = torch.as_tensor(c["lam"], device=dev)
        mu = torch.as_tensor(c["mu"], device=dev)
        keep = (lam, mu)
        coeffs = fea.make_coeffs(lam=lam, mu=mu, f_kind=_fk(c["f_kind"]), f_param=c["f_param"])
    else:
        kind = fea.FEA_DIFFUSION_MASS if c["mass"] else fea.FEA_POISSON
        form = fea.make_form(kind, c["order"], c["mass"])
        kap = None if c["kappa"] is None else torch.as_tensor(c["kappa"], device=dev)
        keep = (kap,)
        coeffs = fea.make_coeffs(kappa=kap, f_kind=_fk(c["f_kind"]), f_param=c["f_param"])
    quad = fea.make_quadrature(c["npts"], prec)
    vals, rhs = m.assemble(form, coeffs, quad)
    torch.cuda.synchronize()
    m.check()
    rp, ci = m.pattern_tensors(c["order"], c["ndpn"])
    out = dict(rp=rp.cpu().numpy(), ci=ci.cpu().numpy(), vals=vals.cpu().numpy(), rhs=rhs.cpu().numpy(),
               mesh=m, keep=keep)
    return out


def _fk(name):
    return {"zero": 0, None: 0, "const": 1, "sinprod": 2}[name]
