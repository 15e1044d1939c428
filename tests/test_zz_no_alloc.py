"""fea_assemble_noalloc, the allocation-free variant of fea_assemble for
callers that cannot let a library call cudaMalloc (device memory reserved
by another allocator, or loops that cannot take the synchronisation of an
allocation).  Its scratch is a fixed device array inside the library.

Called through the C-ABI twice in a row on the same inputs, it must give
bitwise what fea_assemble gives with the same element and scatter launches
(the fused element kernel and the local-row scatter), agree with the CPU
oracle within the FP64 parity tolerance, and leave the device's free memory
unchanged.  Meshes too large for the fixed array, and misaligned arguments,
are rejected before anything runs.  This file sorts last so that a run
stopping at the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

from common import TOL_FP64, TOL_MIXED, case, oracle_system, row_scaled_error, vec_scaled_error

pytestmark = pytest.mark.gpu


def _setup(kind, n, prec):
    import torch
    from paper_1802_03433_gb300 import fea
    c = case(kind, n, seed=11)
    m = fea.Mesh(c["coords"], c["tets"])
    keep = []
    if c["form"] == "elasticity":
        lam, mu = torch.as_tensor(c["lam"], device="cuda"), torch.as_tensor(c["mu"], device="cuda")
        keep += [lam, mu]
        co = fea.make_coeffs(lam=lam, mu=mu, f_kind=1, f_param=c["f_param"])
        form = fea.make_form(fea.FEA_ELASTICITY, 1)
    else:
        kap = None if c["kappa"] is None else torch.as_tensor(c["kappa"], device="cuda")
        keep.append(kap)
        co = fea.make_coeffs(kappa=kap, f_kind=2, f_param=c["f_param"])
        form = fea.make_form(fea.FEA_DIFFUSION_MASS if c["mass"] else fea.FEA_POISSON, c["order"], c["mass"])
    q = fea.make_quadrature(c["npts"], prec)
    # the reference call takes the launches noalloc takes: the fused element
    # kernel and the local-row scatter chosen automatically
    fea.fea_mesh_set_load_split(m.h, 0)
    if hasattr(fea, "fea_mesh_set_scatter"):
        fea.fea_mesh_set_scatter(m.h, fea.FEA_SCATTER_LOCAL_ROWS)
    return fea, m, form, co, q, keep, c


@pytest.mark.parametrize("kind,n,prec", [("p1_kappa", 8, 0), ("p2_diffmass", 5, 0), ("elasticity", 4, 0),
                                         ("p2_diffmass", 5, 1), ("elasticity", 4, 1)])
def test_noalloc_matches_fea_assemble_twice(kind, n, prec):
    import torch
    fea, m, form, co, q, keep, c = _setup(kind, n, prec)
    ref_v, ref_r = m.assemble(form, co, q)
    ref_v, ref_r = ref_v.clone(), ref_r.clone()
    torch.cuda.synchronize()
    o = oracle_system(c)
    tol = TOL_FP64 if prec == 0 else TOL_MIXED
    v = torch.full_like(ref_v, np.nan)
    r = torch.full_like(ref_r, np.nan)
    fea.fea_assemble_noalloc(m.h, form, co, q, v, r)  # the first call on the device takes the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        v.fill_(np.nan)
        r.fill_(np.nan)
        fea.fea_assemble_noalloc(m.h, form, co, q, v, r)
        torch.cuda.synchronize()
        m.check()
        assert torch.cuda.mem_get_info()[0] == free0  # nothing was allocated
        assert torch.equal(v, ref_v) and torch.equal(r, ref_r)
        assert row_scaled_error(o["rp"], o["vals"], v.cpu().numpy()) <= tol
        assert vec_scaled_error(o["rhs"], r.cpu().numpy()) <= tol
    m.close()


def test_noalloc_rejects_meshes_above_the_fixed_scratch():
    import torch
    fea, m, form, co, q, keep, c = _setup("p2_diffmass", 40, 0)  # 384,000 P2 tets ~ 400 MB of scratch
    ndof, nnz = m.pattern(2)
    v = torch.empty(nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_assemble_noalloc(m.h, form, co, q, v, None)
    assert ei.value.status == 1 and "fixed" in str(ei.value)
    m.close()


def test_noalloc_rejects_misaligned_arguments_before_any_launch():
    """A values, rhs or coefficient pointer off its 8-byte alignment is refused
    on the host (FEA_ERR_ARG); the output is left untouched."""
    import torch
    fea, m, form, co, q, keep, c = _setup("p1_kappa", 4, 0)
    ndof, nnz = m.pattern(1)
    v = torch.full((nnz + 1,), 7.0, dtype=torch.float64, device="cuda")
    r = torch.full((ndof + 1,), 7.0, dtype=torch.float64, device="cuda")
    L = fea.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    off = C.c_void_p(v.data_ptr() + 4)
    st = L.fea_assemble_noalloc(m.h, C.byref(form), C.byref(co), C.byref(q), off, C.c_void_p(r.data_ptr()), s)
    assert st == 1 and "misaligned" in L.fea_last_error().decode()
    st = L.fea_assemble_noalloc(m.h, C.byref(form), C.byref(co), C.byref(q), C.c_void_p(v.data_ptr()),
                                C.c_void_p(r.data_ptr() + 4), s)
    assert st == 1
    kap = torch.ones(c["tets"].shape[1] + 1, dtype=torch.float64, device="cuda")
    bad = fea.make_coeffs(kappa=kap, f_kind=2, f_param=c["f_param"])
    bad.kappa = kap.data_ptr() + 4
    st = L.fea_assemble_noalloc(m.h, C.byref(form), C.byref(bad), C.byref(q), C.c_void_p(v.data_ptr()),
                                C.c_void_p(r.data_ptr()), s)
    assert st == 1 and "aligned" in L.fea_last_error().decode()
    torch.cuda.synchronize()
    assert bool((v == 7.0).all()) and bool((r == 7.0).all())
    m.close()
