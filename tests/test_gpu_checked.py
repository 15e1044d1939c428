"""The bounds-checked build (libfea_checked.so: build_lib.build(checked=True),
loaded with FEA_CHECKED=1).

- Every vertex gather of the element kernels and every shared-memory slot,
  CSR position and partial-sum index of the scatters is checked there; on
  valid meshes no check fails, and the results are bitwise those of the
  normal build (the checks only guard accesses, they change no arithmetic).
  The checked library runs in a child process (the binding picks the library
  when it loads), on the same seeded inputs as the normal one here.
- A failing check latches DEV_ERR_INDEX instead of touching memory:
  fea_diag_checked_gather reads src[idx] through the same check; with idx
  past the logical length n (still inside the buffer, which holds 2n values)
  nothing is read, out[0] is -1 and fea_mesh_check reports FEA_ERR_INDEX.
  The normal build launches nothing there and says so."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from common import case, gpu_system
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [("p1_kappa", 6, 0, 0), ("p2_diffmass", 4, 0, 0), ("p2_diffmass", 4, 1, 0), ("elasticity", 5, 0, 0),
         ("elasticity", 5, 1, 0), ("elasticity", 5, 0, 1)]


def systems(out_path):
    """Assemble every case (and the 2-D example and one backward pass) with
    whichever library the binding loaded; save the arrays to out_path."""
    import torch
    from paper_1802_03433_gb300 import fea
    res = {}
    for kind, n, prec, local in CASES:
        c = case(kind, n, seed=41)
        m = fea.Mesh(c["coords"], c["tets"])
        if local:
            fea.fea_mesh_set_scatter(m.h, fea.FEA_SCATTER_LOCAL_ROWS)
        g = gpu_system(c, prec=prec, mesh=m)
        key = f"{kind}_{n}_{prec}_{local}"
        res[key + "_v"], res[key + "_r"] = g["vals"], g["rhs"]
        m.close()
    coords, tris = mg.tri_square(16, 0.2, 3)
    m = fea.Mesh(coords, tris)
    v, r = m.assemble_2d(fea.make_form2d())
    torch.cuda.synchronize()
    m.check()
    res["tri_v"], res["tri_r"] = v.cpu().numpy(), r.cpu().numpy()
    m.close()
    c = case("p1_kappa", 5, seed=42)
    m = fea.Mesh(c["coords"], c["tets"])
    _, nnz = m.pattern(1)
    rng = np.random.default_rng(42)
    gV = torch.as_tensor(rng.standard_normal(nnz), device="cuda")
    gF = torch.as_tensor(rng.standard_normal(c["coords"].shape[1]), device="cuda")
    gk = torch.empty(c["tets"].shape[1], dtype=torch.float64, device="cuda")
    gx = torch.empty((3, c["coords"].shape[1]), dtype=torch.float64, device="cuda")
    co = fea.make_coeffs(kappa=torch.as_tensor(c["kappa"], device="cuda"), f_kind=fea.FEA_LOAD_SINPROD,
                         f_param=c["f_param"])
    fea.fea_assemble_backward(m.h, fea.make_form(fea.FEA_POISSON, 1), co, fea.make_quadrature(c["npts"]), gV, gF,
                              gk, gx)
    torch.cuda.synchronize()
    m.check()
    res["adj_k"], res["adj_x"] = gk.cpu().numpy(), gx.cpu().numpy()
    m.close()
    np.savez(out_path, **res)


def diag(out_path):
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(2)
    m = fea.Mesh(coords, tets)
    n = 64
    src = torch.arange(2 * n, dtype=torch.float64, device="cuda")  # 2n held, n logical
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    res = {}
    res["checked"] = fea.fea_diag_checked_gather(m.h, src, n, 5, out)
    torch.cuda.synchronize()
    res["in_range"] = float(out[0])
    m.check()
    fea.fea_diag_checked_gather(m.h, src, n, n + 3, out)
    torch.cuda.synchronize()
    res["past_end"] = float(out[0])
    try:
        m.check()
        res["status"] = 0
    except fea.FeaError as e:
        res["status"] = e.status
    m.check()  # the bit was cleared by the previous check
    m.close()
    np.savez(out_path, **res)


def _run_checked(fn_name, tmp):
    from paper_1802_03433_gb300 import build_lib
    build_lib.build(checked=True)
    out = os.path.join(tmp, fn_name + ".npz")
    code = (f"import sys; sys.path[:0] = [{ROOT!r}, {os.path.join(ROOT, 'tests')!r}]; "
            f"import test_gpu_checked as t; t.{fn_name}({out!r})")
    env = dict(os.environ, FEA_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return dict(np.load(out))


def test_checked_build_gives_bitwise_the_normal_results():
    with tempfile.TemporaryDirectory() as tmp:
        got = _run_checked("systems", tmp)
        mine = os.path.join(tmp, "normal.npz")
        systems(mine)
        want = dict(np.load(mine))
    assert sorted(got) == sorted(want)
    for k in want:
        assert np.array_equal(got[k].view(np.uint64), want[k].view(np.uint64)), k


def test_failed_check_latches_the_index_error_and_reads_nothing():
    with tempfile.TemporaryDirectory() as tmp:
        r = _run_checked("diag", tmp)
    assert bool(r["checked"])
    assert float(r["in_range"]) == 5.0
    assert float(r["past_end"]) == -1.0
    assert int(r["status"]) == 2  # FEA_ERR_INDEX


def test_normal_build_launches_no_unchecked_read():
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tets, _ = mg.make_cube(2)
    m = fea.Mesh(coords, tets)
    src = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    assert not fea.fea_diag_checked_gather(m.h, src, 4, 6, out)
    torch.cuda.synchronize()
    assert float(out[0]) == 7.0
    m.check()
    m.close()
