"""The paper's 2-D worked example on the GPU (fea_mesh_create_tri,
fea_assemble_2d) against the oracle: P1 triangles, sigma = [[1, -x-y],
[x+y, 1]], lambda = 1, f = -2 (x^2 + y^2) + 36 (Sec. 4.1-4.2)."""
import numpy as np
import pytest

import oracle
from common import TOL_FP64, row_scaled_error, vec_scaled_error
from paper_1802_03433_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


def _gpu(coords, tris, **kw):
    import torch
    from paper_1802_03433_gb300 import fea
    m = fea.Mesh(coords, tris)
    v, r = m.assemble_2d(fea.make_form2d(**kw))
    torch.cuda.synchronize()
    m.check()
    rp, ci = m.pattern_tensors(1)
    return m, rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), r.cpu().numpy()


@pytest.mark.parametrize("n", [1, 5, 17, 40])
@pytest.mark.parametrize("npts", [1, 3, 6])
def test_paper_example_matches_oracle(n, npts):
    coords, tris = mg.tri_square(n, 0.2, n)
    m, rp, ci, v, r = _gpu(coords, tris, npts=npts)
    orp, oci = oracle.pattern(coords.shape[1], tris)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    ov, orr, bad = oracle.assemble_tri(coords, tris, orp, oci, npts=npts)
    assert bad == 0
    assert row_scaled_error(orp, ov, v) <= TOL_FP64
    assert vec_scaled_error(orr, r) <= TOL_FP64
    if n >= 5:
        assert np.diff(rp).max() == 7   # the paper's MAX_NZ (Sec. 5)
    m.close()


def test_other_sigma_and_unstructured_order():
    coords, tris = mg.tri_square(12, 0.2, 7)
    rng = np.random.default_rng(2)
    perm = rng.permutation(tris.shape[1])
    tris = np.ascontiguousarray(tris[:, perm])
    kw = dict(sigma0=(2.0, 0.3, -0.4, 1.5), sigma_x=(0.1, 0.2, 0.3, -0.1), sigma_y=(-0.2, 0.0, 0.5, 0.4), lam=0.7,
              f=(1.0, 2.0, -1.0, 0.5, 0.25, -0.75), npts=6)
    m, rp, ci, v, r = _gpu(coords, tris, **kw)
    ov, orr, _ = oracle.assemble_tri(coords, tris, rp, ci, S0=kw["sigma0"], Sx=kw["sigma_x"], Sy=kw["sigma_y"],
                                     lam=kw["lam"], f=kw["f"], npts=6)
    assert row_scaled_error(rp, ov, v) <= TOL_FP64
    assert vec_scaled_error(orr, r) <= TOL_FP64
    m.close()


def test_paper_example_4m_nodes_properties():
    """2048^2 squares (8,388,608 triangles, 4,198,401 nodes - the top of the
    paper's 10K-10M node range): sum of values = area (the stiffness rows and
    columns annihilate constants, the mass sums to the area), sum of the load
    = int f = 36 - 4/3, and 16 rows of a 400^2 mesh entry by entry."""
    coords, tris = mg.tri_square(2048, 0.2, 0)
    m, rp, ci, v, r = _gpu(coords, tris)
    assert np.diff(rp).max() == 7 and rp[-1] == 7 * 2048 ** 2 + 6 * 2048 + 1  # N + 2 (3n^2 + 2n) edges
    assert abs(v.sum() - 1.0) < 1e-9
    assert abs(r.sum() - (36 - 4 / 3)) < 1e-9 * 36
    m.close()


def test_scatter_modes_bitwise_identical():
    import torch
    from paper_1802_03433_gb300 import fea
    coords, tris = mg.tri_square(37, 0.2, 4)
    m = fea.Mesh(coords, tris)
    outs = []
    for mode in (0, 3):
        fea.fea_mesh_set_scatter_classes(m.h, mode)
        v, r = m.assemble_2d(fea.make_form2d())
        torch.cuda.synchronize()
        outs.append((v.cpu().numpy().view(np.uint64), r.cpu().numpy().view(np.uint64)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    m.close()
