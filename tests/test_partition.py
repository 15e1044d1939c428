"""Row partition of a mesh over several GPUs (fea_partition; host only, no
GPU needed here).  Checked on the CPU: the owned node ranges tile the mesh,
each part's element set is exactly the elements with a vertex in its range
(its own plus the ghost layer), its local numbering keeps the global order,
and - with the CPU oracle assembling each part's sub-mesh - the owned rows of
the parts, put together, are bitwise the rows of the whole mesh.  The
bookkeeping runs as a world-size-2 gloo job, as the ranks of a multi-GPU run
would."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1802_03433_gb300 import meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fea():
    import torch  # noqa: F401  (CUDA runtime first)
    from paper_1802_03433_gb300 import build_lib, fea
    build_lib.build()
    return fea


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1802_03433_gb300 import fea
    from paper_1802_03433_gb300 import meshgen as mg
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    coords, tets, _ = mg.make_cube(6, 0.2, 1)
    p = fea.fea_partition(tets, coords.shape[1], world, rank)
    # every rank learns every part's range and element count
    mine = torch.tensor([p["lo"], p["hi"], p["elems"].size, p["nodes"].size], dtype=torch.int64)
    allp = [torch.zeros(4, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allp, mine)
    q.put((rank, [t.tolist() for t in allp], p["elems"].tolist(), p["nodes"].tolist(), p["sub_tets"].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_bookkeeping_gloo(fea):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    coords, tets, _ = mg.make_cube(6, 0.2, 1)
    N, E = coords.shape[1], tets.shape[1]
    ranges = res[0][1]
    assert ranges == res[1][1]  # every rank saw the same table
    # the owned ranges tile [0, N) in rank order
    assert ranges[0][0] == 0 and ranges[-1][1] == N
    assert all(ranges[k][1] == ranges[k + 1][0] for k in range(len(ranges) - 1))
    for rank, _, elems, nodes, sub in res:
        lo, hi = ranges[rank][0], ranges[rank][1]
        want = np.flatnonzero(((tets >= lo) & (tets < hi)).any(axis=0))
        np.testing.assert_array_equal(np.array(elems), want)  # own + ghost elements, exactly
        want_nodes = np.union1d(np.unique(tets[:, want]), np.arange(lo, hi))
        np.testing.assert_array_equal(np.array(nodes), want_nodes)
        np.testing.assert_array_equal(np.array(nodes)[np.array(sub)], tets[:, want])  # local -> global
    # ghosts: the two parts share the layer of elements that straddle the cut
    shared = np.intersect1d(res[0][2], res[1][2])
    straddle = np.flatnonzero(((tets < ranges[0][1]).any(axis=0)) & ((tets >= ranges[1][0]).any(axis=0)))
    np.testing.assert_array_equal(shared, straddle)
    assert 0 < shared.size < E


@pytest.mark.parametrize("kind,ndpn,nparts", [("p1_kappa", 1, 3), ("elasticity", 3, 2), ("elasticity", 3, 4)])
def test_owned_rows_of_the_parts_are_the_whole_mesh_rows(fea, kind, ndpn, nparts):
    """The oracle on each part's sub-mesh: the owned rows, concatenated in
    part order, are bitwise the oracle's rows of the whole mesh (same
    elements in the same order, same coordinates)."""
    from common import case
    c = case(kind, 5, seed=21)
    coords, tets = c["coords"], c["tets"]
    N = coords.shape[1]
    rp, ci = oracle.pattern(N, tets, ndpn=ndpn)
    kw = dict(f_kind=c["f_kind"], f_param=c["f_param"], npts=c["npts"])
    if kind == "elasticity":
        vals, rhs, _ = oracle.assemble(coords, tets, 1, tets, rp, ci, kind="elasticity", lam=c["lam"], mu=c["mu"], **kw)
    else:
        vals, rhs, _ = oracle.assemble(coords, tets, 1, tets, rp, ci, kappa=c["kappa"], **kw)
    lens, cols, vs, rh = [], [], [], []
    for part in range(nparts):
        p = fea.fea_partition(tets, N, nparts, part)
        sc = np.ascontiguousarray(coords[:, p["nodes"]])
        st = p["sub_tets"]
        srp, sci = oracle.pattern(p["nodes"].size, st, ndpn=ndpn)
        if kind == "elasticity":
            sv, sr, _ = oracle.assemble(sc, st, 1, st, srp, sci, kind="elasticity", lam=c["lam"][p["elems"]],
                                        mu=c["mu"][p["elems"]], **kw)
        else:
            sv, sr, _ = oracle.assemble(sc, st, 1, st, srp, sci, kappa=c["kappa"][p["elems"]], **kw)
        r0, ln, cc, vv = fea.owned_rows(p, srp, sci, sv, ndpn)
        assert r0 == ndpn * p["lo"]
        lens.append(ln)
        cols.append(cc)
        vs.append(vv)
        a = int(np.searchsorted(p["nodes"], p["lo"]))
        rh.append(sr[ndpn * a: ndpn * a + ndpn * (p["hi"] - p["lo"])])
    np.testing.assert_array_equal(np.concatenate(lens), np.diff(rp))
    np.testing.assert_array_equal(np.concatenate(cols), ci)
    assert np.array_equal(np.concatenate(vs).view(np.uint64), vals.view(np.uint64))
    assert np.array_equal(np.concatenate(rh).view(np.uint64), rhs.view(np.uint64))


def test_partition_rejects_bad_arguments(fea):
    coords, tets, _ = mg.make_cube(2)
    N = coords.shape[1]
    for nparts, part in ((0, 0), (2, 2), (2, -1)):
        with pytest.raises(fea.FeaError) as ei:
            fea.fea_partition(tets, N, nparts, part)
        assert ei.value.status == 1
    bad = tets.copy()
    bad[1, 3] = N + 5
    with pytest.raises(fea.FeaError) as ei:
        fea.fea_partition(bad, N, 2, 0)
    assert ei.value.status == 2
    # more parts than nodes: some parts own nothing and take no element
    p = fea.fea_partition(tets, N, N + 3, 0)
    assert p["lo"] == p["hi"] == 0 and p["elems"].size == 0


# ---------------------------------------------------------------- batch meshes over several GPUs
def _lpt_bound(m):
    return 4.0 / 3.0 - 1.0 / (3.0 * m)  # Graham's bound for longest processing time first


def test_batch_partition_assigns_every_mesh_and_meets_grahams_bound(fea):
    import itertools
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(1, 8))
        m = int(rng.integers(2, 4))
        cost = rng.integers(1, 50, size=n).astype(np.float64)
        part, load = fea.fea_partition_batch(cost, m)
        assert part.shape == (n,) and set(part.tolist()) <= set(range(m))
        np.testing.assert_array_equal(load, [cost[part == p].sum() for p in range(m)])
        # the best assignment by brute force
        opt = min(max(cost[np.array(a) == p].sum() for p in range(m)) for a in itertools.product(range(m), repeat=n))
        assert load.max() <= _lpt_bound(m) * opt + 1e-12
        again, _ = fea.fea_partition_batch(cost, m)
        np.testing.assert_array_equal(part, again)  # deterministic


def test_batch_partition_special_cases(fea):
    # equal costs: k meshes per part; one part: everything on it; no meshes
    part, load = fea.fea_partition_batch(np.ones(12), 4)
    assert np.bincount(part, minlength=4).tolist() == [3, 3, 3, 3]
    part, load = fea.fea_partition_batch([3.0, 1.0, 2.0], 1)
    assert part.tolist() == [0, 0, 0] and load.tolist() == [6.0]
    part, load = fea.fea_partition_batch(np.zeros(0), 3)
    assert part.size == 0 and load.tolist() == [0.0, 0.0, 0.0]
    # the largest mesh goes first, to part 0; the next to part 1
    part, _ = fea.fea_partition_batch([1.0, 5.0, 4.0], 2)
    assert part.tolist() == [1, 0, 1]


def test_batch_partition_rejects_bad_arguments(fea):
    for cost, m in (([1.0, -1.0], 2), ([1.0, float("nan")], 2), ([1.0, float("inf")], 2), ([1.0], 0)):
        with pytest.raises(fea.FeaError):
            fea.fea_partition_batch(cost, m)


def _batch_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1802_03433_gb300 import fea
    from paper_1802_03433_gb300 import meshgen as mg
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sides, orders = mg.batch_sides()
    cost = 6.0 * sides.astype(np.float64) ** 3 * np.where(orders == 2, 3.6, 1.0)
    part, load = fea.fea_partition_batch(cost, world)
    mine = torch.tensor(np.flatnonzero(part == rank), dtype=torch.int64)
    n = torch.tensor([mine.numel()], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, n)
    q.put((rank, mine.tolist(), [int(c) for c in counts], load.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_partition_gloo(fea):
    """Two ranks split the 256-mesh batch by LPT on their own: their mesh sets
    are disjoint, cover the batch, and their loads are within Graham's bound
    of the perfect split."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_batch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    sides, orders = mg.batch_sides()
    (_, m0, c0, l0), (_, m1, c1, l1) = res
    assert c0 == c1 == [len(m0), len(m1)] and l0 == l1
    assert not set(m0) & set(m1) and sorted(m0 + m1) == list(range(sides.size))
    assert max(l0) <= _lpt_bound(2) * (sum(l0) / 2)


# ---------------------------------------------------------------- adjoint of a partitioned mesh
def _adjoint_case(n=5, seed=23):
    from common import case
    c = case("p1_kappa", n, seed=seed)
    N = c["coords"].shape[1]
    rp, ci = oracle.pattern(N, c["tets"])
    rng = np.random.default_rng(seed + 1)
    v, w, g = rng.standard_normal(N), rng.standard_normal(N), rng.standard_normal(N)
    rows = np.repeat(np.arange(N), np.diff(rp))
    gV = v[rows] * w[ci]  # L = v^T K w + g^T f
    return c, N, rp, ci, gV, g


@pytest.mark.parametrize("nparts", [2, 3])
def test_adjoint_by_parts_gives_the_whole_mesh_gradient(fea, nparts):
    """The oracle's dual-number gradient on each part's sub-mesh, with the
    whole mesh's dL/dvalues taken at the sub-mesh's entries (sub_positions):
    dL/dx of the owned nodes and dL/dkappa of every element of the part are
    bitwise those of the whole mesh."""
    c, N, rp, ci, gV, g = _adjoint_case()
    kw = dict(kappa=c["kappa"], f_kind=c["f_kind"], f_param=c["f_param"], npts=c["npts"])
    gk, gx = oracle.assemble_grad(c["coords"], c["tets"], 1, c["tets"], rp, ci, gV, g, **kw)
    covered = np.zeros(N, dtype=bool)
    for part in range(nparts):
        p = fea.fea_partition(c["tets"], N, nparts, part)
        st = p["sub_tets"]
        srp, sci = oracle.pattern(p["nodes"].size, st)
        pos = fea.sub_positions(p, srp, sci, rp, ci)
        kw_p = dict(kw, kappa=c["kappa"][p["elems"]])
        sgk, sgx = oracle.assemble_grad(np.ascontiguousarray(c["coords"][:, p["nodes"]]), st, 1, st, srp, sci,
                                        gV[pos], g[p["nodes"]], **kw_p)
        assert np.array_equal(sgk.view(np.uint64), gk[p["elems"]].view(np.uint64))
        a, b = np.searchsorted(p["nodes"], [p["lo"], p["hi"]])
        assert np.array_equal(sgx[:, a:b].view(np.uint64), gx[:, p["lo"]:p["hi"]].view(np.uint64))
        covered[p["lo"]:p["hi"]] = True
    assert covered.all()


def test_sub_positions_rejects_a_foreign_pattern(fea):
    c, N, rp, ci, _, _ = _adjoint_case(n=3)
    p = fea.fea_partition(c["tets"], N, 2, 0)
    srp, sci = oracle.pattern(p["nodes"].size, p["sub_tets"])
    # the global pattern of another mesh does not hold the sub-mesh's entries
    c2 = mg.make_cube(2)
    rp2, ci2 = oracle.pattern(c2[0].shape[1], c2[1])
    with pytest.raises(ValueError):
        fea.sub_positions(p, srp, sci, rp2, ci2)


@pytest.mark.parametrize("ndpn,nparts", [(1, 3), (3, 2)])
def test_sub_positions_point_at_the_same_global_entries(fea, ndpn, nparts):
    """Every entry of a part's sub-mesh pattern maps to the whole mesh's entry
    of the same global row and column (scalar and 3 dofs per node)."""
    coords, tets, _ = mg.make_cube(4, 0.2, 3)
    N = coords.shape[1]
    rp, ci = oracle.pattern(N, tets, ndpn=ndpn)
    grow_of = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    for part in range(nparts):
        p = fea.fea_partition(tets, N, nparts, part)
        srp, sci = oracle.pattern(p["nodes"].size, p["sub_tets"], ndpn=ndpn)
        pos = fea.sub_positions(p, srp, sci, rp, ci, ndpn)
        srow = np.repeat(np.arange(srp.size - 1), np.diff(srp))
        want_row = ndpn * p["nodes"][srow // ndpn] + srow % ndpn
        want_col = ndpn * p["nodes"][sci // ndpn] + sci % ndpn
        np.testing.assert_array_equal(grow_of[pos], want_row)
        np.testing.assert_array_equal(ci[pos], want_col)
        assert np.unique(pos).size == pos.size
