"""Parity at the full benchmark sizes, in the configuration bench.py times.

The whole tree (every node of the 2.87M, 2M and 4.19M-particle sets) and
every group are compared bit for bit; interaction lists and forces are
compared on a seeded sample of groups the oracle walks one by one.  The
512-system forest of the batch benchmark is compared system by system on a
seeded sample of its systems.
"""
import numpy as np
import pytest

import nbsynth
from tests.gpu_common import oracle_tree_arrays, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("workload,theta", [("halomix2.87m", None), ("cosmo2m", 0.5),
                                            ("cosmo2m", 1.0), ("halomix4.19m", None)])
def test_full_size_tree_lists_forces(oracle_lib, workload, theta):
    import paper_0909_0541_gb300 as nb
    ps, w = nbsynth.workload(workload)
    theta = w["theta"] if theta is None else theta
    n_crit, eps = w["n_crit"], w["eps"]
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit)
    ctx.build_tree(pos, mass)
    ctx.walk_groups(theta, n_crit)
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device=dev)
    pot = torch.empty(ps.n, dtype=torch.float32, device=dev)
    ctx.forces(eps, acc, pot, "fp32")
    acc, pot = acc.cpu().numpy(), pot.cpu().numpy()
    t = ctx.copy_tree()
    gg = ctx.copy_groups()

    T = oracle_lib.Tree(ps.pos, ps.mass)
    o = oracle_tree_arrays(T)
    assert np.array_equal(t["perm"], o["perm"])
    for k in ("level", "first", "count", "next", "parent", "nchild"):
        assert np.array_equal(t[k], o[k]), k
    assert np.array_equal(t["M"], o["M"]) and np.array_equal(t["com"], o["com"])
    cell = o["is_cell"] == 1
    assert np.array_equal(t["l"][cell], o["l"][cell]) and np.array_equal(t["s"][cell], o["s"][cell])

    gnode = T.groups(n_crit)
    box = T.group_boxes(gnode)
    assert np.array_equal(gg["gnode"], gnode) and np.array_equal(gg["box"], box)

    e = T.export()
    leaf_of_slot = np.flatnonzero(e["is_cell"] == 0)
    sel = np.random.default_rng(5).choice(len(gnode), 48, replace=False)
    for k in sel:
        ref = T.walk_group(gnode[k], box[k], theta)
        f, c = e["first"][gnode[k]], e["count"][gnode[k]]
        own = np.isin(ref, leaf_of_slot[f:f + c])
        assert own.sum() == c
        ids, _ = ctx.copy_list(k)
        assert np.array_equal(np.sort(ids), ref[~own])
    a32, p32, _, _, am = T.forces(n_crit, theta, eps, gsel=sel, with_amag=True, coords32=True)
    a64, _, _, _ = T.forces(n_crit, theta, eps, gsel=sel)
    rows = np.concatenate([e["order"][e["first"][gnode[k]]:e["first"][gnode[k]] + e["count"][gnode[k]]]
                           for k in sel])
    d = np.linalg.norm(acc[rows].astype(np.float64) - a32[rows], axis=1)
    assert np.all(d <= 1e-5 * am[rows])
    assert np.all(np.abs(pot[rows] - p32[rows]) <= 1e-5 * np.abs(p32[rows]))
    assert np.median(rel_err(acc[rows], a64[rows])) < 1e-6
    ctx.close()


def test_full_batch512_sampled_systems(oracle_lib):
    """The 512-system forest (7.66M particles) as the batch benchmark builds
    it: for 12 seeded systems, the system's part of the forest (order,
    topology, moments, groups, boxes), four of its lists and all its forces
    against the system's own oracle tree."""
    import paper_0909_0541_gb300 as nb
    systems = nbsynth.batched_systems(512)
    off = np.r_[0, np.cumsum([ps.n for ps in systems])].astype(np.int64)
    eps, theta, n_crit = 1.0 / 64, 0.75, 256
    dev = torch.device("cuda")
    pos = np.concatenate([ps.pos for ps in systems])
    mass = np.concatenate([ps.mass for ps in systems])
    ctx = nb.NBody(len(pos), eps=eps, theta=theta, n_crit=n_crit, max_systems=len(systems))
    ctx.build_tree_batched(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                           torch.from_numpy(off).to(dev))
    ctx.walk_groups(theta, n_crit)
    acc = torch.empty((len(pos), 3), dtype=torch.float32, device=dev)
    ctx.forces(eps, acc)
    acc = acc.cpu().numpy()
    t = ctx.copy_tree()
    gg = ctx.copy_groups()
    roots = np.flatnonzero(t["parent"] == -1)   # one per system, in preorder
    assert len(roots) == len(systems)
    ends = np.r_[roots[1:], len(t["parent"])]
    rng = np.random.default_rng(9)
    for s in np.sort(rng.choice(len(systems), 12, replace=False)):
        ps = systems[s]
        T = oracle_lib.Tree(ps.pos, ps.mass)
        o = oracle_tree_arrays(T)
        node0, nn = roots[s], ends[s] - roots[s]
        assert nn == T.nnodes
        sl = slice(node0, node0 + nn)
        assert np.array_equal(t["perm"][off[s]:off[s + 1]] - off[s], o["perm"])
        assert np.array_equal(t["first"][sl] - off[s], o["first"])
        for k in ("level", "count", "nchild"):
            assert np.array_equal(t[k][sl], o[k]), (s, k)
        assert np.array_equal(t["M"][sl], o["M"]) and np.array_equal(t["com"][sl], o["com"])
        mine = np.flatnonzero((gg["gfirst"] >= off[s]) & (gg["gfirst"] < off[s + 1]))
        gnode = T.groups(n_crit)
        assert np.array_equal(gg["gnode"][mine] - node0, gnode)
        box = T.group_boxes(gnode)
        assert np.array_equal(gg["box"][mine], box)
        e = T.export()
        leaf = np.flatnonzero(e["is_cell"] == 0)
        for k in rng.choice(len(mine), min(4, len(mine)), replace=False):
            ref = T.walk_group(gnode[k], box[k], theta)
            f, c = e["first"][gnode[k]], e["count"][gnode[k]]
            ref = ref[~np.isin(ref, leaf[f:f + c])]
            ids, _ = ctx.copy_list(mine[k])
            assert np.array_equal(np.sort(ids) - node0, ref)
        a32, _, _, _, am = T.forces(n_crit, theta, eps, with_amag=True, coords32=True)
        d = np.linalg.norm(acc[off[s]:off[s + 1]].astype(np.float64) - a32, axis=1)
        assert np.all(d <= 1e-5 * np.maximum(am, 1e-300))
    ctx.close()
