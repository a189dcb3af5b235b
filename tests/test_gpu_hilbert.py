"""The tree in Peano-Hilbert order (nb_set_key_order, the order Sec. "Test
and Optimization" names as better than Morton's for locality) against the
oracle's tree in the same order (oracle.Tree(..., order="hilbert")).

Bit-exact, as for Morton order: the sorted Peano-Hilbert keys, the particle
order, every node's level, first particle, count, next, parent and number of
children in the curve's depth-first preorder, the FP64 moments, l and s
(s checks the cell corners, which the kernel recovers from the keys by the
inverse transform), the groups and their boxes, and every interaction list
as a set.  Forces at the tree path's bars (1e-5 / 1e-6 of sum_j |a_ij|)
against the oracle's coords32 sum over the Hilbert tree, and equal as sets of
terms to the Morton tree's: the same interaction counts.
"""
import numpy as np
import pytest

import nbsynth
from tests.gpu_common import gpu_run, oracle_tree_arrays
from tests.test_gpu_parity import CASES, assert_lists_equal, assert_tree_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _sorted_hilbert_keys(oracle, T):
    e = T.export()
    return oracle.hilbert_keys(e["q"])[e["order"]]


@pytest.mark.parametrize("name", list(CASES))
def test_hilbert_tree_groups_lists_bit_exact(oracle_lib, name):
    ps, theta, n_crit, eps = CASES[name]()
    g = gpu_run(ps.pos, ps.mass, theta=theta, n_crit=n_crit, eps=eps, key_order="hilbert")
    T = oracle_lib.Tree(ps.pos, ps.mass, order="hilbert")
    assert np.array_equal(g["tree"]["keys"], _sorted_hilbert_keys(oracle_lib, T))
    assert_tree_equal(g, T)
    assert_lists_equal(g, T, theta, n_crit)
    _, _, npp, npc = T.forces(n_crit, theta, eps)
    Tm = oracle_lib.Tree(ps.pos, ps.mass)
    _, _, mpp, mpc = Tm.forces(n_crit, theta, eps)
    st = g["stats"]
    assert (st["n_pp"], st["n_pc"]) == (npp, npc) == (mpp, mpc)
    g["ctx"].close()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp32_comp", 1e-6)])
def test_hilbert_forces_within_tolerance(oracle_lib, precision, tol):
    ps, theta, n_crit, eps = CASES["halomix20000"]()
    g = gpu_run(ps.pos, ps.mass, theta=theta, n_crit=n_crit, eps=eps, precision=precision,
                lists=False, key_order="hilbert")
    T = oracle_lib.Tree(ps.pos, ps.mass, order="hilbert")
    a32, p32, _, _, am = T.forces(n_crit, theta, eps, with_amag=True, coords32=True)
    d = np.linalg.norm(g["acc"].astype(np.float64) - a32, axis=1)
    assert np.all(d <= tol * am)
    assert np.all(np.abs(g["pot"] - p32) <= tol * np.abs(p32))
    g["ctx"].close()


def test_hilbert_edge_sizes_and_coincident_points(oracle_lib):
    rng = np.random.default_rng(21)
    for n in (1, 2, 3, 33, 4097):
        pos = rng.normal(size=(n, 3))
        if n > 10:
            pos[5:9] = pos[4]            # a depth-21 bucket of coincident particles
        mass = rng.uniform(0.5, 2, n).astype(np.float32)
        for n_crit in (1, 16):
            g = gpu_run(pos, mass, theta=0.7, n_crit=n_crit, eps=0.05, max_n=5000,
                        key_order="hilbert")
            T = oracle_lib.Tree(pos, mass, order="hilbert")
            assert_tree_equal(g, T)
            assert_lists_equal(g, T, 0.7, n_crit)
            g["ctx"].close()


def test_switching_order_back_gives_the_morton_tree(oracle_lib):
    """One context built in Hilbert order, then in Morton order again."""
    import paper_0909_0541_gb300 as nb
    ps, theta, n_crit, eps = CASES["cube4097"]()
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n)
    ctx.set_key_order("hilbert")
    ctx.build_tree(pos, mass)
    ctx.set_key_order("morton")
    ctx.build_tree(pos, mass)
    t = ctx.copy_tree()
    o = oracle_tree_arrays(oracle_lib.Tree(ps.pos, ps.mass))
    assert np.array_equal(t["perm"], o["perm"]) and np.array_equal(t["next"], o["next"])
    ctx.close()


@pytest.mark.slow
def test_hilbert_full_size_tree_and_sampled_lists(oracle_lib):
    """The 2.87M halo mix in Hilbert order: every node and group bit-exact,
    48 sampled groups' lists against the oracle's walk."""
    import paper_0909_0541_gb300 as nb
    ps, w = nbsynth.workload("halomix2.87m")
    theta, n_crit, eps = w["theta"], w["n_crit"], w["eps"]
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit)
    ctx.set_key_order("hilbert")
    ctx.build_tree(pos, mass)
    ctx.walk_groups(theta, n_crit)
    t = ctx.copy_tree()
    gg = ctx.copy_groups()
    T = oracle_lib.Tree(ps.pos, ps.mass, order="hilbert")
    o = oracle_tree_arrays(T)
    assert np.array_equal(t["keys"], _sorted_hilbert_keys(oracle_lib, T))
    assert np.array_equal(t["perm"], o["perm"])
    for k in ("level", "first", "count", "next", "parent", "nchild"):
        assert np.array_equal(t[k], o[k]), k
    assert np.array_equal(t["M"], o["M"]) and np.array_equal(t["com"], o["com"])
    cell = o["is_cell"] == 1
    assert np.array_equal(t["s"][cell], o["s"][cell])
    gnode = T.groups(n_crit)
    box = T.group_boxes(gnode)
    assert np.array_equal(gg["gnode"], gnode) and np.array_equal(gg["box"], box)
    e = T.export()
    leaf_of_slot = np.flatnonzero(e["is_cell"] == 0)
    for k in np.random.default_rng(6).choice(len(gnode), 48, replace=False):
        ref = T.walk_group(gnode[k], box[k], theta)
        f, c = e["first"][gnode[k]], e["count"][gnode[k]]
        own = np.isin(ref, leaf_of_slot[f:f + c])
        ids, _ = ctx.copy_list(k)
        assert np.array_equal(np.sort(ids), ref[~own])
    ctx.close()
