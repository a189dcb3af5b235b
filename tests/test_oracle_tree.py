"""Pins for the oracle's tree code: grid, Morton keys, topology, moments,
next/more threading, groups, interaction lists and force accuracy.

Every check here recomputes what it needs from the definitions in numpy
(brute-force bit interleaving, prefix enumeration, exact dyadic sums, the
FP32 opening test) rather than re-calling the oracle routine it checks."""
import numpy as np
import pytest

import nbsynth

LEVELS = 21


def np_morton(q):
    """Brute-force interleave in numpy, independent of the C routine."""
    q = q.astype(np.uint64)
    key = np.zeros(q.shape[0], np.uint64)
    for b in range(LEVELS - 1, -1, -1):
        for a in range(3):
            key = (key << np.uint64(1)) | ((q[:, a] >> np.uint64(b)) & np.uint64(1))
    return key


def clustered_small(n=6000, seed=3):
    """Uniform points plus a tight clump and exactly coincident particles,
    so that deep chains and depth-21 buckets occur."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1, 1, (n, 3))
    pos[: n // 10] = 0.3 + 1e-5 * rng.normal(size=(n // 10, 3))
    pos[n // 10: n // 10 + 7] = pos[n // 10 + 7]          # 8 coincident
    pos[-3:] = pos[-4]                                    # 4 coincident
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return pos, mass


def dyadic_set(n=4096, seed=9):
    rng = np.random.default_rng(seed)
    pos = rng.integers(-1024, 1024, (n, 3)).astype(np.float64) / 1024.0
    mass = np.full(n, 1.0 / n, np.float32)
    return pos, mass


@pytest.fixture(scope="module")
def plummer_tree(oracle_lib):
    ps = nbsynth.plummer(16384, nbsynth.BASE_SEED + 1)
    return ps, oracle_lib.Tree(ps.pos, ps.mass)


@pytest.fixture(scope="module")
def clump_tree(oracle_lib):
    pos, mass = clustered_small()
    return pos, mass, oracle_lib.Tree(pos, mass)


def test_root_cube_and_grid_contain_particles(oracle_lib, clump_tree):
    pos, mass, T = clump_tree
    q = T.export()["q"]
    assert q.min() >= 0 and q.max() < 2 ** LEVELS
    assert np.all(pos >= T.corner) and np.all(pos < T.corner + T.L)
    h = T.L / 2 ** LEVELS
    lo = T.corner + q * h
    # each particle lies in its grid cell (to FP64 rounding of the quotient)
    assert np.all(pos >= lo - 1e-12 * T.L) and np.all(pos <= lo + h + 1e-12 * T.L)
    ext = (pos.max(0) - pos.min(0)).max()
    assert T.L == ext * (1 + 2.0 ** -20)
    assert np.array_equal(T.centre, 0.5 * (pos.min(0) + pos.max(0)))


def test_morton_keys_match_brute_force(oracle_lib, clump_tree):
    _, _, T = clump_tree
    q = T.export()["q"]
    assert np.array_equal(oracle_lib.morton_keys(q), np_morton(q))


@pytest.mark.parametrize("which", ["plummer", "clump", "dyadic"])
def test_dfs_leaf_order_is_sorted_key_order(oracle_lib, plummer_tree, clump_tree, which):
    if which == "plummer":
        T = plummer_tree[1]
    elif which == "clump":
        T = clump_tree[2]
    else:
        T = oracle_lib.Tree(*dyadic_set())
    e = T.export()
    keys = np_morton(e["q"])
    assert np.array_equal(e["order"], np.argsort(keys, kind="stable"))
    # particle leaves appear in preorder in sorted-slot order
    leaves = np.flatnonzero(e["is_cell"] == 0)
    assert np.array_equal(e["first"][leaves], np.arange(T.n))


def brute_cells(keys_sorted):
    """(level, first, count) of every key prefix shared by >= 2 particles."""
    out = set()
    n = keys_sorted.shape[0]
    for lev in range(LEVELS + 1):
        pre = keys_sorted >> np.uint64(3 * (LEVELS - lev))
        starts = np.flatnonzero(np.r_[True, pre[1:] != pre[:-1]])
        counts = np.diff(np.r_[starts, n])
        for s, c in zip(starts[counts >= 2], counts[counts >= 2]):
            out.add((lev, int(s), int(c)))
    return out


@pytest.mark.parametrize("which", ["plummer", "clump"])
def test_topology_matches_prefix_enumeration(plummer_tree, clump_tree, which):
    T = plummer_tree[1] if which == "plummer" else clump_tree[2]
    e = T.export()
    keys = np.sort(np_morton(e["q"]))
    cells = np.flatnonzero(e["is_cell"] == 1)
    got = set(zip(e["level"][cells].tolist(), e["first"][cells].tolist(),
                  e["count"][cells].tolist()))
    assert got == brute_cells(keys)
    assert T.ncells == len(cells) and T.nnodes == len(cells) + T.n


def test_bucket_cells_exist_for_coincident_particles(clump_tree):
    _, _, T = clump_tree
    e = T.export()
    buckets = np.flatnonzero((e["is_cell"] == 1) & (e["level"] == LEVELS))
    assert set(e["count"][buckets].tolist()) >= {8, 4}
    for b in buckets:      # members are the next count nodes, all particle leaves
        c = e["count"][b]
        assert np.all(e["is_cell"][b + 1: b + 1 + c] == 0)
        assert e["nchild"][b] == c


def test_next_more_parent_threading(plummer_tree, clump_tree):
    for T in (plummer_tree[1], clump_tree[2]):
        e = T.export()
        nn = T.nnodes
        cell = e["is_cell"] == 1
        assert np.array_equal(e["more"][cell], np.flatnonzero(cell) + 1)
        assert np.all(e["more"][~cell] == -1)
        # subtree sizes from parent pointers (children follow parents in preorder)
        size = np.ones(nn, np.int64)
        par = e["parent"]
        for u in range(nn - 1, 0, -1):
            size[par[u]] += size[u]
        nxt = np.arange(nn) + size
        nxt[nxt == nn] = -1
        assert np.array_equal(e["next"], nxt)
        assert np.all(par[1:] < np.arange(1, nn)) and par[0] == -1
        # particle counts add up over children
        cnt = np.zeros(nn, np.int64)
        np.add.at(cnt, par[1:], e["count"][1:])
        assert np.array_equal(cnt[cell], e["count"][cell])
        nch = np.bincount(par[1:], minlength=nn)
        assert np.array_equal(nch[cell], e["nchild"][cell])


def test_moments_exact_on_dyadic_input(oracle_lib):
    pos, mass = dyadic_set()
    T = oracle_lib.Tree(pos, mass)
    e = T.export()
    order = e["order"]
    for u in np.flatnonzero(e["is_cell"] == 1):
        mem = order[e["first"][u]: e["first"][u] + e["count"][u]]
        M = mass[mem].astype(np.float64).sum()
        assert e["M"][u] == M
        com = (mass[mem].astype(np.float64)[:, None] * pos[mem]).sum(0) / M
        assert np.array_equal(e["com"][u], com)
        lev = e["level"][u]
        lc = T.L / 2.0 ** lev
        assert e["l"][u] == np.float32(lc)
        corner = e["q"][mem[0]] >> (LEVELS - lev)
        g = T.corner + (corner + 0.5) * lc
        assert np.all(np.abs(com - g) <= 0.5 * lc * (1 + 1e-12))
        assert e["s"][u] == np.float32(np.sqrt(((com - g) ** 2).sum()))
        assert np.array_equal(e["comf"][u], com.astype(np.float32))


def test_groups_partition_and_rule(plummer_tree, clump_tree):
    for T in (plummer_tree[1], clump_tree[2]):
        e = T.export()
        for n_crit in (1, 16, 64, 1000):
            g = T.groups(n_crit)
            assert np.all(np.diff(g) > 0)
            cnt = e["count"][g]
            assert np.all(cnt <= n_crit)
            par = e["parent"][g]
            assert np.all((par == -1) | (e["count"][np.maximum(par, 0)] > n_crit))
            assert np.array_equal(e["first"][g], np.r_[0, np.cumsum(cnt)[:-1]])
            assert cnt.sum() == T.n


def group_boxes_numpy(T, gnode):
    e = T.export()
    out = []
    for u in gnode:
        mem = e["order"][e["first"][u]: e["first"][u] + e["count"][u]]
        x = T.pos[mem].astype(np.float32)
        lo, hi = x.min(0), x.max(0)
        c = (0.5 * (lo.astype(np.float64) + hi.astype(np.float64))).astype(np.float32)
        out.append(np.r_[lo, hi, c])
    return np.array(out, np.float32)


def mac_far_numpy(e, u, box, theta):
    """The group opening test in numpy float32, one rounding per operation."""
    f = np.float32
    invth = f(1.0 / theta) if theta > 0 else f(np.inf)
    c = e["comf"][u]
    below = box[:3] - c
    above = c - box[3:6]
    ex = np.maximum(np.maximum(below, above), f(0))
    d2 = f(ex[0] * ex[0])
    d2 = f(d2 + f(ex[1] * ex[1]))
    d2 = f(d2 + f(ex[2] * ex[2]))
    w = f(f(e["l"][u] * invth) + e["s"][u])
    return bool(d2 > f(w * w))


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.75, 1.0])
def test_lists_partition_and_mac(plummer_tree, theta):
    ps, T = plummer_tree
    e = T.export()
    n_crit = 64
    gnode, box, off, ent = T.all_lists(n_crit, theta)
    assert np.array_equal(box, group_boxes_numpy(T, gnode))
    rng = np.random.default_rng(1)
    par = e["parent"]
    total_m = ps.mass.astype(np.float64)
    for g in rng.choice(len(gnode), 24, replace=False):
        lst = ent[off[g]: off[g + 1]]
        assert np.array_equal(lst, T.walk_group(gnode[g], box[g], theta, mode=0))
        assert np.all(np.diff(lst) > 0)       # depth-first order = preorder ids
        # partition: every particle covered exactly once
        cover = np.zeros(T.n, np.int64)
        for u in lst:
            cover[e["first"][u]: e["first"][u] + e["count"][u]] += 1
        assert np.all(cover == 1)
        # opening test: accepted cells pass and do not hold the group; every
        # proper ancestor of an entry was opened (fails, or holds the group)
        gfirst = e["first"][gnode[g]]
        opened = set()
        for u in lst:
            if e["is_cell"][u]:
                assert mac_far_numpy(e, u, box[g], theta)
                assert not (e["first"][u] <= gfirst < e["first"][u] + e["count"][u])
            a = par[u]
            while a != -1 and a not in opened:
                opened.add(a)
                a = par[a]
        for a in opened:
            holds = e["first"][a] <= gfirst < e["first"][a] + e["count"][a]
            assert holds or not mac_far_numpy(e, a, box[g], theta)
        if theta == 0.0:
            leaves = np.flatnonzero(e["is_cell"] == 0)
            assert np.array_equal(lst, leaves)


def test_theta_zero_reproduces_direct_sum(oracle_lib):
    ps = nbsynth.plummer(2048, 4)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    eps = 1.0 / 64
    a, p, npp, npc = T.forces(32, 0.0, eps)
    ad, pd = oracle_lib.direct(ps.pos, ps.mass, eps)
    assert npc == 0 and npp == ps.n * (ps.n - 1)
    assert np.max(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)) < 1e-12
    assert np.max(np.abs(p - pd) / np.abs(pd)) < 1e-13


@pytest.mark.parametrize("theta", [0.5, 0.75, 1.0])
def test_ncrit_one_equals_per_particle_walk(plummer_tree, theta):
    ps, T = plummer_tree
    gnode = T.groups(1)
    assert len(gnode) == T.n
    box = T.group_boxes(gnode)
    e = T.export()
    for g in np.random.default_rng(2).choice(T.n, 40, replace=False):
        slot = e["first"][gnode[g]]
        assert np.array_equal(T.walk_group(gnode[g], box[g], theta),
                              T.walk_particle(slot, theta))


def test_force_error_level_and_monotone_in_theta(oracle_lib):
    # random points in a cube, per-particle walk (n_crit = 1) as in the paper.
    # The paper puts the tree method's mean relative error at theta 0.5-0.6
    # near 2e-4 without saying of which quantity; a loose pin: within a
    # factor 20 of it (a dropped term or wrong sign gives O(1) errors).
    ps = nbsynth.uniform_cube(1 << 15, 7)
    eps = 1e-4
    sel = np.random.default_rng(0).choice(ps.n, 2048, replace=False)
    ad, _ = oracle_lib.direct(ps.pos, ps.mass, eps, targets=sel)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    prev = 0.0
    for theta in (0.3, 0.5, 0.7, 0.9):
        a, _, _, _ = T.forces(1, theta, eps)
        err = np.linalg.norm(a[sel] - ad, axis=1) / np.linalg.norm(ad, axis=1)
        assert err.mean() > prev
        prev = err.mean()
        if theta == 0.5:
            assert 1e-5 < err.mean() < 4e-3
    # groups only tighten the opening test, so the error drops
    a1, _, _, _ = T.forces(1, 0.7, eps)
    a64, _, _, _ = T.forces(64, 0.7, eps)
    e1 = np.linalg.norm(a1[sel] - ad, axis=1) / np.linalg.norm(ad, axis=1)
    e64 = np.linalg.norm(a64[sel] - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert np.median(e64) < np.median(e1)


def test_tiny_and_degenerate_inputs(oracle_lib):
    # one particle: the root is a particle leaf, its list is itself, force 0
    T = oracle_lib.Tree(np.array([[0.5, 0.5, 0.5]]), np.array([1.0], np.float32))
    assert T.nnodes == 1 and T.ncells == 0 and T.L == 1.0
    a, p, npp, npc = T.forces(8, 0.6, 0.1)
    assert np.all(a == 0) and p[0] == 0 and npp == 0 and npc == 0
    # all particles coincident: one depth-21 bucket under a chain of cells
    pos = np.tile([[0.1, -0.2, 0.3]], (5, 1))
    T = oracle_lib.Tree(pos, np.ones(5, np.float32))
    e = T.export()
    assert T.ncells == LEVELS + 1 and e["level"][T.ncells - 1] == LEVELS
    a, p, _, _ = T.forces(2, 0.6, 0.5)
    assert np.allclose(a, 0) and np.allclose(p, -4 / 0.5)


def test_coords32_mode(oracle_lib):
    # dyadic positions, theta 0: the group-relative FP32 coordinates are exact,
    # so the sum equals the FP64-position sum bit for bit
    pos, mass = dyadic_set(2048)
    T = oracle_lib.Tree(pos, mass)
    a64, p64, _, _ = T.forces(32, 0.0, 0.01)
    a32, p32, _, _ = T.forces(32, 0.0, 0.01, coords32=True)
    assert np.array_equal(a64, a32) and np.array_equal(p64, p32)
    # general input: differs only by FP32 representation of the coordinates
    ps = nbsynth.plummer(4000, 3)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    a64, _, _, _, am = T.forces(64, 0.75, 1 / 64, with_amag=True)
    a32, _, _, _ = T.forces(64, 0.75, 1 / 64, coords32=True)
    d = np.linalg.norm(a64 - a32, axis=1)
    assert np.all(d <= 1e-5 * am) and np.median(d / am) < 1e-7
    assert not np.array_equal(a64, a32)


# ---- Peano-Hilbert keys (the alternative order of Sec. "Test and
# Optimization"), pinned by the defining properties of the curve

def _level_cells(lv):
    g = np.arange(1 << lv)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)


@pytest.mark.parametrize("lv", [1, 2, 3, 4])
def test_hilbert_keys_visit_every_cell_once_through_faces(oracle_lib, lv):
    """At every level the top 3 lv key bits order the 8^lv cells as one path
    from the origin that enters each cell once and steps across one face at
    a time."""
    L = 21
    c = _level_cells(lv)
    k = oracle_lib.hilbert_keys((c << (L - lv)).astype(np.int32))
    top = (k >> np.uint64(3 * (L - lv))).astype(np.int64)
    assert np.array_equal(np.sort(top), np.arange(8 ** lv))
    path = c[np.argsort(top)]
    assert np.array_equal(path[0], [0, 0, 0])
    assert np.all(np.abs(np.diff(path, axis=0)).sum(1) == 1)


def test_hilbert_keys_adjacent_at_full_resolution(oracle_lib):
    """Around random grid points: the keys one above and one below a point's
    key belong to two of its six face neighbours."""
    L = 21
    rng = np.random.default_rng(11)
    q = rng.integers(1, (1 << L) - 1, (300, 3)).astype(np.int32)
    k = oracle_lib.hilbert_keys(q).astype(np.int64)
    steps = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    nb = oracle_lib.hilbert_keys((q[:, None, :] + steps[None]).reshape(-1, 3).astype(np.int32))
    nb = nb.astype(np.int64).reshape(-1, 6)
    for i in range(len(q)):
        assert k[i] + 1 in nb[i] and k[i] - 1 in nb[i]


def test_hilbert_keys_nest_by_level(oracle_lib):
    """Points of one aligned sub-cube at level lv share their top 3 lv key
    bits, so each sub-cube is one contiguous key range (what the tree build
    needs of any key order)."""
    L = 21
    rng = np.random.default_rng(12)
    for lv in (1, 3, 7, 12, 20):
        base = rng.integers(0, 1 << lv, (40, 3)) << (L - lv)
        off = rng.integers(0, 1 << (L - lv), (40, 5, 3))
        q = (base[:, None, :] + off).reshape(-1, 3).astype(np.int32)
        top = oracle_lib.hilbert_keys(q) >> np.uint64(3 * (L - lv))
        assert np.all(top.reshape(40, 5) == top.reshape(40, 5)[:, :1])


# ---- the oracle's tree in Peano-Hilbert order: the same octree, its nodes
# visited in another order

def _node_ids(T):
    """A name for every node that does not depend on the visiting order:
    (level, corner) for cells, the caller index for particles."""
    e = T.export()
    c = T.corners()
    out = []
    for u in range(T.nnodes):
        if e["is_cell"][u]:
            out.append(("c", int(e["level"][u]), *map(int, c[u])))
        else:
            out.append(("p", int(e["order"][e["first"][u]])))
    return out


@pytest.fixture(scope="module")
def two_orders(oracle_lib):
    pos, mass = clustered_small()
    return (oracle_lib.Tree(pos, mass), oracle_lib.Tree(pos, mass, order="hilbert"))


def test_hilbert_tree_has_the_same_cells_and_members(two_orders):
    TM, TH = two_orders
    assert TM.nnodes == TH.nnodes and TM.ncells == TH.ncells
    em, eh = TM.export(), TH.export()
    im, ih = _node_ids(TM), _node_ids(TH)
    assert sorted(im) == sorted(ih)
    where = {k: u for u, k in enumerate(im)}
    for u, k in enumerate(ih):
        v = where[k]
        assert eh["count"][u] == em["count"][v] and eh["nchild"][u] == em["nchild"][v]
        assert eh["l"][u] == em["l"][v]
        mh = np.sort(eh["order"][eh["first"][u]: eh["first"][u] + eh["count"][u]])
        mm = np.sort(em["order"][em["first"][v]: em["first"][v] + em["count"][v]])
        assert np.array_equal(mh, mm)
        # the masses and first moments are the same sums in another order
        assert eh["M"][u] == pytest.approx(em["M"][v], rel=1e-14)
        assert np.allclose(eh["com"][u], em["com"][v], rtol=0, atol=1e-13 * TM.L)


def test_hilbert_leaf_order_is_sorted_hilbert_key_order(oracle_lib, two_orders):
    """Depth-first leaf order = particles sorted by Peano-Hilbert key, ties
    (particles in one depth-21 bucket) in input order."""
    TM, TH = two_orders
    e = TH.export()
    k = oracle_lib.hilbert_keys(e["q"])
    assert np.array_equal(e["order"], np.argsort(k, kind="stable"))
    assert not np.array_equal(e["order"], TM.export()["order"])   # a different order


@pytest.mark.parametrize("theta", [0.0, 0.6, 1.0])
def test_hilbert_lists_walk_the_same_cells(two_orders, theta):
    """The recursive and iterative walks agree in Hilbert order too, and a
    group's list names the same cells and particles as in Morton order."""
    TM, TH = two_orders
    im, ih = _node_ids(TM), _node_ids(TH)
    gm, bm, om, lm = TM.all_lists(32, theta)
    gh, bh, oh, lh = TH.all_lists(32, theta)
    assert sorted(im[u] for u in gm) == sorted(ih[u] for u in gh)
    where = {im[u]: g for g, u in enumerate(gm)}
    rng = np.random.default_rng(3)
    for g in rng.choice(len(gh), min(30, len(gh)), replace=False):
        lst = lh[oh[g]: oh[g + 1]]
        assert np.array_equal(lst, TH.walk_group(gh[g], bh[g], theta, mode=0))
        assert np.all(np.diff(lst) > 0)
        gmo = where[ih[gh[g]]]
        assert np.array_equal(bh[g], bm[gmo])
        assert sorted(ih[u] for u in lst) == sorted(im[u] for u in lm[om[gmo]: om[gmo + 1]])


def test_hilbert_forces_match_morton(two_orders):
    TM, TH = two_orders
    am, pm, ppm, pcm = TM.forces(32, 0.6, 1e-3)
    ah, ph, pph, pch = TH.forces(32, 0.6, 1e-3)
    assert (ppm, pcm) == (pph, pch)
    scale = np.linalg.norm(am, axis=1).max()
    assert np.abs(ah - am).max() <= 1e-12 * scale
    assert np.abs(ph - pm).max() <= 1e-12 * np.abs(pm).max()
