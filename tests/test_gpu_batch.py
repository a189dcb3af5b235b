"""Batches of independent systems as one forest, CUDA-graph replay of
leapfrog steps, and the autotuner."""
import numpy as np
import pytest

import nbsynth
from tests.gpu_common import oracle_tree_arrays, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def batch(nsys=12, seed=5, lo=64, hi=3000):
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(lo), np.log(hi), nsys)).astype(int)
    ns[0] = 1                                    # a one-particle system
    systems = [(nbsynth.plummer if k % 2 == 0 else nbsynth.hernquist)(int(m), 100 + k)
               if m > 1 else nbsynth.two_body(1.0) for k, m in enumerate(ns)]
    systems[0] = nbsynth.ParticleSet(systems[0].pos[:1], systems[0].vel[:1],
                                     systems[0].mass[:1], "one")
    off = np.r_[0, np.cumsum([s.n for s in systems])].astype(np.int64)
    pos = np.concatenate([s.pos for s in systems])
    vel = np.concatenate([s.vel for s in systems])
    mass = np.concatenate([s.mass for s in systems])
    return systems, off, pos, vel, mass


def test_forest_matches_per_system_oracle(oracle_lib):
    import paper_0909_0541_gb300 as nb
    systems, off, pos, vel, mass = batch()
    dev = torch.device("cuda")
    eps, theta, n_crit = 1 / 64, 0.7, 32
    ctx = nb.NBody(len(pos), eps=eps, theta=theta, n_crit=n_crit, max_systems=len(systems))
    ctx.build_tree_batched(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                           torch.from_numpy(off).to(dev))
    ctx.walk_groups(theta, n_crit)
    acc = torch.empty((len(pos), 3), dtype=torch.float32, device=dev)
    ctx.forces(eps, acc)
    acc = acc.cpu().numpy()
    t = ctx.copy_tree()
    gg = ctx.copy_groups()
    node0 = 0
    for s, ps in enumerate(systems):
        T = oracle_lib.Tree(ps.pos, ps.mass)
        o = oracle_tree_arrays(T)
        nn = T.nnodes
        sl = slice(node0, node0 + nn)
        assert np.array_equal(t["perm"][off[s]:off[s + 1]] - off[s], o["perm"])
        assert np.array_equal(t["first"][sl] - off[s], o["first"])
        for k in ("level", "count", "nchild"):
            assert np.array_equal(t[k][sl], o[k]), (s, k)
        par = t["parent"][sl]
        assert np.array_equal(np.where(par >= 0, par - node0, -1), o["parent"])
        nxt = t["next"][sl]
        nxt = np.where((nxt < 0) | (nxt >= node0 + nn), -1, nxt - node0)
        assert np.array_equal(nxt, o["next"])
        assert np.array_equal(t["M"][sl], o["M"]) and np.array_equal(t["com"][sl], o["com"])
        assert np.array_equal(t["root"][8 * s:8 * s + 3], T.centre) and t["root"][8 * s + 3] == T.L
        # groups and lists of this system
        mine = np.flatnonzero((gg["gfirst"] >= off[s]) & (gg["gfirst"] < off[s + 1]))
        gnode = T.groups(n_crit)
        assert np.array_equal(gg["gnode"][mine] - node0, gnode)
        box = T.group_boxes(gnode)
        assert np.array_equal(gg["box"][mine], box)
        e = T.export()
        leaf = np.flatnonzero(e["is_cell"] == 0)
        for k, g in enumerate(mine):
            ref = T.walk_group(gnode[k], box[k], theta)
            f, c = e["first"][gnode[k]], e["count"][gnode[k]]
            ref = ref[~np.isin(ref, leaf[f:f + c])]
            ids, _ = ctx.copy_list(g)
            assert np.array_equal(np.sort(ids) - node0, ref)
        a32, _, _, _, am = T.forces(n_crit, theta, eps, with_amag=True, coords32=True)
        d = np.linalg.norm(acc[off[s]:off[s + 1]].astype(np.float64) - a32, axis=1)
        assert np.all(d <= 1e-5 * np.maximum(am, 1e-300))
        node0 += nn
    assert node0 == ctx.stats()["n_nodes"]


def test_batched_leapfrog_and_graph_replay(oracle_lib):
    import paper_0909_0541_gb300 as nb
    systems, off, pos, vel, mass = batch(16, 9, 200, 2000)
    dev = torch.device("cuda")
    eps, theta, n_crit, dt = 1 / 64, 0.6, 64, 1 / 128
    P = torch.from_numpy(pos).to(dev)
    V = torch.from_numpy(vel).to(dev)
    M = torch.from_numpy(mass).to(dev)
    O = torch.from_numpy(off).to(dev)
    s = torch.cuda.Stream()
    ctx = nb.NBody(len(pos), eps=eps, theta=theta, n_crit=n_crit, max_systems=16, stream=s)
    with torch.cuda.stream(s):
        ctx.leapfrog_step_batched(P, V, M, O, dt)
    s.synchronize()
    for k, ps in enumerate(systems):
        xo, vo, ao = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, eps, dt, 1, use_tree=True,
                                         theta=theta, n_crit=n_crit)
        amax = np.abs(ao).max() if len(ao) > 1 else 1.0
        assert np.max(np.abs(P.cpu().numpy()[off[k]:off[k + 1]] - xo)) <= dt * dt * 1e-4 * amax + 1e-15
    # eager reference: a second context runs 1 + 6 steps from the same start
    P2 = torch.from_numpy(pos).to(dev)
    V2 = torch.from_numpy(vel).to(dev)
    ctx2 = nb.NBody(len(pos), eps=eps, theta=theta, n_crit=n_crit, max_systems=16, stream=s)
    with torch.cuda.stream(s):
        for _ in range(7):
            ctx2.leapfrog_step_batched(P2, V2, M, O, dt)
        # the first context: capture 3 steps after its first and replay twice
        ctx.graph_capture_leapfrog(P, V, M, dt, 3, offsets=O)
        ctx.graph_launch()
        ctx.graph_launch()
        ctx.sync_status()
    s.synchronize()
    assert torch.equal(P, P2) and torch.equal(V, V2)


def test_autotune_picks_a_candidate():
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(50000, 3)
    dev = torch.device("cuda")
    P = torch.from_numpy(ps.pos).to(dev)
    M = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=1 / 64, theta=0.7)
    pick, table = ctx.autotune(P, M, 1 / 64, 0.7, n_crits=(16, 64, 256), reps=2)
    best = pick["n_crit"]
    assert best in (16, 64, 256) and pick["rows"] in (1, 2)
    assert pick["tile"] in (32, 64) and pick["block"] in (256, 128)
    assert len(table) == 3 * 8
    assert table[(best, pick["rows"], pick["tile"], pick["block"])] == min(table.values())
    # the chosen force shape gives the same accelerations as the default one
    ctx.build_tree(P, M)
    ctx.walk_groups(0.7, best)
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device=dev)
    ctx.forces(1 / 64, acc)
    assert torch.isfinite(acc).all()
    ref = nb.NBody(ps.n, eps=1 / 64, theta=0.7)
    ref.build_tree(P, M)
    ref.walk_groups(0.7, best)
    acc0 = torch.empty_like(acc)
    ref.forces(1 / 64, acc0)
    # 64-target items with 32-record tiles sum in the default order (bit-equal);
    # other shapes split the sources among streams differently
    if pick["rows"] == 2 and pick["tile"] == 32:
        assert torch.equal(acc, acc0)
    else:
        scale = acc0.norm(dim=1).max().item()
        assert (acc - acc0).norm(dim=1).max().item() <= 1e-5 * scale


def test_autotune_a_forest(oracle_lib):
    """The autotuner on a batch: it builds the forest, keeps the fastest
    (n_crit, item width), and a batched step with it still matches every
    system's oracle step."""
    import paper_0909_0541_gb300 as nb
    systems, off, pos, vel, mass = batch(10, 9, 300, 4000)
    dev = torch.device("cuda")
    eps, theta, dt = 1 / 64, 0.6, 1 / 128
    P = torch.from_numpy(pos).to(dev)
    V = torch.from_numpy(vel).to(dev)
    M = torch.from_numpy(mass).to(dev)
    O = torch.from_numpy(off).to(dev)
    ctx = nb.NBody(len(pos), eps=eps, theta=theta, n_crit=64, max_systems=len(systems))
    pick, table = ctx.autotune(P, M, eps, theta, n_crits=(16, 64, 256), reps=2, offsets=O)
    best = pick["n_crit"]
    assert best in (16, 64, 256) and pick["rows"] in (1, 2)
    assert table[(best, pick["rows"], pick["tile"], pick["block"])] == min(table.values())
    ctx.leapfrog_step_batched(P, V, M, O, dt)
    for k, ps in enumerate(systems):
        xo, vo, ao = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, eps, dt, 1, use_tree=True,
                                         theta=theta, n_crit=best)
        amax = np.abs(ao).max() if len(ao) > 1 else 1.0
        assert np.max(np.abs(P.cpu().numpy()[off[k]:off[k + 1]] - xo)) <= dt * dt * 1e-4 * amax + 1e-15
