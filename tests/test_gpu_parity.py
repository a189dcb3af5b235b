"""CUDA path vs the CPU oracle on the same seeded inputs.

Bit-exact: sorted order, tree topology, FP64 moments, l, s, groups, group
boxes and every interaction list.  The CUDA walk is breadth-first and leaves
the group's own particles to the force kernel, so each GPU list, sorted, must
equal the oracle's depth-first list (ascending node ids) minus the group's
own particles, which must all be in the oracle's list.

Forces, for every particle:
* arithmetic parity against the oracle's FP64 sum over the same lists and the
  same group-relative FP32 coordinates and FP32 masses (oracle coords32
  mode): the bar is 1e-5 relative for plain FP32 sums and 1e-6 for
  compensated (or FP64-accumulated) sums.  A rounded sum's error scales with
  the sum of its terms' magnitudes, A_i = sum_j |a_ij|, not with |a_i|
  (which cancellation can make arbitrarily small), so the bound is
  |a_i(gpu) - a_i(oracle)| <= tol * A_i; every potential (a sum of
  same-signed terms) must be within tol relative;
* against the oracle's FP64 sum over the exact FP64 positions, which adds
  the FP32 coordinate representation: the median of |da|/|a| is at most a
  tenth of tol and the potential within 10 tol.
"""
import numpy as np
import pytest

import nbsynth
from tests.gpu_common import gpu_run, oracle_external_lists, oracle_tree_arrays, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def clump_set(n=6000, seed=3):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1, 1, (n, 3))
    pos[: n // 10] = 0.3 + 1e-5 * rng.normal(size=(n // 10, 3))
    pos[n // 10: n // 10 + 7] = pos[n // 10 + 7]
    pos[-3:] = pos[-4]
    mass = rng.uniform(0.5, 1.5, n).astype(np.float32)
    return pos, mass


CASES = {
    "plummer16k": lambda: (nbsynth.plummer(16384, nbsynth.BASE_SEED + 1), 0.75, 64, 1 / 64),
    "cube4097": lambda: (nbsynth.uniform_cube(4097, 11), 0.6, 32, 1e-3),
    "cosmo12345": lambda: (nbsynth.clustered_cosmo(12345, 13, n_halos=20,
                                                   mlo=1e-3, mhi=1e-2), 0.75, 256, 1e-3),
    "halomix20000": lambda: (nbsynth.halo_mix(20000, 14, n_halos=50), 0.6, 128, 5e-4),
}


def assert_tree_equal(g, T):
    o = oracle_tree_arrays(T)
    t = g["tree"]
    assert np.array_equal(t["perm"], o["perm"])
    for k in ("level", "first", "count", "next", "parent", "nchild"):
        assert np.array_equal(t[k], o[k]), k
    cell = o["is_cell"] == 1
    assert np.array_equal(t["M"], o["M"])
    assert np.array_equal(t["com"], o["com"])
    assert np.array_equal(t["l"][cell], o["l"][cell])
    assert np.array_equal(t["s"][cell], o["s"][cell])
    assert np.array_equal(t["root"][:3], T.centre) and t["root"][3] == T.L
    assert np.array_equal(t["root"][4:7], T.corner)


def assert_lists_equal(g, T, theta, n_crit):
    gnode, box, off, ent, own = oracle_external_lists(T, n_crit, theta)
    gg = g["groups"]
    assert np.array_equal(gg["gnode"], gnode)
    assert np.array_equal(gg["box"], box)
    e = T.export()
    assert np.array_equal(gg["gfirst"], e["first"][gnode])
    assert np.array_equal(gg["gcount"], e["count"][gnode])
    assert np.array_equal(own, e["count"][gnode])      # own particles all in the list
    if theta > 0:
        assert np.all(gg["invtheta"] == np.float32(1.0 / theta))
    else:
        assert np.all(np.isinf(gg["invtheta"]))
    L = g["lists"]
    assert np.array_equal(L["offsets"], off)
    xm = L["xm"]
    for k in range(len(gnode)):
        a, b = off[k], off[k + 1]
        order = np.argsort(L["entries"][a:b], kind="stable")
        assert np.array_equal(L["entries"][a:b][order], ent[a:b])
        xm[a:b] = xm[a:b][order]
    # FP32 source records: group-relative position within 2 ulp, exact mass
    gid = np.repeat(np.arange(len(gnode)), np.diff(off))
    rel = e["com"][ent] - box[gid, 6:9].astype(np.float64)
    assert np.all(np.abs(xm[:, :3] - rel) <= 2.0 ** -22 * np.abs(rel) + 1e-45)
    assert np.array_equal(xm[:, 3], e["M"][ent].astype(np.float32))


@pytest.mark.parametrize("name", list(CASES))
def test_tree_groups_lists_bit_exact(oracle_lib, name):
    ps, theta, n_crit, eps = CASES[name]()
    g = gpu_run(ps.pos, ps.mass, theta=theta, n_crit=n_crit, eps=eps)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    assert_tree_equal(g, T)
    assert_lists_equal(g, T, theta, n_crit)
    st = g["stats"]
    _, _, npp, npc = T.forces(n_crit, theta, eps, gsel=np.zeros(0, np.int64))
    a, p, npp, npc = T.forces(n_crit, theta, eps)
    assert st["n_pp"] == npp and st["n_pc"] == npc
    assert st["n_cells"] == T.ncells and st["n_nodes"] == T.nnodes


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp32_comp", 1e-6),
                                           ("fp64acc", 1e-6)])
def test_forces_within_tolerance(oracle_lib, name, precision, tol):
    ps, theta, n_crit, eps = CASES[name]()
    g = gpu_run(ps.pos, ps.mass, theta=theta, n_crit=n_crit, eps=eps,
                precision=precision, lists=False)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    a32, p32, _, _, amag = T.forces(n_crit, theta, eps, with_amag=True, coords32=True)
    a64, p64, _, _ = T.forces(n_crit, theta, eps)
    d = np.linalg.norm(g["acc"].astype(np.float64) - a32, axis=1)
    ep = np.abs(g["pot"] - p32) / np.abs(p32)
    ea = rel_err(g["acc"], a64)
    ep64 = np.abs(g["pot"] - p64) / np.abs(p64)
    # the literal per-particle bar |da_i| / |a_i| <= tol, and how far the
    # particles that miss it are from cancellation (A_i / |a_i|)
    amod = np.linalg.norm(a32, axis=1)
    lit = d / np.where(amod > 0, amod, 1.0)
    miss = lit > tol
    print(f"{name} {precision}: |da|/A max {(d / amag).max():.2e}, pot max {ep.max():.2e}; "
          f"vs FP64 positions |da|/|a| median {np.median(ea):.2e} p99.9 "
          f"{np.percentile(ea, 99.9):.2e}, pot max {ep64.max():.2e}; literal |da|/|a| <= tol "
          f"for {1.0 - miss.mean():.6f} of particles, max A/|a| among the rest "
          f"{(amag[miss] / amod[miss]).max() if miss.any() else 0.0:.3g}")
    assert np.all(d <= tol * amag)
    assert np.all(ep <= tol)
    assert np.median(ea) <= tol / 10
    assert np.all(ep64 <= 10 * tol)


def test_edge_sizes(oracle_lib):
    rng = np.random.default_rng(8)
    # 3071..3073 and 4095, 4096 straddle the radix sort's tiles (3072 keys in the
    # context's single-pass sort, 4096 in the caller-buffer sort)
    for n in (1, 2, 3, 31, 33, 64, 65, 3071, 3072, 3073, 4095, 4096):
        pos = rng.normal(size=(n, 3))
        mass = rng.uniform(0.5, 2, n).astype(np.float32)
        for n_crit in (1, 8, 4096):
            g = gpu_run(pos, mass, theta=0.7, n_crit=n_crit, eps=0.05, max_n=5000)
            T = oracle_lib.Tree(pos, mass)
            assert_tree_equal(g, T)
            assert_lists_equal(g, T, 0.7, n_crit)
            a, p, _, _, am = T.forces(n_crit, 0.7, 0.05, with_amag=True, coords32=True)
            if n == 1:
                assert np.all(g["acc"] == 0) and g["pot"][0] == 0
            else:
                d = np.linalg.norm(g["acc"].astype(np.float64) - a, axis=1)
                assert np.all(d <= 1e-5 * am)


def test_coincident_particles_and_zero_softening(oracle_lib):
    pos, mass = clump_set()
    for eps in (0.0, 1e-4):
        g = gpu_run(pos, mass, theta=0.6, n_crit=16, eps=eps)
        T = oracle_lib.Tree(pos, mass)
        assert_tree_equal(g, T)
        assert_lists_equal(g, T, 0.6, 16)
        a, p, _, _, am = T.forces(16, 0.6, eps, with_amag=True, coords32=True)
        assert np.all(np.isfinite(g["acc"])) and np.all(np.isfinite(g["pot"]))
        d = np.linalg.norm(g["acc"].astype(np.float64) - a, axis=1)
        assert np.all(d <= 1e-5 * am)
        assert np.all(np.abs(g["pot"] - p) <= 1e-5 * np.abs(p))


@pytest.mark.parametrize("order", ["morton", "hilbert"])
def test_level21_bucket_of_more_than_eight_coincident_particles(oracle_lib, order):
    """A level-21 cell keeps all its coincident particles as children (here
    40 at one point and 9 at another): topology, moments, lists and forces
    against the oracle, with the bucket as a group (n_crit 64) and split into
    one-particle groups (n_crit 16)."""
    ps = nbsynth.uniform_cube(5000, 23)
    pos = ps.pos.copy()
    pos[1000:1040] = pos[3]
    pos[2000:2009] = pos[4000]
    for n_crit in (16, 64):
        for eps in (0.0, 1e-3):
            g = gpu_run(pos, ps.mass, theta=0.6, n_crit=n_crit, eps=eps, key_order=order)
            T = oracle_lib.Tree(pos, ps.mass, order=order)
            assert_tree_equal(g, T)
            assert_lists_equal(g, T, 0.6, n_crit)
            assert int(g["tree"]["nchild"].max()) == 41
            a, p, _, _, am = T.forces(n_crit, 0.6, eps, with_amag=True, coords32=True)
            d = np.linalg.norm(g["acc"].astype(np.float64) - a, axis=1)
            assert np.all(np.isfinite(g["acc"])) and np.all(d <= 1e-5 * am)
            g["ctx"].close()


def test_theta_zero_is_direct_sum(oracle_lib):
    ps = nbsynth.plummer(3000, 4)
    eps = 1 / 64
    g = gpu_run(ps.pos, ps.mass, theta=0.0, n_crit=64, eps=eps, precision="fp32_comp")
    T = oracle_lib.Tree(ps.pos, ps.mass)
    a32, p32, _, _, am = T.forces(64, 0.0, eps, with_amag=True, coords32=True)
    ad, pd = oracle_lib.direct(ps.pos, ps.mass, eps)
    assert g["stats"]["n_pc"] == 0 and g["stats"]["n_pp"] == ps.n * (ps.n - 1)
    d = np.linalg.norm(g["acc"].astype(np.float64) - a32, axis=1)
    assert np.all(d <= 1e-6 * am)
    assert np.all(np.abs(g["pot"] - p32) <= 1e-6 * np.abs(p32))
    assert np.median(rel_err(g["acc"], ad)) < 1e-7


def test_ncrit_one_is_per_particle_walk(oracle_lib):
    ps = nbsynth.plummer(2000, 5)
    g = gpu_run(ps.pos, ps.mass, theta=0.8, n_crit=1, eps=1 / 64)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    L = g["lists"]
    e = T.export()
    gn = g["groups"]["gnode"]
    for k in range(0, ps.n, 97):
        slot = e["first"][gn[k]]
        ref = T.walk_particle(slot, 0.8)
        ref = ref[ref != gn[k]]           # the group's own particle
        got = np.sort(L["entries"][L["offsets"][k]:L["offsets"][k + 1]])
        assert np.array_equal(got, ref)


def test_direct_sum_judge(oracle_lib):
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.halo_mix(30000, 21, n_halos=40)
    eps = 5e-4
    tg = np.random.default_rng(1).choice(ps.n, 300, replace=False)
    ad, pd = oracle_lib.direct(ps.pos, ps.mass, eps, targets=tg)
    dev = torch.device("cuda")
    acc, pot = nb.direct_sum(torch.from_numpy(ps.pos).to(dev),
                             torch.from_numpy(ps.mass).to(dev), eps,
                             torch.from_numpy(tg).to(dev))
    assert np.max(rel_err(acc.cpu().numpy(), ad)) < 1e-12
    assert np.max(np.abs(pot.cpu().numpy() - pd) / np.abs(pd)) < 1e-12


def test_nonfinite_position_is_reported():
    import paper_0909_0541_gb300 as nb
    pos = np.random.default_rng(0).normal(size=(100, 3))
    pos[17, 1] = np.nan
    dev = torch.device("cuda")
    ctx = nb.NBody(100)
    with pytest.raises(nb.NBError) as ei:
        ctx.build_tree(torch.from_numpy(pos).to(dev),
                       torch.ones(100, dtype=torch.float32, device=dev))
    assert ei.value.code == -5


def test_call_order_and_arguments():
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    ctx = nb.NBody(10)
    acc = torch.zeros((10, 3), dtype=torch.float32, device=dev)
    with pytest.raises(nb.NBError) as ei:
        ctx.walk_groups(0.5, 8)
    assert ei.value.code == -6
    with pytest.raises(nb.NBError) as ei:
        ctx.forces(0.1, acc)
    assert ei.value.code == -6
    pos = torch.zeros((11, 3), dtype=torch.float64, device=dev)
    with pytest.raises(nb.NBError) as ei:
        ctx.build_tree(pos, torch.ones(11, dtype=torch.float32, device=dev))
    assert ei.value.code == -1


def test_list_storage_sized_by_counting_walk():
    """The first synchronising walk of a context only counts, so the list
    storage is allocated once: capacity = longest list + 1/4, in 256s."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(16384, 5)
    dev = torch.device("cuda")
    P = torch.from_numpy(ps.pos).to(dev)
    M = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=1 / 64, theta=0.75, n_crit=64)
    ctx.build_tree(P, M)
    ctx.walk_groups(0.75, 64)
    st = ctx.stats()
    need = st["max_list"]
    assert st["list_capacity"] == max(256, (need + need // 4 + 255) // 256 * 256)
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device=dev)
    ctx.forces(1 / 64, acc)
    ctx.sync_status()
    assert bool(torch.isfinite(acc).all())


def test_bounded_wait_gives_up_and_context_survives(oracle_lib):
    """The bottom-up moments make a warp wait for other warps' cells.  The
    wait is bounded: a warp waiting on a count that nothing raises gives up
    after the poll limit and latches NB_ERR_INTERNAL (-8), and the context
    then builds a tree that still matches the oracle bit for bit."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(3000, 21)
    dev = torch.device("cuda")
    ctx = nb.NBody(ps.n)
    assert ctx.selftest_wait(2000) == -8
    ctx.build_tree(torch.from_numpy(ps.pos).to(dev), torch.from_numpy(ps.mass).to(dev))
    ctx.sync_status()
    assert_tree_equal(dict(tree=ctx.copy_tree()), oracle_lib.Tree(ps.pos, ps.mass))


@pytest.mark.parametrize("name", list(CASES))
def test_fused_walk_force_equals_list_path(name):
    """The fused walk-and-force pass (no lists in device memory) sums the same
    sources in the same 32-record tiles as the list path: accelerations,
    potentials and interaction counts agree bit for bit."""
    import paper_0909_0541_gb300 as nb
    ps, theta, n_crit, eps = CASES[name]()
    g = gpu_run(ps.pos, ps.mass, theta=theta, n_crit=n_crit, eps=eps, lists=False)
    dev = torch.device("cuda")
    ctx = nb.NBody(ps.n)
    ctx.build_tree(torch.from_numpy(ps.pos).to(dev), torch.from_numpy(ps.mass).to(dev))
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device=dev)
    pot = torch.zeros(ps.n, dtype=torch.float32, device=dev)
    ctx.forces_fused(theta, n_crit, eps, acc, pot)
    st = ctx.stats()
    assert np.array_equal(acc.cpu().numpy(), g["acc"])
    assert np.array_equal(pot.cpu().numpy(), g["pot"])
    assert st["n_pp"] == g["stats"]["n_pp"] and st["n_pc"] == g["stats"]["n_pc"]
    with pytest.raises(nb.NBError) as ei:   # no lists were left behind
        ctx.forces(eps, acc)
    assert ei.value.code == -6


def test_fused_pass_against_oracle_at_theta_above_zero(oracle_lib):
    """The fused pass compared directly with the oracle (not only with the list
    path) at theta 0.6: the coords32 FP64 sum over the oracle's lists, at the
    FP32 bar 1e-5 of sum_j |a_ij|, and the same interaction counts."""
    import paper_0909_0541_gb300 as nb
    ps, theta, n_crit, eps = CASES["halomix20000"]()
    dev = torch.device("cuda")
    ctx = nb.NBody(ps.n)
    ctx.build_tree(torch.from_numpy(ps.pos).to(dev), torch.from_numpy(ps.mass).to(dev))
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device=dev)
    pot = torch.zeros(ps.n, dtype=torch.float32, device=dev)
    ctx.forces_fused(theta, n_crit, eps, acc, pot)
    st = ctx.stats()
    T = oracle_lib.Tree(ps.pos, ps.mass)
    a32, p32, npp, npc, am = T.forces(n_crit, theta, eps, with_amag=True, coords32=True)
    assert (st["n_pp"], st["n_pc"]) == (npp, npc)
    d = np.linalg.norm(acc.cpu().numpy().astype(np.float64) - a32, axis=1)
    assert np.all(d <= 1e-5 * am)
    assert np.all(np.abs(pot.cpu().numpy() - p32) <= 1e-5 * np.abs(p32))
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32_comp", "fp64acc"])
def test_fused_precision_modes_equal_list_path(precision):
    import paper_0909_0541_gb300 as nb
    ps, theta, n_crit, eps = CASES["halomix20000"]()
    g = gpu_run(ps.pos, ps.mass, theta=theta, n_crit=n_crit, eps=eps, precision=precision,
                lists=False)
    dev = torch.device("cuda")
    ctx = nb.NBody(ps.n)
    ctx.build_tree(torch.from_numpy(ps.pos).to(dev), torch.from_numpy(ps.mass).to(dev))
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device=dev)
    ctx.forces_fused(theta, n_crit, eps, acc, None, precision)
    assert np.array_equal(acc.cpu().numpy(), g["acc"])


def test_fused_leapfrog_steps_equal_list_steps():
    """nb_set_fused: leapfrog steps through the fused pass give the same bits
    as through lists, eager and captured in a CUDA graph."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(16384, nbsynth.BASE_SEED + 1)
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    out = []
    for fused in (False, True):
        P = torch.from_numpy(ps.pos).to(dev)
        V = torch.from_numpy(ps.vel).to(dev)
        M = torch.from_numpy(ps.mass).to(dev)
        stream.wait_stream(torch.cuda.current_stream())
        ctx = nb.NBody(ps.n, eps=1 / 64, theta=0.75, n_crit=64, stream=stream)
        ctx.set_fused(fused)
        with torch.cuda.stream(stream):
            ctx.leapfrog_step(P, V, M, 1 / 128)
            ctx.set_sync_checks(False)
            ctx.graph_capture_leapfrog(P, V, M, 1 / 128, 3)
            ctx.graph_launch()
            ctx.leapfrog_step(P, V, M, 1 / 128)
            stream.synchronize()
            ctx.sync_status()
        out.append((P.cpu().numpy(), V.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_wide_frontier_grows_the_walk_queues(oracle_lib):
    """theta = 0 opens every cell, so on a 40,000-particle cube a frontier
    holds all 32,768 nodes of depth 5: more than the 4096-entry queues a
    context of this size starts with.  The walk reports the overflow, the
    queues grow and the walk is redone; the list path and the fused pass
    then both reproduce the direct sum."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.uniform_cube(40000, 17)
    dev = torch.device("cuda")
    P = torch.from_numpy(ps.pos).to(dev)
    M = torch.from_numpy(ps.mass).to(dev)
    eps = 1e-3
    ctx = nb.NBody(ps.n)
    ctx.build_tree(P, M)
    ctx.walk_groups(0.0, 4096)
    st = ctx.stats()
    assert st["list_entries"] == sum(ps.n - c for c in ctx.copy_groups()["gcount"])
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device=dev)
    ctx.forces(eps, acc)
    fresh = nb.NBody(ps.n)   # the fused pass grows its own context's queues
    fresh.build_tree(P, M)
    accf = torch.zeros_like(acc)
    fresh.forces_fused(0.0, 4096, eps, accf)
    assert torch.equal(acc, accf)
    tg = np.random.default_rng(3).choice(ps.n, 400, replace=False)
    ad, _, am = oracle_lib.direct(ps.pos, ps.mass, eps, tg, with_amag=True)
    d = np.linalg.norm(acc.cpu().numpy()[tg].astype(np.float64) - ad, axis=1)
    assert np.all(d <= 1e-5 * am)
