"""The overlapped walk and force (nb_walk_forces: one persistent launch in
which warps take force items of groups already walked, else the next walk)
gives the same bits as nb_walk_groups + nb_forces: every list and every
item's sums are computed the same way; only the order in which warps take
them changes."""
import numpy as np
import pytest

import nbsynth
from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _ctx(ps, **kw):
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, **kw)
    return ctx, pos, mass


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp32_comp"])
def test_walk_forces_equal_the_separate_calls(name, precision):
    ps, theta, n_crit, eps = CASES[name]()
    ctx, pos, mass = _ctx(ps)
    dev = pos.device
    a0 = torch.zeros((ps.n, 3), dtype=torch.float32, device=dev)
    p0 = torch.zeros(ps.n, dtype=torch.float32, device=dev)
    ctx.build_tree(pos, mass)
    ctx.walk_groups(theta, n_crit)             # sizes the list storage
    ctx.forces(eps, a0, p0, precision)
    s0 = ctx.stats()
    lists0 = ctx.copy_lists()
    a1 = torch.zeros_like(a0)
    p1 = torch.zeros_like(p0)
    ctx.walk_forces(theta, n_crit, eps, a1, p1, precision)
    s1 = ctx.stats()
    assert torch.equal(a0, a1) and torch.equal(p0, p1)
    assert (s0["n_pp"], s0["n_pc"], s0["list_entries"]) == (s1["n_pp"], s1["n_pc"],
                                                             s1["list_entries"])
    lists1 = ctx.copy_lists()
    assert np.array_equal(lists0["offsets"], lists1["offsets"])
    assert np.array_equal(lists0["entries"], lists1["entries"])
    # with the synchronising checks off as well (the mode of captured steps)
    ctx.set_sync_checks(False)
    a2 = torch.zeros_like(a0)
    ctx.walk_forces(theta, n_crit, eps, a2, None, precision)
    ctx.sync_status()
    assert torch.equal(a0, a2)
    ctx.close()


def test_walk_forces_without_list_storage():
    """The first call on a fresh context (no list storage yet): synchronising,
    it walks and sums separately; without synchronising checks it refuses."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(5000, 91)
    ctx, pos, mass = _ctx(ps)
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device=pos.device)
    ctx.build_tree(pos, mass)
    ctx.set_sync_checks(False)
    with pytest.raises(nb.NBError) as ei:
        ctx.walk_forces(0.6, 64, 0.01, acc)
    assert ei.value.code == -3                # CAPACITY
    ctx.set_sync_checks(True)
    ctx.walk_forces(0.6, 64, 0.01, acc)
    ref = torch.zeros_like(acc)
    ctx.walk_groups(0.6, 64)
    ctx.forces(0.01, ref)
    assert torch.equal(acc, ref)
    with pytest.raises(nb.NBError) as ei:
        ctx.walk_forces(0.6, 64, 0.01, acc, None, "fp64acc")
    assert ei.value.code == -1
    ctx.close()


def test_overlapped_leapfrog_steps_equal_plain_steps():
    """Eight KDK steps with the overlapped force passes (synchronising checks
    off after the first) and eight without: the same positions and
    velocities, bit for bit."""
    ps = nbsynth.halo_mix(60000, 92, n_halos=40)
    out = []
    for overlap in (False, True):
        ctx, pos, mass = _ctx(ps, eps=5e-4, theta=0.6, n_crit=128)
        vel = torch.from_numpy(ps.vel).to(pos.device)
        ctx.set_overlap(overlap)
        ctx.leapfrog_step(pos, vel, mass, 1.0 / 1024)
        ctx.set_sync_checks(False)
        for _ in range(7):
            ctx.leapfrog_step(pos, vel, mass, 1.0 / 1024)
        ctx.sync_status()
        out.append((pos.cpu().numpy(), vel.cpu().numpy(), ctx.stats()["n_pp_total"]))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_overlapped_batch_forest():
    """A forest of 24 systems: the overlapped pass equals the separate one."""
    import paper_0909_0541_gb300 as nb
    systems = nbsynth.batched_systems(24)
    off = np.r_[0, np.cumsum([p.n for p in systems])].astype(np.int64)
    pos = np.concatenate([p.pos for p in systems])
    mass = np.concatenate([p.mass for p in systems])
    dev = torch.device("cuda")
    ctx = nb.NBody(len(pos), max_systems=len(systems))
    ctx.build_tree_batched(torch.from_numpy(pos).to(dev), torch.from_numpy(mass).to(dev),
                           torch.from_numpy(off).to(dev))
    a0 = torch.zeros((len(pos), 3), dtype=torch.float32, device=dev)
    ctx.walk_groups(0.75, 64)
    ctx.forces(1 / 64, a0)
    a1 = torch.zeros_like(a0)
    ctx.walk_forces(0.75, 64, 1 / 64, a1)
    assert torch.equal(a0, a1)
    ctx.close()
