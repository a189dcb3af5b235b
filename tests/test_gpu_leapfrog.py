"""nb_leapfrog_step against the oracle's FP64 KDK leapfrog with tree forces,
and against the FP64 direct-sum leapfrog on the Plummer 16k configuration
(eps 1/64, theta 0.75, n_crit 64, dt 1/128)."""
import numpy as np
import pytest

import nbsynth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_one_step_plummer16k(oracle_lib):
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(16384, nbsynth.BASE_SEED + 1)
    eps, theta, n_crit, dt = 1.0 / 64, 0.75, 64, 1.0 / 128
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    vel = torch.from_numpy(ps.vel).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit)
    ctx.leapfrog_step(pos, vel, mass, dt)
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device=dev)
    ctx.leapfrog_acc(acc)
    x1, v1, a1 = pos.cpu().numpy(), vel.cpu().numpy(), acc.cpu().numpy()
    xo, vo, ao = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, eps, dt, 1, use_tree=True,
                                     theta=theta, n_crit=n_crit)
    amax = np.abs(ao).max()
    # kicks carry the force error (<= 1e-5 relative of the summed magnitudes)
    assert np.max(np.abs(v1 - vo)) <= dt * 1e-5 * 10 * amax
    assert np.max(np.abs(x1 - xo)) <= dt * dt * 1e-5 * 10 * amax
    # accelerations at the new positions
    assert np.median(np.linalg.norm(a1 - ao, axis=1) / np.linalg.norm(ao, axis=1)) < 1e-6
    # against the FP64 direct-sum step: the tree's own error at theta 0.75
    xd, vd, ad = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, eps, dt, 1)
    err = np.linalg.norm(a1 - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert 1e-4 < np.median(err) < 5e-3
    ctx.close()


def test_many_steps_conserve_energy(oracle_lib):
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(4096, 77)
    eps, theta, n_crit, dt = 1.0 / 64, 0.6, 64, 1.0 / 128
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    vel = torch.from_numpy(ps.vel).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit, sync_checks=True)

    def energy(p, v):
        _, pot = oracle_lib.direct(p, ps.mass, eps)
        m = ps.mass.astype(np.float64)
        return 0.5 * (m * (v ** 2).sum(1)).sum() + 0.5 * (m * pot).sum()

    e0 = energy(ps.pos, ps.vel)
    for _ in range(64):
        ctx.leapfrog_step(pos, vel, mass, dt)
    e1 = energy(pos.cpu().numpy(), vel.cpu().numpy())
    assert abs(e1 - e0) < 2e-3 * abs(e0)
    # reversibility: 64 steps back with negated velocities
    vel.neg_()
    ctx.leapfrog_reset()
    for _ in range(64):
        ctx.leapfrog_step(pos, vel, mass, dt)
    assert np.max(np.abs(pos.cpu().numpy() - ps.pos)) < 1e-4
    ctx.close()


def test_host_buffer_step_equals_device_step():
    """nb_leapfrog_step_host (the library does the copies, positions leave on
    a second stream after the drift) gives the same bits as nb_leapfrog_step
    on device buffers, step after step, with and without synchronising
    checks."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(20000, 31)
    eps, theta, n_crit, dt = 1.0 / 64, 0.75, 64, 1.0 / 128
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    vel = torch.from_numpy(ps.vel).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    a = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit, stream=stream)
    b = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit, stream=stream)
    hpos = torch.from_numpy(ps.pos.copy()).pin_memory()
    hvel = torch.from_numpy(ps.vel.copy()).pin_memory()
    hmass = torch.from_numpy(ps.mass.copy()).pin_memory()
    with torch.cuda.stream(stream):
        for k in range(4):
            if k == 2:
                a.set_sync_checks(False)
                b.set_sync_checks(False)
            a.leapfrog_step(pos, vel, mass, dt)
            b.leapfrog_step_host(hpos, hvel, hmass, dt)
        stream.synchronize()
        a.sync_status()
        b.sync_status()
    assert np.array_equal(pos.cpu().numpy(), hpos.numpy())
    assert np.array_equal(vel.cpu().numpy(), hvel.numpy())
    with pytest.raises(TypeError):
        b.leapfrog_step_host(hpos.float(), hvel, hmass, dt)


def test_graph_replay_times_its_phases_and_equals_eager_steps():
    """Three KDK steps captured in a CUDA graph with timing on: two launches
    give the same bits as six eager steps (inside the graph a step's second
    kick runs with the next step's first kick and drift); nb_get_timing
    reports each phase of the last launch twice (build, walk, force once per
    step; integrate 4 times per launch: the first kick and drift, two joined
    passes, the last kick) and the captured kernels twice; eager phases after
    that are timed on their own."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(20000, 33)
    eps, theta, n_crit, dt = 1.0 / 64, 0.75, 64, 1.0 / 128
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    out = []
    for graph in (False, True):
        pos = torch.from_numpy(ps.pos).to(dev)
        vel = torch.from_numpy(ps.vel).to(dev)
        mass = torch.from_numpy(ps.mass).to(dev)
        stream.wait_stream(torch.cuda.current_stream())
        ctx = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit, stream=stream)
        with torch.cuda.stream(stream):
            ctx.leapfrog_step(pos, vel, mass, dt)
            ctx.set_sync_checks(False)
            if graph:
                ctx.set_timing(True)
                ctx.graph_capture_leapfrog(pos, vel, mass, dt, 3)
                ctx.get_timing()
                ctx.graph_launch()
                ctx.graph_launch()
                tm = ctx.get_timing()
                assert tm["launches"] > 0 and tm["launches"] % 2 == 0
                for phase, calls in (("build", 6), ("walk", 6), ("force", 6),
                                     ("integrate", 8)):
                    assert tm[phase][1] == calls, (phase, tm[phase])
                    assert tm[phase][0] > 0.0
                ctx.leapfrog_step(pos, vel, mass, dt)
                tm = ctx.get_timing()
                assert tm["force"][1] == 1 and tm["integrate"][1] == 2
                assert tm["launches"] > 0
                ctx.set_timing(False)
            else:
                for _ in range(7):
                    ctx.leapfrog_step(pos, vel, mass, dt)
            stream.synchronize()
            ctx.sync_status()
        out.append((pos.cpu().numpy(), vel.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_graph_dropped_when_list_storage_is_reallocated():
    """A captured graph holds the list storage's addresses: a later
    synchronising walk that needs more room reallocates it and must drop the
    graph (replaying it would touch freed memory), so the next launch is
    refused with NB_ERR_STATE and a new capture works."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(6000, 93)
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    vel = torch.from_numpy(ps.vel).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    stream = torch.cuda.Stream(device=dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(stream):
        ctx = nb.NBody(ps.n, eps=1 / 64, theta=0.75, n_crit=64, stream=stream)
        ctx.leapfrog_step(pos, vel, mass, 1 / 128)
        ctx.graph_capture_leapfrog(pos, vel, mass, 1 / 128, 2)
        ctx.graph_launch()
        ctx.sync_status()
        ctx.build_tree(pos, mass)
        ctx.walk_groups(0.0, 64)          # every list holds every particle: more room
        with pytest.raises(nb.NBError) as ei:
            ctx.graph_launch()
        assert ei.value.code == -6        # STATE: capture again
        ctx.leapfrog_reset()
        ctx.leapfrog_step(pos, vel, mass, 1 / 128)
        ctx.graph_capture_leapfrog(pos, vel, mass, 1 / 128, 2)
        ctx.graph_launch()
        ctx.sync_status()
        ctx.close()


@pytest.mark.parametrize("dt,offset", [(1.0 / 128, 0), (0.01, 0), (1.0 / 128, 1)])
def test_kick_and_drift_are_the_fp64_formulas(dt, offset):
    """The kick v + fl64(a) (dt/2) and the drift x + v dt, each operation
    rounded on its own, bit for bit: 16-byte aligned buffers (four components
    per thread and round) and buffers one double off that alignment (one
    component at a time); zero, negative-zero and subnormal velocities
    included."""
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(6000, 41)
    eps, theta, n_crit = 1.0 / 64, 0.7, 64
    v0 = ps.vel.copy()
    v0[:7, 0] = 0.0
    v0[7:14, 1] = -0.0
    v0[14:21, 2] = 3e-310
    v0[21:28, 0] = -2.5e-308
    dev = torch.device("cuda")

    def placed(a):   # a device copy whose data pointer is `offset` doubles past 16-byte alignment
        flat = torch.empty(a.size + offset, dtype=torch.float64, device=dev)
        view = flat[offset:].view(a.shape)
        view.copy_(torch.from_numpy(a))
        assert (view.data_ptr() % 16 == 0) == (offset == 0)
        return view

    pos, vel = placed(ps.pos), placed(v0)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=eps, theta=theta, n_crit=n_crit)
    a0 = torch.empty((ps.n, 3), dtype=torch.float32, device=dev)
    ctx.build_tree(pos, mass)
    ctx.walk_groups(theta, n_crit)
    ctx.forces(eps, a0)
    ctx.leapfrog_step(pos, vel, mass, dt)
    a1 = torch.empty_like(a0)
    ctx.leapfrog_acc(a1)
    h = 0.5 * dt
    vh = v0 + a0.cpu().numpy().astype(np.float64) * h
    x1 = ps.pos + vh * dt
    v1 = vh + a1.cpu().numpy().astype(np.float64) * h
    assert np.array_equal(pos.cpu().numpy(), x1)
    assert np.array_equal(vel.cpu().numpy(), v1)
    ctx.close()
