"""Quadrupole cells on the GPU (nb_set_quadrupole: "any high order moment" of
Sec. "Oct-tree Method") against the oracle's quadrupole tree code.

* Q of every node: the device folds children by the parallel-axis theorem,
  the oracle sums over members by the definition, both in FP64; they agree
  to 1e-10 of M l^2 (the cell's mass times its side squared bounds |Q|).
  Particles have Q = 0 exactly.
* Lists: the same sets of nodes as without quadrupoles (the opening test is
  unchanged), bit-exact against the oracle's walk.
* Forces: against the oracle's FP64 sum with the quadrupole term over the same
  group-relative FP32 coordinates (coords32), at the tree path's bars: 1e-5
  (FP32) and 1e-6 (compensated) of sum_j |a_ij|, potentials relative.
"""
import numpy as np
import pytest

import nbsynth
from tests.gpu_common import oracle_tree_arrays
from tests.test_gpu_parity import CASES, assert_lists_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def run(pos, mass, theta, n_crit, eps, precision="fp32", lists=True):
    import paper_0909_0541_gb300 as nb
    n = pos.shape[0]
    dev = torch.device("cuda")
    p = torch.from_numpy(np.ascontiguousarray(pos, np.float64)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(mass, np.float32)).to(dev)
    ctx = nb.NBody(max(n, 1))
    ctx.set_quadrupole(True)
    ctx.build_tree(p, m)
    ctx.walk_groups(theta, n_crit)
    acc = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    pot = torch.zeros(n, dtype=torch.float32, device=dev)
    ctx.forces(eps, acc, pot, precision)
    out = dict(acc=acc.cpu().numpy().astype(np.float64), pot=pot.cpu().numpy().astype(np.float64),
               stats=ctx.stats(), Q=ctx.copy_quadrupoles())
    if lists:
        out["tree"] = ctx.copy_tree()
        out["groups"] = ctx.copy_groups()
        out["lists"] = ctx.copy_lists(with_xm=True)
    ctx.close()
    return out


def assert_q_close(Q, T):
    e = T.export()
    Qo = T.quadrupoles()
    cell = e["is_cell"] == 1
    assert np.all(Q[~cell] == 0.0)
    scale = e["M"] * e["l"].astype(np.float64) ** 2
    d = np.abs(Q - Qo).max(axis=1)
    assert np.all(d[cell] <= 1e-10 * scale[cell] + 1e-300), float(np.max(d[cell] / scale[cell]))


def pair_and_target():
    """Two equal masses at +-s on the z axis and a light far target on it."""
    pos = np.array([[0.0, 0.0, 0.1], [0.0, 0.0, -0.1], [0.0, 0.0, 3.0]])
    mass = np.array([0.5, 0.5, 1e-6], np.float32)
    return pos, mass


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp32_comp", 1e-6)])
def test_quadrupole_forces_and_lists(oracle_lib, name, precision, tol):
    ps, theta, n_crit, eps = CASES[name]()
    g = run(ps.pos, ps.mass, theta, n_crit, eps, precision, lists=precision == "fp32")
    T = oracle_lib.Tree(ps.pos, ps.mass)
    assert_q_close(g["Q"], T)
    if precision == "fp32":
        assert_lists_equal(g, T, theta, n_crit)
    a, p, npp, npc, am = T.forces_quad(n_crit, theta, eps, with_amag=True, coords32=True)
    assert (g["stats"]["n_pp"], g["stats"]["n_pc"]) == (npp, npc)
    d = np.linalg.norm(g["acc"] - a, axis=1)
    assert np.all(d <= tol * am), float(np.max(d / am))
    assert np.all(np.abs(g["pot"] - p) <= tol * np.abs(p))
    # the quadrupole term is really there: the monopole sum differs by far more
    a0, _, _, _ = T.forces(n_crit, theta, eps, coords32=True)
    assert np.median(np.linalg.norm(a0 - a, axis=1) / am) > 10 * tol


def test_quadrupole_closed_form_far_pair(oracle_lib):
    """A light target far out on the axis of an equal-mass pair (eps 0,
    n_crit 1, the pair's cell accepted): a_z = -2m/d^2 - 6 m s^2 / d^4 and
    phi = -2m/d - 2 m s^2 / d^3 to FP32 rounding."""
    pos, mass = pair_and_target()
    g = run(pos, mass, 1.0, 1, 0.0, lists=False)
    assert g["stats"]["n_pc"] >= 1
    m, s, d = 0.5, 0.1, 3.0
    az = -2 * m / d ** 2 - 6 * m * s ** 2 / d ** 4
    ph = -2 * m / d - 2 * m * s ** 2 / d ** 3
    assert abs(g["acc"][2, 2] - az) <= 1e-6 * abs(az)
    assert abs(g["pot"][2] - ph) <= 1e-6 * abs(ph)
    assert abs(g["acc"][2, 0]) < 1e-12 and abs(g["acc"][2, 1]) < 1e-12


def test_quadrupole_theta_zero_is_direct_sum(oracle_lib):
    ps = nbsynth.uniform_cube(3000, 81)
    g = run(ps.pos, ps.mass, 0.0, 64, 1e-3, "fp32_comp", lists=False)
    a, _, am = oracle_lib.direct(ps.pos, ps.mass, 1e-3, with_amag=True)
    assert g["stats"]["n_pc"] == 0
    assert np.all(np.linalg.norm(g["acc"] - a, axis=1) <= 1e-5 * am)


def test_quadrupole_state_and_arguments():
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(2000, 82)
    dev = torch.device("cuda")
    p = torch.from_numpy(ps.pos).to(dev)
    m = torch.from_numpy(ps.mass).to(dev)
    acc = torch.zeros((ps.n, 3), dtype=torch.float32, device=dev)
    ctx = nb.NBody(ps.n)
    ctx.build_tree(p, m)              # built without quadrupoles
    ctx.set_quadrupole(True)
    with pytest.raises(nb.NBError) as ei:
        ctx.walk_groups(0.6, 64)
    assert ei.value.code == -6        # STATE: rebuild first
    ctx.build_tree(p, m)
    ctx.walk_groups(0.6, 64)
    with pytest.raises(nb.NBError) as ei:
        ctx.forces(0.01, acc, None, "fp64acc")
    assert ei.value.code == -1
    with pytest.raises(nb.NBError) as ei:
        ctx.forces_fused(0.6, 64, 0.01, acc)
    assert ei.value.code == -1
    ctx.forces(0.01, acc)
    ctx.set_quadrupole(False)         # back to the monopole on the same lists
    ctx.forces(0.01, acc)
    ctx.close()


@pytest.mark.slow
def test_quadrupole_full_size_moments_and_sampled_lists(oracle_lib):
    """The 2.87M halo mix: every node's Q against the oracle's, and 32
    sampled groups' lists against the oracle's walk."""
    import paper_0909_0541_gb300 as nb
    ps, w = nbsynth.workload("halomix2.87m")
    theta, n_crit = w["theta"], w["n_crit"]
    dev = torch.device("cuda")
    ctx = nb.NBody(ps.n, n_crit=n_crit)
    ctx.set_quadrupole(True)
    ctx.build_tree(torch.from_numpy(ps.pos).to(dev), torch.from_numpy(ps.mass).to(dev))
    ctx.walk_groups(theta, n_crit)
    Q = ctx.copy_quadrupoles()
    T = oracle_lib.Tree(ps.pos, ps.mass)
    assert_q_close(Q, T)
    e = T.export()
    leaf_of_slot = np.flatnonzero(e["is_cell"] == 0)
    gnode = T.groups(n_crit)
    box = T.group_boxes(gnode)
    for k in np.random.default_rng(7).choice(len(gnode), 32, replace=False):
        ref = T.walk_group(gnode[k], box[k], theta)
        f, c = e["first"][gnode[k]], e["count"][gnode[k]]
        ids, _ = ctx.copy_list(k)
        assert np.array_equal(np.sort(ids), ref[~np.isin(ref, leaf_of_slot[f:f + c])])
    ctx.close()
