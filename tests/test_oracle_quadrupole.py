"""Pins for the oracle's quadrupole cell moments and the quadrupole
particle-cell term (the "any high order moment" remark of Sec. "Oct-tree
Method"; the paper itself uses the monopole).  Q_ab = sum m (3 d_a d_b -
|d|^2 delta_ab) about the centre of mass; the term adds -r.Q.r / (2 R^5) to
the potential and Q r / R^5 - 5 (r.Q.r) r / (2 R^7) to the acceleration,
r = x_i - COM, R^2 = |r|^2 + eps^2."""
import numpy as np
import pytest

import nbsynth

IDX = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4,
       (1, 2): 5, (2, 1): 5}


def full(q):
    return np.array([[q[IDX[a, b]] for b in range(3)] for a in range(3)])


def test_two_body_closed_form(oracle_lib):
    m, s = 0.5, 0.3
    pos = np.array([[0.0, 0.0, s], [0.0, 0.0, -s]])
    T = oracle_lib.Tree(pos, np.array([m, m], np.float32))
    Q = T.quadrupoles()[0]
    assert np.allclose(Q, [-2 * m * s * s, -2 * m * s * s, 4 * m * s * s, 0, 0, 0],
                       rtol=1e-15, atol=1e-17)


def test_traceless_and_parallel_axis(oracle_lib):
    """Every cell's Q is traceless, and equals the sum over its children of
    their Q shifted to the parent's centre of mass (parallel-axis theorem),
    a different route to the same moments."""
    ps = nbsynth.plummer(3000, 6)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    e = T.export()
    Q = T.quadrupoles()
    cells = np.flatnonzero(e["is_cell"] == 1)
    scale = np.abs(Q).max()
    assert np.abs(Q[cells, :3].sum(1)).max() <= 1e-12 * scale
    assert np.all(Q[e["is_cell"] == 0] == 0.0)
    par = e["parent"]
    rng = np.random.default_rng(0)
    for u in rng.choice(cells, 200, replace=False):
        kids = np.flatnonzero(par == u)
        acc = np.zeros((3, 3))
        for c in kids:
            D = e["com"][c] - e["com"][u]
            acc += full(Q[c]) + e["M"][c] * (3 * np.outer(D, D) - D @ D * np.eye(3))
        assert np.allclose(full(Q[u]), acc, rtol=0, atol=1e-11 * scale)


def test_far_two_body_cell_on_axis(oracle_lib):
    """A light target far up the axis of an equal-mass pair sees the pair as
    one cell: its acceleration is the monopole plus quadrupole closed form
    -2m/d^2 - 6 m s^2 / d^4 (eps = 0), and its potential -2m/d - 2 m s^2/d^3."""
    m, s, d = 0.5, 0.3, 100.0
    pos = np.array([[0.0, 0.0, s], [0.0, 0.0, -s], [0.0, 0.0, d]])
    mass = np.array([m, m, 1e-30], np.float32)
    T = oracle_lib.Tree(pos, mass)
    acc, pot, npp, npc = T.forces_quad(1, 1.0, 0.0)
    assert npc >= 1                       # the pair entered as one cell
    assert acc[2, 2] == pytest.approx(-2 * m / d**2 - 6 * m * s * s / d**4, rel=1e-13)
    assert abs(acc[2, 0]) < 1e-20 and abs(acc[2, 1]) < 1e-20
    assert pot[2] == pytest.approx(-2 * m / d - 2 * m * s * s / d**3, rel=1e-13)
    mono = T.forces(1, 1.0, 0.0)[0]
    exact = -m / (d - s) ** 2 - m / (d + s) ** 2
    assert abs(acc[2, 2] - exact) < 0.01 * abs(mono[2, 2] - exact)


def test_quadrupole_lowers_the_tree_error(oracle_lib):
    ps = nbsynth.plummer(4000, 3)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    ad = oracle_lib.direct(ps.pos, ps.mass, 1 / 64)[0]
    norm = np.linalg.norm(ad, axis=1)
    for theta in (0.4, 0.6, 0.8):
        e1 = np.linalg.norm(T.forces(32, theta, 1 / 64)[0] - ad, axis=1) / norm
        e2 = np.linalg.norm(T.forces_quad(32, theta, 1 / 64)[0] - ad, axis=1) / norm
        assert np.median(e2) < 0.5 * np.median(e1)
    a0 = T.forces_quad(32, 0.0, 1 / 64)[0]        # theta 0: no cell is accepted
    assert np.abs(a0 - ad).max() <= 1e-12 * norm.max()
