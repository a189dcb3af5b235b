"""Pins for the oracle's FP64 kick-drift-kick leapfrog: Kepler orbit closed
form, energy conservation and exact time reversibility."""
import math

import numpy as np

import nbsynth


def energy(pos, vel, mass):
    m = mass.astype(np.float64)
    ke = 0.5 * (m * (vel ** 2).sum(1)).sum()
    d = np.linalg.norm(pos[0] - pos[1])
    return ke - m[0] * m[1] / d


def test_kepler_circular_orbit_period_and_energy(oracle_lib):
    # G (m1 + m2) = 1, separation 1: period 2 pi, closed orbit
    ps = nbsynth.two_body(1.0, 0.3, 0.7)
    nsteps = 4000
    dt = 2 * math.pi / nsteps
    e0 = energy(ps.pos, ps.vel, ps.mass)
    pos, vel, _ = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, 0.0, dt, nsteps)
    assert np.max(np.abs(pos - ps.pos)) < 1e-5
    assert abs(energy(pos, vel, ps.mass) - e0) < 1e-9 * abs(e0)
    # half a period: bodies on the opposite side
    pos2, _, _ = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, 0.0, dt, nsteps // 2)
    assert np.max(np.abs(pos2 + ps.pos)) < 1e-5


def test_time_reversible(oracle_lib):
    ps = nbsynth.plummer(64, 21)
    eps, dt = 0.05, 1.0 / 128
    pos, vel, acc = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, eps, dt, 50)
    pos2, vel2, _ = oracle_lib.leapfrog(pos, -vel, ps.mass, eps, dt, 50, acc=acc)
    assert np.max(np.abs(pos2 - ps.pos)) < 1e-12
    assert np.max(np.abs(-vel2 - ps.vel)) < 1e-12


def test_tree_leapfrog_energy_drift(oracle_lib):
    ps = nbsynth.plummer(2048, nbsynth.BASE_SEED + 1)
    eps, dt = 1.0 / 64, 1.0 / 128

    def etot(p, v):
        _, pot = oracle_lib.direct(p, ps.mass, eps)
        m = ps.mass.astype(np.float64)
        return 0.5 * (m * (v ** 2).sum(1)).sum() + 0.5 * (m * pot).sum()

    e0 = etot(ps.pos, ps.vel)
    pos, vel, _ = oracle_lib.leapfrog(ps.pos, ps.vel, ps.mass, eps, dt, 20,
                                      use_tree=True, theta=0.75, n_crit=64)
    assert abs(etot(pos, vel) - e0) < 2e-3 * abs(e0)
