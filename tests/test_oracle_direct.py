"""Pins for the oracle's FP64 direct sum, Eq. (gravity), against closed forms,
invariants and a long-double brute force."""
import json
import math
import os

import numpy as np
import pytest

import nbsynth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.mark.parametrize("sep,eps", [(1.0, 0.0), (0.37, 0.1), (2.5, 1.0 / 64),
                                     (1e-3, 5e-4), (0.0, 0.25)])
def test_two_body_closed_form(oracle_lib, sep, eps):
    # |a_1| = m_2 r / (r^2 + eps^2)^{3/2} towards body 2; phi_1 = -m_2 / sqrt(r^2+eps^2)
    ps = nbsynth.two_body(sep, m1=0.25, m2=0.75, circular=False)
    acc, pot = oracle_lib.direct(ps.pos, ps.mass, eps)
    r2e = sep * sep + eps * eps
    for i, j in ((0, 1), (1, 0)):
        mj = float(ps.mass[j])
        expect_ax = mj * (ps.pos[j, 0] - ps.pos[i, 0]) / r2e ** 1.5
        assert acc[i, 0] == pytest.approx(expect_ax, rel=1e-14, abs=0)
        assert acc[i, 1] == 0.0 and acc[i, 2] == 0.0
        assert pot[i] == pytest.approx(-mj / math.sqrt(r2e), rel=1e-14)


def test_coincident_unsoftened_pair_contributes_nothing(oracle_lib):
    pos = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    mass = np.array([1, 1, 1], np.float32)
    acc, pot = oracle_lib.direct(pos, mass, 0.0)
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(pot))
    assert acc[0, 0] == pytest.approx(1.0) and pot[0] == pytest.approx(-1.0)


def test_zero_net_force(oracle_lib):
    ps = nbsynth.plummer(3000, 11)
    acc, _ = oracle_lib.direct(ps.pos, ps.mass, 1.0 / 64)
    net = (ps.mass.astype(np.float64)[:, None] * acc).sum(0)
    scale = (ps.mass.astype(np.float64)[:, None] * np.abs(acc)).sum(0)
    assert np.all(np.abs(net) < 1e-13 * scale)


def test_long_double_brute_force(oracle_lib):
    rng = np.random.default_rng(5)
    pos = rng.normal(size=(48, 3))
    mass = rng.uniform(0.1, 1.0, 48).astype(np.float32)
    for eps in (0.0, 0.05):
        a1, p1 = oracle_lib.direct(pos, mass, eps)
        a2, p2 = oracle_lib.direct_ld(pos, mass, eps)
        assert np.max(np.abs(a1 - a2) / np.linalg.norm(a2, axis=1)[:, None]) < 1e-13
        assert np.max(np.abs(p1 - p2) / np.abs(p2)) < 1e-14


def test_magnitude_sum_bounds_the_acceleration(oracle_lib):
    # sum_j |a_ij| >= |sum_j a_ij| (triangle inequality), equal for two bodies
    ps = nbsynth.plummer(500, 12)
    acc, _, am = oracle_lib.direct(ps.pos, ps.mass, 0.01, with_amag=True)
    assert np.all(am >= np.linalg.norm(acc, axis=1) * (1 - 1e-14))
    tb = nbsynth.two_body(0.7, 0.4, 0.6, circular=False)
    acc, _, am = oracle_lib.direct(tb.pos, tb.mass, 0.1, with_amag=True)
    assert np.allclose(am, np.linalg.norm(acc, axis=1), rtol=1e-15)


def test_targets_subset(oracle_lib):
    ps = nbsynth.uniform_sphere(500, 3)
    a, p = oracle_lib.direct(ps.pos, ps.mass, 0.01)
    idx = np.array([7, 0, 499, 250])
    a2, p2 = oracle_lib.direct(ps.pos, ps.mass, 0.01, targets=idx)
    assert np.array_equal(a[idx], a2) and np.array_equal(p[idx], p2)


def test_plummer_potential_closed_form(oracle_lib):
    # truncated Plummer (a = M = 1, cut at r = 20, renormalised to unit mass):
    # phi(r) = (-1/sqrt(r^2+1) + 1/sqrt(401) - M20/20) / M20, M20 = 20^3/401^{3/2}
    ps = nbsynth.plummer(16384, nbsynth.BASE_SEED + 1)
    _, pot = oracle_lib.direct(ps.pos, ps.mass, 1.0 / 64)
    r = np.linalg.norm(ps.pos, axis=1)
    m20 = 8000.0 / 401.0 ** 1.5
    phi_t = (-1.0 / np.sqrt(r * r + 1) + 1 / math.sqrt(401.0) - m20 / 20) / m20
    edges = [0.1, 0.3, 0.6, 1.0, 1.5, 2.5, 4.0]
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (r >= lo) & (r < hi)
        assert m.sum() > 200
        # sampling noise of a 16k-particle realisation is well below 1 %
        assert abs(pot[m].mean() - phi_t[m].mean()) < 0.01 * abs(phi_t[m].mean())


def test_uniform_sphere_interior_potential(oracle_lib):
    # phi(r) = -M (3 R^2 - r^2) / (2 R^3) inside a uniform sphere
    ps = nbsynth.uniform_sphere(20000, 17)
    _, pot = oracle_lib.direct(ps.pos, ps.mass, 1e-3)
    r = np.linalg.norm(ps.pos, axis=1)
    edges = np.linspace(0.2, 0.9, 8)
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (r >= lo) & (r < hi)
        expect = np.mean(-(3.0 - r[m] ** 2) / 2.0)
        assert abs(pot[m].mean() - expect) < 0.01 * abs(expect)


def test_paper_flop_convention_fixture():
    here = os.path.join(os.path.dirname(__file__), "golden", "paper_figures.json")
    fig = json.load(open(here))
    assert fig["flops_per_interaction"]["value"] == 38
    # the run's sustained speed follows from its own figures (Sec. Cosmological Simulation)
    g = 38 * fig["cosmo_run_interactions"]["value"] / fig["cosmo_run_wallclock_s"]["value"] / 1e9
    assert abs(g - fig["cosmo_run_gflops"]["value"]) < 0.1
