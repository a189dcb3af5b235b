"""Pins for the oracle's neighbour search by the general treewalk (Sec.
"General Treewalk"): the fixed-radius neighbours j != i, |x_j - x_i| <= h.
The tree forms (one walk per particle, one per group) must equal the
brute-force definition exactly; the definition itself is pinned by closed
forms on a lattice, symmetry and the limiting radii."""
import numpy as np
import pytest

import nbsynth


def lattice(m=7, a=0.25, jitter_seed=None):
    g = np.arange(m) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    return pos, np.full(len(pos), 1.0 / len(pos), np.float32)


def counts(off):
    return np.diff(off)


@pytest.mark.parametrize("h_over_a, expect", [(1.0, 6), (1.5, 18), (1.8, 26)])
def test_lattice_interior_counts(oracle_lib, h_over_a, expect):
    """On a cubic lattice of spacing a (exact in binary) an interior point has
    6 neighbours at h = a (the face neighbours, at distance exactly h), 18 at
    1.5 a (plus the edge ones at a sqrt 2) and 26 at 1.8 a (plus the corners
    at a sqrt 3)."""
    m, a = 7, 0.25
    pos, mass = lattice(m, a)
    T = oracle_lib.Tree(pos, mass)
    q = np.rint(pos / a).astype(int)
    interior = np.all((q >= 2) & (q <= m - 3), axis=1)
    for off, _ in (oracle_lib.neighbours_brute(pos, h_over_a * a), T.neighbours(h_over_a * a),
                   T.neighbours(h_over_a * a, group_form=True, n_crit=16)):
        assert np.all(counts(off)[interior] == expect)


@pytest.mark.parametrize("order", ["morton", "hilbert"])
@pytest.mark.parametrize("case", ["plummer", "halos", "lattice"])
def test_tree_forms_equal_the_definition(oracle_lib, order, case):
    if case == "plummer":
        ps = nbsynth.plummer(3000, 2)
        pos, mass, hs = ps.pos, ps.mass, (0.05, 0.2, 0.6)
    elif case == "halos":
        ps = nbsynth.halo_mix(6000, 4, n_halos=10)
        pos, mass, hs = ps.pos, ps.mass, (0.002, 0.01)
    else:
        pos, mass = lattice(6, 0.25)
        hs = (0.25, 0.5)
    T = oracle_lib.Tree(pos, mass, order=order)
    for h in hs:
        ob, ib = oracle_lib.neighbours_brute(pos, h)
        for off, idx in (T.neighbours(h), T.neighbours(h, group_form=True, n_crit=32),
                         T.neighbours(h, group_form=True, n_crit=1)):
            assert np.array_equal(off, ob) and np.array_equal(idx, ib)


def test_neighbour_relation_is_symmetric(oracle_lib):
    ps = nbsynth.halo_mix(4000, 9, n_halos=8)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    off, idx = T.neighbours(0.01, group_form=True)
    i = np.repeat(np.arange(T.n), counts(off))
    pairs = set(zip(i.tolist(), idx.tolist()))
    assert len(pairs) == len(idx) and len(idx) % 2 == 0
    assert all((j, k) in pairs for k, j in pairs)
    assert np.all(idx != i)


def test_limiting_radii(oracle_lib):
    """h = 0 finds exactly the coincident copies; a radius beyond the
    system finds every other particle."""
    rng = np.random.default_rng(2)
    base = rng.uniform(-1, 1, (200, 3))
    mult = rng.integers(1, 4, 200)
    pos = np.repeat(base, mult, axis=0)
    mass = np.full(len(pos), 1.0, np.float32)
    T = oracle_lib.Tree(pos, mass)
    for off, _ in (T.neighbours(0.0), T.neighbours(0.0, group_form=True, n_crit=8)):
        assert np.array_equal(counts(off), np.repeat(mult - 1, mult))
    off, _ = T.neighbours(10.0, group_form=True)
    assert np.all(counts(off) == len(pos) - 1)
