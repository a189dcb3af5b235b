"""Fixed-radius neighbours by the general treewalk on the GPU
(nb_neighbours; Sec. "General Treewalk") against the definition.

The neighbour sets are fixed by the definition (j != i, |x_j - x_i|^2 <= h^2
summed (x, y) then z in FP64), and both sides take every decision in FP64
with the same operations: the CSR offsets and the ascending caller indices
must equal the oracle's brute force (or, at 300k particles, the oracle's
tree form, itself pinned against the brute force) element for element.
"""
import numpy as np
import pytest

import nbsynth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def lattice(m=7, a=0.25):
    g = np.arange(m) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    return pos, np.full(len(pos), 1.0 / len(pos), np.float32)


def gpu_neigh(pos, mass, h, n_crit=64, order="morton"):
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    ctx = nb.NBody(max(len(pos), 1))
    ctx.set_key_order(order)
    ctx.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).to(dev),
                   torch.from_numpy(np.ascontiguousarray(mass, np.float32)).to(dev))
    off, idx = ctx.neighbours(h, n_crit)
    ctx.close()
    return off.cpu().numpy(), idx.cpu().numpy().astype(np.int64)


CASES = [
    ("cube", lambda: nbsynth.uniform_cube(4097, 11), (0.02, 0.08)),
    ("plummer", lambda: nbsynth.plummer(16384, 5), (0.01, 0.05)),
    ("halos", lambda: nbsynth.halo_mix(20000, 14, n_halos=50), (0.001, 0.005)),
]


@pytest.mark.parametrize("n_crit", [1, 64, 4096])
@pytest.mark.parametrize("name,make,hs", CASES)
def test_neighbours_equal_the_definition(oracle_lib, name, make, hs, n_crit):
    ps = make()
    for h in hs:
        ob, ib = oracle_lib.neighbours_brute(ps.pos, h)
        off, idx = gpu_neigh(ps.pos, ps.mass, h, n_crit)
        assert np.array_equal(off, ob) and np.array_equal(idx, ib), (name, h, n_crit)


def test_neighbours_hilbert_order_and_coincident_points(oracle_lib):
    ps = nbsynth.uniform_cube(3000, 12)
    pos = ps.pos.copy()
    pos[100:110] = pos[7]                       # eleven particles at one point
    for h in (0.0, 0.05):                       # h = 0: exactly the coincident copies
        ob, ib = oracle_lib.neighbours_brute(pos, h)
        off, idx = gpu_neigh(pos, ps.mass, h, 32, order="hilbert")
        assert np.array_equal(off, ob) and np.array_equal(idx, ib)
        if h == 0.0:
            assert np.diff(off)[7] == 10 and np.diff(off).sum() == 110


@pytest.mark.parametrize("h_over_a, expect", [(1.0, 6), (1.5, 18), (1.8, 26)])
def test_lattice_closed_forms(h_over_a, expect):
    m, a = 7, 0.25
    pos, mass = lattice(m, a)
    off, idx = gpu_neigh(pos, mass, h_over_a * a, 16)
    q = np.rint(pos / a).astype(int)
    interior = np.all((q >= 2) & (q <= m - 3), axis=1)
    assert np.all(np.diff(off)[interior] == expect)


def test_edge_sizes_and_everyone(oracle_lib):
    rng = np.random.default_rng(3)
    for n in (1, 2, 33):
        pos = rng.normal(size=(n, 3))
        mass = np.ones(n, np.float32)
        off, idx = gpu_neigh(pos, mass, 100.0, 8)     # a radius beyond the system
        assert np.array_equal(np.diff(off), np.full(n, n - 1))
        ob, ib = oracle_lib.neighbours_brute(pos, 100.0)
        assert np.array_equal(off, ob) and np.array_equal(idx, ib)


@pytest.mark.slow
def test_neighbours_300k_against_the_oracle_tree(oracle_lib):
    ps = nbsynth.halo_mix(300_000, 15, n_halos=200)
    h = 0.003
    T = oracle_lib.Tree(ps.pos, ps.mass)
    ob, ib = T.neighbours(h, group_form=True, n_crit=64)
    off, idx = gpu_neigh(ps.pos, ps.mass, h, 128)
    assert np.array_equal(off, ob) and np.array_equal(idx, ib)
