"""nb_morton_order_noalloc: Morton keys and sort order without any device
allocation.

Some callers cannot call cudaMalloc: it synchronises the device and is not
allowed while a stream is being captured, and when another allocator (such as
a framework's caching allocator) already holds most of the device memory it
can fail.  This entry point serves them from a static scratch array inside the
library.  The test calls it through the C ABI twice in a row, on two particle
sets of different size, and checks each result bit for bit against the keys
and order nb_build_tree produces for the same positions (integer results:
the bar is bit-exact).  It also covers the smallest inputs (one and two
particles), a NaN coordinate (NB_ERR_NONFINITE) and a clean call right after
it, which must succeed: the error word left by the failed call is cleared.  It lives in its own file so that pytest collects it
after every other test.
"""
import numpy as np
import pytest

import nbsynth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_noalloc_order_matches_build_tree_on_two_calls():
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    sets = [nbsynth.halo_mix(300_000, 31, n_halos=100), nbsynth.plummer(5000, 32)]
    for ps in sets:
        pos = torch.from_numpy(ps.pos).to(dev)
        mass = torch.from_numpy(ps.mass).to(dev)
        keys = torch.empty(ps.n, dtype=torch.int64, device=dev)
        perm = torch.empty(ps.n, dtype=torch.int32, device=dev)
        nb.morton_order_noalloc(pos, keys, perm)
        ctx = nb.NBody(ps.n)
        ctx.build_tree(pos, mass)
        ref = ctx.copy_tree()
        ctx.close()
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref["keys"])
        assert np.array_equal(perm.cpu().numpy(), ref["perm"])


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import paper_0909_0541_gb300 as nb
    n = nb.NOALLOC_MAX_N + 1
    dev = torch.device("cuda")
    pos = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    with pytest.raises(nb.NBError) as ei:
        nb.morton_order_noalloc(pos, keys, perm)
    assert ei.value.code == -1


def _build_tree_order(pos_t):
    import paper_0909_0541_gb300 as nb
    n = int(pos_t.shape[0])
    mass = torch.ones(n, dtype=torch.float32, device=pos_t.device)
    ctx = nb.NBody(max(n, 1))
    ctx.build_tree(pos_t, mass)
    ref = ctx.copy_tree()
    ctx.close()
    return ref["keys"], ref["perm"]


def _noalloc(pos_t):
    import paper_0909_0541_gb300 as nb
    n = int(pos_t.shape[0])
    keys = torch.empty(n, dtype=torch.int64, device=pos_t.device)
    perm = torch.empty(n, dtype=torch.int32, device=pos_t.device)
    nb.morton_order_noalloc(pos_t, keys, perm)
    return keys.cpu().numpy().view(np.uint64), perm.cpu().numpy()


def test_noalloc_smallest_inputs():
    dev = torch.device("cuda")
    for pos in (np.array([[0.25, -1.0, 3.0]]), np.array([[1.0, 1.0, 1.0], [0.0, 0.0, 0.0]])):
        p = torch.from_numpy(pos).to(dev)
        k, q = _noalloc(p)
        rk, rq = _build_tree_order(p)
        assert np.array_equal(k, rk) and np.array_equal(q, rq)


def test_noalloc_nan_then_clean_call():
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    ps = nbsynth.plummer(4000, 33)
    bad = ps.pos.copy()
    bad[123, 2] = np.nan
    with pytest.raises(nb.NBError) as ei:
        _noalloc(torch.from_numpy(bad).to(dev))
    assert ei.value.code == -5          # NB_ERR_NONFINITE
    p = torch.from_numpy(ps.pos).to(dev)
    k, q = _noalloc(p)                  # the next clean call succeeds
    rk, rq = _build_tree_order(p)
    assert np.array_equal(k, rk) and np.array_equal(q, rq)
