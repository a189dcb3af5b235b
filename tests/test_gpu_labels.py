"""The learned theta's label rule on the device (nb_theta_fit_curves,
nb_theta_allocate, nb_error_stats, nb_column_stats) against the oracle's
FP64 numpy statement of the same rule (oracle/labels.py).

Bars: the fitted curves agree to 1e-9 (relative on the cost curve, absolute
on ln error: the device solves standardised normal equations by Cholesky,
the oracle uses np.linalg.lstsq, so only rounding differs).  Labels are
integer decisions made in FP64 on both sides: they must be equal wherever the
oracle's best choice beats the runner-up by more than 1e-9 of the objective's
scale, the exchange rate must agree to 1e-9 relative, and the weighted
median must be identical (it is one of the inputs).  Error statistics are
exact: the same FP32 errors, the same order statistics.
"""
import numpy as np
import pytest

from oracle import labels as olab

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def synthetic(S=5000, T=19, seed=3):
    """Curves with a known dependence on two features plus noise, and
    unrelated feature columns (one constant)."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(S, 16)).astype(np.float32)
    X[:, 7] = 2.5                                   # a constant column
    size = rng.integers(8, 257, S).astype(np.float32)
    grid = np.round(np.arange(0.30, 0.30 + 0.05 * T - 1e-9, 0.05), 2).astype(np.float32)
    lnK = -7.0 + 0.8 * X[:, 0] - 0.3 * X[:, 3] + 0.5 * rng.normal(size=S)
    E = np.exp(lnK[None, :] + 2.0 * np.log(grid)[:, None]).astype(np.float32)
    C = (size[None, :] * (size[None, :] + 400.0 * np.exp(0.2 * X[:, 1])[None, :]
                          * grid[:, None] ** -3.0)).astype(np.float32)
    return X, E, C, size, grid


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("cols", [[0, 1, 2, 3, 4, 5, 11], list(range(12)), []])
def test_fit_curves_match_lstsq(cols):
    import paper_0909_0541_gb300 as nb
    X, E, C, size, grid = synthetic()
    pe, pc = nb.theta_fit_curves(_dev(X), _dev(E), _dev(C), cols)
    PE, PC = olab.fit_curves(X, E, C, cols)
    assert np.allclose(pe.cpu().numpy(), PE, rtol=0, atol=1e-9)
    assert np.allclose(pc.cpu().numpy(), PC, rtol=1e-9, atol=0)


@pytest.mark.parametrize("rule", ["measured", "predicted"])
def test_allocation_matches_oracle(rule):
    import paper_0909_0541_gb300 as nb
    X, E, C, size, grid = synthetic()
    cols = [0, 1, 2, 3, 4, 5, 11]
    if rule == "predicted":
        pred = nb.theta_fit_curves(_dev(X), _dev(E), _dev(C), cols)
        PE, PC = olab.fit_curves(X, E, C, cols)
        args = (1e-3, 1e9, 60)
    else:
        pred, PE, PC = None, None, None
        args = (1.0, 1e6, 40)
    lab, lam, wm = nb.theta_allocate(_dev(E), _dev(C), _dev(size), _dev(grid), 1e-3, *args,
                                     pred=pred)
    rlab, rlam, rwm = olab.allocate(E, C, size, grid, 1e-3, *args, PE, PC)
    assert abs(lam - rlam) <= 1e-9 * rlam
    assert wm == rwm and wm <= 1e-3
    # equal wherever the oracle's choice is not a near-tie
    PE_ = np.log(np.maximum(E.astype(np.float64), 1e-9)) if PE is None else PE
    PC_ = C.astype(np.float64) if PC is None else PC
    obj = PC_ / size[None, :].astype(np.float64) + rlam * PE_
    srt = np.sort(obj, axis=0)
    clear = (srt[1] - srt[0]) > 1e-9 * np.abs(srt[0])
    got = lab.cpu().numpy()
    assert np.array_equal(got[clear], rlab[clear])
    assert clear.mean() > 0.99


def test_allocation_particle_median_matches_oracle():
    """The bisection held on the median over particles (per-particle errors
    and group offsets) instead of the weighted median of group medians."""
    import paper_0909_0541_gb300 as nb
    X, E, C, size, grid = synthetic(S=3000)
    rng = np.random.default_rng(9)
    poff = np.r_[0, np.cumsum(size.astype(np.int64))].astype(np.int64)
    P = int(poff[-1])
    gid = np.repeat(np.arange(len(size)), size.astype(np.int64))
    perr = (E[:, gid] * np.exp(0.4 * rng.normal(size=(E.shape[0], P)))).astype(np.float32)
    lab, lam, st = nb.theta_allocate(_dev(E), _dev(C), _dev(size), _dev(grid), 1e-3, 1.0, 1e6,
                                     40, perr=_dev(perr), poff=_dev(poff))
    rlab, rlam, rst = olab.allocate(E, C, size, grid, 1e-3, 1.0, 1e6, 40, perr=perr, poff=poff)
    assert abs(lam - rlam) <= 1e-9 * rlam and st == rst and st <= 1e-3
    obj = C.astype(np.float64) / size[None, :] + rlam * np.log(np.maximum(E, 1e-9))
    srt = np.sort(obj, axis=0)
    clear = (srt[1] - srt[0]) > 1e-9 * np.abs(srt[0])
    assert np.array_equal(lab.cpu().numpy()[clear], rlab[clear])
    bad = poff.copy()
    bad[5] = bad[6] + 1                                 # decreasing offsets: rejected
    with pytest.raises(nb.NBError):
        nb.theta_allocate(_dev(E), _dev(C), _dev(size), _dev(grid), 1e-3, 1.0, 1e6, 40,
                          perr=_dev(perr), poff=_dev(bad))


def test_allocation_edge_sizes():
    import paper_0909_0541_gb300 as nb
    X, E, C, size, grid = synthetic(S=1)
    lab, lam, wm = nb.theta_allocate(_dev(E), _dev(C), _dev(size), _dev(grid), 1e-3, 1.0, 1e6, 40)
    rlab, rlam, rwm = olab.allocate(E, C, size, grid, 1e-3, 1.0, 1e6, 40)
    assert np.array_equal(lab.cpu().numpy(), rlab) and wm == rwm
    with pytest.raises(nb.NBError):
        nb.theta_allocate(_dev(E), _dev(C), _dev(size), _dev(grid), 1e-3, 0.0, 1e6, 40)


@pytest.mark.parametrize("nt", [1, 2, 7, 8192, 100003])
def test_error_stats_exact(nt):
    import paper_0909_0541_gb300 as nb
    rng = np.random.default_rng(nt)
    n = nt + 11
    acc = rng.normal(size=(n, 3)).astype(np.float32)
    tg = rng.choice(n, nt, replace=False).astype(np.int64)
    ref = acc[tg].astype(np.float64) * (1.0 + 1e-3 * rng.normal(size=(nt, 1)))
    ref[0] = 0.0 if nt > 3 else ref[0]                 # |ref| = 0 counts as 1
    med, q99 = nb.error_stats(_dev(acc), _dev(ref), _dev(tg), q=0.99)
    d = np.linalg.norm(acc[tg].astype(np.float64) - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    e = (d / np.where(r > 0, r, 1.0)).astype(np.float32)
    rmed, rq = olab.error_stats(e, 0.99)
    assert med == rmed and q99 == rq


def test_column_stats():
    import paper_0909_0541_gb300 as nb
    X, *_ = synthetic()
    mu, sd = nb.column_stats(_dev(X), 12)
    Xd = X[:, :12].astype(np.float64)
    assert np.allclose(mu.cpu().numpy(), Xd.mean(0), rtol=1e-12, atol=1e-15)
    assert np.allclose(sd.cpu().numpy(), Xd.std(0), rtol=1e-12, atol=1e-15)
