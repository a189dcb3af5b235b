"""The learned opening angle without a GPU: the oracle's label rule
(oracle/labels.py) on synthetic curves whose best allocation is known, its
least-squares fit and weighted median against closed forms, and the flat
parameter layout the host hands to the network's kernels."""
import numpy as np

import nbsynth
from oracle import labels, mlp
from paper_0909_0541_gb300 import MLP_NPARAM, learn


def curves(S=400, seed=0):
    """Two kinds of group with the same cost curve whose errors differ by a
    factor 16 at every theta (error = K theta^2, cost = 1000 n_g theta^-3)."""
    rng = np.random.default_rng(seed)
    kind = rng.integers(0, 2, S)
    size = rng.integers(8, 64, S).astype(np.float64)
    grid = learn.THETA_GRID.astype(np.float64)
    K = np.where(kind == 1, 0.25, 4.0) * 1e-3 / 0.6 ** 2
    E = K[None, :] * grid[:, None] ** 2
    C = 1000.0 * size[None, :] * grid[:, None] ** -3.0
    X = np.zeros((S, 16), np.float32)
    X[:, 0] = kind
    X[:, 1] = np.log(size)
    return X, E, C, size, kind, grid


def test_predicted_labels_meet_the_budget_and_beat_one_theta():
    X, E, C, size, kind, grid = curves()
    PE, PC = labels.fit_curves(X, E, C, [0, 1])
    lab, lam, werr = labels.allocate(E, C, size, grid, learn.BUDGET, 1e-3, 1e9, 60, PE, PC)
    t = np.searchsorted(learn.THETA_GRID, lab)
    cols = np.arange(len(lab))
    assert labels.weighted_median(E[t, cols], size) <= learn.BUDGET
    assert werr <= learn.BUDGET and lam > 0
    # groups with the same predicted curves get the same theta (up to a tie
    # between neighbouring grid points)
    for k in (0, 1):
        assert lab[kind == k].max() - lab[kind == k].min() <= 0.051
    # and the allocation costs less than the best single theta within budget.
    # (Under a median budget the cheapest allocation may meet it with one kind
    # alone: the exchange rate trades the other kind's error for cost.)
    ok = [k for k in range(len(grid)) if labels.weighted_median(E[k], size) <= learn.BUDGET]
    best_single = min(C[k].sum() for k in ok)
    assert C[t, cols].sum() < best_single


def test_fit_curves_is_least_squares():
    """Residuals of the fit are orthogonal to every column and the intercept
    (the normal equations), on noisy data."""
    rng = np.random.default_rng(4)
    S, T = 300, 5
    X = rng.normal(size=(S, 16))
    E = np.exp(rng.normal(size=(T, S)) - 7.0)
    C = np.exp(rng.normal(size=(T, S)) + 8.0)
    PE, PC = labels.fit_curves(X, E, C, [1, 4, 9])
    A = np.c_[X[:, [1, 4, 9]], np.ones(S)]
    assert np.abs(A.T @ (np.log(E + 1e-15) - PE).T).max() < 1e-8
    assert np.abs(A.T @ (np.log(C + 1.0) - np.log(PC)).T).max() < 1e-8


def test_weighted_median():
    v = np.array([5.0, 1.0, 3.0])
    assert labels.weighted_median(v, np.array([1.0, 1.0, 1.0])) == 3.0
    assert labels.weighted_median(v, np.array([1.0, 10.0, 1.0])) == 1.0
    # half the weight exactly at a value: that value
    assert labels.weighted_median(np.array([1.0, 2.0, 3.0, 4.0]), np.ones(4)) == 2.0
    assert labels.error_stats([4.0, 1.0, 3.0, 2.0], 0.75) == (2.5, 3.0)


def test_host_parameter_packing_matches_the_oracle_layout():
    """learn.pack_params (what the product hands to nb_mlp_*) and the
    oracle's pack_params write the same flat layout; a zero spread becomes 1
    so the normalisation never divides by zero."""
    w = nbsynth.mlp_initial_weights(7)
    rng = np.random.default_rng(8)
    b = {k: rng.normal(0, 0.1, 64) for k in ("b1", "b2", "b3")}
    mu = rng.normal(0, 1, 12)
    sigma = rng.uniform(0.5, 2.0, 12)
    w_all = dict(w, **b, b4=0.25)
    host = learn.pack_params(w_all, mu, sigma)
    ref = mlp.pack_params(w["W1"], b["b1"], w["W2"], b["b2"], w["W3"], b["b3"], w["w4"],
                          0.25, mu, sigma)
    assert host.dtype == np.float32 and host.shape == (MLP_NPARAM,) == ref.shape
    assert np.array_equal(host, ref)
    sigma0 = sigma.copy()
    sigma0[[2, 5]] = 0.0
    packed = mlp.unpack(learn.pack_params(w_all, mu, sigma0))
    assert np.all(packed["sigma"][[2, 5]] == 1.0)
    assert np.all(packed["sigma"][12:] == 1.0) and np.all(packed["mu"][12:] == 0.0)
    assert np.all(packed["W1"][:, 12:] == 0.0)
