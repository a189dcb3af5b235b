"""FP64 reference of the learned opening angle's label rule (test
infrastructure: only tests/ may import it).

The paper fixes one theta for all particles (Eq. mac) and shows its cost /
accuracy trade (Table theta); the per-group theta is the project's addition
(reading g19).  For S sampled groups and an ascending theta grid, E[t, g] is
group g's measured median |da|/|a| against the FP64 direct sum and C[t, g]
its cost.  The label of g is the grid theta minimising

    PC[t, g] / n_g + lambda * PE[t, g]

with (PE, PC) = (ln max(E, 1e-9), C) for the measured curves, or the curves
the features predict: ordinary least squares of ln(E + 1e-15) and of
ln(C + 1) on the chosen feature columns plus an intercept (PE = the fit,
PC = exp of the fit).  lambda is bisected in ln space so that the
n_g-weighted median of the measured errors E at the chosen thetas meets the
budget (or, as an option, the plain median over the judged particles of
their own errors at their group's theta); the labels are those of the
bracket's upper end.  Written as plain
numpy: np.linalg.lstsq for the fit, np.argmin for the choice (first minimum
on ties), a stable sort and a cumulative sum for the weighted median.
"""
from __future__ import annotations

import numpy as np


def weighted_median(v, w):
    """The first value, in ascending order, at which the running weight
    reaches half the total."""
    v = np.asarray(v, np.float64)
    w = np.asarray(w, np.float64)
    o = np.argsort(v, kind="stable")
    cw = np.cumsum(w[o])
    return float(v[o][np.searchsorted(cw, 0.5 * cw[-1])])


def fit_curves(X, E, C, cols):
    """(PE, PC), each (T, S): least-squares predictions from the feature
    columns `cols` of X (S, >= max(cols)+1) plus an intercept."""
    F = np.asarray(X, np.float64)[:, list(cols)]
    A = np.c_[F, np.ones(len(F))]
    T, S = E.shape
    PE, PC = np.zeros((T, S)), np.zeros((T, S))
    for t in range(T):
        ce, *_ = np.linalg.lstsq(A, np.log(np.asarray(E[t], np.float64) + 1e-15), rcond=None)
        cc, *_ = np.linalg.lstsq(A, np.log(np.asarray(C[t], np.float64) + 1.0), rcond=None)
        PE[t], PC[t] = A @ ce, np.exp(A @ cc)
    return PE, PC


def choose(lam, PE, PC, size):
    """Grid index chosen for every group at exchange rate lam."""
    return np.argmin(PC / np.asarray(size, np.float64)[None, :] + lam * PE, axis=0)


def allocate(E, C, size, grid, budget, lam_lo, lam_hi, iters, PE=None, PC=None,
             perr=None, poff=None):
    """(labels (S,), lambda, statistic) of the rule above.  The statistic
    held at the budget is the n_g-weighted median of the groups' errors E,
    or, with perr (T, P) and poff (S + 1): the median over the judged
    particles of their own errors at their group's theta."""
    E = np.asarray(E, np.float64)
    C = np.asarray(C, np.float64)
    size = np.asarray(size, np.float64)
    if PE is None:
        PE = np.log(np.maximum(E, 1e-9))
    if PC is None:
        PC = C
    col = np.arange(E.shape[1])
    if perr is not None:
        perr = np.asarray(perr, np.float64)
        group_of = np.repeat(col, np.diff(poff))
        pcol = np.arange(perr.shape[1])

    def stat(lam):
        t = choose(lam, PE, PC, size)
        if perr is None:
            return t, weighted_median(E[t, col], size)
        return t, float(np.median(perr[t[group_of], pcol]))

    lo, hi = float(lam_lo), float(lam_hi)
    for _ in range(iters):
        mid = float(np.sqrt(lo * hi))
        if stat(mid)[1] > budget:
            lo = mid
        else:
            hi = mid
    t, werr = stat(hi)
    return np.asarray(grid, np.float32)[t], hi, werr


def error_stats(err, q):
    """(median, nearest-rank q-quantile: the ceil(q n)-th smallest)."""
    e = np.sort(np.asarray(err, np.float64))
    n = len(e)
    k = max(int(np.ceil(q * n)), 1)
    return float(np.median(e)), float(e[k - 1])
