"""Learned per-group opening angle: training data, training, evaluation.

The paper uses one global theta (Eq. mac, Sec. "Our GPU implementation");
this module drives the learned form through the C ABI.  Every computation
runs in libnb's kernels: the probe walk (features), the tree walk and force
sum at each theta of a grid, the FP64 direct-sum judge, per-group median
errors, labels, and the tensor-core network's training and inference.  What
remains here is orchestration: choosing which groups to judge (seeded draws),
index bookkeeping, and the shuffles handed to the trainer.

Labels: each sampled group is walked and summed at every theta of the grid
0.30, 0.35, ..., 1.20, giving its median |da|/|a| against the FP64 direct
sum, e(theta), and its interactions, c(theta).  Its label is the grid theta
minimising c / n_g + lambda ln e: one exchange rate between interactions and
error for all groups, so that groups whose error barely grows with theta
(dense regions, where near neighbours dominate the force) open fewer cells
and groups whose error grows fast keep a small theta.  lambda is bisected so
that the n_g-weighted median of the labelled errors meets the budget (1e-3).
(Requiring every group's own median to meet the budget costs as much as one
fixed theta at the same global median error.)  The curves are the measured
ones, or the ones the features predict (least squares); the fit, the choice,
the weighted median and the bisection all run in libnb (nb_theta_fit_curves,
nb_theta_allocate).  The network maps the features to theta in [0.3, 1.2];
the fixed-theta walk is the fallback for non-finite output.
"""
from __future__ import annotations

import numpy as np

from . import (MLP_NPARAM, NBody, column_stats, direct_sum, error_stats, group_errors,
               mlp_train, theta_allocate, theta_fit_curves)

THETA_GRID = np.round(np.arange(0.30, 1.2001, 0.05), 2).astype(np.float32)
BUDGET = 1e-3
NIN = 12
OFF = dict(W1=0, b1=1024, W2=1088, b2=5184, W3=5248, b3=9344, w4=9408, b4=9920, mu=9928,
           sigma=9944)


def pack_params(w: dict, mu, sigma) -> np.ndarray:
    """Flat FP32 parameters (layout of include/nb.h) from initial weights
    w (W1 64x12, W2, W3 64x64, w4 64, biases) and feature mean / spread."""
    p = np.zeros(MLP_NPARAM, np.float64)
    W1 = np.zeros((64, 16))
    W1[:, :NIN] = w["W1"]
    p[OFF["W1"]:OFF["W1"] + 1024] = W1.ravel()
    p[OFF["b1"]:OFF["b1"] + 64] = w["b1"]
    p[OFF["W2"]:OFF["W2"] + 4096] = np.ravel(w["W2"])
    p[OFF["b2"]:OFF["b2"] + 64] = w["b2"]
    p[OFF["W3"]:OFF["W3"] + 4096] = np.ravel(w["W3"])
    p[OFF["b3"]:OFF["b3"] + 64] = w["b3"]
    p[OFF["w4"]:OFF["w4"] + 64] = w["w4"]
    p[OFF["b4"]] = w["b4"]
    p[OFF["mu"]:OFF["mu"] + NIN] = mu
    sg = np.ones(16)
    sg[:NIN] = np.where(np.asarray(sigma) > 0, sigma, 1.0)
    p[OFF["sigma"]:OFF["sigma"] + 16] = sg
    return p.astype(np.float32)


def judge_targets(ctx: NBody, groups: np.ndarray, per_group=0, seed=0):
    """Caller indices of the judged members of `groups` (in group order), the
    offsets of each group's rows, and the groups' sizes.  per_group > 0 judges
    a seeded random subset of at most that many members per group."""
    gg = ctx.copy_groups()
    perm = ctx.copy_perm()
    first, count = gg["gfirst"][groups], gg["gcount"][groups]
    rng = np.random.default_rng(seed)
    rows = []
    for f, c in zip(first, count):
        m = perm[f:f + c]
        if per_group and c > per_group:
            m = m[np.sort(rng.choice(c, per_group, replace=False))]
        rows.append(m)
    targets = np.concatenate(rows).astype(np.int64)
    off = np.r_[0, np.cumsum([len(r) for r in rows])].astype(np.int64)
    return targets, off, count.astype(np.float32)


TREE_COLS = [0, 1, 2, 3, 4, 5, 11]   # the features of feature mode 1 (no walk)


def make_dataset(pos, mass, eps, n_crit, n_sample, seed, grid=THETA_GRID, budget=BUDGET,
                 ctx: NBody | None = None, feature_mode=0, label_rule="measured",
                 walk_weight=0.0, label_stat="groups", judge_per_group=0):
    """(features (S,16), labels (S,), info) for S seeded random groups of the
    particle set (pos, mass: CUDA tensors); info holds the error and cost
    curves, the group sizes, the sampled groups and the exchange rate.
    feature_mode: 0 probe-walk features, 1 tree-only features.  label_rule:
    "measured" (the allocation over each group's measured curves) or
    "predicted" (over the curves the features predict, least squares on the
    features of the feature mode).  A group's cost at a theta is its
    interactions, n_g (list length + n_g), plus walk_weight x list length: the
    walk's time per list entry in units of the force's time per interaction
    (0: interactions only).  label_stat: the error statistic the exchange rate
    is bisected on, "groups" (n_g-weighted median of group medians) or
    "particles" (median over the judged particles).  judge_per_group > 0 judges
    at most that many seeded members of each group against the direct sum."""
    import torch
    n = int(pos.shape[0])
    own = ctx is None
    ctx = ctx or NBody(n, eps=eps, n_crit=n_crit)
    ctx.build_tree(pos, mass)
    ctx.set_feature_mode(feature_mode)
    feat = ctx.group_features(n_crit)
    G = int(feat.shape[0])
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(G, min(n_sample, G), replace=False))
    targets, off, size = judge_targets(ctx, sel, judge_per_group, seed + 17)
    dev = pos.device
    t_dev = torch.from_numpy(targets).to(dev)
    o_dev = torch.from_numpy(off).to(dev)
    ref, _ = direct_sum(pos, mass, eps, t_dev)
    acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    errs = torch.empty((len(grid), len(sel)), dtype=torch.float32, device=dev)
    perr = torch.empty((len(grid), len(targets)), dtype=torch.float32, device=dev) \
        if label_stat == "particles" else None
    cost = np.zeros((len(grid), len(sel)), np.float32)
    for t, th in enumerate(grid):
        ctx.walk_groups(float(th), n_crit)
        ctx.forces(eps, acc)
        errs[t] = group_errors(acc, ref, t_dev, o_dev)
        if perr is not None:
            error_stats(acc, ref, t_dev, err_out=perr[t])
        ln = ctx.copy_group_lengths()[sel]
        cost[t] = size * (ln + size) + walk_weight * ln
    grid_d = torch.from_numpy(np.asarray(grid, np.float32)).to(dev)
    cost_d = torch.from_numpy(cost).to(dev)
    size_d = torch.from_numpy(size).to(dev)
    X = feat[torch.from_numpy(sel).to(dev)].contiguous()
    if label_rule == "predicted":
        cols = TREE_COLS if feature_mode == 1 else list(range(NIN))
        pred = theta_fit_curves(X, errs, cost_d, cols)
        labels, hi, werr = theta_allocate(errs, cost_d, size_d, grid_d, budget, 1e-3, 1e9, 60,
                                          pred=pred, perr=perr, poff=o_dev)
    else:
        labels, hi, werr = theta_allocate(errs, cost_d, size_d, grid_d, budget, 1.0, 1e6, 40,
                                          perr=perr, poff=o_dev)
    E = errs.cpu().numpy()
    if own:
        ctx.close()
    info = dict(errors=E, cost=cost, size=size, groups=sel, lam=hi, labelled_error=werr)
    return X, labels, info


def train(X, y, epochs=150, batch=256, lr=2e-3, seed=5):
    """Fresh network (seeded initial weights) trained on (X, y).  Returns
    (params CUDA tensor, per-epoch mean loss)."""
    import torch

    import nbsynth
    S = int(X.shape[0])
    mu, sd = column_stats(X, NIN)
    params = torch.from_numpy(pack_params(nbsynth.mlp_initial_weights(seed), mu.cpu().numpy(),
                                          sd.cpu().numpy())).to(X.device)
    rng = np.random.default_rng(seed + 1)
    order = torch.from_numpy(np.stack([rng.permutation(S) for _ in range(epochs)])
                             .astype(np.int32)).to(X.device)
    hist = mlp_train(params, X, y, order, epochs, batch, lr)
    steps = S // batch
    return params, (hist / (steps * batch)).cpu().numpy()


def median_error(acc, ref, targets):
    """Median |da|/|a| of acc at targets against the FP64 direct-sum
    reference ref (nb_error_stats)."""
    return error_stats(acc, ref, targets)[0] if int(ref.shape[0]) else 0.0


def step_cost(ctx: NBody, n_crit, eps, acc, theta=None, params=None, fallback=0.6):
    """Walk + force once (fixed theta, or the network's per-group theta);
    returns (interactions, milliseconds of the walk and force phases)."""
    ctx.set_timing(True)
    ctx.get_timing()
    if params is None:
        ctx.walk_groups(theta, n_crit)
    else:
        ctx.walk_groups_learned(n_crit, params, fallback)
    ctx.forces(eps, acc)
    tm = ctx.get_timing()
    ctx.set_timing(False)
    st = ctx.stats()
    return st["n_pp"] + st["n_pc"], tm["walk"][0] + tm["force"][0]


def calibrate(ctx: NBody, params, n_crit, eps, acc, ref, targets, target_err,
              lo=-4.0, hi=4.0, iters=14, fallback=0.6):
    """Shift of the output bias b4 (a common offset of every group's logit)
    bisected so that the learned walk's median error over `targets` equals
    target_err; ctx holds the tree of the calibration set.  The labels bound
    a weighted median of per-group medians, and this matches the global
    median instead.  Returns (calibrated parameters, shift)."""
    base = params.clone()
    p = params.clone()
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        p.copy_(base)
        p[OFF["b4"]] += mid
        ctx.walk_groups_learned(n_crit, p, fallback)
        ctx.forces(eps, acc)
        if median_error(acc, ref, targets) > target_err:
            hi = mid
        else:
            lo = mid
    p.copy_(base)
    p[OFF["b4"]] += lo
    return p, lo


def matched_fixed_theta(ctx: NBody, n_crit, eps, acc, ref, targets, target_err,
                        lo=0.3, hi=1.2, iters=12):
    """Bisection for the fixed theta whose median error equals target_err."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        ctx.walk_groups(mid, n_crit)
        ctx.forces(eps, acc)
        if median_error(acc, ref, targets) > target_err:
            hi = mid
        else:
            lo = mid
    return lo
