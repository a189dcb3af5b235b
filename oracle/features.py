"""FP64 reference of the learned-theta features of each group.

TEST INFRASTRUCTURE.  Features come from the oracle's own probe walk (the
group walk at theta = 1.2, the group's own particles removed) and its tree,
following the definition in include/nb.h: ln n_g; ln(box side / L + 1e-7)
for x, y, z; ln n_g - sum ln(side / L + 1e-4); ln(|box centre - root
centre| / L + 1e-6); ln(list length + 1); accepted cells / list length;
ln(min, mean, max distance from the box centre to accepted cells' centres of
mass / L + 1e-7); depth of the group node / 22.  tree_features gives the
tree-only set (feature mode 1): the same formulas for the features that need
no walk, zeros for the rest.
"""
from __future__ import annotations

import numpy as np

PROBE_THETA = 1.2


def group_features(T, n_crit, groups=None):
    """(len(groups), 12) features of the selected groups (all when None)."""
    e = T.export()
    gnode = T.groups(n_crit)
    box = T.group_boxes(gnode)
    leaf_of_slot = np.flatnonzero(e["is_cell"] == 0)
    depth = np.zeros(T.nnodes, np.int64)
    par = e["parent"]
    for u in range(1, T.nnodes):
        depth[u] = depth[par[u]] + 1
    L = T.L
    sel = np.arange(len(gnode)) if groups is None else np.asarray(groups)
    out = np.zeros((len(sel), 12))
    for r, k in enumerate(sel):
        u = gnode[k]
        lst = T.walk_group(u, box[k], PROBE_THETA)
        f, c = e["first"][u], e["count"][u]
        lst = lst[~np.isin(lst, leaf_of_slot[f:f + c])]
        cells = lst[e["is_cell"][lst] == 1]
        lo, hi, ctr = box[k, 0:3].astype(np.float64), box[k, 3:6].astype(np.float64), \
            box[k, 6:9].astype(np.float64)
        side = (hi - lo) / L
        d = np.linalg.norm(e["com"][cells] - ctr, axis=1) if len(cells) else np.zeros(0)
        out[r, 0] = np.log(c)
        out[r, 1:4] = np.log(side + 1e-7)
        out[r, 4] = np.log(c) - np.log(side + 1e-4).sum()
        out[r, 5] = np.log(np.linalg.norm(ctr - T.centre) / L + 1e-6)
        out[r, 6] = np.log(len(lst) + 1.0)
        out[r, 7] = len(cells) / len(lst) if len(lst) else 0.0
        if len(cells):
            out[r, 8] = np.log(d.min() / L + 1e-7)
            out[r, 9] = np.log(d.mean() / L + 1e-7)
            out[r, 10] = np.log(d.max() / L + 1e-7)
        else:
            out[r, 8:11] = np.log(1e-7)
        out[r, 11] = depth[u] / 22.0
    return out


def tree_features(T, n_crit, groups=None):
    """(len(groups), 12) tree-only features (feature mode 1): the features
    above that need no walk (0-5 and 11), the walk-based ones (6-10) zero."""
    e = T.export()
    gnode = T.groups(n_crit)
    box = T.group_boxes(gnode)
    depth = np.zeros(T.nnodes, np.int64)
    par = e["parent"]
    for u in range(1, T.nnodes):
        depth[u] = depth[par[u]] + 1
    L = T.L
    sel = np.arange(len(gnode)) if groups is None else np.asarray(groups)
    out = np.zeros((len(sel), 12))
    for r, k in enumerate(sel):
        u = gnode[k]
        c = e["count"][u]
        lo, hi, ctr = box[k, 0:3].astype(np.float64), box[k, 3:6].astype(np.float64), \
            box[k, 6:9].astype(np.float64)
        side = (hi - lo) / L
        out[r, 0] = np.log(c)
        out[r, 1:4] = np.log(side + 1e-7)
        out[r, 4] = np.log(c) - np.log(side + 1e-4).sum()
        out[r, 5] = np.log(np.linalg.norm(ctr - T.centre) / L + 1e-6)
        out[r, 11] = depth[u] / 22.0
    return out
