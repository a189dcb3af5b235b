"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
on a seeded particle set and run the oracle on the same inputs."""
from __future__ import annotations

import numpy as np


def gpu_run(pos, mass, *, theta, n_crit, eps, precision="fp32", max_n=None,
            lists=True, key_order="morton"):
    import torch

    import paper_0909_0541_gb300 as nb
    n = pos.shape[0]
    dev = torch.device("cuda")
    p = torch.from_numpy(np.ascontiguousarray(pos, np.float64)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(mass, np.float32)).to(dev)
    ctx = nb.NBody(max_n or max(n, 1))
    ctx.set_key_order(key_order)
    ctx.build_tree(p, m)
    ctx.walk_groups(theta, n_crit)
    acc = torch.zeros((n, 3), dtype=torch.float32, device=dev)
    pot = torch.zeros(n, dtype=torch.float32, device=dev)
    ctx.forces(eps, acc, pot, precision)
    out = dict(ctx=ctx, acc=acc.cpu().numpy(), pot=pot.cpu().numpy(),
               stats=ctx.stats())
    if lists:
        out["tree"] = ctx.copy_tree()
        out["groups"] = ctx.copy_groups()
        out["lists"] = ctx.copy_lists(with_xm=True)
    return out


def oracle_tree_arrays(T):
    """Oracle export converted to the GPU export's conventions."""
    e = T.export()
    cell = e["is_cell"] == 1
    return dict(
        perm=e["order"], level=np.where(cell, e["level"], -1),
        first=e["first"], count=e["count"], next=e["next"], parent=e["parent"],
        nchild=e["nchild"], M=e["M"], com=e["com"], l=np.where(cell, e["l"], 0),
        s=np.where(cell, e["s"], 0), is_cell=e["is_cell"])


def oracle_external_lists(T, n_crit, theta):
    """The oracle's depth-first lists with each group's own particles removed
    (the CUDA walk lists sources outside the group; the force kernel sums the
    group's members directly).  Returns (gnode, box, offsets, entries, own)
    where own[k] is the number of own particles found in group k's list."""
    gnode, box, off, ent = T.all_lists(n_crit, theta)
    e = T.export()
    leaf_of_slot = np.flatnonzero(e["is_cell"] == 0)
    out, offs, own = [], [0], []
    for k in range(len(gnode)):
        lst = ent[off[k]:off[k + 1]]
        f, c = e["first"][gnode[k]], e["count"][gnode[k]]
        mine = np.isin(lst, leaf_of_slot[f:f + c])
        own.append(int(mine.sum()))
        out.append(lst[~mine])
        offs.append(offs[-1] + int((~mine).sum()))
    ent2 = np.concatenate(out) if out else np.zeros(0, np.int64)
    return gnode, box, np.array(offs, np.int64), ent2, np.array(own)


def rel_err(a, ref):
    """Per-particle |a - ref| / |ref| (rows of ref with zero norm use 1)."""
    d = np.linalg.norm(np.asarray(a, np.float64) - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    return d / np.where(r > 0, r, 1.0)
