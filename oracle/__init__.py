"""CPU oracle for the oct-tree gravity path (arXiv:0909.0541).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_0909_0541_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``nb_oracle.c`` (plain C, FP64 where the method is
defined in FP64, FP32 with separately rounded operations where the opening
test is defined in FP32).  This module only compiles it and marshals numpy
arrays.  ``mlp.py`` holds the FP64 reference of the learned opening-angle
network.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
          "-shared", "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (seconds).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _P(t):
    return C.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i64, f64, f32 = C.c_int64, C.c_double, C.c_float
            vp = C.c_void_p
            L.or_num_threads.restype = C.c_int
            L.or_direct.argtypes = [i64, vp, vp, f64, i64, vp, vp, vp, vp]
            L.or_direct_ld.argtypes = [i64, vp, vp, f64, vp, vp]
            L.or_root_cube.argtypes = [i64, vp, vp]
            L.or_quantize.argtypes = [i64, vp, vp, vp]
            L.or_morton_keys.argtypes = [i64, vp, vp]
            L.or_hilbert_keys.argtypes = [i64, vp, vp]
            L.or_tree_build.restype = vp
            L.or_tree_build.argtypes = [i64, vp, vp]
            L.or_tree_build_order.restype = vp
            L.or_tree_build_order.argtypes = [i64, vp, vp, C.c_int]
            L.or_tree_corners.argtypes = [vp, vp]
            L.or_tree_export_quad.restype = C.c_int
            L.or_tree_export_quad.argtypes = [vp, vp]
            L.or_tree_forces_quad.restype = C.c_int
            L.or_tree_forces_quad.argtypes = [vp, i64, f64, f64, vp, vp, vp, vp, vp, C.c_int]
            L.or_neighbours.restype = i64
            L.or_neighbours.argtypes = [vp, f64, C.c_int, i64, vp, vp, i64]
            L.or_neighbours_brute.restype = i64
            L.or_neighbours_brute.argtypes = [i64, vp, f64, vp, vp, i64]
            L.or_tree_free.argtypes = [vp]
            L.or_tree_nnodes.restype = i64
            L.or_tree_nnodes.argtypes = [vp]
            L.or_tree_ncells.restype = i64
            L.or_tree_ncells.argtypes = [vp]
            L.or_tree_root.argtypes = [vp, vp]
            L.or_tree_export.argtypes = [vp] * 16
            L.or_groups.restype = i64
            L.or_groups.argtypes = [vp, i64, vp]
            L.or_group_boxes.argtypes = [vp, i64, vp, vp]
            L.or_walk_group.restype = i64
            L.or_walk_group.argtypes = [vp, i64, vp, f64, C.c_int, vp, i64]
            L.or_walk_particle.restype = i64
            L.or_walk_particle.argtypes = [vp, i64, f64, vp, i64]
            L.or_all_lists.restype = i64
            L.or_all_lists.argtypes = [vp, i64, vp, vp, f64, vp, vp, i64]
            L.or_tree_forces.argtypes = [vp, i64, f64, vp, f64, i64, vp, vp,
                                         vp, vp, vp, vp, C.c_int]
            L.or_leapfrog.argtypes = [i64, vp, vp, vp, f64, f64, i64, C.c_int,
                                      f64, i64, vp, C.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _pos(pos):
    return np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)


def _mass(mass):
    return np.ascontiguousarray(mass, dtype=np.float32).reshape(-1)


def num_threads() -> int:
    return int(lib().or_num_threads())


def direct(pos, mass, eps, targets=None, with_amag=False):
    """FP64 direct sum of Eq. (gravity) (physical signs, G = 1) for the
    particles `targets` (all when None).  Returns (acc (nt,3), pot (nt,)),
    plus sum_j |a_ij| per target when with_amag."""
    pos, mass = _pos(pos), _mass(mass)
    n = pos.shape[0]
    if targets is None:
        nt, tg = n, None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        nt = tg.shape[0]
    acc = np.zeros((nt, 3))
    pot = np.zeros(nt)
    am = np.zeros(nt) if with_amag else None
    rc = lib().or_direct(n, _ptr(pos), _ptr(mass), float(eps), nt, _ptr(tg),
                         _ptr(acc), _ptr(pot), _ptr(am))
    assert rc == 0
    return (acc, pot, am) if with_amag else (acc, pot)


def direct_ld(pos, mass, eps):
    """The same sum in long double (tiny N only)."""
    pos, mass = _pos(pos), _mass(mass)
    n = pos.shape[0]
    acc = np.zeros((n, 3))
    pot = np.zeros(n)
    lib().or_direct_ld(n, _ptr(pos), _ptr(mass), float(eps), _ptr(acc), _ptr(pot))
    return acc, pot


def root_cube(pos):
    """(centre[3], L, corner[3]) of the root cell."""
    pos = _pos(pos)
    out = np.zeros(7)
    lib().or_root_cube(pos.shape[0], _ptr(pos), _ptr(out))
    return out[:3].copy(), float(out[3]), out[4:].copy()


def quantize(pos):
    pos = _pos(pos)
    out = np.zeros(7)
    lib().or_root_cube(pos.shape[0], _ptr(pos), _ptr(out))
    q = np.zeros((pos.shape[0], 3), dtype=np.int32)
    lib().or_quantize(pos.shape[0], _ptr(pos), _ptr(out), _ptr(q))
    return q


def morton_keys(q):
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1, 3)
    k = np.zeros(q.shape[0], dtype=np.uint64)
    lib().or_morton_keys(q.shape[0], _ptr(q), _ptr(k))
    return k


def neighbours_brute(pos, h):
    """The definition of the neighbour sets, every pair tested: (offsets,
    caller indices in ascending order)."""
    pos = _pos(pos)
    n = pos.shape[0]
    off = np.zeros(n + 1, np.int64)
    tot = int(lib().or_neighbours_brute(n, _ptr(pos), float(h), _ptr(off), None, 0))
    idx = np.zeros(max(tot, 1), np.int64)
    lib().or_neighbours_brute(n, _ptr(pos), float(h), _ptr(off), _ptr(idx), tot)
    return off, idx[:tot]


def hilbert_keys(q):
    """Peano-Hilbert keys (63 bits, 21 levels) of grid coordinates."""
    q = np.ascontiguousarray(q, dtype=np.int32).reshape(-1, 3)
    k = np.zeros(q.shape[0], dtype=np.uint64)
    lib().or_hilbert_keys(q.shape[0], _ptr(q), _ptr(k))
    return k


class Tree:
    """The oracle's oct-tree over (pos, mass); nodes in depth-first preorder.
    order: "morton" visits children in octant order, "hilbert" in
    Peano-Hilbert order (the same cells, numbered in another order)."""

    ORDERS = {"morton": 0, "hilbert": 1}

    def __init__(self, pos, mass, order="morton"):
        self.pos = _pos(pos)
        self.mass = _mass(mass)
        self.n = self.pos.shape[0]
        self.key_order = order
        self._h = lib().or_tree_build_order(self.n, _ptr(self.pos), _ptr(self.mass),
                                            self.ORDERS[order])
        if not self._h:
            raise MemoryError("oracle tree build failed")
        self.nnodes = int(lib().or_tree_nnodes(self._h))
        self.ncells = int(lib().or_tree_ncells(self._h))
        r = np.zeros(7)
        lib().or_tree_root(self._h, _ptr(r))
        self.centre, self.L, self.corner = r[:3].copy(), float(r[3]), r[4:].copy()
        self._exp = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_tree_free(h)
            self._h = None

    def corners(self):
        """Integer corner of every node at its level (zeros for particles)."""
        c = np.zeros((self.nnodes, 3), np.int32)
        lib().or_tree_corners(self._h, _ptr(c))
        return c

    def quadrupoles(self):
        """Traceless quadrupole of every node about its centre of mass,
        (xx, yy, zz, xy, xz, yz), FP64; zeros for particles."""
        Q = np.zeros((self.nnodes, 6))
        assert lib().or_tree_export_quad(self._h, _ptr(Q)) == 0
        return Q

    def forces_quad(self, n_crit, theta, eps, with_amag=False, coords32=False):
        """forces() with the quadrupole term of every accepted cell:
        (acc, pot, npp, npc), plus sum_j |a_ij| of the monopole terms when
        with_amag; coords32 as in forces()."""
        acc = np.full((self.n, 3), np.nan)
        pot = np.full(self.n, np.nan)
        am = np.full(self.n, np.nan) if with_amag else None
        npp, npc = C.c_int64(0), C.c_int64(0)
        rc = lib().or_tree_forces_quad(self._h, int(n_crit), float(theta), float(eps),
                                       _ptr(acc), _ptr(pot), _ptr(am), C.byref(npp),
                                       C.byref(npc), 1 if coords32 else 0)
        assert rc == 0
        out = (acc, pot, int(npp.value), int(npc.value))
        return out + (am,) if with_amag else out

    def neighbours(self, h, group_form=False, n_crit=64):
        """Fixed-radius neighbours by the general treewalk: (offsets n+1,
        sorted caller indices), j != i with |x_j - x_i| <= h in FP64.
        group_form walks once per group of <= n_crit particles."""
        off = np.zeros(self.n + 1, np.int64)
        tot = int(lib().or_neighbours(self._h, float(h), 1 if group_form else 0,
                                      int(n_crit), _ptr(off), None, 0))
        assert tot >= 0
        idx = np.zeros(max(tot, 1), np.int64)
        lib().or_neighbours(self._h, float(h), 1 if group_form else 0, int(n_crit),
                            _ptr(off), _ptr(idx), tot)
        return off, idx[:tot]

    def export(self):
        if self._exp is None:
            nn, n = self.nnodes, self.n
            d = dict(
                order=np.zeros(n, np.int64), q=np.zeros((n, 3), np.int32),
                is_cell=np.zeros(nn, np.int8), level=np.zeros(nn, np.int32),
                first=np.zeros(nn, np.int64), count=np.zeros(nn, np.int64),
                next=np.zeros(nn, np.int64), more=np.zeros(nn, np.int64),
                parent=np.zeros(nn, np.int64), nchild=np.zeros(nn, np.int32),
                M=np.zeros(nn), com=np.zeros((nn, 3)),
                l=np.zeros(nn, np.float32), s=np.zeros(nn, np.float32),
                comf=np.zeros((nn, 3), np.float32))
            keys = ["order", "q", "is_cell", "level", "first", "count", "next",
                    "more", "parent", "nchild", "M", "com", "l", "s", "comf"]
            lib().or_tree_export(self._h, *[_ptr(d[k]) for k in keys])
            self._exp = d
        return self._exp

    def groups(self, n_crit):
        G = int(lib().or_groups(self._h, int(n_crit), None))
        g = np.zeros(max(G, 1), np.int64)
        lib().or_groups(self._h, int(n_crit), _ptr(g))
        return g[:G]

    def group_boxes(self, gnode):
        gnode = np.ascontiguousarray(gnode, dtype=np.int64)
        box = np.zeros((gnode.shape[0], 9), np.float32)
        lib().or_group_boxes(self._h, gnode.shape[0], _ptr(gnode), _ptr(box))
        return box

    def walk_group(self, gnode, box, theta, mode=1):
        box = np.ascontiguousarray(box, dtype=np.float32)
        n = int(lib().or_walk_group(self._h, int(gnode), _ptr(box), float(theta),
                                    int(mode), None, 0))
        out = np.zeros(max(n, 1), np.int64)
        lib().or_walk_group(self._h, int(gnode), _ptr(box), float(theta),
                            int(mode), _ptr(out), n)
        return out[:n]

    def walk_particle(self, slot, theta):
        n = int(lib().or_walk_particle(self._h, int(slot), float(theta), None, 0))
        out = np.zeros(max(n, 1), np.int64)
        lib().or_walk_particle(self._h, int(slot), float(theta), _ptr(out), n)
        return out[:n]

    def all_lists(self, n_crit, theta):
        """(gnode, box, offsets (G+1), entries) for every group."""
        gnode = self.groups(n_crit)
        box = self.group_boxes(gnode)
        G = gnode.shape[0]
        off = np.zeros(G + 1, np.int64)
        tot = int(lib().or_all_lists(self._h, G, _ptr(gnode), _ptr(box),
                                     float(theta), _ptr(off), None, 0))
        ent = np.zeros(max(tot, 1), np.int64)
        lib().or_all_lists(self._h, G, _ptr(gnode), _ptr(box), float(theta),
                           _ptr(off), _ptr(ent), tot)
        return gnode, box, off, ent[:tot]

    def forces(self, n_crit, theta, eps, gsel=None, theta_g=None, with_amag=False,
               coords32=False):
        """FP64 forces over the group lists.  Returns (acc, pot, npp, npc),
        and sum_j |a_ij| per particle last when with_amag; rows of particles
        outside the selected groups stay NaN.  coords32: sum over the
        group-relative FP32 coordinates and FP32 masses instead of the FP64
        positions (isolates arithmetic from representation error)."""
        acc = np.full((self.n, 3), np.nan)
        pot = np.full(self.n, np.nan)
        am = np.full(self.n, np.nan) if with_amag else None
        npp, npc = C.c_int64(0), C.c_int64(0)
        gs = None if gsel is None else np.ascontiguousarray(gsel, np.int64)
        tg = None if theta_g is None else np.ascontiguousarray(theta_g, np.float32)
        rc = lib().or_tree_forces(self._h, int(n_crit), float(theta), _ptr(tg),
                                  float(eps), 0 if gs is None else gs.shape[0],
                                  _ptr(gs), _ptr(acc), _ptr(pot), _ptr(am),
                                  C.byref(npp), C.byref(npc), 1 if coords32 else 0)
        assert rc == 0
        out = (acc, pot, int(npp.value), int(npc.value))
        return out + (am,) if with_amag else out


def leapfrog(pos, vel, mass, eps, dt, nsteps, use_tree=False, theta=0.75,
             n_crit=64, acc=None):
    """FP64 kick-drift-kick steps.  Returns (pos, vel, acc) after nsteps."""
    pos = _pos(pos).copy()
    vel = _pos(vel).copy()
    mass = _mass(mass)
    have = acc is not None
    acc = np.zeros_like(pos) if acc is None else _pos(acc).copy()
    rc = lib().or_leapfrog(pos.shape[0], _ptr(pos), _ptr(vel), _ptr(mass),
                           float(eps), float(dt), int(nsteps), int(use_tree),
                           float(theta), int(n_crit), _ptr(acc), int(have))
    assert rc == 0
    return pos, vel, acc
