"""GB300-native oct-tree group walk and softened gravity (arXiv:0909.0541).

A thin ctypes binding over ``libnb.so`` (CUDA for sm_103a, C ABI in
``include/nb.h``).  Every step of the path -- tree build, group walk, force
sum, leapfrog -- runs in the library's kernels; this module only marshals
torch tensors (device memory and streams) into the C calls.  There is no CPU
fallback: importing fails if the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NB_OK = 0
NB_ERR = {
    -1: "INVALID_ARG", -2: "CUDA", -3: "CAPACITY", -4: "WALK_LIMIT",
    -5: "NONFINITE", -6: "STATE", -7: "NOMEM", -8: "INTERNAL",
}
NB_FP32, NB_FP32_COMP, NB_FP64ACC = 0, 1, 2
PRECISION = {"fp32": NB_FP32, "fp32_comp": NB_FP32_COMP, "fp64acc": NB_FP64ACC}
KEY_ORDER = {"morton": 0, "hilbert": 1}

# flops per interaction by the paper's convention (Sec. "A Bare Many-body
# Performance on RV770 GPU")
FLOPS_PER_INTERACTION = 38

EXPORTED = [
    "nb_config_default", "nb_create", "nb_destroy", "nb_set_sync_checks",
    "nb_build_tree", "nb_walk_groups", "nb_forces", "nb_leapfrog_step",
    "nb_leapfrog_reset", "nb_leapfrog_acc", "nb_direct_sum", "nb_sync_status",
    "nb_get_stats", "nb_copy_tree", "nb_copy_groups", "nb_copy_lists",
    "nb_error_string", "nb_set_timing", "nb_get_timing", "nb_morton_order_noalloc", "nb_copy_list", "nb_mlp_workspace_size",
    "nb_mlp_forward", "nb_mlp_grad", "nb_mlp_train", "nb_group_features",
    "nb_walk_groups_learned", "nb_group_errors", "nb_theta_labels",
    "nb_copy_group_lengths", "nb_build_tree_batched", "nb_leapfrog_step_batched",
    "nb_graph_capture_leapfrog", "nb_graph_launch", "nb_autotune", "nb_selftest_wait",
    "nb_leapfrog_step_host", "nb_forces_fused", "nb_set_fused", "nb_set_feature_mode",
    "nb_direct_f32", "nb_direct_f32_workspace_size", "nb_set_key_order",
    "nb_theta_fit_workspace_size", "nb_theta_fit_curves", "nb_theta_allocate_workspace_size",
    "nb_theta_allocate", "nb_error_stats", "nb_column_stats", "nb_set_quadrupole",
    "nb_copy_quadrupoles", "nb_neighbours", "nb_walk_forces", "nb_set_overlap",
]
MLP_NPARAM = 9960
NFEAT_STRIDE = 16
NOALLOC_MAX_N = 1 << 20
PHASES = ("build", "walk", "force", "integrate")


class nb_config(C.Structure):
    _fields_ = [("max_n", C.c_int64), ("list_capacity", C.c_int64),
                ("stream", C.c_void_p), ("sync_checks", C.c_int),
                ("device", C.c_int), ("eps", C.c_float), ("theta", C.c_float),
                ("n_crit", C.c_int), ("precision", C.c_int), ("max_systems", C.c_int64)]


class nb_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_cells", C.c_int64), ("n_nodes", C.c_int64),
                ("n_groups", C.c_int64), ("list_entries", C.c_int64),
                ("max_list", C.c_int64), ("list_capacity", C.c_int64),
                ("n_pp", C.c_int64), ("n_pc", C.c_int64),
                ("max_level", C.c_int32), ("reserved", C.c_int32),
                ("n_pp_total", C.c_int64), ("n_pc_total", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class NBError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {NB_ERR.get(code, code)} "
                         f"({_lib.nb_error_string(code).decode()})")


def _load():
    path = _build.build()
    L = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.nb_config_default.argtypes = [C.POINTER(nb_config), i64]
    L.nb_config_default.restype = None
    L.nb_create.argtypes = [C.POINTER(vp), C.POINTER(nb_config)]
    L.nb_destroy.argtypes = [vp]
    L.nb_set_sync_checks.argtypes = [vp, i32]
    L.nb_build_tree.argtypes = [vp, vp, vp, i64]
    L.nb_walk_groups.argtypes = [vp, C.c_float, i32, vp]
    L.nb_forces.argtypes = [vp, C.c_float, vp, vp, i32]
    L.nb_forces_fused.argtypes = [vp, C.c_float, i32, C.c_float, vp, vp, i32]
    L.nb_set_fused.argtypes = [vp, i32]
    L.nb_set_key_order.argtypes = [vp, i32]
    L.nb_set_quadrupole.argtypes = [vp, i32]
    L.nb_walk_forces.argtypes = [vp, C.c_float, i32, C.c_float, vp, vp, i32]
    L.nb_set_overlap.argtypes = [vp, i32]
    L.nb_neighbours.argtypes = [vp, C.c_double, i32, vp, vp, i64, vp]
    L.nb_copy_quadrupoles.argtypes = [vp, vp]
    L.nb_set_feature_mode.argtypes = [vp, i32]
    L.nb_leapfrog_step.argtypes = [vp, vp, vp, vp, i64, C.c_double]
    L.nb_leapfrog_reset.argtypes = [vp]
    L.nb_leapfrog_step_host.argtypes = [vp, vp, vp, vp, i64, C.c_double]
    L.nb_leapfrog_acc.argtypes = [vp, vp]
    L.nb_direct_sum.argtypes = [vp, vp, i64, C.c_double, vp, i64, vp, vp, vp]
    L.nb_direct_f32_workspace_size.argtypes = [i64]
    L.nb_direct_f32_workspace_size.restype = C.c_size_t
    L.nb_direct_f32.argtypes = [vp, vp, i64, C.c_float, vp, vp, i32, vp, C.c_size_t, vp]
    L.nb_sync_status.argtypes = [vp]
    L.nb_selftest_wait.argtypes = [vp, C.c_uint]
    L.nb_get_stats.argtypes = [vp, C.POINTER(nb_stats)]
    L.nb_copy_tree.argtypes = [vp] * 14
    L.nb_copy_groups.argtypes = [vp] * 6
    L.nb_copy_lists.argtypes = [vp] * 4
    L.nb_copy_list.argtypes = [vp, i64, vp, vp, i64, vp]
    L.nb_set_timing.argtypes = [vp, i32]
    L.nb_get_timing.argtypes = [vp, vp, vp, vp]
    L.nb_morton_order_noalloc.argtypes = [vp, i64, vp, vp, vp]
    L.nb_group_features.argtypes = [vp, i32, vp, i64, vp]
    L.nb_build_tree_batched.argtypes = [vp, vp, vp, vp, i64, i64]
    L.nb_graph_capture_leapfrog.argtypes = [vp, vp, vp, vp, vp, i64, i64, C.c_double, i32]
    L.nb_graph_launch.argtypes = [vp]
    L.nb_autotune.argtypes = [vp, vp, vp, vp, i64, i64, C.c_float, C.c_float, vp, i32, i32, vp, vp,
                              vp, vp, vp]
    L.nb_leapfrog_step_batched.argtypes = [vp, vp, vp, vp, vp, i64, i64, C.c_double]
    L.nb_copy_group_lengths.argtypes = [vp, vp, i64]
    L.nb_walk_groups_learned.argtypes = [vp, i32, vp, C.c_float, vp]
    L.nb_group_errors.argtypes = [vp, vp, vp, vp, i64, vp, vp]
    L.nb_theta_labels.argtypes = [vp, vp, vp, vp, i32, i64, C.c_float, C.c_float, vp, vp]
    L.nb_theta_fit_workspace_size.argtypes = [i64, i32, i32]
    L.nb_theta_fit_workspace_size.restype = C.c_size_t
    L.nb_theta_fit_curves.argtypes = [vp, i64, i32, vp, i32, vp, vp, i32, vp, vp, vp,
                                      C.c_size_t, vp]
    L.nb_theta_allocate_workspace_size.argtypes = [i64, i64]
    L.nb_theta_allocate_workspace_size.restype = C.c_size_t
    L.nb_theta_allocate.argtypes = [vp, vp, vp, vp, vp, vp, i32, i64, C.c_double, C.c_double,
                                    C.c_double, i32, vp, vp, i64, vp, vp, vp, C.c_size_t, vp]
    L.nb_error_stats.argtypes = [vp, vp, vp, i64, C.c_double, vp, vp, vp]
    L.nb_column_stats.argtypes = [vp, i64, i32, i32, vp, vp, vp]
    L.nb_mlp_workspace_size.argtypes = [i64]
    L.nb_mlp_workspace_size.restype = C.c_size_t
    L.nb_mlp_forward.argtypes = [vp, vp, i64, vp, C.c_float, vp, vp]
    L.nb_mlp_grad.argtypes = [vp, vp, vp, i64, vp, vp, vp, vp]
    L.nb_mlp_train.argtypes = [vp, vp, vp, vp, vp, i64, vp, i32, i32, C.c_float, vp, vp, vp, vp]
    L.nb_error_string.argtypes = [i32]
    L.nb_error_string.restype = C.c_char_p
    return L


_lib = _load()


def library_path() -> str:
    return _build.LIB


def _check(rc, where):
    if rc != NB_OK:
        raise NBError(rc, where)


def _dptr(t, dtype, shape_last=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor of the given dtype."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError(f"{name} must have shape (n, {shape_last})")
    return t.data_ptr()


def _hptr(a):
    return None if a is None else a.ctypes.data


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class NBody:
    """One libnb context: storage for up to max_n particles on one GPU."""

    def __init__(self, max_n, *, eps=0.01, theta=0.6, n_crit=64,
                 precision="fp32", list_capacity=0, sync_checks=True,
                 stream=None, device=None, max_systems=1):
        import torch
        dev = torch.cuda.current_device() if device is None else int(device)
        cfg = nb_config()
        _lib.nb_config_default(C.byref(cfg), int(max_n))
        cfg.list_capacity = int(list_capacity)
        cfg.stream = _stream_handle(stream)
        cfg.sync_checks = 1 if sync_checks else 0
        cfg.device = dev
        cfg.eps = float(eps)
        cfg.theta = float(theta)
        cfg.n_crit = int(n_crit)
        cfg.precision = PRECISION.get(precision, precision)
        cfg.max_systems = int(max_systems)
        self.cfg = cfg
        self.max_n = int(max_n)
        h = C.c_void_p()
        _check(_lib.nb_create(C.byref(h), C.byref(cfg)), "nb_create")
        self._h = h
        self.n = 0

    def close(self):
        if getattr(self, "_h", None):
            _lib.nb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the path ---------------------------------------------------------
    def set_sync_checks(self, on: bool):
        _check(_lib.nb_set_sync_checks(self._h, 1 if on else 0), "nb_set_sync_checks")

    def build_tree(self, pos, mass):
        import torch
        n = int(pos.shape[0])
        _check(_lib.nb_build_tree(self._h, _dptr(pos, torch.float64, 3, "pos"),
                                  _dptr(mass, torch.float32, None, "mass"), n),
               "nb_build_tree")
        self.n = n
        self._nsys = 1

    def build_tree_batched(self, pos, mass, offsets):
        """offsets: (n_systems + 1,) int64 CUDA tensor of row offsets."""
        import torch
        n = int(pos.shape[0])
        _check(_lib.nb_build_tree_batched(self._h, _dptr(pos, torch.float64, 3, "pos"),
                                          _dptr(mass, torch.float32, None, "mass"),
                                          _dptr(offsets, torch.int64, None, "offsets"),
                                          int(offsets.shape[0]) - 1, n), "nb_build_tree_batched")
        self.n = n
        self._nsys = int(offsets.shape[0]) - 1

    def leapfrog_step_batched(self, pos, vel, mass, offsets, dt):
        import torch
        _check(_lib.nb_leapfrog_step_batched(self._h, _dptr(pos, torch.float64, 3, "pos"),
                                             _dptr(vel, torch.float64, 3, "vel"),
                                             _dptr(mass, torch.float32, None, "mass"),
                                             _dptr(offsets, torch.int64, None, "offsets"),
                                             int(offsets.shape[0]) - 1, int(pos.shape[0]),
                                             float(dt)), "nb_leapfrog_step_batched")
        self.n = int(pos.shape[0])

    def graph_capture_leapfrog(self, pos, vel, mass, dt, nsteps, offsets=None):
        import torch
        nsys = 1 if offsets is None else int(offsets.shape[0]) - 1
        _check(_lib.nb_graph_capture_leapfrog(
            self._h, _dptr(pos, torch.float64, 3, "pos"), _dptr(vel, torch.float64, 3, "vel"),
            _dptr(mass, torch.float32, None, "mass"),
            _dptr(offsets, torch.int64, None, "offsets"), nsys, int(pos.shape[0]), float(dt),
            int(nsteps)), "nb_graph_capture_leapfrog")

    def graph_launch(self):
        _check(_lib.nb_graph_launch(self._h), "nb_graph_launch")

    def autotune(self, pos, mass, eps, theta, n_crits=(32, 64, 128, 256, 512), reps=3,
                 offsets=None):
        """Times walk + FP32 force over n_crit x item rows (1, 2: 32 or 64
        targets per warp) x j-tile depth (32, 64) x block size (256, 128) and
        keeps the fastest.  Returns ({"n_crit", "rows", "tile", "block"},
        {(n_crit, rows, tile, block): ms}); offsets (int64 CUDA tensor of
        n_systems + 1 row offsets) tunes a batch of systems."""
        import torch
        cand = np.asarray(n_crits, np.int32)
        ms = np.zeros(8 * len(cand), np.float32)
        bn, br, bt, bb = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0)
        nsys = 1 if offsets is None else int(offsets.shape[0]) - 1
        _check(_lib.nb_autotune(self._h, _dptr(pos, torch.float64, 3, "pos"),
                                _dptr(mass, torch.float32, None, "mass"),
                                _dptr(offsets, torch.int64, None, "offsets"), nsys,
                                int(pos.shape[0]),
                                float(eps), float(theta), _hptr(cand), len(cand), int(reps),
                                C.byref(bn), C.byref(br), C.byref(bt), C.byref(bb), _hptr(ms)),
               "nb_autotune")
        table = {}
        for k, c in enumerate(cand):
            for r in range(2):
                for ti, tile in enumerate((32, 64)):
                    for bi, block in enumerate((256, 128)):
                        table[(int(c), r + 1, tile, block)] = float(
                            ms[((k * 2 + r) * 2 + ti) * 2 + bi])
        self.cfg.n_crit = bn.value
        return {"n_crit": bn.value, "rows": br.value, "tile": bt.value,
                "block": bb.value}, table

    def walk_groups(self, theta, n_crit, theta_per_group=None):
        import torch
        _check(_lib.nb_walk_groups(self._h, float(theta), int(n_crit),
                                   _dptr(theta_per_group, torch.float32, None,
                                         "theta_per_group")),
               "nb_walk_groups")

    def forces(self, eps, acc, pot=None, precision="fp32"):
        import torch
        _check(_lib.nb_forces(self._h, float(eps), _dptr(acc, torch.float32, 3, "acc"),
                              _dptr(pot, torch.float32, None, "pot"),
                              PRECISION.get(precision, precision)), "nb_forces")

    def set_feature_mode(self, mode: int):
        """Learned-theta features: 0 from the probe walk, 1 tree-only (no walk)."""
        _check(_lib.nb_set_feature_mode(self._h, int(mode)), "nb_set_feature_mode")

    def set_key_order(self, order: str):
        """Particle order of the next builds: "morton" (default) or "hilbert"."""
        _check(_lib.nb_set_key_order(self._h, KEY_ORDER[order]), "nb_set_key_order")

    def set_quadrupole(self, on: bool):
        """Quadrupole cells from the next build on (nb_set_quadrupole)."""
        _check(_lib.nb_set_quadrupole(self._h, 1 if on else 0), "nb_set_quadrupole")

    def copy_quadrupoles(self) -> np.ndarray:
        """(n_nodes, 6) FP64 quadrupoles of the current tree, preorder."""
        q = np.zeros((self.stats()["n_nodes"], 6))
        _check(_lib.nb_copy_quadrupoles(self._h, _hptr(q)), "nb_copy_quadrupoles")
        return q

    def neighbours(self, h, n_crit=64):
        """(offsets (n+1,) int64, caller indices int32) CUDA tensors of every
        particle's neighbours within h, ascending (nb_neighbours)."""
        import torch
        n = self.n
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        tot = C.c_int64(0)
        _check(_lib.nb_neighbours(self._h, float(h), int(n_crit), off.data_ptr(), None, 0,
                                  C.byref(tot)), "nb_neighbours")
        idx = torch.empty(max(tot.value, 1), dtype=torch.int32, device="cuda")
        _check(_lib.nb_neighbours(self._h, float(h), int(n_crit), off.data_ptr(), idx.data_ptr(),
                                  int(idx.numel()), C.byref(tot)), "nb_neighbours")
        return off, idx[:tot.value]

    def walk_forces(self, theta, n_crit, eps, acc, pot=None, precision="fp32"):
        """Groups, walk and force sum with the walk overlapping the force sum
        in one launch (nb_walk_forces): the same results as walk_groups +
        forces."""
        import torch
        _check(_lib.nb_walk_forces(self._h, float(theta), int(n_crit), float(eps),
                                   _dptr(acc, torch.float32, 3, "acc"),
                                   _dptr(pot, torch.float32, None, "pot"),
                                   PRECISION.get(precision, precision)), "nb_walk_forces")

    def set_overlap(self, on: bool):
        """Leapfrog force passes through walk_forces (nb_set_overlap)."""
        _check(_lib.nb_set_overlap(self._h, 1 if on else 0), "nb_set_overlap")

    def set_fused(self, on: bool):
        """Leapfrog force passes without interaction lists (nb_set_fused)."""
        _check(_lib.nb_set_fused(self._h, 1 if on else 0), "nb_set_fused")

    def forces_fused(self, theta, n_crit, eps, acc, pot=None, precision="fp32"):
        """Groups, walk and force in one pass with no interaction lists in
        device memory (same results as walk_groups + forces)."""
        import torch
        _check(_lib.nb_forces_fused(self._h, float(theta), int(n_crit), float(eps),
                                    _dptr(acc, torch.float32, 3, "acc"),
                                    _dptr(pot, torch.float32, None, "pot"),
                                    PRECISION.get(precision, precision)), "nb_forces_fused")

    def leapfrog_step(self, pos, vel, mass, dt):
        import torch
        _check(_lib.nb_leapfrog_step(self._h, _dptr(pos, torch.float64, 3, "pos"),
                                     _dptr(vel, torch.float64, 3, "vel"),
                                     _dptr(mass, torch.float32, None, "mass"),
                                     int(pos.shape[0]), float(dt)), "nb_leapfrog_step")
        self.n = int(pos.shape[0])

    def leapfrog_step_host(self, pos, vel, mass, dt):
        """One KDK step on host (CPU) tensors or arrays, pinned for overlap:
        pos, vel (n x 3 float64) are updated in place by the library, which
        does the host-device copies itself."""
        def hp(t, dtype, cols, name):
            a = t.numpy() if hasattr(t, "numpy") else t
            if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
                raise TypeError(f"{name} must be a C-contiguous {np.dtype(dtype).name} host array")
            if cols and (a.ndim != 2 or a.shape[1] != cols):
                raise TypeError(f"{name} must be n x {cols}")
            return a.ctypes.data, a.shape[0]
        p, n = hp(pos, np.float64, 3, "pos")
        v, nv = hp(vel, np.float64, 3, "vel")
        m, nm = hp(mass, np.float32, None, "mass")
        if nv != n or nm != n:
            raise ValueError("pos, vel and mass must have the same length")
        _check(_lib.nb_leapfrog_step_host(self._h, p, v, m, int(n), float(dt)),
               "nb_leapfrog_step_host")
        self.n = int(n)

    def leapfrog_reset(self):
        _check(_lib.nb_leapfrog_reset(self._h), "nb_leapfrog_reset")

    def leapfrog_acc(self, acc):
        import torch
        _check(_lib.nb_leapfrog_acc(self._h, _dptr(acc, torch.float32, 3, "acc")),
               "nb_leapfrog_acc")

    def group_features(self, n_crit):
        """(G, 16) float32 CUDA tensor of the probe-walk features."""
        import torch
        G = C.c_int64(0)
        _check(_lib.nb_group_features(self._h, int(n_crit), None, 0, C.byref(G)),
               "nb_group_features")
        feat = torch.empty((max(G.value, 1), NFEAT_STRIDE), dtype=torch.float32, device="cuda")
        _check(_lib.nb_group_features(self._h, int(n_crit), feat.data_ptr(), G.value, None),
               "nb_group_features")
        self.sync_status()
        return feat[:G.value]

    def walk_groups_learned(self, n_crit, params, theta_fallback=0.6, theta_out=None):
        import torch
        _check(_lib.nb_walk_groups_learned(self._h, int(n_crit),
                                           _dptr(params, torch.float32, None, "params"),
                                           float(theta_fallback),
                                           _dptr(theta_out, torch.float32, None, "theta_out")),
               "nb_walk_groups_learned")

    def set_timing(self, on: bool):
        _check(_lib.nb_set_timing(self._h, 1 if on else 0), "nb_set_timing")

    def get_timing(self) -> dict:
        """Per-phase device milliseconds and call counts since the last call,
        and the number of libnb kernel launches in that time.  Phases inside a
        graph captured with timing on count once per graph launch (the last
        launch's times, scaled by the launches since the last call)."""
        ms = np.zeros(4)
        calls = np.zeros(4, np.int64)
        launches = np.zeros(1, np.int64)
        _check(_lib.nb_get_timing(self._h, _hptr(ms), _hptr(calls), _hptr(launches)),
               "nb_get_timing")
        out = {p: (float(ms[i]), int(calls[i])) for i, p in enumerate(PHASES)}
        out["launches"] = int(launches[0])
        return out

    def sync_status(self):
        _check(_lib.nb_sync_status(self._h), "nb_sync_status")

    def selftest_wait(self, spin_limit: int) -> int:
        """Status of one warp's bounded wait on a count nothing raises
        (NB_ERR_INTERNAL when the wait gave up as designed)."""
        return int(_lib.nb_selftest_wait(self._h, int(spin_limit)))

    def stats(self) -> dict:
        st = nb_stats()
        _check(_lib.nb_get_stats(self._h, C.byref(st)), "nb_get_stats")
        return st.as_dict()

    # -- debug export -------------------------------------------------------
    def copy_tree(self) -> dict:
        st = self.stats()
        n, nn = st["n"], st["n_nodes"]
        d = dict(root=np.zeros(max(7, 8 * getattr(self, "_nsys", 1))), keys=np.zeros(n, np.uint64), perm=np.zeros(n, np.int32),
                 level=np.zeros(nn, np.int32), first=np.zeros(nn, np.int32),
                 count=np.zeros(nn, np.int32), next=np.zeros(nn, np.int32),
                 parent=np.zeros(nn, np.int32), nchild=np.zeros(nn, np.int32),
                 M=np.zeros(nn), com=np.zeros((nn, 3)), l=np.zeros(nn, np.float32),
                 s=np.zeros(nn, np.float32))
        keys = ["root", "keys", "perm", "level", "first", "count", "next", "parent",
                "nchild", "M", "com", "l", "s"]
        _check(_lib.nb_copy_tree(self._h, *[_hptr(d[k]) for k in keys]), "nb_copy_tree")
        d["is_cell"] = (d["level"] >= 0).astype(np.int8)
        return d

    def copy_perm(self) -> np.ndarray:
        """Sorted slot -> caller index of the current tree."""
        perm = np.zeros(self.stats()["n"], np.int32)
        _check(_lib.nb_copy_tree(self._h, None, None, _hptr(perm), *([None] * 10)),
               "nb_copy_tree")
        return perm

    def copy_groups(self) -> dict:
        G = self.stats()["n_groups"]
        d = dict(gnode=np.zeros(G, np.int32), gfirst=np.zeros(G, np.int32),
                 gcount=np.zeros(G, np.int32), box=np.zeros((G, 9), np.float32),
                 invtheta=np.zeros(G, np.float32))
        _check(_lib.nb_copy_groups(self._h, *[_hptr(d[k]) for k in
                                              ["gnode", "gfirst", "gcount", "box", "invtheta"]]),
               "nb_copy_groups")
        return d

    def copy_group_lengths(self) -> np.ndarray:
        G = self.stats()["n_groups"]
        out = np.zeros(G, np.int32)
        _check(_lib.nb_copy_group_lengths(self._h, _hptr(out), G), "nb_copy_group_lengths")
        return out

    def copy_list(self, group, with_xm=False):
        """(node ids, FP32 records or None) of one group's list."""
        n = C.c_int64(0)
        _check(_lib.nb_copy_list(self._h, int(group), None, None, 0, C.byref(n)), "nb_copy_list")
        ids = np.zeros(n.value, np.int32)
        xm = np.zeros((n.value, 4), np.float32) if with_xm else None
        _check(_lib.nb_copy_list(self._h, int(group), _hptr(ids), _hptr(xm), n.value,
                                 C.byref(n)), "nb_copy_list")
        return ids, xm

    def copy_lists(self, with_xm=False) -> dict:
        st = self.stats()
        G, tot = st["n_groups"], st["list_entries"]
        d = dict(offsets=np.zeros(G + 1, np.int64), entries=np.zeros(tot, np.int32),
                 xm=np.zeros((tot, 4), np.float32) if with_xm else None)
        _check(_lib.nb_copy_lists(self._h, _hptr(d["offsets"]), _hptr(d["entries"]),
                                  _hptr(d["xm"])), "nb_copy_lists")
        return d


def direct_sum(pos, mass, eps, targets=None, stream=None):
    """FP64 GPU direct sum of Eq. (gravity) for `targets` (int64 indices, all
    when None).  Returns (acc (nt,3) float64, pot (nt,) float64) tensors."""
    import torch
    n = int(pos.shape[0])
    nt = n if targets is None else int(targets.shape[0])
    acc = torch.empty((nt, 3), dtype=torch.float64, device=pos.device)
    pot = torch.empty(nt, dtype=torch.float64, device=pos.device)
    _check(_lib.nb_direct_sum(_dptr(pos, torch.float64, 3, "pos"),
                              _dptr(mass, torch.float32, None, "mass"), n, float(eps),
                              _dptr(targets, torch.int64, None, "targets"), nt,
                              acc.data_ptr(), pot.data_ptr(), _stream_handle(stream)),
           "nb_direct_sum")
    return acc, pot


def direct_f32(pos, mass, eps, precision="fp32", acc=None, pot=None, work=None, stream=None):
    """Brute-force FP32 sum of Eq. (gravity) over all pairs (nb_direct_f32).
    Returns (acc (n,3) float32, pot (n,) float32) CUDA tensors; `work` (uint8
    CUDA tensor of direct_f32_workspace_size(n) bytes) may be passed to reuse
    a workspace, as may acc / pot."""
    import torch
    n = int(pos.shape[0])
    dev = pos.device
    if acc is None:
        acc = torch.empty((n, 3), dtype=torch.float32, device=dev)
    if pot is None:
        pot = torch.empty(n, dtype=torch.float32, device=dev)
    need = direct_f32_workspace_size(n)
    if work is None:
        work = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    _check(_lib.nb_direct_f32(_dptr(pos, torch.float64, 3, "pos"),
                              _dptr(mass, torch.float32, None, "mass"), n, float(eps),
                              _dptr(acc, torch.float32, 3, "acc"),
                              _dptr(pot, torch.float32, None, "pot"),
                              PRECISION.get(precision, precision),
                              _dptr(work, torch.uint8, None, "work"), int(work.numel()),
                              _stream_handle(stream)), "nb_direct_f32")
    return acc, pot


def direct_f32_workspace_size(n) -> int:
    """Workspace bytes nb_direct_f32 needs for n particles on the current device."""
    return int(_lib.nb_direct_f32_workspace_size(int(n)))


def morton_order_noalloc(pos, keys_out, perm_out, stream=None):
    """Sorted Morton keys and sorted slot -> caller index for n <= NOALLOC_MAX_N
    particles, computed without any device allocation (the library's static
    scratch); keys_out (n,) int64 holding uint64 bits, perm_out (n,) int32.
    pos, keys_out and perm_out must be on one device; the call runs with that
    device current, on `stream` (default: that device's current stream)."""
    import torch
    n = int(pos.shape[0])
    for t, name, dt in ((keys_out, "keys_out", torch.int64), (perm_out, "perm_out", torch.int32)):
        if not isinstance(t, torch.Tensor) or t.dim() != 1 or int(t.shape[0]) != n:
            raise ValueError(f"{name} must be a 1-D tensor of {n} elements")
    pp = _dptr(pos, torch.float64, 3, "pos")
    kp = _dptr(keys_out, torch.int64, None, "keys_out")
    qp = _dptr(perm_out, torch.int32, None, "perm_out")
    if keys_out.device != pos.device or perm_out.device != pos.device:
        raise ValueError("pos, keys_out and perm_out must be on the same device")
    with torch.cuda.device(pos.device):
        s = stream if stream is not None else torch.cuda.current_stream(pos.device)
        if s.device != pos.device:
            raise ValueError("stream must belong to the tensors' device")
        _check(_lib.nb_morton_order_noalloc(pp, n, kp, qp, s.cuda_stream),
               "nb_morton_order_noalloc")


# ---------------------------------------------------------------- learned theta
def _workspace(batch, device):
    import torch
    return torch.empty(int(_lib.nb_mlp_workspace_size(int(batch))), dtype=torch.uint8,
                       device=device)


def mlp_forward(params, feat, fallback=0.6, stream=None):
    """theta (n,) for feature rows feat (n, 16) float32 with the network
    parameters params (MLP_NPARAM,) float32."""
    import torch
    n = int(feat.shape[0])
    theta = torch.empty(n, dtype=torch.float32, device=feat.device)
    work = _workspace(max(n, 1), feat.device)
    _check(_lib.nb_mlp_forward(_dptr(params, torch.float32, None, "params"),
                               _dptr(feat, torch.float32, NFEAT_STRIDE, "feat"), n,
                               theta.data_ptr(), float(fallback), work.data_ptr(),
                               _stream_handle(stream)), "nb_mlp_forward")
    return theta


def mlp_grad(params, feat, labels, stream=None):
    """(gradient (MLP_NPARAM,), summed loss) of one batch."""
    import torch
    n = int(feat.shape[0])
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=feat.device)
    loss = torch.empty(1, dtype=torch.float32, device=feat.device)
    work = _workspace(n, feat.device)
    _check(_lib.nb_mlp_grad(_dptr(params, torch.float32, None, "params"),
                            _dptr(feat, torch.float32, NFEAT_STRIDE, "feat"),
                            _dptr(labels, torch.float32, None, "labels"), n,
                            grad.data_ptr(), loss.data_ptr(), work.data_ptr(),
                            _stream_handle(stream)), "nb_mlp_grad")
    return grad, loss


def mlp_train(params, feat, labels, order, epochs, batch, lr, stream=None):
    """Adam training in place on params; order (epochs, n) int32 shuffles.
    Returns the per-epoch summed loss."""
    import torch
    n = int(feat.shape[0])
    dev = feat.device
    m = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=dev)
    v = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=dev)
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=dev)
    hist = torch.empty(int(epochs), dtype=torch.float32, device=dev)
    work = _workspace(batch, dev)
    _check(_lib.nb_mlp_train(_dptr(params, torch.float32, None, "params"), m.data_ptr(),
                             v.data_ptr(), _dptr(feat, torch.float32, NFEAT_STRIDE, "feat"),
                             _dptr(labels, torch.float32, None, "labels"), n,
                             _dptr(order, torch.int32, None, "order"), int(epochs), int(batch),
                             float(lr), grad.data_ptr(), hist.data_ptr(), work.data_ptr(),
                             _stream_handle(stream)), "nb_mlp_train")
    return hist


def group_errors(acc, ref, targets, off, stream=None):
    """Median |da|/|a| per sampled group (see nb_group_errors)."""
    import torch
    S = int(off.shape[0]) - 1
    err = torch.empty(S, dtype=torch.float32, device=acc.device)
    _check(_lib.nb_group_errors(_dptr(acc, torch.float32, 3, "acc"),
                                _dptr(ref, torch.float64, 3, "ref"),
                                _dptr(targets, torch.int64, None, "targets"),
                                _dptr(off, torch.int64, None, "off"), S, err.data_ptr(),
                                _stream_handle(stream)), "nb_group_errors")
    return err


def theta_labels(err, grid, budget=1e-3, cost=None, size=None, lam=0.0, stream=None):
    """Labels from errors (T, S) over a theta grid; with cost (T, S) and size
    (S,) the cost-aware labels at exchange rate lam (see nb_theta_labels)."""
    import torch
    T, S = int(err.shape[0]), int(err.shape[1])
    lab = torch.empty(S, dtype=torch.float32, device=err.device)
    _check(_lib.nb_theta_labels(_dptr(err.contiguous(), torch.float32, None, "err"),
                                None if cost is None else
                                _dptr(cost.contiguous(), torch.float32, None, "cost"),
                                None if size is None else _dptr(size, torch.float32, None, "size"),
                                _dptr(grid, torch.float32, None, "grid"), T, S, float(budget),
                                float(lam), lab.data_ptr(), _stream_handle(stream)),
           "nb_theta_labels")
    return lab


def theta_fit_curves(feat, err, cost, cols, stream=None):
    """Curves predicted from the feature columns `cols` of feat (S, stride)
    float32 for err, cost (T, S) float32: (pred ln error, pred cost), each
    (T, S) float64 CUDA tensors (nb_theta_fit_curves)."""
    import torch
    S, stride = int(feat.shape[0]), int(feat.shape[1])
    T = int(err.shape[0])
    c = np.ascontiguousarray(cols, np.int32)
    dev = feat.device
    pe = torch.empty((T, S), dtype=torch.float64, device=dev)
    pc = torch.empty((T, S), dtype=torch.float64, device=dev)
    need = int(_lib.nb_theta_fit_workspace_size(S, len(c), T))
    work = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    _check(_lib.nb_theta_fit_curves(_dptr(feat, torch.float32, stride, "feat"), S, stride,
                                    _hptr(c), len(c), _dptr(err.contiguous(), torch.float32,
                                                            None, "err"),
                                    _dptr(cost.contiguous(), torch.float32, None, "cost"), T,
                                    pe.data_ptr(), pc.data_ptr(), work.data_ptr(),
                                    int(work.numel()), _stream_handle(stream)),
           "nb_theta_fit_curves")
    return pe, pc


def theta_allocate(err, cost, size, grid, budget, lam_lo, lam_hi, iters, pred=None,
                   perr=None, poff=None, stream=None):
    """Labels (S,) float32 and (lambda, statistic) of the allocation rule
    (nb_theta_allocate); pred = (pred ln error, pred cost) from
    theta_fit_curves, or None for the measured curves; perr (T, P) float32
    per-particle errors with poff (S + 1,) int64 offsets: hold the median
    over particles at the budget instead of the weighted median of group
    medians."""
    import torch
    T, S = int(err.shape[0]), int(err.shape[1])
    P = 0 if perr is None else int(perr.shape[1])
    dev = err.device
    lab = torch.empty(S, dtype=torch.float32, device=dev)
    res = torch.empty(2, dtype=torch.float64, device=dev)
    need = int(_lib.nb_theta_allocate_workspace_size(S, P))
    work = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    pe, pc = pred if pred is not None else (None, None)
    _check(_lib.nb_theta_allocate(
        None if pe is None else _dptr(pe.contiguous(), torch.float64, None, "pred_lnerr"),
        None if pc is None else _dptr(pc.contiguous(), torch.float64, None, "pred_cost"),
        _dptr(err.contiguous(), torch.float32, None, "err"),
        _dptr(cost.contiguous(), torch.float32, None, "cost"),
        _dptr(size, torch.float32, None, "size"), _dptr(grid, torch.float32, None, "grid"),
        T, S, float(budget), float(lam_lo), float(lam_hi), int(iters),
        None if perr is None else _dptr(perr.contiguous(), torch.float32, None, "perr"),
        None if poff is None else _dptr(poff, torch.int64, None, "poff"), P,
        lab.data_ptr(), res.data_ptr(), work.data_ptr(), int(work.numel()),
        _stream_handle(stream)), "nb_theta_allocate")
    r = res.cpu().numpy()
    return lab, float(r[0]), float(r[1])


def error_stats(acc, ref, targets=None, q=0.99, err_out=None, stream=None):
    """(median, nearest-rank q-quantile) of |a - ref| / |ref| over the
    targets (nb_error_stats): acc (n, 3) float32, ref (nt, 3) float64;
    err_out (nt,) float32 receives the per-target errors when given."""
    import torch
    nt = int(ref.shape[0])
    out = torch.empty(2, dtype=torch.float64, device=ref.device)
    err = err_out if err_out is not None else \
        torch.empty(max(nt, 1), dtype=torch.float32, device=ref.device)
    _check(_lib.nb_error_stats(_dptr(acc, torch.float32, 3, "acc"),
                               _dptr(ref, torch.float64, 3, "ref"),
                               _dptr(targets, torch.int64, None, "targets"), nt, float(q),
                               out.data_ptr(), _dptr(err, torch.float32, None, "err_out"),
                               _stream_handle(stream)), "nb_error_stats")
    o = out.cpu().numpy()
    return float(o[0]), float(o[1])


def column_stats(feat, ncols, stream=None):
    """(mean, spread) float64 CUDA tensors of the first ncols columns of feat
    (nb_column_stats)."""
    import torch
    S, stride = int(feat.shape[0]), int(feat.shape[1])
    mu = torch.empty(ncols, dtype=torch.float64, device=feat.device)
    sd = torch.empty(ncols, dtype=torch.float64, device=feat.device)
    _check(_lib.nb_column_stats(_dptr(feat, torch.float32, stride, "feat"), S, stride,
                                int(ncols), mu.data_ptr(), sd.data_ptr(),
                                _stream_handle(stream)), "nb_column_stats")
    return mu, sd
