"""Thin ctypes binding of the C-ABI in ``include/mr_lbm.h``.

Argument marshalling only: every step of the time step runs in the CUDA
kernels of ``libmrlbm.so``.  There is no CPU fallback: if the library is
missing or cannot be loaded, every entry point raises.  Arrays may be numpy
arrays (host memory) or CUDA tensors (device memory, passed by pointer on
the handle's stream).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrlbm.so")

MR_STATUS = {0: "MR_OK", 1: "MR_EINVAL", 2: "MR_ENOMEM", 3: "MR_ECUDA", 4: "MR_ECAPACITY",
             5: "MR_ENOCONV", 6: "MR_ENONFINITE", 7: "MR_ESTATE", 8: "MR_EINTERNAL"}
SCHEMES = {"d1q2_advection": 0, "d1q2_burgers": 1, "d1q3_shallow_water": 2, "d2q4x4_euler": 3,
           "d2q9_ns": 4, "d3q6_advection": 5}
BCS = {"periodic": 0, "copy": 1, "bounce_back": 2, "anti_bounce_back": 3, "bounce_back_velocity": 4}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
FUNCTIONALS = {"ke_sum": 1, "ke_final": 2}
NCONS = {0: 1, 1: 1, 2: 2, 3: 4, 4: 3, 5: 1}
NPOP = {0: 2, 1: 2, 2: 3, 3: 16, 4: 9, 5: 6}
DIM = {0: 1, 1: 1, 2: 1, 3: 2, 4: 2, 5: 3}


class MrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s" % (where, MR_STATUS.get(status, status)))


class MrConfig(C.Structure):
    _fields_ = [
        ("scheme", C.c_int),
        ("lambda_", C.c_double),
        ("s", C.c_double * 16),
        ("phys", C.c_double * 8),
        ("xmin", C.c_double * 3),
        ("xmax", C.c_double * 3),
        ("roots", C.c_int * 3),
        ("min_level", C.c_int),
        ("max_level", C.c_int),
        ("eps", C.c_double),
        ("mu_bar", C.c_int),
        ("pred_s", C.c_int),
        ("bc", C.c_int * 6),
        ("cross_sign", C.c_int),
        ("precision", C.c_int),
        ("leaf_capacity", C.c_longlong),
        ("obstacle", C.c_int),
        ("exact_collision", C.c_int),
    ]


_lib = None


def library():
    """Load libmrlbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmrlbm.so is missing: run __graft_entry__.build() "
                               "(or python -m paper_2103_02903_gb300.build) first")
        L = C.CDLL(LIB_PATH)
        vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.c_double
        L.mr_lbm_create.argtypes = [C.POINTER(MrConfig), vp, C.POINTER(vp)]
        L.mr_lbm_destroy.argtypes = [vp]
        L.mr_lbm_init.argtypes = [vp, vp, i]
        L.mr_lbm_step.argtypes = [vp, i]
        L.mr_lbm_adapt.argtypes = [vp]
        L.mr_lbm_project.argtypes = [vp, i, vp, i]
        L.mr_lbm_project_noalloc.argtypes = [vp, i, vp, i]
        L.mr_lbm_get_leaves.argtypes = [vp, C.POINTER(ll), vp, vp, vp, i]
        L.mr_lbm_set_leaves.argtypes = [vp, ll, vp, vp, vp, i]
        L.mr_lbm_stats.argtypes = [vp, vp, C.POINTER(d), C.POINTER(d)]
        L.mr_lbm_counters.argtypes = [vp, C.POINTER(ll), C.POINTER(ll)]
        L.mr_lbm_launch_count.argtypes = [vp]
        L.mr_lbm_launch_count.restype = ll
        L.mr_lbm_profile_enable.argtypes = [vp, i]
        L.mr_lbm_profile_read.argtypes = [vp, C.POINTER(d), C.POINTER(ll)]
        L.mr_lbm_synchronize.argtypes = [vp]
        L.mr_lbm_strerror.argtypes = [i]
        L.mr_lbm_strerror.restype = C.c_char_p
        L.mr_lbm_flattened_weights.argtypes = [i, i, i, i, i, vp]
        L.mr_lbm_flattened_weights_s.argtypes = [i, i, i, i, i, i, i, vp]
        L.mr_lbm_adjoint.argtypes = [vp, vp, i, i, i, i, C.POINTER(d), vp, vp]
        L.mr_lbm_adjoint.restype = i
        L.mr_lbm_batch_create.argtypes = [C.POINTER(MrConfig), i, vp, C.POINTER(vp)]
        L.mr_lbm_batch_instance.argtypes = [vp, i, C.POINTER(vp)]
        L.mr_lbm_batch_step.argtypes = [vp, i]
        L.mr_lbm_batch_synchronize.argtypes = [vp]
        L.mr_lbm_batch_counters.argtypes = [vp, C.POINTER(ll), C.POINTER(ll)]
        L.mr_lbm_batch_launch_count.argtypes = [vp]
        L.mr_lbm_batch_launch_count.restype = ll
        L.mr_lbm_batch_profile_enable.argtypes = [vp, i]
        L.mr_lbm_batch_profile_read.argtypes = [vp, C.POINTER(d), C.POINTER(ll)]
        L.mr_lbm_batch_destroy.argtypes = [vp]
        L.mr_lbm_batch_parts.argtypes = [vp, C.POINTER(i)]
        L.mr_lbm_batch_get_schedule.argtypes = [vp, i, C.POINTER(i)]
        L.mr_lbm_batch_set_schedule.argtypes = [vp, i, C.POINTER(i)]
        L.mr_lbm_batch_autotune.argtypes = [vp, i, C.POINTER(d), C.POINTER(d)]
        for name in ("mr_lbm_create", "mr_lbm_destroy", "mr_lbm_init", "mr_lbm_step", "mr_lbm_adapt",
                     "mr_lbm_project", "mr_lbm_project_noalloc", "mr_lbm_get_leaves", "mr_lbm_set_leaves", "mr_lbm_stats",
                     "mr_lbm_counters", "mr_lbm_profile_enable", "mr_lbm_profile_read",
                     "mr_lbm_synchronize", "mr_lbm_flattened_weights", "mr_lbm_flattened_weights_s", "mr_lbm_batch_create",
                     "mr_lbm_batch_instance", "mr_lbm_batch_step", "mr_lbm_batch_synchronize",
                     "mr_lbm_batch_counters", "mr_lbm_batch_profile_enable", "mr_lbm_batch_profile_read",
                     "mr_lbm_batch_destroy", "mr_lbm_batch_parts", "mr_lbm_batch_get_schedule",
                     "mr_lbm_batch_set_schedule", "mr_lbm_batch_autotune"):
            getattr(L, name).restype = i
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise MrError(status, where)


def make_config(cfg: Dict, leaf_capacity: int = 0) -> MrConfig:
    c = MrConfig()
    c.scheme = SCHEMES[cfg["scheme"]]
    c.lambda_ = float(cfg["lambda_"])
    for k, v in enumerate(cfg["s"]):
        c.s[k] = float(v)
    for k, v in enumerate(cfg["phys"]):
        c.phys[k] = float(v)
    for a in range(3):
        c.xmin[a] = float(cfg["xmin"][a])
        c.xmax[a] = float(cfg["xmax"][a])
        c.roots[a] = int(cfg["roots"][a])
    c.min_level = int(cfg["min_level"])
    c.max_level = int(cfg["max_level"])
    c.eps = float(cfg["eps"])
    c.mu_bar = int(cfg["mu_bar"])
    c.pred_s = int(cfg.get("pred_s", 1))
    for f in range(6):
        b = cfg["bc"][f]
        c.bc[f] = BCS[b] if isinstance(b, str) else int(b)
    c.cross_sign = int(cfg.get("cross_sign", 1))
    prec = cfg.get("precision", 0)
    c.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    c.leaf_capacity = int(cfg.get("leaf_capacity", leaf_capacity))
    c.obstacle = int(cfg.get("obstacle", 0))
    c.exact_collision = int(cfg.get("exact_collision", 0))
    return c


def _ptr(x):
    """(pointer, on_device) of a numpy array or a CUDA tensor."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    if not (isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]):
        raise ValueError("expected a C-contiguous numpy array or a tensor")
    return C.c_void_p(x.ctypes.data), 0


def flattened_weights(roots: int, level: int, max_level: int, periodic: bool, k: int) -> np.ndarray:
    out = np.zeros(10, np.float64)
    _check(library().mr_lbm_flattened_weights(roots, level, max_level, int(periodic), k,
                                              out.ctypes.data), "mr_lbm_flattened_weights")
    return out


def flattened_weights_s(s: int, half_width: int, roots: int, level: int, max_level: int, periodic: bool,
                        k: int) -> np.ndarray:
    """Weights of f_{k-w..k+w} for the velocities +1 (first 2w+1) and -1 (last 2w+1)."""
    out = np.zeros(4 * half_width + 2, np.float64)
    _check(library().mr_lbm_flattened_weights_s(s, half_width, roots, level, max_level, int(periodic), k,
                                                out.ctypes.data), "mr_lbm_flattened_weights_s")
    return out


class Solver:
    """One adaptive MR-LBM simulation on the current CUDA device."""

    def __init__(self, cfg: Dict, stream: Optional[int] = None, leaf_capacity: int = 0, _borrowed=None):
        self.cfg = dict(cfg)
        self._c = make_config(cfg, leaf_capacity)
        self._owned = _borrowed is None
        if _borrowed is None:
            h = C.c_void_p()
            _check(library().mr_lbm_create(C.byref(self._c), C.c_void_p(stream or 0), C.byref(h)),
                   "mr_lbm_create")
        else:
            h = _borrowed
        self.h = h
        sid = self._c.scheme
        self.d, self.Q, self.ncons = DIM[sid], NPOP[sid], NCONS[sid]
        self.J, self.Jmin = self._c.max_level, self._c.min_level

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                library().mr_lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_cells(self, level: int) -> int:
        n = 1
        for a in range(self.d):
            n *= self.cfg["roots"][a] << level
        return n

    def init(self, conserved):
        if isinstance(conserved, np.ndarray):
            conserved = np.ascontiguousarray(conserved, np.float64)
        p, dev = _ptr(conserved)
        _check(library().mr_lbm_init(self.h, p, dev), "mr_lbm_init")

    def step(self, n: int = 1):
        _check(library().mr_lbm_step(self.h, int(n)), "mr_lbm_step")

    def adapt(self):
        _check(library().mr_lbm_adapt(self.h), "mr_lbm_adapt")

    def project(self, level: int, out=None):
        if out is None:
            out = np.zeros((self.ncons, self.level_cells(level)), np.float64)
        p, dev = _ptr(out)
        _check(library().mr_lbm_project(self.h, int(level), p, dev), "mr_lbm_project")
        return out

    def project_noalloc(self, level: int, out=None):
        """mr_lbm_project without allocation (fixed 16 MiB device scratch)."""
        if out is None:
            out = np.zeros((self.ncons, self.level_cells(level)), np.float64)
        p, dev = _ptr(out)
        _check(library().mr_lbm_project_noalloc(self.h, int(level), p, dev), "mr_lbm_project_noalloc")
        return out

    def num_leaves(self) -> int:
        n = C.c_longlong(0)
        _check(library().mr_lbm_get_leaves(self.h, C.byref(n), None, None, None, 0), "mr_lbm_get_leaves")
        return n.value

    def get_leaves(self):
        """(keys uint64, levels int8, f float64 [Q, n]) sorted by (level, key)."""
        n = self.num_leaves()
        keys = np.zeros(n, np.uint64)
        lev = np.zeros(n, np.int8)
        f = np.zeros((self.Q, n), np.float64)
        nn = C.c_longlong(n)
        _check(library().mr_lbm_get_leaves(self.h, C.byref(nn), keys.ctypes.data, lev.ctypes.data,
                                           f.ctypes.data, 0), "mr_lbm_get_leaves")
        return keys, lev, f

    def get_leaves_into(self, keys, levels, f):
        nn = C.c_longlong(int(keys.shape[0]))
        pk, dev = _ptr(keys)
        pl, _ = _ptr(levels)
        pf, _ = _ptr(f)
        _check(library().mr_lbm_get_leaves(self.h, C.byref(nn), pk, pl, pf, dev), "mr_lbm_get_leaves")
        return nn.value

    def set_leaves(self, keys, levels, f):
        n = int(keys.shape[0])
        if isinstance(keys, np.ndarray):
            keys = np.ascontiguousarray(keys, np.uint64)
            levels = np.ascontiguousarray(levels, np.int8)
            f = np.ascontiguousarray(f, np.float64)
        pk, dev = _ptr(keys)
        pl, _ = _ptr(levels)
        pf, _ = _ptr(f)
        _check(library().mr_lbm_set_leaves(self.h, n, pk, pl, pf, dev), "mr_lbm_set_leaves")

    def stats(self):
        per = np.zeros(self.J + 1, np.int64)
        mesh_or, mem_or = C.c_double(), C.c_double()
        _check(library().mr_lbm_stats(self.h, per.ctypes.data, C.byref(mesh_or), C.byref(mem_or)),
               "mr_lbm_stats")
        return per, mesh_or.value, mem_or.value

    def counters(self):
        a, b = C.c_longlong(), C.c_longlong()
        _check(library().mr_lbm_counters(self.h, C.byref(a), C.byref(b)), "mr_lbm_counters")
        return a.value, b.value

    def launch_count(self) -> int:
        return int(library().mr_lbm_launch_count(self.h))

    def profile_enable(self, on: bool = True):
        _check(library().mr_lbm_profile_enable(self.h, int(on)), "mr_lbm_profile_enable")

    def profile_read(self):
        ms, n = C.c_double(), C.c_longlong()
        _check(library().mr_lbm_profile_read(self.h, C.byref(ms), C.byref(n)), "mr_lbm_profile_read")
        return ms.value, n.value

    def synchronize(self):
        _check(library().mr_lbm_synchronize(self.h), "mr_lbm_synchronize")

    def adjoint(self, conserved0, nsteps: int, checkpoint_every: int = 100, functional: str = "ke_sum",
                gradients: bool = True):
        """mr_lbm_adjoint: (J, dJ/d conserved0 [ncons, N_J], dJ/d s [16]).
        conserved0 is a numpy array (gradient returned as numpy) or a CUDA
        tensor (gradient returned as a CUDA tensor)."""
        kind = FUNCTIONALS[functional] if isinstance(functional, str) else int(functional)
        if isinstance(conserved0, np.ndarray):
            conserved0 = np.ascontiguousarray(conserved0, np.float64)
            grad = np.zeros_like(conserved0) if gradients else None
        else:
            import torch
            grad = torch.zeros_like(conserved0) if gradients else None
        gs = np.zeros(16, np.float64)
        J = C.c_double()
        p, dev = _ptr(conserved0)
        gp, _ = _ptr(grad)
        _check(library().mr_lbm_adjoint(self.h, p, dev, int(nsteps), int(checkpoint_every), kind, C.byref(J), gp,
                                        gs.ctypes.data if gradients else None), "mr_lbm_adjoint")
        return J.value, grad, (gs if gradients else None)


class Batch:
    """Many independent simulations stepped by shared launches
    (mr_lbm_batch_*); ``instances[i]`` is a borrowed Solver for input,
    output and statistics of configuration i."""

    def __init__(self, cfgs, stream: Optional[int] = None):
        n = len(cfgs)
        arr = (MrConfig * n)(*[make_config(c) for c in cfgs])
        b = C.c_void_p()
        _check(library().mr_lbm_batch_create(arr, n, C.c_void_p(stream or 0), C.byref(b)), "mr_lbm_batch_create")
        self.b = b
        self.instances = []
        for i, c in enumerate(cfgs):
            h = C.c_void_p()
            _check(library().mr_lbm_batch_instance(b, i, C.byref(h)), "mr_lbm_batch_instance")
            self.instances.append(Solver(c, _borrowed=h))

    def __len__(self):
        return len(self.instances)

    def step(self, n: int = 1):
        _check(library().mr_lbm_batch_step(self.b, int(n)), "mr_lbm_batch_step")

    def synchronize(self):
        _check(library().mr_lbm_batch_synchronize(self.b), "mr_lbm_batch_synchronize")

    def counters(self):
        a, c = C.c_longlong(), C.c_longlong()
        _check(library().mr_lbm_batch_counters(self.b, C.byref(a), C.byref(c)), "mr_lbm_batch_counters")
        return a.value, c.value

    def launch_count(self) -> int:
        return int(library().mr_lbm_batch_launch_count(self.b))

    def profile_enable(self, on=True):
        _check(library().mr_lbm_batch_profile_enable(self.b, int(on)), "mr_lbm_batch_profile_enable")

    def profile_read(self):
        ms, n = C.c_double(), C.c_longlong()
        _check(library().mr_lbm_batch_profile_read(self.b, C.byref(ms), C.byref(n)), "mr_lbm_batch_profile_read")
        return ms.value, n.value

    NPHASE = 7

    def parts(self) -> int:
        n = C.c_int()
        _check(library().mr_lbm_batch_parts(self.b, C.byref(n)), "mr_lbm_batch_parts")
        return n.value

    def schedule(self):
        """[parts][7] blocks per SM of each phase (mr_lbm_batch_get_schedule)."""
        out = []
        for p in range(self.parts()):
            v = (C.c_int * self.NPHASE)()
            _check(library().mr_lbm_batch_get_schedule(self.b, p, v), "mr_lbm_batch_get_schedule")
            out.append(list(v))
        return out

    def set_schedule(self, part: int, bps):
        v = (C.c_int * self.NPHASE)(*[int(x) for x in bps])
        _check(library().mr_lbm_batch_set_schedule(self.b, part, v), "mr_lbm_batch_set_schedule")

    def autotune(self, trial_steps: int = 4):
        """mr_lbm_batch_autotune: (ms per step before, after)."""
        a, b = C.c_double(), C.c_double()
        _check(library().mr_lbm_batch_autotune(self.b, int(trial_steps), C.byref(a), C.byref(b)),
               "mr_lbm_batch_autotune")
        return a.value, b.value

    def close(self):
        if getattr(self, "b", None):
            for s in self.instances:
                s.h = None
            library().mr_lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- keys
def _spread(v, d):
    v = np.asarray(v, np.uint64)
    out = np.zeros_like(v)
    for b in range(32):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(d * b)
    return out


def _compact(v, d):
    v = np.asarray(v, np.uint64)
    out = np.zeros_like(v)
    for b in range(32):
        out |= ((v >> np.uint64(d * b)) & np.uint64(1)) << np.uint64(b)
    return out


def encode_keys(cfg: Dict, level, ix, iy=None) -> np.ndarray:
    """Keys of the C-ABI (Morton code at the cell's own level with a root prefix)."""
    d = DIM[SCHEMES[cfg["scheme"]]]
    level = np.asarray(level, np.uint64)
    ix = np.asarray(ix, np.uint64)
    if d == 1:
        return ix.astype(np.uint64)
    iy = np.asarray(iy, np.uint64)
    mask = (np.uint64(1) << level) - np.uint64(1)
    root = (ix >> level) + np.uint64(cfg["roots"][0]) * (iy >> level)
    local = _spread(ix & mask, 2) | (_spread(iy & mask, 2) << np.uint64(1))
    return (root << (np.uint64(2) * level)) | local


def encode_keys3(cfg: Dict, level, ix, iy, iz) -> np.ndarray:
    """Keys of a d = 3 scheme: (root << 3l) | 3-way interleave of (x, y, z)
    at the cell's level, root = x >> l + roots_x (y >> l + roots_y (z >> l))."""
    level = np.asarray(level, np.uint64)
    ix, iy, iz = (np.asarray(v, np.uint64) for v in (ix, iy, iz))
    mask = (np.uint64(1) << level) - np.uint64(1)
    root = (ix >> level) + np.uint64(cfg["roots"][0]) * ((iy >> level) + np.uint64(cfg["roots"][1]) * (iz >> level))
    local = _spread(ix & mask, 3) | (_spread(iy & mask, 3) << np.uint64(1)) | (_spread(iz & mask, 3) << np.uint64(2))
    return (root << (np.uint64(3) * level)) | local


def decode_keys3(cfg: Dict, level, keys):
    """(x, y, z) of the keys of a d = 3 scheme."""
    keys = np.asarray(keys, np.uint64)
    level = np.asarray(level, np.uint64)
    root = keys >> (np.uint64(3) * level)
    local = keys & ((np.uint64(1) << (np.uint64(3) * level)) - np.uint64(1))
    rxy = np.uint64(cfg["roots"][0] * cfg["roots"][1])
    rz, rr = root // rxy, root % rxy
    rx, ry = rr % np.uint64(cfg["roots"][0]), rr // np.uint64(cfg["roots"][0])
    x = (rx << level) | _compact(local, 3)
    y = (ry << level) | _compact(local >> np.uint64(1), 3)
    z = (rz << level) | _compact(local >> np.uint64(2), 3)
    return x.astype(np.int64), y.astype(np.int64), z.astype(np.int64)


def decode_keys(cfg: Dict, level, keys):
    """(x, y) of the keys of a d <= 2 scheme (y = 0 in 1D); (x, y, z) for d = 3."""
    d = DIM[SCHEMES[cfg["scheme"]]]
    keys = np.asarray(keys, np.uint64)
    level = np.asarray(level, np.uint64)
    if d == 3:
        return decode_keys3(cfg, level, keys)
    if d == 1:
        return keys.astype(np.int64), np.zeros(keys.shape, np.int64)
    root = keys >> (np.uint64(2) * level)
    local = keys & ((np.uint64(1) << (np.uint64(2) * level)) - np.uint64(1))
    rx = root % np.uint64(cfg["roots"][0])
    ry = root // np.uint64(cfg["roots"][0])
    x = (rx << level) | _compact(local, 2)
    y = (ry << level) | _compact(local >> np.uint64(1), 2)
    return x.astype(np.int64), y.astype(np.int64)
