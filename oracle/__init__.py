"""ctypes binding of the plain C oracle.

TEST INFRASTRUCTURE ONLY.  The oracle is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``;
the product path (``paper_2103_02903_gb300``) never imports it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

_lib = None


class OrConfig(C.Structure):
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
        ("bc", C.c_int * 6),
        ("cross_sign", C.c_int),
        ("obstacle", C.c_int),
        ("exact_collision", C.c_int),
        ("pred_s", C.c_int),
    ]


SCHEMES = {"d1q2_advection": 0, "d1q2_burgers": 1, "d1q3_shallow_water": 2,
           "d2q4x4_euler": 3, "d2q9_ns": 4, "d3q6_advection": 5}
BCS = {"periodic": 0, "copy": 1, "bounce_back": 2, "anti_bounce_back": 3,
       "bounce_back_velocity": 4}


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        vp = C.c_void_p
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        L.or_create.restype = vp
        L.or_create.argtypes = [C.POINTER(OrConfig)]
        L.or_destroy.argtypes = [vp]
        L.or_scheme_info.argtypes = [vp] + [C.POINTER(C.c_int)] * 5
        L.or_init.argtypes = [vp, dp]
        L.or_step.argtypes = [vp, C.c_int]
        L.or_adapt.argtypes = [vp]
        L.or_stream_collide.argtypes = [vp, C.c_int]
        L.or_num_leaves.restype = C.c_longlong
        L.or_num_leaves.argtypes = [vp]
        L.or_get_leaves.argtypes = [vp, ip, ip, ip, ip, dp]
        L.or_set_leaves.argtypes = [vp, C.c_longlong, ip, ip, ip, ip, dp]
        L.or_project.argtypes = [vp, C.c_int, dp]
        L.or_reconstruct.argtypes = [vp, C.c_int, dp]
        L.or_last_margin.restype = C.c_double
        L.or_last_margin.argtypes = [vp]
        L.or_group_norms.argtypes = [vp, C.c_int, dp]
        L.or_prediction_coefficient.restype = C.c_double
        L.or_predict_children.argtypes = [C.c_int, C.c_int, dp, dp]
        L.or_predict_children_s.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
        L.or_prediction_coefficients.argtypes = [C.c_int, dp]
        L.or_check_graded.argtypes = [vp]
        _lib = L
    return _lib


def make_config(cfg: dict) -> OrConfig:
    c = OrConfig()
    c.scheme = SCHEMES[cfg["scheme"]]
    c.lambda_ = float(cfg["lambda_"])
    for i, v in enumerate(cfg["s"]):
        c.s[i] = float(v)
    for i, v in enumerate(cfg["phys"]):
        c.phys[i] = float(v)
    for i in range(3):
        c.xmin[i] = float(cfg["xmin"][i])
        c.xmax[i] = float(cfg["xmax"][i])
        c.roots[i] = int(cfg["roots"][i])
    c.min_level = int(cfg["min_level"])
    c.max_level = int(cfg["max_level"])
    c.eps = float(cfg["eps"])
    c.mu_bar = int(cfg["mu_bar"])
    for i in range(6):
        b = cfg["bc"][i]
        c.bc[i] = BCS[b] if isinstance(b, str) else int(b)
    c.cross_sign = int(cfg.get("cross_sign", 1))
    c.obstacle = int(cfg.get("obstacle", 0))
    c.exact_collision = int(cfg.get("exact_collision", 0))
    c.pred_s = int(cfg.get("pred_s", 1))
    return c


class Oracle:
    """Dense FP64 reference of the adaptive step (test infrastructure)."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.h = lib().or_create(C.byref(self._c))
        if not self.h:
            raise RuntimeError("oracle: invalid configuration")
        v = [C.c_int() for _ in range(5)]
        lib().or_scheme_info(self.h, *[C.byref(x) for x in v])
        self.d, self.q, self.m, self.Q, self.ncons = [x.value for x in v]
        self.J = self._c.max_level
        self.Jmin = self._c.min_level

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def level_shape(self, level):
        return tuple(self.cfg["roots"][a] << level for a in range(self.d))

    def init(self, conserved):
        lib().or_init(self.h, np.ascontiguousarray(conserved, dtype=np.float64).ravel())

    def step(self, n=1):
        if lib().or_step(self.h, n) != 0:
            raise RuntimeError("oracle step failed")

    def adapt(self):
        if lib().or_adapt(self.h) != 0:
            raise RuntimeError("oracle adapt failed")

    def stream_collide(self, collide=True):
        if lib().or_stream_collide(self.h, 1 if collide else 0) != 0:
            raise RuntimeError("oracle stream failed")

    def num_leaves(self):
        return int(lib().or_num_leaves(self.h))

    def leaves(self):
        """Return (level, ix, iy, iz, f[Q, n]) sorted by (level, z, y, x)."""
        n = self.num_leaves()
        lev = np.zeros(n, np.int32)
        ix = np.zeros(n, np.int32)
        iy = np.zeros(n, np.int32)
        iz = np.zeros(n, np.int32)
        f = np.zeros((self.Q, n), np.float64)
        lib().or_get_leaves(self.h, lev, ix, iy, iz, f)
        return lev, ix, iy, iz, f

    def set_leaves(self, level, ix, iy, iz, f):
        n = len(level)
        rc = lib().or_set_leaves(self.h, n, np.ascontiguousarray(level, np.int32),
                                 np.ascontiguousarray(ix, np.int32),
                                 np.ascontiguousarray(iy, np.int32),
                                 np.ascontiguousarray(iz, np.int32),
                                 np.ascontiguousarray(f, np.float64))
        if rc != 0:
            raise ValueError("oracle: leaves do not partition the domain (%d)" % rc)

    def project(self, level):
        shape = self.level_shape(level)
        out = np.zeros(self.ncons * int(np.prod(shape)), np.float64)
        lib().or_project(self.h, level, out)
        return out.reshape(self.ncons, -1)

    def reconstruct(self, level):
        shape = self.level_shape(level)
        out = np.zeros(self.Q * int(np.prod(shape)), np.float64)
        lib().or_reconstruct(self.h, level, out)
        return out.reshape(self.Q, -1)

    def margin(self):
        return float(lib().or_last_margin(self.h))

    def group_norms(self, level):
        out = np.zeros(int(np.prod(self.level_shape(level))), np.float64)
        if lib().or_group_norms(self.h, level, out) != 0:
            raise ValueError("no group norms at this level")
        return out

    def graded(self):
        return bool(lib().or_check_graded(self.h) == 1)


def prediction_coefficient():
    return float(lib().or_prediction_coefficient())


def predict_children(d, stencil, cross_sign=1):
    out = np.zeros(1 << d, np.float64)
    lib().or_predict_children(d, cross_sign, np.ascontiguousarray(stencil, np.float64).ravel(), out)
    return out


def prediction_coefficients(s):
    out = np.zeros(s, np.float64)
    if lib().or_prediction_coefficients(s, out) != 0:
        raise ValueError("s must be 1, 2 or 3")
    return out


def predict_children_s(d, stencil, cross_sign=1, s=1):
    """Children of a (2s+1)^d stencil (x fastest) under the prediction of half-width s."""
    out = np.zeros(1 << d, np.float64)
    st = np.ascontiguousarray(stencil, np.float64).ravel()
    assert st.size == (2 * s + 1) ** d
    if lib().or_predict_children_s(d, cross_sign, s, st, out) != 0:
        raise ValueError("bad d or s")
    return out
