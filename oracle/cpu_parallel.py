"""ctypes binding of the all-core FP64 CPU baseline (``cpu_parallel.c``).

Benchmark infrastructure only (the CPU context of the GPU timings): Jacobi and
u_hat-ordered Gauss-Seidel sweeps of eq. SLscheme3 on every host core.  Shares
no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import build as _build

_LIB = None


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_controls", ctypes.c_int32),
                ("h", ctypes.c_double), ("lam", ctypes.c_double), ("sigma", ctypes.c_double),
                ("cost", ctypes.c_double), ("u_obstacle", ctypes.c_double),
                ("speed", ctypes.c_void_p), ("drift", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("controls", ctypes.c_void_p)]


def lib():
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(_build.build_parallel())
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_int64)
        L.cpb_threads.restype = ctypes.c_int
        L.cpb_fix.argtypes = [P, dp]
        L.cpb_jacobi.restype = ctypes.c_double
        L.cpb_jacobi.argtypes = [P, dp, dp]
        L.cpb_gs.restype = ctypes.c_double
        L.cpb_gs.argtypes = [P, dp, lp, lp, ctypes.c_int32]
        _LIB = L
    return _LIB


def threads() -> int:
    return int(lib().cpb_threads())


class AllCore:
    """The instance's discrete problem (constant sigma and cost, optional drift)."""

    def __init__(self, inst):
        self.n = int(inst.n)
        self.N = self.n * self.n
        dx = 2.0 / (self.n - 1)
        h = inst.h if inst.h > 0 else dx
        beta = 1.0 / (1.0 + inst.lam * h)
        self.h, self.beta = h, beta
        self._speed = np.ascontiguousarray(inst.speed, np.float32)
        self._mask = np.ascontiguousarray(inst.mask, np.uint8)
        self._drift = None if inst.drift is None else np.ascontiguousarray(inst.drift, np.float32)
        self._ctrl = np.ascontiguousarray(inst.controls, np.float64)
        uob = h * inst.cost / (1.0 - beta) if inst.lam > 0 else 1e6
        vp = lambda a: None if a is None else a.ctypes.data
        self._p = _Problem(self.n, self._ctrl.shape[0], h, inst.lam, inst.sigma, inst.cost, uob,
                           vp(self._speed), vp(self._drift), vp(self._mask), vp(self._ctrl))

    def fix(self, u: np.ndarray) -> np.ndarray:
        u = np.array(u, dtype=np.float64, copy=True)
        lib().cpb_fix(ctypes.byref(self._p), u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return u

    def jacobi(self, u: np.ndarray, out: np.ndarray) -> float:
        dp = ctypes.POINTER(ctypes.c_double)
        return lib().cpb_jacobi(ctypes.byref(self._p), u.ctypes.data_as(dp), out.ctypes.data_as(dp))

    def gs_lists(self, uhat: np.ndarray, lists: Optional[int] = None):
        """One node list per block of rows, each sorted by u_hat (free nodes only)."""
        lists = lists or 4 * threads()
        free = np.flatnonzero(self._mask == 0)
        rows = free // self.n
        block = np.minimum(rows * lists // self.n, lists - 1)
        order = np.lexsort((uhat[free], block))
        nodes = np.ascontiguousarray(free[order], np.int64)
        off = np.zeros(lists + 1, np.int64)
        np.cumsum(np.bincount(block, minlength=lists), out=off[1:])
        return nodes, off

    def gs(self, u: np.ndarray, nodes: np.ndarray, off: np.ndarray) -> float:
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_int64)
        return lib().cpb_gs(ctypes.byref(self._p), u.ctypes.data_as(dp), nodes.ctypes.data_as(lp),
                            off.ctypes.data_as(lp), off.size - 1)
