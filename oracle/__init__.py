"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded restatement of the paper's scheme and
pre-computation (Cacace & Falcone, Sections 3-4), used to check the CUDA
solver.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the solver package never does, and the two
share no code (inputs come from ``hjb_inputs``).

Every function states the passage it follows.  All pins are in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Tuple

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        L.orc_node_update.restype = ctypes.c_double
        L.orc_node_update.argtypes = [P(_Problem), P(ctypes.c_double), ctypes.c_int64,
                                      ctypes.c_int, P(ctypes.c_int32)]
        L.orc_node_candidates.restype = None
        L.orc_node_candidates.argtypes = [P(_Problem), P(ctypes.c_double), ctypes.c_int64,
                                          ctypes.c_int, P(ctypes.c_double)]
        L.orc_fix_nonfree.restype = None
        L.orc_fix_nonfree.argtypes = [P(_Problem), P(ctypes.c_double)]
        L.orc_apply.restype = ctypes.c_double
        L.orc_apply.argtypes = [P(_Problem), P(ctypes.c_double), P(ctypes.c_double),
                                P(ctypes.c_int32), ctypes.c_int]
        L.orc_residual.restype = ctypes.c_double
        L.orc_residual.argtypes = [P(_Problem), P(ctypes.c_double)]
        L.orc_sweep_gs.restype = ctypes.c_double
        L.orc_sweep_gs.argtypes = [P(_Problem), P(ctypes.c_double), ctypes.c_int,
                                   P(ctypes.c_int64), ctypes.c_int64]
        L.orc_solve.restype = ctypes.c_int32
        L.orc_solve.argtypes = [P(_Problem), P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                P(ctypes.c_int64), ctypes.c_int64, ctypes.c_double,
                                ctypes.c_int32, P(ctypes.c_double)]
        L.orc_coarse_data.restype = ctypes.c_int32
        L.orc_coarse_data.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_float),
                                      P(ctypes.c_uint8), P(ctypes.c_float), P(ctypes.c_uint8)]
        L.orc_interp_coarse.restype = None
        L.orc_interp_coarse.argtypes = [ctypes.c_int32, P(ctypes.c_double), ctypes.c_int32,
                                        P(ctypes.c_uint8), ctypes.c_double, P(ctypes.c_double)]
        L.orc_synthesis.restype = None
        L.orc_synthesis.argtypes = [P(_Problem), P(ctypes.c_double), P(ctypes.c_uint8)]
        L.orc_synthesis_values.restype = None
        L.orc_synthesis_values.argtypes = [P(_Problem), P(ctypes.c_double), P(ctypes.c_int64),
                                           ctypes.c_int64, P(ctypes.c_double)]
        L.orc_successors.restype = None
        L.orc_successors.argtypes = [P(_Problem), P(ctypes.c_uint8), P(ctypes.c_int32)]
        L.orc_labels.restype = ctypes.c_int32
        L.orc_labels.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_uint8),
                                 P(ctypes.c_int8), ctypes.c_int32, P(ctypes.c_int8)]
        L.orc_band_keys.restype = None
        L.orc_band_keys.argtypes = [ctypes.c_int64, P(ctypes.c_double), P(ctypes.c_uint8),
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                    P(ctypes.c_int32)]
        _LIB = L
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_controls", ctypes.c_int32),
                ("h", ctypes.c_double), ("lam", ctypes.c_double),
                ("sigma", ctypes.c_double), ("cost", ctypes.c_double),
                ("u_obstacle", ctypes.c_double),
                ("speed", ctypes.POINTER(ctypes.c_float)),
                ("drift", ctypes.POINTER(ctypes.c_float)),
                ("mask", ctypes.POINTER(ctypes.c_uint8)),
                ("controls", ctypes.POINTER(ctypes.c_double)),
                ("sigma_field", ctypes.POINTER(ctypes.c_float)),
                ("diffusion", ctypes.c_int32),
                ("cost_field", ctypes.POINTER(ctypes.c_float)),
                ("control_cost", ctypes.POINTER(ctypes.c_double))]


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class Problem:
    """Discrete problem on G: the data of Section 3 (f = b + c a, l, sigma, g = 0 on
    the target) plus the time step h and the discount lambda (beta = 1/(1+lambda h)).

    General terms of Section 5.3: ``sigma_field`` (sigma(x) per node, replacing
    the constant sigma), ``diffusion`` (0: sigma(x) I_2; 1: sigma(x) a, a
    one-dimensional Wiener process along the control), ``cost_field`` (l(x) per
    node, replacing the constant cost) and ``control_cost`` (m(a_m) per control);
    the running cost is l(x) + m(a)."""

    def __init__(self, n: int, controls: np.ndarray, speed: np.ndarray, mask: np.ndarray,
                 h: float = 0.0, lam: float = 1.0, sigma: float = 0.0, cost: float = 1.0,
                 drift: Optional[np.ndarray] = None, u_obstacle: Optional[float] = None,
                 sigma_field: Optional[np.ndarray] = None, diffusion: int = 0,
                 cost_field: Optional[np.ndarray] = None,
                 control_cost: Optional[np.ndarray] = None):
        self.n = int(n)
        self.dx = 2.0 / (n - 1)
        self.h = float(h) if h > 0 else self.dx
        self.lam = float(lam)
        self.sigma = float(sigma)
        self.cost = float(cost)
        self.beta = 1.0 / (1.0 + self.lam * self.h)
        self.controls = np.ascontiguousarray(controls, dtype=np.float64).reshape(-1, 2)
        self.speed = np.ascontiguousarray(speed, dtype=np.float32).reshape(-1)
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self.drift = None if drift is None else np.ascontiguousarray(drift, dtype=np.float32).reshape(-1)
        self.sigma_field = (None if sigma_field is None
                            else np.ascontiguousarray(sigma_field, dtype=np.float32).reshape(-1))
        self.diffusion = int(diffusion)
        self.cost_field = (None if cost_field is None
                           else np.ascontiguousarray(cost_field, dtype=np.float32).reshape(-1))
        self.control_cost = (None if control_cost is None
                             else np.ascontiguousarray(control_cost, dtype=np.float64).reshape(-1))
        if u_obstacle is None:
            u_obstacle = self.u_max if self.lam > 0 else 1e6
        self.u_obstacle = float(u_obstacle)
        assert self.speed.size == n * n and self.mask.size == n * n
        assert self.diffusion in (0, 1)
        assert self.sigma_field is None or self.sigma_field.size == n * n
        assert self.cost_field is None or self.cost_field.size == n * n
        assert self.control_cost is None or self.control_cost.size == self.controls.shape[0]
        fp = ctypes.POINTER(ctypes.c_float)
        self._s = _Problem(self.n, self.controls.shape[0], self.h, self.lam, self.sigma,
                           self.cost, self.u_obstacle, _ptr(self.speed, ctypes.c_float),
                           _ptr(self.drift, ctypes.c_float) if self.drift is not None else fp(),
                           _ptr(self.mask, ctypes.c_uint8), _ptr(self.controls, ctypes.c_double),
                           _ptr(self.sigma_field, ctypes.c_float) if self.sigma_field is not None
                           else fp(), self.diffusion,
                           _ptr(self.cost_field, ctypes.c_float) if self.cost_field is not None
                           else fp(),
                           _ptr(self.control_cost, ctypes.c_double) if self.control_cost is not None
                           else ctypes.POINTER(ctypes.c_double)())

    @classmethod
    def from_instance(cls, inst, **kw) -> "Problem":
        args = dict(h=inst.h, lam=inst.lam, sigma=inst.sigma, cost=inst.cost, drift=inst.drift,
                    sigma_field=getattr(inst, "sigma_field", None),
                    diffusion=getattr(inst, "diffusion", 0),
                    cost_field=getattr(inst, "cost_field", None),
                    control_cost=getattr(inst, "control_cost", None))
        args.update(kw)
        return cls(inst.n, inst.controls, inst.speed, inst.mask, **args)

    @property
    def N(self) -> int:
        return self.n * self.n

    @property
    def l_max(self) -> float:
        """The largest running cost max_x l(x) + max_a m(a)."""
        lx = float(self.cost_field.max()) if self.cost_field is not None else self.cost
        la = float(self.control_cost.max()) if self.control_cost is not None else 0.0
        return lx + la

    @property
    def u_max(self) -> float:
        """h l / (1 - beta) = l (1/lambda + h) with the largest l: a bound on the
        value of never reaching the target."""
        return self.h * self.l_max / (1.0 - self.beta)

    # ------------------------------------------------------------- scheme
    def node_update(self, u: np.ndarray, k: int, scheme: int = 3) -> Tuple[float, int]:
        """u_i <- min_a {...} at one free node (eq. SLscheme2 / SLscheme3)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        am = ctypes.c_int32()
        v = lib().orc_node_update(ctypes.byref(self._s), _ptr(u, ctypes.c_double), int(k),
                                  scheme, ctypes.byref(am))
        return v, am.value

    def node_candidates(self, u: np.ndarray, nodes: np.ndarray, scheme: int = 3) -> np.ndarray:
        """Every control's candidate value at the listed free nodes: (len(nodes), N_A)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty((len(nodes), self.controls.shape[0]))
        row = np.empty(self.controls.shape[0])
        for t, k in enumerate(nodes):
            lib().orc_node_candidates(ctypes.byref(self._s), _ptr(u, ctypes.c_double), int(k),
                                      scheme, _ptr(row, ctypes.c_double))
            out[t] = row
        return out

    def fix_nonfree(self, u: np.ndarray) -> np.ndarray:
        u = np.array(u, dtype=np.float64, copy=True)
        lib().orc_fix_nonfree(ctypes.byref(self._s), _ptr(u, ctypes.c_double))
        return u

    def apply(self, u: np.ndarray, scheme: int = 3) -> Tuple[np.ndarray, np.ndarray, float]:
        """One Jacobi application T u on every free node; returns (T u, argmin, sup |Tu-u|)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        am = np.empty(self.N, dtype=np.int32)
        inc = lib().orc_apply(ctypes.byref(self._s), _ptr(u, ctypes.c_double),
                              _ptr(out, ctypes.c_double), _ptr(am, ctypes.c_int32), scheme)
        return out, am, inc

    def residual(self, u: np.ndarray) -> float:
        """|| T2 u - u ||_inf over free nodes (eq. SLscheme2, the plain fixed point)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        return lib().orc_residual(ctypes.byref(self._s), _ptr(u, ctypes.c_double))

    def sweep_gs(self, u: np.ndarray, scheme: int = 3, order: Optional[np.ndarray] = None) -> float:
        """One in-place Gauss-Seidel sweep (row-major unless an order is given)."""
        assert u.dtype == np.float64 and u.flags.c_contiguous
        if order is not None:
            order = np.ascontiguousarray(order, dtype=np.int64)
        return lib().orc_sweep_gs(ctypes.byref(self._s), _ptr(u, ctypes.c_double), scheme,
                                  _ptr(order, ctypes.c_int64) if order is not None
                                  else ctypes.POINTER(ctypes.c_int64)(),
                                  0 if order is None else order.size)

    def solve(self, u0: Optional[np.ndarray] = None, scheme: int = 3, method: str = "gs",
              order: Optional[np.ndarray] = None, tol: float = 1e-13,
              max_sweeps: int = 100000) -> Tuple[np.ndarray, int, float]:
        """Value iteration to a sup-increment <= tol.  Returns (u, sweeps, last increment);
        sweeps = -1 if max_sweeps was hit."""
        u = np.zeros(self.N) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
        if order is not None:
            order = np.ascontiguousarray(order, dtype=np.int64)
        last = ctypes.c_double()
        s = lib().orc_solve(ctypes.byref(self._s), _ptr(u, ctypes.c_double), scheme,
                            0 if method == "gs" else 1,
                            _ptr(order, ctypes.c_int64) if order is not None
                            else ctypes.POINTER(ctypes.c_int64)(),
                            0 if order is None else order.size, tol, max_sweeps,
                            ctypes.byref(last))
        return u, s, last.value

    # ----------------------------------------------------- pre-computation
    def synthesis(self, uhat: np.ndarray) -> np.ndarray:
        """a*(x_i) = argmin_a {beta u_hat(x_i + h f) + h l} (eq. discrete-synthesis)."""
        uhat = np.ascontiguousarray(uhat, dtype=np.float64)
        a = np.empty(self.N, dtype=np.uint8)
        lib().orc_synthesis(ctypes.byref(self._s), _ptr(uhat, ctypes.c_double), _ptr(a, ctypes.c_uint8))
        return a

    def synthesis_values(self, uhat: np.ndarray, nodes: np.ndarray) -> np.ndarray:
        uhat = np.ascontiguousarray(uhat, dtype=np.float64)
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        vals = np.empty((nodes.size, self.controls.shape[0]))
        lib().orc_synthesis_values(ctypes.byref(self._s), _ptr(uhat, ctypes.c_double),
                                   _ptr(nodes, ctypes.c_int64), nodes.size,
                                   _ptr(vals, ctypes.c_double))
        return vals

    def successors(self, a: np.ndarray) -> np.ndarray:
        """Winner-take-all transport step of eq. discrete-advection (see oracle.c)."""
        a = np.ascontiguousarray(a, dtype=np.uint8)
        succ = np.empty(self.N, dtype=np.int32)
        lib().orc_successors(ctypes.byref(self._s), _ptr(a, ctypes.c_uint8), _ptr(succ, ctypes.c_int32))
        return succ

    def labels(self, succ: np.ndarray, sector: np.ndarray, n_patches: int) -> np.ndarray:
        succ = np.ascontiguousarray(succ, dtype=np.int32)
        sector = np.ascontiguousarray(sector, dtype=np.int8)
        lab = np.empty(self.N, dtype=np.int8)
        rc = lib().orc_labels(self.n, _ptr(succ, ctypes.c_int32), _ptr(self.mask, ctypes.c_uint8),
                              _ptr(sector, ctypes.c_int8), n_patches, _ptr(lab, ctypes.c_int8))
        assert rc == 0
        return lab


# --------------------------------------------------------------- coarse grid

def coarse_data(n: int, nc: int, speed: np.ndarray, mask: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Speed and mask on the nested coarse grid G_c (Section 2)."""
    speed = np.ascontiguousarray(speed, dtype=np.float32)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    sc = np.empty(nc * nc, dtype=np.float32)
    mc = np.empty(nc * nc, dtype=np.uint8)
    rc = lib().orc_coarse_data(n, nc, _ptr(speed, ctypes.c_float), _ptr(mask, ctypes.c_uint8),
                               _ptr(sc, ctypes.c_float), _ptr(mc, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("coarse grid does not nest in the fine grid")
    return sc, mc


def interp_coarse(nc: int, uc: np.ndarray, n: int, mask: np.ndarray, u_obstacle: float) -> np.ndarray:
    """u_hat = Q1 interpolation of u_c on G (Section 4.3, pre-computation)."""
    uc = np.ascontiguousarray(uc, dtype=np.float64)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.empty(n * n)
    lib().orc_interp_coarse(nc, _ptr(uc, ctypes.c_double), n, _ptr(mask, ctypes.c_uint8),
                            u_obstacle, _ptr(out, ctypes.c_double))
    return out


def band_keys(uhat: np.ndarray, mask: np.ndarray, lam: float, width: float, n_bands: int) -> np.ndarray:
    """Causal band index of each free node, by increasing u_hat (Section 4.2)."""
    uhat = np.ascontiguousarray(uhat, dtype=np.float64)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    keys = np.empty(uhat.size, dtype=np.int32)
    lib().orc_band_keys(uhat.size, _ptr(uhat, ctypes.c_double), _ptr(mask, ctypes.c_uint8),
                        lam, width, n_bands, _ptr(keys, ctypes.c_int32))
    return keys


# ------------------------------------------------------- whole pre-computation

def patchy_precompute(inst, tol_c: float = 1e-10, band_factor: float = 1.0,
                      n_bands: int = 1 << 20):
    """The pre-computation list of Section 4.3 on an instance with a coarse grid:
    coarse solve (sigma = 0, from the big initial value), u_hat, a*, successors,
    labels and band keys.  Returns a dict of arrays."""
    n, nc = inst.n, inst.coarse_n
    fine = Problem.from_instance(inst)
    sc, mc = coarse_data(n, nc, inst.speed, inst.mask)
    hc = 2.0 / (nc - 1) if inst.h <= 0 else inst.h * (n - 1) / (nc - 1)
    # the other per-node data on G_c are the fine data at the nested nodes
    r = (n - 1) // (nc - 1)

    def nested(a, comps=1):
        return None if a is None else np.ascontiguousarray(
            np.asarray(a).reshape(n, n, comps)[::r, ::r]).reshape(-1)

    coarse = Problem(nc, inst.controls, sc, mc, h=hc, lam=inst.lam, sigma=0.0,
                     cost=inst.cost, u_obstacle=fine.u_obstacle, drift=nested(inst.drift, 2),
                     cost_field=nested(getattr(inst, "cost_field", None)),
                     control_cost=getattr(inst, "control_cost", None))
    u0 = np.full(nc * nc, coarse.u_max if inst.lam > 0 else 1e6)
    uc, sweeps, _ = coarse.solve(u0, scheme=3, method="gs", tol=tol_c)
    uhat = interp_coarse(nc, uc, n, inst.mask, fine.u_obstacle)
    a = fine.synthesis(uhat)
    succ = fine.successors(a)
    lab = fine.labels(succ, inst.sector, inst.n_patches)
    keys = band_keys(uhat, inst.mask, inst.lam, band_factor * fine.h, n_bands)
    return dict(uc=uc, coarse_sweeps=sweeps, uhat=uhat, a=a, succ=succ, labels=lab, keys=keys,
                coarse=coarse, fine=fine)
