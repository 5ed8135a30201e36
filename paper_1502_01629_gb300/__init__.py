"""GB300 (sm_103a) solver for the Markov-chain semi-Lagrangian value iteration of
the 2-D second-order HJB equation inside the patchy domain decomposition
(Cacace & Falcone, "A dynamic domain decomposition for a class of second order
semi-linear equations").

The compute path is the CUDA library behind the C ABI of ``include/hjb.h``;
this package is its thin binding.  Names follow the C entry points:

    p = Problem(desc_fields..., speed, mask, sector, controls)
    p.coarse_solve(); p.build_patches(); stats = p.solve_patches(tol32, tol64)
    u = p.get_value()

PyTorch, when used, only supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from ._lib import (HJB_ERR_NOT_CONVERGED, HJB_OK, BatchDesc, BatchInst, Desc, HJBError, RegimeInfo, Terms,
                   Stats, check, header_functions, lib)

__all__ = ["Problem", "Batch", "Net", "HJBError", "regime", "kernel_launches", "lib", "header_functions", "trim_memory",
           "HJB_ERR_NOT_CONVERGED"]


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def kernel_launches() -> int:
    """Kernels the library has launched since it was loaded."""
    return int(lib().hjb_kernel_launches())


def regime(dx: float, f_min: float, f_max: float, eps: float) -> dict:
    """Upwind diffusion-ball regime (Section 4.1): Upsilon, omega, alpha bounds,
    tau_dx, the threshold on eps and whether the condition holds.  Host only."""
    out = RegimeInfo()
    check(lib().hjb_regime(dx, f_min, f_max, eps, ctypes.byref(out)), "hjb_regime")
    return {f: getattr(out, f) for f, _ in out._fields_}


def trim_memory() -> None:
    """Return the device memory the library's pool keeps cached from destroyed
    problems and batches (``hjb_trim_memory``)."""
    check(lib().hjb_trim_memory(), "hjb_trim_memory")


class Problem:
    """One problem instance on the GPU (wraps an ``hjb_problem*``).

    The data follow ``hjb_inputs.Instance``: n nodes per side on [-1, 1]^2, the
    control set, speed c(x), mask (0 free, 1 target, 2 obstacle), the boundary
    sectors, and the discretisation knobs (h, lam, sigma, cost, coarse grid, patch
    schedule).  ``sigma_field``, ``diffusion``, ``cost_field`` and ``control_cost``
    select the general terms of Section 5.3 (``hjb_create_problem_general``);
    ``device_inputs=True`` takes torch CUDA tensors (or raw device pointers) for
    the per-node arrays (``hjb_create_problem_device``)."""

    def __init__(self, n: int, controls: np.ndarray, speed: np.ndarray, mask: np.ndarray,
                 sector: Optional[np.ndarray] = None, *, h: float = 0.0, lam: float = 1.0,
                 sigma: float = 0.0, cost: float = 1.0, coarse_n: int = 0, n_patches: int = 1,
                 scheme: int = 3, band_width: float = 1.0, band_window: int = 8,
                 band_group: int = 1, wave_warps: int = 0, resort_passes: int = 0,
                 schedule: int = 0, tile_waves: int = 0, tile_period: int = 0,
                 local_sweeps: int = 0, tile_shape: int = -1, visit: int = 0,
                 drift: Optional[np.ndarray] = None, stream=None, device_inputs: bool = False,
                 sigma_field: Optional[np.ndarray] = None, diffusion: int = 0,
                 cost_field: Optional[np.ndarray] = None,
                 control_cost: Optional[np.ndarray] = None):
        self._h = None
        self.n = int(n)
        self.N = self.n * self.n
        self.controls = _c(controls, np.float64).reshape(-1, 2)
        self.n_controls = self.controls.shape[0]
        self.coarse_n = int(coarse_n)
        self.n_patches = int(n_patches)
        d = Desc()
        d.n, d.n_controls, d.h, d.lam, d.sigma, d.cost = (self.n, self.n_controls, float(h),
                                                         float(lam), float(sigma), float(cost))
        d.coarse_n, d.n_patches, d.scheme = self.coarse_n, self.n_patches, int(scheme)
        d.band_width, d.band_window = float(band_width), int(band_window)
        d.band_group, d.wave_warps, d.resort_passes = int(band_group), int(wave_warps), int(resort_passes)
        d.schedule, d.tile_waves, d.tile_period = int(schedule), int(tile_waves), int(tile_period)
        d.local_sweeps = int(local_sweeps)
        d.tile_shape = int(tile_shape)
        d.visit = int(visit)
        self.desc = d
        st = None
        if stream is not None:
            st = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        handle = ctypes.c_void_p()
        general = (sigma_field is not None or cost_field is not None or control_cost is not None
                   or int(diffusion) != 0)
        if general and device_inputs:
            raise ValueError("the general terms take host arrays")
        if device_inputs:
            # torch CUDA tensors (or raw device pointers as ints)
            ptr = lambda t: None if t is None else ctypes.c_void_p(t if isinstance(t, int) else t.data_ptr())
            rc = lib().hjb_create_problem_device(ctypes.byref(d), ptr(speed), ptr(mask), ptr(sector),
                                                 _p(self.controls), ptr(drift), st,
                                                 ctypes.byref(handle))
        else:
            self._speed = _c(speed, np.float32).reshape(-1)
            self._mask = _c(mask, np.uint8).reshape(-1)
            self._sector = None if sector is None else _c(sector, np.int8).reshape(-1)
            self._drift = None if drift is None else _c(drift, np.float32).reshape(-1)
            if self._speed.size != self.N or self._mask.size != self.N:
                raise ValueError("speed and mask must have n*n entries")
            if general:
                # sigma(x), the diffusion form and l(x) + m(a) of Section 5.3
                self._sigf = None if sigma_field is None else _c(sigma_field, np.float32).reshape(-1)
                self._costf = None if cost_field is None else _c(cost_field, np.float32).reshape(-1)
                self._cctl = None if control_cost is None else _c(control_cost, np.float64).reshape(-1)
                t = Terms()
                t.sigma_field, t.diffusion = _p(self._sigf), int(diffusion)
                t.cost_field, t.control_cost = _p(self._costf), _p(self._cctl)
                rc = lib().hjb_create_problem_general(ctypes.byref(d), _p(self._speed), _p(self._mask),
                                                      _p(self._sector), _p(self.controls),
                                                      _p(self._drift), ctypes.byref(t), st,
                                                      ctypes.byref(handle))
            else:
                rc = lib().hjb_create_problem(ctypes.byref(d), _p(self._speed), _p(self._mask),
                                              _p(self._sector), _p(self.controls), _p(self._drift),
                                              st, ctypes.byref(handle))
        check(rc, "hjb_create_problem")
        self._h = handle

    @classmethod
    def from_instance(cls, inst, **kw) -> "Problem":
        args = dict(h=inst.h, lam=inst.lam, sigma=inst.sigma, cost=inst.cost,
                    coarse_n=inst.coarse_n, n_patches=inst.n_patches, drift=inst.drift,
                    sigma_field=getattr(inst, "sigma_field", None),
                    diffusion=getattr(inst, "diffusion", 0),
                    cost_field=getattr(inst, "cost_field", None),
                    control_cost=getattr(inst, "control_cost", None))
        args.update(kw)
        return cls(inst.n, inst.controls, inst.speed, inst.mask, inst.sector, **args)

    # ------------------------------------------------------------ lifetime
    def close(self):
        if self._h is not None and self._h.value:
            lib().hjb_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ----------------------------------------------------------- solve steps
    @staticmethod
    def _ret(rc: int, st: Stats, where: str, check_conv: bool) -> dict:
        if rc == HJB_ERR_NOT_CONVERGED and not check_conv:
            return st.as_dict()
        check(rc, where)
        return st.as_dict()

    def coarse_solve(self, tol_c: float = 1e-6, max_sweeps: int = 100000,
                     check_conv: bool = True) -> dict:
        st = Stats()
        rc = lib().hjb_coarse_solve(self._h, tol_c, max_sweeps, ctypes.byref(st))
        return self._ret(rc, st, "hjb_coarse_solve", check_conv)

    def build_patches(self) -> dict:
        st = Stats()
        check(lib().hjb_build_patches(self._h, ctypes.byref(st)), "hjb_build_patches")
        return st.as_dict()

    def set_uhat(self, uhat: np.ndarray) -> None:
        """Replace u_hat (``hjb_set_uhat``) and redo the pre-computation after it."""
        uhat = _c(uhat, np.float32).reshape(-1)
        check(lib().hjb_set_uhat(self._h, _p(uhat)), "hjb_set_uhat")

    def set_feedback(self, a: np.ndarray) -> None:
        a = _c(a, np.uint8).reshape(-1)
        check(lib().hjb_set_feedback(self._h, _p(a)), "hjb_set_feedback")

    def solve_patches(self, tol32: float = 5e-7, tol64: float = 1e-6, max_passes: int = 10000,
                      check_conv: bool = True) -> dict:
        st = Stats()
        rc = lib().hjb_solve_patches(self._h, tol32, tol64, max_passes, ctypes.byref(st))
        return self._ret(rc, st, "hjb_solve_patches", check_conv)

    def solve_full(self, precision: int = 32, tol: float = 5e-7, tol64: float = 1e-6,
                   max_sweeps: int = 200000, check_conv: bool = True) -> dict:
        st = Stats()
        rc = lib().hjb_solve_full(self._h, precision, tol, tol64, max_sweeps, ctypes.byref(st))
        return self._ret(rc, st, "hjb_solve_full", check_conv)

    def apply_operator(self, u: np.ndarray, precision: int = 64, scheme: int = 3):
        u = _c(u, np.float64).reshape(-1)
        out = np.empty(self.N)
        am = np.empty(self.N, np.int32)
        check(lib().hjb_apply_operator(self._h, precision, scheme, _p(u), _p(out), _p(am)),
              "hjb_apply_operator")
        return out, am

    def residual(self) -> float:
        r = ctypes.c_double()
        check(lib().hjb_residual(self._h, ctypes.byref(r)), "hjb_residual")
        return r.value

    # -------------------------------------------------------------- state
    def set_value(self, u: np.ndarray) -> None:
        u = _c(u, np.float64).reshape(-1)
        check(lib().hjb_set_value(self._h, _p(u)), "hjb_set_value")

    def get_value(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """The fine value (float64, n^2); into `out` when given (e.g. a buffer in
        pinned host memory reused across solves)."""
        if out is None:
            out = np.empty(self.N)
        elif out.dtype != np.float64 or out.size != self.N or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of n^2 elements")
        check(lib().hjb_get_value(self._h, _p(out)), "hjb_get_value")
        return out

    def get_coarse_value(self) -> np.ndarray:
        out = np.empty(self.coarse_n * self.coarse_n)
        check(lib().hjb_get_coarse_value(self._h, _p(out)), "hjb_get_coarse_value")
        return out

    def get_uhat(self) -> np.ndarray:
        out = np.empty(self.N)
        check(lib().hjb_get_uhat(self._h, _p(out)), "hjb_get_uhat")
        return out

    def get_feedback(self) -> np.ndarray:
        out = np.empty(self.N, np.uint8)
        check(lib().hjb_get_feedback(self._h, _p(out)), "hjb_get_feedback")
        return out

    def get_successors(self) -> np.ndarray:
        out = np.empty(self.N, np.int32)
        check(lib().hjb_get_successors(self._h, _p(out)), "hjb_get_successors")
        return out

    def get_labels(self) -> np.ndarray:
        out = np.empty(self.N, np.int8)
        check(lib().hjb_get_labels(self._h, _p(out)), "hjb_get_labels")
        return out

    def get_order(self):
        nf, nb = ctypes.c_int32(), ctypes.c_int32()
        check(lib().hjb_get_order(self._h, None, None, None, ctypes.byref(nf), ctypes.byref(nb)),
              "hjb_get_order")
        keys = np.empty(self.N, np.int32)
        order = np.empty(nf.value, np.int32)
        off = np.empty(nb.value + 1, np.int32)
        check(lib().hjb_get_order(self._h, _p(keys), _p(order), _p(off), None, None), "hjb_get_order")
        return keys, order, off

    def device_info(self) -> dict:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(lib().hjb_device_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
              "hjb_device_info")
        return {"num_sms": a.value, "wave_blocks32": b.value, "wave_blocks64": c.value}


class Batch:
    """Many independent problems solved together (wraps an ``hjb_batch*``).

    ``instances`` are objects with the fields of ``hjb_inputs.Instance`` (n,
    speed, mask, sector, h, lam, sigma, coarse_n, n_patches); they share the
    control set ``controls``, the running cost and the scheme."""

    def __init__(self, instances, controls: np.ndarray, *, cost: float = 1.0, scheme: int = 3,
                 tile_shape: int = -1, tile_waves: int = 0, tile_period: int = 2,
                 band_width: float = 1.0, schedule: int = 0, stream=None):
        self._h = None
        insts = list(instances)
        self.count = len(insts)
        self.ns = [int(x.n) for x in insts]
        arr = (BatchInst * self.count)()
        for i, x in enumerate(insts):
            arr[i].n, arr[i].coarse_n, arr[i].n_patches, arr[i].reserved = x.n, x.coarse_n, x.n_patches, 0
            arr[i].h, arr[i].lam, arr[i].sigma = x.h, x.lam, x.sigma
        d = BatchDesc()
        controls = _c(controls, np.float64).reshape(-1, 2)
        d.n_controls, d.scheme, d.tile_shape = controls.shape[0], scheme, tile_shape
        d.tile_waves, d.tile_period, d.schedule = tile_waves, tile_period, int(schedule)
        d.cost, d.band_width = cost, band_width
        # one host array per instance (hjb_batch_create_lists): the library copies
        # each into its place on the device, nothing is concatenated here
        keep = [(_c(x.speed, np.float32).reshape(-1), _c(x.mask, np.uint8).reshape(-1),
                 None if x.sector is None else _c(x.sector, np.int8).reshape(-1)) for x in insts]
        for (sp, mk, sc), n in zip(keep, self.ns):
            if sp.size != n * n or mk.size != n * n or (sc is not None and sc.size != n * n):
                raise ValueError("speed, mask and sector must have n*n entries")
        ptrs = lambda k: (ctypes.c_void_p * self.count)(*[a[k].ctypes.data if a[k] is not None else None
                                                          for a in keep])
        speed_l, mask_l = ptrs(0), ptrs(1)
        sector_l = None if any(a[2] is None for a in keep) else ptrs(2)
        h = ctypes.c_void_p()
        st = None
        if stream is not None:
            st = ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
        check(lib().hjb_batch_create_lists(ctypes.byref(d), self.count, ctypes.cast(arr, ctypes.c_void_p),
                                           ctypes.cast(speed_l, ctypes.c_void_p),
                                           ctypes.cast(mask_l, ctypes.c_void_p),
                                           None if sector_l is None else ctypes.cast(sector_l, ctypes.c_void_p),
                                           _p(controls), st, ctypes.byref(h)), "hjb_batch_create_lists")
        self._h = h

    @classmethod
    def from_instances(cls, insts, **kw) -> "Batch":
        return cls(insts, insts[0].controls, cost=insts[0].cost, **kw)

    def close(self):
        if self._h is not None and self._h.value:
            lib().hjb_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, tol_c: float = 1e-6, tol32: float = 2.5e-7, tol64: float = 1e-6,
              max_passes: int = 100000, check_conv: bool = True):
        """The patchy pipeline for every instance; returns (stats, residuals)."""
        st = Stats()
        res = np.empty(self.count)
        rc = lib().hjb_batch_solve(self._h, tol_c, tol32, tol64, max_passes, ctypes.byref(st), _p(res))
        if not (rc == HJB_ERR_NOT_CONVERGED and not check_conv):
            check(rc, "hjb_batch_solve")
        return st.as_dict(), res

    def solve_full(self, tol32: float = 2.5e-7, tol64: float = 1e-6, max_sweeps: int = 200000,
                   check_conv: bool = True):
        """The plain full-grid Jacobi comparator for every instance."""
        st = Stats()
        res = np.empty(self.count)
        rc = lib().hjb_batch_solve_full(self._h, tol32, tol64, max_sweeps, ctypes.byref(st), _p(res))
        if not (rc == HJB_ERR_NOT_CONVERGED and not check_conv):
            check(rc, "hjb_batch_solve_full")
        return st.as_dict(), res

    def autotune(self, tol_c: float = 1e-6, tol32: float = 2.5e-7) -> dict:
        """Time the candidate tile schedules; returns the choice and the times."""
        shape, waves = ctypes.c_int32(), ctypes.c_int32()
        ms = np.zeros(9)
        check(lib().hjb_batch_autotune(self._h, tol_c, tol32, ctypes.byref(shape), ctypes.byref(waves),
                                       _p(ms)), "hjb_batch_autotune")
        names = [f"{s}/B{b}" for s in ("8x8", "8x4", "4x4") for b in (1, 2)]
        names += [f"{s}/worklist" for s in ("8x8", "8x4", "4x4")]
        tried = {k: v for k, v in zip(names, ms.tolist()) if v > 0}
        best = min(tried, key=tried.get)
        return {"tile_shape": shape.value, "tile_waves": waves.value,
                "schedule": 3 if best.endswith("worklist") else 4, "ms": tried}

    def get_value(self, index: int) -> np.ndarray:
        out = np.empty(self.ns[index] ** 2)
        check(lib().hjb_batch_get_value(self._h, index, _p(out)), "hjb_batch_get_value")
        return out

    def get_values(self, out: Optional[np.ndarray] = None) -> list:
        """Every instance's value from one read-back (``hjb_batch_get_values``): a
        list of n_i^2 arrays, views of one buffer (`out`, sum n_i^2 float64, when
        given: e.g. pinned host memory reused across solves)."""
        sizes = [n * n for n in self.ns]
        if out is None:
            out = np.empty(sum(sizes))
        elif out.dtype != np.float64 or out.size != sum(sizes) or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array of sum n_i^2 elements")
        check(lib().hjb_batch_get_values(self._h, _p(out)), "hjb_batch_get_values")
        return np.split(out, np.cumsum(sizes)[:-1])

    def get_feedback(self, index: int) -> np.ndarray:
        out = np.empty(self.ns[index] ** 2, np.uint8)
        check(lib().hjb_batch_get_feedback(self._h, index, _p(out)), "hjb_batch_get_feedback")
        return out

    def get_labels(self, index: int) -> np.ndarray:
        out = np.empty(self.ns[index] ** 2, np.int8)
        check(lib().hjb_batch_get_labels(self._h, index, _p(out)), "hjb_batch_get_labels")
        return out

    def get_uhat(self, index: int) -> np.ndarray:
        out = np.empty(self.ns[index] ** 2, np.float32)
        check(lib().hjb_batch_get_uhat(self._h, index, _p(out)), "hjb_batch_get_uhat")
        return out

    # --------------------------------------------------- coarse / warm start
    def coarse_solve(self, tol_c: float = 1e-6, max_sweeps: int = 100000, check_conv: bool = True):
        """The coarse solves alone; returns (stats, sweeps per instance, fallback flags)."""
        st = Stats()
        sw = np.zeros(self.count, np.int32)
        fb = np.zeros(self.count, np.uint8)
        rc = lib().hjb_batch_coarse_solve(self._h, tol_c, max_sweeps, ctypes.byref(st), _p(sw), _p(fb))
        if not (rc == HJB_ERR_NOT_CONVERGED and not check_conv):
            check(rc, "hjb_batch_coarse_solve")
        return st.as_dict(), sw, fb

    def precompute(self, tol_c: float = 1e-6) -> dict:
        st = Stats()
        check(lib().hjb_batch_precompute(self._h, tol_c, ctypes.byref(st)), "hjb_batch_precompute")
        return st.as_dict()

    def get_coarse_value(self, index: int, nc: int) -> np.ndarray:
        out = np.empty(nc * nc, np.float32)
        check(lib().hjb_batch_get_coarse_value(self._h, index, _p(out)), "hjb_batch_get_coarse_value")
        return out

    def net_inputs(self, x) -> None:
        """Fill the device tensor x (bf16 bits [count][nc][nc][16]) with the network input."""
        check(lib().hjb_batch_net_inputs(self._h, ctypes.c_void_p(x.data_ptr())), "hjb_batch_net_inputs")

    def net_targets(self, tval, tctrl, freem) -> None:
        check(lib().hjb_batch_net_targets(self._h, ctypes.c_void_p(tval.data_ptr()),
                                          ctypes.c_void_p(tctrl.data_ptr()), ctypes.c_void_p(freem.data_ptr())),
              "hjb_batch_net_targets")

    def coarse_warm(self, net_out_ptr, first: int = 0, count: int = 0, k_sweeps: int = 4,
                    fallback_tol: float = 1e-2) -> None:
        """Start later coarse solves of instances [first, first + count) from a
        network output (device pointer or tensor, FP32 [count][nc][nc][48]); None
        restores the plain start for every instance."""
        if net_out_ptr is None:
            check(lib().hjb_batch_coarse_warm(self._h, None, 0, 0, 0, 0.0), "hjb_batch_coarse_warm")
            return
        ptr = net_out_ptr.data_ptr() if hasattr(net_out_ptr, "data_ptr") else int(net_out_ptr)
        check(lib().hjb_batch_coarse_warm(self._h, ctypes.c_void_p(ptr), first, count or self.count, k_sweeps,
                                          fallback_tol), "hjb_batch_coarse_warm")


# layer shapes of the warm-start network: (cin stored, cout)
NET_LAYERS = [(16, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 33)]
NET_IN_REAL = 5
NET_DIL = [1, 2, 4, 8, 16, 32]   # dilation of each layer


class Net:
    """The learned warm start's network on the GPU (wraps an ``hjb_net*``).

    Inputs and targets of ``train_step`` / ``forward`` are device tensors (any
    object with ``data_ptr()``); parameters move through host arrays."""

    def __init__(self, max_batch: int, height: int, width: int, stream=None):
        self._h = None
        self.max_batch, self.H, self.W = max_batch, height, width
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
        check(lib().hjb_net_create(max_batch, height, width, st, ctypes.byref(h)), "hjb_net_create")
        self._h = h
        self.n_params = int(lib().hjb_net_param_count())

    def close(self):
        if self._h is not None and self._h.value:
            lib().hjb_net_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- parameters
    @staticmethod
    def unpack(params: np.ndarray) -> list:
        """[(w (cout, 9, cin), b (cout,)), ...] views of a flat parameter array."""
        out, o = [], 0
        for cin, cout in NET_LAYERS:
            nw = cout * 9 * cin
            out.append((params[o:o + nw].reshape(cout, 9, cin), params[o + nw:o + nw + cout]))
            o += nw + cout
        return out

    @staticmethod
    def pack(layers) -> np.ndarray:
        return np.concatenate([np.concatenate([np.asarray(w, np.float64).reshape(-1),
                                               np.asarray(b, np.float64).reshape(-1)]) for w, b in layers])

    def init_params(self, seed: int) -> np.ndarray:
        """He-normal weights (std sqrt(2 / (9 cin)), cin the real inputs), zero
        biases, zero weights on the padding input channels of layer 0."""
        rng = np.random.default_rng(np.random.PCG64(seed))
        layers = []
        for li, (cin, cout) in enumerate(NET_LAYERS):
            real = NET_IN_REAL if li == 0 else cin
            w = np.zeros((cout, 9, cin))
            w[:, :, :real] = rng.standard_normal((cout, 9, real)) * np.sqrt(2.0 / (9 * real))
            layers.append((w, np.zeros(cout)))
        return self.pack(layers)

    def set_params(self, params: np.ndarray) -> None:
        p = _c(params, np.float32)
        check(lib().hjb_net_set_params(self._h, _p(p)), "hjb_net_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        check(lib().hjb_net_get_params(self._h, _p(out)), "hjb_net_get_params")
        return out.astype(np.float64)

    def get_grads(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        check(lib().hjb_net_get_grads(self._h, _p(out)), "hjb_net_get_grads")
        return out.astype(np.float64)

    # ------------------------------------------------------------- compute
    def forward(self, x, batch: int, host_out: bool = False):
        out = np.empty((batch, self.H, self.W, 48), np.float32) if host_out else None
        check(lib().hjb_net_forward(self._h, batch, ctypes.c_void_p(x.data_ptr()), _p(out)), "hjb_net_forward")
        return out

    def train_step(self, x, tval, tctrl, free, n_free: int, lr: float = 1e-3, w_value: float = 1.0,
                   w_ctrl: float = 0.1):
        batch = int(x.shape[0])
        loss = np.zeros(2)
        check(lib().hjb_net_train_step(self._h, batch, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(tval.data_ptr()), ctypes.c_void_p(tctrl.data_ptr()),
                                       ctypes.c_void_p(free.data_ptr()), int(n_free), lr, w_value, w_ctrl,
                                       _p(loss)), "hjb_net_train_step")
        return float(loss[0]), float(loss[1])

    def output_ptr(self) -> int:
        """Device address of the last forward's output (FP32 [batch][H][W][48])."""
        p = ctypes.c_void_p()
        check(lib().hjb_net_output_device(self._h, ctypes.byref(p)), "hjb_net_output_device")
        return int(p.value)

    def warm_values(self, index: int, mask, scale: float, umax: float, uob: float, u0) -> None:
        check(lib().hjb_net_warm_values(self._h, index, ctypes.c_void_p(mask.data_ptr()), scale, umax, uob,
                                        ctypes.c_void_p(u0.data_ptr())), "hjb_net_warm_values")
