"""Python binding of libenkfmc.so (argument marshalling only).

Every step of the analysis runs in the library's CUDA kernels; this module
only loads the shared library, declares the C signatures of include/enkfmc.h,
and turns torch tensors into device pointers.  There is no fallback: if the
library cannot be loaded, `load()` raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libenkfmc.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTSPD", 4: "EDNONPOS", 5: "ENONFINITE",
          6: "ETIMEOUT", 7: "ECUDA", 8: "ENOTIMPL", 9: "ESTATE"}
FP64, FP32 = 0, 1


class enkfmc_problem(ctypes.Structure):
    _fields_ = [("nlon", c_int32), ("nlat", c_int32), ("nlev", c_int32), ("nvar_3d", c_int32),
                ("nvar_2d", c_int32), ("lon_periodic", c_int32), ("r", c_int32),
                ("vert_reach", c_int32), ("N", c_int32), ("sub_lon", c_int32),
                ("sub_lat", c_int32), ("precision", c_int32), ("ridge_c", c_double),
                ("flags", c_int32)]


class enkfmc_info(ctypes.Structure):
    _fields_ = [("n", c_int64), ("pmax", c_int32), ("nsub", c_int32), ("nblock", c_int32),
                ("hb_max", c_int32), ("ext_rows", c_int64), ("halo_rows", c_int64),
                ("band_elems", c_int64), ("workspace_bytes", c_int64), ("m", c_int64),
                ("tc_chol", c_int32), ("tc_solve", c_int32), ("refine_steps", c_int32),
                ("fp64_rows", c_int32)]


_H = c_void_p
# name -> (restype, argtypes); mirrors include/enkfmc.h
SIGNATURES = {
    "enkfmc_create": (c_int32, [POINTER(c_void_p), POINTER(enkfmc_problem), c_void_p]),
    "enkfmc_destroy": (None, [_H]),
    "enkfmc_check_problem": (c_int32, [POINTER(enkfmc_problem)]),
    "enkfmc_strerror": (c_char_p, [c_int32]),
    "enkfmc_query": (c_int32, [_H, POINTER(enkfmc_info)]),
    "enkfmc_set_stream": (c_int32, [_H, c_void_p]),
    "enkfmc_slot_offsets": (c_int32, [_H, c_void_p, c_void_p, c_void_p]),
    "enkfmc_set_observations": (c_int32, [_H, c_void_p, c_int64]),
    "enkfmc_estimate": (c_int32, [_H, c_void_p, c_void_p, c_void_p]),
    "enkfmc_assemble": (c_int32, [_H, c_void_p, c_void_p, c_void_p, c_void_p]),
    "enkfmc_analyze": (c_int32, [_H, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "enkfmc_analyze_dual": (c_int32, [_H, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p]),
    "enkfmc_cycle_host": (c_int32, [_H, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "enkfmc_forecast_shift": (c_int32, [_H, c_void_p, c_void_p, c_int32, c_int32, c_double]),
    "enkfmc_ensemble_sqerr": (c_int32, [_H, c_void_p, c_void_p, c_void_p]),
    "enkfmc_filter_run": (c_int32, [_H, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_double,
                                    c_void_p]),
    "enkfmc_analyze_adjoint": (c_int32, [_H, c_void_p, c_void_p, c_void_p, c_void_p]),
    "enkfmc_get_status": (c_int32, [_H, POINTER(c_int64)]),
    "enkfmc_export_T_pattern": (c_int32, [_H, c_void_p, c_void_p]),
    "enkfmc_fp64_blocks": (c_int32, [_H, POINTER(c_int32)]),
    "enkfmc_batch_create": (c_int32, [POINTER(c_void_p), c_void_p, c_int32, c_int32, c_void_p]),
    "enkfmc_batch_bind": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p]),
    "enkfmc_batch_capture": (c_int32, [c_void_p]),
    "enkfmc_batch_run": (c_int32, [c_void_p]),
    "enkfmc_batch_get_status": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "enkfmc_batch_query": (c_int32, [c_void_p, POINTER(c_int32), c_void_p]),
    "enkfmc_batch_destroy": (None, [c_void_p]),
    "enkfmc_set_tuning": (c_int32, [_H, c_int32, c_int32]),
    "enkfmc_debug_block": (c_int32, [_H, c_int32, c_void_p, c_int64, POINTER(c_int64),
                                     POINTER(c_int32)]),
    "enkfmc_profile": (c_int32, [_H, c_int32]),
    "enkfmc_profile_read": (c_int32, [_H, c_void_p, c_void_p, c_void_p]),
    "enkfmc_kernel_name": (c_char_p, [c_int32]),
    "enkfmc_work_per_launch": (c_int32, [_H, c_void_p, c_void_p]),
    "enkfmc_estimate_noalloc": (c_int32, [POINTER(enkfmc_problem), c_void_p, c_void_p, c_void_p,
                                          c_void_p]),
}
NKERNEL = 18
FLAG_NO_SOLVE_REFINEMENT = 1
FLAG_SIMT_BAND = 2
FLAG_PLAIN_FP32 = 4
FLAG_REFINE_MASK = 0xF00
TUNE_REGRESS_CTAS_PER_SM = 0
TUNE_REGRESS_KERNEL = 1


def flag_refine_steps(k: int) -> int:
    """ENKFMC_FLAG_REFINE_STEPS(k): k refinement steps of every sub-domain solve."""
    return (int(k) & 0xF) << 8

_LIB = None


class EnkfmcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


def load(path: str | None = None, build_if_stale: bool = True):
    """Load libenkfmc.so (building it in-tree first when sources are newer)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_stale and path is None:
        from . import build as _build
        _build.build()
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libenkfmc.so not found at {p}; run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(code: int, where: str):
    if code != 0:
        raise EnkfmcError(code, where)


def problem_of(w, precision=FP32, flags=0) -> enkfmc_problem:
    """The enkfmc_problem of a workload-like object."""
    return enkfmc_problem(w.nlon, w.nlat, w.nlev, w.nvar_3d, w.nvar_2d, int(bool(w.lon_periodic)),
                          w.r, w.vert_reach, w.N, w.sub_lon, w.sub_lat, precision, w.ridge_c, flags)


def check_problem(w, precision=FP32, flags=0) -> int:
    """enkfmc_check_problem: 0 when the library can run the problem, else its status."""
    p = problem_of(w, precision, flags)
    return int(load().enkfmc_check_problem(ctypes.byref(p)))


class Handle:
    """One problem on the current CUDA device; methods mirror the C entry points."""

    def __init__(self, *, nlon, nlat, nlev, nvar_3d, nvar_2d, r, N, sub_lon, sub_lat,
                 precision=FP32, ridge_c=1e-3, vert_reach=1, lon_periodic=True, stream=None,
                 flags=0):
        self.lib = load()
        self.problem = enkfmc_problem(nlon, nlat, nlev, nvar_3d, nvar_2d, int(bool(lon_periodic)),
                                      r, vert_reach, N, sub_lon, sub_lat, precision, ridge_c,
                                      flags)
        h = c_void_p()
        _check(self.lib.enkfmc_create(ctypes.byref(h), ctypes.byref(self.problem),
                                      c_void_p(stream)), "enkfmc_create")
        self.h = h
        self.precision = precision
        self.info = self.query()

    @classmethod
    def from_workload(cls, w, precision=FP32, stream=None, flags=0):
        return cls(nlon=w.nlon, nlat=w.nlat, nlev=w.nlev, nvar_3d=w.nvar_3d, nvar_2d=w.nvar_2d,
                   r=w.r, N=w.N, sub_lon=w.sub_lon, sub_lat=w.sub_lat, precision=precision,
                   ridge_c=w.ridge_c, vert_reach=w.vert_reach, lon_periodic=w.lon_periodic,
                   stream=stream, flags=flags)

    def close(self):
        if getattr(self, "h", None):
            self.lib.enkfmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self) -> enkfmc_info:
        info = enkfmc_info()
        _check(self.lib.enkfmc_query(self.h, ctypes.byref(info)), "enkfmc_query")
        return info

    def set_stream(self, stream):
        _check(self.lib.enkfmc_set_stream(self.h, c_void_p(stream)), "enkfmc_set_stream")

    def slot_offsets(self):
        pm = self.info.pmax
        dk, dy, dx = (np.zeros(pm, np.int32) for _ in range(3))
        _check(self.lib.enkfmc_slot_offsets(self.h, _ptr(dk), _ptr(dy), _ptr(dx)), "slot_offsets")
        return dk, dy, dx

    def set_observations(self, obs_idx):
        a = np.ascontiguousarray(obs_idx, dtype=np.int32)
        _check(self.lib.enkfmc_set_observations(self.h, _ptr(a) if a.size else None, a.size),
               "enkfmc_set_observations")
        self.info = self.query()

    def estimate(self, Xb, Tvals, D):
        _check(self.lib.enkfmc_estimate(self.h, _ptr(Xb), _ptr(Tvals), _ptr(D)), "enkfmc_estimate")

    def assemble(self, Xb, Tvals, D, R):
        _check(self.lib.enkfmc_assemble(self.h, _ptr(Xb), _ptr(Tvals), _ptr(D), _ptr(R)),
               "enkfmc_assemble")

    def analyze(self, Xb, y, R, Z, Xa):
        _check(self.lib.enkfmc_analyze(self.h, _ptr(Xb), _ptr(y), _ptr(R), _ptr(Z), _ptr(Xa)),
               "enkfmc_analyze")

    def analyze_dual(self, Xb, Tvals, D, y, R, Z, Xa):
        _check(self.lib.enkfmc_analyze_dual(self.h, _ptr(Xb), _ptr(Tvals), _ptr(D), _ptr(y),
                                            _ptr(R), _ptr(Z), _ptr(Xa)), "enkfmc_analyze_dual")

    def analyze_adjoint(self, Xa_bar, y_bar, R_bar, Xb_bar):
        _check(self.lib.enkfmc_analyze_adjoint(self.h, _ptr(Xa_bar), _ptr(y_bar), _ptr(R_bar),
                                               _ptr(Xb_bar)), "enkfmc_analyze_adjoint")

    def cycle_host(self, Xb, y, R, Z, Xa):
        _check(self.lib.enkfmc_cycle_host(self.h, _ptr(Xb), _ptr(y), _ptr(R), _ptr(Z), _ptr(Xa)),
               "enkfmc_cycle_host")

    def forecast_shift(self, X, Xout, nvec: int, shift: int, inflation: float = 1.0):
        _check(self.lib.enkfmc_forecast_shift(self.h, _ptr(X), _ptr(Xout), nvec, shift,
                                              float(inflation)), "enkfmc_forecast_shift")

    def ensemble_sqerr(self, Xa, xref, out):
        _check(self.lib.enkfmc_ensemble_sqerr(self.h, _ptr(Xa), _ptr(xref), _ptr(out)),
               "enkfmc_ensemble_sqerr")

    def filter_run(self, Xb, ys, Zs, R, xrefs, Tvals, D, Xa, M: int, shift: int, sqerr,
                   inflation: float = 1.0):
        _check(self.lib.enkfmc_filter_run(self.h, _ptr(Xb), _ptr(ys), _ptr(Zs), _ptr(R),
                                          _ptr(xrefs), _ptr(Tvals), _ptr(D), _ptr(Xa), M, shift,
                                          float(inflation), _ptr(sqerr)), "enkfmc_filter_run")

    def set_tuning(self, knob: int, value: int):
        _check(self.lib.enkfmc_set_tuning(self.h, knob, value), "enkfmc_set_tuning")

    def get_status(self):
        info = c_int64(0)
        code = self.lib.enkfmc_get_status(self.h, ctypes.byref(info))
        return int(code), int(info.value)

    def fp64_blocks(self) -> int:
        """Blocks the last assemble factored in double precision (synchronises)."""
        c = c_int32(0)
        _check(self.lib.enkfmc_fp64_blocks(self.h, ctypes.byref(c)), "enkfmc_fp64_blocks")
        return int(c.value)

    def check(self, where="device status"):
        code, info = self.get_status()
        if code:
            raise EnkfmcError(code, f"{where} (info {info})")

    def export_T_pattern(self):
        n = self.info.n
        rowptr = np.zeros(n + 1, np.int64)
        _check(self.lib.enkfmc_export_T_pattern(self.h, _ptr(rowptr), None), "export_T_pattern")
        col = np.zeros(max(1, int(rowptr[-1])), np.int32)
        _check(self.lib.enkfmc_export_T_pattern(self.h, _ptr(rowptr), _ptr(col)), "export_T_pattern")
        return rowptr, col[:int(rowptr[-1])]

    def profile(self, enable: bool):
        _check(self.lib.enkfmc_profile(self.h, int(bool(enable))), "enkfmc_profile")

    def profile_read(self, kernels: bool = False):
        """{kind: (calls, total ms)} since the previous read; with kernels=True
        {kind: (calls, CUDA kernels, total ms)}."""
        n = np.zeros(NKERNEL, np.int64)
        nk = np.zeros(NKERNEL, np.int64)
        ms = np.zeros(NKERNEL, np.float64)
        _check(self.lib.enkfmc_profile_read(self.h, _ptr(n), _ptr(nk), _ptr(ms)),
               "enkfmc_profile_read")
        names = [self.lib.enkfmc_kernel_name(k).decode() for k in range(NKERNEL)]
        if kernels:
            return {names[k]: (int(n[k]), int(nk[k]), float(ms[k])) for k in range(NKERNEL)}
        return {names[k]: (int(n[k]), float(ms[k])) for k in range(NKERNEL)}

    def work_per_launch(self):
        """{kernel name: (algorithmic flops, algorithmic bytes)} per launch."""
        f = np.zeros(NKERNEL, np.float64)
        b = np.zeros(NKERNEL, np.float64)
        _check(self.lib.enkfmc_work_per_launch(self.h, _ptr(f), _ptr(b)), "work_per_launch")
        return {self.lib.enkfmc_kernel_name(k).decode(): (float(f[k]), float(b[k]))
                for k in range(NKERNEL)}

    def debug_block(self, b, dtype):
        nb, hb = c_int64(0), c_int32(0)
        _check(self.lib.enkfmc_debug_block(self.h, b, None, 0, ctypes.byref(nb), ctypes.byref(hb)),
               "debug_block")
        buf = np.zeros(nb.value * (hb.value + 1), dtype=dtype)
        _check(self.lib.enkfmc_debug_block(self.h, b, _ptr(buf), buf.size, ctypes.byref(nb),
                                           ctypes.byref(hb)), "debug_block")
        return buf.reshape(nb.value, hb.value + 1), hb.value


class Batch:
    """Independent problems run as one CUDA graph per cycle (enkfmc_batch_*).

    handles: Handle objects (kept alive by the batch); bind() each instance's
    device tensors, capture() once, then run() replays one cycle of all."""

    def __init__(self, handles, nstreams=8, stream=None):
        self.lib = load()
        self.handles = list(handles)
        arr = (c_void_p * len(self.handles))(*[h.h.value for h in self.handles])
        b = c_void_p()
        _check(self.lib.enkfmc_batch_create(ctypes.byref(b), arr, len(self.handles), nstreams,
                                            c_void_p(stream)), "enkfmc_batch_create")
        self.b = b
        self._keep = {}

    def bind(self, i, Xb, T, D, y, R, Z, Xa):
        self._keep[i] = (Xb, T, D, y, R, Z, Xa)
        _check(self.lib.enkfmc_batch_bind(self.b, i, _ptr(Xb), _ptr(T), _ptr(D), _ptr(y),
                                          _ptr(R), _ptr(Z), _ptr(Xa)), "enkfmc_batch_bind")

    def capture(self):
        _check(self.lib.enkfmc_batch_capture(self.b), "enkfmc_batch_capture")

    def run(self):
        _check(self.lib.enkfmc_batch_run(self.b), "enkfmc_batch_run")

    def status(self):
        """(status [nprob], info [nprob]) after synchronising."""
        st = np.zeros(len(self.handles), np.int32)
        info = np.zeros(len(self.handles), np.int64)
        self.lib.enkfmc_batch_get_status(self.b, _ptr(st), _ptr(info))
        return st, info

    def streams(self):
        ns = c_int32(0)
        of = np.zeros(len(self.handles), np.int32)
        _check(self.lib.enkfmc_batch_query(self.b, ctypes.byref(ns), _ptr(of)), "batch_query")
        return int(ns.value), of

    def close(self):
        if getattr(self, "b", None):
            self.lib.enkfmc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
