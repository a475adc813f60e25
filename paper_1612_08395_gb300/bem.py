"""ctypes binding of libbem_gb300.so (include/bem.h): argument marshalling only.

Every array may be a numpy array (host) or a torch tensor (host or CUDA); the
library reads or writes it in place through its data pointer.  Arrays must be
C-contiguous float64 of Ny x Nx elements.  Nothing here computes any part of
the method; a missing library raises ``BemLibraryMissing``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# BEM_DEBUG_CHECKS=1 selects the bounds-checked debug build (build.py)
LIB_PATH = os.path.join(_PKG, "_build_debug" if os.environ.get("BEM_DEBUG_CHECKS", "0") == "1" else "_build",
                        "libbem_gb300.so")

BEM_OK = 0
BEM_EINVAL = -1
BEM_ENOMEM = -2
BEM_ENOCONV = -3
BEM_ENUMERIC = -4
BEM_ETIMEOUT = -5
BEM_ECUDA = -6
BEM_ECANCELED = -7
PREC_FP64 = 0
PREC_FP32 = 1
PREC_FP32_REFINE = 2
_PREC = {"fp64": PREC_FP64, "fp32": PREC_FP32, "fp32_refine": PREC_FP32_REFINE}


class BemLibraryMissing(RuntimeError):
    pass


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bem error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_sweeps", ctypes.c_int), ("flags", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("force", ctypes.c_double), ("area", ctypes.c_double),
                ("contact_radius", ctypes.c_double), ("final_eps", ctypes.c_double),
                ("max_gap_violation", ctypes.c_double), ("depth", ctypes.c_double),
                ("iterations", ctypes.c_int), ("detach_rounds", ctypes.c_int),
                ("contact_count", ctypes.c_int), ("status", ctypes.c_int), ("stalled", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("Px", ctypes.c_int), ("Py", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("k", ctypes.c_double),
                ("nu", ctypes.c_double), ("E0", ctypes.c_double), ("c0", ctypes.c_double),
                ("alpha", ctypes.c_double), ("compliance", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("kernel_launches", ctypes.c_ulonglong),
                ("rows_per_cta", ctypes.c_int), ("cols_per_cta", ctypes.c_int), ("col_radix", ctypes.c_int)]


class Job(ctypes.Structure):
    _fields_ = [("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("k", ctypes.c_double), ("nu", ctypes.c_double),
                ("E0", ctypes.c_double), ("c0", ctypes.c_double), ("profile", ctypes.c_void_p),
                ("d_steps", ctypes.c_void_p), ("nsteps", ctypes.c_int), ("dgamma", ctypes.c_double),
                ("opts", Opts), ("per_step", ctypes.c_void_p), ("final_pressure", ctypes.c_void_p),
                ("tag", ctypes.c_longlong)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_longlong), ("status", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double), ("device", ctypes.c_int)]


class DeviceView(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_size_t), ("used", ctypes.c_size_t), ("evictable", ctypes.c_size_t),
                ("cached_bytes", ctypes.c_size_t), ("idle_workers", ctypes.c_int),
                ("has_cached", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbem_gb300.so (built by paper_1612_08395_gb300/build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise BemLibraryMissing(f"{path} not found: build it with paper_1612_08395_gb300/build.py")
    lib = ctypes.CDLL(path)
    dp, vp, ip = ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int
    lib.bem_create.argtypes = [ip, ip] + [ctypes.c_double] * 6 + [ctypes.POINTER(vp)]
    lib.bem_destroy.argtypes = [vp]
    lib.bem_destroy.restype = None
    lib.bem_last_error.restype = ctypes.c_char_p
    lib.bem_solve.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.POINTER(Opts), vp, ctypes.POINTER(Result)]
    lib.bem_sweep.argtypes = [vp, vp, vp, ip, ctypes.c_double, ctypes.POINTER(Opts),
                              ctypes.POINTER(Result), vp]
    lib.bem_sweep_from.argtypes = [vp, vp, vp, ip, ctypes.c_double, ctypes.POINTER(Opts), vp, vp,
                                   ctypes.POINTER(Result), vp]
    lib.bem_contact_set.argtypes = [vp, vp]
    lib.bem_influence_table.argtypes = [vp, vp]
    lib.bem_spectrum.argtypes = [vp, vp]
    lib.bem_convolve.argtypes = [vp, ip, vp, vp]
    lib.bem_get_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.bem_convolve_noalloc.argtypes = [vp, ip, ip, ctypes.c_double, vp, vp, vp]
    lib.bem_pass_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong), ip]
    lib.bem_pass_work.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    for fn in (lib.bem_alpha, lib.bem_c1_corrected):
        fn.restype = ctypes.c_double
    lib.bem_alpha.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.bem_c1_corrected.argtypes = [ctypes.c_double]
    lib.bem_p_crit.restype = ctypes.c_double
    lib.bem_p_crit.argtypes = [ctypes.c_double] * 6
    lib.bem_set_material.argtypes = [vp] + [ctypes.c_double] * 3
    lib.bem_server_create.argtypes = [ip, ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.bem_server_create_on.argtypes = [ip, ctypes.POINTER(ctypes.c_int), ip, ctypes.c_size_t,
                                         ctypes.POINTER(vp)]
    lib.bem_server_place.argtypes = [ip, ctypes.POINTER(DeviceView), ctypes.c_size_t]
    lib.bem_server_submit.argtypes = [vp, ctypes.POINTER(Job)]
    lib.bem_server_poll.argtypes = [vp, ctypes.POINTER(Completion), ip, ip]
    lib.bem_server_pending.argtypes = [vp]
    lib.bem_server_cancel.argtypes = [vp, ctypes.c_longlong]
    lib.bem_server_loop_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.bem_server_bytes.argtypes = [vp]
    lib.bem_server_bytes.restype = ctypes.c_size_t
    lib.bem_server_footprint.argtypes = [ip, ip]
    lib.bem_server_footprint.restype = ctypes.c_size_t
    lib.bem_server_destroy.argtypes = [vp]
    lib.bem_server_destroy.restype = None
    _lib = lib
    return lib


def _check(rc, allow=()):
    if rc != BEM_OK and rc not in allow:
        raise BemError(rc, load_library().bem_last_error().decode())
    return rc


def _ptr(a, n=None, writable=False):
    """Data pointer of a C-contiguous float64 numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensor must be contiguous float64")
        if n is not None and a.numel() != n:
            raise ValueError(f"expected {n} elements, got {a.numel()}")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise ValueError("array must be a C-contiguous float64 numpy array")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} elements, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data)


def convolve_noalloc(khat, nx, ny, compliance, p, u, stream=None) -> int:
    """bem_convolve_noalloc on device tensors (no allocation inside); returns the status."""
    sp = None if stream is None else getattr(stream, "cuda_stream", stream)
    return load_library().bem_convolve_noalloc(_ptr(khat), nx, ny, compliance, _ptr(p, nx * ny),
                                               _ptr(u, nx * ny, writable=True), sp)


def alpha(k: float, nu: float) -> float:
    return load_library().bem_alpha(k, nu)


def c1_corrected(k: float) -> float:
    return load_library().bem_c1_corrected(k)


def p_crit(k, nu, dgamma, delta, E0=1.0, c0=1.0) -> float:
    return load_library().bem_p_crit(k, nu, E0, c0, dgamma, delta)


FLAG_TIME_PASSES = 1


def make_opts(precision="fp32", tol=0.0, max_iter=0, refine_sweeps=0, stream=None, time_passes=False):
    prec = _PREC[precision] if isinstance(precision, str) else int(precision)
    sp = None
    if stream is not None:
        sp = getattr(stream, "cuda_stream", stream)
    return Opts(tol, max_iter, prec, refine_sweeps, FLAG_TIME_PASSES if time_passes else 0, sp)


class Handle:
    """One solver instance: grid, material and the cached influence spectrum."""

    def __init__(self, nx, ny, dx, dy, k, nu, E0=1.0, c0=1.0):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.bem_create(nx, ny, dx, dy, k, nu, E0, c0, ctypes.byref(h)))
        self._h = h
        self.nx, self.ny = nx, ny

    def close(self):
        if getattr(self, "_h", None):
            load_library().bem_destroy(self._h)
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

    @property
    def n(self):
        return self.nx * self.ny

    def info(self) -> Info:
        inf = Info()
        _check(load_library().bem_get_info(self._h, ctypes.byref(inf)))
        return inf

    def pass_times(self, reset=False):
        """(ms[A, B, C] totals, timed iterations, of which fixed-set) under time_passes."""
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_longlong * 2)()
        _check(load_library().bem_pass_times(self._h, ms, cnt, 1 if reset else 0))
        return list(ms), cnt[0], cnt[1]

    def pass_work(self):
        """(bytes[A, B, C], flops[A, B, C]): average algorithmic work per timed launch
        (read before a pass_times reset)."""
        b = (ctypes.c_double * 3)()
        f = (ctypes.c_double * 3)()
        _check(load_library().bem_pass_work(self._h, b, f))
        return list(b), list(f)

    def influence_table(self) -> np.ndarray:
        inf = self.info()
        out = np.empty((inf.Py // 2 + 1, inf.Px // 2 + 1))
        _check(load_library().bem_influence_table(self._h, _ptr(out, writable=True)))
        return out

    def spectrum(self) -> np.ndarray:
        inf = self.info()
        out = np.empty((inf.Py // 2 + 1, inf.Px // 2 + 1))
        _check(load_library().bem_spectrum(self._h, _ptr(out, writable=True)))
        return out

    def convolve(self, p, precision="fp64", out=None):
        if out is None:
            out = np.empty((self.ny, self.nx)) if isinstance(p, np.ndarray) else p.new_empty(p.shape)
        prec = _PREC[precision] if isinstance(precision, str) else int(precision)
        _check(load_library().bem_convolve(self._h, prec, _ptr(p, self.n),
                                           _ptr(out, self.n, writable=True)))
        return out

    def set_material(self, nu, E0=1.0, c0=1.0):
        _check(load_library().bem_set_material(self._h, nu, E0, c0))

    def solve(self, profile, d, dgamma=0.0, d_preload=None, pressure_out=None, check=True, **opts):
        res = Result()
        o = make_opts(**opts)
        pp = _ptr(pressure_out, self.n, writable=True) if pressure_out is not None else None
        rc = load_library().bem_solve(self._h, _ptr(profile, self.n), d, dgamma,
                                      d if d_preload is None else d_preload, ctypes.byref(o), pp,
                                      ctypes.byref(res))
        if check:
            _check(rc, allow=(BEM_ENOCONV,))
        return res, rc

    def contact_set(self) -> np.ndarray:
        """The held contact set after the last sweep or solve (uint8, Ny x Nx)."""
        out = np.empty((self.ny, self.nx), dtype=np.uint8)
        _check(load_library().bem_contact_set(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def sweep_from(self, profile, d_steps, p_state, S_state=None, dgamma=0.0, final_pressure=None,
                   check=True, **opts):
        """Continue a sweep from a saved state (pressure, and contact set if adhesive)."""
        ds = np.ascontiguousarray(np.asarray(d_steps, dtype=np.float64))
        res = (Result * len(ds))()
        o = make_opts(**opts)
        fp = _ptr(final_pressure, self.n, writable=True) if final_pressure is not None else None
        sp = None
        if S_state is not None:
            S_state = np.ascontiguousarray(S_state, dtype=np.uint8)
            if S_state.size != self.n:
                raise ValueError(f"expected {self.n} elements, got {S_state.size}")
            sp = ctypes.c_void_p(S_state.ctypes.data)
        rc = load_library().bem_sweep_from(self._h, _ptr(profile, self.n), _ptr(ds), len(ds), dgamma,
                                           ctypes.byref(o), _ptr(p_state, self.n), sp, res, fp)
        if check:
            _check(rc, allow=(BEM_ENOCONV,))
        return list(res), rc

    def sweep(self, profile, d_steps, dgamma=0.0, final_pressure=None, check=True, **opts):
        ds = np.ascontiguousarray(np.asarray(d_steps, dtype=np.float64))
        res = (Result * len(ds))()
        o = make_opts(**opts)
        fp = _ptr(final_pressure, self.n, writable=True) if final_pressure is not None else None
        rc = load_library().bem_sweep(self._h, _ptr(profile, self.n), _ptr(ds), len(ds), dgamma,
                                      ctypes.byref(o), res, fp)
        if check:
            _check(rc, allow=(BEM_ENOCONV,))
        return list(res), rc


class Server:
    """bem_server_*: independent sweeps run by native worker threads.

    ``submit`` copies the job description and keeps the arrays it points to
    alive until ``poll`` returns the job's completion, which carries the
    per-step results and the final pressure (if one was asked for).
    """

    def __init__(self, nworkers=4, hbm_budget_bytes=16 << 30, devices=None):
        """nworkers workers on the current device, or (devices = a list of CUDA
        device indices) nworkers workers and a budget of hbm_budget_bytes on each."""
        lib = load_library()
        s = ctypes.c_void_p()
        if devices is None:
            _check(lib.bem_server_create(nworkers, hbm_budget_bytes, ctypes.byref(s)))
        else:
            devs = (ctypes.c_int * len(devices))(*devices)
            _check(lib.bem_server_create_on(len(devices), devs, nworkers, hbm_budget_bytes, ctypes.byref(s)))
        self._s = s
        self._live = {}
        self._next = 0

    def submit(self, nx, ny, dx, dy, k, nu, profile, d_steps, dgamma=0.0, E0=1.0, c0=1.0,
               final_pressure=None, **opts):
        ds = np.ascontiguousarray(np.asarray(d_steps, dtype=np.float64))
        res = (Result * len(ds))()
        tag = self._next
        self._next += 1
        fp = _ptr(final_pressure, nx * ny, writable=True) if final_pressure is not None else None
        job = Job(nx, ny, dx, dy, k, nu, E0, c0, _ptr(profile, nx * ny), _ptr(ds), len(ds), dgamma,
                  make_opts(**opts), ctypes.cast(res, ctypes.c_void_p), fp, tag)
        self._live[tag] = (profile, ds, res, final_pressure)
        _check(load_library().bem_server_submit(self._s, ctypes.byref(job)))
        return tag

    def poll(self, max_n=64, wait_ms=0):
        """Completed jobs as dicts: tag, status, t_submit/t_start/t_end (s), results, pressure."""
        buf = (Completion * max_n)()
        n = load_library().bem_server_poll(self._s, buf, max_n, wait_ms)
        if n < 0:
            _check(n)
        out = []
        for c in buf[:n]:
            profile, ds, res, fp = self._live.pop(c.tag)
            out.append({"tag": c.tag, "status": c.status, "t_submit": c.t_submit, "t_start": c.t_start,
                        "t_end": c.t_end, "device": c.device, "results": list(res), "final_pressure": fp})
        return out

    def cancel(self, tag):
        """Cancel a job that has not started; True when it was still queued."""
        return load_library().bem_server_cancel(self._s, tag) == BEM_OK

    def pending(self):
        return load_library().bem_server_pending(self._s)

    def device_bytes(self):
        return load_library().bem_server_bytes(self._s)

    def loop_stats(self):
        """(batched loop graphs launched, solves' CG loops they carried)."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load_library().bem_server_loop_stats(self._s, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    @staticmethod
    def footprint(nx, ny):
        return load_library().bem_server_footprint(nx, ny)

    @staticmethod
    def place(views, need):
        """bem_server_place on a list of dicts with the DeviceView fields."""
        arr = (DeviceView * len(views))(*[DeviceView(**v) for v in views])
        return load_library().bem_server_place(len(views), arr, need)

    def drain(self, timeout_s=600.0):
        """Poll until every submitted job has completed; returns their completions."""
        import time
        out, t_end = [], time.monotonic() + timeout_s
        while self._live:
            if time.monotonic() > t_end:
                raise TimeoutError(f"{len(self._live)} jobs still pending")
            out += self.poll(wait_ms=100)
        return out

    def close(self):
        if getattr(self, "_s", None):
            load_library().bem_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
