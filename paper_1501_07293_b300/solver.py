"""Thin ctypes binding over libmm_b300.so (declared in include/mm_b300.h).

Argument marshalling only: every step of the field evaluation and of the
time integration runs in the library's CUDA kernels.  Device arrays are torch
tensors (float32, contiguous, on the context's device); host arrays are numpy
arrays.  The library is required: importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

# MM_B300_BOUNDS_CHECK=1 selects the bounds-check build of the library
# (libmm_b300_bc.so: index checks in the kernels that report MM_EBOUNDS)
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "libmm_b300_bc.so" if os.environ.get("MM_B300_BOUNDS_CHECK") == "1" else "libmm_b300.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ETIMEOUT, MM_ENONFINITE, MM_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
MM_EBOUNDS = -7
STATUS_NAMES = {0: "MM_OK", -1: "MM_EINVAL", -2: "MM_ENOMEM", -3: "MM_ECUDA", -4: "MM_ETIMEOUT",
                -5: "MM_ENONFINITE", -6: "MM_EUNSUPPORTED",
                -7: "MM_EBOUNDS"}
MM_FP32, MM_SPLIT_BF16, MM_SPLIT_FP16 = 0, 1, 2
MM_RK4, MM_EULER = 0, 1
MM_ZFORM_AUTO, MM_ZFORM_DIRECT = 0, 1
TERM_EXCHANGE, TERM_ANISOTROPY, TERM_DEMAG, TERM_ZEEMAN, TERM_ALL = 1, 2, 4, 8, 15


class MMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("integrator", ctypes.c_int), ("self_term", ctypes.c_int),
                ("obs_every", ctypes.c_int), ("stream", ctypes.c_void_p), ("tune_cache", ctypes.c_char_p),
                ("zform", ctypes.c_int)]


class Segment(ctypes.Structure):
    """mm_segment: [t_begin, t_end) s, b_begin/b_end (T, linear in between), alpha (< 0: context's)."""
    _fields_ = [("t_begin", ctypes.c_double), ("t_end", ctypes.c_double), ("b_begin", ctypes.c_double * 3),
                ("b_end", ctypes.c_double * 3), ("alpha", ctypes.c_double)]


PROGRAM_MAX = 32
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGNATURES = {
    "mm_default_opts": (None, [ctypes.POINTER(Opts)]),
    "mm_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), _D, _D, _D, _D, _D, _D, ctypes.POINTER(Opts)]),
    "mm_destroy": (None, [_P]),
    "mm_set_stream": (_I, [_P, _P]),
    "mm_padded_dims": (_I, [_P, ctypes.POINTER(_I)]),
    "mm_set_m": (_I, [_P, _P]),
    "mm_get_m": (_I, [_P, _P]),
    "mm_set_field": (_I, [_P, ctypes.POINTER(_D), _P, _P]),
    "mm_set_alpha": (_I, [_P, _D]),
    "mm_set_program": (_I, [_P, _I, ctypes.POINTER(Segment)]),
    "mm_set_time": (_I, [_P, _D]),
    "mm_get_time": (_I, [_P, ctypes.POINTER(_D)]),
    "mm_heff": (_I, [_P, _P, ctypes.c_uint]),
    "mm_step": (_I, [_P, _I, _D]),
    "mm_energy": (_I, [_P, ctypes.POINTER(_D)]),
    "mm_observables": (_I, [_P, ctypes.POINTER(_D)]),
    "mm_step_timed": (_I, [_P, _I, _D, ctypes.POINTER(_D)]),
    "mm_adjoint": (_I, [_P, _I, _D, _I, _P, _P, _P, _P]),
    "mm_set_adjoint_memory": (_I, [_P, _D]),
    "mm_get_series": (_I, [_P, _P, _I, ctypes.POINTER(_I)]),
    "mm_set_tuning": (_I, [_P, _I, _I]),
    "mm_get_tuning": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mm_launch_count": (ctypes.c_longlong, [_P]),
    "mm_build_flags": (_I, []),
    "mm_sync": (_I, [_P]),
    "mm_selftest_wait_timeout": (_I, [_P, ctypes.c_uint]),
    "mm_last_error": (ctypes.c_char_p, [_P]),
    "mm_heff_noalloc": (_I, [ctypes.POINTER(_I), _D, _D, _D, _D, ctypes.POINTER(_D), _I, _P, _P,
                             ctypes.c_uint, _P]),
    "mm_noalloc_status": (_I, [_P]),
    "mm_fp32_probe": (_I, [_I, _I, _P, ctypes.POINTER(_D)]),
    "mm_tensor_eval": (_I, [_P, _I, _P]),
    "mm_noalloc_last_error": (ctypes.c_char_p, []),
    "mm_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), _D, _D, _D, _D, _D, _D, ctypes.POINTER(Opts)]),
    "mm_batch_destroy": (None, [_P]),
    "mm_batch_film": (_P, [_P, _I]),
    "mm_batch_step": (_I, [_P, _I, _D]),
    "mm_batch_run": (_I, [_P, _I, _D, _D, _I, ctypes.POINTER(_I)]),
    "mm_batch_max_dmdt": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "mm_batch_group_count": (_I, [_P]),
    "mm_batch_launch_count": (ctypes.c_longlong, [_P]),
    "mm_batch_last_error": (ctypes.c_char_p, [_P]),
    "mm_batch_set_schedule": (_I, [_P, _I]),
    "mm_batch_get_schedule": (_I, [_P]),
    "mm_batch_sync": (_I, [_P]),
    "mm_batch_selftest_wait_timeout": (_I, [_P, ctypes.c_uint]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -m paper_1501_07293_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a) -> int:
    """Raw address of a torch tensor (device or host) or a numpy array (host)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be C-contiguous float32")
        return a.ctypes.data
    if not a.is_contiguous() or str(a.dtype) != "torch.float32":
        raise ValueError("tensors must be contiguous float32")
    return a.data_ptr()


class Solver:
    """One film on one GPU: owns an mm_ctx."""

    def __init__(self, grid: Sequence[int], delta: float, Ms: float, A: float, Ku: float, alpha: float,
                 gamma: float, integrator: str = "rk4", self_term: bool = True, device=None, stream=None,
                 precision: str = "fp32", obs_every: int = 0, tune_cache: Optional[str] = None,
                 zform: str = "auto"):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.grid = tuple(int(g) for g in grid)
        self.N = self.grid[0] * self.grid[1] * self.grid[2]
        L = lib()
        o = Opts()
        L.mm_default_opts(ctypes.byref(o))
        o.integrator = MM_EULER if integrator == "euler" else MM_RK4
        o.self_term = 1 if self_term else 0
        o.precision = {"fp32": MM_FP32, "split_bf16": MM_SPLIT_BF16, "split_fp16": MM_SPLIT_FP16}[precision]
        o.obs_every = int(obs_every)
        # launch shapes an earlier autotune stored for this size (applied by mm_create)
        o.tune_cache = None if tune_cache is None else os.fsencode(tune_cache)
        o.zform = {"auto": MM_ZFORM_AUTO, "direct": MM_ZFORM_DIRECT}[zform]
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream() if stream is None else stream
            o.stream = s.cuda_stream
            self._stream = s
            ctx = _P()
            g = (_I * 3)(*self.grid)
            rc = L.mm_create(ctypes.byref(ctx), g, float(delta), float(Ms), float(A), float(Ku), float(alpha),
                             float(gamma), ctypes.byref(o))
            if rc != MM_OK:
                raise MMError(rc, L.mm_last_error(None).decode())
        self.ctx = ctx
        self._L = L
        self.precision = precision

    # -- helpers --------------------------------------------------------------
    def _check(self, rc: int):
        if rc != MM_OK:
            raise MMError(rc, self._L.mm_last_error(self.ctx).decode())

    def _vec_shape(self):
        nx, ny, nz = self.grid
        return (3, nz, ny, nx)

    def close(self):
        if getattr(self, "ctx", None):
            self._L.mm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- C ABI wrappers -----------------------------------------------------
    def padded_dims(self):
        p = (_I * 3)()
        self._check(self._L.mm_padded_dims(self.ctx, p))
        return tuple(p)

    def set_m(self, m):
        """m: (3, nz, ny, nx) float32, torch (device or host) or numpy (host)."""
        self._check(self._L.mm_set_m(self.ctx, _ptr(m)))

    def get_m(self, out=None):
        t = self.torch
        if out is None:
            out = t.empty(self._vec_shape(), dtype=t.float32, device=self.device)
        self._check(self._L.mm_get_m(self.ctx, _ptr(out)))
        return out

    def set_field(self, b_ext=(0.0, 0.0, 0.0), h_map=None, ku_map=None):
        b = (_D * 3)(*[float(v) for v in b_ext])
        self._keep = (h_map, ku_map)  # the library copies; keep host buffers alive until then
        self._check(self._L.mm_set_field(self.ctx, b, None if h_map is None else _ptr(h_map),
                                         None if ku_map is None else _ptr(ku_map)))

    def set_alpha(self, alpha: float):
        self._check(self._L.mm_set_alpha(self.ctx, float(alpha)))

    def set_program(self, segments):
        """Field program: iterable of (t_begin, t_end, b_begin[3], b_end[3], alpha); [] removes it."""
        segs = list(segments)
        arr = (Segment * max(1, len(segs)))()
        for i, (t0, t1, b0, b1, al) in enumerate(segs):
            arr[i].t_begin, arr[i].t_end, arr[i].alpha = float(t0), float(t1), float(al)
            for k in range(3):
                arr[i].b_begin[k], arr[i].b_end[k] = float(b0[k]), float(b1[k])
        self._check(self._L.mm_set_program(self.ctx, len(segs), arr))

    def set_time(self, t: float):
        self._check(self._L.mm_set_time(self.ctx, float(t)))

    def series(self, max_records: int = 65536) -> np.ndarray:
        """Observables records (obs_every > 0), oldest first: rows (t, step, <mx>, <my>, <mz>, max|dm/dt|)."""
        buf = np.zeros((max_records, 6), dtype=np.float64)
        n = _I(0)
        self._check(self._L.mm_get_series(self.ctx, buf.ctypes.data, int(max_records), ctypes.byref(n)))
        return buf[:n.value].copy()

    def set_tuning(self, yz_route: int = 0, zt_block: int = 0):
        """y/z launch shape: route 0 built-in / 1 fused / 2 split; z-product ky block (0 built-in)."""
        self._check(self._L.mm_set_tuning(self.ctx, int(yz_route), int(zt_block)))

    def tuning(self):
        """(route in effect: 1 fused / 2 split, ky block of the split pass)."""
        r, k = _I(0), _I(0)
        self._check(self._L.mm_get_tuning(self.ctx, ctypes.byref(r), ctypes.byref(k)))
        return r.value, k.value

    def time(self) -> float:
        """The context clock (s); synchronises."""
        v = _D(0.0)
        self._check(self._L.mm_get_time(self.ctx, ctypes.byref(v)))
        return v.value

    def heff(self, mask: int = TERM_ALL, out=None):
        t = self.torch
        if out is None:
            out = t.empty(self._vec_shape(), dtype=t.float32, device=self.device)
        self._check(self._L.mm_heff(self.ctx, _ptr(out), int(mask)))
        return out

    def step(self, n: int, dt: float):
        self._check(self._L.mm_step(self.ctx, int(n), float(dt)))

    def step_timed(self, n: int, dt: float) -> np.ndarray:
        """Eager, event-bracketed steps; device ms per kernel class [x-fwd, y/z, x-inv+LLG]."""
        ms = (_D * 3)(0.0, 0.0, 0.0)
        self._check(self._L.mm_step_timed(self.ctx, int(n), float(dt), ms))
        return np.array(ms[:])

    def adjoint(self, n: int, dt: float, ckpt_every: int, dL_dm_final, want=("m0", "h", "ku")):
        """mm_adjoint from the current state: returns dict of gradients (device tensors).

        On return the solver holds the final state of the n steps.
        """
        t = self.torch
        nx, ny, nz = self.grid
        out = {}
        gm0 = t.empty(self._vec_shape(), dtype=t.float32, device=self.device) if "m0" in want else None
        gh = t.empty(self._vec_shape(), dtype=t.float32, device=self.device) if "h" in want else None
        gk = t.empty((nz, ny, nx), dtype=t.float32, device=self.device) if "ku" in want else None
        self._check(self._L.mm_adjoint(self.ctx, int(n), float(dt), int(ckpt_every), _ptr(dL_dm_final),
                                       None if gh is None else _ptr(gh), None if gk is None else _ptr(gk),
                                       None if gm0 is None else _ptr(gm0)))
        for k, v in (("m0", gm0), ("h", gh), ("ku", gk)):
            if v is not None:
                out[k] = v
        return out

    def set_adjoint_memory(self, nbytes: float):
        """mm_set_adjoint_memory: bytes of recorded segments mm_adjoint's forward pass may keep."""
        self._check(self._L.mm_set_adjoint_memory(self.ctx, float(nbytes)))

    def energy(self) -> np.ndarray:
        e = (_D * 5)()
        self._check(self._L.mm_energy(self.ctx, e))
        return np.array(e[:])

    def observables(self) -> np.ndarray:
        o = (_D * 5)()
        self._check(self._L.mm_observables(self.ctx, o))
        return np.array(o[:])

    def launch_count(self) -> int:
        return int(self._L.mm_launch_count(self.ctx))

    def sync(self):
        self._check(self._L.mm_sync(self.ctx))

    def selftest_wait_timeout(self, polls: int = 1000):
        """Enqueue a kernel whose bounded wait runs out (see mm_selftest_wait_timeout)."""
        self._check(self._L.mm_selftest_wait_timeout(self.ctx, int(polls)))


def heff_noalloc(grid, delta, Ms, A, Ku, b_ext, m, H, mask: int = TERM_ALL, self_term: bool = True,
                 stream=None):
    """mm_heff_noalloc: effective field of the device state m into the device tensor H.

    No context and no device allocation (the library's static scratch array
    holds every intermediate).  m and H are float32 (3, nz, ny, nx) CUDA
    tensors; calls that overlap on the GPU race on the shared scratch.
    """
    import torch
    L = lib()
    g = (_I * 3)(*[int(v) for v in grid])
    b = (_D * 3)(*[float(v) for v in b_ext])
    s = torch.cuda.current_stream() if stream is None else stream
    rc = L.mm_heff_noalloc(g, float(delta), float(Ms), float(A), float(Ku), b, 1 if self_term else 0,
                           _ptr(m), _ptr(H), int(mask), s.cuda_stream)
    if rc != MM_OK:
        raise MMError(rc, L.mm_noalloc_last_error().decode())
    return H


def tensor_eval(offsets) -> np.ndarray:
    """mm_tensor_eval: the FP64 tensor (xx, yy, zz, xy, xz, yz) at integer offsets
    (an (n, 3) array of I, J, K), as the set-up kernel evaluates it."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    out = np.zeros((off.shape[0], 6), dtype=np.float64)
    rc = lib().mm_tensor_eval(off.ctypes.data, int(off.shape[0]), out.ctypes.data)
    if rc != MM_OK:
        raise MMError(rc, "mm_tensor_eval failed")
    return out


def fp32_probe_tflops(packed: bool, iters: int = 1 << 16, reps: int = 5):
    """Measured FP32 rate (TFLOP/s) of the mm_fp32_probe kernel on the current device:
    the best of `reps` CUDA-event-timed launches after one warm-up launch."""
    import torch
    L = lib()
    s = torch.cuda.current_stream()
    fl = _D()
    best = 0.0
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        rc = L.mm_fp32_probe(1 if packed else 0, int(iters), s.cuda_stream, ctypes.byref(fl))
        e1.record(s)
        if rc != MM_OK:
            raise MMError(rc, "mm_fp32_probe failed")
        torch.cuda.synchronize()
        if r:
            best = max(best, fl.value / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def noalloc_status(stream=None):
    """mm_noalloc_status: synchronise the stream and raise MMError if a kernel of an
    earlier heff_noalloc call on this device flagged a failure (flags are cleared)."""
    import torch
    L = lib()
    s = torch.cuda.current_stream() if stream is None else stream
    rc = L.mm_noalloc_status(s.cuda_stream)
    if rc != MM_OK:
        raise MMError(rc, L.mm_noalloc_last_error().decode())


def noalloc_selftest_wait_timeout(polls: int = 1000):
    """mm_selftest_wait_timeout(NULL, polls): a kernel on the legacy default stream
    whose bounded wait runs out and sets heff_noalloc's timeout flag."""
    rc = lib().mm_selftest_wait_timeout(None, int(polls))
    if rc != MM_OK:
        raise MMError(rc, lib().mm_noalloc_last_error().decode())


class _FilmView(Solver):
    """A film of a Batch: the single-film API on the batch-owned context (not destroyed here)."""

    def __init__(self, batch, index, ctx, grid):
        self.torch = batch.torch
        self.device = batch.device
        self.grid = tuple(grid)
        self.N = grid[0] * grid[1] * grid[2]
        self.ctx = ctx
        self._L = batch._L
        self._stream = batch._stream

    def close(self):
        self.ctx = None


class Batch:
    """Independent films of uneven size advanced together (mm_batch_*)."""

    def __init__(self, grids, delta, Ms, A, Ku, alpha, gamma, device=None, stream=None, precision: str = "fp32"):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.grids = [tuple(int(v) for v in g) for g in grids]
        L = lib()
        o = Opts()
        L.mm_default_opts(ctypes.byref(o))
        o.precision = {"fp32": MM_FP32, "split_bf16": MM_SPLIT_BF16, "split_fp16": MM_SPLIT_FP16}[precision]
        with torch.cuda.device(self.device):
            s = torch.cuda.current_stream() if stream is None else stream
            o.stream = s.cuda_stream
            self._stream = s
            flat = (_I * (3 * len(self.grids)))(*[v for g in self.grids for v in g])
            b = _P()
            rc = L.mm_batch_create(ctypes.byref(b), len(self.grids), flat, float(delta), float(Ms), float(A),
                                   float(Ku), float(alpha), float(gamma), ctypes.byref(o))
            if rc != MM_OK:
                raise MMError(rc, L.mm_batch_last_error(None).decode())
        self.b = b
        self._L = L
        self.films = [_FilmView(self, f, L.mm_batch_film(b, f), g) for f, g in enumerate(self.grids)]

    def _check(self, rc):
        if rc != MM_OK:
            raise MMError(rc, self._L.mm_batch_last_error(self.b).decode())

    def step(self, n: int, dt: float):
        self._check(self._L.mm_batch_step(self.b, int(n), float(dt)))

    def run(self, max_steps: int, dt: float, tol_dmdt: float, check_every: int = 100):
        out = (_I * len(self.grids))()
        self._check(self._L.mm_batch_run(self.b, int(max_steps), float(dt), float(tol_dmdt), int(check_every), out))
        return list(out)

    def max_dmdt(self):
        out = (ctypes.c_float * len(self.grids))()
        self._check(self._L.mm_batch_max_dmdt(self.b, out))
        return np.array(out[:], dtype=np.float64)

    def group_count(self) -> int:
        return int(self._L.mm_batch_group_count(self.b))

    def set_schedule(self, schedule: str):
        """'persistent' (one launch per step over every film) or 'grouped'."""
        self._check(self._L.mm_batch_set_schedule(self.b, 1 if schedule == "persistent" else 0))

    def schedule(self) -> str:
        return "persistent" if self._L.mm_batch_get_schedule(self.b) == 1 else "grouped"

    def sync(self):
        self._check(self._L.mm_batch_sync(self.b))

    def selftest_wait_timeout(self, polls: int = 1000):
        """One persistent launch whose dependency waits run out (mm_batch_selftest_wait_timeout)."""
        self._check(self._L.mm_batch_selftest_wait_timeout(self.b, int(polls)))

    def launch_count(self) -> int:
        return int(self._L.mm_batch_launch_count(self.b))

    def close(self):
        if getattr(self, "b", None):
            for f in self.films:
                f.close()
            self._L.mm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
