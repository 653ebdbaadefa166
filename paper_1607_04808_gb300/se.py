"""Thin ctypes binding of libse.so (include/se.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory and the current stream.  There is no CPU
fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libse.so")

KERNELS = {"stokeslet": 0, "stresslet": 1, "rotlet": 2}
PRECS = {"fp32": 0, "fp64": 1}
STATUS = {
    0: "SE_OK", 1: "SE_ERR_INVALID_ARG", 2: "SE_ERR_OUT_OF_BOX", 3: "SE_ERR_COINCIDENT",
    4: "SE_ERR_OOM", 5: "SE_ERR_CUDA", 6: "SE_ERR_CUFFT", 7: "SE_ERR_TIMEOUT",
    8: "SE_ERR_NOT_SUPPORTED",
}
STAGES = ["bin", "spread", "fft", "scale", "ifft", "gather", "real_setup", "real"]
TEST_SKIP_TILE_COPY = 1  # se.h SE_TEST_SKIP_TILE_COPY
BACK_STAGES = ["adj_bin", "adj_fourier", "adj_gather", "adj_real", "bin", "fourier", "grad_gather", "grad_real"]
BATCH_STAGES = ["bin", "spread", "fft", "scale", "ifft", "gather", "real"]


class SEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class SEParams(ctypes.Structure):
    _fields_ = [
        ("xi", ctypes.c_double), ("rc", ctypes.c_double), ("M", ctypes.c_int), ("P", ctypes.c_int),
        ("deltaL_policy", ctypes.c_int), ("max_fft", ctypes.c_int), ("cell_width", ctypes.c_double),
        ("Mtilde", ctypes.c_int),
        ("Mg", ctypes.c_int), ("eta", ctypes.c_double), ("h", ctypes.c_double),
    ]


class SEPeaks(ctypes.Structure):
    _fields_ = [("fp32_fma_tflops", ctypes.c_double), ("fp32_ffma2_tflops", ctypes.c_double),
                ("fp64_fma_tflops", ctypes.c_double), ("sm_count", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libse.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_SO):
                raise RuntimeError(
                    f"{_SO} is missing: build it with paper_1607_04808_gb300._build.build() "
                    "(or __graft_entry__.build())")
            L = ctypes.CDLL(_SO)
            vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            L.se_plan_create.restype = i32
            L.se_plan_create.argtypes = [i32, i64, dbl, ctypes.POINTER(ctypes.c_double), dbl, i32,
                                         ctypes.POINTER(SEParams), ctypes.POINTER(vp)]
            L.se_plan_create_box.restype = i32
            L.se_plan_create_box.argtypes = [i32, i64, dbl, ctypes.POINTER(ctypes.c_double), dbl, i32,
                                             ctypes.POINTER(SEParams), ctypes.POINTER(vp)]
            L.se_plan_create_periodic.restype = i32
            L.se_plan_create_periodic.argtypes = [i32, i64, dbl, ctypes.POINTER(ctypes.c_double), dbl, i32,
                                                  ctypes.POINTER(SEParams), ctypes.POINTER(vp)]
            L.se_plan_get_grid.restype = i32
            L.se_plan_get_grid.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 4
            L.se_eval.restype = i32
            L.se_eval.argtypes = [vp, vp, vp, vp, vp, vp]
            L.se_eval_real_space.restype = i32
            L.se_eval_real_space.argtypes = [vp, vp, vp, vp, vp, vp]
            L.se_eval_targets.restype = i32
            L.se_eval_targets.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
            L.se_eval_host.restype = i32
            L.se_eval_host.argtypes = [vp, vp, vp, vp, vp, vp]
            L.se_eval_backward.restype = i32
            L.se_eval_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.se_eval_backward_q.restype = i32
            L.se_eval_backward_q.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.se_choose_params_points.restype = i32
            L.se_choose_params_points.argtypes = [i32, i32, i64, ctypes.POINTER(dbl), vp, dbl,
                                                  ctypes.POINTER(SEParams), ctypes.POINTER(SEParams)]
            L.se_choose_params.restype = i32
            L.se_choose_params.argtypes = [i32, i32, i64, dbl, dbl, dbl, ctypes.POINTER(SEParams),
                                           ctypes.POINTER(SEParams)]
            L.se_plan_get_params.restype = i32
            L.se_plan_get_params.argtypes = [vp, ctypes.POINTER(SEParams)]
            L.se_plan_check.restype = i32
            L.se_plan_check.argtypes = [vp]
            L.se_plan_set_timing.restype = i32
            L.se_plan_set_timing.argtypes = [vp, i32]
            L.se_plan_set_overlap.restype = i32
            L.se_plan_set_overlap.argtypes = [vp, i32]
            L.se_plan_set_keep_grid.restype = i32
            L.se_plan_set_keep_grid.argtypes = [vp, i32]
            L.se_plan_set_deterministic.restype = i32
            L.se_plan_set_deterministic.argtypes = [vp, i32]
            L.se_plan_set_test_flags.restype = i32
            L.se_plan_set_test_flags.argtypes = [vp, i32]
            L.se_plan_stage_times.restype = i32
            L.se_plan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32]
            L.se_plan_launch_count.restype = i64
            L.se_plan_launch_count.argtypes = [vp]
            L.se_set_precompute_cache.restype = i32
            L.se_set_precompute_cache.argtypes = [i32, ctypes.c_char_p]
            L.se_plan_precompute_info.restype = i32
            L.se_plan_precompute_info.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
            L.se_plan_destroy.restype = i32
            L.se_batch_create.restype = i32
            L.se_batch_create.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                          i32, dbl, i32, ctypes.POINTER(SEParams), ctypes.POINTER(vp)]
            L.se_batch_eval.restype = i32
            L.se_batch_eval.argtypes = [vp, vp, vp, vp, vp]
            L.se_batch_set_graph.restype = i32
            L.se_batch_set_graph.argtypes = [vp, i32]
            L.se_batch_set_timing.restype = i32
            L.se_batch_set_timing.argtypes = [vp, i32]
            L.se_batch_stage_times.restype = i32
            L.se_batch_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i32]
            L.se_batch_get_params.restype = i32
            L.se_batch_get_params.argtypes = [vp, i32, ctypes.POINTER(SEParams)]
            L.se_batch_check.restype = i32
            L.se_batch_check.argtypes = [vp]
            L.se_batch_launch_count.restype = i64
            L.se_batch_launch_count.argtypes = [vp]
            L.se_batch_destroy.restype = i32
            L.se_batch_destroy.argtypes = [vp]
            L.se_plan_destroy.argtypes = [vp]
            L.se_last_error.restype = ctypes.c_char_p
            L.se_last_error.argtypes = []
            L.se_version.restype = ctypes.c_char_p
            L.se_version.argtypes = []
            L.se_measure_peaks.restype = i32
            L.se_measure_peaks.argtypes = [ctypes.POINTER(SEPeaks)]
            _lib = L
    return _lib


def _check(code: int):
    if code != 0:
        raise SEError(code, lib().se_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A Spectral Ewald plan for N points in a box: box = (x0, y0, z0, L) for the
    cube [x0, x0+L) x [y0, y0+L) x [z0, z0+L) (se_plan_create), or
    (x0, y0, z0, Lx, Ly, Lz) for a rectangular box (se_plan_create_box).
    periodic=True: the triply periodic sums in the cube (x0, y0, z0, L)
    (se_plan_create_periodic)."""

    def __init__(self, kernel: str, N: int, box=(0.0, 0.0, 0.0, 1.0), *, xi: float = 0.0,
                 tol: float = 0.0, prec: str = "fp32", M: int = 0, P: int = 0, rc: float = 0.0,
                 deltaL_policy: int = 0, max_fft: int = 0, periodic: bool = False, cell_width: float = 0.0):
        self.kernel = kernel
        self.kid = KERNELS[kernel]
        self.N = int(N)
        self.prec = prec
        self.dtype = torch.float32 if prec == "fp32" else torch.float64
        self.box = tuple(float(b) for b in box)
        if len(self.box) not in (4, 6) or (periodic and len(self.box) != 4):
            raise ValueError("box: (x0, y0, z0, L) or (x0, y0, z0, Lx, Ly, Lz); periodic plans take a cube")
        self.periodic = bool(periodic)
        prm = SEParams(xi=float(xi), rc=float(rc), M=int(M), P=int(P),
                       deltaL_policy=int(deltaL_policy), max_fft=int(max_fft), cell_width=float(cell_width))
        boxa = (ctypes.c_double * len(self.box))(*self.box)
        if self.periodic:
            create = lib().se_plan_create_periodic
        else:
            create = lib().se_plan_create if len(self.box) == 4 else lib().se_plan_create_box
        h = ctypes.c_void_p()
        _check(create(self.kid, self.N, float(xi), boxa, float(tol), PRECS[prec],
                      ctypes.byref(prm), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def params(self) -> dict:
        p = SEParams()
        _check(lib().se_plan_get_params(self._h, ctypes.byref(p)))
        return {k: getattr(p, k) for k, _ in SEParams._fields_}

    @property
    def grid(self) -> dict:
        """Grid sizes per dimension (se_plan_get_grid): M, Mtilde, Mf, Mg."""
        arrs = [(ctypes.c_int * 3)() for _ in range(4)]
        _check(lib().se_plan_get_grid(self._h, *arrs))
        return {k: tuple(a) for k, a in zip(("M", "Mtilde", "Mf", "Mg"), arrs)}

    def _arg(self, t, name):
        if t is None:
            return None
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and t.shape == (self.N, 3)):
            raise ValueError(f"{name}: expected a contiguous CUDA tensor ({self.N}, 3) of {self.dtype}")
        return t

    def eval(self, x, f, q=None, out=None, stream=None, check=False):
        """u = sum_{n != m} K(x_m - x_n) . f_n (se_eval) on device tensors."""
        x, f, q = self._arg(x, "x"), self._arg(f, "f"), self._arg(q, "q")
        if out is None:
            out = torch.empty_like(x)
        self._arg(out, "out")
        _check(lib().se_eval(self._h, _ptr(x), _ptr(f), _ptr(q), _ptr(out), _stream(stream)))
        if check:
            self.check()
        return out

    def eval_targets(self, x, f, xt, q=None, out=None, stream=None):
        """u at separate target points xt (Nt, 3) from the plan's sources (se_eval_targets)."""
        x, f, q = self._arg(x, "x"), self._arg(f, "f"), self._arg(q, "q")
        if not (xt.is_cuda and xt.dtype == self.dtype and xt.is_contiguous() and xt.dim() == 2 and xt.shape[1] == 3):
            raise ValueError(f"xt: expected a contiguous CUDA tensor (Nt, 3) of {self.dtype}")
        if out is None:
            out = torch.empty_like(xt)
        _check(lib().se_eval_targets(self._h, _ptr(x), _ptr(f), _ptr(q), int(xt.shape[0]), _ptr(xt), _ptr(out),
                                     _stream(stream)))
        return out

    def eval_real_space(self, x, f, q=None, out=None, stream=None):
        """The screened real-space part u^R alone (se_eval_real_space)."""
        x, f, q = self._arg(x, "x"), self._arg(f, "f"), self._arg(q, "q")
        if out is None:
            out = torch.empty_like(x)
        self._arg(out, "out")
        _check(lib().se_eval_real_space(self._h, _ptr(x), _ptr(f), _ptr(q), _ptr(out), _stream(stream)))
        return out

    def eval_host(self, x: np.ndarray, f: np.ndarray, q: np.ndarray | None = None,
                  out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """se_eval_host: host arrays in, host array out (copies inside the call)."""
        dt = np.float32 if self.prec == "fp32" else np.float64

        def host(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                assert a.device.type == "cpu" and a.dtype == self.dtype and a.is_contiguous()
                return a
            a = np.ascontiguousarray(a, dtype=dt)
            assert a.shape == (self.N, 3)
            return a

        def p(a):
            if a is None:
                return None
            return ctypes.c_void_p(a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)

        x, f, q = host(x), host(f), host(q)
        if out is None:
            out = np.empty((self.N, 3), dtype=dt)
        _check(lib().se_eval_host(self._h, p(x), p(f), p(q), p(out), _stream(stream)))
        return out

    def backward(self, x, f, grad_u, want_f=True, want_x=True, stream=None, q=None, want_q=False):
        """Gradients of L = sum grad_u . u (se_eval_backward_q): (grad_f, grad_x), or
        (grad_f, grad_x, grad_q) when want_q (stresslet, which also needs q)."""
        x, f, grad_u = self._arg(x, "x"), self._arg(f, "f"), self._arg(grad_u, "grad_u")
        q = self._arg(q, "q")
        gf = torch.empty_like(x) if want_f else None
        gx = torch.empty_like(x) if want_x else None
        gq = torch.empty_like(x) if want_q else None
        _check(lib().se_eval_backward_q(self._h, _ptr(x), _ptr(f), _ptr(q), _ptr(grad_u), _ptr(gf),
                                        _ptr(gq), _ptr(gx), _stream(stream)))
        return (gf, gx, gq) if want_q else (gf, gx)

    def check(self):
        """se_plan_check: synchronise and raise on a device-side error."""
        _check(lib().se_plan_check(self._h))

    def set_timing(self, on: bool = True):
        _check(lib().se_plan_set_timing(self._h, 1 if on else 0))

    def set_overlap(self, on: bool = True):
        """se_plan_set_overlap: Fourier part and real-space sum on two streams (FP32)."""
        _check(lib().se_plan_set_overlap(self._h, 1 if on else 0))

    def set_keep_grid(self, on: bool = True):
        """se_plan_set_keep_grid: the backward reuses the last evaluation's grid
        when given the same x, f (, q) tensors (their contents unchanged)."""
        _check(lib().se_plan_set_keep_grid(self._h, 1 if on else 0))

    def set_deterministic(self, on: bool = True):
        """se_plan_set_deterministic: bit-identical results call after call
        (stable bin order, atomic-free spreading, full-list real-space sum)."""
        _check(lib().se_plan_set_deterministic(self._h, 1 if on else 0))

    def set_test_flags(self, flags: int):
        """se_plan_set_test_flags (tests of the failure path; 0 restores normal operation)."""
        _check(lib().se_plan_set_test_flags(self._h, int(flags)))

    def stage_times(self, backward: bool = False) -> dict:
        """se_plan_stage_times of the last timed call: se_eval's stages, or with
        backward=True those of se_eval_backward."""
        buf = (ctypes.c_float * 8)()
        n = lib().se_plan_stage_times(self._h, buf, 8)
        names = BACK_STAGES if backward else STAGES
        return {names[i]: buf[i] for i in range(n)}

    def precompute_info(self) -> tuple[float, bool]:
        """(milliseconds, from the cache) of the plan's precomputation."""
        ms, cached = ctypes.c_double(), ctypes.c_int()
        _check(lib().se_plan_precompute_info(self._h, ctypes.byref(ms), ctypes.byref(cached)))
        return ms.value, bool(cached.value)

    def launch_count(self) -> int:
        """se_plan_launch_count: kernels of this library launched by the last call."""
        return int(lib().se_plan_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().se_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent systems with several right-hand sides each (se_batch_create).

    sizes[s] points of system s in the cube boxes[s] = (x0, y0, z0, L); the
    points of all systems are concatenated in x (sumN, 3), the forces in
    f (sumN, n_rhs, 3).
    """

    def __init__(self, kernel: str, sizes, boxes=None, n_rhs: int = 1, *, tol: float = 0.0,
                 prec: str = "fp32", max_fft: int = 0, graph: bool = True):
        self.kernel = kernel
        self.sizes = [int(n) for n in sizes]
        self.S = len(self.sizes)
        self.R = int(n_rhs)
        self.N = sum(self.sizes)
        self.prec = prec
        self.dtype = torch.float32 if prec == "fp32" else torch.float64
        if boxes is None:
            boxes = [(0.0, 0.0, 0.0, 1.0)] * self.S
        flat = [float(v) for b in boxes for v in b]
        if len(flat) != 4 * self.S:
            raise ValueError("boxes: one (x0, y0, z0, L) per system")
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        ns = (ctypes.c_int64 * self.S)(*self.sizes)
        bx = (ctypes.c_double * (4 * self.S))(*flat)
        prm = SEParams(max_fft=int(max_fft))
        h = ctypes.c_void_p()
        _check(lib().se_batch_create(KERNELS[kernel], self.S, ns, bx, self.R, float(tol), PRECS[prec],
                                     ctypes.byref(prm), ctypes.byref(h)))
        self._h = h
        _check(lib().se_batch_set_graph(self._h, 1 if graph else 0))

    def params(self, s: int) -> dict:
        p = SEParams()
        _check(lib().se_batch_get_params(self._h, int(s), ctypes.byref(p)))
        return {k: getattr(p, k) for k, _ in SEParams._fields_}

    def eval(self, x, f, out=None, stream=None, check=False):
        """u for every system and right-hand side (se_batch_eval)."""
        if not (x.is_cuda and x.dtype == self.dtype and x.is_contiguous() and x.shape == (self.N, 3)):
            raise ValueError(f"x: expected a contiguous CUDA tensor ({self.N}, 3) of {self.dtype}")
        shp = (self.N, self.R, 3)
        if not (f.is_cuda and f.dtype == self.dtype and f.is_contiguous() and tuple(f.shape) == shp):
            raise ValueError(f"f: expected a contiguous CUDA tensor {shp} of {self.dtype}")
        if out is None:
            out = torch.empty_like(f)
        _check(lib().se_batch_eval(self._h, _ptr(x), _ptr(f), _ptr(out), _stream(stream)))
        if check:
            self.check()
        return out

    def check(self):
        _check(lib().se_batch_check(self._h))

    def launch_count(self) -> int:
        return int(lib().se_batch_launch_count(self._h))

    def set_timing(self, on: bool) -> None:
        """se_batch_set_timing: stage timing of the following evaluations (no graph while on)."""
        _check(lib().se_batch_set_timing(self._h, 1 if on else 0))

    def stage_times(self) -> dict:
        """se_batch_stage_times of the last timed evaluation."""
        buf = (ctypes.c_float * 7)()
        n = lib().se_batch_stage_times(self._h, buf, 7)
        return {BATCH_STAGES[i]: buf[i] for i in range(n)}

    def close(self):
        if getattr(self, "_h", None):
            lib().se_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SEFunction(torch.autograd.Function):
    """u = SE(x, f[, q]) with gradients for x, f and q through se_eval_backward_q."""

    @staticmethod
    def forward(ctx, x, f, q, plan: Plan):
        ctx.plan = plan
        ctx.has_q = q is not None
        ctx.save_for_backward(x, f, q) if q is not None else ctx.save_for_backward(x, f)
        return plan.eval(x.contiguous(), f.contiguous(), None if q is None else q.contiguous())

    @staticmethod
    def backward(ctx, grad_u):
        if ctx.has_q:
            x, f, q = ctx.saved_tensors
            gf, gx, gq = ctx.plan.backward(x, f, grad_u.contiguous(), want_f=ctx.needs_input_grad[1],
                                           want_x=ctx.needs_input_grad[0], q=q,
                                           want_q=ctx.needs_input_grad[2])
            return gx, gf, gq, None
        x, f = ctx.saved_tensors
        gf, gx = ctx.plan.backward(x, f, grad_u.contiguous(), want_f=ctx.needs_input_grad[1],
                                   want_x=ctx.needs_input_grad[0])
        return gx, gf, None, None


def se_sum(x, f, plan: Plan, q=None):
    """Differentiable u = sum K(x_m - x_n) f_n (stresslet: T(x_m - x_n) f_n q_n)."""
    return SEFunction.apply(x, f, q, plan)


def set_precompute_cache(memory: bool = True, directory: str | None = None):
    """se_set_precompute_cache: share precomputed kernels between plans with equal grids."""
    _check(lib().se_set_precompute_cache(1 if memory else 0,
                                         None if directory is None else str(directory).encode()))


def choose_params(kernel: str, N: int, L: float = 1.0, tol: float = 0.0, prec: str = "fp32",
                  xi: float = 0.0, **overrides) -> dict:
    """Parameters the library would choose (se_choose_params; host only, no GPU needed)."""
    pin = SEParams(**{k: v for k, v in overrides.items()})
    pout = SEParams()
    _check(lib().se_choose_params(KERNELS[kernel], PRECS[prec], int(N), float(L), float(tol), float(xi),
                                  ctypes.byref(pin), ctypes.byref(pout)))
    return {k: getattr(pout, k) for k in ("xi", "rc", "M", "P", "deltaL_policy", "max_fft")}


def choose_params_points(kernel: str, x, box=(0.0, 0.0, 0.0, 1.0), tol: float = 0.0, prec: str = "fp32",
                         **overrides) -> dict:
    """Parameters for these points (se_choose_params_points; host only): x is an
    (N, 3) array or CPU tensor, box (x0, y0, z0, L) or (x0, y0, z0, Lx, Ly, Lz)."""
    import numpy as np
    xa = np.ascontiguousarray(np.asarray(x.cpu() if hasattr(x, "cpu") else x),
                              dtype=np.float32 if prec == "fp32" else np.float64)
    if xa.ndim != 2 or xa.shape[1] != 3:
        raise ValueError("x must be (N, 3)")
    b = tuple(float(v) for v in box)
    if len(b) == 4:
        b = b + (b[3], b[3])
    boxa = (ctypes.c_double * 6)(*b)
    pin = SEParams(**{k: v for k, v in overrides.items()})
    pout = SEParams()
    _check(lib().se_choose_params_points(KERNELS[kernel], PRECS[prec], xa.shape[0], boxa,
                                         xa.ctypes.data_as(ctypes.c_void_p), float(tol), ctypes.byref(pin),
                                         ctypes.byref(pout)))
    return {k: getattr(pout, k) for k in ("xi", "rc", "M", "P", "deltaL_policy", "max_fft", "cell_width")}


def version() -> str:
    return lib().se_version().decode()


def measure_peaks() -> dict:
    """Measured FP32 (scalar and paired) and FP64 FMA rates of the current device
    in TFLOP/s, and its SM count (se_measure_peaks)."""
    out = SEPeaks()
    _check(lib().se_measure_peaks(ctypes.byref(out)))
    return {"fp32_fma_tflops": out.fp32_fma_tflops, "fp32_ffma2_tflops": out.fp32_ffma2_tflops,
            "fp64_fma_tflops": out.fp64_fma_tflops, "sm_count": out.sm_count}
