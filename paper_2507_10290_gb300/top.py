"""ctypes binding of the C ABI in include/top.h (argument marshalling only).

The functions `top_create`, `top_solve`, `top_grad`, `top_destroy`,
`top_strerror` and `top_last_cuda_error` have the names and arguments of the
C entry points.  `Solver` wraps them for torch tensors: torch supplies the
device memory and the stream, every step of the iteration runs in the CUDA
library.  Importing this module loads libtop.so and raises ImportError if it
has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# TOP_CHECKED=1 in the environment selects the bounds-checked build
# (libtop_checked.so: index checks in every kernel, failures as TOP_E_BOUNDS)
CHECKED = os.environ.get("TOP_CHECKED", "0") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "libtop_checked.so" if CHECKED else "libtop.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "top.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the CUDA library is required; there is no CPU fallback)")
_lib = C.CDLL(LIB_PATH)


def _header_constants():
    vals = {}
    with open(HEADER_PATH) as f:
        for m in re.finditer(r"#define\s+(TOP_\w+)\s+(-?\d+)", f.read()):
            vals[m.group(1)] = int(m.group(2))
    return vals


_K = _header_constants()
TOP_OK = _K["TOP_OK"]
TOP_E_INVAL = _K["TOP_E_INVAL"]
TOP_E_NOMEM = _K["TOP_E_NOMEM"]
TOP_E_CUDA = _K["TOP_E_CUDA"]
TOP_E_TIMEOUT = _K["TOP_E_TIMEOUT"]
TOP_E_NOTSUP = _K["TOP_E_NOTSUP"]
TOP_E_STATE = _K["TOP_E_STATE"]
TOP_E_NUMERIC = _K["TOP_E_NUMERIC"]
TOP_E_LIMIT = _K["TOP_E_LIMIT"]
TOP_E_BOUNDS = _K["TOP_E_BOUNDS"]
TOP_NOALLOC_MAX_SEGMENTS = _K["TOP_NOALLOC_MAX_SEGMENTS"]
TOP_NOALLOC_MAX_BATCH = _K["TOP_NOALLOC_MAX_BATCH"]
TOP_API_VERSION = _K["TOP_API_VERSION"]
TOP_CONVERGED, TOP_NOT_CONVERGED, TOP_NONFINITE, TOP_STALLED = 0, 1, 2, 3
TOP_FP32, TOP_FP64 = 0, 1
TOP_PIN, TOP_FREE = 0, 1
TOP_CLOSED_FORM, TOP_NUMERIC = 0, 1
TOP_MEM_DEVICE, TOP_MEM_HOST = 0, 1
TOP_SCHED_AUTO, TOP_SCHED_RESIDENT, TOP_SCHED_STREAM = 0, 1, 2
TOP_NUMERIC_AUTO, TOP_NUMERIC_WARP, TOP_NUMERIC_THREAD = 0, 1, 2
TOP_GEMM_CUDA_CORES, TOP_GEMM_TENSOR = 0, 1
TOP_STREAM_FUSED, TOP_STREAM_PHASES = 0, 1


class top_config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_batch", C.c_int32), ("max_segments", C.c_int32),
                ("max_samples", C.c_int32), ("schedule", C.c_int32), ("segs_per_cta", C.c_int32),
                ("ckpt_interval", C.c_int32), ("numeric_form", C.c_int32), ("gemm_form", C.c_int32),
                ("stream_form", C.c_int32), ("reserved", C.c_int32 * 6)]


class top_problem(C.Structure):
    _fields_ = [("B", C.c_int32), ("memory", C.c_int32), ("seg_offset", C.c_void_p),
                ("waypoints", C.c_void_p), ("durations", C.c_void_p), ("start_state", C.c_void_p),
                ("end_state", C.c_void_p), ("mode", C.c_int32), ("inner", C.c_int32),
                ("rho", C.c_double), ("eps", C.c_double), ("max_iters", C.c_int32),
                ("check_every", C.c_int32),
                ("M_box", C.c_int32), ("vbox", C.c_void_p),
                ("M_ball", C.c_int32), ("ball_c", C.c_void_p), ("ball_r", C.c_void_p),
                ("M_vn", C.c_int32), ("vnorm", C.c_void_p),
                ("M_gen", C.c_int32), ("gen_vmax", C.c_void_p), ("gen_amax", C.c_void_p),
                ("lbfgs_mem", C.c_int32), ("lbfgs_max_iters", C.c_int32), ("lbfgs_tol", C.c_double),
                ("adaptive_rho", C.c_int32), ("rho_mu", C.c_double), ("rho_tau_incr", C.c_double),
                ("rho_tau_decr", C.c_double),
                ("M_poly", C.c_int32), ("F_poly", C.c_int32), ("poly_n", C.c_void_p), ("poly_h", C.c_void_p),
                ("stall_checks", C.c_int32)]


class top_result(C.Structure):
    _fields_ = [("coeffs", C.c_void_p), ("cost", C.c_void_p), ("r_primal", C.c_void_p),
                ("r_dual", C.c_void_p), ("iters", C.c_void_p), ("status", C.c_void_p),
                ("history", C.c_void_p), ("rho", C.c_void_p)]


class top_state(C.Structure):
    _fields_ = [("p", C.c_void_p), ("m", C.c_void_p), ("ybox", C.c_void_p), ("qball", C.c_void_p),
                ("qvn", C.c_void_p), ("iters", C.c_void_p)]


_lib.top_create.argtypes = [C.POINTER(top_config), C.POINTER(C.c_void_p)]
_lib.top_create.restype = C.c_int
_lib.top_solve.argtypes = [C.c_void_p, C.POINTER(top_problem), C.POINTER(top_result), C.c_void_p]
_lib.top_solve.restype = C.c_int
_lib.top_resume.argtypes = [C.c_void_p, C.POINTER(top_problem), C.POINTER(top_state), C.POINTER(top_result),
                            C.POINTER(top_state), C.c_void_p]
_lib.top_resume.restype = C.c_int
_lib.top_grad.argtypes = [C.c_void_p, C.POINTER(top_problem), C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_void_p]
_lib.top_grad.restype = C.c_int
_lib.top_launch_count.argtypes = [C.c_void_p]
_lib.top_launch_count.restype = C.c_int64
_lib.top_destroy.argtypes = [C.c_void_p]
_lib.top_destroy.restype = None
_lib.top_strerror.argtypes = [C.c_int]
_lib.top_strerror.restype = C.c_char_p
_lib.top_last_cuda_error.argtypes = [C.c_void_p]
_lib.top_last_cuda_error.restype = C.c_int
_lib.top_solve_noalloc.argtypes = [C.POINTER(top_problem), C.POINTER(top_result), C.c_int, C.c_void_p]
_lib.top_solve_noalloc.restype = C.c_int
_lib.top_sample.argtypes = [C.c_void_p, C.POINTER(top_problem), C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                            C.c_void_p]
_lib.top_sample.restype = C.c_int
_lib.top_time_alloc.argtypes = [C.c_void_p, C.POINTER(top_problem), C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                C.c_void_p, C.c_void_p]
_lib.top_time_alloc.restype = C.c_int
_lib.top_autotune.argtypes = [C.c_void_p, C.POINTER(top_problem), C.c_int32, C.POINTER(C.c_int32),
                              C.POINTER(C.c_float), C.c_int32, C.c_void_p]
_lib.top_autotune.restype = C.c_int
_lib.top_set_layout.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
_lib.top_set_layout.restype = C.c_int
_lib.top_sync.argtypes = [C.c_void_p, C.c_void_p]
_lib.top_sync.restype = C.c_int
_lib.top_set_profiling.argtypes = [C.c_void_p, C.c_int]
_lib.top_set_profiling.restype = C.c_int
_lib.top_kernel_times.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int]
_lib.top_kernel_times.restype = C.c_int


def top_create(cfg: top_config):
    """int top_create(const top_config*, top_handle**) -> (code, handle)"""
    h = C.c_void_p()
    rc = _lib.top_create(C.byref(cfg), C.byref(h))
    return rc, h


def top_solve(handle, problem: top_problem, result: top_result, stream: int = 0) -> int:
    return _lib.top_solve(handle, C.byref(problem), C.byref(result), C.c_void_p(stream))


def top_resume(handle, problem: top_problem, start, result: top_result, save, stream: int = 0) -> int:
    """int top_resume(h, pb, from, res, to, stream); start / save: top_state or None"""
    return _lib.top_resume(handle, C.byref(problem), None if start is None else C.byref(start), C.byref(result),
                           None if save is None else C.byref(save), C.c_void_p(stream))


def top_grad(handle, problem: top_problem, dJ: int, dwaypoints: int, ddurations: int, stream: int = 0) -> int:
    return _lib.top_grad(handle, C.byref(problem), C.c_void_p(dJ), C.c_void_p(dwaypoints),
                         C.c_void_p(ddurations), C.c_void_p(stream))


def top_destroy(handle) -> None:
    _lib.top_destroy(handle)


def top_strerror(code: int) -> str:
    return _lib.top_strerror(int(code)).decode()


def top_last_cuda_error(handle) -> int:
    return _lib.top_last_cuda_error(handle)


def top_solve_noalloc(problem: top_problem, result: top_result, precision: int, stream: int = 0) -> int:
    """int top_solve_noalloc(const top_problem*, top_result*, int precision, void* stream):
    the solve for callers that cannot allocate device memory (fixed scratch, no handle)."""
    return _lib.top_solve_noalloc(C.byref(problem), C.byref(result), int(precision), C.c_void_p(stream))


def top_sample(handle, problem: top_problem, coeffs: int, M: int, order: int, out: int, stream: int = 0) -> int:
    """int top_sample(top_handle*, const top_problem*, const double* coeffs, int M, int order, double* out,
    void* stream): trajectories sampled at M uniform times."""
    return _lib.top_sample(handle, C.byref(problem), C.c_void_p(coeffs), int(M), int(order), C.c_void_p(out),
                           C.c_void_p(stream))


def top_time_alloc(handle, problem: top_problem, k_T: float, lr: float, steps: int, durations_io: int,
                   result, stream: int = 0) -> int:
    """int top_time_alloc(top_handle*, const top_problem*, double k_T, double lr, int steps,
    double* durations_io, top_result* res, void* stream): outer time allocation."""
    return _lib.top_time_alloc(handle, C.byref(problem), float(k_T), float(lr), int(steps),
                               C.c_void_p(durations_io), None if result is None else C.byref(result),
                               C.c_void_p(stream))


def top_autotune(handle, problem: top_problem, iters: int, n_ms: int = 7, stream: int = 0):
    """int top_autotune(top_handle*, const top_problem*, int iters, int* out_segs_per_cta, float* ms, int n_ms,
    void* stream) -> (code, chosen segments per CTA, [ms per capacity 512, 448, ..., 128])."""
    out = C.c_int32(0)
    buf = (C.c_float * n_ms)()
    rc = _lib.top_autotune(handle, C.byref(problem), int(iters), C.byref(out), buf, int(n_ms), C.c_void_p(stream))
    return rc, int(out.value), [float(x) for x in buf]


def top_set_layout(handle, B: int, host_seg_offset) -> int:
    """int top_set_layout(top_handle*, int B, const int32_t* host_seg_offset): capture-safe mode
    (host_seg_offset: a contiguous int32 numpy array of B+1 entries, or None with B = 0)."""
    ptr = None if host_seg_offset is None else host_seg_offset.ctypes.data
    return _lib.top_set_layout(handle, int(B), C.c_void_p(ptr))


def top_sync(handle, stream: int = 0) -> int:
    """int top_sync(top_handle*, void* stream): error flag of the last capture-safe top_solve."""
    return _lib.top_sync(handle, C.c_void_p(stream))


def top_launch_count(handle) -> int:
    """int64_t top_launch_count(const top_handle*): kernels launched by top_solve so far."""
    return int(_lib.top_launch_count(handle))


def top_set_profiling(handle, enable: bool) -> int:
    return _lib.top_set_profiling(handle, int(bool(enable)))


def top_kernel_times(handle, n: int = 4):
    """(code, [ms...]) of the last top_solve's kernels: precompute, resident, streaming, cluster-resident."""
    buf = (C.c_float * n)()
    rc = _lib.top_kernel_times(handle, buf, n)
    return rc, [float(x) for x in buf]


class TopError(RuntimeError):
    def __init__(self, code: int, where: str, cuda: int = 0):
        msg = f"{where}: {top_strerror(code)} ({code})"
        if cuda:
            msg += f", cudaError {cuda}"
        super().__init__(msg)
        self.code = code


def _ptr(t):
    return None if t is None else t.data_ptr()


class Solver:
    """One handle of the library, sized for a batch capacity.

    precision: "fp32" (FP32 iteration, FP64 KKT inverses and cost) or "fp64".
    """

    def __init__(self, max_batch: int, max_segments: int, precision: str = "fp32", max_samples: int = 16,
                 schedule: str = "auto", segs_per_cta: int = 0, ckpt_interval: int = 10,
                 numeric_form: str = "auto", gemm_form: str = "cuda_cores", stream_form: str = "fused"):
        import torch  # device memory and streams only
        self.torch = torch
        cfg = top_config()
        cfg.precision = {"fp32": TOP_FP32, "fp64": TOP_FP64}[precision]
        cfg.max_batch = int(max_batch)
        cfg.max_segments = int(max(1, max_segments))
        cfg.max_samples = int(max_samples)
        cfg.schedule = {"auto": TOP_SCHED_AUTO, "resident": TOP_SCHED_RESIDENT, "stream": TOP_SCHED_STREAM}[schedule]
        cfg.segs_per_cta = int(segs_per_cta)
        cfg.ckpt_interval = int(ckpt_interval)
        cfg.numeric_form = {"auto": TOP_NUMERIC_AUTO, "warp": TOP_NUMERIC_WARP,
                            "thread": TOP_NUMERIC_THREAD}[numeric_form]
        cfg.gemm_form = {"cuda_cores": TOP_GEMM_CUDA_CORES, "tensor": TOP_GEMM_TENSOR}[gemm_form]
        cfg.stream_form = {"fused": TOP_STREAM_FUSED, "phases": TOP_STREAM_PHASES}[stream_form]
        self.precision = precision
        rc, h = top_create(cfg)
        if rc != TOP_OK:
            raise TopError(rc, "top_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            top_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- marshalling --------------------------------------------------------
    def device_inputs(self, w, device="cuda"):
        """Copy a Workload's arrays into device tensors (FP64, ABI layout)."""
        torch = self.torch

        def t(x, dtype=torch.float64):
            return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)

        return {
            "seg_offset": t(w.seg_offset, torch.int32), "waypoints": t(w.waypoints), "durations": t(w.durations),
            "start_state": t(w.start_state), "end_state": t(w.end_state),
            "vbox": t(getattr(w, "vbox", None)), "ball_c": t(getattr(w, "ball_c", None)),
            "ball_r": t(getattr(w, "ball_r", None)), "vnorm": t(getattr(w, "vnorm", None)),
            "gen_vmax": t(getattr(w, "gen_vmax", None)), "gen_amax": t(getattr(w, "gen_amax", None)),
            "poly_n": t(getattr(w, "poly_n", None)), "poly_h": t(getattr(w, "poly_h", None)),
        }

    def make_problem(self, w, tensors, memory=TOP_MEM_DEVICE, max_iters=None, eps=None, check_every=1,
                     stall_checks=0):
        pb = top_problem()
        pb.B = int(np.asarray(w.seg_offset).shape[0] - 1)
        pb.memory = memory
        for k in ("seg_offset", "waypoints", "durations", "start_state", "end_state", "vbox", "ball_c",
                  "ball_r", "vnorm", "gen_vmax", "gen_amax", "poly_n", "poly_h"):
            x = tensors.get(k)
            if x is None:
                setattr(pb, k, None)
            elif memory == TOP_MEM_DEVICE:
                setattr(pb, k, x.data_ptr())
            else:
                setattr(pb, k, x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr())
        pb.mode = {"pin": TOP_PIN, "free": TOP_FREE}[w.mode]
        pb.inner = {"closed": TOP_CLOSED_FORM, "numeric": TOP_NUMERIC}[getattr(w, "inner", "closed")]
        pb.rho = float(w.rho)
        pb.eps = float(w.eps if eps is None else eps)
        pb.max_iters = int(w.max_iters if max_iters is None else max_iters)
        pb.check_every = int(check_every)
        pb.M_box = int(getattr(w, "M_box", 0) or 0)
        pb.M_ball = int(getattr(w, "M_ball", 0) or 0)
        pb.M_vn = int(getattr(w, "M_vn", 0) or 0)
        pb.M_gen = int(getattr(w, "M_gen", 0) or 0)
        pb.lbfgs_mem = int(getattr(w, "lbfgs_mem", 0) or 0)
        pb.lbfgs_max_iters = int(getattr(w, "lbfgs_max_iters", 0) or 0)
        pb.lbfgs_tol = float(getattr(w, "lbfgs_tol", 0.0) or 0.0)
        pb.adaptive_rho = int(bool(getattr(w, "adaptive_rho", False)))
        pb.rho_mu = float(getattr(w, "rho_mu", 0.0) or 0.0)
        pb.rho_tau_incr = float(getattr(w, "rho_tau_incr", 0.0) or 0.0)
        pb.rho_tau_decr = float(getattr(w, "rho_tau_decr", 0.0) or 0.0)
        pb.M_poly = int(getattr(w, "M_poly", 0) or 0)
        pb.F_poly = int(getattr(w, "F_poly", 0) or 0)
        pb.stall_checks = int(stall_checks)
        return pb

    def alloc_result(self, B: int, S: int, max_iters: int = 0, history: bool = False, device="cuda"):
        torch = self.torch
        out = {
            "coeffs": torch.empty((S, 3, 8), dtype=torch.float64, device=device),
            "cost": torch.empty(B, dtype=torch.float64, device=device),
            "r_primal": torch.empty(B, dtype=torch.float64, device=device),
            "r_dual": torch.empty(B, dtype=torch.float64, device=device),
            "iters": torch.empty(B, dtype=torch.int32, device=device),
            "status": torch.empty(B, dtype=torch.int32, device=device),
            "rho": torch.empty(B, dtype=torch.float64, device=device),
        }
        if history:
            out["history"] = torch.full((max(1, max_iters), B, 2), float("nan"), dtype=torch.float64, device=device)
        return out

    @staticmethod
    def result_struct(out):
        r = top_result()
        for k in ("coeffs", "cost", "r_primal", "r_dual", "iters", "status", "history", "rho"):
            x = out.get(k)
            setattr(r, k, None if x is None else (x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()))
        return r

    def alloc_state(self, w, device="cuda"):
        """Buffers for an iteration state (top_state) of this workload's layout."""
        torch = self.torch
        B = int(np.asarray(w.seg_offset).shape[0] - 1)
        S = int(np.asarray(w.seg_offset)[-1])
        z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=device)  # noqa: E731
        st = {"p": z(S + B, 3, 7), "m": z(S + B, 3, 7), "iters": torch.zeros(B, dtype=torch.int32, device=device)}
        if getattr(w, "M_box", 0):
            st["ybox"] = z(S, 6 * w.M_box)
        if getattr(w, "M_ball", 0):
            st["qball"] = z(S, w.M_ball, 3)
        if getattr(w, "M_vn", 0):
            st["qvn"] = z(S, w.M_vn, 3)
        return st

    @staticmethod
    def state_struct(st):
        if st is None:
            return None
        x = top_state()
        for k in ("p", "m", "ybox", "qball", "qvn", "iters"):
            v = st.get(k)
            setattr(x, k, None if v is None else (v.ctypes.data if isinstance(v, np.ndarray) else v.data_ptr()))
        return x

    def resume(self, w, start=None, save=True, max_iters=None, eps=None, check_every: int = 1, stream=None,
               tensors=None, out=None, stall_checks: int = 0, history: bool = False):
        """top_resume: solve from the state `start` (None: Init) and return (outputs, saved state or None)."""
        torch = self.torch
        tensors = tensors if tensors is not None else self.device_inputs(w)
        K = int(w.max_iters if max_iters is None else max_iters)
        B = int(np.asarray(w.seg_offset).shape[0] - 1)
        S = int(np.asarray(w.seg_offset)[-1])
        out = out if out is not None else self.alloc_result(B, S, K, history)
        saved = self.alloc_state(w) if save else None
        pb = self.make_problem(w, tensors, TOP_MEM_DEVICE, max_iters=K, eps=eps, check_every=check_every,
                               stall_checks=stall_checks)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = top_resume(self.handle, pb, self.state_struct(start), self.result_struct(out), self.state_struct(saved), s)
        if rc != TOP_OK:
            raise TopError(rc, "top_resume", top_last_cuda_error(self.handle))
        return out, saved

    def solve(self, w, history: bool = False, max_iters=None, eps=None, check_every: int = 1, stream=None,
              tensors=None, out=None, stall_checks: int = 0):
        """Solve a Workload on the GPU; returns a dict of device tensors."""
        torch = self.torch
        tensors = tensors if tensors is not None else self.device_inputs(w)
        K = int(w.max_iters if max_iters is None else max_iters)
        B = int(np.asarray(w.seg_offset).shape[0] - 1)
        S = int(np.asarray(w.seg_offset)[-1])
        out = out if out is not None else self.alloc_result(B, S, K, history)
        pb = self.make_problem(w, tensors, TOP_MEM_DEVICE, max_iters=K, eps=eps, check_every=check_every,
                               stall_checks=stall_checks)
        r = self.result_struct(out)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = top_solve(self.handle, pb, r, s)
        if rc != TOP_OK:
            raise TopError(rc, "top_solve", top_last_cuda_error(self.handle))
        return out

    def grad(self, w, dJ=None, max_iters=None, tensors=None, stream=None):
        """d(sum_b dJ[b] J_b)/d(waypoints, durations) through max_iters unrolled iterations
        (top_grad); returns device tensors (dwaypoints [S+B,3], ddurations [S])."""
        torch = self.torch
        tensors = tensors if tensors is not None else self.device_inputs(w)
        B = int(np.asarray(w.seg_offset).shape[0] - 1)
        S = int(np.asarray(w.seg_offset)[-1])
        if dJ is None:
            dJ = torch.ones(B, dtype=torch.float64, device="cuda")
        dJ = torch.as_tensor(dJ, dtype=torch.float64, device="cuda").contiguous()
        dw = torch.empty((S + B, 3), dtype=torch.float64, device="cuda")
        dT = torch.empty(S, dtype=torch.float64, device="cuda")
        pb = self.make_problem(w, tensors, TOP_MEM_DEVICE, max_iters=max_iters, eps=0.0)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = top_grad(self.handle, pb, dJ.data_ptr(), dw.data_ptr(), dT.data_ptr(), s)
        if rc != TOP_OK:
            raise TopError(rc, "top_grad", top_last_cuda_error(self.handle))
        return dw, dT

    def autotune(self, w, iters: int = 20, tensors=None, stream=None, gemm=False):
        """top_autotune on this batch: returns (segments per CTA chosen, {capacity: ms}); with
        gemm=True also {"cuda_cores": ms, "tensor": ms} of the two gemm forms at that capacity
        (negative where the choice does not apply)."""
        torch = self.torch
        tensors = tensors if tensors is not None else self.device_inputs(w)
        pb = self.make_problem(w, tensors, TOP_MEM_DEVICE)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc, best, ms = top_autotune(self.handle, pb, iters, 9, s)
        if rc != TOP_OK:
            raise TopError(rc, "top_autotune", top_last_cuda_error(self.handle))
        caps = {512 - 64 * q: t for q, t in enumerate(ms[:7])}
        if gemm:
            return best, caps, {"cuda_cores": ms[7], "tensor": ms[8]}
        return best, caps

    def sample(self, w, coeffs, M: int, order: int = 0, tensors=None, stream=None):
        """Every trajectory of w with coefficients `coeffs` ([S,3,8] device tensor)
        sampled at M uniform times (top_sample); returns a [B, M, 3] device tensor."""
        torch = self.torch
        tensors = tensors if tensors is not None else self.device_inputs(w)
        B = int(np.asarray(w.seg_offset).shape[0] - 1)
        out = torch.empty((B, M, 3), dtype=torch.float64, device="cuda")
        pb = self.make_problem(w, tensors, TOP_MEM_DEVICE)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = top_sample(self.handle, pb, coeffs.contiguous().data_ptr(), M, order, out.data_ptr(), s)
        if rc != TOP_OK:
            raise TopError(rc, "top_sample", top_last_cuda_error(self.handle))
        return out

    def time_alloc(self, w, k_T: float, lr: float, steps: int, max_iters=None, tensors=None, stream=None,
                   result: bool = True):
        """Outer time allocation (top_time_alloc): returns (durations [S] device
        tensor, solve outputs with them or None)."""
        torch = self.torch
        tensors = tensors if tensors is not None else self.device_inputs(w)
        B = int(np.asarray(w.seg_offset).shape[0] - 1)
        S = int(np.asarray(w.seg_offset)[-1])
        K = int(w.max_iters if max_iters is None else max_iters)
        T = tensors["durations"].clone()
        out = self.alloc_result(B, S, K) if result else None
        pb = self.make_problem(w, tensors, TOP_MEM_DEVICE, max_iters=K, eps=0.0)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = top_time_alloc(self.handle, pb, k_T, lr, steps, T.data_ptr(),
                            self.result_struct(out) if result else None, s)
        if rc != TOP_OK:
            raise TopError(rc, "top_time_alloc", top_last_cuda_error(self.handle))
        return T, out

    def solve_host(self, w, history: bool = False, max_iters=None, eps=None, check_every: int = 1,
                   arrays=None, out=None, stream=None):
        """Solve with HOST buffers (numpy): the library stages the copies itself."""
        B = int(np.asarray(w.seg_offset).shape[0] - 1)
        S = int(np.asarray(w.seg_offset)[-1])
        K = int(w.max_iters if max_iters is None else max_iters)
        if arrays is None:
            arrays = {
                "seg_offset": np.ascontiguousarray(w.seg_offset, dtype=np.int32),
                "waypoints": np.ascontiguousarray(w.waypoints, dtype=np.float64),
                "durations": np.ascontiguousarray(w.durations, dtype=np.float64),
                "start_state": np.ascontiguousarray(w.start_state, dtype=np.float64),
                "end_state": np.ascontiguousarray(w.end_state, dtype=np.float64),
            }
            for k in ("vbox", "ball_c", "ball_r", "vnorm", "gen_vmax", "gen_amax", "poly_n", "poly_h"):
                x = getattr(w, k, None)
                arrays[k] = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        if out is None:
            out = {"coeffs": np.empty((S, 3, 8)), "cost": np.empty(B), "r_primal": np.empty(B),
                   "r_dual": np.empty(B), "iters": np.empty(B, np.int32), "status": np.empty(B, np.int32),
                   "rho": np.empty(B)}
            if history:
                out["history"] = np.full((max(1, K), B, 2), np.nan)
        pb = self.make_problem(w, arrays, TOP_MEM_HOST, max_iters=K, eps=eps, check_every=check_every)
        r = self.result_struct(out)
        s = stream if stream is not None else self.torch.cuda.current_stream().cuda_stream
        rc = top_solve(self.handle, pb, r, s)
        if rc != TOP_OK:
            raise TopError(rc, "top_solve", top_last_cuda_error(self.handle))
        return out
