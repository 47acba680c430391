"""ctypes wrapper of top_oracle.c (test infrastructure only).

`solve(w)` runs the literal serial CADMM of the paper on a workload object
(any object with the attributes of `Workload`: seg_offset, waypoints,
durations, start_state, end_state, mode, inner, rho, eps, max_iters and the
optional constraint families) and returns numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "top_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {}
_LOCK = threading.Lock()

_VARIANTS = {
    "double": ("liboracle.so", []),
    "long double": ("liboracle_ld.so", ["-DOR_REAL=long double", "-DOR_LONG"]),
}


def build(force: bool = False) -> None:
    """Compile both precision variants of the oracle with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    for name, flags in _VARIANTS.values():
        out = os.path.join(_BUILD, name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               *flags, "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)


class _Problem(C.Structure):
    _fields_ = [
        ("B", C.c_int32), ("seg_offset", C.c_void_p), ("waypoints", C.c_void_p),
        ("durations", C.c_void_p), ("start_state", C.c_void_p), ("end_state", C.c_void_p),
        ("mode", C.c_int32), ("inner", C.c_int32), ("rho", C.c_double), ("eps", C.c_double),
        ("max_iters", C.c_int32),
        ("M_box", C.c_int32), ("vbox", C.c_void_p),
        ("M_ball", C.c_int32), ("ball_c", C.c_void_p), ("ball_r", C.c_void_p),
        ("M_vn", C.c_int32), ("vnorm", C.c_void_p),
        ("M_gen", C.c_int32), ("gen_vmax", C.c_void_p), ("gen_amax", C.c_void_p),
        ("lbfgs_tol", C.c_double), ("lbfgs_max_iters", C.c_int32), ("lbfgs_mem", C.c_int32),
        ("adaptive_rho", C.c_int32), ("rho_mu", C.c_double), ("rho_tau_incr", C.c_double),
        ("rho_tau_decr", C.c_double),
        ("M_poly", C.c_int32), ("F_poly", C.c_int32), ("poly_n", C.c_void_p), ("poly_h", C.c_void_p),
    ]


class _Result(C.Structure):
    _fields_ = [
        ("coeffs", C.c_void_p), ("cost", C.c_void_p), ("r_primal", C.c_void_p),
        ("r_dual", C.c_void_p), ("iters", C.c_void_p), ("status", C.c_void_p),
        ("history", C.c_void_p), ("z", C.c_void_p), ("u", C.c_void_p),
        ("s", C.c_void_p), ("v", C.c_void_p), ("phi_b", C.c_void_p), ("w_b", C.c_void_p),
        ("phi_v", C.c_void_p), ("w_v", C.c_void_p), ("y_gen", C.c_void_p),
        ("inner_iters", C.c_void_p), ("rho_hist", C.c_void_p), ("rho_final", C.c_void_p),
    ]


def build_variant(source_text: str, out_dir: str, flags=()) -> str:
    """Compile a modified copy of the oracle source (used by the tests that
    plant mistakes to show that the pins catch them); returns the .so path."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "variant.c")
    with open(src, "w") as f:
        f.write(source_text)
    out = os.path.join(out_dir, "libvariant.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", *flags, "-o", out, src, "-lm"],
                   check=True)
    return out


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _lib(real: str = "double"):
    with _LOCK:
        if real not in _LIBS:
            if real in _VARIANTS:
                build()
                path = os.path.join(_BUILD, _VARIANTS[real][0])
            else:
                path = real  # an explicit library path (planted-mistake variants)
            lib = C.CDLL(path)
            lib.oracle_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Result)]
            lib.oracle_solve.restype = C.c_int
            lib.oracle_segment_cond.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int,
                                                C.POINTER(C.c_double)]
            lib.oracle_segment_cond.restype = C.c_int
            lib.oracle_real_bytes.restype = C.c_int
            lib.oracle_project_ball.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
            lib.oracle_project_ball.restype = None
            lib.oracle_numeric_local.argtypes = [C.POINTER(_Problem), C.c_int, C.c_int,
                                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.oracle_numeric_local.restype = C.c_int
            _LIBS[real] = lib
        return _LIBS[real]


def real_bytes(real: str = "double") -> int:
    return int(_lib(real).oracle_real_bytes())


def _f64(x, shape=None):
    if x is None:
        return None
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _make_problem(w, keep, lbfgs_tol, lbfgs_max_iters, lbfgs_mem, max_iters=None):
    B = int(np.asarray(w.seg_offset).shape[0] - 1)
    S = int(np.asarray(w.seg_offset)[-1])
    arrs = {
        "seg_offset": np.ascontiguousarray(np.asarray(w.seg_offset, dtype=np.int32)),
        "waypoints": _f64(w.waypoints, (S + B, 3)),
        "durations": _f64(w.durations, (S,)),
        "start_state": _f64(w.start_state, (B, 4, 3)),
        "end_state": _f64(w.end_state, (B, 4, 3)),
        "vbox": _f64(getattr(w, "vbox", None)),
        "ball_c": _f64(getattr(w, "ball_c", None)),
        "ball_r": _f64(getattr(w, "ball_r", None)),
        "vnorm": _f64(getattr(w, "vnorm", None)),
        "gen_vmax": _f64(getattr(w, "gen_vmax", None)),
        "gen_amax": _f64(getattr(w, "gen_amax", None)),
        "poly_n": _f64(getattr(w, "poly_n", None)),
        "poly_h": _f64(getattr(w, "poly_h", None)),
    }
    keep.extend(a for a in arrs.values() if a is not None)
    pb = _Problem()
    pb.B = B
    for k, a in arrs.items():
        setattr(pb, k, _ptr(a))
    pb.mode = {"pin": 0, "free": 1}[w.mode]
    pb.inner = {"closed": 0, "numeric": 1}[getattr(w, "inner", "closed")]
    pb.rho = float(w.rho)
    pb.eps = float(getattr(w, "eps", 0.0))
    pb.max_iters = int(w.max_iters if max_iters is None else max_iters)
    pb.M_box = int(getattr(w, "M_box", 0) or 0)
    pb.M_ball = int(getattr(w, "M_ball", 0) or 0)
    pb.M_vn = int(getattr(w, "M_vn", 0) or 0)
    pb.M_gen = int(getattr(w, "M_gen", 0) or 0)
    pb.lbfgs_tol = float(lbfgs_tol)
    pb.lbfgs_max_iters = int(lbfgs_max_iters)
    pb.lbfgs_mem = int(lbfgs_mem)
    pb.adaptive_rho = int(bool(getattr(w, "adaptive_rho", False)))
    pb.rho_mu = float(getattr(w, "rho_mu", 10.0))
    pb.rho_tau_incr = float(getattr(w, "rho_tau_incr", 1.1))
    pb.rho_tau_decr = float(getattr(w, "rho_tau_decr", 1.1))
    pb.M_poly = int(getattr(w, "M_poly", 0) or 0)
    pb.F_poly = int(getattr(w, "F_poly", 0) or 0)
    return pb, B, S


def solve(w, *, real: str = "double", state: bool = False, history: bool = False,
          max_iters=None, lbfgs_tol: float = 1e-12, lbfgs_max_iters: int = 2000,
          lbfgs_mem: int = 8) -> dict:
    """Run the oracle CADMM on every trajectory of `w` (serially).

    Returns a dict with coeffs [S,3,8] (raw monomial basis in t - t_{i-1}),
    cost [B], r_primal [B], r_dual [B], iters [B], status [B]; with
    `history`, history [iters,B,2]; with `state`, z [S+B,3,7], u [S,42],
    s / v [S,6*M_box], phi_b / w_b [S,M_ball,3], phi_v / w_v [S,M_vn,3],
    y_gen [S,M_gen,2], inner_iters [S].
    """
    keep = []
    pb, B, S = _make_problem(w, keep, lbfgs_tol, lbfgs_max_iters, lbfgs_mem, max_iters)
    K = pb.max_iters
    out = {
        "coeffs": np.zeros((S, 3, 8)), "cost": np.zeros(B), "r_primal": np.zeros(B),
        "r_dual": np.zeros(B), "iters": np.zeros(B, np.int32), "status": np.zeros(B, np.int32),
    }
    res = _Result()
    for k in ("coeffs", "cost", "r_primal", "r_dual", "iters", "status"):
        setattr(res, k, _ptr(out[k]))
    if history:
        out["history"] = np.zeros((max(K, 1), B, 2))
        res.history = _ptr(out["history"])
        out["rho_hist"] = np.zeros((max(K, 1), B))
        res.rho_hist = _ptr(out["rho_hist"])
    out["rho_final"] = np.zeros(B)
    res.rho_final = _ptr(out["rho_final"])
    if state:
        Mb, Mq, Mv, Mg = pb.M_box, pb.M_ball, pb.M_vn, pb.M_gen
        out.update({
            "z": np.zeros((S + B, 3, 7)), "u": np.zeros((S, 42)),
            "s": np.zeros((S, 6 * Mb + pb.F_poly * pb.M_poly)), "v": np.zeros((S, 6 * Mb + pb.F_poly * pb.M_poly)),
            "phi_b": np.zeros((S, Mq, 3)), "w_b": np.zeros((S, Mq, 3)),
            "phi_v": np.zeros((S, Mv, 3)), "w_v": np.zeros((S, Mv, 3)),
            "y_gen": np.zeros((S, Mg, 2)), "inner_iters": np.zeros(S, np.int32),
        })
        for k in ("z", "u", "s", "v", "phi_b", "w_b", "phi_v", "w_v", "y_gen", "inner_iters"):
            setattr(res, k, _ptr(out[k]))
    rc = _lib(real).oracle_solve(C.byref(pb), C.byref(res))
    if rc != 0:
        raise RuntimeError(f"oracle_solve failed with code {rc}")
    if history:
        kmax = int(out["iters"].max()) if B else 0
        out["history"] = out["history"][:kmax]
        out["rho_hist"] = out["rho_hist"][:kmax]
    return out


def segment_cond(w, b: int, i: int, real: str = "double"):
    """(cond(K), cond(S K S)) of the local matrix of segment i of trajectory b."""
    keep = []
    pb, _, _ = _make_problem(w, keep, 1e-12, 1, 8)
    out = (C.c_double * 2)()
    rc = _lib(real).oracle_segment_cond(C.byref(pb), int(b), int(i), out)
    if rc != 0:
        raise RuntimeError("local matrix not positive definite")
    return float(out[0]), float(out[1])


def project_ball(q, o, rad, real: str = "double"):
    """The oracle's projection onto ||phi - o|| <= rad (o = None: centred at 0)."""
    qa = _f64(q, (3,))
    oa = None if o is None else _f64(o, (3,))
    out = np.zeros(3)
    _lib(real).oracle_project_ball(_ptr(qa), _ptr(oa), float(rad), _ptr(out))
    return out


def numeric_local(w, b: int, i: int, zt, u, y, lbfgs_tol: float = 1e-13,
                  lbfgs_max_iters: int = 5000, lbfgs_mem: int = 8, real: str = "double"):
    """One numerical local step of segment i of trajectory b; returns (c[24], iterations)."""
    keep = []
    pb, _, _ = _make_problem(w, keep, lbfgs_tol, lbfgs_max_iters, lbfgs_mem)
    zt = _f64(zt, (42,)); u = _f64(u, (42,)); y = _f64(y, (-1,))
    out = np.zeros(24)
    it = _lib(real).oracle_numeric_local(C.byref(pb), int(b), int(i), _ptr(zt), _ptr(u), _ptr(y), _ptr(out))
    if it < 0:
        raise RuntimeError("local matrix not positive definite")
    return out, int(it)
