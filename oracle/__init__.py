"""CPU oracle for the TOP consensus-ADMM iteration.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its binding) imports, links or runs anything in this package; only the
tests, the smoke check and the CPU-baseline leg of the benchmark do.

  capi         ctypes wrapper around top_oracle.c: the literal serial FP64
               CADMM of the paper (Algorithm 1, Eq. 18-21), plus a long
               double build of the same source to bound its own rounding.
  centralized  numpy/scipy solutions of the whole (centralised) problem that
               the CADMM fixed point must equal: the pinned spline system,
               the single free polynomial, the dense KKT system and a
               brute-force active-set QP for tiny inputs.
"""
from .capi import build, solve, segment_cond, real_bytes, project_ball, numeric_local  # noqa: F401
