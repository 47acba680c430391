"""One speed bound ||v(t_ij)|| <= v_max through both constraint paths of the
paper: the projection of Eq. 14 / 18f-g (closed-form local step) and the
numerical step of Eq. 15-17 (L-BFGS local step), on the same synthetic
instance (the comparison of Table III).  Each path is held to the oracle at
a fixed iteration count with the bound active on several segments; the
timing comparison itself is a line of `bench.py --suite`."""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import T, TOL, compare, solver, to_np  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("inner", ["closed", "numeric"])
def test_each_path_against_the_oracle(T, precision, inner):
    # a bound at 0.8 x the median chord speed acts on several segments in the
    # first iterations while every local L-BFGS solve still reaches its tolerance
    g0 = W.speed_limit(seed=3, N=32, M=8)
    chord = np.linalg.norm(np.diff(g0.waypoints, axis=0), axis=1) / g0.durations
    w = W.speed_limit(seed=3, N=32, M=8, inner=inner, max_iters=40, vmax=0.8 * float(np.median(chord)))
    kw = dict(lbfgs_tol=1e-12, lbfgs_max_iters=5000) if inner == "numeric" else {}
    w = w.with_(lbfgs_tol=1e-12 if precision == "fp64" else 1e-6, lbfgs_max_iters=5000) if inner == "numeric" else w
    o = oracle.solve(w, state=inner == "numeric", **kw)
    if inner == "numeric":
        assert (o["inner_iters"] > 0).sum() >= 3, "the bound must be active on several segments"
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision,form", [("fp32", "thread"), ("fp64", "thread"), ("fp32", "warp")])
def test_numerical_step_in_the_other_form(T, precision, form):
    """The thread-per-segment form of the numerical step (TOP_NUMERIC_THREAD;
    the default is one warp per segment) in both precisions, and the warp form
    named explicitly, held to the oracle like the default form."""
    from test_parity_gpu import _solvers
    key = ("numeric-form", precision, form)
    if key not in _solvers:
        _solvers[key] = T.Solver(64, 4096, precision=precision, max_samples=16, numeric_form=form)
    g0 = W.speed_limit(seed=3, N=32, M=8)
    chord = np.linalg.norm(np.diff(g0.waypoints, axis=0), axis=1) / g0.durations
    w = W.speed_limit(seed=3, N=32, M=8, inner="numeric", max_iters=40, vmax=0.8 * float(np.median(chord)))
    w = w.with_(lbfgs_tol=1e-12 if precision == "fp64" else 1e-6, lbfgs_max_iters=5000)
    o = oracle.solve(w, state=True, lbfgs_tol=1e-12, lbfgs_max_iters=5000)
    assert (o["inner_iters"] > 0).sum() >= 3
    g = to_np(_solvers[key].solve(w))
    compare(g, o, w, TOL[precision])
