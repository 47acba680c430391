"""GPU parity of residual-balancing rho (UpdateRho, Eq. 22) against the oracle.

On the FP64 path the per-trajectory rho sequence is decided by the same
comparisons of FP64 residual norms on both sides, so the final rho must be
identical and the coefficients within the FP64 tolerance.  On the FP32 path
the residual norms carry a few percent of cancellation error, so a decision
near the factor mu may go the other way.  There the tests take (a) the early
phase of PIN problems, where every decision has a wide margin, with the same
rho sequence required, and (b) FREE problems run to a tight tolerance, whose
optimum does not depend on the rho schedule.
"""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import T, TOL, compare, solver, to_np  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

EDGE_NS = [1, 0, 2, 3, 33, 31, 32, 64, 0, 5, 127, 1]


def _stream_solver(T, precision):
    key = ("stream", precision)
    from test_parity_gpu import _solvers
    if key not in _solvers:
        _solvers[key] = T.Solver(256, 200000, precision=precision, max_samples=16, schedule="stream")
    return _solvers[key]


def check_rho(g, o):
    assert np.array_equal(g["rho"], o["rho_final"]), (g["rho"], o["rho_final"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fixed_rho_is_reported(T, precision):
    w = W.tiny(seed=4, N=[3, 0, 9], mode="pin").with_(max_iters=20, rho=2.5)
    g = to_np(solver(T, precision).solve(w))
    assert np.all(g["rho"] == 2.5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rule_that_never_fires_equals_fixed_rho(T, precision):
    w = W.tiny(seed=12, N=EDGE_NS, mode="pin").with_(max_iters=60)
    a = to_np(solver(T, precision).solve(w))
    b = to_np(solver(T, precision).solve(w.with_(adaptive_rho=True, rho_mu=1e300)))
    for k in ("coeffs", "cost", "iters", "status"):
        assert np.array_equal(a[k], b[k]), k
    assert np.all(b["rho"] == w.rho)


@pytest.mark.parametrize("mode", ["pin", "free"])
def test_resident_fp64_edge_shapes(T, mode):
    w = W.tiny(seed=12, N=EDGE_NS, mode=mode).with_(max_iters=200, adaptive_rho=True)
    o = oracle.solve(w)
    assert (o["rho_final"] != w.rho).sum() >= 5, "rho must move on most trajectories"
    g = to_np(solver(T, "fp64").solve(w))
    compare(g, o, w, TOL["fp64"])
    check_rho(g, o)


def test_resident_fp64_batch_subset(T):
    w = W.batch(B=16, seed=3).with_(adaptive_rho=True)
    o = oracle.solve(w)
    g = to_np(solver(T, "fp64").solve(w))
    compare(g, o, w, TOL["fp64"])
    check_rho(g, o)


def test_resident_fp64_box_ball_velocity_families(T):
    w = W.corridor(N=64).with_(adaptive_rho=True)
    o = oracle.solve(w)
    g = to_np(solver(T, "fp64").solve(w))
    compare(g, o, w, TOL["fp64"])
    check_rho(g, o)
    v = W.tiny(seed=21, N=[6, 9], mode="free", step=3.0).with_(M_vn=8, vnorm=np.array([2.0, 2.5]),
                                                                max_iters=150, adaptive_rho=True)
    o = oracle.solve(v)
    g = to_np(solver(T, "fp64").solve(v))
    compare(g, o, v, TOL["fp64"])
    check_rho(g, o)


@pytest.mark.parametrize("mode", ["pin", "free"])
def test_streaming_fp64(T, mode):
    w = W.tiny(seed=12, N=EDGE_NS, mode=mode).with_(max_iters=200, adaptive_rho=True)
    o = oracle.solve(w)
    g = to_np(_stream_solver(T, "fp64").solve(w))
    compare(g, o, w, TOL["fp64"])
    check_rho(g, o)
    c = W.corridor(N=64).with_(adaptive_rho=True)
    o = oracle.solve(c)
    g = to_np(_stream_solver(T, "fp64").solve(c))
    compare(g, o, c, TOL["fp64"])
    check_rho(g, o)


def test_streaming_fp64_numerical_step(T):
    """20 iterations from rho = 100: rho falls at every iteration (r_d > mu r_p),
    so every iteration rebuilds the L-BFGS preconditioner G(rho)."""
    w = W.general(N=100, v_nom=3.0).with_(max_iters=20, rho=100.0, lbfgs_max_iters=2000, lbfgs_tol=1e-12,
                                          adaptive_rho=True)
    o = oracle.solve(w, state=True, lbfgs_tol=1e-12, lbfgs_max_iters=2000)
    assert (o["inner_iters"] > 0).sum() >= 3, "the bounds must be active somewhere"
    assert o["rho_final"][0] < 20.0
    g = to_np(solver(T, "fp64").solve(w))
    compare(g, o, w, TOL["fp64"])
    check_rho(g, o)


def test_stopping_rule_and_history_fp64(T):
    w = W.tiny(seed=1, N=[8, 5, 12], mode="free", T_range=(0.8, 1.6)).with_(eps=1e-3, max_iters=5000,
                                                                         adaptive_rho=True)
    o = oracle.solve(w, history=True)
    g = to_np(solver(T, "fp64").solve(w, history=True, check_every=7))  # ignored: every iteration
    compare(g, o, w, TOL["fp64"])
    check_rho(g, o)
    for b in range(w.B):
        kb = int(o["iters"][b])
        scale = np.abs(o["history"][:kb, b]).max(axis=0)
        assert np.all(np.abs(g["history"][:kb, b] - o["history"][:kb, b]) <= 1e-9 * scale)


@pytest.mark.parametrize("schedule", ["auto", "stream"])
@pytest.mark.parametrize("mode", ["pin", "free"])
def test_fp32_decisive_phase(T, schedule, mode):
    """The first 30 iterations of problems where every decision of Eq. 22 has
    a margin of at least 15% against mu (checked on the oracle's history),
    well above the FP32 error of the residual norms: the same rho sequence."""
    w = W.tiny(seed=19, N=[1, 0, 3, 33, 31, 32, 64, 0, 5, 127, 1], mode=mode).with_(
        max_iters=30, adaptive_rho=True)
    o = oracle.solve(w, history=True)
    rp, rd = o["history"][..., 0], o["history"][..., 1]
    with np.errstate(divide="ignore", invalid="ignore"):
        m = np.minimum(np.abs(np.log(rp / (10 * rd))), np.abs(np.log(rd / (10 * rp))))
    assert np.nanmin(m) > 0.15
    s = solver(T, "fp32") if schedule == "auto" else _stream_solver(T, "fp32")
    g = to_np(s.solve(w))
    compare(g, o, w, TOL["fp32"])
    check_rho(g, o)


@pytest.mark.parametrize("schedule", ["auto", "stream"])
def test_fp32_free_mode_reaches_the_optimum(T, schedule):
    """Run to a tight tolerance, FREE interior waypoints: the optimum (one
    polynomial through the two boundary states, P3) does not depend on the
    rho schedule, and the FP32 path reaches it within the FP32 tolerance."""
    from oracle import centralized as CZ
    w = W.tiny(seed=1, N=[8, 5, 12], mode="free", T_range=(0.8, 1.6)).with_(
        eps=3e-6, max_iters=20000, adaptive_rho=True)
    s = solver(T, "fp32") if schedule == "auto" else _stream_solver(T, "fp32")
    g = to_np(s.solve(w))
    assert np.all(g["rho"] != w.rho)  # (the FP32 residuals may stall above eps: no status check)
    for b in range(w.B):
        sub = w.subset([b])
        ref = CZ.free_polynomial(sub.durations, sub.start_state[0], sub.end_state[0])
        s0, s1 = w.seg_offset[b], w.seg_offset[b + 1]
        err = np.linalg.norm((g["coeffs"][s0:s1] - ref) * sub.durations[:, None, None] ** np.arange(8)) / \
            np.linalg.norm(ref * sub.durations[:, None, None] ** np.arange(8))
        assert err < TOL["fp32"], (b, err)


def test_host_memory_returns_rho(T):
    w = W.tiny(seed=5, N=[10, 3, 20], mode="pin").with_(max_iters=80, adaptive_rho=True)
    s = solver(T, "fp64")
    gd = to_np(s.solve(w))
    gh = s.solve_host(w)
    for k in ("coeffs", "cost", "iters", "status", "rho"):
        assert np.array_equal(gd[k], gh[k]), k


def test_gradient_rejects_adaptive_rho(T):
    s = solver(T, "fp64")
    w = W.tiny(seed=5, N=[4], mode="pin").with_(max_iters=5, adaptive_rho=True)
    with pytest.raises(T.TopError) as e:
        s.grad(w)
    assert e.value.code == T.TOP_E_NOTSUP


def test_bad_rule_parameters_are_rejected(T):
    s = solver(T, "fp64")
    w = W.tiny(seed=5, N=[4], mode="pin").with_(max_iters=5, adaptive_rho=True)
    for bad in ({"rho_mu": 0.5}, {"rho_tau_incr": 0.9}, {"rho_tau_decr": float("nan")}):
        with pytest.raises(T.TopError) as e:
            s.solve(w.with_(**bad))
        assert e.value.code == T.TOP_E_INVAL


def test_full_batch_adaptive_to_tolerance_sampled(T):
    """The 4096-trajectory FREE batch with residual balancing run to eps = 1e-4
    in FP32 (the benchmark's `full_adaptive` run), held at six sampled
    trajectories (three short, three long) to the FP64 oracle run on those
    trajectories alone.  Trajectories are independent (their rho, residual
    sums and stop decisions are per trajectory, summed in an order fixed by
    the trajectory's own segments), so each sample is the same problem in
    both.  Near the threshold FP32 and FP64 may stop a few checks apart: both
    must converge, within 25 % of each other's iteration count, to
    coefficients that agree to the accuracy the stopping rule allows (1e-2
    time-normalised; the converged FREE solutions are the same polynomial)."""
    w = W.batch(seed=0).with_(mode="free", eps=1e-4, max_iters=30000, adaptive_rho=True)
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision="fp32", max_samples=0)
    g = to_np(s.solve(w))
    s.close()
    Nb = np.diff(w.seg_offset)
    ids = [int(b) for b in np.where(Nb <= 40)[0][:3]] + [int(b) for b in np.where(Nb >= 400)[0][:2]] + \
        [int(b) for b in np.where((Nb >= 150) & (Nb < 250))[0][:1]]
    assert (g["status"] == 0).sum() >= 4090
    for b in ids:
        o = oracle.solve(w.subset([b]))
        assert int(o["status"][0]) == 0 and int(g["status"][b]) == 0, (b, o["status"], g["status"][b])
        gi, oi = int(g["iters"][b]), int(o["iters"][0])
        assert abs(gi - oi) <= 0.25 * oi, (b, gi, oi)
        s0, s1 = int(w.seg_offset[b]), int(w.seg_offset[b + 1])
        T_b = w.durations[s0:s1][:, None, None] ** np.arange(8)[None, None, :]
        a, r = g["coeffs"][s0:s1] * T_b, o["coeffs"] * T_b
        assert np.linalg.norm(a - r) <= 1e-2 * np.linalg.norm(r), (b, np.linalg.norm(a - r) / np.linalg.norm(r))
