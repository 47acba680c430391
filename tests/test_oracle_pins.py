"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle (top_oracle.c through oracle.capi) against
something other than itself: exact closed forms, the centralised optimum
that the CADMM fixed point must equal (Sec. III-D.2: the CADMM solution
space contains the optimum and ADMM converges to it), projections'
defining properties, KKT certificates built from independent numpy
matrices, and a long double re-run for the oracle's own rounding.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import centralized as CZ
from paper_2507_10290_gb300 import workloads as W

GOLDEN = __file__.rsplit("/", 1)[0] + "/golden/rest_to_rest_min_snap.txt"


def scaled_relerr(c, ref, T):
    """||c - ref|| / ||ref|| on time-normalised coefficients c_k T_i^k."""
    sc = np.asarray(T)[:, None, None] ** np.arange(8)[None, None, :]
    return float(np.linalg.norm((c - ref) * sc) / np.linalg.norm(ref * sc))


def read_golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *rest = line.split()
        vals[key] = rest
    return vals


# ---------------------------------------------------------------- P1 ----

def test_golden_rest_to_rest_closed_form_exact():
    """The golden smootherstep polynomial meets the 8 rest boundary conditions
    and its snap integral / speed ratio are the stated exact constants."""
    g = read_golden()
    s = [Fraction(int(x)) for x in g["coeffs"]]

    def deriv(poly, r):
        out = list(poly)
        for _ in range(r):
            out = [k * out[k] for k in range(1, len(out))]
        return out

    def ev(poly, t):
        return sum(ck * t ** k for k, ck in enumerate(poly))

    for r in range(4):
        assert ev(deriv(s, r), Fraction(0)) == (0 if r else 0)
        assert ev(deriv(s, r), Fraction(1)) == (1 if r == 0 else 0)
    snap = deriv(s, 4)
    sq = [Fraction(0)] * (2 * len(snap) - 1)
    for i, a in enumerate(snap):
        for j, b in enumerate(snap):
            sq[i + j] += a * b
    integral = sum(ck / (k + 1) for k, ck in enumerate(sq))
    assert integral == Fraction(int(g["snap_integral"][0]))
    vel = deriv(s, 1)
    assert ev(vel, Fraction(1, 2)) / 1 == Fraction(g["peak_to_mean_speed"][0])
    # s'(tau) = 140 tau^3 (1 - tau)^3 >= 0: the peak is at tau = 1/2
    assert vel == [0, 0, 0, 140, -420, 420, -140]


@pytest.mark.parametrize("mode", ["pin", "free"])
def test_p1_single_segment_matches_closed_form(mode):
    g = read_golden()
    s = np.array([float(x) for x in g["coeffs"]])
    rng = np.random.default_rng(7)
    for _ in range(3):
        P = rng.uniform(-5, 5, size=(2, 3))
        T = rng.uniform(0.6, 1.8)
        w = W.tiny(N=1, mode=mode).with_(
            waypoints=P, durations=np.array([T]),
            start_state=np.concatenate([P[None, :1], np.zeros((1, 3, 3))], axis=1),
            end_state=np.concatenate([P[None, 1:], np.zeros((1, 3, 3))], axis=1),
            rho=1e5 / T ** 7, max_iters=500)
        r = oracle.solve(w)
        d = P[1] - P[0]
        ref = np.zeros((1, 3, 8))
        for a in range(3):
            ref[0, a] = d[a] * s / T ** np.arange(8)
            ref[0, a, 0] += P[0, a]
        assert scaled_relerr(r["coeffs"], ref, [T]) < 1e-11
        J_ref = float(g["snap_integral"][0]) * float(d @ d) / T ** 7
        assert abs(r["cost"][0] - J_ref) <= 1e-10 * J_ref


# ----------------------------------------------------- centralised aids ----

def test_centralized_solvers_agree_and_meet_conditions():
    w = W.tiny(seed=3, N=6, mode="pin", T_range=(0.5, 1.5))
    P, T, s0, s1 = w.waypoints, w.durations, w.start_state[0], w.end_state[0]
    c = CZ.pin_spline(P, T, s0, s1)
    # interpolation, boundary orders 0..3 and C^6 continuity
    for a in range(3):
        for r in range(4):
            assert abs(c[0, a] @ CZ.deriv_row(r, 0) - s0[r, a]) < 1e-9
            assert abs(c[-1, a] @ CZ.deriv_row(r, T[-1]) - s1[r, a]) < 1e-9
        for j in range(1, len(T)):
            assert abs(c[j, a] @ CZ.deriv_row(0, 0) - P[j, a]) < 1e-9
            for r in range(7):
                left = c[j - 1, a] @ CZ.deriv_row(r, T[j - 1])
                right = c[j, a] @ CZ.deriv_row(r, 0)
                assert abs(left - right) < 1e-7 * max(1, abs(left))
    kk, _ = CZ.kkt_qp(P, T, s0, s1, "pin")
    assert scaled_relerr(kk, c, T) < 1e-7
    f = CZ.free_polynomial(T, s0, s1)
    kk, _ = CZ.kkt_qp(P, T, s0, s1, "free")
    assert scaled_relerr(kk, f, T) < 1e-7
    # single segment: both equal the closed-form smootherstep
    g = read_golden()
    sm = np.array([float(x) for x in g["coeffs"]])
    d = P[-1] - P[0]
    for sol in (CZ.pin_spline(P[[0, -1]], T[:1], s0, s1), CZ.free_polynomial(T[:1], s0, s1)):
        ref = np.zeros((1, 3, 8))
        for a in range(3):
            ref[0, a] = d[a] * sm / T[0] ** np.arange(8)
            ref[0, a, 0] += P[0, a]
        assert scaled_relerr(sol, ref, T[:1]) < 1e-12


# ---------------------------------------------------------------- P2/P3 --

def test_p2_pin_mode_converges_to_spline():
    w = W.tiny(seed=1, N=2, mode="pin", T_range=(0.8, 1.6)).with_(rho=1.0, max_iters=300000)
    r = oracle.solve(w)
    ref = CZ.pin_spline(w.waypoints, w.durations, w.start_state[0], w.end_state[0])
    assert scaled_relerr(r["coeffs"], ref, w.durations) < 1e-6


def test_p3_free_mode_converges_to_single_polynomial():
    w = W.tiny(seed=1, N=8, mode="free", T_range=(0.8, 1.6)).with_(rho=1.0, max_iters=20000)
    r = oracle.solve(w)
    ref = CZ.free_polynomial(w.durations, w.start_state[0], w.end_state[0])
    assert scaled_relerr(r["coeffs"], ref, w.durations) < 1e-10
    J = CZ.segment_cost(ref, w.durations)
    assert abs(r["cost"][0] - J) < 1e-9 * J


# ---------------------------------------------------------------- P5/P6 --

def _box_instance():
    """Tiny FREE instance whose box limit is 80% of the unconstrained peak axis speed."""
    w = W.tiny(seed=5, N=3, mode="free", T_range=(0.9, 1.3), step=2.0)
    free = CZ.free_polynomial(w.durations, w.start_state[0], w.end_state[0])
    M = 2
    peak = max(abs(free[i, a] @ CZ.deriv_row(1, (j + 1) * w.durations[i] / M))
               for i in range(3) for a in range(3) for j in range(M))
    return w.with_(M_box=M, vbox=np.array([0.8 * peak]), rho=10.0, max_iters=100000)


def test_p5_box_constrained_matches_active_set_qp():
    w = _box_instance()
    P, T = w.waypoints, w.durations
    c_ref, act = CZ.active_set_qp(P, T, w.start_state[0], w.end_state[0], "free", w.M_box,
                                  float(w.vbox[0]))
    assert c_ref is not None and len(act) > 0, "the instance must have active box rows"
    r = oracle.solve(w)
    assert scaled_relerr(r["coeffs"], c_ref, T) < 1e-6


def test_p6_kkt_certificate_of_converged_box_problem():
    w = _box_instance()
    r = oracle.solve(w, state=True)
    T, rho, M = w.durations, w.rho, w.M_box
    N = len(T)
    c = r["coeffs"]
    scale = 0.0
    for i in range(N):
        Mt = np.zeros((42, 24))
        E = np.ones(42)
        for a in range(3):
            for side in range(2):
                for rr in range(7):
                    row = a * 14 + side * 7 + rr
                    Mt[row, a * 8:(a + 1) * 8] = CZ.deriv_row(rr, T[i] if side else 0.0)
                    if (side == 0 and i == 0 or side == 1 and i == N - 1) and rr >= 4:
                        E[row] = 0
        Ao, b = [], []
        for j in range(1, M + 1):
            for a in range(3):
                for sg in (1.0, -1.0):
                    row = np.zeros(24)
                    row[a * 8:(a + 1) * 8] = sg * CZ.deriv_row(1, j * T[i] / M)
                    Ao.append(row); b.append(float(w.vbox[0]))
        Ao, b = np.array(Ao), np.array(b)
        Qt = np.zeros((24, 24))
        for a in range(3):
            Qt[a * 8:(a + 1) * 8, a * 8:(a + 1) * 8] = CZ.snap_gram(T[i])
        ci = c[i].reshape(24)
        mu = rho * r["v"][i]
        stat = 2 * Qt @ ci + rho * Mt.T @ (E * r["u"][i]) + Ao.T @ mu
        scale = max(scale, float(np.abs(2 * Qt @ ci).max()))
        assert np.abs(stat).max() < 1e-6 * scale
        assert mu.min() > -1e-9 * scale                       # dual feasibility
        assert (Ao @ ci - b).max() < 1e-7                     # primal feasibility
        assert np.abs(mu * (Ao @ ci - b)).max() < 1e-6 * scale  # complementarity
    # consensus stationarity: the two sides' multipliers cancel at free rows
    u = r["u"]
    for j in range(1, N):
        for a in range(3):
            end = u[j - 1, a * 14 + 7: a * 14 + 14]
            start = u[j, a * 14: a * 14 + 7]
            assert np.abs(end + start).max() < 1e-9 * max(1, np.abs(end).max())


# ---------------------------------------------------------------- P7 ----

def test_p7_ball_projection_properties():
    rng = np.random.default_rng(11)
    for _ in range(200):
        o = rng.normal(size=3) if rng.random() < 0.7 else None
        rad = rng.uniform(0.2, 3.0)
        q1, q2 = rng.normal(scale=3.0, size=(2, 3))
        p1 = oracle.project_ball(q1, o, rad)
        p2 = oracle.project_ball(q2, o, rad)
        oc = np.zeros(3) if o is None else o
        assert np.linalg.norm(p1 - oc) <= rad * (1 + 1e-12)                 # feasible
        assert np.allclose(oracle.project_ball(p1, o, rad), p1, atol=1e-12)  # idempotent
        assert np.linalg.norm(p1 - p2) <= np.linalg.norm(q1 - q2) + 1e-12   # non-expansive
        if np.linalg.norm(q1 - oc) <= rad:
            assert np.allclose(p1, q1, atol=0)                              # identity inside
        # brute force: no sampled feasible point is closer to q1
        dirs = rng.normal(size=(2000, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        pts = oc + dirs * rad * rng.uniform(0, 1, size=(2000, 1)) ** (1 / 3)
        pts = np.vstack([pts, oc + dirs * rad])
        assert np.linalg.norm(p1 - q1) <= np.linalg.norm(pts - q1, axis=1).min() + 1e-12


# ---------------------------------------------------------------- P8 ----

def test_p8_dual_invariants():
    w = W.tiny(seed=2, N=5, mode="free", T_range=(0.6, 1.4)).with_(max_iters=37)
    r1 = oracle.solve(w, state=True)
    r2 = oracle.solve(w.with_(max_iters=38), state=True)
    T = w.durations
    for j in range(1, 5):
        for a in range(3):
            for rr in range(7):
                e, s = a * 14 + 7 + rr, a * 14 + rr
                # free rows: u_end + u_start = 0 after every iteration
                assert abs(r2["u"][j - 1, e] + r2["u"][j, s]) < 1e-9 * max(1, abs(r2["u"][j - 1, e]))
                # the end-side increment is half the junction gap (Eq. 18b, 18c)
                left = r2["coeffs"][j - 1, a] @ CZ.deriv_row(rr, T[j - 1])
                right = r2["coeffs"][j, a] @ CZ.deriv_row(rr, 0.0)
                inc = r2["u"][j - 1, e] - r1["u"][j - 1, e]
                assert abs(inc - 0.5 * (left - right)) < 1e-8 * max(1, abs(left), abs(right))


def test_pin_rows_and_ends_fixed():
    w = W.tiny(seed=4, N=4, mode="pin").with_(max_iters=25)
    r = oracle.solve(w, state=True)
    z = r["z"]
    assert np.allclose(z[:, :, 0], w.waypoints, atol=0)
    assert np.allclose(z[0, :, :4], w.start_state[0].T, atol=0)
    assert np.allclose(z[-1, :, :4], w.end_state[0].T, atol=0)
    assert np.all(z[0, :, 4:] == 0) and np.all(z[-1, :, 4:] == 0)


# ---------------------------------------------------------------- P9 ----

def test_p9_long_double_rerun_bounds_rounding():
    assert oracle.real_bytes("double") == 8 and oracle.real_bytes("long double") >= 10
    for w in (W.single_box(), W.corridor(N=16).with_(max_iters=100)):
        rd = oracle.solve(w)
        rl = oracle.solve(w, real="long double")
        err = scaled_relerr(rd["coeffs"], rl["coeffs"], w.durations)
        assert err < 1e-11, err
        assert abs(rd["cost"][0] - rl["cost"][0]) < 1e-11 * abs(rl["cost"][0])
    # Jacobi equilibration is what keeps it small
    w = W.corridor(N=16)
    raw, eq = oracle.segment_cond(w, 0, 3)
    assert raw > 1e4 * eq and eq < 1e4


# ---------------------------------------------------- numerical step ----

def test_numeric_step_with_inactive_bounds_equals_closed_form():
    w = W.tiny(seed=8, N=6, mode="pin").with_(max_iters=60)
    rc = oracle.solve(w)
    wn = w.with_(inner="numeric", M_gen=8, gen_vmax=np.array([1e6]), gen_amax=np.array([1e6]))
    rn = oracle.solve(wn, state=True)
    assert scaled_relerr(rn["coeffs"], rc["coeffs"], w.durations) < 1e-12
    assert np.all(rn["y_gen"] == 0)


def _numpy_F(c, T, first, last, zt, u, y, rho, M, vmax, amax):
    """F of Eq. 16 for one segment, from independent numpy matrices."""
    Mt = np.zeros((42, 24))
    E = np.ones(42)
    for a in range(3):
        for side in range(2):
            for rr in range(7):
                row = a * 14 + side * 7 + rr
                Mt[row, a * 8:(a + 1) * 8] = CZ.deriv_row(rr, T if side else 0.0)
                if (side == 0 and first or side == 1 and last) and rr >= 4:
                    E[row] = 0
    G = CZ.snap_gram(T)
    F = sum(c[a * 8:(a + 1) * 8] @ G @ c[a * 8:(a + 1) * 8] for a in range(3))
    res = E * (Mt @ c - zt + u)
    F += rho / 2 * res @ res
    for j in range(M):
        t = (j + 1) * T / M
        for order, gmax, yy in ((1, vmax, y[j, 0]), (2, amax, y[j, 1])):
            vec = np.array([c[a * 8:(a + 1) * 8] @ CZ.deriv_row(order, t) for a in range(3)])
            h = vec @ vec - gmax ** 2
            g = max(0.0, h) ** 2
            F += rho / 2 * g * g + yy * g
    return F


def test_numeric_local_step_is_stationary_point():
    """With active norm bounds, the L-BFGS result is a minimiser of an independently
    coded F: central differences of F vanish there and F is lower than nearby."""
    w = W.tiny(seed=9, N=3, mode="pin", step=6.0, T_range=(0.8, 1.0)).with_(
        inner="numeric", M_gen=6, gen_vmax=np.array([4.0]), gen_amax=np.array([8.0]), rho=1e4)
    rng = np.random.default_rng(0)
    i = 1
    T = w.durations[i]
    # consensus target: the boundary derivatives of the pinned spline (fast: |v| > 4)
    spl = CZ.pin_spline(w.waypoints, w.durations, w.start_state[0], w.end_state[0])
    zt = np.zeros(42)
    for a in range(3):
        for rr in range(7):
            zt[a * 14 + rr] = spl[i, a] @ CZ.deriv_row(rr, 0.0)
            zt[a * 14 + 7 + rr] = spl[i, a] @ CZ.deriv_row(rr, T)
    u = rng.normal(scale=0.01, size=42)
    y = np.abs(rng.normal(size=(6, 2)))
    c, it = oracle.numeric_local(w, 0, i, zt, u, y)
    assert it > 0
    args = (T, False, False, zt, u, y, 1e4, 6, 4.0, 8.0)
    # the bounds are active at the minimiser
    vel = [np.linalg.norm([c[a * 8:(a + 1) * 8] @ CZ.deriv_row(1, (j + 1) * T / 6) for a in range(3)])
           for j in range(6)]
    assert max(vel) > 4.0
    F0 = _numpy_F(c, *args)
    # scale each coordinate by the curvature of the quadratic part
    Hd = np.array([max(1e-12, (_numpy_F(c + e, *args) + _numpy_F(c - e, *args) - 2 * F0))
                   for e in np.eye(24) * 1e-3]) / 1e-6
    h = 1e-4 / np.sqrt(Hd)
    grad = np.array([(_numpy_F(c + h[k] * np.eye(24)[k], *args) - _numpy_F(c - h[k] * np.eye(24)[k], *args))
                     / (2 * h[k]) for k in range(24)])
    gscaled = np.abs(grad / np.sqrt(Hd))
    c_q = oracle.numeric_local(w.with_(gen_vmax=np.array([1e6]), gen_amax=np.array([1e6])), 0, i, zt, u, y)[0]
    assert _numpy_F(c_q, *args) > F0   # the constraint terms moved the minimiser
    assert gscaled.max() < 1e-5 * max(1.0, math.sqrt(abs(F0)))
    for _ in range(50):
        d = rng.normal(size=24) * h * 10
        assert _numpy_F(c + d, *args) >= F0 - 1e-9 * abs(F0)


def test_numeric_duals_nondecreasing():
    w = W.tiny(seed=9, N=4, mode="pin", step=4.0, T_range=(0.8, 1.0)).with_(
        inner="numeric", M_gen=4, gen_vmax=np.array([4.0]), gen_amax=np.array([8.0]), max_iters=5,
        rho=1e4)
    r5 = oracle.solve(w, state=True)
    r6 = oracle.solve(w.with_(max_iters=6), state=True)
    assert np.all(r5["y_gen"] >= 0) and r5["y_gen"].max() > 0
    assert np.all(r6["y_gen"] >= r5["y_gen"])


# ---------------------------------------------------------- stopping ----

def test_stopping_rule_and_history():
    w = W.tiny(seed=1, N=8, mode="free", T_range=(0.8, 1.6)).with_(eps=1e-3, max_iters=5000)
    r = oracle.solve(w, history=True)
    k = int(r["iters"][0])
    h = r["history"][:, 0]
    N = 8
    assert r["status"][0] == 0 and 0 < k < 5000
    assert h[k - 1, 0] < N * 1e-3 and h[k - 1, 1] < N * 1e-3
    assert not (h[: k - 1, 0] < N * 1e-3).__and__(h[: k - 1, 1] < N * 1e-3).any()
    assert r["r_primal"][0] == h[k - 1, 0] and r["r_dual"][0] == h[k - 1, 1]


def test_batch_is_per_trajectory_and_handles_empty():
    a = W.tiny(seed=6, N=[3, 0, 5, 1], mode="pin").with_(max_iters=40)
    r = oracle.solve(a)
    assert r["cost"][1] == 0 and r["iters"][1] == 0
    for b in (0, 2, 3):
        rb = oracle.solve(a.subset([b]))
        s0, s1 = a.seg_offset[b], a.seg_offset[b + 1]
        assert np.array_equal(rb["coeffs"], r["coeffs"][s0:s1])
        assert rb["cost"][0] == r["cost"][b]


# ------------------------------------------------- adaptive rho (Eq. 22) --

def _consensus_rows(T, first, last):
    """M~ (42 x 24) and the end mask E of one segment, rows (a, side, r)."""
    Mt = np.zeros((42, 24))
    E = np.ones(42)
    for a in range(3):
        for side in range(2):
            for rr in range(7):
                row = a * 14 + side * 7 + rr
                Mt[row, a * 8:(a + 1) * 8] = CZ.deriv_row(rr, T if side else 0.0)
                if ((side == 0 and first) or (side == 1 and last)) and rr >= 4:
                    E[row] = 0
    return Mt, E


def test_adaptive_rho_never_triggered_equals_fixed_rho():
    w = W.tiny(seed=2, N=[5, 9], mode="pin").with_(max_iters=80)
    r0 = oracle.solve(w)
    r1 = oracle.solve(w.with_(adaptive_rho=True, rho_mu=1e300))
    assert np.array_equal(r0["coeffs"], r1["coeffs"]) and np.array_equal(r0["cost"], r1["cost"])


def adaptive_rule_violations(lib=None):
    """Count of iterations whose next rho breaks Eq. 22 (mu = 10, tau = 1.1),
    and the numbers of increases and decreases of rho seen, over a run that
    starts at rho = 1 (r_d dominates) and one at rho = 1e-3 (r_p dominates)."""
    bad, up, down = 0, 0, 0
    for rho0 in (1.0, 1e-3):
        w = W.tiny(seed=3, N=[12], mode="pin").with_(max_iters=400, adaptive_rho=True, rho=rho0)
        r = oracle.solve(w, history=True, **({} if lib is None else {"real": lib}))
        rho, h = r["rho_hist"][:, 0], r["history"][:, 0]
        bad += rho[0] != rho0
        for k in range(len(rho) - 1):
            rp, rd = h[k]
            expect = rho[k] * 1.1 if rp > 10 * rd else (rho[k] / 1.1 if rd > 10 * rp else rho[k])
            bad += abs(rho[k + 1] - expect) > 1e-14 * expect
            up += rho[k + 1] > rho[k]
            down += rho[k + 1] < rho[k]
    return bad, up, down


def test_adaptive_rho_follows_the_update_rule():
    """rho_{k+1} = 1.1 rho_k if r_p > 10 r_d, rho_k / 1.1 if r_d > 10 r_p, else rho_k (Eq. 22)."""
    bad, up, down = adaptive_rule_violations()
    assert bad == 0 and up > 10 and down > 10


def test_adaptive_rho_reaches_the_same_fixed_point():
    """The schedule of rho changes the path, not the limit: FREE mode still ends
    at the single polynomial (P3).  On small PIN instances the rule settles at
    rho ~ 0.027, where plain ADMM is slow, so PIN-like behaviour is pinned by the
    box-KKT certificate below instead."""
    w = W.tiny(seed=1, N=8, mode="free", T_range=(0.8, 1.6)).with_(max_iters=30000, adaptive_rho=True)
    r = oracle.solve(w)
    assert r["rho_final"][0] != 1.0
    ref = CZ.free_polynomial(w.durations, w.start_state[0], w.end_state[0])
    assert scaled_relerr(r["coeffs"], ref, w.durations) < 1e-8


def adaptive_kkt_error(lib=None):
    """Stationarity of the converged box problem with the final rho and the
    final scaled duals (y = rho u, mu = rho v), relative to |2 Qt c|."""
    w = _box_instance().with_(adaptive_rho=True, max_iters=100000, rho=10.0)
    r = oracle.solve(w, state=True, **({} if lib is None else {"real": lib}))
    rho = r["rho_final"][0]
    T, M = w.durations, w.M_box
    N = len(T)
    worst = 0.0
    for i in range(N):
        Mt, E = _consensus_rows(T[i], i == 0, i == N - 1)
        Ao = []
        for j in range(1, M + 1):
            for a in range(3):
                for sg in (1.0, -1.0):
                    row = np.zeros(24)
                    row[a * 8:(a + 1) * 8] = sg * CZ.deriv_row(1, j * T[i] / M)
                    Ao.append(row)
        Ao = np.array(Ao)
        Qt = np.zeros((24, 24))
        for a in range(3):
            Qt[a * 8:(a + 1) * 8, a * 8:(a + 1) * 8] = CZ.snap_gram(T[i])
        ci = r["coeffs"][i].reshape(24)
        stat = 2 * Qt @ ci + rho * Mt.T @ (E * r["u"][i]) + Ao.T @ (rho * r["v"][i])
        worst = max(worst, np.abs(stat).max() / np.abs(2 * Qt @ ci).max())
    return worst, rho


def test_adaptive_rho_keeps_box_kkt_certificate():
    err, rho = adaptive_kkt_error()
    assert rho != 10.0 and err < 1e-5


def adaptive_dual_continuity_error(lib=None):
    """Across a change of rho the unscaled consensus dual y = rho u follows
    y+ = y + rho_k E (M~ c+ - z+) exactly (Eq. 18c in unscaled form), however the
    scaled copy is stored.  Returns the largest relative violation over the
    first few changes of rho in a box-constrained FREE run."""
    w = _box_instance().with_(adaptive_rho=True)
    kw = {} if lib is None else {"real": lib}
    hist = oracle.solve(w.with_(max_iters=200), history=True, **kw)["rho_hist"][:, 0]
    changes = [k for k in range(1, len(hist)) if hist[k] != hist[k - 1]][:4]
    if not changes:
        return np.inf
    worst = 0.0
    N = len(w.durations)
    for m1 in changes:           # rho changed after iteration m1 - 1 (0-based)
        a = oracle.solve(w.with_(max_iters=m1 - 1), state=True, **kw)
        b = oracle.solve(w.with_(max_iters=m1), state=True, **kw)
        rho_a, rho_b = a["rho_final"][0], b["rho_final"][0]
        for i in range(N):
            Mt, E = _consensus_rows(w.durations[i], i == 0, i == N - 1)
            zt = np.concatenate([b["z"][i][ax].tolist() + b["z"][i + 1][ax].tolist() for ax in range(3)])
            y_next = rho_a * (a["u"][i] + E * (Mt @ b["coeffs"][i].reshape(24) - zt))
            err = np.abs(rho_b * b["u"][i] - y_next).max() / max(np.abs(y_next).max(), 1e-30)
            worst = max(worst, err)
    return worst


def test_adaptive_rho_unscaled_dual_is_continuous():
    assert adaptive_dual_continuity_error() < 1e-12


# ------------------------------------------- polytope corridors (Eq. 8-10) --

def _polytope_instance():
    """Tiny FREE instance inside tight polytopes (F=6 faces, M=4 samples):
    two rows are active at the optimum; rho = 10 converges to 1e-9."""
    w0 = W.tiny(seed=5, N=3, mode="free", T_range=(0.9, 1.3), step=2.0)
    return W.with_polytopes(w0, F=6, M=4, seed=1, margin=(0.05, 0.2)).with_(max_iters=200000, eps=1e-9, rho=10.0)


def polytope_kkt_errors(lib=None):
    """KKT conditions of the sampled-polytope QP at the converged oracle state,
    with every matrix rebuilt here from the basis: stationarity with
    lambda = rho u and mu = rho v, dual feasibility mu >= 0, primal feasibility,
    complementarity (each relative to |2 Qt c|), and the number of active rows."""
    w = _polytope_instance()
    r = oracle.solve(w, state=True, **({} if lib is None else {"real": lib}))
    rho = w.rho
    T, M, F = w.durations, w.M_poly, w.F_poly
    N = len(T)
    worst = {"stat": 0.0, "dual": 0.0, "primal": 0.0, "compl": 0.0}
    active = 0
    for i in range(N):
        Mt, E = _consensus_rows(T[i], i == 0, i == N - 1)
        A, h = [], []
        for j in range(1, M + 1):
            beta = CZ.deriv_row(0, j * T[i] / M)
            for f in range(F):
                A.append(np.kron(w.poly_n[i, f], beta))
                h.append(w.poly_h[i, f])
        A, h = np.array(A), np.array(h)
        Qt = np.zeros((24, 24))
        for a in range(3):
            Qt[a * 8:(a + 1) * 8, a * 8:(a + 1) * 8] = CZ.snap_gram(T[i])
        ci = r["coeffs"][i].reshape(24)
        mu = rho * r["v"][i]
        scale = np.abs(2 * Qt @ ci).max()
        stat = 2 * Qt @ ci + rho * Mt.T @ (E * r["u"][i]) + A.T @ mu
        worst["stat"] = max(worst["stat"], np.abs(stat).max() / scale)
        worst["dual"] = max(worst["dual"], max(0.0, -mu.min()) / scale)
        worst["primal"] = max(worst["primal"], max(0.0, (A @ ci - h).max()))
        worst["compl"] = max(worst["compl"], np.abs(mu * (A @ ci - h)).max() / scale)
        active += int((mu > 1e-6 * scale).sum())
    return worst, active, r


def test_polytope_kkt_certificate():
    worst, active, r = polytope_kkt_errors()
    assert r["status"][0] == 0
    assert active >= 2, "the polytopes must bind"
    assert worst["stat"] < 1e-6 and worst["dual"] < 1e-9 and worst["primal"] < 1e-7 and worst["compl"] < 1e-6, worst


def _rotation(seed):
    Qm, Rm = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    Qm = Qm * np.sign(np.diag(Rm))[None, :]
    return Qm * np.sign(np.linalg.det(Qm))


def polytope_rotation_error(lib=None):
    """Rotating the waypoints, boundary states and face normals by R rotates
    every iterate: c'_i[a, k] = sum_b R[a, b] c_i[b, k] (the ADMM of Eq. 18 with
    rotation-invariant rows is rotation-equivariant)."""
    w = _polytope_instance().with_(max_iters=300, eps=0.0)
    R = _rotation(11)
    wr = w.with_(waypoints=w.waypoints @ R.T, start_state=w.start_state @ R.T, end_state=w.end_state @ R.T,
                 poly_n=w.poly_n @ R.T)
    kw = {} if lib is None else {"real": lib}
    a = oracle.solve(w, **kw)["coeffs"]
    b = oracle.solve(wr, **kw)["coeffs"]
    rot = np.einsum("ab,ibk->iak", R, a)
    return float(np.abs(rot - b).max() / np.abs(a).max())


def test_polytope_rotation_equivariance():
    assert polytope_rotation_error() < 1e-11


def test_inactive_polytopes_keep_the_free_fixed_point():
    w0 = W.tiny(seed=5, N=3, mode="free", T_range=(0.9, 1.3), step=2.0)
    w = W.with_polytopes(w0, F=8, M=4, seed=2, margin=(50.0, 60.0)).with_(max_iters=100000, eps=1e-10)
    r = oracle.solve(w)
    ref = CZ.free_polynomial(w.durations, w.start_state[0], w.end_state[0])
    assert scaled_relerr(r["coeffs"], ref, w.durations) < 1e-9


# ------------------------------- quadratic rows inside the iteration (Eq. 18f-g) --

def _ball_instance():
    """Tiny FREE instance with a ball corridor per segment (Sec. III-C.2 with the
    centre shift of reading R8): centre at the chord midpoint of the unconstrained
    optimum, radius 85 % of its farthest sample (the trajectory's fixed end stays
    strictly inside), so that some samples bind; rho = 10 converges to ~1e-8."""
    w = W.tiny(seed=5, N=3, mode="free", T_range=(0.9, 1.3), step=2.0)
    free = CZ.free_polynomial(w.durations, w.start_state[0], w.end_state[0])
    N, M = len(w.durations), 2
    cen, rad = np.zeros((N, 3)), np.zeros(N)
    for i in range(N):
        T = w.durations[i]
        pts = np.array([[free[i, a] @ CZ.deriv_row(0, (j + 1) * T / M) for a in range(3)] for j in range(M)])
        start = np.array([free[i, a] @ CZ.deriv_row(0, 0.0) for a in range(3)])
        cen[i] = 0.5 * (start + pts[-1])
        rad[i] = 0.85 * np.linalg.norm(pts - cen[i], axis=1).max()
    rad[-1] = max(rad[-1], 1.05 * np.linalg.norm(w.waypoints[-1] - cen[-1]))
    return w.with_(M_ball=M, ball_c=cen, ball_r=rad, rho=10.0, max_iters=200000)


def _vn_instance():
    """Tiny FREE instance whose speed bound ||v(t_ij)|| <= v_max (projection
    family, Eq. 18f-g with the centre at 0) is 85 % of the unconstrained peak
    sampled speed; rho = 10 converges to ~1e-9."""
    w = W.tiny(seed=5, N=3, mode="free", T_range=(0.9, 1.3), step=2.0)
    free = CZ.free_polynomial(w.durations, w.start_state[0], w.end_state[0])
    N, M = len(w.durations), 3
    peak = max(np.linalg.norm([free[i, a] @ CZ.deriv_row(1, (j + 1) * w.durations[i] / M) for a in range(3)])
               for i in range(N) for j in range(M))
    return w.with_(M_vn=M, vnorm=np.array([0.85 * peak]), rho=10.0, max_iters=100000)


def quadratic_row_errors(kind, lib=None):
    """The converged oracle on a ball-corridor ("ball") or velocity-norm ("vn")
    instance against (i) the exact optimum of the same QCQP from its Lagrange
    dual (`centralized.norm_ball_qp`, nothing shared with the oracle), and
    (ii) the KKT certificate of Eq. 18 at the fixed point, every matrix rebuilt
    here from the basis:
      stationarity  2 Qt c + rho Mt^T (E u) + rho sum_j A_j^T w_j = 0
                    (A_j = I_3 (x) beta^{(r)}(t_j)^T, r = 0 ball, 1 velocity;
                    nu_j = rho w_j is the multiplier of sample j),
      nu_j along the outward normal at phi_j: w_j = lam_j (phi_j - o), lam_j >= 0,
      complementarity: lam_j > 0 only where ||phi_j - o|| = rad,
      the split holds: A_j c = phi_j, and A_j c is feasible.
    Returns (relative distance to the QCQP optimum, worst certificate violations,
    number of binding samples)."""
    w = _ball_instance() if kind == "ball" else _vn_instance()
    r = oracle.solve(w, state=True, **({} if lib is None else {"real": lib}))
    T, rho = w.durations, w.rho
    N = len(T)
    if kind == "ball":
        M, order, cen, rad = w.M_ball, 0, w.ball_c, w.ball_r
        phi, wd = r["phi_b"], r["w_b"]
    else:
        M, order, cen, rad = w.M_vn, 1, np.zeros((N, 3)), np.full(N, float(w.vnorm[0]))
        phi, wd = r["phi_v"], r["w_v"]
    c_ref, mu, g = CZ.norm_ball_qp(w.waypoints, T, w.start_state[0], w.end_state[0], "free", M, order, cen, rad)
    dist = scaled_relerr(r["coeffs"], c_ref, T)
    worst = {"stat": 0.0, "normal": 0.0, "compl": 0.0, "split": 0.0, "feas": 0.0}
    binding = 0
    for i in range(N):
        Mt, E = _consensus_rows(T[i], i == 0, i == N - 1)
        Qt = np.zeros((24, 24))
        for a in range(3):
            Qt[a * 8:(a + 1) * 8, a * 8:(a + 1) * 8] = CZ.snap_gram(T[i])
        ci = r["coeffs"][i].reshape(24)
        scale = np.abs(2 * Qt @ ci).max()
        stat = 2 * Qt @ ci + rho * Mt.T @ (E * r["u"][i])
        for j in range(M):
            A = np.kron(np.eye(3), CZ.deriv_row(order, (j + 1) * T[i] / M)[None, :])
            stat += rho * A.T @ wd[i, j]
            d = phi[i, j] - cen[i]
            nw = np.linalg.norm(wd[i, j])
            worst["split"] = max(worst["split"], np.abs(A @ ci - phi[i, j]).max() / max(1.0, np.abs(phi[i, j]).max()))
            worst["feas"] = max(worst["feas"], np.linalg.norm(A @ ci - cen[i]) - rad[i])
            if nw > 1e-8 * max(1.0, np.abs(wd).max()):
                binding += 1
                cosang = float(wd[i, j] @ d) / (nw * np.linalg.norm(d))
                worst["normal"] = max(worst["normal"], 1.0 - cosang)
                worst["compl"] = max(worst["compl"], abs(np.linalg.norm(d) - rad[i]) / rad[i])
        worst["stat"] = max(worst["stat"], np.abs(stat).max() / scale)
    return dist, worst, binding, r


def _quadratic_rows_ok(kind, lib=None):
    dist, worst, binding, r = quadratic_row_errors(kind, lib)
    return (binding >= 1 and dist < 1e-6 and worst["stat"] < 1e-6 and worst["normal"] < 1e-9
            and worst["compl"] < 1e-7 and worst["split"] < 1e-7 and worst["feas"] < 1e-7)


@pytest.mark.parametrize("kind", ["ball", "vn"])
def test_quadratic_rows_reach_the_qcqp_optimum_with_a_kkt_certificate(kind):
    dist, worst, binding, r = quadratic_row_errors(kind)
    assert binding >= 1, "the instance must have binding samples"
    assert dist < 1e-6, dist
    assert worst["stat"] < 1e-6 and worst["normal"] < 1e-9 and worst["compl"] < 1e-7, worst
    assert worst["split"] < 1e-7 and worst["feas"] < 1e-7, worst


# ------------------------------------------- residual values (Eq. 19-20) --

def residual_errors(lib=None, K=23):
    """||r_p|| and ||r_d|| reported after iteration K+1 (and in the history),
    recomputed here from the returned coefficients and junction states with
    matrices built from the basis:
      r_p^2 = sum over interior junctions, axes and orders 0..6 of
              (sigma_j^{(r)}(T_j) - sigma_{j+1}^{(r)}(0))^2            (Eq. 19)
      r_d^2 = sum_i || rho Mt_i^T E_i (zt_i^{K+1} - zt_i^K) ||^2          (Eq. 20, R10)
    on a batch of one PIN and one FREE trajectory with rho != 1 and box rows.
    Returns the largest relative error."""
    kw = {} if lib is None else {"real": lib}
    w = W.tiny(seed=12, N=[4, 6], mode="pin", T_range=(0.6, 1.4)).with_(rho=3.7)
    w = w.with_(M_box=3, vbox=np.array([2.0, 2.0]))
    worst = 0.0
    for mode in ("pin", "free"):
        wm = w.with_(mode=mode)
        a = oracle.solve(wm.with_(max_iters=K), state=True, **kw)
        b = oracle.solve(wm.with_(max_iters=K + 1), state=True, history=True, **kw)
        off = wm.seg_offset
        for t in range(wm.B):
            s0, s1 = int(off[t]), int(off[t + 1])
            N = s1 - s0
            T = wm.durations[s0:s1]
            c = b["coeffs"][s0:s1]
            rp2 = 0.0
            for j in range(1, N):
                for ax in range(3):
                    for rr in range(7):
                        gap = c[j - 1, ax] @ CZ.deriv_row(rr, T[j - 1]) - c[j, ax] @ CZ.deriv_row(rr, 0.0)
                        rp2 += gap * gap
            rd2 = 0.0
            za, zb = a["z"][s0 + t:s1 + t + 1], b["z"][s0 + t:s1 + t + 1]
            for i in range(N):
                Mt, E = _consensus_rows(T[i], i == 0, i == N - 1)
                dz = np.concatenate([np.concatenate([zb[i + side, ax] - za[i + side, ax] for side in (0, 1)])
                                     for ax in range(3)])
                v = wm.rho * Mt.T @ (E * dz)
                rd2 += v @ v
            for got, ref in ((b["r_primal"][t], np.sqrt(rp2)), (b["r_dual"][t], np.sqrt(rd2)),
                             (b["history"][K, t, 0], np.sqrt(rp2)), (b["history"][K, t, 1], np.sqrt(rd2))):
                worst = max(worst, abs(got - ref) / max(ref, 1e-300))
            if rd2 == 0.0 or rp2 == 0.0:
                worst = np.inf  # the instance must exercise both residuals
    return worst


def test_residuals_equal_their_definition():
    assert residual_errors() < 1e-10


# ------------------------------------------- numerical-step dual (Eq. 17) --

def numeric_dual_error(lib=None, K=20):
    """y^{K+1} - y^K = rho g(c^{K+1}) per sample and bound (Eq. 17 with the dual
    update of Eq. 7c, reading R9), g = max(0, ||sigma^{(r)}(t_j)||^2 - g_max^2)^2,
    recomputed here from the returned coefficients; rho = 1e4, so that a
    missing factor rho is visible.  Returns the largest relative error."""
    kw = {} if lib is None else {"real": lib}
    w = W.tiny(seed=9, N=4, mode="pin", step=4.0, T_range=(0.8, 1.0)).with_(
        inner="numeric", M_gen=4, gen_vmax=np.array([4.0]), gen_amax=np.array([8.0]), rho=1e4)
    a = oracle.solve(w.with_(max_iters=K), state=True, **kw)
    b = oracle.solve(w.with_(max_iters=K + 1), state=True, **kw)
    worst, active = 0.0, 0
    for i in range(w.S):
        T = w.durations[i]
        for j in range(w.M_gen):
            t = (j + 1) * T / w.M_gen
            for col, order, gmax in ((0, 1, 4.0), (1, 2, 8.0)):
                vec = np.array([b["coeffs"][i, ax] @ CZ.deriv_row(order, t) for ax in range(3)])
                g = max(0.0, vec @ vec - gmax ** 2) ** 2
                inc = b["y_gen"][i, j, col] - a["y_gen"][i, j, col]
                ref = w.rho * g
                active += ref > 0
                worst = max(worst, abs(inc - ref) / max(abs(ref), 1e-12 * abs(b["y_gen"]).max(), 1e-300))
    return worst if active else np.inf


def test_numeric_dual_step_is_rho_times_g():
    assert numeric_dual_error() < 1e-9
