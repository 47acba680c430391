"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Both sides get the same seeded inputs and run the same number of CADMM
iterations; coefficients are compared on the time-normalised scale
c_k T^k (relative 2-norm over the batch), costs relative, iteration counts
and statuses exactly.  Tolerances: 1e-9 for the FP64 path, 1e-4 for the
FP32 path (FP32 state with FP64 KKT inverses and FP64 cost), over the batch,
per trajectory and per segment (`compare`).
"""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4}


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2507_10290_gb300 import build
    build.build()
    from paper_2507_10290_gb300 import top
    return top


_solvers = {}


def solver(T, precision, max_batch=4096, max_segments=1100000, max_samples=16):
    key = (precision, max_batch, max_segments, max_samples)
    if key not in _solvers:
        _solvers[key] = T.Solver(max_batch, max_segments, precision=precision, max_samples=max_samples)
    return _solvers[key]


def to_np(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def scaled(c, T):
    return c * np.asarray(T)[:, None, None] ** np.arange(8)[None, None, :]


def _coefficient_cost(dc, w):
    """Per trajectory, sum_i dc_i^T Qt(T_i) dc_i (the min-snap cost of a set of
    coefficients, here a difference), from Q(T)_kl = F(k,4) F(l,4) T^(k+l-7) / (k+l-7)
    on the time-normalised coefficients."""
    T = np.asarray(w.durations)
    k = np.arange(8)
    F4 = np.array([np.prod(np.arange(kk - 3, kk + 1)) if kk >= 4 else 0.0 for kk in k])
    e = k[:, None] + k[None, :] - 7
    Qh = np.where((k[:, None] >= 4) & (k[None, :] >= 4), np.outer(F4, F4) / np.where(e > 0, e, 1), 0.0)
    dh = dc * T[:, None, None] ** k[None, None, :]
    per_seg = np.einsum("sak,kl,sal->s", dh, Qh, dh) * T ** -7.0
    off = np.asarray(w.seg_offset)
    return np.array([per_seg[off[b]:off[b + 1]].sum() for b in range(w.B)])


def _boundary_scales(c, w):
    """Per trajectory, the sizes of the stacked vectors that Eq. 19 and Eq. 20
    take differences of, from coefficients c [S,3,8] (raw basis):
      X_p = || stack_i (beta~(T_i) c_i, beta~(0) c_i) ||      (Eq. 19)
      X_d = || stack_i rho Mt_i^T Mt_i c_i ||                  (Eq. 20 with z~ ~ Mt c)
    A relative error e in the coefficients moves ||r_p|| and ||r_d|| by about
    e X_p and e X_d, however small the residuals themselves are."""
    T = np.asarray(w.durations)
    k = np.arange(8)
    fall = np.array([[np.prod(np.arange(kk - r + 1, kk + 1)) if kk >= r else 0.0 for kk in k] for r in range(7)])
    S = len(T)
    with np.errstate(invalid="ignore"):
        powT = np.where(k[None, None, :] >= np.arange(7)[None, :, None],
                        T[:, None, None] ** np.clip(k[None, None, :] - np.arange(7)[None, :, None], 0, None), 0.0)
    MT = fall[None] * powT                      # [S, 7, 8]: rows r of beta^{(r)}(T)
    M0 = np.zeros((S, 7, 8))
    M0[:, np.arange(7), np.arange(7)] = fall[np.arange(7), np.arange(7)]
    eT = np.einsum("srk,sak->sar", MT, c)       # [S, 3, 7]
    e0 = np.einsum("srk,sak->sar", M0, c)
    mtm = np.einsum("srk,sar->sak", MT, eT) + np.einsum("srk,sar->sak", M0, e0)
    off = np.asarray(w.seg_offset)
    xp = np.array([np.sqrt(np.sum(eT[off[b]:off[b + 1]] ** 2) + np.sum(e0[off[b]:off[b + 1]] ** 2))
                   for b in range(w.B)])
    xd = np.array([w.rho * np.sqrt(np.sum(mtm[off[b]:off[b + 1]] ** 2)) for b in range(w.B)])
    return xp, xd


def compare(g, o, w, tol, check_iters=True):
    """Holds the GPU result g to the oracle's o; returns (batch coefficient
    error, batch cost error) after asserting:
      - coefficients (time-normalised c_k T_i^k): relative 2-norm over the
        batch and per trajectory <= tol; per segment, the error norm against
        the trajectory's RMS segment norm <= 10 tol (the trajectory bound
        alone allows up to sqrt(N_b) tol in one segment: this catches one
        wrong segment in a long trajectory);
      - cost: over the batch max|dJ| <= tol max|J|; per trajectory
        |dJ_b| <= tol J_b + 2 sqrt(J_b D_b) + D_b, D_b = sum_i dc_i^T Qt(T_i) dc_i
        the cost of the coefficient difference: J(c + dc) - J(c) = 2 c^T Qt dc
        + dc^T Qt dc, so the cost may move by what the (already bounded)
        coefficient difference implies, plus tol (empty trajectories: both 0);
      - iteration counts and statuses exactly (unless check_iters is False);
      - residuals: per trajectory |dr| <= rtol r + tol X, rtol = 1e-3 (FP32)
        or 1e-7 (FP64), X the size of the stacked vectors whose difference
        the residual is (_boundary_scales): Eq. 19-20 are norms of
        differences of O(|z|) quantities, so a residual is as accurate as the
        coefficients it is formed from, and no more, once it is much smaller
        than X."""
    T = w.durations
    off = np.asarray(w.seg_offset)
    if w.S:
        ref = scaled(o["coeffs"], T)
        got = scaled(g["coeffs"], T)
        err = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
        assert err <= tol, f"coefficient error {err:.3e} > {tol:.1e}"
        seg_d = np.linalg.norm((got - ref).reshape(w.S, -1), axis=1)
        seg_n = np.linalg.norm(ref.reshape(w.S, -1), axis=1)
        for b in range(w.B):
            s0, s1 = int(off[b]), int(off[b + 1])
            if s1 == s0:
                continue
            nb = float(np.linalg.norm(seg_n[s0:s1]))
            eb = float(np.linalg.norm(seg_d[s0:s1])) / max(nb, 1e-300)
            assert eb <= tol, f"trajectory {b}: coefficient error {eb:.3e} > {tol:.1e}"
            rms = nb / np.sqrt(s1 - s0)
            es = float(seg_d[s0:s1].max()) / max(rms, 1e-300)
            assert es <= 10 * tol, (f"trajectory {b}: worst segment error {es:.3e} (of the RMS segment norm) "
                                    f"> {10 * tol:.1e}")
    else:
        err = 0.0
    cref = np.abs(o["cost"]).max() if len(o["cost"]) else 0.0
    cerr = float(np.abs(g["cost"] - o["cost"]).max() / max(cref, 1e-300)) if len(o["cost"]) else 0.0
    assert cerr <= tol, f"cost error {cerr:.3e} > {tol:.1e}"
    dcost = _coefficient_cost(np.asarray(g["coeffs"]) - np.asarray(o["coeffs"]), w) if w.S else np.zeros(w.B)
    for b in range(w.B):
        jb = abs(float(o["cost"][b]))
        d = abs(float(g["cost"][b]) - float(o["cost"][b]))
        bound = tol * jb + 2.0 * np.sqrt(jb * dcost[b]) + dcost[b]
        assert d <= bound * (1 + 1e-9) or (jb == 0.0 and d == 0.0), \
            f"trajectory {b}: cost error {d:.3e} > {bound:.3e} (J = {jb:.3e}, cost of the coefficient difference {dcost[b]:.3e})"
    if check_iters:
        assert np.array_equal(g["iters"], o["iters"]), (g["iters"], o["iters"])
        assert np.array_equal(g["status"], o["status"]), (g["status"], o["status"])
    rtol = 1e-7 if tol <= 1e-9 else 1e-3
    if w.S:
        xp, xd = _boundary_scales(o["coeffs"], w)
        for key, X in (("r_primal", xp), ("r_dual", xd)):
            d = np.abs(g[key] - o[key])
            bound = rtol * np.abs(o[key]) + tol * X
            worst = int(np.argmax(d - bound))
            assert np.all(d <= bound), (f"{key} of trajectory {worst}: |d| = {d[worst]:.3e}, r = {o[key][worst]:.3e}, "
                                        f"X = {X[worst]:.3e}")
    return err, cerr


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_box_N8(T, precision):
    w = W.single_box()
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", ["pin", "free"])
def test_edge_shapes(T, precision, mode):
    # ragged batch: single-segment, empty, lengths straddling warps and a CTA
    Ns = [1, 0, 2, 3, 33, 31, 32, 64, 0, 5, 127, 1]
    w = W.tiny(seed=12, N=Ns, mode=mode).with_(max_iters=60)
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_and_one_iteration(T, precision):
    w = W.tiny(seed=3, N=[4, 7], mode="pin")
    for K in (0, 1):
        o = oracle.solve(w.with_(max_iters=K))
        g = to_np(solver(T, precision).solve(w, max_iters=K))
        compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_subset_300_iterations(T, precision):
    full = W.batch(B=64)
    w = full
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_shared_durations(T, precision):
    """Trajectories whose segments share one duration: the precompute inverts
    the first interior segment and reuses it for the other interior segments
    of that duration.  Shared batch, lengths 0..6 around the first/last
    special cases, one interior duration changed, with and without sample rows."""
    w = W.batch(B=48, shared_T=True, n_min=8, n_max=64)
    compare(to_np(solver(T, precision).solve(w)), oracle.solve(w), w, TOL[precision])
    Ns = [0, 1, 2, 3, 4, 5, 6, 9]
    e = W.tiny(seed=31, N=Ns, mode="pin")
    off = e.seg_offset
    Tn = e.durations.copy()
    for b in range(len(Ns)):
        Tn[off[b]:off[b + 1]] = 0.7 + 0.1 * b
    Tn[off[7] + 4] = 1.3                     # one interior segment differs
    Tn[off[6] + 1] = 0.9                     # the reference segment itself differs
    e = e.with_(durations=Tn, max_iters=120)
    for case in (e, e.with_(mode="free", M_box=8, vbox=np.full(len(Ns), 1.2))):
        compare(to_np(solver(T, precision).solve(case)), oracle.solve(case), case, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_corridor_box_and_ball(T, precision):
    N = 64 if precision == "fp64" else 128
    w = W.corridor(N=N)
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_velocity_norm_projection(T, precision):
    w = W.tiny(seed=21, N=[6, 9], mode="free", step=3.0).with_(M_vn=8, vnorm=np.array([2.0, 2.5]),
                                                                max_iters=150)
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


def test_stopping_rule_and_history_fp64(T):
    w = W.tiny(seed=1, N=[8, 5, 12], mode="free", T_range=(0.8, 1.6)).with_(eps=1e-3, max_iters=5000)
    o = oracle.solve(w, history=True)
    g = to_np(solver(T, "fp64").solve(w, history=True, check_every=1))
    compare(g, o, w, TOL["fp64"])
    k = int(o["iters"].max())
    for b in range(w.B):
        kb = int(o["iters"][b])
        # residuals are differences of O(|z|) quantities: absolute rounding ~ 1e-9 of their peak
        scale = np.abs(o["history"][:kb, b]).max(axis=0)
        assert np.all(np.abs(g["history"][:kb, b] - o["history"][:kb, b]) <= 1e-9 * scale)


def test_host_memory_path_matches_device_path(T):
    w = W.tiny(seed=5, N=[10, 3, 20], mode="pin").with_(max_iters=80)
    s = solver(T, "fp32")
    gd = to_np(s.solve(w))
    gh = s.solve_host(w)
    for k in ("coeffs", "cost", "r_primal", "r_dual", "iters", "status"):
        assert np.array_equal(gd[k], gh[k]), k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_run_to_run_deterministic(T, precision):
    w = W.batch(B=32, seed=4).with_(max_iters=50)
    s = solver(T, precision)
    a = to_np(s.solve(w))
    b = to_np(s.solve(w))
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_invalid_inputs_are_rejected(T):
    s = solver(T, "fp32", max_batch=8, max_segments=64)
    w = W.tiny(seed=2, N=[4, 4], mode="pin")
    bad = w.with_(durations=np.where(np.arange(8) == 3, -1.0, w.durations))
    with pytest.raises(T.TopError) as e:
        s.solve(bad)
    assert e.value.code == T.TOP_E_INVAL
    big = W.tiny(seed=2, N=[40, 40], mode="pin")
    with pytest.raises(T.TopError) as e:
        s.solve(big)
    assert e.value.code == T.TOP_E_NOMEM
    num = w.with_(inner="numeric", M_box=2, vbox=np.array([1.0, 1.0]), M_gen=2,
                  gen_vmax=np.ones(2), gen_amax=np.ones(2))
    with pytest.raises(T.TopError) as e:
        s.solve(num)
    assert e.value.code == T.TOP_E_NOTSUP
    # the handle still works afterwards
    o = oracle.solve(w)
    compare(to_np(s.solve(w)), o, w, TOL["fp32"])


def test_full_size_batch_sampled(T):
    """The 4096-trajectory workload at full size, 300 iterations, FP32: sampled
    trajectories against the oracle (each trajectory is independent)."""
    w = W.batch()
    g = to_np(solver(T, "fp32").solve(w))
    rng = np.random.default_rng(0)
    ids = sorted(rng.choice(w.B, size=12, replace=False).tolist())
    sub = w.subset(ids)
    o = oracle.solve(sub)
    gs = {k: v[ids] for k, v in g.items() if k != "coeffs"}
    segs = np.concatenate([np.arange(w.seg_offset[b], w.seg_offset[b + 1]) for b in ids])
    gs["coeffs"] = g["coeffs"][segs]
    compare(gs, o, sub, TOL["fp32"])
    assert np.all(np.isfinite(g["coeffs"])) and np.all(g["iters"] == 300)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_numerical_step_with_active_bounds(T, precision, tol):
    """General norm bounds through the L-BFGS local step (Sec. III-C.3), with
    bounds active on several segments; both sides solve every local problem
    to a tight tolerance, so they agree at the inner optimum."""
    w = W.general(N=100, v_nom=3.0).with_(max_iters=100, rho=100.0, lbfgs_max_iters=2000,
                                          lbfgs_tol=1e-12 if precision == "fp64" else 1e-6)
    o = oracle.solve(w, state=True, lbfgs_tol=1e-12, lbfgs_max_iters=2000)
    assert (o["inner_iters"] > 0).sum() >= 3, "the bounds must be active somewhere"
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, tol)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_numerical_step_inactive_equals_closed_form(T, precision):
    w = W.tiny(seed=8, N=[6, 40, 3], mode="pin").with_(max_iters=60)
    wn = w.with_(inner="numeric", M_gen=8, gen_vmax=np.full(3, 1e6), gen_amax=np.full(3, 1e6))
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(wn))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_corridor_full_size_streaming(T, precision):
    """The 1024-segment corridor workload at full size (box + ball rows at 16
    samples, FREE waypoints, 200 iterations): longer than one CTA holds, so it
    runs in the streaming form."""
    w = W.corridor()
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_general_bounds_long_trajectory(T, precision):
    """The general-bounds workload at N = 1000 through the numerical step."""
    w = W.general(N=1000)
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("B,N", [(2, 4500), (6, 2300)])
def test_streaming_sums_over_several_chunks(T, B, N):
    """Streaming trajectories longer than one block of the residual sums
    (2048 segments, FP64, residuals every 10 iterations): the residuals of
    every evaluated iteration, the iteration at which the stopping rule
    (Eq. 21) fires and the coefficients there agree with the oracle.  With six
    streaming trajectories the kernels also find each segment's trajectory
    through the per-solve map instead of the search."""
    key = ("stream-chunks", B, N)
    if key not in _solvers:
        _solvers[key] = T.Solver(B, B * N, precision="fp64", max_samples=0, schedule="stream")
    s = _solvers[key]
    K, cev = 80, 10
    w = W.batch(seed=3, B=B, fixed_N=N).with_(mode="free", max_iters=K)
    o = oracle.solve(w, history=True)  # eps = 0: the residuals of every iteration
    checks = np.arange(cev - 1, K, cev)
    m = o["history"][:, :, :].max(axis=2)  # [K, B]: the larger residual
    # a threshold that trajectory 0 first meets at a check inside the run
    j = 1 + int(np.argmin(m[checks[1:-1], 0]))
    assert m[checks[j], 0] < m[checks[:j], 0].min()
    eps = m[checks[j], 0] * (1 + 1e-6) / N
    expect_it = np.full(B, K)
    expect_st = np.ones(B, np.int32)
    for b in range(B):
        hit = [k for k in checks if m[k, b] < N * eps]
        if hit:
            expect_it[b], expect_st[b] = hit[0] + 1, 0
    assert expect_it[0] == checks[j] + 1 < K
    g = to_np(s.solve(w.with_(eps=eps), history=True, check_every=cev))
    assert np.array_equal(g["iters"], expect_it) and np.array_equal(g["status"], expect_st)
    for b in range(B):
        ks = [k for k in checks if k < expect_it[b]]
        scale = np.abs(o["history"][ks, b]).max(axis=0)
        assert np.all(np.abs(g["history"][ks, b] - o["history"][ks, b]) <= 1e-9 * scale)
    # the coefficients where each trajectory stopped
    for it in sorted(set(expect_it.tolist())):
        sel = [b for b in range(B) if expect_it[b] == it]
        ws = w.subset(sel).with_(max_iters=int(it))
        os_ = oracle.solve(ws)
        off = np.asarray(w.seg_offset)
        gs = {"coeffs": np.concatenate([g["coeffs"][off[b]:off[b + 1]] for b in sel]),
              "cost": g["cost"][sel], "r_primal": g["r_primal"][sel], "r_dual": g["r_dual"][sel],
              "iters": os_["iters"], "status": os_["status"]}
        compare(gs, os_, ws, TOL["fp64"])


def test_large_host_memory_results_equal_device_results(T):
    """138,519 segments (26.6 MB of coefficients staged back to the host): the
    host-buffer call returns exactly what the device-buffer call does."""
    w = W.batch(B=512).with_(max_iters=10)
    s = solver(T, "fp32")
    gd = to_np(s.solve(w))
    gh = s.solve_host(w)
    assert gd["coeffs"].nbytes > (16 << 20)
    for k in ("coeffs", "cost", "r_primal", "r_dual", "iters", "status"):
        assert np.array_equal(gd[k], gh[k]), k


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pin_with_box_rows_does_not_converge(T, precision):
    """The single-box workload with PIN waypoints: pinned positions plus the
    velocity box leave (almost) no feasible trajectory, and the iteration does
    not reach eps = 1e-4 in 3000 iterations, on the oracle as on the GPU.  The
    status says so (TOP_NOT_CONVERGED), the results of the last iteration are
    written and finite, and they match the oracle's after the same iterations."""
    w = W.single_box().with_(mode="pin", eps=1e-4, max_iters=3000)
    o = oracle.solve(w)
    assert o["status"][0] == T.TOP_NOT_CONVERGED
    g = to_np(solver(T, precision).solve(w))
    assert g["status"][0] == T.TOP_NOT_CONVERGED and g["iters"][0] == 3000
    assert np.all(np.isfinite(g["coeffs"])) and g["r_primal"][0] > 1.0
    compare(g, o, w, TOL[precision])


def test_full_capacity_fits_shared_memory(T):
    """The 512-segment resident CTA (FP32, no inequality rows, 128 trajectory
    slots) fits the opt-in shared memory: the autotuner can time it."""
    w = W.batch(B=32)
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision="fp32")
    best, caps = s.autotune(w, iters=3)
    s.close()
    assert caps[512] > 0, caps


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_capacity_edges(T, precision):
    """Lengths at the edges of a resident CTA (FP32 holds 512 segments, FP64
    256): 255, 256, 257, 511, 512 and 513 segments with a single segment
    between them, so each form boundary (resident, 2-CTA cluster) is crossed."""
    w = W.tiny(seed=31, N=[255, 1, 256, 257, 511, 512, 513], mode="pin").with_(max_iters=40)
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])
