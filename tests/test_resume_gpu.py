"""top_resume: the iteration state saved after K1 iterations and resumed
for K2 more reproduces one run of K1 + K2 iterations bit for bit (resident
packs and thread-block clusters, FP32 and FP64); the saved state is the
paper's (z, u) and row states, checked against the oracle's; a state saved in
FP32 continues in FP64 (the hand-off of a tolerance run)."""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import T, TOL, compare, to_np  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _solver(T, w, precision, **kw):
    return T.Solver(max_batch=w.B, max_segments=w.S, precision=precision, max_samples=16, **kw)


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _split_run(T, w, precision, K1, K2):
    s = _solver(T, w, precision)
    full, st_full = s.resume(w, max_iters=K1 + K2)
    a, st1 = s.resume(w, max_iters=K1)
    b, st2 = s.resume(w, start=st1, max_iters=K2)
    s.close()
    return _np(full), _np(st_full), _np(b), _np(st2)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", ["pin", "free"])
def test_resume_resident_is_bit_exact(T, precision, mode):
    w = W.tiny(seed=12, N=[1, 0, 2, 3, 33, 31, 64, 5, 127], mode=mode).with_(max_iters=80)
    if mode == "free":  # box rows as well
        w = w.with_(M_box=4, vbox=np.full(w.B, 1.5))
    full, st_full, b, st2 = _split_run(T, w, precision, 30, 50)
    for k in ("coeffs", "cost"):
        assert np.array_equal(full[k], b[k]), k
    for k in st_full:
        assert np.array_equal(st_full[k], st2[k]), k
    assert np.array_equal(b["iters"], np.where(np.diff(w.seg_offset) > 0, 50, 0))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_resume_in_clusters_is_bit_exact(T, precision):
    """The corridor workload (1024 segments, box and ball rows) runs in a
    thread-block cluster; the ball rows' first-iteration case is crossed."""
    w = W.corridor(N=1024).with_(max_iters=60)
    full, st_full, b, st2 = _split_run(T, w, precision, 1, 59)
    for k in ("coeffs", "cost"):
        assert np.array_equal(full[k], b[k]), k
    for k in st_full:
        assert np.array_equal(st_full[k], st2[k]), k


def test_saved_state_is_the_oracles_state(T):
    """p_j = z_j - u(start side of segment j), m_j = z_j - u(end side of segment
    j - 1), box rows y = v - s, ball rows q = phi + w (FP64, 1e-9 of the scale)."""
    w = W.corridor(N=12).with_(max_iters=40)
    w = w.with_(M_box=8, vbox=np.full(w.B, 3.0))
    s = _solver(T, w, "fp64")
    _, st = s.resume(w)
    s.close()
    st = _np(st)
    o = oracle.solve(w, state=True)
    off = np.asarray(w.seg_offset)
    for b in range(w.B):
        s0, s1 = int(off[b]), int(off[b + 1])
        N = s1 - s0
        for j in range(N + 1):
            jg = s0 + b + j
            z = o["z"][jg]  # [3][7]
            uS = o["u"][s0 + j].reshape(3, 2, 7)[:, 0, :] if j < N else None
            uE = o["u"][s0 + j - 1].reshape(3, 2, 7)[:, 1, :] if j > 0 else None
            p_ref = z - uS if uS is not None else np.where(np.arange(7) < 4, z, 0.0)
            m_ref = z - uE if uE is not None else np.where(np.arange(7) < 4, z, 0.0)
            if j == 0:
                p_ref = np.where(np.arange(7) < 4, p_ref, 0.0)
            if j == N:
                m_ref = np.where(np.arange(7) < 4, m_ref, 0.0)
            scale = max(1.0, np.abs(z).max())
            assert np.abs(st["p"][jg] - p_ref).max() <= 1e-9 * scale, (b, j, "p")
            assert np.abs(st["m"][jg] - m_ref).max() <= 1e-9 * scale, (b, j, "m")
    y_ref = o["v"] - o["s"]
    assert np.abs(st["ybox"] - y_ref).max() <= 1e-9 * max(1.0, np.abs(y_ref).max())
    q_ref = o["phi_b"] + o["w_b"]
    assert np.abs(st["qball"] - q_ref).max() <= 1e-9 * max(1.0, np.abs(q_ref).max())
    assert np.all(st["iters"] == 40)


def test_fp32_state_continues_in_fp64(T):
    """The hand-off of a tolerance run: FP32 for K1 iterations (held to the
    oracle at K1 with the FP32 tolerance), its state resumed by an FP64 handle
    for K2 more (held to the oracle's K1 + K2 run with the FP32 tolerance: the
    FP32 phase's rounding is carried over)."""
    w = W.corridor(N=64).with_(max_iters=200)
    s32 = _solver(T, w, "fp32")
    a, st = s32.resume(w, max_iters=120)
    s32.close()
    o1 = oracle.solve(w.with_(max_iters=120))
    compare(_np(a), o1, w, TOL["fp32"])
    s64 = _solver(T, w, "fp64")
    b, _ = s64.resume(w, start=st, max_iters=80, save=False)
    s64.close()
    o2 = oracle.solve(w.with_(max_iters=200))
    b = _np(b)
    b["iters"] = b["iters"] + 120
    compare(b, o2, w, TOL["fp32"])


def test_resume_rejects_what_it_cannot_save(T):
    w = W.tiny(seed=3, N=[4, 7], mode="pin").with_(max_iters=10)
    s = _solver(T, w, "fp32")
    for bad in (w.with_(adaptive_rho=True),
                w.with_(inner="numeric", M_gen=4, gen_vmax=np.full(2, 1e6), gen_amax=np.full(2, 1e6))):
        with pytest.raises(T.TopError) as e:
            s.resume(bad)
        assert e.value.code == T.TOP_E_NOTSUP
    s.close()
    st = _solver(T, w, "fp32", schedule="stream")
    with pytest.raises(T.TopError) as e:
        st.resume(w)
    assert e.value.code == T.TOP_E_NOTSUP
    st.close()


def _stall_stop(history, tol, cev, W_, cap):
    """The stall rule written out: at each check iteration k (k + 1 a multiple
    of cev), each of ||r_p||, ||r_d|| that falls below 0.99 of its own best so
    far becomes the new best; a check where neither does is one more check
    without progress; the run stops after W_ such checks in a row.  Returns the
    iteration count at the stop."""
    bp, bd, cnt = 1e300, 1e300, 0
    for k in range(cev - 1, cap, cev):
        rp, rd = history[k]
        if rp < tol and rd < tol:
            return None  # converged first
        ip, id_ = rp < 0.99 * bp, rd < 0.99 * bd
        if ip:
            bp = rp
        if id_:
            bd = rd
        if ip or id_:
            cnt = 0
        else:
            cnt += 1
            if cnt >= W_:
                return k + 1
    return None


@pytest.mark.parametrize("case", ["single_box", "corridor"])
def test_stall_rule_stops_where_its_definition_says(T, case):
    """FP32 at eps = 1e-4 does not reach the tolerance on these workloads (its
    residual floor): the stall rule stops the trajectory with TOP_STALLED at
    the iteration the rule's definition gives from the recorded residual
    history (resident packs for single_box, a cluster for the corridor), and
    FP64 resumed from that state converges."""
    w = W.single_box() if case == "single_box" else W.corridor(N=600)
    cev, W_, cap, eps = 10, 30, 20000, 1e-4
    s32 = _solver(T, w, "fp32")
    a, st = s32.resume(w, eps=eps, max_iters=cap, check_every=cev, stall_checks=W_, history=True)
    s32.close()
    a = _np(a)
    assert int(a["status"][0]) == T.TOP_STALLED, a["status"]
    K1 = int(a["iters"][0])
    assert K1 == _stall_stop(a["history"][:, 0, :], w.S * eps, cev, W_, cap)
    s64 = _solver(T, w, "fp64")
    b, _ = s64.resume(w, start=st, eps=eps, max_iters=cap - K1, check_every=cev, save=False)
    s64.close()
    assert int(_np(b)["status"][0]) == T.TOP_CONVERGED


def test_stall_rule_off_and_invalid(T):
    w = W.single_box().with_(max_iters=300)
    s = _solver(T, w, "fp32")
    g = _np(s.solve(w, eps=1e-4, check_every=10))  # stall_checks = 0: the run goes to max_iters
    assert int(g["status"][0]) == T.TOP_NOT_CONVERGED and int(g["iters"][0]) == 300
    with pytest.raises(T.TopError) as e:
        s.solve(w, eps=1e-4, stall_checks=-1)
    assert e.value.code == T.TOP_E_INVAL
    s.close()
