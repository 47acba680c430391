"""GPU adjoint (top_grad) against central finite differences of the CPU oracle.

J(P, T) = sum_b dJ_b J_b after exactly K closed-form iterations; the oracle's
unrolled map is differenced in FP64.  FP64 adjoint: 1e-6 relative to the
gradient's norm (FD step 1e-4); FP32 adjoint: 1e-3 (FD step 1e-3, the
benchmark's tolerance).  At the benchmark's size (256 x 256, K = 100) the
check is on random directions of sampled trajectories.
"""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_2507_10290_gb300 import build
    build.build()
    from paper_2507_10290_gb300 import top
    return top


def oracle_J(w, dJ):
    return float(np.dot(dJ, oracle.solve(w)["cost"]))


def fd_gradient(w, dJ, h):
    """Central differences of the oracle's sum dJ_b J_b in every waypoint and duration."""
    gP = np.zeros_like(w.waypoints)
    gT = np.zeros_like(w.durations)
    for idx in np.ndindex(*w.waypoints.shape):
        Pp, Pm = w.waypoints.copy(), w.waypoints.copy()
        Pp[idx] += h
        Pm[idx] -= h
        gP[idx] = (oracle_J(w.with_(waypoints=Pp), dJ) - oracle_J(w.with_(waypoints=Pm), dJ)) / (2 * h)
    for i in range(len(w.durations)):
        Tp, Tm = w.durations.copy(), w.durations.copy()
        Tp[i] += h
        Tm[i] -= h
        gT[i] = (oracle_J(w.with_(durations=Tp), dJ) - oracle_J(w.with_(durations=Tm), dJ)) / (2 * h)
    return gP, gT


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("mode", ["pin", "free"])
@pytest.mark.parametrize("precision,h,tol", [("fp64", 1e-4, 1e-6), ("fp32", 1e-3, 1e-3)])
def test_full_gradient_small(T, mode, precision, h, tol):
    w = W.tiny(seed=31, N=[3, 5, 1], mode=mode, T_range=(0.6, 1.2)).with_(max_iters=30, rho=1.0)
    dJ = np.array([1.0, 0.5, 2.0])
    gP, gT = fd_gradient(w, dJ, h)
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision=precision)
    dw, dT = s.grad(w, dJ=dJ)
    dw, dT = dw.cpu().numpy(), dT.cpu().numpy()
    s.close()
    assert rel(dT, gT) < tol, (rel(dT, gT), dT, gT)
    assert rel(dw, gP) < tol, (rel(dw, gP),)
    # the trajectory's end waypoints do not enter (the boundary states do)
    for b in range(w.B):
        assert np.all(dw[w.seg_offset[b] + b] == 0) and np.all(dw[w.seg_offset[b + 1] + b] == 0)


def _box_case():
    """Two FREE trajectories whose box limit is 45 % of the unconstrained peak
    axis speed: six box rows are active after 40 iterations (central
    differences with h = 1e-4 and 1e-5 agree to 3e-8, no kink nearby)."""
    from oracle import centralized as C
    w = W.tiny(seed=41, N=[3, 4], mode="free", T_range=(0.7, 1.2), step=2.0).with_(max_iters=40, rho=3.0)
    vb = []
    for b in range(w.B):
        sub = w.subset([b])
        fr = C.free_polynomial(sub.durations, sub.start_state[0], sub.end_state[0])
        pk = max(abs(fr[i, a] @ C.deriv_row(1, (j + 1) * sub.durations[i] / 4))
                 for i in range(sub.S) for a in range(3) for j in range(4))
        vb.append(0.45 * pk)
    return w.with_(M_box=4, vbox=np.array(vb))


ROW_CASES = {
    "box": _box_case,
    # the corridor recipe at N = 5: ball rows at 16 samples, 14 of them projected
    "ball": lambda: W.corridor(N=5).with_(max_iters=25, rho=3.0, M_box=0, vbox=None),
    # a speed bound through the projection, 13 samples projected
    "vnorm": lambda: W.tiny(seed=21, N=[6, 4], mode="free", step=3.0).with_(
        M_vn=6, vnorm=np.array([2.0, 2.5]), max_iters=25, rho=3.0),
}


@pytest.mark.parametrize("case", sorted(ROW_CASES))
@pytest.mark.parametrize("precision,h,tol", [("fp64", 1e-4, 1e-6), ("fp32", 1e-3, 1e-3)])
def test_gradient_through_inequality_rows(T, case, precision, h, tol):
    """The adjoint through the slack / projection steps (Eq. 18d-g) against
    central differences of the oracle's unrolled map, every waypoint and
    duration."""
    w = ROW_CASES[case]()
    dJ = np.linspace(1.0, 2.0, w.B)
    gP, gT = fd_gradient(w, dJ, h)
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision=precision, max_samples=16)
    dw, dT = s.grad(w, dJ=dJ)
    dw, dT = dw.cpu().numpy(), dT.cpu().numpy()
    s.close()
    assert rel(dT, gT) < tol, (rel(dT, gT), dT, gT)
    assert rel(dw, gP) < tol, (rel(dw, gP),)


def test_time_allocation_in_a_corridor(T):
    """Outer time allocation with box and ball rows: F = J + k_T sum T falls
    (evaluated by the oracle at the initial and the final durations)."""
    w = W.corridor(N=8).with_(max_iters=60, rho=3.0)
    kT = 5.0
    s = T.Solver(max_batch=1, max_segments=w.S, precision="fp64", max_samples=16)
    Tout, out = s.time_alloc(w, k_T=kT, lr=0.05, steps=5)
    s.close()
    Tout = np.asarray(Tout.cpu().numpy() if hasattr(Tout, "cpu") else Tout)
    F0 = oracle.solve(w)["cost"][0] + kT * w.durations.sum()
    F1 = oracle.solve(w.with_(durations=Tout))["cost"][0] + kT * Tout.sum()
    assert np.all(Tout > 0) and F1 < F0, (F0, F1)


def test_directional_derivatives_full_size(T):
    """256 x 256, K = 100, FP32: random directions on sampled trajectories."""
    w = W.grad_batch()
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision="fp32")
    dJ = np.ones(w.B)
    dw, dT = s.grad(w, dJ=dJ)
    dw, dT = dw.cpu().numpy(), dT.cpu().numpy()
    s.close()
    assert np.all(np.isfinite(dw)) and np.all(np.isfinite(dT))
    rng = np.random.default_rng(5)
    h = 1e-3
    for b in rng.choice(w.B, size=3, replace=False):
        sub = w.subset([b])
        s0, s1 = w.seg_offset[b], w.seg_offset[b + 1]
        gw = dw[s0 + b: s1 + b + 1]
        gt = dT[s0:s1]
        for _ in range(3):
            vP = rng.normal(size=sub.waypoints.shape)
            vT = rng.normal(size=sub.durations.shape) * 0.1
            Jp = oracle.solve(sub.with_(waypoints=sub.waypoints + h * vP, durations=sub.durations + h * vT))["cost"][0]
            Jm = oracle.solve(sub.with_(waypoints=sub.waypoints - h * vP, durations=sub.durations - h * vT))["cost"][0]
            fd = (Jp - Jm) / (2 * h)
            ad = float(np.sum(gw * vP) + np.sum(gt * vT))
            assert abs(ad - fd) <= 1e-3 * max(abs(fd), 1e-12), (b, ad, fd)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-3)])
def test_converged_gradient_equals_the_centralized_qp_gradient(T, precision, tol):
    """Six PIN segments, rho = 10, K = 1000: the iteration has reached its
    fixed point (the unrolled cost equals the centralized optimum to 1e-12),
    so the adjoint must equal the gradient of the optimal value J*(P, T) of
    the centralized QP, here central differences (h = 1e-5, FP64) of its
    direct solve (the C^6 spline of the optimality conditions)."""
    from oracle import centralized as C
    w0 = W.tiny(seed=4, N=[6], mode="pin", T_range=(1.6, 2.4), step=2.0)
    w = w0.with_(durations=1.4 * w0.durations, max_iters=1000, rho=10.0)

    def Jstar(P, Td):
        return C.segment_cost(C.pin_spline(P, Td, w.start_state[0], w.end_state[0]), Td)

    assert abs(oracle.solve(w)["cost"][0] / Jstar(w.waypoints, w.durations) - 1) < 1e-10
    h = 1e-5
    gP = np.zeros_like(w.waypoints)
    gT = np.zeros_like(w.durations)
    for idx in np.ndindex(*w.waypoints.shape):
        Pp, Pm = w.waypoints.copy(), w.waypoints.copy()
        Pp[idx] += h
        Pm[idx] -= h
        gP[idx] = (Jstar(Pp, w.durations) - Jstar(Pm, w.durations)) / (2 * h)
    for i in range(w.S):
        Tp, Tm = w.durations.copy(), w.durations.copy()
        Tp[i] += h
        Tm[i] -= h
        gT[i] = (Jstar(w.waypoints, Tp) - Jstar(w.waypoints, Tm)) / (2 * h)
    s = T.Solver(max_batch=1, max_segments=w.S, precision=precision)
    dw, dT = s.grad(w)
    s.close()
    dw, dT = dw.cpu().numpy(), dT.cpu().numpy()
    assert rel(dT, gT) < tol, (rel(dT, gT), dT, gT)
    assert rel(dw, gP) < tol, rel(dw, gP)


@pytest.mark.parametrize("mode", ["pin", "free"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_resident_and_streaming_adjoints_agree(T, mode, precision, tol):
    """The one-launch resident adjoint (trajectories that fit one CTA) and the
    streaming adjoint (any length) differentiate the same iteration: ragged
    lengths, an empty trajectory, K not a multiple of the checkpoint interval."""
    w = W.tiny(seed=33, N=[1, 0, 2, 7, 33, 64, 5], mode=mode, T_range=(0.6, 1.4)).with_(max_iters=37)
    dJ = np.linspace(0.5, 2.0, w.B)
    out = []
    for schedule in ("auto", "stream"):
        s = T.Solver(max_batch=w.B, max_segments=w.S, precision=precision, schedule=schedule)
        dw, dT = s.grad(w, dJ=dJ)
        out.append((dw.cpu().numpy(), dT.cpu().numpy()))
        s.close()
    (rw, rT), (sw, sT) = out
    assert np.all(np.isfinite(rw)) and np.all(np.isfinite(rT))
    assert rel(rT, sT) < tol, rel(rT, sT)
    assert rel(rw, sw) < tol, rel(rw, sw)


def test_long_trajectory_gradient_uses_the_streaming_adjoint(T):
    """A trajectory longer than a resident adjoint CTA holds: the streaming
    adjoint, checked along random directions against the oracle."""
    w = W.tiny(seed=35, N=[300, 4], mode="pin", T_range=(0.6, 1.4)).with_(max_iters=12)
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision="fp64")
    dw, dT = s.grad(w)
    dw, dT = dw.cpu().numpy(), dT.cpu().numpy()
    s.close()
    rng = np.random.default_rng(2)
    h = 1e-4
    for _ in range(2):
        vP = rng.normal(size=w.waypoints.shape)
        vT = rng.normal(size=w.durations.shape) * 0.1
        Jp = oracle.solve(w.with_(waypoints=w.waypoints + h * vP, durations=w.durations + h * vT))["cost"].sum()
        Jm = oracle.solve(w.with_(waypoints=w.waypoints - h * vP, durations=w.durations - h * vT))["cost"].sum()
        fd = (Jp - Jm) / (2 * h)
        ad = float(np.sum(dw * vP) + np.sum(dT * vT))
        assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


def test_autograd_function_matches_top_grad(T):
    import torch
    from paper_2507_10290_gb300.autograd import TopCost
    w = W.tiny(seed=7, N=[4, 6], mode="pin").with_(max_iters=20)
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision="fp64")
    P = torch.tensor(w.waypoints, dtype=torch.float64, device="cuda", requires_grad=True)
    Td = torch.tensor(w.durations, dtype=torch.float64, device="cuda", requires_grad=True)
    cost = TopCost.apply(P, Td, s, w)
    ref = oracle.solve(w)["cost"]
    assert np.allclose(cost.detach().cpu().numpy(), ref, rtol=1e-9)
    (cost * torch.tensor([1.0, 3.0], device="cuda", dtype=torch.float64)).sum().backward()
    dw, dT = s.grad(w, dJ=np.array([1.0, 3.0]))
    assert torch.allclose(P.grad, dw) and torch.allclose(Td.grad, dT)
    # inputs on the CPU: the gradients come back there, in the inputs' dtype
    Pc = torch.tensor(w.waypoints, dtype=torch.float32, requires_grad=True)
    Tc = torch.tensor(w.durations, dtype=torch.float64, requires_grad=True)
    TopCost.apply(Pc, Tc, s, w).sum().backward()
    assert Pc.grad.device.type == "cpu" and Pc.grad.dtype == torch.float32 and Tc.grad.device.type == "cpu"
    s.close()
