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
    s.close()
