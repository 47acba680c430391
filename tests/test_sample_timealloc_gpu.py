"""Trajectory sampling (top_sample) and the outer time allocation
(top_time_alloc) on the GPU.

Sampling is checked against the plain definition sigma_i(t) = sum_k c_k (t -
t_{i-1})^k and its derivatives evaluated here in numpy; the similarity
metric of Sec. IV-A.2 (e_simi = lg sum_m |p_m - p_m^ref|, 8192 samples) on
GPU coefficients is compared with the same metric on the oracle's.  The
time allocation is checked against the closed-form optimum of a single
rest-to-rest segment, J(T) = 100800 |dP|^2 / T^7 (the golden smootherstep),
and for several segments against a stationarity and a finite-difference
minimum test on the oracle.  Both use a rho and an iteration count at which
the inner iteration has converged, so that J after K iterations is the
optimum's cost.
"""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import T, solver, to_np  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def eval_piecewise(coeffs, durations, off, M, order):
    """numpy: derivative `order` at t_m = m T_b / (M - 1), later segment at junctions."""
    B = len(off) - 1
    out = np.zeros((B, M, 3))
    k = np.arange(8)
    fall = np.array([np.prod(np.arange(kk - order + 1, kk + 1)) if kk >= order else 0 for kk in k], dtype=float)
    for b in range(B):
        g0, g1 = off[b], off[b + 1]
        if g1 == g0:
            continue
        Tb = durations[g0:g1]
        starts = np.concatenate([[0.0], np.cumsum(Tb)[:-1]])
        total = Tb.sum()
        for m in range(M):
            t = total if m == M - 1 else m * total / (M - 1)
            i = int(np.searchsorted(starts, t, side="right") - 1)
            tau = t - starts[i]
            powers = np.where(k >= order, tau ** np.maximum(k - order, 0), 0.0)
            out[b, m] = coeffs[g0 + i] @ (fall * powers)
    return out


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_sample_matches_the_definition(T, order):
    w = W.tiny(seed=3, N=[4, 0, 1, 7], mode="pin")
    rng = np.random.default_rng(order)
    coeffs = rng.normal(size=(w.S, 3, 8))
    s = solver(T, "fp64")
    import torch
    got = s.sample(w, torch.as_tensor(coeffs, device="cuda"), 33, order).cpu().numpy()
    ref = eval_piecewise(coeffs, w.durations, w.seg_offset, 33, order)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    assert np.all(got[1] == 0.0)


def e_simi(samples, ref):
    return float(np.log10(np.linalg.norm(samples - ref, axis=-1).sum()))


def test_similarity_metric_on_the_curve_matches_the_oracle(T):
    """e_simi of the trajectory after 600 iterations, GPU (FP64) against the
    oracle's coefficients sampled by the same definition."""
    Mref = 8192
    for N in (8, 32):
        w = W.curve(N=N, max_iters=600)
        o = oracle.solve(w)
        s = solver(T, "fp64")
        g = s.solve(w)
        samp = s.sample(w, g["coeffs"], Mref, 0).cpu().numpy()[0]
        tt = np.linspace(0.0, 1.0, Mref)
        ref = W.trefoil(tt, 0, w.notes["scale"])
        ours = e_simi(samp, ref)
        theirs = e_simi(eval_piecewise(o["coeffs"], w.durations, w.seg_offset, Mref, 0)[0], ref)
        assert abs(ours - theirs) < 1e-6, (N, ours, theirs)


def _single_segment(T0):
    P = np.array([[0.3, -1.0, 2.0], [2.5, 1.5, -1.0]])
    z = np.zeros((1, 3, 3))
    return W.tiny(N=1, mode="pin").with_(
        waypoints=P, durations=np.array([T0]), start_state=np.concatenate([P[None, :1], z], axis=1),
        end_state=np.concatenate([P[None, 1:], z], axis=1), max_iters=300, rho=1e5 / 2.0 ** 7), P[1] - P[0]


def test_time_allocation_reaches_the_closed_form_optimum(T):
    """F(T) = 100800 |dP|^2 / T^7 + k_T T has its minimum at
    T* = (7 * 100800 |dP|^2 / k_T)^(1/8); k_T is chosen so that T* = 2."""
    w, d = _single_segment(2.6)
    Tstar = 2.0
    kT = 7 * 100800 * float(d @ d) / Tstar ** 8
    s = solver(T, "fp64")
    Tout, out = s.time_alloc(w, k_T=kT, lr=0.5 / (8 * kT * Tstar), steps=80)
    Tout = Tout.cpu().numpy()
    assert abs(Tout[0] - Tstar) < 1e-6 * Tstar, Tout
    J = to_np(out)["cost"][0]
    assert abs(J - 100800 * float(d @ d) / Tout[0] ** 7) < 1e-8 * J


def test_time_allocation_on_several_segments_is_a_local_minimum(T):
    """Five PIN segments, rho = 10 and 1000 iterations (the inner iteration is
    converged to ~1e-12 at these durations), k_T = 40: the outer loop ends at a
    stationary point of F, and the oracle's F grows along every coordinate."""
    w0 = W.tiny(seed=4, N=[5], mode="pin", T_range=(1.6, 2.4), step=2.0)
    w = w0.with_(durations=1.4 * w0.durations, max_iters=1000, rho=10.0)
    kT = 40.0
    s = solver(T, "fp64")
    Tout, _ = s.time_alloc(w, k_T=kT, lr=0.3 / (8 * kT * float(w.durations.mean())), steps=300, result=False)
    Tf = Tout.cpu().numpy()
    wf = w.with_(durations=Tf)
    _, dT = s.grad(wf)
    dF = dT.cpu().numpy() + kT
    assert np.abs(dF).max() < 1e-3 * kT, dF
    F0 = oracle.solve(wf)["cost"][0] + kT * Tf.sum()
    for i in range(len(Tf)):
        for h in (-1e-3, 1e-3):
            Tp = Tf.copy()
            Tp[i] *= 1 + h
            Fp = oracle.solve(wf.with_(durations=Tp))["cost"][0] + kT * Tp.sum()
            assert Fp > F0 - 1e-9 * F0, (i, h)
