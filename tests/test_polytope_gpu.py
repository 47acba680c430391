"""GPU parity of the polytope-corridor family (Sec. III-C.1, Eq. 8-10, 18d-e)
against the oracle.

The library factorises each segment's local matrix in the eigenbasis of
sum_f n_f n_f^T, where the axis-coupling polytope rows make it block
diagonal; the oracle assembles and factorises the full 24 x 24 matrix.  Same
seeded inputs, same iteration count; tolerances 1e-9 (FP64) and 1e-4 (FP32).
"""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import T, TOL, compare, solver, to_np  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

EDGE_NS = [3, 9, 1, 0, 17, 40, 2]


def edge_case(mode, **extra):
    w = W.tiny(seed=12, N=EDGE_NS, mode=mode).with_(max_iters=150, **extra)
    return W.with_polytopes(w, F=8, M=4, seed=3, margin=(0.05, 0.5))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", ["free", "pin"])
def test_polytopes_edge_shapes(T, precision, mode):
    w = edge_case(mode)
    o = oracle.solve(w, state=True)
    assert (o["v"] > 1e-9).sum() > 20, "the polytopes must bind"
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_polytopes_with_box_and_ball_rows(T, precision):
    B = len(EDGE_NS)
    S = sum(EDGE_NS)
    w = edge_case("free", M_box=4, vbox=np.full(B, 2.5))
    rng = np.random.default_rng(4)
    off = np.concatenate([[0], np.cumsum(EDGE_NS)])
    centres = np.zeros((S, 3))
    for b in range(B):
        for g in range(off[b], off[b + 1]):
            centres[g] = 0.5 * (w.waypoints[g + b] + w.waypoints[g + b + 1])
    radii = 0.6 * np.linalg.norm(np.diff(w.waypoints, axis=0), axis=1)
    radii = np.concatenate([radii[off[b] + b: off[b + 1] + b] for b in range(B)]) + rng.uniform(0.5, 1.0, S)
    w = w.with_(M_ball=4, ball_c=centres, ball_r=radii)
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_polytope_corridor_full_size(T, precision):
    """The 1024-segment polytope corridor (F = 8 faces at 8 samples, box rows at
    16 samples), 200 iterations."""
    w = W.polytope_corridor()
    o = oracle.solve(w)
    g = to_np(solver(T, precision).solve(w))
    compare(g, o, w, TOL[precision])


def test_rotation_equivariance_on_the_gpu(T):
    w = W.with_polytopes(W.tiny(seed=5, N=[3, 6], mode="free", T_range=(0.9, 1.3), step=2.0),
                         F=6, M=4, seed=1, margin=(0.05, 0.2)).with_(max_iters=300)
    Qm, Rm = np.linalg.qr(np.random.default_rng(11).normal(size=(3, 3)))
    R = Qm * np.sign(np.diag(Rm))[None, :]
    R = R * np.sign(np.linalg.det(R))
    wr = w.with_(waypoints=w.waypoints @ R.T, start_state=w.start_state @ R.T, end_state=w.end_state @ R.T,
                 poly_n=w.poly_n @ R.T)
    s = solver(T, "fp64")
    a = to_np(s.solve(w))["coeffs"]
    b = to_np(s.solve(wr))["coeffs"]
    assert np.abs(np.einsum("ab,ibk->iak", R, a) - b).max() < 1e-9 * np.abs(a).max()


def test_host_memory_path(T):
    w = edge_case("free")
    s = solver(T, "fp64")
    gd = to_np(s.solve(w))
    gh = s.solve_host(w)
    for k in ("coeffs", "cost", "iters", "status"):
        assert np.array_equal(gd[k], gh[k]), k


def test_unsupported_combinations(T):
    s = solver(T, "fp64")
    w = edge_case("free")
    for bad in (w.with_(adaptive_rho=True), w.with_(F_poly=0)):
        with pytest.raises(T.TopError) as e:
            s.solve(bad)
        assert e.value.code in (T.TOP_E_NOTSUP, T.TOP_E_INVAL)
    with pytest.raises(T.TopError) as e:
        s.grad(w)
    assert e.value.code == T.TOP_E_NOTSUP


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cluster_and_streaming_forms_agree_on_polytopes(T, precision):
    """Polytope trajectories run in clusters (one CTA for short ones) by
    default; the streaming form computes the same iteration."""
    from test_parity_gpu import _solvers
    key = ("stream-poly", precision)
    if key not in _solvers:
        _solvers[key] = T.Solver(64, 200000, precision=precision, max_samples=16, schedule="stream")
    w = edge_case("free", M_box=4, vbox=np.full(len(EDGE_NS), 2.5))
    T.top_set_profiling(solver(T, precision).handle, True)
    a = to_np(solver(T, precision).solve(w))
    rc, ms = T.top_kernel_times(solver(T, precision).handle, 4)
    T.top_set_profiling(solver(T, precision).handle, False)
    assert ms[3] > 0.0 and ms[2] == 0.0, ms
    b = to_np(_solvers[key].solve(w))
    sc = w.durations[:, None, None] ** np.arange(8)
    tol = 1e-11 if precision == "fp64" else 2e-5
    assert np.linalg.norm((a["coeffs"] - b["coeffs"]) * sc) <= tol * np.linalg.norm(b["coeffs"] * sc)
