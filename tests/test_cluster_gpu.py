"""GPU parity of the cluster-resident form (one trajectory per thread-block
cluster, distributed shared memory at the CTA boundaries) against the oracle.

A handle with 64 segments per CTA sends trajectories of 65 .. 1024 segments
through clusters of 2 .. 16 CTAs, while shorter ones stay resident and longer
ones stream; every form must agree with the oracle (FP64 1e-9, FP32 1e-4) and
the cluster kernel must actually have run.
"""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import T, TOL, compare, to_np  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

NS = [0, 1, 5, 64, 65, 128, 129, 200, 333, 1024, 1025, 40]


def small_cta_solver(T, precision, schedule="auto"):
    from test_parity_gpu import _solvers
    key = ("cta64", precision, schedule)
    if key not in _solvers:
        _solvers[key] = T.Solver(64, 20000, precision=precision, max_samples=16, segs_per_cta=64, schedule=schedule)
    return _solvers[key]


def solve_profiled(T, s, w, **kw):
    T.top_set_profiling(s.handle, True)
    g = to_np(s.solve(w, **kw))
    rc, ms = T.top_kernel_times(s.handle, 4)
    T.top_set_profiling(s.handle, False)
    return g, ms


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", ["pin", "free"])
def test_cluster_form_matches_the_oracle(T, precision, mode):
    w = W.tiny(seed=21, N=NS, mode=mode).with_(max_iters=120)
    o = oracle.solve(w)
    g, ms = solve_profiled(T, small_cta_solver(T, precision), w)
    assert ms[3] > 0.0, "the cluster-resident kernel did not run"
    assert ms[2] > 0.0, "the 1025-segment trajectory must stream"
    compare(g, o, w, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cluster_form_with_box_and_ball_rows(T, precision):
    w = W.corridor(N=300).with_(max_iters=120)
    o = oracle.solve(w)
    g, ms = solve_profiled(T, small_cta_solver(T, precision), w)
    assert ms[3] > 0.0
    compare(g, o, w, TOL[precision])


def test_cluster_stopping_rule_and_history_fp64(T):
    w = W.tiny(seed=1, N=[150, 70, 300], mode="free", T_range=(0.8, 1.6)).with_(eps=1e-3, max_iters=20000)
    o = oracle.solve(w, history=True)
    g, ms = solve_profiled(T, small_cta_solver(T, "fp64"), w, history=True, check_every=1)
    assert ms[3] > 0.0
    compare(g, o, w, TOL["fp64"])
    for b in range(w.B):
        kb = int(o["iters"][b])
        scale = np.abs(o["history"][:kb, b]).max(axis=0)
        assert np.all(np.abs(g["history"][:kb, b] - o["history"][:kb, b]) <= 1e-9 * scale)


def test_cluster_and_streaming_forms_agree(T):
    w = W.tiny(seed=4, N=[700, 90], mode="pin").with_(max_iters=100)
    a = to_np(small_cta_solver(T, "fp64").solve(w))
    b = to_np(small_cta_solver(T, "fp64", schedule="stream").solve(w))
    sc = w.durations[:, None, None] ** np.arange(8)
    assert np.linalg.norm((a["coeffs"] - b["coeffs"]) * sc) <= 1e-11 * np.linalg.norm(a["coeffs"] * sc)
    assert np.array_equal(a["iters"], b["iters"])


def test_default_capacity_corridor_runs_in_clusters(T):
    """The 1024-segment corridor (box + ball rows at 16 samples) on the default
    handle: more segments than one CTA holds, so it runs in a cluster."""
    from test_parity_gpu import solver
    w = W.corridor()
    s = solver(T, "fp32")
    g, ms = solve_profiled(T, s, w)
    assert ms[3] > 0.0
    o = oracle.solve(w)
    compare(g, o, w, TOL["fp32"])


@pytest.mark.parametrize("N", [600, 2600])
def test_lanes_per_segment_corridors_fp32(T, N):
    """FP32 corridors with box and ball rows (32 sample rows per segment): the
    cluster kernel splits each segment's rows over 4 lanes (N = 600: 128
    segments per CTA) or 2 (N = 2600: longer than 16 CTAs of 128), and must
    still match the oracle with no streaming."""
    from test_parity_gpu import solver
    w = W.corridor(N=N).with_(max_iters=150)
    g, ms = solve_profiled(T, solver(T, "fp32"), w)
    assert ms[3] > 0.0 and ms[2] == 0.0
    o = oracle.solve(w)
    compare(g, o, w, TOL["fp32"])


@pytest.mark.parametrize("mode", ["pin", "free"])
def test_cluster_form_with_adaptive_rho_fp64(T, mode):
    """Residual balancing (Eq. 22) inside clusters: rank 0 applies the rule,
    every CTA rescales its state; final rho identical to the oracle's."""
    w = W.tiny(seed=21, N=NS, mode=mode).with_(max_iters=150, adaptive_rho=True)
    o = oracle.solve(w)
    g, ms = solve_profiled(T, small_cta_solver(T, "fp64"), w)
    assert ms[3] > 0.0
    compare(g, o, w, TOL["fp64"])
    assert np.array_equal(g["rho"], o["rho_final"]), (g["rho"], o["rho_final"])
    c = W.corridor(N=300).with_(max_iters=150, adaptive_rho=True)
    o = oracle.solve(c)
    g, ms = solve_profiled(T, small_cta_solver(T, "fp64"), c)
    assert ms[3] > 0.0
    compare(g, o, c, TOL["fp64"])
    assert np.array_equal(g["rho"], o["rho_final"])


def test_autotuner_picks_a_fitting_capacity_and_keeps_parity(T):
    w = W.batch(B=48, seed=7).with_(max_iters=40)
    s = T.Solver(64, 30000, precision="fp32", max_samples=0)
    best, table = s.autotune(w, iters=10)
    assert best in table and table[best] > 0
    assert all(v < 0 or v >= table[best] for v in table.values())
    o = oracle.solve(w)
    compare(to_np(s.solve(w)), o, w, TOL["fp32"])
    s.close()


def test_graph_capture_replays_top_solve(T):
    """Capture-safe mode: a whole top_solve (precompute, resident packs and a
    cluster) recorded into a CUDA graph and replayed gives the same outputs."""
    import torch
    w = W.tiny(seed=3, N=[40, 7, 300, 64, 12], mode="pin").with_(max_iters=60)
    s = T.Solver(8, 1000, precision="fp32", max_samples=0, segs_per_cta=64)
    tensors = s.device_inputs(w)
    out = s.alloc_result(w.B, w.S, 60)
    off = np.ascontiguousarray(w.seg_offset, dtype=np.int32)
    assert T.top_set_layout(s.handle, w.B, off) == T.TOP_OK
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        s.solve(w, tensors=tensors, out=out, stream=stream.cuda_stream)  # workspace, plan, attributes
    torch.cuda.synchronize()
    assert T.top_sync(s.handle, stream.cuda_stream) == T.TOP_OK
    ref = {k: v.clone() for k, v in out.items()}
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        s.solve(w, tensors=tensors, out=out, stream=stream.cuda_stream)
    for v in out.values():
        v.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert T.top_sync(s.handle, stream.cuda_stream) == T.TOP_OK
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    o = oracle.solve(w)
    compare(to_np(out), o, w, TOL["fp32"])
    assert T.top_set_layout(s.handle, 0, None) == T.TOP_OK
    s.close()


def test_launch_count(T):
    """top_launch_count: a fixed-rho solve whose trajectories all fit one CTA
    launches fill (the final rho), mark, invert, copy and resident; a long one
    adds one cluster launch; the streaming form (three trajectories, 100
    iterations, residuals on the last only) launches the four precompute
    kernels, its set-up, one fused local step per iteration (two kernels per
    iteration, local step and junction, with one launch per phase), the last
    iteration's junction update and residual evaluation, and the output."""
    s = small_cta_solver(T, "fp32")
    w = W.tiny(seed=2, N=[5, 9, 40], mode="pin").with_(max_iters=30)
    c0 = T.top_launch_count(s.handle)
    s.solve(w)
    assert T.top_launch_count(s.handle) - c0 == 5
    w2 = W.tiny(seed=2, N=[5, 200], mode="pin").with_(max_iters=30)  # 200 > 64 per CTA: a cluster
    c0 = T.top_launch_count(s.handle)
    g, ms = solve_profiled(T, s, w2)
    assert ms[3] > 0.0
    assert T.top_launch_count(s.handle) - c0 == 6
    st = small_cta_solver(T, "fp32", schedule="stream")
    c0 = T.top_launch_count(st.handle)
    st.solve(w.with_(max_iters=100))
    assert T.top_launch_count(st.handle) - c0 == 4 + 1 + 100 + 3 + 2
    sp = T.Solver(64, 20000, precision="fp32", max_samples=16, segs_per_cta=64, schedule="stream",
                  stream_form="phases")
    c0 = T.top_launch_count(sp.handle)
    sp.solve(w.with_(max_iters=100))
    assert T.top_launch_count(sp.handle) - c0 == 4 + 1 + 2 * 100 + 2 + 2
    sp.close()
    assert T.top_launch_count(None) == -1
