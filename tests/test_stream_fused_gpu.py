"""The fused streaming iteration against one launch per phase.

With top_config.stream_form = TOP_STREAM_FUSED (the default) an iteration
without a residual evaluation leaves its junction update (Eq. 18b-c) to the
start of the next iteration's local step, which reads the junction state and
the segments' end values from one half of the workspace and writes the other.
The arithmetic is the same as with TOP_STREAM_PHASES (a local-step launch and a
junction launch per iteration), so every result must agree bit for bit: on the
closed-form families, the polytope rows, the numerical step with violated
bounds (work list of the warp form), with and without periodic residual checks
and the stopping rule, over more iterations than one recorded graph block.
"""
import numpy as np
import pytest

from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2507_10290_gb300 import build
    build.build()
    from paper_2507_10290_gb300 import top
    return top


def _speed_numeric():
    g0 = W.speed_limit(seed=3, N=64, M=8)
    chord = np.linalg.norm(np.diff(g0.waypoints, axis=0), axis=1) / g0.durations
    return W.speed_limit(seed=3, N=64, M=8, inner="numeric", max_iters=90, vmax=0.8 * float(np.median(chord)))


CASES = {
    "batch PIN": (lambda: W.batch(B=12, seed=2, n_min=300, n_max=700).with_(max_iters=75), {}),
    "batch FREE to eps, checks every 10": (
        lambda: W.batch(B=12, seed=2, n_min=300, n_max=700).with_(mode="free", max_iters=260, eps=2e-3),
        {"check_every": 10, "history": True}),
    "batch FREE, checks every 3": (
        lambda: W.batch(B=6, seed=4, n_min=200, n_max=400).with_(mode="free", max_iters=120, eps=1e-9),
        {"check_every": 3}),
    "corridor box + ball": (lambda: W.corridor(N=600).with_(max_iters=80), {}),
    "polytope corridor": (lambda: W.polytope_corridor(N=300).with_(max_iters=70), {}),
    "numerical step, bound active": (_speed_numeric, {}),
}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(CASES))
def test_fused_iterations_equal_one_launch_per_phase(T, precision, name):
    make, kw = CASES[name]
    w = make()
    out = {}
    for form in ("fused", "phases"):
        s = T.Solver(max_batch=w.B, max_segments=w.S, precision=precision, max_samples=16, schedule="stream",
                     stream_form=form)
        T.top_set_profiling(s.handle, True)
        out[form] = to_np(s.solve(w, **kw))
        rc, ms = T.top_kernel_times(s.handle, 4)
        assert ms[2] > 0.0 and ms[1] == 0.0 and ms[3] == 0.0, ms  # the streaming form ran
        s.close()
    for k in out["phases"]:  # (the history holds NaN on the iterations without an evaluation)
        a, b = out["fused"][k], out["phases"][k]
        assert np.array_equal(a, b, equal_nan=a.dtype.kind == "f"), (name, k)
