"""The tensor-core form of the local step's product (top_config.gemm_form).

Where the 32 segments of a warp share one inverse G (interior segments of one
trajectory with one duration), TOP_GEMM_TENSOR runs the warp's G * RHS
(8 x 96) as mma.sync m16n8k8 tiles in split TF32 (hi*hi + hi*lo + lo*hi).  It
is held to the oracle at the FP32 tolerance; where no warp shares an inverse
it must leave every result bit for bit as the CUDA-core form computes it, and
where warps do share one it must change the rounding (so the tensor path ran).
"""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import TOL, compare, scaled, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2507_10290_gb300 import build
    build.build()
    from paper_2507_10290_gb300 import top
    return top


def _solve(T, w, form):
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision="fp32", gemm_form=form)
    out = to_np(s.solve(w))
    s.close()
    return out


@pytest.mark.parametrize("mode", ["pin", "free"])
def test_shared_durations_on_tensor_cores_match_the_oracle(T, mode):
    # 48 trajectories with one duration each, 40..300 segments: most warps share one inverse
    w = W.batch(B=48, n_min=40, n_max=300, shared_T=True).with_(max_iters=200)
    w = w.with_(mode=mode)
    o = oracle.solve(w)
    g = _solve(T, w, "tensor")
    compare(g, o, w, TOL["fp32"])
    c = _solve(T, w, "cuda_cores")
    a, b = scaled(g["coeffs"], w.durations), scaled(c["coeffs"], w.durations)
    diff = np.linalg.norm(a - b) / np.linalg.norm(b)
    # a different rounding (so the tensor path ran), each within the FP32 tolerance of the oracle
    assert 0.0 < diff < 2 * TOL["fp32"], diff


def test_no_shared_inverse_leaves_results_bit_identical(T):
    # per-segment durations: no warp shares an inverse, so every warp takes the CUDA-core product
    w = W.batch(B=24, n_min=8, n_max=200).with_(max_iters=100)
    g = _solve(T, w, "tensor")
    c = _solve(T, w, "cuda_cores")
    for k in ("coeffs", "cost", "r_primal", "r_dual", "iters", "status"):
        assert np.array_equal(g[k], c[k]), k


def _ragged_shared(Ns=(1, 2, 3, 33, 34, 35, 64, 65, 66, 97, 130, 31), mode="pin"):
    # lengths around warp and trajectory boundaries, one duration per trajectory
    w = W.tiny(seed=7, N=list(Ns), mode=mode)
    return w.with_(durations=np.repeat(np.linspace(0.6, 1.4, len(Ns)), Ns))


def test_ragged_shared_batch(T):
    # warps that straddle trajectories or hold their first / last segments take the CUDA-core product
    w = _ragged_shared().with_(max_iters=300)
    o = oracle.solve(w)
    compare(_solve(T, w, "tensor"), o, w, TOL["fp32"])


def test_stopping_rule_with_tensor_cores(T):
    # trajectories stop at different iterations: a warp with stopped segments leaves the tensor path
    # (FREE waypoints: the oracle stops these between 1 and 6157 iterations)
    w = _ragged_shared(Ns=(1, 33, 34, 35, 64, 65, 66, 97, 130, 31), mode="free").with_(max_iters=20000, eps=1e-3)
    g = _solve(T, w, "tensor")
    c = _solve(T, w, "cuda_cores")
    assert np.all(g["status"] == 0) and np.all(c["status"] == 0)
    assert len(set(g["iters"].tolist())) > 5  # stopped at different iterations
    a, b = scaled(g["coeffs"], w.durations), scaled(c["coeffs"], w.durations)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-3


def test_autotune_times_both_forms(T):
    w = W.batch(B=64, shared_T=True)
    s = T.Solver(max_batch=w.B, max_segments=w.S, precision="fp32")
    best, caps, forms = s.autotune(w, iters=20, gemm=True)
    assert best in caps and caps[best] > 0
    assert forms["cuda_cores"] > 0 and forms["tensor"] > 0
    s.close()
    # with box rows the choice does not apply: both entries negative
    wb = W.single_box()
    s = T.Solver(max_batch=1, max_segments=wb.S, precision="fp32")
    _, _, forms = s.autotune(wb, iters=5, gemm=True)
    assert forms["cuda_cores"] < 0 and forms["tensor"] < 0
    s.close()
