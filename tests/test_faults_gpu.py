"""Host-side fault injection on the GPU path: corrupt inputs and failing
allocations give error codes or per-trajectory statuses, never a device
fault, and the handle (and the GPU) stay usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_2507_10290_gb300 import workloads as W

from test_parity_gpu import T, TOL, compare, solver, to_np  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_waypoint_marks_only_its_trajectory(T, precision):
    w = W.tiny(seed=6, N=[5, 9, 4], mode="pin").with_(max_iters=40)
    P = w.waypoints.copy()
    P[5 + 1 + 3] = np.nan  # an interior waypoint of the second trajectory
    bad = w.with_(waypoints=P)
    g = to_np(solver(T, precision).solve(bad))
    assert g["status"][1] == T.TOP_NONFINITE
    ok = [0, 2]
    o = oracle.solve(w.subset(ok))
    segs = np.concatenate([np.arange(w.seg_offset[b], w.seg_offset[b + 1]) for b in ok])
    sub = {k: v[ok] for k, v in g.items() if k != "coeffs"}
    sub["coeffs"] = g["coeffs"][segs]
    compare(sub, o, w.subset(ok), TOL[precision])


def test_corrupt_offsets_and_durations_are_rejected(T):
    import torch
    s = solver(T, "fp32")
    w = W.tiny(seed=2, N=[4, 4], mode="pin")
    tensors = s.device_inputs(w)
    bad_off = tensors["seg_offset"].clone()
    bad_off[1] = 9  # 0, 9, 8: not monotone
    with pytest.raises(T.TopError) as e:
        s.solve(w, tensors={**tensors, "seg_offset": bad_off})
    assert e.value.code == T.TOP_E_INVAL
    for val in (0.0, float("inf"), float("nan")):
        T_bad = tensors["durations"].clone()
        T_bad[3] = val
        with pytest.raises(T.TopError) as e:
            s.solve(w, tensors={**tensors, "durations": T_bad})
        assert e.value.code == T.TOP_E_INVAL, val
    # still usable
    compare(to_np(s.solve(w)), oracle.solve(w), w, TOL["fp32"])
    assert torch.cuda.is_available()


def test_failing_allocation_reports_nomem(T):
    cfg = T.top_config()
    cfg.precision = T.TOP_FP32
    cfg.max_batch = 1 << 20
    cfg.max_segments = (1 << 31) - 1  # [36][S] floats alone would be ~300 GB
    cfg.max_samples = 16
    rc, h = T.top_create(cfg)
    assert rc == T.TOP_E_NOMEM and not h.value
    s = T.Solver(4, 64, precision="fp32")  # the device is fine afterwards
    w = W.tiny(seed=1, N=[3, 5], mode="free").with_(max_iters=20)
    compare(to_np(s.solve(w)), oracle.solve(w), w, TOL["fp32"])
    s.close()


def test_empty_batch_and_zero_iterations(T):
    s = solver(T, "fp64")
    w = W.tiny(seed=1, N=[0, 0], mode="pin")
    g = to_np(s.solve(w))
    assert np.all(g["status"] == 0) and np.all(g["iters"] == 0) and np.all(g["cost"] == 0)
