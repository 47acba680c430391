"""top_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (a host framework whose allocator forbids side allocations, a
real-time loop that must not call cudaMalloc, a process with a fixed memory
budget) cannot create a handle, because top_create allocates a workspace.
top_solve_noalloc keeps its scratch in one fixed-size device array instead.
This test calls it through the C ABI and checks it against the handle-based
top_solve and against the CPU oracle on the same inputs, twice in a row (the
second call reuses the array the first one left behind; around it the free
device memory and torch's reserved memory must not change), and checks that a
problem beyond the fixed limit is rejected with TOP_E_LIMIT.  The file is
named to run last.
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


def noalloc_solve(T, w, precision, memory=None):
    """One call of top_solve_noalloc on freshly allocated inputs and outputs;
    with `memory` (a list), appends the (free device bytes, torch reserved
    bytes) seen just before and just after the call."""
    import torch
    s = T.Solver.__new__(T.Solver)  # marshalling helpers only; no handle is created
    s.torch = torch
    tensors = s.device_inputs(w)
    out = s.alloc_result(w.B, w.S, w.max_iters)
    pb = s.make_problem(w, tensors, T.TOP_MEM_DEVICE)
    r = T.Solver.result_struct(out)
    prec = T.TOP_FP64 if precision == "fp64" else T.TOP_FP32
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved())
    rc = T.top_solve_noalloc(pb, r, prec, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved())
    if memory is not None:
        memory.append((before, after))
    return rc, {k: v.cpu().numpy() for k, v in out.items()}


def scaled(c, durations):
    return c * np.asarray(durations)[:, None, None] ** np.arange(8)[None, None, :]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_top_solve_twice(T, precision):
    cases = [
        W.tiny(seed=12, N=[1, 0, 2, 3, 33, 31, 64, 5, 127], mode="pin").with_(max_iters=80),
        W.single_box(),
    ]
    for w in cases:
        ref_solver = T.Solver(max_batch=w.B, max_segments=w.S, precision=precision, max_samples=16)
        ref = {k: v.cpu().numpy() for k, v in ref_solver.solve(w).items()}
        ref_solver.close()
        orc = oracle.solve(w)
        memory = []
        for call in range(2):
            rc, got = noalloc_solve(T, w, precision, memory)
            assert rc == T.TOP_OK, (call, T.top_strerror(rc))
            for other in (ref, orc):  # the handle-based solve and the CPU oracle
                err = np.linalg.norm(scaled(got["coeffs"] - other["coeffs"], w.durations)) / \
                    np.linalg.norm(scaled(other["coeffs"], w.durations))
                assert err <= TOL[precision], (call, err)
                assert np.max(np.abs(got["cost"] - other["cost"])) <= TOL[precision] * np.max(np.abs(other["cost"]))
                assert np.array_equal(got["iters"], other["iters"]) and np.array_equal(got["status"], other["status"])
        # the second call finds its array resident and allocates nothing
        before, after = memory[1]
        assert before == after, (before, after)


def test_noalloc_rejects_problems_beyond_its_limit(T):
    n = T.TOP_NOALLOC_MAX_SEGMENTS // 256 + 1
    w = W.batch(B=n, fixed_N=256, seed=3).with_(max_iters=2)
    assert w.S > T.TOP_NOALLOC_MAX_SEGMENTS
    rc, _ = noalloc_solve(T, w, "fp32")
    assert rc == T.TOP_E_LIMIT
    # and a valid call still works afterwards
    small = W.tiny(seed=4, N=[6, 9], mode="free").with_(max_iters=20)
    rc, _ = noalloc_solve(T, small, "fp32")
    assert rc == T.TOP_OK
