"""The seeded input generators shared by the oracle and the GPU path (host
logic only): sizes and layouts the kernels rely on, the geometric promises
each recipe makes (corridors contain the chord ends, consecutive balls and
polytopes overlap at the shared waypoint, repaired durations respect the
speed limits), determinism per trajectory stream, and subset consistency."""
import numpy as np

from paper_2507_10290_gb300 import workloads as W


def test_batch_layout_and_per_trajectory_streams():
    w = W.batch(B=64)
    off = w.seg_offset
    assert off[0] == 0 and np.all(np.diff(off) >= 8) and np.all(np.diff(off) <= 512)
    assert w.waypoints.shape == (w.S + w.B, 3) and w.durations.shape == (w.S,)
    assert np.all((w.durations >= 0.3) & (w.durations <= 1.5))
    # trajectory b draws from its own stream: a smaller batch reproduces its prefix
    v = W.batch(B=16)
    assert np.array_equal(v.seg_offset, off[:17])
    assert np.array_equal(v.durations, w.durations[:off[16]])
    # rest boundary states at the trajectory's first and last waypoint
    for b in range(w.B):
        assert np.array_equal(w.start_state[b, 0], w.waypoints[off[b] + b])
        assert np.array_equal(w.end_state[b, 0], w.waypoints[off[b + 1] + b])
        assert not w.start_state[b, 1:].any() and not w.end_state[b, 1:].any()


def test_shared_durations_are_constant_per_trajectory():
    w = W.batch(B=32, shared_T=True)
    off = w.seg_offset
    for b in range(w.B):
        T = w.durations[off[b]:off[b + 1]]
        assert np.all(T == T[0])
    assert len(np.unique(w.durations)) == w.B


def test_subset_keeps_every_per_segment_and_per_trajectory_array():
    w = W.with_polytopes(W.batch(B=12, n_min=3, n_max=9), F=7, M=4, seed=2)
    ids = [7, 0, 11]
    s = w.subset(ids)
    off = w.seg_offset
    segs = np.concatenate([np.arange(off[b], off[b + 1]) for b in ids])
    pts = np.concatenate([np.arange(off[b] + b, off[b + 1] + b + 1) for b in ids])
    assert np.array_equal(s.durations, w.durations[segs])
    assert np.array_equal(s.waypoints, w.waypoints[pts])
    assert np.array_equal(s.poly_n, w.poly_n[segs]) and np.array_equal(s.poly_h, w.poly_h[segs])
    assert np.array_equal(s.start_state, w.start_state[ids])
    assert np.array_equal(np.diff(s.seg_offset), np.diff(off)[ids])


def test_corridor_balls_contain_the_chord_ends_and_overlap():
    w = W.corridor(N=256)
    P, c, r = w.waypoints, w.ball_c, w.ball_r
    for i in range(w.S):
        assert np.linalg.norm(P[i] - c[i]) < r[i] and np.linalg.norm(P[i + 1] - c[i]) < r[i]
    # consecutive balls share the waypoint between them
    for i in range(w.S - 1):
        assert np.linalg.norm(c[i] - c[i + 1]) < r[i] + r[i + 1]
    # the repaired durations allow the chord at 80 % of the axis speed limit
    chord_speed = np.max(np.abs(np.diff(P, axis=0)), axis=1) / w.durations
    assert np.all(chord_speed <= 0.8 * w.vbox[0] + 1e-12)


def test_polytopes_contain_both_chord_ends_with_unit_normals():
    w = W.with_polytopes(W.batch(B=6, n_min=4, n_max=12), F=9, M=4, seed=5)
    off = w.seg_offset
    assert np.allclose(np.linalg.norm(w.poly_n, axis=2), 1.0)
    for b in range(w.B):
        for g in range(off[b], off[b + 1]):
            ends = w.waypoints[[g + b, g + b + 1]]
            assert np.all(w.poly_n[g] @ ends.T < w.poly_h[g][:, None])
    # the first six faces are the two sides of an orthonormal frame: bounded polytopes
    R = w.poly_n[0, :3]
    assert np.allclose(R @ R.T, np.eye(3)) and np.allclose(w.poly_n[0, 3:6], -R)


def test_curve_boundary_states_follow_the_trefoil():
    w = W.curve(N=32)
    Ttot = w.notes["T_total"]
    assert np.isclose(w.durations.sum(), Ttot) and np.allclose(w.durations, Ttot / 32)
    # the analytic derivative matches a central difference of the curve itself
    h = 1e-6
    for order in (1, 2):
        fd = (W.trefoil([0.3 + h], order - 1) - W.trefoil([0.3 - h], order - 1)) / (2 * h)
        assert np.allclose(fd, W.trefoil([0.3], order), rtol=1e-6, atol=1e-6)
    assert np.allclose(w.start_state[0, 1], W.trefoil([0.0], 1)[0] / Ttot)
    assert np.allclose(w.waypoints[[0, -1]], W.trefoil([0.0, 1.0], 0))


def test_generators_are_deterministic():
    for make in (lambda: W.single_box(), lambda: W.corridor(N=64), lambda: W.general(N=200),
                 lambda: W.speed_limit(N=32), lambda: W.polytope_corridor(N=32)):
        a, b = make(), make()
        for k in ("waypoints", "durations", "start_state", "end_state", "ball_r", "poly_h"):
            x, y = getattr(a, k), getattr(b, k)
            assert (x is None and y is None) or np.array_equal(x, y), k
