"""Seeded synthetic trajectory-optimisation inputs.

This module draws inputs only: waypoints, segment durations, boundary
states and constraint parameters.  It holds none of the optimiser's
arithmetic, so that both the CUDA library and the CPU oracle can be fed the
same arrays.

The paper's own workloads (RRT* paths, FIRI corridors built from point-cloud
maps, flight logs; Sec. IV) are not available.  The generators below stand
in for them with the shapes the paper's problem statement fixes (Sec. III-B,
Eq. 2: waypoints P in R^{3 x (N+1)}, durations T_i > 0, rest boundary states
of order p-1 = 3) and the sizes of the five benchmark workloads:

  single_box      1 trajectory, N = 8,  P ~ U[-10,10]^3, T ~ U[0.5,2],
                  FREE waypoints, |v_axis| <= 3 at 8 samples per segment
  corridor        1 trajectory, N = 1024, random-walk waypoints (step
                  N(0, 1.5^2) per axis), T ~ U[0.3,1.5], FREE waypoints,
                  |v_axis| <= 3 and ball corridors ||p - o_i|| <= r_i at 16
                  samples per segment
  batch           4096 trajectories, N_b ~ U{8..512}, random-walk waypoints,
                  T ~ U[0.3,1.5] per segment (or one T per trajectory),
                  PIN waypoints, no inequality constraints
  grad_batch      256 x N = 256, as `batch`, for the adjoint
  general         1 trajectory, N = 100000, random-walk waypoints, PIN
                  waypoints, ||v|| <= 4 and ||a|| <= 8 at 16 samples per
                  segment through the numerical (L-BFGS) local step
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

P_ORDER = 4  # boundary states carry derivative orders 0..3


@dataclass
class Workload:
    """A batch of trajectory problems in the library's input layout.

    seg_offset  int32 [B+1]   trajectory b owns segments seg_offset[b] .. seg_offset[b+1]-1
    waypoints   f64 [S+B, 3]  trajectory b owns rows seg_offset[b]+b .. seg_offset[b+1]+b
    durations   f64 [S]       T_i > 0
    start_state f64 [B, 4, 3] derivative order r (0..3) x axis
    end_state   f64 [B, 4, 3]
    """

    name: str
    seg_offset: np.ndarray
    waypoints: np.ndarray
    durations: np.ndarray
    start_state: np.ndarray
    end_state: np.ndarray
    mode: str = "pin"          # "pin" | "free"
    inner: str = "closed"      # "closed" | "numeric"
    rho: float = 1.0
    eps: float = 0.0
    max_iters: int = 200
    M_box: int = 0
    vbox: Optional[np.ndarray] = None      # [B]
    M_ball: int = 0
    ball_c: Optional[np.ndarray] = None    # [S, 3]
    ball_r: Optional[np.ndarray] = None    # [S]
    M_vn: int = 0
    vnorm: Optional[np.ndarray] = None     # [B]
    M_gen: int = 0
    gen_vmax: Optional[np.ndarray] = None  # [B]
    gen_amax: Optional[np.ndarray] = None  # [B]
    M_poly: int = 0                          # polytope corridor: samples per segment
    F_poly: int = 0                          # faces per segment polytope
    poly_n: Optional[np.ndarray] = None      # [S, F, 3] face normals
    poly_h: Optional[np.ndarray] = None      # [S, F] offsets: n_f . p(t_ij) <= h_f
    adaptive_rho: bool = False  # UpdateRho of Eq. 22 (mu, tau_incr, tau_decr as the paper: 10, 1.1, 1.1)
    rho_mu: float = 10.0
    rho_tau_incr: float = 1.1
    rho_tau_decr: float = 1.1
    lbfgs_mem: int = 0          # numerical step settings (0 = the solver's default)
    lbfgs_max_iters: int = 0
    lbfgs_tol: float = 0.0
    notes: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.seg_offset.shape[0] - 1)

    @property
    def S(self) -> int:
        return int(self.seg_offset[-1])

    def n_segments(self) -> np.ndarray:
        return np.diff(self.seg_offset).astype(np.int64)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def subset(self, traj_ids) -> "Workload":
        """The sub-batch made of the listed trajectories, in that order."""
        traj_ids = [int(b) for b in traj_ids]
        off = self.seg_offset
        segs, pts, offs = [], [], [0]
        for b in traj_ids:
            s0, s1 = int(off[b]), int(off[b + 1])
            segs.append(np.arange(s0, s1))
            pts.append(np.arange(s0 + b, s1 + b + 1))
            offs.append(offs[-1] + (s1 - s0))
        seg_idx = np.concatenate(segs) if segs else np.zeros(0, np.int64)
        pt_idx = np.concatenate(pts) if pts else np.zeros(0, np.int64)

        def per_b(x):
            return None if x is None else np.ascontiguousarray(x[traj_ids])

        def per_s(x):
            return None if x is None else np.ascontiguousarray(x[seg_idx])

        return replace(
            self,
            name=f"{self.name}[subset {len(traj_ids)}]",
            seg_offset=np.asarray(offs, np.int32),
            waypoints=np.ascontiguousarray(self.waypoints[pt_idx]),
            durations=np.ascontiguousarray(self.durations[seg_idx]),
            start_state=per_b(self.start_state),
            end_state=per_b(self.end_state),
            vbox=per_b(self.vbox),
            ball_c=per_s(self.ball_c),
            ball_r=per_s(self.ball_r),
            vnorm=per_b(self.vnorm),
            gen_vmax=per_b(self.gen_vmax),
            gen_amax=per_b(self.gen_amax),
            poly_n=per_s(self.poly_n),
            poly_h=per_s(self.poly_h),
        )


def _rest_states(first: np.ndarray, last: np.ndarray):
    """Rest boundary states (position given, velocity/acceleration/jerk zero)."""
    B = first.shape[0]
    s = np.zeros((B, P_ORDER, 3))
    e = np.zeros((B, P_ORDER, 3))
    s[:, 0, :] = first
    e[:, 0, :] = last
    return s, e


def _random_walk(rng: np.random.Generator, n: int, step: float = 1.5) -> np.ndarray:
    steps = rng.normal(0.0, step, size=(n, 3))
    return np.concatenate([np.zeros((1, 3)), np.cumsum(steps, axis=0)], axis=0)


def single_box(seed: int = 0) -> Workload:
    """1 trajectory, N = 8, FREE waypoints, |v_axis| <= 3 at 8 samples."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(-10.0, 10.0, size=(9, 3))
    T = rng.uniform(0.5, 2.0, size=8)
    # duration repair: the straight line must be possible at 80% of the limit
    alpha = max(1.0, 1.25 * float(np.max(np.abs(P[8] - P[0]))) / (3.0 * float(T.sum())))
    T = T * alpha
    s, e = _rest_states(P[None, 0], P[None, 8])
    return Workload(
        name="single_box N=8", seg_offset=np.array([0, 8], np.int32), waypoints=P,
        durations=T, start_state=s, end_state=e, mode="free", rho=1.0, max_iters=200,
        M_box=8, vbox=np.array([3.0]), notes={"duration_scale": alpha},
    )


def corridor(seed: int = 0, N: int = 1024) -> Workload:
    """1 trajectory, N segments, FREE waypoints, box velocity + ball corridors at 16 samples."""
    rng = np.random.default_rng(seed)
    P = _random_walk(rng, N)
    T = rng.uniform(0.3, 1.5, size=N)
    d = np.diff(P, axis=0)
    T = np.maximum(T, 1.25 * np.max(np.abs(d), axis=1) / 3.0)
    centres = 0.5 * (P[:-1] + P[1:])
    r_draw = rng.uniform(1.0, 3.0, size=N)
    radii = np.maximum(r_draw, 0.55 * np.linalg.norm(d, axis=1))
    s, e = _rest_states(P[None, 0], P[None, N])
    return Workload(
        name=f"corridor N={N}", seg_offset=np.array([0, N], np.int32), waypoints=P,
        durations=T, start_state=s, end_state=e, mode="free", rho=1.0, max_iters=200,
        M_box=16, vbox=np.array([3.0]), M_ball=16, ball_c=centres, ball_r=radii,
        notes={"radius_clamped": int(np.sum(radii > r_draw))},
    )


def batch(seed: int = 0, B: int = 4096, n_min: int = 8, n_max: int = 512,
          shared_T: bool = False, fixed_N: Optional[int] = None) -> Workload:
    """B trajectories with uneven segment counts, PIN waypoints, no inequalities.

    Trajectory b draws its waypoints and durations from its own stream
    (seed, b), so any subset reproduces exactly.
    """
    master = np.random.default_rng(seed)
    if fixed_N is None:
        Nb = master.integers(n_min, n_max + 1, size=B)
    else:
        Nb = np.full(B, int(fixed_N))
    off = np.zeros(B + 1, np.int64)
    off[1:] = np.cumsum(Nb)
    S = int(off[-1])
    P = np.empty((S + B, 3))
    T = np.empty(S)
    for b in range(B):
        rb = np.random.default_rng([seed, b])
        n = int(Nb[b])
        P[off[b] + b: off[b + 1] + b + 1] = _random_walk(rb, n)
        if shared_T:
            T[off[b]:off[b + 1]] = rb.uniform(0.3, 1.5)
        else:
            T[off[b]:off[b + 1]] = rb.uniform(0.3, 1.5, size=n)
    first = P[off[:-1] + np.arange(B)]
    last = P[off[1:] + np.arange(B)]
    s, e = _rest_states(first, last)
    kind = "shared-T" if shared_T else "per-segment T"
    return Workload(
        name=f"batch B={B} S={S} ({kind})", seg_offset=off.astype(np.int32), waypoints=P,
        durations=T, start_state=s, end_state=e, mode="pin", rho=1.0, max_iters=300,
    )


def grad_batch(seed: int = 0, B: int = 256, N: int = 256) -> Workload:
    """B x N trajectories for the adjoint through K = 100 iterations."""
    w = batch(seed=seed, B=B, fixed_N=N)
    return w.with_(name=f"grad_batch B={B} N={N}", max_iters=100)


def general(seed: int = 0, N: int = 100000, v_nom: float = 1.0) -> Workload:
    """1 trajectory, N segments, PIN waypoints, ||v|| <= 4, ||a|| <= 8 by the numerical step.

    In PIN mode the feasible set of the equality constraints is one point
    (the unique C^6 degree-7 spline through the waypoints), so the norm
    bounds can only be met if that spline meets them.  Durations are
    therefore drawn as U[0.3, 1.5] and lengthened to at least
    ||P_i - P_{i-1}|| / v_nom (a nominal speed a quarter of the bound).
    """
    rng = np.random.default_rng(seed)
    P = _random_walk(rng, N)
    T = rng.uniform(0.3, 1.5, size=N)
    T = np.maximum(T, np.linalg.norm(np.diff(P, axis=0), axis=1) / v_nom)
    s, e = _rest_states(P[None, 0], P[None, N])
    return Workload(
        name=f"general N={N}", seg_offset=np.array([0, N], np.int32), waypoints=P,
        durations=T, start_state=s, end_state=e, mode="pin", inner="numeric", rho=1.0,
        max_iters=200, M_gen=16, gen_vmax=np.array([4.0]), gen_amax=np.array([8.0]),
    )


def with_polytopes(w: Workload, F: int = 8, M: int = 8, seed: int = 0, margin=(0.3, 1.5)) -> Workload:
    """Polytope corridors around every segment's chord, standing in for the
    paper's FIRI corridors (which need point-cloud maps): per segment, the six
    faces of a randomly rotated cube plus F - 6 faces with random unit normals,
    each offset to the farther chord end plus a margin ~ U[margin], so both
    waypoints (hence the chord) lie inside and consecutive polytopes overlap
    at the shared waypoint.  Normals are never axis-aligned in general, so the
    rows n_f^T (x) beta(t)^T couple the three axes."""
    if F < 6:
        raise ValueError("F >= 6 (the rotated cube keeps every polytope bounded)")
    rng = np.random.default_rng([seed, 7])
    off = np.asarray(w.seg_offset)
    S = int(off[-1])
    n = np.zeros((S, F, 3))
    h = np.zeros((S, F))
    for b in range(len(off) - 1):
        for g in range(int(off[b]), int(off[b + 1])):
            Qm, Rm = np.linalg.qr(rng.normal(size=(3, 3)))
            Qm = Qm * np.sign(np.diag(Rm))[None, :]
            faces = np.concatenate([Qm.T, -Qm.T, rng.normal(size=(F - 6, 3))], axis=0)
            faces /= np.linalg.norm(faces, axis=1, keepdims=True)
            ends = w.waypoints[[g + b, g + b + 1]]                 # [2, 3]
            n[g] = faces
            h[g] = (faces @ ends.T).max(axis=1) + rng.uniform(margin[0], margin[1], size=F)
    return w.with_(name=f"{w.name} + polytopes F={F} M={M}", M_poly=M, F_poly=F, poly_n=n, poly_h=h)


def polytope_corridor(seed: int = 0, N: int = 1024, F: int = 8, M: int = 8) -> Workload:
    """1 trajectory, N segments: the corridor recipe's random walk and
    durations, FREE waypoints, |v_axis| <= 3 at 16 samples, and a polytope of
    F faces around every chord sampled at M points (with_polytopes)."""
    w = corridor(seed=seed, N=N).with_(M_ball=0, ball_c=None, ball_r=None)
    return with_polytopes(w, F=F, M=M, seed=seed).with_(name=f"polytope_corridor N={N} F={F} M={M}")


def trefoil(s, order: int = 0, scale: float = 5.0) -> np.ndarray:
    """Derivative `order` (0..3) with respect to s of the reference curve
    r(s) = scale (sin 2 pi s + 2 sin 4 pi s, cos 2 pi s - 2 cos 4 pi s, -sin 6 pi s),
    s in [0, 1]: a trefoil knot, the stand-in for the paper's parameterized
    curve.  Returns [len(s), 3]."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))

    def d(fn, w):  # order-th derivative of fn(w s), fn in {sin, cos}
        ph = order * np.pi / 2.0
        base = np.sin(w * s + ph) if fn == "sin" else np.cos(w * s + ph)
        return w ** order * base

    tp = 2.0 * np.pi
    x = d("sin", tp) + 2.0 * d("sin", 2 * tp)
    y = d("cos", tp) - 2.0 * d("cos", 2 * tp)
    z = -d("sin", 3 * tp)
    return scale * np.stack([x, y, z], axis=1)


def curve(N: int = 256, T_total: Optional[float] = None, scale: float = 5.0, max_iters: int = 3000) -> Workload:
    """The segment-count experiment (Sec. IV-A.2): N + 1 points sampled
    uniformly in the parameter of the reference curve (trefoil), PIN waypoints
    so the trajectory passes through them, uniform durations T_total / N
    (default 0.5 s per segment, which keeps T^-r moderate at every N), and the
    curve's own velocity, acceleration and jerk (time t = s T_total) as the
    boundary states."""
    if T_total is None:
        T_total = 0.5 * N
    sN = np.linspace(0.0, 1.0, N + 1)
    P = trefoil(sN, 0, scale)
    s = np.zeros((1, P_ORDER, 3))
    e = np.zeros((1, P_ORDER, 3))
    for r in range(P_ORDER):
        s[0, r] = trefoil([0.0], r, scale)[0] / T_total ** r
        e[0, r] = trefoil([1.0], r, scale)[0] / T_total ** r
    return Workload(name=f"curve N={N}", seg_offset=np.array([0, N], np.int32), waypoints=P,
                    durations=np.full(N, T_total / N), start_state=s, end_state=e, mode="pin", rho=1.0,
                    max_iters=max_iters, notes={"T_total": T_total, "scale": scale})


def speed_limit(seed: int = 0, N: int = 256, M: int = 16, inner: str = "closed", vmax_factor: float = 1.6,
                max_iters: int = 200, vmax: Optional[float] = None) -> Workload:
    """1 trajectory, N segments, FREE waypoints, one speed bound ||v(t_ij)|| <= v_max
    through either constraint path of the paper: the projection of Eq. 14 /
    18f-g (inner="closed": the velocity-norm family) or the numerical step of
    Eq. 15-17 (inner="numeric": the general family with an acceleration bound
    too large to act).  Same geometry for both, from the same seed: random
    walk (step N(0, 1.5^2)), T ~ U[0.3, 1.5] lengthened to ||dP||_inf / 3.
    With free interior waypoints the trajectory only has to join the two
    boundary states in the total time, so v_max is set from that: vmax_factor
    x ||P_N - P_0|| / sum(T) (a rest-to-rest motion peaks well above its mean
    speed, so the bound acts for factors below about 2).  An explicit `vmax`
    overrides the rule."""
    rng = np.random.default_rng(seed)
    P = _random_walk(rng, N)
    T = rng.uniform(0.3, 1.5, size=N)
    dP = np.diff(P, axis=0)
    T = np.maximum(T, np.abs(dP).max(axis=1) / 3.0)
    if vmax is None:
        vmax = float(vmax_factor * np.linalg.norm(P[N] - P[0]) / T.sum())
    s, e = _rest_states(P[None, 0], P[None, N])
    common = dict(seg_offset=np.array([0, N], np.int32), waypoints=P, durations=T, start_state=s, end_state=e,
                  mode="free", rho=1.0, max_iters=max_iters)
    if inner == "closed":
        return Workload(name=f"speed_limit N={N} (projection)", inner="closed", M_vn=M,
                        vnorm=np.array([vmax]), **common)
    return Workload(name=f"speed_limit N={N} (numerical step)", inner="numeric", M_gen=M,
                    gen_vmax=np.array([vmax]), gen_amax=np.array([1e6]), **common)


def tiny(seed: int = 0, N: int = 3, mode: str = "pin", T_range=(0.5, 1.5), B: int = 1,
         step: float = 1.5) -> Workload:
    """Small random instances for edge-case tests."""
    master = np.random.default_rng(seed)
    Nb = np.full(B, N) if np.isscalar(N) else np.asarray(N)
    B = len(Nb)
    off = np.zeros(B + 1, np.int64)
    off[1:] = np.cumsum(Nb)
    S = int(off[-1])
    P = np.empty((S + B, 3))
    T = np.empty(S)
    for b in range(B):
        n = int(Nb[b])
        P[off[b] + b: off[b + 1] + b + 1] = _random_walk(master, n, step)
        T[off[b]:off[b + 1]] = master.uniform(*T_range, size=n)
    first = P[off[:-1] + np.arange(B)]
    last = P[off[1:] + np.arange(B)]
    s, e = _rest_states(first, last)
    return Workload(
        name=f"tiny N={list(map(int, Nb))}", seg_offset=off.astype(np.int32), waypoints=P,
        durations=T, start_state=s, end_state=e, mode=mode, rho=1.0, max_iters=50,
    )
