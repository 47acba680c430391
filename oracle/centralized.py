"""Centralised solutions of the trajectory problem (test infrastructure only).

These solve the whole problem of Sec. III-B (Eq. 2) at once, with their own
basis code (nothing shared with top_oracle.c), so that the CADMM fixed point
of the oracle can be checked against them:

  pin_spline      PIN mode, no inequalities: the square linear system
                  (boundary orders 0..3, interior positions pinned, C^6
                  continuity) whose unique solution is the min-snap spline
                  (the optimality conditions of Sec. III-D.2); sparse LU.
  free_polynomial FREE mode, no inequalities: one degree-7 polynomial over
                  [0, sum T] meeting the 8 boundary conditions per axis,
                  re-expanded per segment by a Taylor shift.
  kkt_qp          any equality set + fixed active inequality rows: the dense
                  KKT system of the whole QP (numpy.linalg.solve).
  active_set_qp   brute force over the active sets of a tiny box-constrained
                  problem: the exact constrained optimum.
  norm_ball_qp    a tiny problem with sampled norm bounds ||sigma^(r)(t_ij) - o_i||
                  <= rad_i (ball corridor: r = 0; velocity norm: r = 1, o = 0),
                  solved through its Lagrange dual (maximised over the
                  multipliers mu >= 0, each dual evaluation one equality-
                  constrained linear KKT solve), then polished by Newton's
                  method on the multipliers of the binding samples.

Coefficients are returned in the raw monomial basis of each segment,
shape [N, 3, 8]:  sigma_i(t) = sum_k c[i, a, k] (t - t_{i-1})^k.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

NC = 8   # coefficients per axis (degree 7)
ND = 7   # continuity orders 0..6
PO = 4   # boundary orders 0..3


def deriv_row(r: int, t: float) -> np.ndarray:
    """d^r/dt^r of (1, t, ..., t^7) evaluated at t."""
    row = np.zeros(NC)
    for k in range(r, NC):
        row[k] = math.factorial(k) / math.factorial(k - r) * t ** (k - r)
    return row


def snap_gram(T: float) -> np.ndarray:
    """int_0^T (d^4 beta)(d^4 beta)^T dt by 8-point Gauss-Legendre (exact for degree 6)."""
    x, wq = np.polynomial.legendre.leggauss(8)
    t = 0.5 * T * (x + 1.0)
    G = np.zeros((NC, NC))
    for tq, wgt in zip(t, wq):
        d = deriv_row(4, tq)
        G += 0.5 * T * wgt * np.outer(d, d)
    return G


def segment_cost(c: np.ndarray, T: np.ndarray) -> float:
    return float(sum(c[i, a] @ snap_gram(T[i]) @ c[i, a] for i in range(len(T)) for a in range(3)))


def pin_spline(P: np.ndarray, T: np.ndarray, start: np.ndarray, end: np.ndarray) -> np.ndarray:
    """Unique C^6 piecewise degree-7 curve through all waypoints (PIN mode fixed point)."""
    N = len(T)
    out = np.zeros((N, 3, NC))
    for a in range(3):
        rows, cols, vals, rhs = [], [], [], []
        eq = 0

        def put(seg, row_vec, val):
            nonlocal eq
            for k in range(NC):
                if row_vec[k] != 0.0:
                    rows.append(eq); cols.append(seg * NC + k); vals.append(row_vec[k])
            rhs.append(val)
            eq += 1

        for r in range(PO):
            put(0, deriv_row(r, 0.0), start[r, a])
        for j in range(1, N):
            put(j - 1, deriv_row(0, T[j - 1]), P[j, a])
            put(j, deriv_row(0, 0.0), P[j, a])
            for r in range(1, ND):
                left = deriv_row(r, T[j - 1])
                right = -deriv_row(r, 0.0)
                for k in range(NC):
                    if left[k] != 0.0:
                        rows.append(eq); cols.append((j - 1) * NC + k); vals.append(left[k])
                    if right[k] != 0.0:
                        rows.append(eq); cols.append(j * NC + k); vals.append(right[k])
                rhs.append(0.0)
                eq += 1
        for r in range(PO):
            put(N - 1, deriv_row(r, T[N - 1]), end[r, a])
        A = sp.csc_matrix((vals, (rows, cols)), shape=(eq, N * NC))
        assert eq == N * NC
        x = spla.spsolve(A, np.asarray(rhs))
        out[:, a, :] = x.reshape(N, NC)
    return out


def taylor_shift(coef: np.ndarray, t0: float) -> np.ndarray:
    """Coefficients of p(t0 + t) in powers of t, for p(t) = sum coef[k] t^k."""
    n = len(coef)
    out = np.zeros(n)
    for j in range(n):
        out[j] = sum(math.comb(k, j) * coef[k] * t0 ** (k - j) for k in range(j, n))
    return out


def free_polynomial(T: np.ndarray, start: np.ndarray, end: np.ndarray) -> np.ndarray:
    """FREE mode fixed point: one degree-7 polynomial over [0, sum T] per axis."""
    N = len(T)
    Ttot = float(np.sum(T))
    A = np.array([deriv_row(r, 0.0) for r in range(PO)] + [deriv_row(r, Ttot) for r in range(PO)])
    t0 = np.concatenate([[0.0], np.cumsum(T)[:-1]])
    out = np.zeros((N, 3, NC))
    for a in range(3):
        coef = np.linalg.solve(A, np.concatenate([start[:, a], end[:, a]]))
        for i in range(N):
            out[i, a] = taylor_shift(coef, t0[i])
    return out


def _equalities(P, T, start, end, mode):
    """Rows (dense over all N*24 unknowns) of the equality constraints of Eq. 2."""
    N = len(T)
    n = N * 3 * NC

    def idx(i, a):
        return i * 3 * NC + a * NC

    A, b = [], []
    for a in range(3):
        for r in range(PO):
            row = np.zeros(n); row[idx(0, a):idx(0, a) + NC] = deriv_row(r, 0.0)
            A.append(row); b.append(start[r, a])
            row = np.zeros(n); row[idx(N - 1, a):idx(N - 1, a) + NC] = deriv_row(r, T[N - 1])
            A.append(row); b.append(end[r, a])
        for j in range(1, N):
            for r in range(ND):
                row = np.zeros(n)
                row[idx(j - 1, a):idx(j - 1, a) + NC] = deriv_row(r, T[j - 1])
                row[idx(j, a):idx(j, a) + NC] -= deriv_row(r, 0.0)
                A.append(row); b.append(0.0)
            if mode == "pin":
                row = np.zeros(n); row[idx(j, a):idx(j, a) + NC] = deriv_row(0, 0.0)
                A.append(row); b.append(P[j, a])
    return np.array(A), np.array(b)


def _hessian(T):
    N = len(T)
    H = np.zeros((N * 3 * NC, N * 3 * NC))
    for i in range(N):
        G = snap_gram(T[i])
        for a in range(3):
            o = i * 3 * NC + a * NC
            H[o:o + NC, o:o + NC] = 2.0 * G
    return H


def box_rows(T, M, vmax):
    """Linear rows +-v_axis(t_ij) <= vmax, t_ij = j T_i / M (dense over all unknowns)."""
    N = len(T)
    n = N * 3 * NC
    G, h = [], []
    for i in range(N):
        for j in range(1, M + 1):
            t = j * T[i] / M
            for a in range(3):
                for sgn in (1.0, -1.0):
                    row = np.zeros(n)
                    o = i * 3 * NC + a * NC
                    row[o:o + NC] = sgn * deriv_row(1, t)
                    G.append(row); h.append(vmax)
    return np.array(G), np.array(h)


def kkt_qp(P, T, start, end, mode, G_act=None, h_act=None):
    """min sum c^T Qt c s.t. the equalities of Eq. 2 and G_act c = h_act; returns (c, multipliers)."""
    A, b = _equalities(P, T, start, end, mode)
    if G_act is not None and len(G_act):
        A = np.vstack([A, G_act]); b = np.concatenate([b, h_act])
    H = _hessian(T)
    N = len(T)
    # solve in time-normalised unknowns x_k = c_k T^k with unit-norm rows (conditioning only)
    D = np.concatenate([[T[i] ** -k for a in range(3) for k in range(NC)] for i in range(N)])
    Hs = D[:, None] * H * D[None, :]
    As = A * D[None, :]
    rs = 1.0 / np.linalg.norm(As, axis=1)
    As = As * rs[:, None]
    sigma = 1.0 / np.max(np.diag(Hs))
    n, m = H.shape[0], A.shape[0]
    KKT = np.zeros((n + m, n + m))
    KKT[:n, :n] = Hs * sigma
    KKT[:n, n:] = As.T
    KKT[n:, :n] = As
    sol = np.linalg.lstsq(KKT, np.concatenate([np.zeros(n), b * rs]), rcond=None)[0]
    c = (D * sol[:n]).reshape(N, 3, NC)
    lam = sol[n:] * rs / sigma
    return c, lam


def active_set_qp(P, T, start, end, mode, M, vmax, tol=1e-9):
    """Exact optimum of a tiny box-constrained QP by enumerating active sets.

    The problem separates by axis (the cost, the equalities and the box rows
    each act on one axis), so the enumeration runs axis by axis.  Returns
    (c [N,3,8], active row indices into box_rows) or (None, None).
    """
    G, h = box_rows(T, M, vmax)
    A, b_eq = _equalities(P, T, start, end, mode)
    H = _hessian(T)
    N = len(T)
    cols_of = [np.concatenate([np.arange(i * 3 * NC + a * NC, i * 3 * NC + (a + 1) * NC)
                               for i in range(N)]) for a in range(3)]
    c_all = np.zeros(N * 3 * NC)
    act_all = []
    for a in range(3):
        cols = cols_of[a]
        eq_rows = np.where(np.abs(A[:, cols]).sum(axis=1) > 0)[0]
        box_rows_a = np.where(np.abs(G[:, cols]).sum(axis=1) > 0)[0]
        Aa, ba = A[np.ix_(eq_rows, cols)], b_eq[eq_rows]
        Ga, ha = G[np.ix_(box_rows_a, cols)], h[box_rows_a]
        Ha = H[np.ix_(cols, cols)]
        D = np.concatenate([[T[i] ** -k for k in range(NC)] for i in range(N)])
        n = len(cols)
        found = None
        for size in range(0, len(ha) + 1):
            for act in itertools.combinations(range(len(ha)), size):
                act = list(act)
                if any((box_rows_a[i] ^ 1) in box_rows_a[act] for i in act):
                    continue  # a row and its mirror cannot both be active
                Aall = np.vstack([Aa, Ga[act]]) if act else Aa
                ball = np.concatenate([ba, ha[act]]) if act else ba
                As = Aall * D[None, :]
                rs = 1.0 / np.linalg.norm(As, axis=1)
                As = As * rs[:, None]
                Hs = D[:, None] * Ha * D[None, :]
                sigma = 1.0 / np.max(np.diag(Hs))
                m = As.shape[0]
                KKT = np.zeros((n + m, n + m))
                KKT[:n, :n] = Hs * sigma
                KKT[:n, n:] = As.T
                KKT[n:, :n] = As
                sol = np.linalg.lstsq(KKT, np.concatenate([np.zeros(n), ball * rs]), rcond=None)[0]
                x = D * sol[:n]
                lam = sol[n:] * rs / sigma
                if np.abs(Aall @ x - ball).max() > 1e-7 * max(1.0, np.abs(ball).max()):
                    continue  # equalities + this active set are inconsistent
                if np.any(Ga @ x > ha + tol):
                    continue
                if np.any(lam[len(ba):] < -tol):
                    continue
                found = (x, [int(box_rows_a[i]) for i in act])
                break
            if found is not None:
                break
        if found is None:
            return None, None
        c_all[cols] = found[0]
        act_all += found[1]
    return c_all.reshape(N, 3, NC), sorted(act_all)


def norm_ball_qp(P, T, start, end, mode, M, order, centres, radii):
    """Exact optimum of min sum c^T Qt c under the equalities of Eq. 2 and the
    sampled norm bounds ||sigma_i^{(order)}(t_ij) - centres[i]|| <= radii[i],
    t_ij = j T_i / M, j = 1..M.

    The problem is a convex QCQP with a strictly feasible point, so strong
    duality holds: for multipliers mu >= 0 the Lagrangian is a quadratic in c
    whose equality-constrained minimiser c(mu) is one linear KKT solve, and
    the dual function d(mu) = L(c(mu), mu) is concave with gradient
    ||G_j c(mu) - o_j||^2 - rad_j^2.  d is maximised by L-BFGS-B over mu >= 0;
    the multipliers of the binding samples are then refined by Newton's
    method on ||G_j c(mu) - o_j||^2 = rad_j^2.  Returns (c [N,3,8], mu [N*M],
    g [N*M] = ||G_j c - o_j|| - rad_j).
    """
    import scipy.optimize as so

    A, b = _equalities(P, T, start, end, mode)
    H = _hessian(T)
    N = len(T)
    n = N * 3 * NC
    # time-normalised unknowns and unit-norm equality rows (conditioning only)
    D = np.concatenate([[T[i] ** -k for a in range(3) for k in range(NC)] for i in range(N)])
    Hs = D[:, None] * H * D[None, :]
    As = A * D[None, :]
    rs = 1.0 / np.linalg.norm(As, axis=1)
    As = As * rs[:, None]
    bs = b * rs
    m = As.shape[0]
    Gs, os_, rad = [], [], []
    for i in range(N):
        for j in range(1, M + 1):
            row = deriv_row(order, j * T[i] / M)
            G = np.zeros((3, n))
            for a in range(3):
                o = i * 3 * NC + a * NC
                G[a, o:o + NC] = row
            Gs.append(G * D[None, :])
            os_.append(np.asarray(centres[i], dtype=float))
            rad.append(float(radii[i]))
    J = len(Gs)

    def c_of(mu):
        K = Hs.copy()
        rhs = np.zeros(n)
        for G, o, mj in zip(Gs, os_, mu):
            K += 2.0 * mj * G.T @ G
            rhs += 2.0 * mj * G.T @ o
        KKT = np.zeros((n + m, n + m))
        KKT[:n, :n] = K
        KKT[:n, n:] = As.T
        KKT[n:, :n] = As
        return np.linalg.solve(KKT, np.concatenate([rhs, bs]))[:n]

    def gaps(x):
        return np.array([np.sum((G @ x - o) ** 2) - r * r for G, o, r in zip(Gs, os_, rad)])

    def neg_dual(mu):
        x = c_of(mu)
        g = gaps(x)
        return -(0.5 * x @ Hs @ x + mu @ g), -g

    res = so.minimize(neg_dual, np.zeros(J), jac=True, method="L-BFGS-B", bounds=[(0.0, None)] * J,
                      options=dict(ftol=0.0, gtol=1e-14, maxiter=20000))
    mu = np.array(res.x)
    act = np.where(mu > 1e-9 * max(1.0, mu.max()))[0]
    if len(act):
        def f(ma):
            full = np.zeros(J)
            full[act] = ma
            return gaps(c_of(full))[act]
        sol = so.root(f, mu[act], method="hybr", options=dict(xtol=1e-15))
        # hybr may report "no further improvement" at full precision: judge by the residual
        if np.all(sol.x >= 0) and np.abs(f(sol.x)).max() <= np.abs(f(mu[act])).max():
            mu = np.zeros(J)
            mu[act] = sol.x
    x = c_of(mu)
    g = np.array([np.linalg.norm(G @ x - o) - r for G, o, r in zip(Gs, os_, rad)])
    return (D * x).reshape(N, 3, NC), mu, g
