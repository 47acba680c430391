"""The oracle's pins catch plausible mistakes.

Each case copies the oracle source, plants one mistake by a textual edit
(a dropped factor, a flipped sign, a wrong index or exponent, a missing
mask), compiles the copy on the CPU into a temporary directory and checks
that at least one pin (closed form, centralised fixed point, active-set
optimum, projection property, numerical-step stationarity) rejects it.  The
unmodified source passes the same checks.
"""
import numpy as np
import pytest

import oracle
from oracle import capi
from oracle import centralized as CZ
from paper_2507_10290_gb300 import workloads as W

from test_oracle_pins import (_box_instance, _numpy_F, _quadratic_rows_ok, adaptive_dual_continuity_error,
                              adaptive_kkt_error, adaptive_rule_violations, numeric_dual_error, polytope_kkt_errors,
                              polytope_rotation_error, read_golden, residual_errors, scaled_relerr)


def pin_closed_form(lib):
    g = read_golden()
    s = np.array([float(x) for x in g["coeffs"]])
    P = np.array([[0.3, -1.0, 2.0], [2.5, 1.5, -1.0]])
    T = 1.3
    for mode in ("free", "pin"):
        w = W.tiny(N=1, mode=mode).with_(
            waypoints=P, durations=np.array([T]),
            start_state=np.concatenate([P[None, :1], np.zeros((1, 3, 3))], axis=1),
            end_state=np.concatenate([P[None, 1:], np.zeros((1, 3, 3))], axis=1),
            rho=1e5 / T ** 7, max_iters=500)
        r = oracle.solve(w, real=lib)
        d = P[1] - P[0]
        ref = np.zeros((1, 3, 8))
        for a in range(3):
            ref[0, a] = d[a] * s / T ** np.arange(8)
            ref[0, a, 0] += P[0, a]
        J = 100800 * float(d @ d) / T ** 7
        if not (scaled_relerr(r["coeffs"], ref, [T]) < 1e-9 and abs(r["cost"][0] - J) < 1e-9 * J):
            return False
    return True


def pin_free_fixed_point(lib):
    w = W.tiny(seed=1, N=8, mode="free", T_range=(0.8, 1.6)).with_(rho=1.0, max_iters=20000)
    r = oracle.solve(w, real=lib)
    ref = CZ.free_polynomial(w.durations, w.start_state[0], w.end_state[0])
    return scaled_relerr(r["coeffs"], ref, w.durations) < 1e-8


def pin_pin_fixed_point(lib):
    w = W.tiny(seed=1, N=2, mode="pin", T_range=(0.8, 1.6)).with_(rho=1.0, max_iters=300000)
    r = oracle.solve(w, real=lib)
    ref = CZ.pin_spline(w.waypoints, w.durations, w.start_state[0], w.end_state[0])
    return scaled_relerr(r["coeffs"], ref, w.durations) < 1e-5


def pin_active_set(lib):
    w = _box_instance()
    c_ref, _ = CZ.active_set_qp(w.waypoints, w.durations, w.start_state[0], w.end_state[0], "free",
                                w.M_box, float(w.vbox[0]))
    r = oracle.solve(w, real=lib)
    return scaled_relerr(r["coeffs"], c_ref, w.durations) < 1e-6


def pin_projection(lib):
    rng = np.random.default_rng(3)
    for _ in range(50):
        o = rng.normal(size=3)
        rad = rng.uniform(0.2, 2.0)
        q = rng.normal(scale=3.0, size=3)
        p = capi.project_ball(q, o, rad, real=lib)
        if np.linalg.norm(p - o) > rad * (1 + 1e-12):
            return False
        if not np.allclose(capi.project_ball(p, o, rad, real=lib), p, atol=1e-12):
            return False
        # the projection is on the segment from o to q
        d = (q - o) / np.linalg.norm(q - o)
        if np.linalg.norm(q - o) > rad and abs(np.linalg.norm(p - o) - rad) > 1e-12:
            return False
        if np.linalg.norm(np.cross(p - o, d)) > 1e-9:
            return False
    return True


def pin_numeric_stationary(lib):
    w = W.tiny(seed=9, N=3, mode="pin", step=6.0, T_range=(0.8, 1.0)).with_(
        inner="numeric", M_gen=6, gen_vmax=np.array([4.0]), gen_amax=np.array([8.0]), rho=1e4)
    i, T = 1, w.durations[1]
    spl = CZ.pin_spline(w.waypoints, w.durations, w.start_state[0], w.end_state[0])
    zt = np.zeros(42)
    for a in range(3):
        for rr in range(7):
            zt[a * 14 + rr] = spl[i, a] @ CZ.deriv_row(rr, 0.0)
            zt[a * 14 + 7 + rr] = spl[i, a] @ CZ.deriv_row(rr, T)
    rng = np.random.default_rng(0)
    u = rng.normal(scale=0.01, size=42)
    y = np.abs(rng.normal(size=(6, 2)))
    c, _ = capi.numeric_local(w, 0, i, zt, u, y, real=lib)
    args = (T, False, False, zt, u, y, 1e4, 6, 4.0, 8.0)
    F0 = _numpy_F(c, *args)
    for _ in range(200):
        d = rng.normal(size=24) * 1e-4 * np.abs(c).clip(1e-3)
        if _numpy_F(c + d, *args) < F0 - 1e-9 * abs(F0):
            return False
    return True


def pin_adaptive_rule(lib):
    bad, up, down = adaptive_rule_violations(lib)
    return bad == 0 and up > 10 and down > 10


def pin_adaptive_kkt(lib):
    err, rho = adaptive_kkt_error(lib)
    return rho != 10.0 and err < 1e-5


def pin_adaptive_dual(lib):
    return adaptive_dual_continuity_error(lib) < 1e-12


def pin_polytope_kkt(lib):
    worst, active, r = polytope_kkt_errors(lib)
    return (r["status"][0] == 0 and active >= 2 and worst["stat"] < 1e-6 and worst["dual"] < 1e-9
            and worst["primal"] < 1e-7 and worst["compl"] < 1e-6)


def pin_polytope_rotation(lib):
    return polytope_rotation_error(lib) < 1e-11


def pin_residuals(lib):
    return residual_errors(lib) < 1e-10


def pin_numeric_dual(lib):
    return numeric_dual_error(lib) < 1e-9


def pin_ball_corridor(lib):
    return _quadratic_rows_ok("ball", lib)


def pin_velocity_norm(lib):
    return _quadratic_rows_ok("vn", lib)


# cheap pins first: a planted mistake stops at the first pin that rejects it
ALL_PINS = [pin_projection, pin_residuals, pin_closed_form, pin_numeric_dual, pin_numeric_stationary,
            pin_free_fixed_point, pin_active_set, pin_velocity_norm, pin_ball_corridor, pin_pin_fixed_point,
            pin_adaptive_rule, pin_adaptive_dual, pin_adaptive_kkt, pin_polytope_rotation, pin_polytope_kkt]

PLANTS = {
    "rhs without rho": ("for (int l = 0; l < NL; ++l) rhs[l] *= rho;\n        chol_solve",
                        "for (int l = 0; l < NL; ++l) rhs[l] *= 1;\n        chol_solve"),
    "u update sign": ("u[(size_t)i * NR + q] += sd[i].E[q] * (Mc[q]",
                      "u[(size_t)i * NR + q] -= sd[i].E[q] * (Mc[q]"),
    "consensus weight": ("z[(j * AX + a) * ND + r] = (left + right) / 2;",
                         "z[(j * AX + a) * ND + r] = (2 * left + right) / 3;"),
    "end mask missing": ("if (side == 1 && last && r >= PO) e = 0;", ";"),
    "Q exponent": ("int e = k + l - 2 * PO + 1;", "int e = k + l - 2 * PO + 2;"),
    "M row at wrong end": ("beta_rk(r, k, side ? T : (real)0)", "beta_rk(r, k, side ? (real)0 : T)"),
    "slack sign": ("real sn = -(Ac[q] - sd[i].b[q] + v[idx]);", "real sn = (Ac[q] - sd[i].b[q] + v[idx]);"),
    "dual v misses slack": ("v[idx] = v[idx] + Ac[q] + s[idx] - sd[i].b[q];",
                            "v[idx] = v[idx] + Ac[q] - sd[i].b[q];"),
    "projection scale": ("real f = ratio > 1 ? sqrt_r(1 / ratio) : (real)1;",
                         "real f = ratio > 1 ? 1 / ratio : (real)1;"),
    "penalty gradient": ("real coef = (rho * g + y) * 4 * h;", "real coef = (rho * g + y) * 2 * h;"),
    "velocity sample row": ("sample_matrix(1, t, sd->Agv + (size_t)j * 3 * NL);",
                            "sample_matrix(2, t, sd->Agv + (size_t)j * 3 * NL);"),
    "scaled duals kept on rho change": ("const real f = rho / rn;", "const real f = 1;"),
    "rho rule inverted": ("rn = rho * (real)pb->rho_tau_incr;", "rn = rho / (real)pb->rho_tau_incr;"),
    "K kept at old rho": ("if (refactor_segment(&sd[i], pb, rho) != 0)",
                          "if (0 && refactor_segment(&sd[i], pb, rho) != 0)"),
    "polytope normal on the wrong axis": ("sd->Ao[row * NL + a * NC + k] = (real)nf[a] * beta_rk(0, k, t);",
                                          "sd->Ao[row * NL + a * NC + k] = (real)nf[(a + 1) % 3] * beta_rk(0, k, t);"),
    "polytope rows on velocity": ("sd->Ao[row * NL + a * NC + k] = (real)nf[a] * beta_rk(0, k, t);",
                                  "sd->Ao[row * NL + a * NC + k] = (real)nf[a] * beta_rk(1, k, t);"),
    "polytope offset sign": ("sd->b[row] = pb->poly_h[(size_t)gi * pb->F_poly + f];",
                             "sd->b[row] = -pb->poly_h[(size_t)gi * pb->F_poly + f];"),
    # quadratic rows inside the iteration (Eq. 18a, 18f-g)
    "ball rhs with +w": ("d3[a] = phb[((size_t)i * Mq + j) * 3 + a] - wb[((size_t)i * Mq + j) * 3 + a];",
                         "d3[a] = phb[((size_t)i * Mq + j) * 3 + a] + wb[((size_t)i * Mq + j) * 3 + a];"),
    "velocity-norm rhs with +w": ("d3[a] = phv[((size_t)i * Mv + j) * 3 + a] - wv[((size_t)i * Mv + j) * 3 + a];",
                                  "d3[a] = phv[((size_t)i * Mv + j) * 3 + a] + wv[((size_t)i * Mv + j) * 3 + a];"),
    "velocity-norm rows on position": ("sample_matrix(1, t, sd->Av + (size_t)j * 3 * NL);",
                                       "sample_matrix(0, t, sd->Av + (size_t)j * 3 * NL);"),
    "ball rows missing from K": ("sample_matrix(0, t, sd->Ab + (size_t)j * 3 * NL);\n      add_AtA(sd->K, sd->Ab + (size_t)j * 3 * NL, 3, rho);",
                                 "sample_matrix(0, t, sd->Ab + (size_t)j * 3 * NL);"),
    "velocity-norm rows missing from K": ("sample_matrix(1, t, sd->Av + (size_t)j * 3 * NL);\n      add_AtA(sd->K, sd->Av + (size_t)j * 3 * NL, 3, rho);",
                                          "sample_matrix(1, t, sd->Av + (size_t)j * 3 * NL);"),
    "ball dual forgets its past": ("wb[((size_t)i * Mq + j) * 3 + a] = qv[a] - ph[a];",
                                   "wb[((size_t)i * Mq + j) * 3 + a] = w3[a] - ph[a];"),
    # residuals (Eq. 19-20)
    "r_d without rho": ("matvec_t_add(sd[i].Mt, NR, dz, rho, rdv);", "matvec_t_add(sd[i].Mt, NR, dz, 1, rdv);"),
    "r_d without M^T": ("matvec_t_add(sd[i].Mt, NR, dz, rho, rdv);\n      rd2 += dotn(rdv, rdv, NL);",
                        "for (int q = 0; q < NR; ++q) rd2 += rho * rho * dz[q] * dz[q];"),
    "r_d from the end side only": ("dz[q] = sd[i].E[q] * (z[zi] - zo[zi]);",
                                   "dz[q] = side ? sd[i].E[q] * (z[zi] - zo[zi]) : 0;"),
    "r_p over orders < p only": ("rp2 += gap * gap;                                       /* Eq. 19 */",
                                 "if (r < PO) rp2 += gap * gap;"),
    # numerical-step dual (Eq. 17)
    "numeric dual without rho": ("yg[((size_t)i * Mg + j) * 2 + g2] += rho * g;",
                                 "yg[((size_t)i * Mg + j) * 2 + g2] += g;"),
}


def test_unmodified_source_passes_every_pin(tmp_path):
    lib = capi.build_variant(capi.source_text(), str(tmp_path / "clean"))
    for pin in ALL_PINS:
        assert pin(lib), pin.__name__


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = PLANTS[name]
    src = capi.source_text()
    assert src.count(old) == 1, f"plant site for {name!r} not unique"
    lib = capi.build_variant(src.replace(old, new), str(tmp_path / name.replace(" ", "_")))
    assert any(not pin(lib) for pin in ALL_PINS), f"no pin caught {name!r}"
