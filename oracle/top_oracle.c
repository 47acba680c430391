/*
 * top_oracle.c -- plain, slow, serial reference of the TOP consensus-ADMM
 * (CADMM) trajectory optimiser.  TEST INFRASTRUCTURE ONLY: the product path
 * (the CUDA library) never links, loads or calls this file; only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark do.
 *
 * It follows the paper (arXiv 2507.10290, "TOP: Trajectory Optimization via
 * Parallel Optimization towards Constant Time Complexity") literally:
 *   - cost  sum_i c_i^T Qt(T_i) c_i,  Qt = I_3 (x) Q,  Q(T) = int_0^T beta^(p) beta^(p)T
 *     (Sec. III-D, definition of Q under Eq. 18),
 *   - consensus map Mt = I_3 (x) M,  M(t) = (beta^0(0)..beta^(d-1)(0), beta^0(t)..beta^(d-1)(t))^T
 *     (Sec. III-D, definition of M under Eq. 18),
 *   - the closed-form local step of Eq. 18a with the projections of Eq. 18d-g,
 *   - the consensus average (Eq. 18b) and the scaled dual update (Eq. 18c),
 *   - the numerical local step of Sec. III-C.3 (Eq. 15-17) solved with L-BFGS,
 *   - primal / dual residuals (Eq. 19-20) and the stopping rule (Eq. 21),
 *   - optionally the residual-balancing update of rho (UpdateRho, Eq. 22),
 *   - linear rows from velocity boxes and from polytope corridors with
 *     arbitrary face normals (Eq. 8-10, 18d-e),
 * all with dense matrices built entry by entry (the 24x24 local matrix of
 * Eq. 18a, the 42x24 consensus map, the 2*3*M x 24 linear-constraint matrix,
 * the 3x24 sample matrices), solved with a Cholesky factorisation of the
 * Jacobi-equilibrated local matrix.
 *
 * Readings where the paper is silent or garbled (each one is listed in the
 * design notes of the repository with its justification):
 *   R1  degree 2p-1 = 7 (8 coefficients per axis), consensus derivative
 *       orders 0..2p-2 = 0..6 (d = 7 rows per axis and end), from the
 *       optimality conditions of Sec. III-D.2.
 *   R2  the fixed end junctions z_0, z_N only define orders < p; the
 *       consensus rows of order >= p at the start of the first segment and
 *       at the end of the last segment are dropped (mask E).
 *   R3  two waypoint modes: PIN fixes the position rows of interior
 *       junctions to the waypoints, FREE only uses them to initialise z.
 *   R4  the right-hand side of Eq. 18a carries the factor rho that the
 *       derivation from the augmented Lagrangian (Eq. 6) gives.
 *   R5  samples at t_ij = j*T_i/M, j = 1..M.
 *   R6  Init: z position rows = waypoints, other rows 0, ends from the
 *       boundary states; u = s = v = phi = w = y = 0.
 *   R7  loop until ||r_p|| < N*eps and ||r_d|| < N*eps (the loop condition
 *       of Algorithm 1 is printed inverted); eps = 0 runs max_iters.
 *   R8  ball corridor ||p(t) - o|| <= r: the projection of Eq. 14 shifted
 *       to the centre o.
 *   R9  general convex constraints use g0 = ||A c||^2 - g_max^2 and
 *       g = max(0, g0)^2 (Eq. 15); y <- y + rho*g (Eq. 17 "updated like
 *       Eq. 7c").  L-BFGS: memory m, initial inverse Hessian = inverse of
 *       the quadratic part's Hessian (2 Qt + rho Mt^T E Mt), Armijo
 *       backtracking (c1 = 1e-4, halving), started from the minimiser of the
 *       quadratic part, stopped when g^T K^-1 g <= tol^2 rhs^T K^-1 rhs.
 *   R10 dual residual stacked per segment: rho * Mt_i^T E_i (zt_i^{k+1} - zt_i^k).
 *   R13 UpdateRho runs after the stopping test of each iteration; when rho
 *       changes, the unscaled duals rho*u, rho*v, rho*w are kept (every
 *       scaled dual is multiplied by rho_old / rho_new) and each segment's
 *       local matrix is assembled and factorised again for the new rho.
 *
 * Parity unpinned: the iterate path of the L-BFGS numerical step.  Only its
 * result is pinned (stationarity of an independently coded objective, and
 * equality with the closed form where no bound is active), so GPU/oracle
 * parity of that step holds where every local solve reaches its tolerance
 * before its iteration cap.
 *
 * Compile-time type: OR_REAL (default double; the oracle's own rounding is
 * bounded by re-running it with OR_REAL = long double).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef OR_REAL
#define OR_REAL double
#endif
typedef OR_REAL real;

#define AX 3          /* m: flat-output axes (x, y, z) */
#define PO 4          /* p: control order, minimum snap */
#define NC 8          /* coefficients per axis: degree 2p-1 = 7 */
#define ND 7          /* consensus derivative orders 0..2p-2 */
#define NL (AX * NC)  /* 24 local unknowns per segment */
#define NR (AX * 2 * ND) /* 42 consensus rows per segment */

enum { OR_PIN = 0, OR_FREE = 1 };
enum { OR_CLOSED = 0, OR_NUMERIC = 1 };
enum { OR_CONVERGED = 0, OR_NOT_CONVERGED = 1, OR_NONFINITE = 2 };

typedef struct or_problem {
  int32_t B;
  const int32_t *seg_offset; /* [B+1] CSR over segments */
  const double *waypoints;   /* [S+B][3]: N_b+1 points per trajectory */
  const double *durations;   /* [S] */
  const double *start_state; /* [B][4][3]: derivative order r, axis a */
  const double *end_state;   /* [B][4][3] */
  int32_t mode;              /* OR_PIN | OR_FREE */
  int32_t inner;             /* OR_CLOSED | OR_NUMERIC */
  double rho;
  double eps;                /* stopping tolerance (E_r = E_d = N*eps); 0 = run max_iters */
  int32_t max_iters;
  int32_t M_box;  const double *vbox;             /* [B] |v_axis| <= vbox, linear rows */
  int32_t M_ball; const double *ball_c;           /* [S][3] */
  const double *ball_r;                           /* [S] */
  int32_t M_vn;   const double *vnorm;            /* [B] ||v|| <= vnorm, projection */
  int32_t M_gen;  const double *gen_vmax;         /* [B] ||v|| <= vmax, numerical step */
  const double *gen_amax;                         /* [B] ||a|| <= amax, numerical step */
  double lbfgs_tol;          /* relative infinity-norm gradient tolerance */
  int32_t lbfgs_max_iters;
  int32_t lbfgs_mem;
  /* adaptive penalty (Sec. III-D.4, Eq. 22); 0 keeps rho fixed */
  int32_t adaptive_rho;
  double rho_mu, rho_tau_incr, rho_tau_decr;
  /* polytope corridor (Sec. III-C.1, Eq. 8-10, 18d-e): segment i must satisfy
     n_f^T p(t_ij) <= h_f for its F_poly faces at M_poly samples; the rows
     n_f^T (x) beta(t_ij)^T follow the box rows in the linear-row block */
  int32_t M_poly, F_poly;
  const double *poly_n;      /* [S][F_poly][3] face normals */
  const double *poly_h;      /* [S][F_poly] offsets */
} or_problem;

typedef struct or_result {
  double *coeffs;     /* [S][3][8]: sigma_i(t) = sum_k coeffs[i][a][k] (t - t_{i-1})^k */
  double *cost;       /* [B] */
  double *r_primal;   /* [B] ||r_p|| of the last iteration */
  double *r_dual;     /* [B] ||r_d|| of the last iteration */
  int32_t *iters;     /* [B] */
  int32_t *status;    /* [B] */
  double *history;    /* optional [max_iters][B][2] (||r_p||, ||r_d||) */
  /* optional state after the last iteration */
  double *z;          /* [S+B][3][7] */
  double *u;          /* [S][42] row (a, side, r) = a*14 + side*7 + r */
  double *s, *v;      /* [S][6*M_box + F_poly*M_poly]: box row ((j*3)+a)*2 + sign, then
                         polytope row 6*M_box + j*F_poly + f */
  double *phi_b, *w_b;/* [S][M_ball][3] */
  double *phi_v, *w_v;/* [S][M_vn][3] */
  double *y_gen;      /* [S][M_gen][2] (velocity, acceleration) */
  int32_t *inner_iters; /* [S] L-BFGS iterations summed over the run */
  double *rho_hist;   /* optional [max_iters][B]: rho used in each iteration */
  double *rho_final;  /* optional [B]: rho after the last update */
} or_result;

/* ------------------------------------------------------------------ */
/* basis (Sec. III-D, Eq. 18 and the definitions below it)             */
/* ------------------------------------------------------------------ */

/* k! / (k-r)! */
static real falling(int k, int r) {
  real f = 1;
  for (int i = 0; i < r; ++i) f *= (real)(k - i);
  return f;
}

static real rpow(real t, int e) {
  real v = 1;
  for (int i = 0; i < e; ++i) v *= t;
  return v;
}

/* entry k of beta^{(r)}(t), beta(t) = (1, t, ..., t^7) */
static real beta_rk(int r, int k, real t) {
  if (k < r) return 0;
  return falling(k, r) * rpow(t, k - r);
}

/* Q(T) = int_0^T beta^{(p)}(tau) beta^{(p)}(tau)^T dtau, entry (k, l) */
static real q_entry(int k, int l, real T) {
  if (k < PO || l < PO) return 0;
  int e = k + l - 2 * PO + 1;
  return falling(k, PO) * falling(l, PO) * rpow(T, e) / (real)e;
}

/* ------------------------------------------------------------------ */
/* small dense linear algebra                                          */
/* ------------------------------------------------------------------ */

static real sqrt_r(real x) {
#ifdef OR_LONG
  return sqrtl(x);
#else
  return sqrt(x);
#endif
}

/* Jacobi-equilibrated Cholesky: S = diag(K)^-1/2, L L^T = S K S.
 * returns 0 on success, -1 if not positive definite. */
static int chol_equil(int n, const real *K, real *L, real *S) {
  for (int i = 0; i < n; ++i) {
    if (!(K[i * n + i] > 0)) return -1;
    S[i] = 1 / sqrt_r(K[i * n + i]);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) L[i * n + j] = 0;
  for (int j = 0; j < n; ++j) {
    real d = S[j] * K[j * n + j] * S[j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0)) return -1;
    real ljj = sqrt_r(d);
    L[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      real a = S[i] * K[i * n + j] * S[j];
      for (int k = 0; k < j; ++k) a -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = a / ljj;
    }
  }
  return 0;
}

/* solve K x = r using the factors of chol_equil */
static void chol_solve(int n, const real *L, const real *S, const real *r, real *x) {
  real w[NL];
  for (int i = 0; i < n; ++i) {
    real a = S[i] * r[i];
    for (int k = 0; k < i; ++k) a -= L[i * n + k] * w[k];
    w[i] = a / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    real a = w[i];
    for (int k = i + 1; k < n; ++k) a -= L[k * n + i] * x[k];
    x[i] = a / L[i * n + i];
  }
  for (int i = 0; i < n; ++i) x[i] *= S[i];
}

/* ------------------------------------------------------------------ */
/* per-segment literal matrices                                        */
/* ------------------------------------------------------------------ */

typedef struct seg_data {
  real T;
  real Mt[NR * NL];  /* \tilde M(T) = I_3 (x) M(T) */
  real E[NR];        /* consensus row mask (R2) */
  real Qt[NL * NL];  /* \tilde Q(T) */
  real K[NL * NL];   /* matrix of Eq. 18a */
  real L[NL * NL], S[NL];
  int nbox;
  real *Ao, *b;      /* [nbox][NL], [nbox] */
  real *Ab;          /* [M_ball][3][NL] position sample matrices */
  real *Av;          /* [M_vn][3][NL] velocity sample matrices */
  real *Agv, *Aga;   /* [M_gen][3][NL] velocity / acceleration sample matrices */
} seg_data;

static int row_of(int a, int side, int r) { return a * 2 * ND + side * ND + r; }

/* fill the 3 x NL matrix I_3 (x) beta^{(r)}(t)^T */
static void sample_matrix(int r, real t, real *A) {
  for (int i = 0; i < 3 * NL; ++i) A[i] = 0;
  for (int a = 0; a < AX; ++a)
    for (int k = 0; k < NC; ++k) A[a * NL + a * NC + k] = beta_rk(r, k, t);
}

/* A^T A accumulated into K with weight w */
static void add_AtA(real *K, const real *A, int rows, real w) {
  for (int i = 0; i < NL; ++i)
    for (int j = 0; j < NL; ++j) {
      real acc = 0;
      for (int q = 0; q < rows; ++q) acc += A[q * NL + i] * A[q * NL + j];
      K[i * NL + j] += w * acc;
    }
}

static int build_segment(seg_data *sd, const or_problem *pb, int b, int gi, int first, int last) {
  real T = pb->durations[gi];
  real rho = pb->rho;
  sd->T = T;
  /* consensus map and mask */
  for (int i = 0; i < NR * NL; ++i) sd->Mt[i] = 0;
  for (int a = 0; a < AX; ++a)
    for (int side = 0; side < 2; ++side)
      for (int r = 0; r < ND; ++r) {
        int row = row_of(a, side, r);
        for (int k = 0; k < NC; ++k)
          sd->Mt[row * NL + a * NC + k] = beta_rk(r, k, side ? T : (real)0);
        real e = 1;
        if (side == 0 && first && r >= PO) e = 0;
        if (side == 1 && last && r >= PO) e = 0;
        sd->E[row] = e;
      }
  /* cost matrix */
  for (int i = 0; i < NL * NL; ++i) sd->Qt[i] = 0;
  for (int a = 0; a < AX; ++a)
    for (int k = 0; k < NC; ++k)
      for (int l = 0; l < NC; ++l) sd->Qt[(a * NC + k) * NL + a * NC + l] = q_entry(k, l, T);
  /* K = 2 Qt + rho Mt^T E Mt + rho Ao^T Ao + rho sum A^T A  (Eq. 18a) */
  for (int i = 0; i < NL * NL; ++i) sd->K[i] = 2 * sd->Qt[i];
  for (int i = 0; i < NL; ++i)
    for (int j = 0; j < NL; ++j) {
      real acc = 0;
      for (int q = 0; q < NR; ++q) acc += sd->Mt[q * NL + i] * sd->E[q] * sd->Mt[q * NL + j];
      sd->K[i * NL + j] += rho * acc;
    }
  const int npoly = pb->M_poly > 0 ? pb->F_poly * pb->M_poly : 0;
  sd->nbox = 6 * pb->M_box + npoly;
  sd->Ao = sd->b = sd->Ab = sd->Av = sd->Agv = sd->Aga = NULL;
  if (sd->nbox > 0) {
    sd->Ao = (real *)calloc((size_t)sd->nbox * NL, sizeof(real));
    sd->b = (real *)calloc((size_t)sd->nbox, sizeof(real));
    for (int j = 0; j < pb->M_poly && npoly; ++j) {
      real t = (real)(j + 1) * T / (real)pb->M_poly;
      for (int f = 0; f < pb->F_poly; ++f) {
        int row = 6 * pb->M_box + j * pb->F_poly + f;
        const double *nf = pb->poly_n + ((size_t)gi * pb->F_poly + f) * 3;
        for (int a = 0; a < AX; ++a)
          for (int k = 0; k < NC; ++k) sd->Ao[row * NL + a * NC + k] = (real)nf[a] * beta_rk(0, k, t);
        sd->b[row] = pb->poly_h[(size_t)gi * pb->F_poly + f];
      }
    }
    for (int j = 0; j < pb->M_box; ++j) {
      real t = (real)(j + 1) * T / (real)pb->M_box;
      for (int a = 0; a < AX; ++a)
        for (int sg = 0; sg < 2; ++sg) {
          int row = (j * 3 + a) * 2 + sg;
          real sign = sg == 0 ? (real)1 : (real)-1;
          for (int k = 0; k < NC; ++k) sd->Ao[row * NL + a * NC + k] = sign * beta_rk(1, k, t);
          sd->b[row] = pb->vbox[b];
        }
    }
    add_AtA(sd->K, sd->Ao, sd->nbox, rho);
  }
  if (pb->M_ball > 0) {
    sd->Ab = (real *)calloc((size_t)pb->M_ball * 3 * NL, sizeof(real));
    for (int j = 0; j < pb->M_ball; ++j) {
      real t = (real)(j + 1) * T / (real)pb->M_ball;
      sample_matrix(0, t, sd->Ab + (size_t)j * 3 * NL);
      add_AtA(sd->K, sd->Ab + (size_t)j * 3 * NL, 3, rho);
    }
  }
  if (pb->M_vn > 0) {
    sd->Av = (real *)calloc((size_t)pb->M_vn * 3 * NL, sizeof(real));
    for (int j = 0; j < pb->M_vn; ++j) {
      real t = (real)(j + 1) * T / (real)pb->M_vn;
      sample_matrix(1, t, sd->Av + (size_t)j * 3 * NL);
      add_AtA(sd->K, sd->Av + (size_t)j * 3 * NL, 3, rho);
    }
  }
  if (pb->M_gen > 0) {
    sd->Agv = (real *)calloc((size_t)pb->M_gen * 3 * NL, sizeof(real));
    sd->Aga = (real *)calloc((size_t)pb->M_gen * 3 * NL, sizeof(real));
    for (int j = 0; j < pb->M_gen; ++j) {
      real t = (real)(j + 1) * T / (real)pb->M_gen;
      sample_matrix(1, t, sd->Agv + (size_t)j * 3 * NL);
      sample_matrix(2, t, sd->Aga + (size_t)j * 3 * NL);
    }
  }
  return chol_equil(NL, sd->K, sd->L, sd->S);
}

static void free_segment(seg_data *sd) {
  free(sd->Ao); free(sd->b); free(sd->Ab); free(sd->Av); free(sd->Agv); free(sd->Aga);
}

/* the matrix of Eq. 18a for another penalty rho (adaptive rho, Eq. 22),
 * assembled from the stored matrices and factored again */
static int refactor_segment(seg_data *sd, const or_problem *pb, real rho) {
  for (int i = 0; i < NL * NL; ++i) sd->K[i] = 2 * sd->Qt[i];
  for (int i = 0; i < NL; ++i)
    for (int j = 0; j < NL; ++j) {
      real acc = 0;
      for (int q = 0; q < NR; ++q) acc += sd->Mt[q * NL + i] * sd->E[q] * sd->Mt[q * NL + j];
      sd->K[i * NL + j] += rho * acc;
    }
  if (sd->Ao) add_AtA(sd->K, sd->Ao, sd->nbox, rho);
  for (int j = 0; j < pb->M_ball; ++j) add_AtA(sd->K, sd->Ab + (size_t)j * 3 * NL, 3, rho);
  for (int j = 0; j < pb->M_vn; ++j) add_AtA(sd->K, sd->Av + (size_t)j * 3 * NL, 3, rho);
  return chol_equil(NL, sd->K, sd->L, sd->S);
}

/* y = A x  (rows x NL) */
static void matvec(const real *A, int rows, const real *x, real *y) {
  for (int q = 0; q < rows; ++q) {
    real acc = 0;
    for (int i = 0; i < NL; ++i) acc += A[q * NL + i] * x[i];
    y[q] = acc;
  }
}

/* x += w * A^T y */
static void matvec_t_add(const real *A, int rows, const real *y, real w, real *x) {
  for (int i = 0; i < NL; ++i) {
    real acc = 0;
    for (int q = 0; q < rows; ++q) acc += A[q * NL + i] * y[q];
    x[i] += w * acc;
  }
}

/* projection onto {phi : ||phi - o||^2 <= rad^2}  (Eq. 14, shifted by o: R8) */
static void project_ball(const real *q, const real *o, real rad, real *phi) {
  real d[3], n2 = 0;
  for (int a = 0; a < 3; ++a) { d[a] = q[a] - (o ? o[a] : 0); n2 += d[a] * d[a]; }
  real ratio = n2 / (rad * rad);
  real f = ratio > 1 ? sqrt_r(1 / ratio) : (real)1;
  for (int a = 0; a < 3; ++a) phi[a] = (o ? o[a] : 0) + f * d[a];
}

/* ------------------------------------------------------------------ */
/* numerical local step (Sec. III-C.3, Eq. 15-17)                      */
/* ------------------------------------------------------------------ */

typedef struct num_ctx {
  const seg_data *sd;
  const real *zt, *u;   /* consensus target and scaled dual, 42 each */
  const real *y;        /* [M_gen][2] */
  int M_gen;
  real rho, vmax, amax;
} num_ctx;

/* g0 = ||A c||^2 - gmax^2, g = max(0, g0)^2; adds rho/2 g^2 + y g and its gradient */
static real gen_term(const real *A, const real *c, real gmax, real rho, real y, real *grad) {
  real w[3];
  matvec(A, 3, c, w);
  real h = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] - gmax * gmax;
  if (!(h > 0)) return 0;
  real g = h * h;
  real coef = (rho * g + y) * 4 * h; /* d/dc (rho/2 g^2 + y g) = (rho g + y) * 2h * 2 A^T w */
  matvec_t_add(A, 3, w, coef, grad);
  return rho / 2 * g * g + y * g;
}

/* F(c) of Eq. 16 restricted to segment i, with its gradient */
static real num_eval(const num_ctx *cx, const real *c, real *grad) {
  const seg_data *sd = cx->sd;
  real F = 0;
  for (int i = 0; i < NL; ++i) {
    real acc = 0;
    for (int j = 0; j < NL; ++j) acc += sd->Qt[i * NL + j] * c[j];
    F += c[i] * acc;
    grad[i] = 2 * acc;
  }
  real res[NR];
  matvec(sd->Mt, NR, c, res);
  for (int q = 0; q < NR; ++q) {
    res[q] = sd->E[q] * (res[q] - cx->zt[q] + cx->u[q]);
    F += cx->rho / 2 * res[q] * res[q];
  }
  matvec_t_add(sd->Mt, NR, res, cx->rho, grad);
  for (int j = 0; j < cx->M_gen; ++j) {
    F += gen_term(sd->Agv + (size_t)j * 3 * NL, c, cx->vmax, cx->rho, cx->y[j * 2 + 0], grad);
    F += gen_term(sd->Aga + (size_t)j * 3 * NL, c, cx->amax, cx->rho, cx->y[j * 2 + 1], grad);
  }
  return F;
}

static real dotn(const real *a, const real *b, int n) {
  real acc = 0;
  for (int i = 0; i < n; ++i) acc += a[i] * b[i];
  return acc;
}

/* L-BFGS (R9) on F with the initial inverse-Hessian approximation
 * H0 = K^-1, K = 2 Qt + rho Mt^T E Mt the Hessian of F's quadratic part
 * (factored by chol_equil); c in/out is the start point / minimiser.  Stops
 * when g^T K^-1 g <= tol^2 * scale.  Returns the iteration count. */
static int lbfgs_solve(const num_ctx *cx, real *c, real tol, real scale, int max_it, int mem) {
  const seg_data *sd = cx->sd;
  real g[NL], xn[NL], gn[NL], d[NL], q[NL], alpha[64];
  real *sv = (real *)calloc((size_t)mem * NL, sizeof(real));
  real *yv = (real *)calloc((size_t)mem * NL, sizeof(real));
  real *rh = (real *)calloc((size_t)mem, sizeof(real));
  int npair = 0, head = 0, it = 0;
  real f = num_eval(cx, c, g);
  for (it = 0; it < max_it; ++it) {
    chol_solve(NL, sd->L, sd->S, g, d);
    if (!(dotn(g, d, NL) > tol * tol * scale)) break;
    /* two-loop recursion, H0 = K^-1 */
    for (int i = 0; i < NL; ++i) q[i] = g[i];
    for (int k = 0; k < npair; ++k) {
      int idx = (head - 1 - k + mem) % mem;
      alpha[k] = rh[idx] * dotn(sv + idx * NL, q, NL);
      for (int i = 0; i < NL; ++i) q[i] -= alpha[k] * yv[idx * NL + i];
    }
    chol_solve(NL, sd->L, sd->S, q, d);
    for (int k = npair - 1; k >= 0; --k) {
      int idx = (head - 1 - k + mem) % mem;
      real beta = rh[idx] * dotn(yv + idx * NL, d, NL);
      for (int i = 0; i < NL; ++i) d[i] += (alpha[k] - beta) * sv[idx * NL + i];
    }
    for (int i = 0; i < NL; ++i) d[i] = -d[i];
    real gd = dotn(g, d, NL);
    if (!(gd < 0)) { /* not a descent direction: restart from -K^-1 g */
      chol_solve(NL, sd->L, sd->S, g, d);
      for (int i = 0; i < NL; ++i) d[i] = -d[i];
      gd = dotn(g, d, NL);
      npair = 0;
    }
    /* Armijo backtracking, c1 = 1e-4, halving */
    real step = 1, fn = f;
    int ok = 0;
    for (int bt = 0; bt < 60; ++bt) {
      for (int i = 0; i < NL; ++i) xn[i] = c[i] + step * d[i];
      fn = num_eval(cx, xn, gn);
      if (fn <= f + (real)1e-4 * step * gd) { ok = 1; break; }
      step /= 2;
    }
    if (!ok) break;
    real sy = 0;
    real sk[NL], yk[NL];
    for (int i = 0; i < NL; ++i) { sk[i] = xn[i] - c[i]; yk[i] = gn[i] - g[i]; sy += sk[i] * yk[i]; }
    if (sy > 0) {
      memcpy(sv + head * NL, sk, sizeof(sk));
      memcpy(yv + head * NL, yk, sizeof(yk));
      rh[head] = 1 / sy;
      head = (head + 1) % mem;
      if (npair < mem) ++npair;
    }
    memcpy(c, xn, sizeof(xn));
    memcpy(g, gn, sizeof(gn));
    f = fn;
  }
  free(sv); free(yv); free(rh);
  return it;
}

/* ------------------------------------------------------------------ */
/* the CADMM iteration (Algorithm 1 with Eq. 18)                       */
/* ------------------------------------------------------------------ */

static int isfin(real x) { return x == x && x - x == 0; }

static int solve_one(const or_problem *pb, or_result *res, int b) {
  const int s0 = pb->seg_offset[b];
  const int N = pb->seg_offset[b + 1] - s0;
  const double *P = pb->waypoints + (size_t)(s0 + b) * 3;
  real rho = pb->rho;
  const int Mb = pb->M_box, Mq = pb->M_ball, Mv = pb->M_vn, Mg = pb->M_gen;
  const int nbox = 6 * Mb + (pb->M_poly > 0 ? pb->F_poly * pb->M_poly : 0);  /* linear rows (box, polytope) */
  if (N <= 0) {
    res->cost[b] = 0; res->r_primal[b] = 0; res->r_dual[b] = 0;
    res->iters[b] = 0; res->status[b] = OR_CONVERGED;
    if (res->rho_final) res->rho_final[b] = (double)rho;  /* no iteration, no update */
    return 0;
  }
  seg_data *sd = (seg_data *)calloc((size_t)N, sizeof(seg_data));
  for (int i = 0; i < N; ++i)
    if (build_segment(&sd[i], pb, b, s0 + i, i == 0, i == N - 1) != 0) {
      for (int q = 0; q <= i; ++q) free_segment(&sd[q]);
      free(sd);
      return -1;
    }
  /* variables (R6) */
  real *z = (real *)calloc((size_t)(N + 1) * AX * ND, sizeof(real));  /* z[j][a][r] */
  real *zo = (real *)calloc((size_t)(N + 1) * AX * ND, sizeof(real));
  real *u = (real *)calloc((size_t)N * NR, sizeof(real));
  real *c = (real *)calloc((size_t)N * NL, sizeof(real));
  real *s = (real *)calloc((size_t)N * (nbox ? nbox : 1), sizeof(real));
  real *v = (real *)calloc((size_t)N * (nbox ? nbox : 1), sizeof(real));
  real *phb = (real *)calloc((size_t)N * (Mq ? Mq : 1) * 3, sizeof(real));
  real *wb = (real *)calloc((size_t)N * (Mq ? Mq : 1) * 3, sizeof(real));
  real *phv = (real *)calloc((size_t)N * (Mv ? Mv : 1) * 3, sizeof(real));
  real *wv = (real *)calloc((size_t)N * (Mv ? Mv : 1) * 3, sizeof(real));
  real *yg = (real *)calloc((size_t)N * (Mg ? Mg : 1) * 2, sizeof(real));
  int *inner_it = (int *)calloc((size_t)N, sizeof(int));
  for (int j = 0; j <= N; ++j)
    for (int a = 0; a < AX; ++a) z[(j * AX + a) * ND + 0] = P[j * 3 + a];
  for (int a = 0; a < AX; ++a)
    for (int r = 0; r < PO; ++r) {
      z[(0 * AX + a) * ND + r] = pb->start_state[((size_t)b * PO + r) * 3 + a];
      z[(N * AX + a) * ND + r] = pb->end_state[((size_t)b * PO + r) * 3 + a];
    }
  const real eps_tol = (real)N * (real)pb->eps;
  int k = 0, status = OR_NOT_CONVERGED;
  real rp = 0, rd = 0;
  for (k = 0; k < pb->max_iters; ++k) {
    /* --- local step, all segments (ClosedFormSolve / NumericSolve) --- */
    for (int i = 0; i < N; ++i) {
      real zt[NR], rhs[NL];
      for (int a = 0; a < AX; ++a)
        for (int side = 0; side < 2; ++side)
          for (int r = 0; r < ND; ++r) zt[row_of(a, side, r)] = z[((i + side) * AX + a) * ND + r];
      /* rhs = rho [Mt^T E (zt - u) + Ao^T (b - s - v) + sum A^T (phi - w)]  (Eq. 18a, R4) */
      real t42[NR];
      for (int q = 0; q < NR; ++q) t42[q] = sd[i].E[q] * (zt[q] - u[(size_t)i * NR + q]);
      for (int l = 0; l < NL; ++l) rhs[l] = 0;
      matvec_t_add(sd[i].Mt, NR, t42, 1, rhs);
      if (pb->inner == OR_CLOSED) {
        if (nbox) {
          real *tb = (real *)malloc(sizeof(real) * nbox);
          for (int q = 0; q < nbox; ++q)
            tb[q] = sd[i].b[q] - s[(size_t)i * nbox + q] - v[(size_t)i * nbox + q];
          matvec_t_add(sd[i].Ao, nbox, tb, 1, rhs);
          free(tb);
        }
        for (int j = 0; j < Mq; ++j) {
          real d3[3];
          for (int a = 0; a < 3; ++a)
            d3[a] = phb[((size_t)i * Mq + j) * 3 + a] - wb[((size_t)i * Mq + j) * 3 + a];
          matvec_t_add(sd[i].Ab + (size_t)j * 3 * NL, 3, d3, 1, rhs);
        }
        for (int j = 0; j < Mv; ++j) {
          real d3[3];
          for (int a = 0; a < 3; ++a)
            d3[a] = phv[((size_t)i * Mv + j) * 3 + a] - wv[((size_t)i * Mv + j) * 3 + a];
          matvec_t_add(sd[i].Av + (size_t)j * 3 * NL, 3, d3, 1, rhs);
        }
        for (int l = 0; l < NL; ++l) rhs[l] *= rho;
        chol_solve(NL, sd[i].L, sd[i].S, rhs, c + (size_t)i * NL);
        /* phi, w (Eq. 18f, 18g) */
        for (int j = 0; j < Mq; ++j) {
          real w3[3], qv[3], ph[3];
          matvec(sd[i].Ab + (size_t)j * 3 * NL, 3, c + (size_t)i * NL, w3);
          for (int a = 0; a < 3; ++a) qv[a] = w3[a] + wb[((size_t)i * Mq + j) * 3 + a];
          real o[3];
          for (int a = 0; a < 3; ++a) o[a] = pb->ball_c[(size_t)(s0 + i) * 3 + a];
          project_ball(qv, o, pb->ball_r[s0 + i], ph);
          for (int a = 0; a < 3; ++a) {
            phb[((size_t)i * Mq + j) * 3 + a] = ph[a];
            wb[((size_t)i * Mq + j) * 3 + a] = qv[a] - ph[a];
          }
        }
        for (int j = 0; j < Mv; ++j) {
          real w3[3], qv[3], ph[3];
          matvec(sd[i].Av + (size_t)j * 3 * NL, 3, c + (size_t)i * NL, w3);
          for (int a = 0; a < 3; ++a) qv[a] = w3[a] + wv[((size_t)i * Mv + j) * 3 + a];
          project_ball(qv, NULL, pb->vnorm[b], ph);
          for (int a = 0; a < 3; ++a) {
            phv[((size_t)i * Mv + j) * 3 + a] = ph[a];
            wv[((size_t)i * Mv + j) * 3 + a] = qv[a] - ph[a];
          }
        }
      } else {
        /* start from the minimiser of the quadratic part (R9) */
        for (int l = 0; l < NL; ++l) rhs[l] *= rho;
        real c0[NL];
        chol_solve(NL, sd[i].L, sd[i].S, rhs, c0);
        num_ctx cx;
        cx.sd = &sd[i]; cx.zt = zt; cx.u = u + (size_t)i * NR; cx.y = yg + (size_t)i * Mg * 2;
        cx.M_gen = Mg; cx.rho = rho; cx.vmax = pb->gen_vmax[b]; cx.amax = pb->gen_amax[b];
        /* tolerance relative to the linear term's size in the K^-1 metric */
        real scale = dotn(rhs, c0, NL);
        if (!(scale > 0)) scale = 1;
        inner_it[i] += lbfgs_solve(&cx, c0, (real)pb->lbfgs_tol, scale, pb->lbfgs_max_iters,
                                   pb->lbfgs_mem > 0 ? pb->lbfgs_mem : 8);
        memcpy(c + (size_t)i * NL, c0, sizeof(c0));
      }
    }
    /* --- consensus (Eq. 18b), pinned rows fixed (R3) --- */
    memcpy(zo, z, sizeof(real) * (size_t)(N + 1) * AX * ND);
    real rp2 = 0;
    for (int j = 1; j < N; ++j) {
      real eL[NR], eR[NR];
      matvec(sd[j - 1].Mt, NR, c + (size_t)(j - 1) * NL, eL);  /* segment j-1 end rows */
      matvec(sd[j].Mt, NR, c + (size_t)j * NL, eR);            /* segment j start rows */
      for (int a = 0; a < AX; ++a)
        for (int r = 0; r < ND; ++r) {
          real left = eL[row_of(a, 1, r)], right = eR[row_of(a, 0, r)];
          real gap = left - right;
          rp2 += gap * gap;                                       /* Eq. 19 */
          if (pb->mode == OR_PIN && r == 0) continue;
          z[(j * AX + a) * ND + r] = (left + right) / 2;
        }
    }
    /* --- dual residual (Eq. 20, R10) --- */
    real rd2 = 0;
    for (int i = 0; i < N; ++i) {
      real dz[NR], rdv[NL];
      for (int a = 0; a < AX; ++a)
        for (int side = 0; side < 2; ++side)
          for (int r = 0; r < ND; ++r) {
            int q = row_of(a, side, r);
            size_t zi = ((size_t)(i + side) * AX + a) * ND + r;
            dz[q] = sd[i].E[q] * (z[zi] - zo[zi]);
          }
      for (int l = 0; l < NL; ++l) rdv[l] = 0;
      matvec_t_add(sd[i].Mt, NR, dz, rho, rdv);
      rd2 += dotn(rdv, rdv, NL);
    }
    /* --- slack, duals (Eq. 18c-e) --- */
    for (int i = 0; i < N; ++i) {
      real Mc[NR];
      matvec(sd[i].Mt, NR, c + (size_t)i * NL, Mc);
      for (int a = 0; a < AX; ++a)
        for (int side = 0; side < 2; ++side)
          for (int r = 0; r < ND; ++r) {
            int q = row_of(a, side, r);
            u[(size_t)i * NR + q] += sd[i].E[q] * (Mc[q] - z[((size_t)(i + side) * AX + a) * ND + r]);
          }
      if (nbox && pb->inner == OR_CLOSED) {
        real *Ac = (real *)malloc(sizeof(real) * nbox);
        matvec(sd[i].Ao, nbox, c + (size_t)i * NL, Ac);
        for (int q = 0; q < nbox; ++q) {
          size_t idx = (size_t)i * nbox + q;
          real sn = -(Ac[q] - sd[i].b[q] + v[idx]);
          s[idx] = sn > 0 ? sn : 0;                               /* Eq. 18d */
          v[idx] = v[idx] + Ac[q] + s[idx] - sd[i].b[q];           /* Eq. 18e */
        }
        free(Ac);
      }
      if (pb->inner == OR_NUMERIC) {
        for (int j = 0; j < Mg; ++j) {
          for (int g2 = 0; g2 < 2; ++g2) {
            const real *A = (g2 ? sd[i].Aga : sd[i].Agv) + (size_t)j * 3 * NL;
            real gmax = g2 ? pb->gen_amax[b] : pb->gen_vmax[b];
            real w3[3];
            matvec(A, 3, c + (size_t)i * NL, w3);
            real h = w3[0] * w3[0] + w3[1] * w3[1] + w3[2] * w3[2] - gmax * gmax;
            real g = h > 0 ? h * h : 0;
            yg[((size_t)i * Mg + j) * 2 + g2] += rho * g;          /* Eq. 17 dual, R9 */
          }
        }
      }
    }
    rp = sqrt_r(rp2); rd = sqrt_r(rd2);
    if (res->history) {
      res->history[((size_t)k * pb->B + b) * 2 + 0] = (double)rp;
      res->history[((size_t)k * pb->B + b) * 2 + 1] = (double)rd;
    }
    if (res->rho_hist) res->rho_hist[(size_t)k * pb->B + b] = (double)rho;
    if (!isfin(rp) || !isfin(rd)) { status = OR_NONFINITE; ++k; break; }
    if (pb->eps > 0 && rp < eps_tol && rd < eps_tol) { status = OR_CONVERGED; ++k; break; }
    if (pb->adaptive_rho) {
      /* UpdateRho (Eq. 22): keep the two residuals within a factor mu */
      real rn = rho;
      if (rp > (real)pb->rho_mu * rd) rn = rho * (real)pb->rho_tau_incr;
      else if (rd > (real)pb->rho_mu * rp) rn = rho / (real)pb->rho_tau_decr;
      if (rn != rho) {
        /* the scaled duals hold y / rho: keep the unscaled y fixed across
           the change, so every scaled dual is multiplied by rho_old / rho_new */
        const real f = rho / rn;
        for (size_t q = 0; q < (size_t)N * NR; ++q) u[q] *= f;
        for (size_t q = 0; q < (size_t)N * nbox; ++q) v[q] *= f;
        for (size_t q = 0; q < (size_t)N * Mq * 3; ++q) wb[q] *= f;
        for (size_t q = 0; q < (size_t)N * Mv * 3; ++q) wv[q] *= f;
        rho = rn;
        for (int i = 0; i < N; ++i)
          if (refactor_segment(&sd[i], pb, rho) != 0) { status = OR_NONFINITE; break; }
      }
    }
  }
  if (res->rho_final) res->rho_final[b] = (double)rho;
  /* outputs */
  real J = 0;
  for (int i = 0; i < N; ++i) {
    const real *ci = c + (size_t)i * NL;
    for (int a = 0; a < NL; ++a) {
      real acc = 0;
      for (int q = 0; q < NL; ++q) acc += sd[i].Qt[a * NL + q] * ci[q];
      J += ci[a] * acc;
    }
    for (int l = 0; l < NL; ++l) res->coeffs[(size_t)(s0 + i) * NL + l] = (double)ci[l];
  }
  res->cost[b] = (double)J;
  res->r_primal[b] = (double)rp;
  res->r_dual[b] = (double)rd;
  res->iters[b] = k;
  res->status[b] = status;
  if (res->z)
    for (int j = 0; j <= N; ++j)
      for (int q = 0; q < AX * ND; ++q) res->z[((size_t)(s0 + b + j)) * AX * ND + q] = (double)z[(size_t)j * AX * ND + q];
  if (res->u)
    for (size_t q = 0; q < (size_t)N * NR; ++q) res->u[(size_t)s0 * NR + q] = (double)u[q];
  if (res->s && nbox)
    for (size_t q = 0; q < (size_t)N * nbox; ++q) {
      res->s[(size_t)s0 * nbox + q] = (double)s[q];
      res->v[(size_t)s0 * nbox + q] = (double)v[q];
    }
  if (res->phi_b && Mq)
    for (size_t q = 0; q < (size_t)N * Mq * 3; ++q) {
      res->phi_b[(size_t)s0 * Mq * 3 + q] = (double)phb[q];
      res->w_b[(size_t)s0 * Mq * 3 + q] = (double)wb[q];
    }
  if (res->phi_v && Mv)
    for (size_t q = 0; q < (size_t)N * Mv * 3; ++q) {
      res->phi_v[(size_t)s0 * Mv * 3 + q] = (double)phv[q];
      res->w_v[(size_t)s0 * Mv * 3 + q] = (double)wv[q];
    }
  if (res->y_gen && Mg)
    for (size_t q = 0; q < (size_t)N * Mg * 2; ++q) res->y_gen[(size_t)s0 * Mg * 2 + q] = (double)yg[q];
  if (res->inner_iters)
    for (int i = 0; i < N; ++i) res->inner_iters[s0 + i] = inner_it[i];
  for (int i = 0; i < N; ++i) free_segment(&sd[i]);
  free(sd); free(z); free(zo); free(u); free(c); free(s); free(v);
  free(phb); free(wb); free(phv); free(wv); free(yg); free(inner_it);
  return 0;
}

/* Solve every trajectory of the batch, one after the other.
 * returns 0, or -1 if some local matrix is not positive definite, or -2 on
 * an invalid argument. */
int oracle_solve(const or_problem *pb, or_result *res) {
  if (!pb || !res || pb->B < 0 || pb->max_iters < 0 || !(pb->rho > 0)) return -2;
  if (pb->inner == OR_NUMERIC && (pb->M_box || pb->M_ball || pb->M_vn)) return -2;
  if (pb->inner == OR_CLOSED && pb->M_gen) return -2;
  for (int b = 0; b < pb->B; ++b)
    if (pb->seg_offset[b + 1] < pb->seg_offset[b]) return -2;
  for (int b = 0; b < pb->B; ++b)
    if (solve_one(pb, res, b) != 0) return -1;
  return 0;
}

/* Condition number (2-norm, by power iteration on K and K^-1) of the local
 * matrix of segment gi, raw and Jacobi-equilibrated; used by the tests to
 * state the oracle's own accuracy.  out[0] = cond(K), out[1] = cond(SKS). */
int oracle_segment_cond(const or_problem *pb, int b, int i_local, double *out) {
  int s0 = pb->seg_offset[b], N = pb->seg_offset[b + 1] - s0;
  seg_data sd;
  if (build_segment(&sd, pb, b, s0 + i_local, i_local == 0, i_local == N - 1) != 0) return -1;
  for (int pass = 0; pass < 2; ++pass) {
    real A[NL * NL];
    for (int i = 0; i < NL; ++i)
      for (int j = 0; j < NL; ++j)
        A[i * NL + j] = pass ? sd.S[i] * sd.K[i * NL + j] * sd.S[j] : sd.K[i * NL + j];
    real Lf[NL * NL], Sf[NL];
    chol_equil(NL, A, Lf, Sf);
    real x[NL], y[NL], lmax = 0, lmin_inv = 0;
    for (int i = 0; i < NL; ++i) x[i] = 1 + (real)i / NL;
    for (int it = 0; it < 2000; ++it) {
      matvec(A, NL, x, y);
      real n = sqrt_r(dotn(y, y, NL));
      for (int i = 0; i < NL; ++i) x[i] = y[i] / n;
      lmax = n;
    }
    for (int i = 0; i < NL; ++i) x[i] = 1 + (real)i / NL;
    for (int it = 0; it < 2000; ++it) {
      chol_solve(NL, Lf, Sf, x, y);
      real n = sqrt_r(dotn(y, y, NL));
      for (int i = 0; i < NL; ++i) x[i] = y[i] / n;
      lmin_inv = n;
    }
    out[pass] = (double)(lmax * lmin_inv);
  }
  free_segment(&sd);
  return 0;
}

/* sizeof(real) so that the tests can tell which precision they loaded */
int oracle_real_bytes(void) { return (int)sizeof(real); }

/* ------------------------------------------------------------------ */
/* hooks for the oracle's own pins                                     */
/* ------------------------------------------------------------------ */

/* projection of q onto the ball ||phi - o|| <= rad (o may be NULL) */
void oracle_project_ball(const double *q, const double *o, double rad, double *phi) {
  real qr[3], orr[3], ph[3];
  for (int a = 0; a < 3; ++a) { qr[a] = q[a]; orr[a] = o ? o[a] : 0; }
  project_ball(qr, o ? orr : NULL, (real)rad, ph);
  for (int a = 0; a < 3; ++a) phi[a] = (double)ph[a];
}

/* one numerical local step (L-BFGS on F of Eq. 16) of segment i_local of
 * trajectory b for the given consensus target zt[42], scaled dual u[42] and
 * general-constraint duals y[M_gen][2]; writes c[24], returns the L-BFGS
 * iteration count or -1. */
int oracle_numeric_local(const or_problem *pb, int b, int i_local, const double *zt,
                         const double *u, const double *y, double *c_out) {
  int s0 = pb->seg_offset[b], N = pb->seg_offset[b + 1] - s0;
  seg_data sd;
  if (build_segment(&sd, pb, b, s0 + i_local, i_local == 0, i_local == N - 1) != 0) return -1;
  real ztr[NR], ur[NR], rhs[NL], t42[NR], c0[NL];
  real *yr = (real *)calloc((size_t)(pb->M_gen ? pb->M_gen : 1) * 2, sizeof(real));
  for (int q = 0; q < NR; ++q) { ztr[q] = zt[q]; ur[q] = u[q]; }
  for (int q = 0; q < 2 * pb->M_gen; ++q) yr[q] = y[q];
  for (int q = 0; q < NR; ++q) t42[q] = sd.E[q] * (ztr[q] - ur[q]);
  for (int l = 0; l < NL; ++l) rhs[l] = 0;
  matvec_t_add(sd.Mt, NR, t42, pb->rho, rhs);
  chol_solve(NL, sd.L, sd.S, rhs, c0);
  num_ctx cx;
  cx.sd = &sd; cx.zt = ztr; cx.u = ur; cx.y = yr; cx.M_gen = pb->M_gen; cx.rho = pb->rho;
  cx.vmax = pb->gen_vmax[b]; cx.amax = pb->gen_amax[b];
  real scale = dotn(rhs, c0, NL);
  if (!(scale > 0)) scale = 1;
  int it = lbfgs_solve(&cx, c0, (real)pb->lbfgs_tol, scale, pb->lbfgs_max_iters,
                       pb->lbfgs_mem > 0 ? pb->lbfgs_mem : 8);
  for (int l = 0; l < NL; ++l) c_out[l] = (double)c0[l];
  free(yr);
  free_segment(&sd);
  return it;
}
