/*
 * ucac_oracle.c -- FP64 CPU oracle for one inner sweep of the two-level
 * component ADMM for UC-ACOPF (Zhang, Kim, Kim: "On Solving Unit Commitment
 * with AC Optimal Power Flow on GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke entry and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library: both read the same raw grid arrays
 * and each derives everything else on its own.
 *
 * Every routine follows the paper's order of steps (Sec. III-A, Eq. step:uc
 * .. step:y, Algorithm 1; Sec. III-B, Algorithm 2).  Where the paper defers a
 * subproblem to prior work the reading taken here is stated beside it:
 *   R1-R4  coupling rows (Eq. uc_duplicate..ramp_up, Eq. coupling),
 *   R5     generator x-update, solved by nested 1-D bisection,
 *   R6     branch x-update, augmented Lagrangian + damped projected Newton,
 *   R7     x-bar^UC update, 27-face box-QP enumeration,
 *   R8     bus x-bar^OPF update, explicit 2x2 multiplier solve,
 *   R9-R12 z, y, residuals, outer update.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -o liboracle.so ucac_oracle.c -lm
 * (-ffp-contract=off keeps every product and sum separately rounded, so the
 * UC stage costs reproduce bit for bit the evaluation order stated below).
 * Built a second time with -fopenmp (liboracle_omp.so), the independent
 * per-(period, generator) and per-(period, line) subproblems of the x-step
 * run on all host cores (OpenMP over components); every other step, and
 * every sum, stays sequential, so both builds give the same bits.
 *
 * Parity status of each function is given in its header comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- input -- */
typedef struct orc_grid {
  int32_t n_bus, n_branch, n_gen, T, ref_bus;
  const double *Pd, *Qd;                      /* [T][n_bus] */
  const double *Gs, *Bs, *Vmin, *Vmax;        /* [n_bus] */
  const int32_t *br_from, *br_to;             /* [n_branch] */
  const double *br_r, *br_x, *br_b, *br_rate; /* [n_branch] */
  const int32_t *gen_bus;                     /* [n_gen] */
  const double *Pmin, *Pmax, *Qmin, *Qmax, *c2, *c1, *c0, *c_su, *c_sd, *RU, *RD, *SU, *SD;
  const int32_t *TU, *TD, *u0, *L0, *F0;
  const double *p0;
  double base_mva;
} orc_grid;

typedef struct orc_params {
  double rho_pq, rho_va, rho_uc;
  double eps_in, eps_out, tau, theta, beta0, lam_max;
  double eta, omega_rel, c_init_rel, c_max_rel;
  double rho_mu, rho_tau;             /* adaptive penalty: balance ratio and factor */
  int32_t K_AL, K_N, L_max, uc_relax; /* uc_relax: box relaxation of the UC step */
  int32_t rho_every, pad;             /* adaptive penalty: check period (0: off) */
} orc_params;

/* ------------------------------------------------------- UC DP (Alg. 2) -- */
/*
 * Stage cost L_t(a,b) of Sec. III-B, with a = u^on_{t-1}, b = u^on_t, su/sd
 * eliminated as su = max(0,b-a), sd = max(0,a-b).  The AL terms of the
 * duplicate rows (Eq. uc_duplicate) are written in target form
 * rho/2 (u_k - tau_k)^2 with tau_k = ubar_k - z_k - y_k/rho (the constant
 * dropped is independent of u).  Evaluation order (fixed, separately rounded):
 *   e_k = u_k - tau_k
 *   q   = ((e_on*e_on) + (e_su*e_su)) + (e_sd*e_sd)
 *   L   = ((c0*b + csu*su) + csd*sd) + (0.5*rho)*q
 * Parity pinned: brute force over all schedules (tests).
 */
EXPORT void orc_uc_stagecost(int T, double c0, double csu, double csd, double rho,
                             const double *tau_on, const double *tau_su, const double *tau_sd,
                             double *L /* [T][4], index a*2+b */) {
  double hr = 0.5 * rho;
  for (int t = 0; t < T; ++t) {
    for (int a = 0; a < 2; ++a) {
      for (int b = 0; b < 2; ++b) {
        double su = (b > a) ? 1.0 : 0.0;
        double sd = (a > b) ? 1.0 : 0.0;
        double bb = (double)b;
        double e_on = bb - tau_on[t];
        double e_su = su - tau_su[t];
        double e_sd = sd - tau_sd[t];
        double q = ((e_on * e_on) + (e_su * e_su)) + (e_sd * e_sd);
        double lin = ((c0 * bb + csu * su) + csd * sd);
        L[t * 4 + a * 2 + b] = lin + hr * q;
      }
    }
  }
}

/*
 * Algorithm 2 (backward induction over t = T..1 with the two options "stay"
 * (Eq. c_keep_formula) and "switch and hold for T_min periods"
 * (Eq. c_switch_formula); stay is chosen when c_stay <= c_switch).
 * Readings: c_{T+1,s} = 0; a switch whose hold window passes T holds to T;
 * the first K0 periods are forced to the initial state u0 (K0 = L_g if u0=1,
 * F_g if u0=0), which is the "break" branch of Algorithm 2.
 * The switch cost is summed as (L(s,1-s) + sum_{t'} L(1-s,1-s) ascending t')
 * + c_next, left to right.
 * Returns c_{1,u0}; writes u^on_t (0/1) for t = 1..T.
 * Parity pinned: brute-force enumeration of all 2^T schedules (tests).
 */
EXPORT double orc_dp(int T, int TU, int TD, int u0, int K0, const double *L, int32_t *u_on) {
  double *c = (double *)calloc((size_t)(T + 2) * 2, sizeof(double));
  unsigned char *dec = (unsigned char *)calloc((size_t)(T + 2) * 2, 1);
  /* c[t][s] for t = 1..T+1 (1-based) */
#define C_(t, s) c[(size_t)(t) * 2 + (s)]
#define D_(t, s) dec[(size_t)(t) * 2 + (s)]
#define LL(t, a, b) L[(size_t)((t)-1) * 4 + (a) * 2 + (b)]
  C_(T + 1, 0) = 0.0;
  C_(T + 1, 1) = 0.0;
  if (K0 < 0) K0 = 0;
  if (K0 > T) K0 = T;
  for (int t = T; t >= K0 + 1; --t) {
    for (int s = 0; s < 2; ++s) {
      int ns = 1 - s;
      double stay = LL(t, s, s) + C_(t + 1, s);
      int Tm = (ns == 1) ? TU : TD;
      if (Tm < 1) Tm = 1;
      int e = t + Tm - 1;
      if (e > T) e = T;
      double sw = LL(t, s, ns);
      for (int tp = t + 1; tp <= e; ++tp) sw = sw + LL(tp, ns, ns);
      sw = sw + C_(e + 1, ns);
      if (stay <= sw) {
        C_(t, s) = stay;
        D_(t, s) = 0;
      } else {
        C_(t, s) = sw;
        D_(t, s) = 1;
      }
    }
  }
  double cost;
  if (K0 > 0) {
    double acc = LL(1, u0, u0);
    for (int t = 2; t <= K0; ++t) acc = acc + LL(t, u0, u0);
    cost = acc + C_(K0 + 1, u0);
  } else {
    cost = C_(1, u0);
  }
  for (int t = 1; t <= K0; ++t) u_on[t - 1] = u0;
  int s = u0, t = K0 + 1;
  while (t <= T) {
    if (D_(t, s) == 0) {
      u_on[t - 1] = s;
      t += 1;
    } else {
      int ns = 1 - s;
      int Tm = (ns == 1) ? TU : TD;
      if (Tm < 1) Tm = 1;
      int e = t + Tm - 1;
      if (e > T) e = T;
      for (int k = t; k <= e; ++k) u_on[k - 1] = ns;
      s = ns;
      t = e + 1;
    }
  }
#undef C_
#undef D_
#undef LL
  free(c);
  free(dec);
  return cost;
}

/* ------------------------------------------------- generator (R5) ------ */
/*
 * Generator x-update for one (t,g): minimise over p in [0,Pmax] (Eq.
 * acopf_gen_p_bounds), q in [min(0,Qmin),Qmax], phat in [0,Pmax] (the local
 * copy of p_{t-1}) and the six slacks s >= 0 of Eq. pg_lo..ramp_up
 *   c2' p^2 + c1' p + sum_r rho/2 (a_r(x) - t_r)^2
 * over the rows pl,pu,ql,qu,rd,ru (F2) and gp,gq,tc (F3).  Eliminating each
 * slack in closed form leaves a convex C^1 piecewise quadratic; q separates.
 * Solved here by nested bisection on the monotone derivatives (a different
 * method from the CUDA path's piece enumeration).
 * prm = {c2', c1', rho, Pmax, qlo, qhi, p0}; tg = {t_pl,t_pu,t_ql,t_qu,t_rd,
 * t_ru,t_gp,t_gq,t_tc}; out = {p,q,phat,s_pl,s_pu,s_ql,s_qu,s_rd,s_ru}.
 * Parity pinned: KKT residual, dense grid, closed form when no slack row is
 * active (tests).
 */
static double dmin0(double v) { return v < 0.0 ? v : 0.0; }
static double dmax0(double v) { return v > 0.0 ? v : 0.0; }

typedef struct {
  double c2, c1, rho, pmax, t_pl, t_pu, t_rd, t_ru, t_gp, t_tc;
} genp_t;

static double gen_Fp(const genp_t *G, double p) {
  return 2.0 * G->c2 * p + G->c1 + G->rho * (p - G->t_gp) + G->rho * dmin0(p - G->t_pl) +
         G->rho * dmax0(p - G->t_pu);
}
static double gen_Hp(const genp_t *G, double d) {
  return G->rho * dmin0(d - G->t_rd) + G->rho * dmax0(d - G->t_ru);
}

/* root of an increasing function on [lo,hi] by bisection (clamped) */
#define BISECT_ITERS 200
static double gen_phat_star(const genp_t *G, double p) {
  /* d/dphat [rho/2 (phat - t_tc)^2 + H(p - phat)] = rho (phat - t_tc) - H'(p - phat) */
  double lo = 0.0, hi = G->pmax;
  double flo = G->rho * (lo - G->t_tc) - gen_Hp(G, p - lo);
  if (flo >= 0.0) return lo;
  double fhi = G->rho * (hi - G->t_tc) - gen_Hp(G, p - hi);
  if (fhi <= 0.0) return hi;
  for (int k = 0; k < BISECT_ITERS; ++k) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double fm = G->rho * (mid - G->t_tc) - gen_Hp(G, p - mid);
    if (fm > 0.0) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

static double gen_outer_deriv(const genp_t *G, int has_prev, double p0, double p, double *ph_out) {
  double ph = has_prev ? gen_phat_star(G, p) : p0;
  if (ph_out) *ph_out = ph;
  return gen_Fp(G, p) + gen_Hp(G, p - ph);
}

EXPORT void orc_gen_solve(const double *prm, int has_prev, const double *tg, double *out) {
  genp_t G;
  G.c2 = prm[0];
  G.c1 = prm[1];
  G.rho = prm[2];
  G.pmax = prm[3];
  double qlo = prm[4], qhi = prm[5], p0 = prm[6];
  G.t_pl = tg[0];
  G.t_pu = tg[1];
  G.t_rd = tg[4];
  G.t_ru = tg[5];
  G.t_gp = tg[6];
  G.t_tc = tg[8];
  double t_ql = tg[2], t_qu = tg[3], t_gq = tg[7];
  double rho = G.rho;
  /* q: derivative rho(q - t_gq) + rho min(0,q - t_ql) + rho max(0,q - t_qu) */
  double q;
  {
    double lo = qlo, hi = qhi;
#define QD(v) (rho * ((v)-t_gq) + rho * dmin0((v)-t_ql) + rho * dmax0((v)-t_qu))
    if (QD(lo) >= 0.0) q = lo;
    else if (QD(hi) <= 0.0) q = hi;
    else {
      for (int k = 0; k < BISECT_ITERS; ++k) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (QD(mid) > 0.0) hi = mid; else lo = mid;
      }
      q = 0.5 * (lo + hi);
    }
#undef QD
  }
  /* p: G(p) = min_phat [...] is convex C^1 with G'(p) = F'(p) + H'(p - phat*(p)) */
  double p, ph;
  {
    double lo = 0.0, hi = G.pmax;
    if (gen_outer_deriv(&G, has_prev, p0, lo, NULL) >= 0.0) p = lo;
    else if (gen_outer_deriv(&G, has_prev, p0, hi, NULL) <= 0.0) p = hi;
    else {
      for (int k = 0; k < BISECT_ITERS; ++k) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (gen_outer_deriv(&G, has_prev, p0, mid, NULL) > 0.0) hi = mid; else lo = mid;
      }
      p = 0.5 * (lo + hi);
    }
    gen_outer_deriv(&G, has_prev, p0, p, &ph);
  }
  double d = p - ph;
  out[0] = p;
  out[1] = q;
  out[2] = ph;
  out[3] = dmax0(p - G.t_pl);  /* s_pl */
  out[4] = dmax0(G.t_pu - p);  /* s_pu */
  out[5] = dmax0(q - t_ql);    /* s_ql */
  out[6] = dmax0(t_qu - q);    /* s_qu */
  out[7] = dmax0(d - G.t_rd);  /* s_rd */
  out[8] = dmax0(G.t_ru - d);  /* s_ru */
}

/* --------------------------------------------------------- branch (R6) --- */
/*
 * Branch x-update for one (t, line ij).  Variables
 *   v = (w_i, w_j, wR_ij, wI_ij, theta_i, theta_j, sigma_ij, sigma_ji)
 * with bounds Vmin^2 <= w <= Vmax^2 (Eq. uc_acopf_w_bound),
 * |wR|,|wI| <= Vmax_i Vmax_j, |theta| <= 2 pi, 0 <= sigma <= rate^2.
 * Flows are linear in v (Eq. acopf, the four flow equations; the second pair
 * read as the j->i direction).  Equalities
 *   h0 = wR^2 + wI^2 - w_i w_j,  h1 = theta_i - theta_j - atan2(wI, wR),
 *   h2 = p_ij^2 + q_ij^2 + sigma_ij - rate^2, h3 = same for ji
 * (Eq. acopf: the product and angle equations and the two line limits with
 * slacks).  Objective: the eight consensus-row AL terms rho/2 (a_r - t_r)^2
 * plus mu^T h + c/2 |h|^2.
 * Augmented-Lagrangian outer loop (<= K_AL): inner solve, mu += c h, stop
 * when |h|_inf <= eta; c *= 10 (capped) when |h| fell by less than 4x.
 * Inner loop (<= K_N): damped projected Newton with an epsilon-active set,
 * Levenberg-Marquardt damping adapted by the ratio of actual to predicted
 * decrease (a trust-region rule); stop when the projected gradient
 * |P(v - g) - v|_inf <= omega.
 * The CUDA path runs the same algorithm; parity is pinned independently by
 * KKT/second-order checks, grid search and exact AC points (tests).
 */
typedef struct {
  double Gii, Bii, Gij, Bij, Gjj, Bjj, Gji, Bji, rate2;
  double lo[8], hi[8];
} brc_t;

typedef struct {
  double tg[8];
  double rpq, rva;
  double mu[4];
  double c;
} brp_t;

static void br_flows(const brc_t *K, const double *v, double *a) {
  a[0] = K->Gii * v[0] + K->Gij * v[2] + K->Bij * v[3];
  a[1] = -K->Bii * v[0] - K->Bij * v[2] + K->Gij * v[3];
  a[2] = K->Gjj * v[1] + K->Gji * v[2] - K->Bji * v[3];
  a[3] = -K->Bjj * v[1] - K->Bji * v[2] - K->Gji * v[3];
}

static void br_cons(const brc_t *K, const double *v, const double *a, double *h) {
  h[0] = v[2] * v[2] + v[3] * v[3] - v[0] * v[1];
  h[1] = v[4] - v[5] - atan2(v[3], v[2]);
  h[2] = a[0] * a[0] + a[1] * a[1] + v[6] - K->rate2;
  h[3] = a[2] * a[2] + a[3] * a[3] + v[7] - K->rate2;
}

static double br_phi(const brc_t *K, const brp_t *P, const double *v) {
  double a[4], h[4];
  br_flows(K, v, a);
  br_cons(K, v, a, h);
  double f = 0.0;
  for (int r = 0; r < 4; ++r) f += 0.5 * P->rpq * (a[r] - P->tg[r]) * (a[r] - P->tg[r]);
  f += 0.5 * P->rva * (v[0] - P->tg[4]) * (v[0] - P->tg[4]);
  f += 0.5 * P->rva * (v[1] - P->tg[5]) * (v[1] - P->tg[5]);
  f += 0.5 * P->rva * (v[4] - P->tg[6]) * (v[4] - P->tg[6]);
  f += 0.5 * P->rva * (v[5] - P->tg[7]) * (v[5] - P->tg[7]);
  for (int k = 0; k < 4; ++k) f += P->mu[k] * h[k] + 0.5 * P->c * h[k] * h[k];
  return f;
}

/* gradient g[8] and Hessian H[8][8] of the inner objective */
static void br_derivs(const brc_t *K, const brp_t *P, const double *v, double *g, double H[8][8]) {
  double a[4], h[4];
  br_flows(K, v, a);
  br_cons(K, v, a, h);
  double da[4][8];
  memset(da, 0, sizeof(da));
  da[0][0] = K->Gii; da[0][2] = K->Gij; da[0][3] = K->Bij;
  da[1][0] = -K->Bii; da[1][2] = -K->Bij; da[1][3] = K->Gij;
  da[2][1] = K->Gjj; da[2][2] = K->Gji; da[2][3] = -K->Bji;
  da[3][1] = -K->Bjj; da[3][2] = -K->Bji; da[3][3] = -K->Gji;
  double dh[4][8];
  memset(dh, 0, sizeof(dh));
  double r2 = v[2] * v[2] + v[3] * v[3];
  dh[0][0] = -v[1]; dh[0][1] = -v[0]; dh[0][2] = 2.0 * v[2]; dh[0][3] = 2.0 * v[3];
  if (r2 > 1e-300) {
    dh[1][2] = v[3] / r2;
    dh[1][3] = -v[2] / r2;
  }
  dh[1][4] = 1.0; dh[1][5] = -1.0;
  for (int i = 0; i < 8; ++i) {
    dh[2][i] = 2.0 * a[0] * da[0][i] + 2.0 * a[1] * da[1][i];
    dh[3][i] = 2.0 * a[2] * da[2][i] + 2.0 * a[3] * da[3][i];
  }
  dh[2][6] += 1.0;
  dh[3][7] += 1.0;
  for (int i = 0; i < 8; ++i) {
    g[i] = 0.0;
    for (int j = 0; j < 8; ++j) H[i][j] = 0.0;
  }
  /* consensus rows */
  for (int r = 0; r < 4; ++r) {
    double e = a[r] - P->tg[r];
    for (int i = 0; i < 8; ++i) {
      g[i] += P->rpq * e * da[r][i];
      for (int j = 0; j < 8; ++j) H[i][j] += P->rpq * da[r][i] * da[r][j];
    }
  }
  g[0] += P->rva * (v[0] - P->tg[4]);
  g[1] += P->rva * (v[1] - P->tg[5]);
  g[4] += P->rva * (v[4] - P->tg[6]);
  g[5] += P->rva * (v[5] - P->tg[7]);
  H[0][0] += P->rva; H[1][1] += P->rva; H[4][4] += P->rva; H[5][5] += P->rva;
  /* constraint terms: (mu + c h) grad h, (mu + c h) hess h + c grad h grad h^T */
  for (int k = 0; k < 4; ++k) {
    double lam = P->mu[k] + P->c * h[k];
    for (int i = 0; i < 8; ++i) {
      g[i] += lam * dh[k][i];
      for (int j = 0; j < 8; ++j) H[i][j] += P->c * dh[k][i] * dh[k][j];
    }
    if (k == 0) {
      H[0][1] += -lam; H[1][0] += -lam; H[2][2] += 2.0 * lam; H[3][3] += 2.0 * lam;
    } else if (k == 1) {
      if (r2 > 1e-300) {
        double r4 = r2 * r2;
        H[2][2] += lam * (-2.0 * v[2] * v[3] / r4);
        H[3][3] += lam * (2.0 * v[2] * v[3] / r4);
        H[2][3] += lam * ((v[2] * v[2] - v[3] * v[3]) / r4);
        H[3][2] += lam * ((v[2] * v[2] - v[3] * v[3]) / r4);
      }
    } else {
      int r0 = (k == 2) ? 0 : 2;
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j)
          H[i][j] += lam * 2.0 * (da[r0][i] * da[r0][j] + da[r0 + 1][i] * da[r0 + 1][j]);
    }
  }
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* dense Cholesky on an n x n SPD matrix (row-major, stride 8); 0 on failure */
static int chol_solve(int n, double A[8][8], double *b) {
  double Lm[8][8];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Lm[i][j] = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = A[j][j];
    for (int k = 0; k < j; ++k) s -= Lm[j][k] * Lm[j][k];
    if (!(s > 0.0)) return 0;
    double d = sqrt(s);
    Lm[j][j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i][j];
      for (int k = 0; k < j; ++k) t -= Lm[i][k] * Lm[j][k];
      Lm[i][j] = t / d;
    }
  }
  double y[8];
  for (int i = 0; i < n; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= Lm[i][k] * y[k];
    y[i] = t / Lm[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = y[i];
    for (int k = i + 1; k < n; ++k) t -= Lm[k][i] * b[k];
    b[i] = t / Lm[i][i];
  }
  return 1;
}

/* projected-gradient stationarity |P(v - g) - v|_inf */
static double br_pg(const brc_t *K, const double *v, const double *g) {
  double m = 0.0;
  for (int i = 0; i < 8; ++i) {
    double d = fabs(clampd(v[i] - g[i], K->lo[i], K->hi[i]) - v[i]);
    if (d > m) m = d;
  }
  return m;
}

/*
 * Inner solve of the AL subproblem (reading R6): projected Newton with an
 * epsilon-active set and a trust radius on the step.
 *   1. stationarity test |P(v - g) - v|_inf <= omega;
 *   2. active set A: within eps of a bound with the gradient pointing out
 *      (eps = min(1e-6, diagonally scaled projected-gradient size)); active
 *      coordinates move onto their bound;
 *   3. Newton step on the free set from the Cholesky factor of H_FF (shifted
 *      by lambda I, lambda = 1e-10 max diag H growing x10, only when H_FF is
 *      not positive definite);
 *   4. an undamped step of size <= 1e-9 (1 + |v|_inf), or one whose predicted
 *      decrease is <= 1e-12 (1 + |phi|) (below the rounding level of phi, where
 *      the ratio test cannot judge it), is taken as the final, quadratically
 *      convergent step;
 *   5. otherwise the step is cut to the radius Delta (inf-norm), projected onto
 *      the box, and accepted when actual >= 1e-4 x predicted decrease; Delta is
 *      doubled after a very successful radius-limited step and set to a quarter
 *      of the rejected step's length after a failure.
 * Returns iterations used; *conv = 1 when 1 or 4 ended the loop.
 */
static int br_inner(const brc_t *K, const brp_t *P, double *v, int K_N, double omega, double *Delta, int *conv) {
  double g[8], H[8][8];
  double f = br_phi(K, P, v);
  br_derivs(K, P, v, g, H);
  int it = 0;
  *conv = 0;
  for (; it < K_N; ++it) {
    double pg = br_pg(K, v, g);
    if (pg <= omega) {
      *conv = 1;
      break;
    }
    double hmax = 0.0, vmax = 0.0;
    for (int i = 0; i < 8; ++i) {
      if (H[i][i] > hmax) hmax = H[i][i];
      if (fabs(v[i]) > vmax) vmax = fabs(v[i]);
    }
    double eps = 0.0;
    for (int i = 0; i < 8; ++i) {
      double di = (H[i][i] > 0.0) ? g[i] / H[i][i] : g[i];
      double sz = fabs(clampd(v[i] - di, K->lo[i], K->hi[i]) - v[i]);
      if (sz > eps) eps = sz;
    }
    if (eps > 1e-6) eps = 1e-6;
    int act[8], fr[8], nf = 0;
    double d[8];
    for (int i = 0; i < 8; ++i) {
      act[i] = 0;
      d[i] = 0.0;
      if (v[i] <= K->lo[i] + eps && g[i] > 0.0) {
        act[i] = 1;
        d[i] = K->lo[i] - v[i];
      } else if (v[i] >= K->hi[i] - eps && g[i] < 0.0) {
        act[i] = 1;
        d[i] = K->hi[i] - v[i];
      } else {
        fr[nf++] = i;
      }
    }
    double lm = 0.0, rhs[8];
    int ok = 0;
    for (int tries = 0; tries < 40; ++tries) {
      double A[8][8];
      for (int a = 0; a < nf; ++a) {
        int i = fr[a];
        double r = -g[i];
        for (int j = 0; j < 8; ++j)
          if (act[j]) r -= H[i][j] * d[j];
        rhs[a] = r;
        for (int b = 0; b < nf; ++b) A[a][b] = H[i][fr[b]];
        A[a][a] += lm;
      }
      if (nf == 0 || chol_solve(nf, A, rhs)) {
        ok = 1;
        break;
      }
      lm = (lm == 0.0) ? 1e-10 * hmax : 10.0 * lm;
    }
    if (!ok) break;
    for (int a = 0; a < nf; ++a) d[fr[a]] = rhs[a];
    double dn = 0.0;
    for (int i = 0; i < 8; ++i)
      if (fabs(d[i]) > dn) dn = fabs(d[i]);
    double vt[8], s[8];
    double predN = 0.0; /* decrease predicted by the full undamped step */
    if (lm == 0.0) {
      double gd = 0.0, dHd = 0.0;
      for (int i = 0; i < 8; ++i) {
        gd += g[i] * d[i];
        double t = 0.0;
        for (int j = 0; j < 8; ++j) t += H[i][j] * d[j];
        dHd += d[i] * t;
      }
      predN = -(gd + 0.5 * dHd);
    }
    if (lm == 0.0 && (dn <= 1e-9 * (1.0 + vmax) || predN <= 1e-12 * (1.0 + fabs(f)))) {
      for (int i = 0; i < 8; ++i) v[i] = clampd(v[i] + d[i], K->lo[i], K->hi[i]);
      *conv = 1;
      ++it;
      break;
    }
    double scale = (dn > *Delta) ? *Delta / dn : 1.0;
    double smax = 0.0;
    for (int i = 0; i < 8; ++i) {
      vt[i] = clampd(v[i] + scale * d[i], K->lo[i], K->hi[i]);
      s[i] = vt[i] - v[i];
      if (fabs(s[i]) > smax) smax = fabs(s[i]);
    }
    double gs = 0.0, sHs = 0.0;
    for (int i = 0; i < 8; ++i) {
      gs += g[i] * s[i];
      double t = 0.0;
      for (int j = 0; j < 8; ++j) t += H[i][j] * s[j];
      sHs += s[i] * t;
    }
    double pred = -(gs + 0.5 * sHs);
    double ft = br_phi(K, P, vt);
    double ared = f - ft;
    if (pred > 0.0 && ared >= 1e-4 * pred) {
      for (int i = 0; i < 8; ++i) v[i] = vt[i];
      f = ft;
      br_derivs(K, P, v, g, H);
      if (ared >= 0.75 * pred && scale < 1.0) *Delta = 2.0 * *Delta;
    } else {
      *Delta = 0.25 * smax;
      if (*Delta <= 1e-15 * (1.0 + vmax)) break; /* stalled */
    }
  }
  return it;
}

/*
 * cst = {Gii,Bii,Gij,Bij,Gjj,Bjj,Gji,Bji,rate2, lo[8], hi[8]} (25 doubles)
 * v[8], mu[4], *c are the warm start on input and the result on output.
 * info[0] = Newton iterations, info[1] = AL iterations, info[2] = status
 * (0 converged, 1 iteration cap).  a_out[8] = the eight row values.
 */
EXPORT void orc_branch_solve(const double *cst, const double *tgt, double rho_pq, double rho_va,
                             double eta, double omega, double c_max, int K_AL, int K_N,
                             double *v, double *mu, double *c, double *a_out, int32_t *info) {
  brc_t K;
  K.Gii = cst[0]; K.Bii = cst[1]; K.Gij = cst[2]; K.Bij = cst[3];
  K.Gjj = cst[4]; K.Bjj = cst[5]; K.Gji = cst[6]; K.Bji = cst[7];
  K.rate2 = cst[8];
  for (int i = 0; i < 8; ++i) {
    K.lo[i] = cst[9 + i];
    K.hi[i] = cst[17 + i];
  }
  brp_t P;
  for (int r = 0; r < 8; ++r) P.tg[r] = tgt[r];
  P.rpq = rho_pq;
  P.rva = rho_va;
  for (int k = 0; k < 4; ++k) P.mu[k] = mu[k];
  P.c = *c;
  for (int i = 0; i < 8; ++i) v[i] = clampd(v[i], K.lo[i], K.hi[i]);
  double a[4], h[4];
  br_flows(&K, v, a);
  br_cons(&K, v, a, h);
  double hprev = INFINITY; /* c grows only when consecutive AL rounds stall */
  double Delta = 1.0;      /* trust radius, kept across the AL rounds of this solve */
  int newton = 0, al = 0, status = 1;
  for (al = 0; al < K_AL;) {
    int conv = 0;
    if (Delta < 1e-3) Delta = 1e-3;
    newton += br_inner(&K, &P, v, K_N, omega, &Delta, &conv);
    br_flows(&K, v, a);
    br_cons(&K, v, a, h);
    double hn = 0.0;
    for (int k = 0; k < 4; ++k) {
      P.mu[k] += P.c * h[k];
      if (fabs(h[k]) > hn) hn = fabs(h[k]);
    }
    ++al;
    if (hn <= eta && conv) {
      status = 0;
      break;
    }
    if (hn > 0.25 * hprev) {
      P.c = 10.0 * P.c;
      if (P.c > c_max) P.c = c_max;
    }
    hprev = hn;
  }
  for (int k = 0; k < 4; ++k) mu[k] = P.mu[k];
  *c = P.c;
  br_flows(&K, v, a);
  for (int r = 0; r < 4; ++r) a_out[r] = a[r];
  a_out[4] = v[0];
  a_out[5] = v[1];
  a_out[6] = v[4];
  a_out[7] = v[5];
  info[0] = newton;
  info[1] = al;
  info[2] = status;
}

/* ------------------------------------------------------------ bus (R8) --- */
/*
 * Bus x-bar^OPF update for one (t,i): minimise sum_v W_v/2 (v - m_v)^2 subject
 * to the two linear balance equations of Eq. acopf (P and Q balance)
 *   sum_v aP_v v = Pd,  sum_v aQ_v v = Qd.
 * Stationarity v = m - (nuP aP + nuQ aQ)/W and the 2x2 system for (nuP,nuQ)
 * are solved explicitly.
 * Parity pinned: generic dense KKT solve and balance residual (tests).
 */
EXPORT void orc_bus_solve(int n, const double *W, const double *m, const double *aP, const double *aQ,
                          double Pd, double Qd, double *v) {
  double M00 = 0.0, M01 = 0.0, M11 = 0.0, r0 = 0.0, r1 = 0.0;
  for (int k = 0; k < n; ++k) {
    M00 += aP[k] * aP[k] / W[k];
    M01 += aP[k] * aQ[k] / W[k];
    M11 += aQ[k] * aQ[k] / W[k];
    r0 += aP[k] * m[k];
    r1 += aQ[k] * m[k];
  }
  r0 -= Pd;
  r1 -= Qd;
  double nuP, nuQ;
  if (M01 == 0.0) {
    nuP = (M00 > 0.0) ? r0 / M00 : 0.0;
    nuQ = (M11 > 0.0) ? r1 / M11 : 0.0;
  } else {
    double det = M00 * M11 - M01 * M01;
    nuP = (M11 * r0 - M01 * r1) / det;
    nuQ = (M00 * r1 - M01 * r0) / det;
  }
  for (int k = 0; k < n; ++k) v[k] = m[k] - (nuP * aP[k] + nuQ * aQ[k]) / W[k];
}

/* ---------------------------------------------------------- x-bar UC (R7) - */
/*
 * Minimise 1/2 x^T H x - g^T x over [0,1]^n (n <= 3) by enumerating the 3^n
 * faces (each coordinate free, at 0 or at 1): on each face solve the reduced
 * linear system; keep candidates inside the box whose fixed coordinates have
 * KKT-consistent gradient signs; return the one of least objective (falling
 * back to the least objective among box-feasible candidates).
 * Parity pinned: dense grid + KKT (tests).
 */
static int solve_small(int n, double A[3][3], double *b) {
  /* Gaussian elimination with partial pivoting */
  int piv[3] = {0, 1, 2};
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
    if (A[p][k] == 0.0) return 0;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t;
      }
      double t = b[k]; b[k] = b[p]; b[p] = t;
      int ti = piv[k]; piv[k] = piv[p]; piv[p] = ti;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i][k] / A[k][k];
      for (int j = k; j < n; ++j) A[i][j] -= f * A[k][j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = b[i];
    for (int j = i + 1; j < n; ++j) t -= A[i][j] * b[j];
    b[i] = t / A[i][i];
  }
  return 1;
}

EXPORT void orc_boxqp(int n, const double *Hf, const double *gv, double *x) {
  double best = INFINITY, bestf = INFINITY;
  double xb[3] = {0, 0, 0}, xf[3] = {0, 0, 0};
  int have = 0, havef = 0;
  int nf = 1;
  for (int i = 0; i < n; ++i) nf *= 3;
  double scale = 0.0;
  for (int i = 0; i < n; ++i) {
    if (fabs(gv[i]) > scale) scale = fabs(gv[i]);
    for (int j = 0; j < n; ++j)
      if (fabs(Hf[i * n + j]) > scale) scale = fabs(Hf[i * n + j]);
  }
  double tolx = 1e-12, tolg = 1e-12 * scale;
  for (int face = 0; face < nf; ++face) {
    int st[3], code = face;
    for (int i = 0; i < n; ++i) {
      st[i] = code % 3; /* 0 free, 1 at 0, 2 at 1 */
      code /= 3;
    }
    double xc[3];
    int fr[3], m = 0;
    for (int i = 0; i < n; ++i) {
      if (st[i] == 0) fr[m++] = i;
      xc[i] = (st[i] == 2) ? 1.0 : 0.0;
    }
    if (m > 0) {
      double A[3][3], b[3];
      for (int a = 0; a < m; ++a) {
        int i = fr[a];
        double r = gv[i];
        for (int j = 0; j < n; ++j)
          if (st[j] != 0) r -= Hf[i * n + j] * xc[j];
        b[a] = r;
        for (int c = 0; c < m; ++c) A[a][c] = Hf[i * n + fr[c]];
      }
      if (!solve_small(m, A, b)) continue;
      for (int a = 0; a < m; ++a) xc[fr[a]] = b[a];
    }
    int inbox = 1;
    for (int i = 0; i < n; ++i)
      if (xc[i] < -tolx || xc[i] > 1.0 + tolx) inbox = 0;
    if (!inbox) continue;
    double fval = 0.0, gr[3];
    for (int i = 0; i < n; ++i) {
      double t = 0.0;
      for (int j = 0; j < n; ++j) t += Hf[i * n + j] * xc[j];
      gr[i] = t - gv[i];
      fval += 0.5 * xc[i] * t - gv[i] * xc[i];
    }
    int kkt = 1;
    for (int i = 0; i < n; ++i) {
      if (st[i] == 1 && gr[i] < -tolg) kkt = 0;
      if (st[i] == 2 && gr[i] > tolg) kkt = 0;
    }
    if (fval < bestf) {
      bestf = fval;
      for (int i = 0; i < n; ++i) xf[i] = xc[i];
      havef = 1;
    }
    if (kkt && fval < best) {
      best = fval;
      for (int i = 0; i < n; ++i) xb[i] = xc[i];
      have = 1;
    }
  }
  for (int i = 0; i < n; ++i) {
    double r = have ? xb[i] : (havef ? xf[i] : 0.0);
    x[i] = clampd(r, 0.0, 1.0);
  }
}

/* ------------------------------------------------------------ instance --- */
/*
 * Coupling rows (R1-R4).  Every row r is c_r = a_r(x) - b_r(xbar) with the AL
 * term y_r (c_r + z_r) + rho_r/2 (c_r + z_r)^2 (the inner augmented Lagrangian
 * of Sec. III-A).  Per (t,g), 0-based t:
 *   ON,SU,SD  a = u_k                     b = ubar_k                 (rho_uc)
 *   PL  a = p - s_pl                      b = Pmin ubar_on_t          (rho_pq)
 *   PU  a = p + s_pu                      b = Pmax ubar_on_t
 *   QL  a = q - s_ql                      b = Qmin ubar_on_t
 *   QU  a = q + s_qu                      b = Qmax ubar_on_t
 *   RD  a = (p - phat) - s_rd             b = -RD ubar_on_t - SD ubar_sd_t
 *   RU  a = (p - phat) + s_ru             b = RU ubar_on_{t-1} + SU ubar_su_t
 *   GP  a = p                             b = pbar_t
 *   GQ  a = q                             b = qbar_t
 *   TC  a = phat_t   (t >= 1 only)        b = pbar_{t-1}
 * (phat_0 = p0 and ubar_on_{-1} = u0 are data.)  Per (t, line):
 *   0..3 flows p_ij,q_ij,p_ji,q_ji minus their bus-side copies (rho_pq)
 *   4,5  w_i, w_j minus wbar_from, wbar_to; 6,7 theta_i, theta_j minus
 *        thetabar_from, thetabar_to (rho_va).
 * The ramp-down row follows the inequality of Eq. uc_acopf_gen_ramp_down_ineq
 * (the equality form printed with the reformulation disagrees with it).
 */
enum { GR_ON, GR_SU, GR_SD, GR_PL, GR_PU, GR_QL, GR_QU, GR_RD, GR_RU, GR_GP, GR_GQ, GR_TC, NGR };
enum { NBR = 8 };
enum { NG_FIELDS = 17, NB_FIELDS = 17, NU_FIELDS = 2, NCTRL = 12 };
enum { F_P, F_Q, F_PH, F_SPL, F_SPU, F_SQL, F_SQU, F_SRD, F_SRU, F_UON, F_USU, F_USD, F_PBAR, F_QBAR,
       F_UBON, F_UBSU, F_UBSD };
enum { FB_V0 = 0, FB_MU0 = 8, FB_C = 12, FB_FB0 = 13 };
enum { FU_W, FU_TH };
enum { C_BETA, C_ZPREV, C_LIN, C_KOUT, C_PEND, C_BNEXT, C_DONE, C_RPQ, C_RVA, C_RUC, C_RCNT, C_RLOG };

typedef struct {
  int nb, nl, ng, T, ref;
  orc_params P;
  double base;
  double *Pd, *Qd, *Gs, *Bs, *Vmin, *Vmax;
  int *bf, *bt;
  double *rate2;
  double *Y; /* [nl][8] Gii,Bii,Gij,Bij,Gjj,Bjj,Gji,Bji */
  double *blo, *bhi; /* [nl][8] */
  int *gbus;
  double *Pmin, *Pmax, *Qmin, *Qmax, *qlo, *qhi, *c2p, *c1p, *c0, *csu, *csd, *RU, *RD, *SU, *SD, *p0;
  int *TU, *TD, *u0, *L0, *F0;
  int *inc_ptr, *inc_br, *inc_side, *gen_ptr, *gen_idx;
  double *G;            /* [NG_FIELDS][T][ng] */
  double *GY, *GZ, *GL; /* [NGR][T][ng] */
  double *B;            /* [NB_FIELDS][T][nl] */
  double *BY, *BZ, *BL; /* [NBR][T][nl] */
  double *U;            /* [NU_FIELDS][T][nb] */
  double ctrl[NCTRL];
  double *GA, *GB, *BA, *BB, *GBold, *BBold;
  double res[6]; /* r_p, r_d, z_norm, inf_norm, objective, z_rms */
  long newton_total, al_total, br_fail, sweeps;
} orc_inst;

#define GIX(I, f, t, g) ((size_t)((f) * (I)->T + (t)) * (size_t)(I)->ng + (size_t)(g))
#define BIX(I, f, t, l) ((size_t)((f) * (I)->T + (t)) * (size_t)(I)->nl + (size_t)(l))
#define UIX(I, f, t, i) ((size_t)((f) * (I)->T + (t)) * (size_t)(I)->nb + (size_t)(i))

static double *dup_d(const double *s, size_t n) {
  double *d = (double *)malloc(n * sizeof(double) + 8);
  memcpy(d, s, n * sizeof(double));
  return d;
}
static int *dup_i(const int32_t *s, size_t n) {
  int *d = (int *)malloc(n * sizeof(int) + 8);
  for (size_t k = 0; k < n; ++k) d[k] = s[k];
  return d;
}
static double grow_rho(const orc_inst *I, int r) { return (r <= GR_SD) ? I->P.rho_uc : I->P.rho_pq; }
static double brow_rho(const orc_inst *I, int k) { return (k < 4) ? I->P.rho_pq : I->P.rho_va; }

EXPORT void orc_default_params(orc_params *p) {
  p->rho_pq = 5e3; p->rho_va = 1e4; p->rho_uc = 1e4;
  p->eps_in = 1e-4; p->eps_out = 1e-4; p->tau = 6.0; p->theta = 0.8;
  p->beta0 = 1e3; p->lam_max = 1e12;
  p->eta = 1e-12; p->omega_rel = 1e-12; p->c_init_rel = 1e4; p->c_max_rel = 1e6;
  p->K_AL = 50; p->K_N = 50; p->L_max = 1000; p->uc_relax = 0;
  p->rho_every = 0; p->pad = 0; p->rho_mu = 10.0; p->rho_tau = 2.0;
}

EXPORT long orc_state_size(const void *h) {
  const orc_inst *I = (const orc_inst *)h;
  return (long)I->T * ((long)(NG_FIELDS + 3 * NGR) * I->ng + (long)(NB_FIELDS + 3 * NBR) * I->nl +
                       (long)NU_FIELDS * I->nb) + NCTRL;
}

static void compute_b(const orc_inst *I, double *GB, double *BB) {
  int T = I->T, ng = I->ng, nl = I->nl;
  for (int t = 0; t < T; ++t)
    for (int g = 0; g < ng; ++g) {
      double ubon = I->G[GIX(I, F_UBON, t, g)], ubsu = I->G[GIX(I, F_UBSU, t, g)];
      double ubsd = I->G[GIX(I, F_UBSD, t, g)];
      double ubon_prev = (t > 0) ? I->G[GIX(I, F_UBON, t - 1, g)] : (double)I->u0[g];
      GB[GIX(I, GR_ON, t, g)] = ubon;
      GB[GIX(I, GR_SU, t, g)] = ubsu;
      GB[GIX(I, GR_SD, t, g)] = ubsd;
      GB[GIX(I, GR_PL, t, g)] = I->Pmin[g] * ubon;
      GB[GIX(I, GR_PU, t, g)] = I->Pmax[g] * ubon;
      GB[GIX(I, GR_QL, t, g)] = I->Qmin[g] * ubon;
      GB[GIX(I, GR_QU, t, g)] = I->Qmax[g] * ubon;
      GB[GIX(I, GR_RD, t, g)] = (-I->RD[g] * ubon) - I->SD[g] * ubsd;
      GB[GIX(I, GR_RU, t, g)] = I->RU[g] * ubon_prev + I->SU[g] * ubsu;
      GB[GIX(I, GR_GP, t, g)] = I->G[GIX(I, F_PBAR, t, g)];
      GB[GIX(I, GR_GQ, t, g)] = I->G[GIX(I, F_QBAR, t, g)];
      GB[GIX(I, GR_TC, t, g)] = (t > 0) ? I->G[GIX(I, F_PBAR, t - 1, g)] : 0.0;
    }
  for (int t = 0; t < T; ++t)
    for (int l = 0; l < nl; ++l) {
      for (int k = 0; k < 4; ++k) BB[BIX(I, k, t, l)] = I->B[BIX(I, FB_FB0 + k, t, l)];
      BB[BIX(I, 4, t, l)] = I->U[UIX(I, FU_W, t, I->bf[l])];
      BB[BIX(I, 5, t, l)] = I->U[UIX(I, FU_W, t, I->bt[l])];
      BB[BIX(I, 6, t, l)] = I->U[UIX(I, FU_TH, t, I->bf[l])];
      BB[BIX(I, 7, t, l)] = I->U[UIX(I, FU_TH, t, I->bt[l])];
    }
}

static void compute_a(const orc_inst *I, double *GA, double *BA) {
  int T = I->T, ng = I->ng, nl = I->nl;
  for (int t = 0; t < T; ++t)
    for (int g = 0; g < ng; ++g) {
      double p = I->G[GIX(I, F_P, t, g)], q = I->G[GIX(I, F_Q, t, g)], ph = I->G[GIX(I, F_PH, t, g)];
      double d = p - ph;
      GA[GIX(I, GR_ON, t, g)] = I->G[GIX(I, F_UON, t, g)];
      GA[GIX(I, GR_SU, t, g)] = I->G[GIX(I, F_USU, t, g)];
      GA[GIX(I, GR_SD, t, g)] = I->G[GIX(I, F_USD, t, g)];
      GA[GIX(I, GR_PL, t, g)] = p - I->G[GIX(I, F_SPL, t, g)];
      GA[GIX(I, GR_PU, t, g)] = p + I->G[GIX(I, F_SPU, t, g)];
      GA[GIX(I, GR_QL, t, g)] = q - I->G[GIX(I, F_SQL, t, g)];
      GA[GIX(I, GR_QU, t, g)] = q + I->G[GIX(I, F_SQU, t, g)];
      GA[GIX(I, GR_RD, t, g)] = d - I->G[GIX(I, F_SRD, t, g)];
      GA[GIX(I, GR_RU, t, g)] = d + I->G[GIX(I, F_SRU, t, g)];
      GA[GIX(I, GR_GP, t, g)] = p;
      GA[GIX(I, GR_GQ, t, g)] = q;
      GA[GIX(I, GR_TC, t, g)] = (t > 0) ? ph : 0.0;
    }
  for (int t = 0; t < T; ++t)
    for (int l = 0; l < nl; ++l) {
      const double *Yl = I->Y + (size_t)l * 8;
      double v[8], a[4];
      for (int k = 0; k < 8; ++k) v[k] = I->B[BIX(I, FB_V0 + k, t, l)];
      a[0] = Yl[0] * v[0] + Yl[2] * v[2] + Yl[3] * v[3];
      a[1] = -Yl[1] * v[0] - Yl[3] * v[2] + Yl[2] * v[3];
      a[2] = Yl[4] * v[1] + Yl[6] * v[2] - Yl[7] * v[3];
      a[3] = -Yl[5] * v[1] - Yl[7] * v[2] - Yl[6] * v[3];
      for (int k = 0; k < 4; ++k) BA[BIX(I, k, t, l)] = a[k];
      BA[BIX(I, 4, t, l)] = v[0];
      BA[BIX(I, 5, t, l)] = v[1];
      BA[BIX(I, 6, t, l)] = v[4];
      BA[BIX(I, 7, t, l)] = v[5];
    }
}

EXPORT void orc_destroy(void *h);

/* Returns NULL on invalid data (disconnected grid, r = x = 0, bad bounds or indices). */
EXPORT void *orc_create(const orc_grid *g, const orc_params *prm) {
  int nb = g->n_bus, nl = g->n_branch, ng = g->n_gen, T = g->T;
  if (nb < 1 || nl < 0 || ng < 0 || T < 1 || g->ref_bus < 0 || g->ref_bus >= nb) return NULL;
  for (int l = 0; l < nl; ++l) {
    if (g->br_from[l] < 0 || g->br_from[l] >= nb || g->br_to[l] < 0 || g->br_to[l] >= nb) return NULL;
    if (g->br_from[l] == g->br_to[l]) return NULL;
    if (!(g->br_r[l] * g->br_r[l] + g->br_x[l] * g->br_x[l] > 0.0)) return NULL;
    if (!(g->br_rate[l] > 0.0)) return NULL;
  }
  for (int i = 0; i < nb; ++i)
    if (!(g->Vmin[i] > 0.0 && g->Vmin[i] <= g->Vmax[i])) return NULL;
  for (int k = 0; k < ng; ++k) {
    if (g->gen_bus[k] < 0 || g->gen_bus[k] >= nb) return NULL;
    if (!(g->Pmin[k] <= g->Pmax[k] && g->Pmax[k] > 0.0 && g->Qmin[k] <= g->Qmax[k])) return NULL;
    if (g->u0[k] != 0 && g->u0[k] != 1) return NULL;
  }
  for (size_t k = 0; k < (size_t)T * nb; ++k)
    if (!isfinite(g->Pd[k]) || !isfinite(g->Qd[k])) return NULL;
  /* connectivity */
  {
    int *par = (int *)malloc(sizeof(int) * nb);
    for (int i = 0; i < nb; ++i) par[i] = i;
    for (int l = 0; l < nl; ++l) {
      int a = g->br_from[l], b = g->br_to[l];
      while (par[a] != a) a = par[a];
      while (par[b] != b) b = par[b];
      if (a != b) par[a] = b;
    }
    int roots = 0;
    for (int i = 0; i < nb; ++i)
      if (par[i] == i) ++roots;
    free(par);
    if (roots != 1) return NULL;
  }
  orc_inst *I = (orc_inst *)calloc(1, sizeof(orc_inst));
  I->nb = nb; I->nl = nl; I->ng = ng; I->T = T; I->ref = g->ref_bus;
  if (prm) I->P = *prm; else orc_default_params(&I->P);
  I->base = g->base_mva;
  I->Pd = dup_d(g->Pd, (size_t)T * nb);
  I->Qd = dup_d(g->Qd, (size_t)T * nb);
  I->Gs = dup_d(g->Gs, nb); I->Bs = dup_d(g->Bs, nb);
  I->Vmin = dup_d(g->Vmin, nb); I->Vmax = dup_d(g->Vmax, nb);
  I->bf = dup_i(g->br_from, nl); I->bt = dup_i(g->br_to, nl);
  I->rate2 = (double *)malloc(sizeof(double) * (nl + 1));
  I->Y = (double *)malloc(sizeof(double) * 8 * (nl + 1));
  I->blo = (double *)malloc(sizeof(double) * 8 * (nl + 1));
  I->bhi = (double *)malloc(sizeof(double) * 8 * (nl + 1));
  const double twopi = 6.283185307179586476925286766559;
  for (int l = 0; l < nl; ++l) {
    /* series admittance y = 1/(r + jx); Y_ii = y + j b/2, Y_ij = -y (no taps) */
    double r = g->br_r[l], x = g->br_x[l], z2 = r * r + x * x;
    double gs = r / z2, bs = -x / z2, bc = g->br_b[l];
    double *Yl = I->Y + (size_t)l * 8;
    Yl[0] = gs; Yl[1] = bs + 0.5 * bc; Yl[2] = -gs; Yl[3] = -bs;
    Yl[4] = gs; Yl[5] = bs + 0.5 * bc; Yl[6] = -gs; Yl[7] = -bs;
    I->rate2[l] = g->br_rate[l] * g->br_rate[l];
    int i = g->br_from[l], j = g->br_to[l];
    double vv = g->Vmax[i] * g->Vmax[j];
    double lo[8] = {g->Vmin[i] * g->Vmin[i], g->Vmin[j] * g->Vmin[j], -vv, -vv, -twopi, -twopi, 0.0, 0.0};
    double hi[8] = {g->Vmax[i] * g->Vmax[i], g->Vmax[j] * g->Vmax[j], vv, vv, twopi, twopi, I->rate2[l], I->rate2[l]};
    for (int k = 0; k < 8; ++k) {
      I->blo[(size_t)l * 8 + k] = lo[k];
      I->bhi[(size_t)l * 8 + k] = hi[k];
    }
  }
  I->gbus = dup_i(g->gen_bus, ng);
  I->Pmin = dup_d(g->Pmin, ng); I->Pmax = dup_d(g->Pmax, ng);
  I->Qmin = dup_d(g->Qmin, ng); I->Qmax = dup_d(g->Qmax, ng);
  I->qlo = (double *)malloc(sizeof(double) * (ng + 1));
  I->qhi = (double *)malloc(sizeof(double) * (ng + 1));
  I->c2p = (double *)malloc(sizeof(double) * (ng + 1));
  I->c1p = (double *)malloc(sizeof(double) * (ng + 1));
  for (int k = 0; k < ng; ++k) {
    I->qlo[k] = (g->Qmin[k] < 0.0) ? g->Qmin[k] : 0.0;
    I->qhi[k] = g->Qmax[k];
    I->c2p[k] = g->c2[k] * g->base_mva * g->base_mva; /* $/h per p.u.^2 */
    I->c1p[k] = g->c1[k] * g->base_mva;
  }
  I->c0 = dup_d(g->c0, ng); I->csu = dup_d(g->c_su, ng); I->csd = dup_d(g->c_sd, ng);
  I->RU = dup_d(g->RU, ng); I->RD = dup_d(g->RD, ng); I->SU = dup_d(g->SU, ng); I->SD = dup_d(g->SD, ng);
  I->p0 = dup_d(g->p0, ng);
  I->TU = dup_i(g->TU, ng); I->TD = dup_i(g->TD, ng); I->u0 = dup_i(g->u0, ng);
  I->L0 = dup_i(g->L0, ng); I->F0 = dup_i(g->F0, ng);
  /* adjacency */
  I->inc_ptr = (int *)calloc(nb + 1, sizeof(int));
  I->inc_br = (int *)malloc(sizeof(int) * (2 * nl + 1));
  I->inc_side = (int *)malloc(sizeof(int) * (2 * nl + 1));
  for (int l = 0; l < nl; ++l) {
    I->inc_ptr[I->bf[l] + 1]++;
    I->inc_ptr[I->bt[l] + 1]++;
  }
  for (int i = 0; i < nb; ++i) I->inc_ptr[i + 1] += I->inc_ptr[i];
  {
    int *fill = (int *)calloc(nb, sizeof(int));
    for (int l = 0; l < nl; ++l) {
      int i = I->bf[l], p = I->inc_ptr[i] + fill[i]++;
      I->inc_br[p] = l; I->inc_side[p] = 0;
      i = I->bt[l]; p = I->inc_ptr[i] + fill[i]++;
      I->inc_br[p] = l; I->inc_side[p] = 1;
    }
    free(fill);
  }
  I->gen_ptr = (int *)calloc(nb + 1, sizeof(int));
  I->gen_idx = (int *)malloc(sizeof(int) * (ng + 1));
  for (int k = 0; k < ng; ++k) I->gen_ptr[I->gbus[k] + 1]++;
  for (int i = 0; i < nb; ++i) I->gen_ptr[i + 1] += I->gen_ptr[i];
  {
    int *fill = (int *)calloc(nb, sizeof(int));
    for (int k = 0; k < ng; ++k) {
      int i = I->gbus[k];
      I->gen_idx[I->gen_ptr[i] + fill[i]++] = k;
    }
    free(fill);
  }
  /* state */
  size_t GN = (size_t)T * ng, BN = (size_t)T * nl, UN = (size_t)T * nb;
  I->G = (double *)calloc(NG_FIELDS * GN + 1, sizeof(double));
  I->GY = (double *)calloc(NGR * GN + 1, sizeof(double));
  I->GZ = (double *)calloc(NGR * GN + 1, sizeof(double));
  I->GL = (double *)calloc(NGR * GN + 1, sizeof(double));
  I->GA = (double *)calloc(NGR * GN + 1, sizeof(double));
  I->GB = (double *)calloc(NGR * GN + 1, sizeof(double));
  I->GBold = (double *)calloc(NGR * GN + 1, sizeof(double));
  I->B = (double *)calloc(NB_FIELDS * BN + 1, sizeof(double));
  I->BY = (double *)calloc(NBR * BN + 1, sizeof(double));
  I->BZ = (double *)calloc(NBR * BN + 1, sizeof(double));
  I->BL = (double *)calloc(NBR * BN + 1, sizeof(double));
  I->BA = (double *)calloc(NBR * BN + 1, sizeof(double));
  I->BB = (double *)calloc(NBR * BN + 1, sizeof(double));
  I->BBold = (double *)calloc(NBR * BN + 1, sizeof(double));
  I->U = (double *)calloc(NU_FIELDS * UN + 1, sizeof(double));
  /* cold start (Sec. IV-A): p, q, |V| at the middle of their bounds, angles 0,
     flows from the initial voltages; UC all on (reading R13).
     Parity pinned: rebuilt from the text with complex phasors of the pi
     model, per-bus voltage bands, charging and a positive reactive floor
     (tests). */
  double cpen0 = I->P.c_init_rel * ((I->P.rho_pq > I->P.rho_va) ? I->P.rho_pq : I->P.rho_va);
  for (int t = 0; t < T; ++t)
    for (int k = 0; k < ng; ++k) {
      double p = 0.5 * I->Pmax[k], q = 0.5 * (I->qlo[k] + I->qhi[k]);
      I->G[GIX(I, F_P, t, k)] = p;
      I->G[GIX(I, F_Q, t, k)] = q;
      I->G[GIX(I, F_PH, t, k)] = (t > 0) ? 0.5 * I->Pmax[k] : I->p0[k];
      I->G[GIX(I, F_UON, t, k)] = 1.0;
      I->G[GIX(I, F_PBAR, t, k)] = p;
      I->G[GIX(I, F_QBAR, t, k)] = q;
      I->G[GIX(I, F_UBON, t, k)] = 1.0;
    }
  for (int t = 0; t < T; ++t) {
    for (int i = 0; i < nb; ++i) {
      double V = 0.5 * (I->Vmin[i] + I->Vmax[i]);
      I->U[UIX(I, FU_W, t, i)] = V * V;
      I->U[UIX(I, FU_TH, t, i)] = 0.0;
    }
    for (int l = 0; l < nl; ++l) {
      int i = I->bf[l], j = I->bt[l];
      double Vi = 0.5 * (I->Vmin[i] + I->Vmax[i]), Vj = 0.5 * (I->Vmin[j] + I->Vmax[j]);
      double v[8] = {Vi * Vi, Vj * Vj, Vi * Vj, 0.0, 0.0, 0.0, 0.0, 0.0};
      const double *Yl = I->Y + (size_t)l * 8;
      double a[4];
      a[0] = Yl[0] * v[0] + Yl[2] * v[2] + Yl[3] * v[3];
      a[1] = -Yl[1] * v[0] - Yl[3] * v[2] + Yl[2] * v[3];
      a[2] = Yl[4] * v[1] + Yl[6] * v[2] - Yl[7] * v[3];
      a[3] = -Yl[5] * v[1] - Yl[7] * v[2] - Yl[6] * v[3];
      v[6] = clampd(I->rate2[l] - a[0] * a[0] - a[1] * a[1], 0.0, I->rate2[l]);
      v[7] = clampd(I->rate2[l] - a[2] * a[2] - a[3] * a[3], 0.0, I->rate2[l]);
      for (int k = 0; k < 8; ++k) I->B[BIX(I, FB_V0 + k, t, l)] = v[k];
      I->B[BIX(I, FB_C, t, l)] = cpen0;
      for (int k = 0; k < 4; ++k) I->B[BIX(I, FB_FB0 + k, t, l)] = a[k];
    }
  }
  I->ctrl[C_BETA] = I->P.beta0;
  I->ctrl[C_ZPREV] = -1.0;
  I->ctrl[C_BNEXT] = I->P.beta0;
  I->ctrl[C_RPQ] = I->P.rho_pq;
  I->ctrl[C_RVA] = I->P.rho_va;
  I->ctrl[C_RUC] = I->P.rho_uc;
  return I;
}

EXPORT void orc_destroy(void *h) {
  orc_inst *I = (orc_inst *)h;
  if (!I) return;
  void *ptrs[] = {I->Pd, I->Qd, I->Gs, I->Bs, I->Vmin, I->Vmax, I->bf, I->bt, I->rate2, I->Y, I->blo,
                  I->bhi, I->gbus, I->Pmin, I->Pmax, I->Qmin, I->Qmax, I->qlo, I->qhi, I->c2p, I->c1p,
                  I->c0, I->csu, I->csd, I->RU, I->RD, I->SU, I->SD, I->p0, I->TU, I->TD, I->u0, I->L0,
                  I->F0, I->inc_ptr, I->inc_br, I->inc_side, I->gen_ptr, I->gen_idx, I->G, I->GY, I->GZ,
                  I->GL, I->GA, I->GB, I->GBold, I->B, I->BY, I->BZ, I->BL, I->BA, I->BB, I->BBold, I->U};
  for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
  free(I);
}

/* Canonical state order: G fields, GY, GZ, GL, B fields, BY, BZ, BL, U, ctrl. */
EXPORT void orc_state_get(const void *h, double *buf) {
  const orc_inst *I = (const orc_inst *)h;
  size_t GN = (size_t)I->T * I->ng, BN = (size_t)I->T * I->nl, UN = (size_t)I->T * I->nb, o = 0;
  memcpy(buf + o, I->G, NG_FIELDS * GN * 8); o += NG_FIELDS * GN;
  memcpy(buf + o, I->GY, NGR * GN * 8); o += NGR * GN;
  memcpy(buf + o, I->GZ, NGR * GN * 8); o += NGR * GN;
  memcpy(buf + o, I->GL, NGR * GN * 8); o += NGR * GN;
  memcpy(buf + o, I->B, NB_FIELDS * BN * 8); o += NB_FIELDS * BN;
  memcpy(buf + o, I->BY, NBR * BN * 8); o += NBR * BN;
  memcpy(buf + o, I->BZ, NBR * BN * 8); o += NBR * BN;
  memcpy(buf + o, I->BL, NBR * BN * 8); o += NBR * BN;
  memcpy(buf + o, I->U, NU_FIELDS * UN * 8); o += NU_FIELDS * UN;
  memcpy(buf + o, I->ctrl, NCTRL * 8);
}

EXPORT void orc_state_set(void *h, const double *buf) {
  orc_inst *I = (orc_inst *)h;
  size_t GN = (size_t)I->T * I->ng, BN = (size_t)I->T * I->nl, UN = (size_t)I->T * I->nb, o = 0;
  memcpy(I->G, buf + o, NG_FIELDS * GN * 8); o += NG_FIELDS * GN;
  memcpy(I->GY, buf + o, NGR * GN * 8); o += NGR * GN;
  memcpy(I->GZ, buf + o, NGR * GN * 8); o += NGR * GN;
  memcpy(I->GL, buf + o, NGR * GN * 8); o += NGR * GN;
  memcpy(I->B, buf + o, NB_FIELDS * BN * 8); o += NB_FIELDS * BN;
  memcpy(I->BY, buf + o, NBR * BN * 8); o += NBR * BN;
  memcpy(I->BZ, buf + o, NBR * BN * 8); o += NBR * BN;
  memcpy(I->BL, buf + o, NBR * BN * 8); o += NBR * BN;
  memcpy(I->U, buf + o, NU_FIELDS * UN * 8); o += NU_FIELDS * UN;
  memcpy(I->ctrl, buf + o, NCTRL * 8);
  /* the current penalties travel with the state (adaptive penalty) */
  I->P.rho_pq = I->ctrl[C_RPQ];
  I->P.rho_va = I->ctrl[C_RVA];
  I->P.rho_uc = I->ctrl[C_RUC];
}

/* Kahan-compensated accumulator */
typedef struct { double s, c; } ksum_t;
static void kadd(ksum_t *k, double x) {
  double y = x - k->c, t = k->s + y;
  k->c = (t - k->s) - y;
  k->s = t;
}

/* x-step targets: t_r = b_r - z_r - y_r/rho_r, evaluated as (b - z) - y/rho */
static double tgt_of(double b, double z, double y, double rho) { return (b - z) - y / rho; }
/* x-bar-step targets: m_r = a_r + z_r + y_r/rho_r, evaluated as (a + z) + y/rho */
static double mtg_of(double a, double z, double y, double rho) { return (a + z) + y / rho; }

/*
 * One inner sweep (Eq. step:uc .. step:y, Algorithm 1 inner loop body), then
 * the residuals and the inner/outer control (readings R11, R12).  A pending
 * outer update (Eq. step:outer) decided at the end of the previous sweep is
 * applied before this sweep's z-step; the x-step does not read lambda or
 * beta, so this is the order of Algorithm 1.
 */
EXPORT void orc_sweep(void *h) {
  orc_inst *I = (orc_inst *)h;
  /* Algorithm 1 ends at convergence: an instance whose last sweep met both
     stopping tests takes no further sweep, so its iterate, residuals and
     counters stay those of that sweep */
  if (I->ctrl[C_DONE] != 0.0) return;
  int T = I->T, ng = I->ng, nl = I->nl, nb = I->nb;
  const orc_params *P = &I->P;
  compute_b(I, I->GB, I->BB);
  /* ---- x^UC: Algorithm 2 per generator (Eq. step:uc) */
  {
    double *ton = (double *)malloc(sizeof(double) * T), *tsu = (double *)malloc(sizeof(double) * T);
    double *tsd = (double *)malloc(sizeof(double) * T), *L = (double *)malloc(sizeof(double) * 4 * T);
    int32_t *u = (int32_t *)malloc(sizeof(int32_t) * T);
    for (int g = 0; g < ng; ++g) {
      for (int t = 0; t < T; ++t) {
        ton[t] = tgt_of(I->GB[GIX(I, GR_ON, t, g)], I->GZ[GIX(I, GR_ON, t, g)], I->GY[GIX(I, GR_ON, t, g)], P->rho_uc);
        tsu[t] = tgt_of(I->GB[GIX(I, GR_SU, t, g)], I->GZ[GIX(I, GR_SU, t, g)], I->GY[GIX(I, GR_SU, t, g)], P->rho_uc);
        tsd[t] = tgt_of(I->GB[GIX(I, GR_SD, t, g)], I->GZ[GIX(I, GR_SD, t, g)], I->GY[GIX(I, GR_SD, t, g)], P->rho_uc);
      }
      if (P->uc_relax) {
        /* box relaxation of Eq. set:UC (integrality, the start-up/shut-down
           equation and the minimum times dropped): each row minimises
           c u + rho/2 (u - tau)^2 over [0, 1] */
        for (int t = 0; t < T; ++t) {
          const double on = clampd(ton[t] - I->c0[g] / P->rho_uc, 0.0, 1.0);
          const double su = clampd(tsu[t] - I->csu[g] / P->rho_uc, 0.0, 1.0);
          const double sd = clampd(tsd[t] - I->csd[g] / P->rho_uc, 0.0, 1.0);
          I->G[GIX(I, F_UON, t, g)] = on;
          I->G[GIX(I, F_USU, t, g)] = su;
          I->G[GIX(I, F_USD, t, g)] = sd;
        }
        continue;
      }
      orc_uc_stagecost(T, I->c0[g], I->csu[g], I->csd[g], P->rho_uc, ton, tsu, tsd, L);
      int K0 = I->u0[g] ? I->L0[g] : I->F0[g];
      orc_dp(T, I->TU[g], I->TD[g], I->u0[g], K0, L, u);
      int prev = I->u0[g];
      for (int t = 0; t < T; ++t) {
        I->G[GIX(I, F_UON, t, g)] = (double)u[t];
        I->G[GIX(I, F_USU, t, g)] = (u[t] > prev) ? 1.0 : 0.0;
        I->G[GIX(I, F_USD, t, g)] = (prev > u[t]) ? 1.0 : 0.0;
        prev = u[t];
      }
    }
    free(ton); free(tsu); free(tsd); free(L); free(u);
  }
  /* ---- x^OPF generators (Eq. step:opf, R5) */
#pragma omp parallel for collapse(2) schedule(static)
  for (int t = 0; t < T; ++t)
    for (int g = 0; g < ng; ++g) {
      double prm[7] = {I->c2p[g], I->c1p[g], P->rho_pq, I->Pmax[g], I->qlo[g], I->qhi[g], I->p0[g]};
      double tg[9];
      const int rows[9] = {GR_PL, GR_PU, GR_QL, GR_QU, GR_RD, GR_RU, GR_GP, GR_GQ, GR_TC};
      for (int k = 0; k < 9; ++k) {
        int r = rows[k];
        tg[k] = tgt_of(I->GB[GIX(I, r, t, g)], I->GZ[GIX(I, r, t, g)], I->GY[GIX(I, r, t, g)], P->rho_pq);
      }
      if (t == 0) tg[8] = 0.0;
      double out[9];
      orc_gen_solve(prm, t > 0, tg, out);
      const int flds[9] = {F_P, F_Q, F_PH, F_SPL, F_SPU, F_SQL, F_SQU, F_SRD, F_SRU};
      for (int k = 0; k < 9; ++k) I->G[GIX(I, flds[k], t, g)] = out[k];
    }
  /* ---- x^OPF lines (Eq. step:opf, R6) */
  {
    double rmax = (P->rho_pq > P->rho_va) ? P->rho_pq : P->rho_va;
    double omega = P->omega_rel * rmax, cmax = P->c_max_rel * rmax;
    long nw = 0, na = 0, nf = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 16) reduction(+ : nw, na, nf)
    for (int t = 0; t < T; ++t)
      for (int l = 0; l < nl; ++l) {
        double cst[25], tg[8], v[8], mu[4], c, a[8];
        int32_t info[3];
        for (int k = 0; k < 8; ++k) cst[k] = I->Y[(size_t)l * 8 + k];
        cst[8] = I->rate2[l];
        for (int k = 0; k < 8; ++k) {
          cst[9 + k] = I->blo[(size_t)l * 8 + k];
          cst[17 + k] = I->bhi[(size_t)l * 8 + k];
        }
        for (int k = 0; k < 8; ++k)
          tg[k] = tgt_of(I->BB[BIX(I, k, t, l)], I->BZ[BIX(I, k, t, l)], I->BY[BIX(I, k, t, l)], brow_rho(I, k));
        for (int k = 0; k < 8; ++k) v[k] = I->B[BIX(I, FB_V0 + k, t, l)];
        for (int k = 0; k < 4; ++k) mu[k] = I->B[BIX(I, FB_MU0 + k, t, l)];
        c = I->B[BIX(I, FB_C, t, l)];
        orc_branch_solve(cst, tg, P->rho_pq, P->rho_va, P->eta, omega, cmax, P->K_AL, P->K_N, v, mu, &c, a, info);
        for (int k = 0; k < 8; ++k) I->B[BIX(I, FB_V0 + k, t, l)] = v[k];
        for (int k = 0; k < 4; ++k) I->B[BIX(I, FB_MU0 + k, t, l)] = mu[k];
        I->B[BIX(I, FB_C, t, l)] = c;
        nw += info[0];
        na += info[1];
        if (info[2] != 0) nf++;
      }
    I->newton_total += nw;
    I->al_total += na;
    I->br_fail += nf;
  }
  compute_a(I, I->GA, I->BA);
  /* ---- pending outer update (Eq. step:outer), decided when the inner level
     terminated in the previous sweep: lambda <- clip(lambda + beta z), then
     beta <- beta_next.  Parity pinned: lambda and beta followed by hand over a
     run, both sides of the strict beta comparison (tests). */
  if (I->ctrl[C_PEND] != 0.0) {
    double beta = I->ctrl[C_BETA], lm = P->lam_max;
    for (size_t k = 0; k < (size_t)NGR * T * ng; ++k) I->GL[k] = clampd(I->GL[k] + beta * I->GZ[k], -lm, lm);
    for (size_t k = 0; k < (size_t)NBR * T * nl; ++k) I->BL[k] = clampd(I->BL[k] + beta * I->BZ[k], -lm, lm);
    I->ctrl[C_BETA] = I->ctrl[C_BNEXT];
    I->ctrl[C_PEND] = 0.0;
  }
  memcpy(I->GBold, I->GB, sizeof(double) * NGR * (size_t)T * ng);
  memcpy(I->BBold, I->BB, sizeof(double) * NBR * (size_t)T * nl);
  /* ---- x-bar^OPF: bus subproblems (Eq. step:opf_bar, R8) */
  {
    int maxv = 2 * ng + 2 * 2 * nl + 4;
    double *W = (double *)malloc(sizeof(double) * maxv), *m = (double *)malloc(sizeof(double) * maxv);
    double *aP = (double *)malloc(sizeof(double) * maxv), *aQ = (double *)malloc(sizeof(double) * maxv);
    double *vv = (double *)malloc(sizeof(double) * maxv);
    for (int t = 0; t < T; ++t)
      for (int i = 0; i < nb; ++i) {
        int n = 0;
        for (int q = I->gen_ptr[i]; q < I->gen_ptr[i + 1]; ++q) {
          int g = I->gen_idx[q];
          double mgp = mtg_of(I->GA[GIX(I, GR_GP, t, g)], I->GZ[GIX(I, GR_GP, t, g)], I->GY[GIX(I, GR_GP, t, g)], P->rho_pq);
          double Wp = P->rho_pq, num = P->rho_pq * mgp;
          if (t < T - 1) {
            double mtc = mtg_of(I->GA[GIX(I, GR_TC, t + 1, g)], I->GZ[GIX(I, GR_TC, t + 1, g)],
                                I->GY[GIX(I, GR_TC, t + 1, g)], P->rho_pq);
            Wp += P->rho_pq;
            num += P->rho_pq * mtc;
          }
          W[n] = Wp; m[n] = num / Wp; aP[n] = 1.0; aQ[n] = 0.0; ++n;
          W[n] = P->rho_pq;
          m[n] = mtg_of(I->GA[GIX(I, GR_GQ, t, g)], I->GZ[GIX(I, GR_GQ, t, g)], I->GY[GIX(I, GR_GQ, t, g)], P->rho_pq);
          aP[n] = 0.0; aQ[n] = 1.0; ++n;
        }
        int deg = I->inc_ptr[i + 1] - I->inc_ptr[i];
        double mw = 0.0, mth = 0.0;
        for (int q = I->inc_ptr[i]; q < I->inc_ptr[i + 1]; ++q) {
          int l = I->inc_br[q], sd = I->inc_side[q];
          int rp = sd ? 2 : 0, rq = rp + 1, rw = sd ? 5 : 4, rt = sd ? 7 : 6;
          W[n] = P->rho_pq;
          m[n] = mtg_of(I->BA[BIX(I, rp, t, l)], I->BZ[BIX(I, rp, t, l)], I->BY[BIX(I, rp, t, l)], P->rho_pq);
          aP[n] = -1.0; aQ[n] = 0.0; ++n;
          W[n] = P->rho_pq;
          m[n] = mtg_of(I->BA[BIX(I, rq, t, l)], I->BZ[BIX(I, rq, t, l)], I->BY[BIX(I, rq, t, l)], P->rho_pq);
          aP[n] = 0.0; aQ[n] = -1.0; ++n;
          mw += mtg_of(I->BA[BIX(I, rw, t, l)], I->BZ[BIX(I, rw, t, l)], I->BY[BIX(I, rw, t, l)], P->rho_va);
          mth += mtg_of(I->BA[BIX(I, rt, t, l)], I->BZ[BIX(I, rt, t, l)], I->BY[BIX(I, rt, t, l)], P->rho_va);
        }
        W[n] = P->rho_va * deg; m[n] = mw / deg; aP[n] = -I->Gs[i]; aQ[n] = I->Bs[i]; ++n;
        orc_bus_solve(n, W, m, aP, aQ, I->Pd[(size_t)t * nb + i], I->Qd[(size_t)t * nb + i], vv);
        n = 0;
        for (int q = I->gen_ptr[i]; q < I->gen_ptr[i + 1]; ++q) {
          int g = I->gen_idx[q];
          I->G[GIX(I, F_PBAR, t, g)] = vv[n++];
          I->G[GIX(I, F_QBAR, t, g)] = vv[n++];
        }
        for (int q = I->inc_ptr[i]; q < I->inc_ptr[i + 1]; ++q) {
          int l = I->inc_br[q], sd = I->inc_side[q];
          int rp = sd ? 2 : 0;
          I->B[BIX(I, FB_FB0 + rp, t, l)] = vv[n++];
          I->B[BIX(I, FB_FB0 + rp + 1, t, l)] = vv[n++];
        }
        I->U[UIX(I, FU_W, t, i)] = vv[n++];
        I->U[UIX(I, FU_TH, t, i)] = (i == I->ref) ? 0.0 : mth / deg;
      }
    free(W); free(m); free(aP); free(aQ); free(vv);
  }
  /* ---- x-bar^UC (Eq. step:uc_bar, R7) */
  for (int g = 0; g < ng; ++g) {
#define MG(r, t) mtg_of(I->GA[GIX(I, r, t, g)], I->GZ[GIX(I, r, t, g)], I->GY[GIX(I, r, t, g)], grow_rho(I, r))
    for (int tau = 0; tau < T; ++tau) {
      int n = (tau < T - 1) ? 3 : 2;
      double H[9] = {0}, gv[3] = {0};
      double e[3];
#define ADDROW(w, mm, e0, e1, e2)                                      \
  do {                                                                 \
    e[0] = (e0); e[1] = (e1); e[2] = (e2);                             \
    for (int a_ = 0; a_ < n; ++a_) {                                   \
      gv[a_] += (w) * (mm) * e[a_];                                    \
      for (int b_ = 0; b_ < n; ++b_) H[a_ * n + b_] += (w) * e[a_] * e[b_]; \
    }                                                                  \
  } while (0)
      ADDROW(P->rho_uc, MG(GR_ON, tau), 1.0, 0.0, 0.0);
      ADDROW(P->rho_uc, MG(GR_SD, tau), 0.0, 1.0, 0.0);
      ADDROW(P->rho_pq, MG(GR_PL, tau), I->Pmin[g], 0.0, 0.0);
      ADDROW(P->rho_pq, MG(GR_PU, tau), I->Pmax[g], 0.0, 0.0);
      ADDROW(P->rho_pq, MG(GR_QL, tau), I->Qmin[g], 0.0, 0.0);
      ADDROW(P->rho_pq, MG(GR_QU, tau), I->Qmax[g], 0.0, 0.0);
      ADDROW(P->rho_pq, MG(GR_RD, tau), -I->RD[g], -I->SD[g], 0.0);
      if (tau < T - 1) {
        ADDROW(P->rho_uc, MG(GR_SU, tau + 1), 0.0, 0.0, 1.0);
        ADDROW(P->rho_pq, MG(GR_RU, tau + 1), I->RU[g], 0.0, I->SU[g]);
      }
#undef ADDROW
      double x[3];
      orc_boxqp(n, H, gv, x);
      I->G[GIX(I, F_UBON, tau, g)] = x[0];
      I->G[GIX(I, F_UBSD, tau, g)] = x[1];
      if (tau < T - 1) I->G[GIX(I, F_UBSU, tau + 1, g)] = x[2];
    }
    {
      double Hs = P->rho_uc + P->rho_pq * I->SU[g] * I->SU[g];
      double gs = P->rho_uc * MG(GR_SU, 0) + P->rho_pq * I->SU[g] * (MG(GR_RU, 0) - I->RU[g] * (double)I->u0[g]);
      I->G[GIX(I, F_UBSU, 0, g)] = clampd(gs / Hs, 0.0, 1.0);
    }
#undef MG
  }
  compute_b(I, I->GB, I->BB);
  /* ---- z (Eq. step:z, R9), y (Eq. step:y, R10), residuals (R11) */
  ksum_t sp = {0, 0}, sd = {0, 0}, sz = {0, 0}, so = {0, 0};
  double inf = 0.0;
  double beta = I->ctrl[C_BETA];
  long mrows = 0;
  for (int r = 0; r < NGR; ++r)
    for (int t = 0; t < T; ++t)
      for (int g = 0; g < ng; ++g) {
        if (r == GR_TC && t == 0) continue;
        size_t k = GIX(I, r, t, g);
        double rho = grow_rho(I, r);
        double c = I->GA[k] - I->GB[k];
        double z = -(I->GL[k] + I->GY[k] + rho * c) / (beta + rho);
        I->GZ[k] = z;
        I->GY[k] = I->GY[k] + rho * (c + z);
        kadd(&sp, (c + z) * (c + z));
        kadd(&sd, (I->GB[k] - I->GBold[k]) * (I->GB[k] - I->GBold[k]));
        kadd(&sz, z * z);
        if (fabs(c) > inf) inf = fabs(c);
        ++mrows;
      }
  for (int r = 0; r < NBR; ++r)
    for (int t = 0; t < T; ++t)
      for (int l = 0; l < nl; ++l) {
        size_t k = BIX(I, r, t, l);
        double rho = brow_rho(I, r);
        double c = I->BA[k] - I->BB[k];
        double z = -(I->BL[k] + I->BY[k] + rho * c) / (beta + rho);
        I->BZ[k] = z;
        I->BY[k] = I->BY[k] + rho * (c + z);
        kadd(&sp, (c + z) * (c + z));
        kadd(&sd, (I->BB[k] - I->BBold[k]) * (I->BB[k] - I->BBold[k]));
        kadd(&sz, z * z);
        if (fabs(c) > inf) inf = fabs(c);
        ++mrows;
      }
  for (int t = 0; t < T; ++t)
    for (int g = 0; g < ng; ++g) {
      double p = I->G[GIX(I, F_P, t, g)];
      kadd(&so, I->c2p[g] * p * p + I->c1p[g] * p + I->c0[g] * I->G[GIX(I, F_UON, t, g)] +
                    I->csu[g] * I->G[GIX(I, F_USU, t, g)] + I->csd[g] * I->G[GIX(I, F_USD, t, g)]);
    }
  double mr = (double)mrows;
  I->res[0] = sqrt(sp.s / mr);
  I->res[1] = sqrt(sd.s / mr);
  I->res[2] = sqrt(sz.s);
  I->res[3] = inf;
  I->res[4] = so.s;
  I->res[5] = sqrt(sz.s / mr);
  I->sweeps++;
  /* ---- inner/outer control (Algorithm 1; readings R11, R12) */
  I->ctrl[C_LIN] += 1.0;
  int inner_ok = (I->res[0] <= P->eps_in) && (I->res[1] <= P->eps_in);
  if (inner_ok || I->ctrl[C_LIN] >= (double)P->L_max) {
    if (inner_ok && I->res[5] <= P->eps_out) {
      I->ctrl[C_DONE] = 1.0;
    } else {
      double zn = I->res[2];
      double bnext = (I->ctrl[C_ZPREV] >= 0.0 && zn > P->theta * I->ctrl[C_ZPREV]) ? P->tau * I->ctrl[C_BETA]
                                                                                    : I->ctrl[C_BETA];
      I->ctrl[C_PEND] = 1.0;
      I->ctrl[C_BNEXT] = bnext;
      I->ctrl[C_ZPREV] = zn;
      I->ctrl[C_KOUT] += 1.0;
      I->ctrl[C_LIN] = 0.0;
    }
  }
  /* adaptive penalty by residual balancing (future work named in Sec. V):
     every rho_every sweeps the three penalties grow by rho_tau when
     r_p > rho_mu r_d and shrink by it when r_d > rho_mu r_p, at most 6 net
     steps either way from the initial penalties */
  if (P->rho_every > 0 && I->ctrl[C_DONE] == 0.0) {
    I->ctrl[C_RCNT] += 1.0;
    if (I->ctrl[C_RCNT] >= (double)P->rho_every) {
      I->ctrl[C_RCNT] = 0.0;
      double sc = 1.0;
      if (I->res[0] > P->rho_mu * I->res[1] && I->ctrl[C_RLOG] < 6.0) sc = P->rho_tau;
      else if (I->res[1] > P->rho_mu * I->res[0] && I->ctrl[C_RLOG] > -6.0) sc = 1.0 / P->rho_tau;
      if (sc != 1.0) {
        I->ctrl[C_RLOG] += (sc > 1.0) ? 1.0 : -1.0;
        I->ctrl[C_RPQ] *= sc;
        I->ctrl[C_RVA] *= sc;
        I->ctrl[C_RUC] *= sc;
        I->P.rho_pq = I->ctrl[C_RPQ];
        I->P.rho_va = I->ctrl[C_RVA];
        I->P.rho_uc = I->ctrl[C_RUC];
      }
    }
  }
}

/* Threads of the x-step subproblem loops: n > 0 sets them (OpenMP build
   only); returns the number in use (1 for the plain build). */
EXPORT int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* out = {r_p, r_d, z_norm, inf_norm, objective, z_rms}; stats = {sweeps, newton, al, branch_fail} */
EXPORT void orc_residuals(const void *h, double *out, long *stats) {
  const orc_inst *I = (const orc_inst *)h;
  for (int k = 0; k < 6; ++k) out[k] = I->res[k];
  if (stats) {
    stats[0] = I->sweeps;
    stats[1] = I->newton_total;
    stats[2] = I->al_total;
    stats[3] = I->br_fail;
  }
}

/* Row values of the current iterate (for checks): a and b per row, canonical row order. */
EXPORT void orc_rows(void *h, double *GA, double *GB, double *BA, double *BB) {
  orc_inst *I = (orc_inst *)h;
  compute_a(I, I->GA, I->BA);
  compute_b(I, I->GB, I->BB);
  size_t GN = (size_t)NGR * I->T * I->ng, BN = (size_t)NBR * I->T * I->nl;
  memcpy(GA, I->GA, GN * 8); memcpy(GB, I->GB, GN * 8);
  memcpy(BA, I->BA, BN * 8); memcpy(BB, I->BB, BN * 8);
}

/*
 * Algorithm 2 for n_gen generators over T periods, inputs [T][n_gen]
 * (duplicate-row targets tau = ubar - z - y/rho), outputs u_on [T][n_gen] and
 * the DP cost per generator: the stage costs and the DP above, one generator
 * after another.  The CPU reference of the DP-only workload of Fig. 1.
 */
EXPORT void orc_ucdp_batch(int ng, int T, double rho, const double *tau_on, const double *tau_su,
                           const double *tau_sd, const double *c0, const double *csu, const double *csd,
                           const int32_t *TU, const int32_t *TD, const int32_t *u0, const int32_t *K0,
                           int8_t *u_on, double *cost) {
  double *ton = (double *)malloc(sizeof(double) * T), *tsu = (double *)malloc(sizeof(double) * T);
  double *tsd = (double *)malloc(sizeof(double) * T), *L = (double *)malloc(sizeof(double) * 4 * T);
  int32_t *u = (int32_t *)malloc(sizeof(int32_t) * T);
  for (int g = 0; g < ng; ++g) {
    for (int t = 0; t < T; ++t) {
      ton[t] = tau_on[(size_t)t * ng + g];
      tsu[t] = tau_su[(size_t)t * ng + g];
      tsd[t] = tau_sd[(size_t)t * ng + g];
    }
    orc_uc_stagecost(T, c0[g], csu[g], csd[g], rho, ton, tsu, tsd, L);
    int k0 = K0[g] < 0 ? 0 : (K0[g] > T ? T : K0[g]);
    cost[g] = orc_dp(T, TU[g] < 1 ? 1 : TU[g], TD[g] < 1 ? 1 : TD[g], u0[g] ? 1 : 0, k0, L, u);
    for (int t = 0; t < T; ++t) u_on[(size_t)t * ng + g] = (int8_t)u[t];
  }
  free(ton); free(tsu); free(tsd); free(L); free(u);
}
