// k_line_polar.cuh -- line x-update per (t, line ij) solved in polar form.
//
// The line subproblem (variables w_i, w_j, wR, wI, theta_i, theta_j and the
// line-limit slacks; the product equation wR^2 + wI^2 = w_i w_j and the angle
// equation theta_i - theta_j = atan2(wI, wR) of Eq. acopf) is parametrised by
// x = (V_i, V_j, d):
//   w_i = V_i^2, w_j = V_j^2, wR = V_i V_j cos d, wI = V_i V_j sin d,
// which satisfies both equations identically for |d| < pi.  The angle copies
// enter only through d = theta_i - theta_j and their own consensus rows, so
// their common mode has the closed form theta_i + theta_j = t_6 + t_7 and the
// two angle rows contribute rho_va/4 (d - (t_6 - t_7))^2.  The line limits
// p^2 + q^2 <= rate^2 (the slack form of Eq. uc_acopf_ij/ji_limit) are handled
// by the augmented Lagrangian for inequalities,
//   psi(g) = (max(0, mu + c g)^2 - mu^2) / (2c),  mu <- max(0, mu + c g),
// and are inactive on most lines, where one Newton solve ends the subproblem.
// This is the same subproblem as the W-form kernel (same feasible set and
// objective, hence the same KKT points); only the coordinates differ.
// The voltage bounds Vmin <= V <= Vmax are Eq. uc_acopf_w_bound; the angle
// bounds |theta| <= 2 pi of the W-form are never active and are dropped.
//
// Inner solver per x (3 variables): the same projected Newton method with an
// epsilon-active set, Cholesky (shifted only when not positive definite), a
// trust radius and the final-step rule as the W-form kernel.  Persistent
// kernel with per-lane work fetching (see k_branch.cuh).
#pragma once
#include "common.cuh"

namespace ucac {

struct PolK {
  double al[4], be[4], ga[4], ka[4];  // a_r = al V_i^2 + be V_j^2 + V_i V_j (ga cos d + ka sin d)
  double rate2, lo0, hi0, lo1, hi1;
};

struct PolP {
  double tg[8];
  double rpq, rva;
  double mu[2];  // line-limit multipliers (ij, ji)
  double c;
};

struct PolEval {
  double f, a[4];
};

// objective, and when D, gradient and Hessian (3x3) at x
template <bool D>
__device__ __forceinline__ PolEval pol_eval(const PolK &K, const PolP &P, const double (&x)[3], double (&g)[3],
                                            double (&H)[3][3]) {
  const double Vi = x[0], Vj = x[1], d = x[2];
  double s, c;
  sincos(d, &s, &c);
  const double Pv = Vi * Vj;
  PolEval R;
  R.f = 0.0;
  if (D) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g[i] = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) H[i][j] = 0.0;
    }
  }
  double da[4][3], d2a[4][6];  // Hessian of a_r packed (00,01,02,11,12,22)
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const double E = K.ga[r] * c + K.ka[r] * s;
    const double Ed = K.ka[r] * c - K.ga[r] * s;
    const double a = K.al[r] * Vi * Vi + K.be[r] * Vj * Vj + Pv * E;
    R.a[r] = a;
    const double e = a - P.tg[r];
    R.f += 0.5 * P.rpq * e * e;
    if (D) {
      da[r][0] = 2.0 * K.al[r] * Vi + Vj * E;
      da[r][1] = 2.0 * K.be[r] * Vj + Vi * E;
      da[r][2] = Pv * Ed;
      d2a[r][0] = 2.0 * K.al[r];
      d2a[r][1] = E;
      d2a[r][2] = Vj * Ed;
      d2a[r][3] = 2.0 * K.be[r];
      d2a[r][4] = Vi * Ed;
      d2a[r][5] = -Pv * E;
      const double pe = P.rpq * e;
#pragma unroll
      for (int i = 0; i < 3; ++i) g[i] += pe * da[r][i];
      H[0][0] += P.rpq * da[r][0] * da[r][0] + pe * d2a[r][0];
      H[0][1] += P.rpq * da[r][0] * da[r][1] + pe * d2a[r][1];
      H[0][2] += P.rpq * da[r][0] * da[r][2] + pe * d2a[r][2];
      H[1][1] += P.rpq * da[r][1] * da[r][1] + pe * d2a[r][3];
      H[1][2] += P.rpq * da[r][1] * da[r][2] + pe * d2a[r][4];
      H[2][2] += P.rpq * da[r][2] * da[r][2] + pe * d2a[r][5];
    }
  }
  // voltage-magnitude rows (w = V^2) and the angle rows (common mode eliminated)
  const double ewi = Vi * Vi - P.tg[4], ewj = Vj * Vj - P.tg[5], et = d - (P.tg[6] - P.tg[7]);
  R.f += 0.5 * P.rva * (ewi * ewi + ewj * ewj) + 0.25 * P.rva * et * et;
  if (D) {
    g[0] += 2.0 * P.rva * ewi * Vi;
    g[1] += 2.0 * P.rva * ewj * Vj;
    g[2] += 0.5 * P.rva * et;
    H[0][0] += P.rva * (4.0 * Vi * Vi + 2.0 * ewi);
    H[1][1] += P.rva * (4.0 * Vj * Vj + 2.0 * ewj);
    H[2][2] += 0.5 * P.rva;
  }
  // line limits g_k = a_{2k}^2 + a_{2k+1}^2 - rate^2 <= 0, inequality AL
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r0 = 2 * k, r1 = 2 * k + 1;
    const double gk = R.a[r0] * R.a[r0] + R.a[r1] * R.a[r1] - K.rate2;
    const double m = P.mu[k] + P.c * gk;
    if (m > 0.0) {
      R.f += (m * m - P.mu[k] * P.mu[k]) / (2.0 * P.c);
      if (D) {
        double dg[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) dg[i] = 2.0 * (R.a[r0] * da[r0][i] + R.a[r1] * da[r1][i]);
#pragma unroll
        for (int i = 0; i < 3; ++i) g[i] += m * dg[i];
        // m * d2g + c dg dg^T, d2g = 2 (da da^T + a d2a) summed over the pair
        const int pk[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = i; j < 3; ++j) {
            const double d2g = 2.0 * (da[r0][i] * da[r0][j] + R.a[r0] * d2a[r0][pk[i][j]] + da[r1][i] * da[r1][j] +
                                      R.a[r1] * d2a[r1][pk[i][j]]);
            H[i][j] += m * d2g + P.c * dg[i] * dg[j];
          }
      }
    } else {
      R.f -= P.mu[k] * P.mu[k] / (2.0 * P.c);
    }
  }
  if (D) {
    H[1][0] = H[0][1];
    H[2][0] = H[0][2];
    H[2][1] = H[1][2];
  }
  return R;
}

__device__ __forceinline__ double pol_lo(const PolK &K, int i) { return i == 0 ? K.lo0 : (i == 1 ? K.lo1 : -3.14159265358979); }
__device__ __forceinline__ double pol_hi(const PolK &K, int i) { return i == 0 ? K.hi0 : (i == 1 ? K.hi1 : 3.14159265358979); }

// 3x3 Cholesky solve of the masked Newton system; false when not positive definite
__device__ __forceinline__ bool chol3(double (&A)[3][3], double (&b)[3]) {
  const double s0 = A[0][0];
  if (!(s0 > 0.0)) return false;
  const double L00 = sqrt(s0), i0 = 1.0 / L00;
  const double L10 = A[1][0] * i0, L20 = A[2][0] * i0;
  const double s1 = A[1][1] - L10 * L10;
  if (!(s1 > 0.0)) return false;
  const double L11 = sqrt(s1), i1 = 1.0 / L11;
  const double L21 = (A[2][1] - L20 * L10) * i1;
  const double s2 = A[2][2] - L20 * L20 - L21 * L21;
  if (!(s2 > 0.0)) return false;
  const double L22 = sqrt(s2), i2 = 1.0 / L22;
  const double y0 = b[0] * i0, y1 = (b[1] - L10 * y0) * i1, y2 = (b[2] - L20 * y0 - L21 * y1) * i2;
  b[2] = y2 * i2;
  b[1] = (y1 - L21 * b[2]) * i1;
  b[0] = (y0 - L10 * b[1] - L20 * b[2]) * i0;
  return true;
}

__device__ __forceinline__ int pol_newton_iter(const PolK &K, const PolP &P, double (&x)[3], double &f,
                                               const double (&g)[3], const double (&H)[3][3], double &Delta,
                                               double omega, bool &accepted, int &counted) {
  accepted = false;
  counted = 0;
  double pg = 0.0, hmax = 0.0, xmax = 0.0, eps = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double lo = pol_lo(K, i), hi = pol_hi(K, i);
    pg = fmax(pg, fabs(clampd(x[i] - g[i], lo, hi) - x[i]));
    hmax = fmax(hmax, H[i][i]);
    xmax = fmax(xmax, fabs(x[i]));
    const double di = (H[i][i] > 0.0) ? g[i] / H[i][i] : g[i];
    eps = fmax(eps, fabs(clampd(x[i] - di, lo, hi) - x[i]));
  }
  if (pg <= omega) return NI_CONV;
  eps = fmin(eps, 1e-6);
  bool act[3];
  double d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double lo = pol_lo(K, i), hi = pol_hi(K, i);
    act[i] = false;
    d[i] = 0.0;
    if (x[i] <= lo + eps && g[i] > 0.0) {
      act[i] = true;
      d[i] = lo - x[i];
    } else if (x[i] >= hi - eps && g[i] < 0.0) {
      act[i] = true;
      d[i] = hi - x[i];
    }
  }
  double lm = 0.0, y[3];
  bool ok = false;
  for (int tries = 0; tries < 40; ++tries) {
    double A[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double r = -g[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (act[j]) r -= H[i][j] * d[j];
        A[i][j] = (act[i] || act[j]) ? ((i == j) ? 1.0 : 0.0) : H[i][j];
      }
      if (!act[i]) A[i][i] += lm;
      y[i] = act[i] ? d[i] : r;
    }
    if (chol3(A, y)) {
      ok = true;
      break;
    }
    lm = (lm == 0.0) ? 1e-10 * hmax : 10.0 * lm;
  }
  if (!ok) return NI_STOP;
  double dn = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    d[i] = y[i];
    dn = fmax(dn, fabs(d[i]));
  }
  counted = 1;
  if (lm == 0.0) {
    double gd = 0.0, dHd = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gd += g[i] * d[i];
      dHd += d[i] * (H[i][0] * d[0] + H[i][1] * d[1] + H[i][2] * d[2]);
    }
    const double predN = -(gd + 0.5 * dHd);
    if (dn <= 1e-9 * (1.0 + xmax) || predN <= 1e-12 * (1.0 + fabs(f))) {
#pragma unroll
      for (int i = 0; i < 3; ++i) x[i] = clampd(x[i] + d[i], pol_lo(K, i), pol_hi(K, i));
      return NI_CONV;
    }
  }
  const double scale = (dn > Delta) ? Delta / dn : 1.0;
  double xt[3], s[3], smax = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    xt[i] = clampd(x[i] + scale * d[i], pol_lo(K, i), pol_hi(K, i));
    s[i] = xt[i] - x[i];
    smax = fmax(smax, fabs(s[i]));
  }
  double gs = 0.0, sHs = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gs += g[i] * s[i];
    sHs += s[i] * (H[i][0] * s[0] + H[i][1] * s[1] + H[i][2] * s[2]);
  }
  const double pred = -(gs + 0.5 * sHs);
  double gd_[3], Hd_[3][3];
  const double ft = pol_eval<false>(K, P, xt, gd_, Hd_).f;
  const double ared = f - ft;
  if (pred > 0.0 && ared >= 1e-4 * pred) {
#pragma unroll
    for (int i = 0; i < 3; ++i) x[i] = xt[i];
    f = ft;
    accepted = true;
    if (ared >= 0.75 * pred && scale < 1.0) Delta = 2.0 * Delta;
    return NI_CONT;
  }
  Delta = 0.25 * smax;
  if (Delta <= 1e-15 * (1.0 + xmax)) {
    counted = 0;
    return NI_STOP;
  }
  return NI_CONT;
}

template <int BS>
__global__ void __launch_bounds__(BS) k_line_polar(Dev S) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long NBP = S.NBP, NL = S.NL;
  const double eta = S.prm.eta;
  const int K_N = S.prm.K_N, K_AL = S.prm.K_AL;
  bool active = true;
  long long bp = -1;
  int k = 0, itn = 0, al = 0, newton = 0;
  bool need_f = false, need_gH = false;
  double f = 0.0, Delta = 1.0, hprev = INFINITY, omega = 0.0, cmax = 0.0;
  double x[3], g[3], H[3][3];
  PolK K;
  PolP P;
  while (true) {
    const bool want = active && bp < 0;
    const unsigned m = __ballot_sync(FULL, want);
    if (m) {
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(S.bp_counter, (unsigned long long)__popc(m));
      base = __shfl_sync(FULL, base, leader);
      if (want) {
        const long long item = (long long)base + __popc(m & ((1u << lane) - 1u));
        if (item >= NBP) {
          active = false;
        } else {
          bp = item;
          k = find_instance(S, bp);
          const Inst &I = S.inst[k];
          const int loc = (int)(bp - I.bpo);
          const int t = loc / I.nl, l = loc - t * I.nl;
          const long long lg = (long long)I.lo + l;
          const double Gii = S.BC[(BC_Y0 + 0) * NL + lg], Bii = S.BC[(BC_Y0 + 1) * NL + lg];
          const double Gij = S.BC[(BC_Y0 + 2) * NL + lg], Bij = S.BC[(BC_Y0 + 3) * NL + lg];
          const double Gjj = S.BC[(BC_Y0 + 4) * NL + lg], Bjj = S.BC[(BC_Y0 + 5) * NL + lg];
          const double Gji = S.BC[(BC_Y0 + 6) * NL + lg], Bji = S.BC[(BC_Y0 + 7) * NL + lg];
          K.al[0] = Gii;  K.be[0] = 0.0;  K.ga[0] = Gij;  K.ka[0] = Bij;
          K.al[1] = -Bii; K.be[1] = 0.0;  K.ga[1] = -Bij; K.ka[1] = Gij;
          K.al[2] = 0.0;  K.be[2] = Gjj;  K.ga[2] = Gji;  K.ka[2] = -Bji;
          K.al[3] = 0.0;  K.be[3] = -Bjj; K.ga[3] = -Bji; K.ka[3] = -Gji;
          K.rate2 = S.BC[BC_RATE2 * NL + lg];
          K.lo0 = sqrt(S.BC[(BC_LO + 0) * NL + lg]);
          K.hi0 = sqrt(S.BC[(BC_HI + 0) * NL + lg]);
          K.lo1 = sqrt(S.BC[(BC_LO + 1) * NL + lg]);
          K.hi1 = sqrt(S.BC[(BC_HI + 1) * NL + lg]);
#pragma unroll
          for (int r = 0; r < 8; ++r) P.tg[r] = S.BT[r * NBP + bp];
          P.rpq = I.rpq;
          P.rva = I.rva;
          P.mu[0] = fmax(S.B[(FB_MU0 + 2) * NBP + bp], 0.0);
          P.mu[1] = fmax(S.B[(FB_MU0 + 3) * NBP + bp], 0.0);
          P.c = S.B[FB_C * NBP + bp];
          // warm start from the stored iterate: V = sqrt(w), d = theta_i - theta_j
          x[0] = clampd(sqrt(fmax(S.B[(FB_V0 + 0) * NBP + bp], 0.0)), K.lo0, K.hi0);
          x[1] = clampd(sqrt(fmax(S.B[(FB_V0 + 1) * NBP + bp], 0.0)), K.lo1, K.hi1);
          x[2] = clampd(S.B[(FB_V0 + 4) * NBP + bp] - S.B[(FB_V0 + 5) * NBP + bp], pol_lo(K, 2), pol_hi(K, 2));
          const double rmax = fmax(I.rpq, I.rva);
          omega = S.prm.omega_rel * rmax;
          cmax = S.prm.c_max_rel * rmax;
          hprev = INFINITY;
          Delta = 1.0;
          itn = al = newton = 0;
          need_f = need_gH = true;
        }
      }
    }
    if (__ballot_sync(FULL, active) == 0) break;
    if (active) {
      if (need_gH) {
        f = pol_eval<true>(K, P, x, g, H).f;
      } else if (need_f) {
        double gd_[3], Hd_[3][3];
        f = pol_eval<false>(K, P, x, gd_, Hd_).f;
      }
      need_f = need_gH = false;
      bool accepted;
      int counted;
      const int out = pol_newton_iter(K, P, x, f, g, H, Delta, omega, accepted, counted);
      newton += counted;
      need_gH = accepted;
      ++itn;
      if (out != NI_CONT || itn >= K_N) {
        const bool conv = (out == NI_CONV);
        double gd_[3], Hd_[3][3];
        const PolEval E = pol_eval<false>(K, P, x, gd_, Hd_);
        double hn = 0.0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const double gk = E.a[2 * q] * E.a[2 * q] + E.a[2 * q + 1] * E.a[2 * q + 1] - K.rate2;
          const double mn = fmax(0.0, P.mu[q] + P.c * gk);
          hn = fmax(hn, fabs(mn - P.mu[q]) / P.c);
          P.mu[q] = mn;
        }
        ++al;
        const bool done = (hn <= eta && conv);
        if (done || al >= K_AL) {
          double s, c;
          sincos(x[2], &s, &c);
          const double Pv = x[0] * x[1], tm = 0.5 * (P.tg[6] + P.tg[7]);
          const double v8[8] = {x[0] * x[0], x[1] * x[1], Pv * c, Pv * s, tm + 0.5 * x[2], tm - 0.5 * x[2],
                                clampd(K.rate2 - E.a[0] * E.a[0] - E.a[1] * E.a[1], 0.0, K.rate2),
                                clampd(K.rate2 - E.a[2] * E.a[2] - E.a[3] * E.a[3], 0.0, K.rate2)};
#pragma unroll
          for (int i = 0; i < 8; ++i) S.B[(FB_V0 + i) * NBP + bp] = v8[i];
          S.B[(FB_MU0 + 0) * NBP + bp] = 0.0;
          S.B[(FB_MU0 + 1) * NBP + bp] = 0.0;
          S.B[(FB_MU0 + 2) * NBP + bp] = P.mu[0];
          S.B[(FB_MU0 + 3) * NBP + bp] = P.mu[1];
          S.B[FB_C * NBP + bp] = P.c;
#pragma unroll
          for (int r = 0; r < 4; ++r) S.BA[r * NBP + bp] = E.a[r];
          S.BA[4 * NBP + bp] = v8[0];
          S.BA[5 * NBP + bp] = v8[1];
          S.BA[6 * NBP + bp] = v8[4];
          S.BA[7 * NBP + bp] = v8[5];
          long long *st = S.bstat + (long long)k * 3;
          atomicAdd((unsigned long long *)&st[0], (unsigned long long)newton);
          atomicAdd((unsigned long long *)&st[1], (unsigned long long)al);
          if (!done) atomicAdd((unsigned long long *)&st[2], 1ull);
          bp = -1;
        } else {
          if (hn > 0.25 * hprev) P.c = fmin(10.0 * P.c, cmax);
          hprev = hn;
          Delta = fmax(Delta, 1e-3);
          itn = 0;
          need_f = need_gH = true;
        }
      }
    }
  }
}

}  // namespace ucac
