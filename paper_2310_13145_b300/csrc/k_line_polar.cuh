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
// trust radius and the final-step rule as the W-form kernel; in addition an
// undamped step of size <= 1e-4 (1 + |x|) inside the radius is accepted
// without the ratio test (its model error is at the rounding level).
// Precision split (B300's FP64 pipe is 1/64 of its FP32 pipe): the iterate,
// flows, residuals, gradient and objective are FP64 -- they fix the converged
// point -- while the Hessian and the Newton system are FP32 on lanes whose
// line limits are inactive (condition number ~1e3-1e4, so the direction is
// accurate to ~1e-4 and Newton still converges in a step or two); lanes with
// an active limit (penalty c up to 1e6 rho, condition up to ~1e9) keep the
// FP64 Hessian.  After the last (tiny) step the flows and cos/sin are updated
// to first order from the last evaluation instead of being re-evaluated (the
// error is the square of a step below 1e-9).  Persistent kernel with per-lane
// work fetching (see k_branch.cuh).
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

// last full evaluation: flows, their gradients (FP32: used only for the
// first-order update after a tiny step), cos/sin and the point
struct PolLast {
  double a[4], c, s, x[3];
  float da[4][3];
  bool lim;  // a line-limit term is active: the FP64 Hessian is in use
};

__device__ __forceinline__ double pol_lo(const PolK &K, int i) { return i == 0 ? K.lo0 : (i == 1 ? K.lo1 : -3.14159265358979); }
__device__ __forceinline__ double pol_hi(const PolK &K, int i) { return i == 0 ? K.hi0 : (i == 1 ? K.hi1 : 3.14159265358979); }

// objective (and flows, cos/sin) at x
__device__ __forceinline__ double pol_obj(const PolK &K, const PolP &P, const double (&x)[3], double (&a)[4],
                                          double &c, double &s) {
  const double Vi = x[0], Vj = x[1], d = x[2];
  sincos(d, &s, &c);
  const double Pv = Vi * Vj;
  double f = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = K.al[r] * Vi * Vi + K.be[r] * Vj * Vj + Pv * (K.ga[r] * c + K.ka[r] * s);
    const double e = a[r] - P.tg[r];
    f += 0.5 * P.rpq * e * e;
  }
  const double ewi = Vi * Vi - P.tg[4], ewj = Vj * Vj - P.tg[5], et = d - (P.tg[6] - P.tg[7]);
  f += 0.5 * P.rva * (ewi * ewi + ewj * ewj) + 0.25 * P.rva * et * et;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double gk = a[2 * k] * a[2 * k] + a[2 * k + 1] * a[2 * k + 1] - K.rate2;
    const double m = P.mu[k] + P.c * gk;
    f += (m > 0.0) ? (m * m - P.mu[k] * P.mu[k]) / (2.0 * P.c) : -P.mu[k] * P.mu[k] / (2.0 * P.c);
  }
  return f;
}

// objective, gradient (FP64) and Hessian (FP32 Hf, or FP64 Hd when a line
// limit is active) at x; fills L
__device__ __forceinline__ double pol_full(const PolK &K, const PolP &P, const double (&x)[3], double (&g)[3],
                                           float (&Hf)[6], double (&Hd)[6], PolLast &L) {
  const double Vi = x[0], Vj = x[1], d = x[2];
  double s, c;
  sincos(d, &s, &c);
  L.c = c;
  L.s = s;
  L.x[0] = Vi;
  L.x[1] = Vj;
  L.x[2] = d;
  const double Pv = Vi * Vj;
  double f = 0.0;
  g[0] = g[1] = g[2] = 0.0;
  double da[4][3], E[4], Ed[4], pe[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    E[r] = K.ga[r] * c + K.ka[r] * s;
    Ed[r] = K.ka[r] * c - K.ga[r] * s;
    const double a = K.al[r] * Vi * Vi + K.be[r] * Vj * Vj + Pv * E[r];
    L.a[r] = a;
    const double e = a - P.tg[r];
    f += 0.5 * P.rpq * e * e;
    da[r][0] = 2.0 * K.al[r] * Vi + Vj * E[r];
    da[r][1] = 2.0 * K.be[r] * Vj + Vi * E[r];
    da[r][2] = Pv * Ed[r];
    pe[r] = P.rpq * e;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g[i] += pe[r] * da[r][i];
      L.da[r][i] = (float)da[r][i];
    }
  }
  const double ewi = Vi * Vi - P.tg[4], ewj = Vj * Vj - P.tg[5], et = d - (P.tg[6] - P.tg[7]);
  f += 0.5 * P.rva * (ewi * ewi + ewj * ewj) + 0.25 * P.rva * et * et;
  g[0] += 2.0 * P.rva * ewi * Vi;
  g[1] += 2.0 * P.rva * ewj * Vj;
  g[2] += 0.5 * P.rva * et;
  double m[2];
  bool lim = false;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r0 = 2 * k, r1 = 2 * k + 1;
    const double gk = L.a[r0] * L.a[r0] + L.a[r1] * L.a[r1] - K.rate2;
    m[k] = P.mu[k] + P.c * gk;
    if (m[k] > 0.0) {
      lim = true;
      f += (m[k] * m[k] - P.mu[k] * P.mu[k]) / (2.0 * P.c);
#pragma unroll
      for (int i = 0; i < 3; ++i) g[i] += m[k] * 2.0 * (L.a[r0] * da[r0][i] + L.a[r1] * da[r1][i]);
    } else {
      f -= P.mu[k] * P.mu[k] / (2.0 * P.c);
    }
  }
  L.lim = lim;
  // packed symmetric index: 0:(0,0) 1:(0,1) 2:(0,2) 3:(1,1) 4:(1,2) 5:(2,2)
  const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
  if (!lim) {
    const float fVi = (float)Vi, fVj = (float)Vj, fP = (float)Pv, rpq = (float)P.rpq, rva = (float)P.rva;
#pragma unroll
    for (int q = 0; q < 6; ++q) Hf[q] = 0.0f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float fE = (float)E[r], fEd = (float)Ed[r], fpe = (float)pe[r];
      const float d2[6] = {2.0f * (float)K.al[r], fE, fVj * fEd, 2.0f * (float)K.be[r], fVi * fEd, -fP * fE};
#pragma unroll
      for (int q = 0; q < 6; ++q) Hf[q] += rpq * L.da[r][pi_[q]] * L.da[r][pj_[q]] + fpe * d2[q];
    }
    Hf[0] += rva * (4.0f * fVi * fVi + 2.0f * (float)ewi);
    Hf[3] += rva * (4.0f * fVj * fVj + 2.0f * (float)ewj);
    Hf[5] += 0.5f * rva;
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) Hd[q] = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double d2[6] = {2.0 * K.al[r], E[r], Vj * Ed[r], 2.0 * K.be[r], Vi * Ed[r], -Pv * E[r]};
#pragma unroll
      for (int q = 0; q < 6; ++q) Hd[q] += P.rpq * da[r][pi_[q]] * da[r][pj_[q]] + pe[r] * d2[q];
    }
    Hd[0] += P.rva * (4.0 * Vi * Vi + 2.0 * ewi);
    Hd[3] += P.rva * (4.0 * Vj * Vj + 2.0 * ewj);
    Hd[5] += 0.5 * P.rva;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (m[k] > 0.0) {
        const int r0 = 2 * k, r1 = 2 * k + 1;
        double dg[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) dg[i] = 2.0 * (L.a[r0] * da[r0][i] + L.a[r1] * da[r1][i]);
        const double d2r0[6] = {2.0 * K.al[r0], E[r0], Vj * Ed[r0], 2.0 * K.be[r0], Vi * Ed[r0], -Pv * E[r0]};
        const double d2r1[6] = {2.0 * K.al[r1], E[r1], Vj * Ed[r1], 2.0 * K.be[r1], Vi * Ed[r1], -Pv * E[r1]};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const int i = pi_[q], j = pj_[q];
          const double d2g = 2.0 * (da[r0][i] * da[r0][j] + L.a[r0] * d2r0[q] + da[r1][i] * da[r1][j] +
                                    L.a[r1] * d2r1[q]);
          Hd[q] += m[k] * d2g + P.c * dg[i] * dg[j];
        }
      }
    }
  }
  return f;
}

// masked 3x3 Cholesky solve (packed symmetric A), T = float or double
template <typename T>
__device__ __forceinline__ bool chol3p(const T (&A)[6], T (&b)[3]) {
  const T s0 = A[0];
  if (!(s0 > T(0))) return false;
  const T L00 = sqrt(s0), i0 = T(1) / L00;
  const T L10 = A[1] * i0, L20 = A[2] * i0;
  const T s1 = A[3] - L10 * L10;
  if (!(s1 > T(0))) return false;
  const T L11 = sqrt(s1), i1 = T(1) / L11;
  const T L21 = (A[4] - L20 * L10) * i1;
  const T s2 = A[5] - L20 * L20 - L21 * L21;
  if (!(s2 > T(0))) return false;
  const T L22 = sqrt(s2), i2 = T(1) / L22;
  const T y0 = b[0] * i0, y1 = (b[1] - L10 * y0) * i1, y2 = (b[2] - L20 * y0 - L21 * y1) * i2;
  b[2] = y2 * i2;
  b[1] = (y1 - L21 * b[2]) * i1;
  b[0] = (y0 - L10 * b[1] - L20 * b[2]) * i0;
  return true;
}

template <typename T>
__device__ __forceinline__ T hq(const T (&H)[6], int i, int j) {
  const int q = (i == j) ? (i == 0 ? 0 : (i == 1 ? 3 : 5)) : ((i + j == 1) ? 1 : ((i + j == 2) ? 2 : 4));
  return H[q];
}

// one Newton iteration with the Hessian H of type T (see newton_iter of the
// W-form kernel for the steps)
template <typename T>
__device__ __forceinline__ int pol_iter(const PolK &K, const PolP &P, double (&x)[3], double &f, const double (&g)[3],
                                        const T (&H)[6], double &Delta, double omega, bool &accepted, int &counted) {
  accepted = false;
  counted = 0;
  double pg = 0.0, xmax = 0.0;
  T hmax = T(0), eps = T(0), dlo[3], dhi[3], gt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double lo = pol_lo(K, i), hi = pol_hi(K, i);
    pg = fmax(pg, fabs(clampd(x[i] - g[i], lo, hi) - x[i]));
    xmax = fmax(xmax, fabs(x[i]));
    dlo[i] = (T)(x[i] - lo);
    dhi[i] = (T)(hi - x[i]);
    gt[i] = (T)g[i];
    const T hii = hq(H, i, i);
    hmax = hmax > hii ? hmax : hii;
    const T di = (hii > T(0)) ? gt[i] / hii : gt[i];
    const T st = (-di < -dlo[i]) ? -dlo[i] : ((-di > dhi[i]) ? dhi[i] : -di);
    const T ast = st < T(0) ? -st : st;
    eps = eps > ast ? eps : ast;
  }
  if (pg <= omega) return NI_CONV;
  eps = eps < T(1e-6) ? eps : T(1e-6);
  bool act[3];
  T d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    act[i] = false;
    d[i] = T(0);
    if (dlo[i] <= eps && gt[i] > T(0)) {
      act[i] = true;
      d[i] = -dlo[i] * T(1.000001);  // onto the bound (clamped below)
    } else if (dhi[i] <= eps && gt[i] < T(0)) {
      act[i] = true;
      d[i] = dhi[i] * T(1.000001);
    }
  }
  T lm = T(0), y[3];
  bool ok = false;
  for (int tries = 0; tries < 40; ++tries) {
    T A[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int i = (q < 3) ? 0 : ((q < 5) ? 1 : 2), j = (q == 0) ? 0 : ((q == 1 || q == 3) ? 1 : 2);
      A[q] = (act[i] || act[j]) ? ((i == j) ? T(1) : T(0)) : H[q];
      if (i == j && !act[i]) A[q] += lm;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T r = -gt[i];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (act[j]) r -= hq(H, i, j) * d[j];
      y[i] = act[i] ? d[i] : r;
    }
    if (chol3p(A, y)) {
      ok = true;
      break;
    }
    lm = (lm == T(0)) ? T(1e-10) * hmax : T(10) * lm;
  }
  if (!ok) return NI_STOP;
  T dn = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    d[i] = y[i];
    const T ad = d[i] < T(0) ? -d[i] : d[i];
    dn = dn > ad ? dn : ad;
  }
  counted = 1;
  if (lm == T(0)) {
    T gd = T(0), dHd = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      gd += gt[i] * d[i];
      dHd += d[i] * (hq(H, i, 0) * d[0] + hq(H, i, 1) * d[1] + hq(H, i, 2) * d[2]);
    }
    const T predN = -(gd + T(0.5) * dHd);
    if ((double)dn <= 1e-9 * (1.0 + xmax) || (double)predN <= 1e-12 * (1.0 + fabs(f))) {
#pragma unroll
      for (int i = 0; i < 3; ++i) x[i] = clampd(x[i] + (double)d[i], pol_lo(K, i), pol_hi(K, i));
      return NI_CONV;
    }
    if ((double)dn <= 1e-4 * (1.0 + xmax) && (double)dn <= Delta) {
#pragma unroll
      for (int i = 0; i < 3; ++i) x[i] = clampd(x[i] + (double)d[i], pol_lo(K, i), pol_hi(K, i));
      accepted = true;
      return NI_CONT;
    }
  }
  const double scale = ((double)dn > Delta) ? Delta / (double)dn : 1.0;
  double xt[3], smax = 0.0;
  T sv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    xt[i] = clampd(x[i] + scale * (double)d[i], pol_lo(K, i), pol_hi(K, i));
    const double si = xt[i] - x[i];
    sv[i] = (T)si;
    smax = fmax(smax, fabs(si));
  }
  T gs = T(0), sHs = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gs += gt[i] * sv[i];
    sHs += sv[i] * (hq(H, i, 0) * sv[0] + hq(H, i, 1) * sv[1] + hq(H, i, 2) * sv[2]);
  }
  const double pred = -(double)(gs + T(0.5) * sHs);
  double at[4], ct, stn;
  const double ft = pol_obj(K, P, xt, at, ct, stn);
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
  // per-lane statistics, flushed to the instance's counters when the lane
  // moves to another instance or retires (consecutive items mostly share one)
  int acc_k = -1;
  unsigned long long acc_nw = 0, acc_al = 0, acc_cap = 0;
  auto flush = [&]() {
    if (acc_k >= 0) {
      unsigned long long *st = (unsigned long long *)(S.bstat + (long long)acc_k * 3);
      atomicAdd(&st[0], acc_nw);
      atomicAdd(&st[1], acc_al);
      if (acc_cap) atomicAdd(&st[2], acc_cap);
    }
    acc_nw = acc_al = acc_cap = 0;
  };
  bool need_full = false;
  double f = 0.0, Delta = 1.0, hprev = INFINITY, omega = 0.0, cmax = 0.0;
  double x[3], g[3], Hd[6];
  float Hf[6];
  PolLast L;
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
          flush();
        } else {
          bp = item;
          k = find_instance(S, bp);
          if (k != acc_k) {
            flush();
            acc_k = k;
          }
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
          K.lo0 = S.BC[(BC_VB + 0) * NL + lg];
          K.hi0 = S.BC[(BC_VB + 1) * NL + lg];
          K.lo1 = S.BC[(BC_VB + 2) * NL + lg];
          K.hi1 = S.BC[(BC_VB + 3) * NL + lg];
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
          need_full = true;
        }
      }
    }
    if (__ballot_sync(FULL, active) == 0) break;
    if (active) {
      if (need_full) f = pol_full(K, P, x, g, Hf, Hd, L);
      need_full = false;
      bool accepted;
      int counted;
      const int out = L.lim ? pol_iter<double>(K, P, x, f, g, Hd, Delta, omega, accepted, counted)
                            : pol_iter<float>(K, P, x, f, g, Hf, Delta, omega, accepted, counted);
      newton += counted;
      need_full = accepted;
      ++itn;
      if (out != NI_CONT || itn >= K_N) {
        const bool conv = (out == NI_CONV);
        // flows and cos/sin at x: first order from the last evaluation after a
        // converged (tiny final) step, a fresh evaluation otherwise
        double a[4], c, sn;
        if (conv) {
          const double dx0 = x[0] - L.x[0], dx1 = x[1] - L.x[1], dx2 = x[2] - L.x[2];
#pragma unroll
          for (int r = 0; r < 4; ++r)
            a[r] = L.a[r] + (double)L.da[r][0] * dx0 + (double)L.da[r][1] * dx1 + (double)L.da[r][2] * dx2;
          c = L.c - L.s * dx2;
          sn = L.s + L.c * dx2;
        } else {
          pol_obj(K, P, x, a, c, sn);
        }
        double hn = 0.0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const double gk = a[2 * q] * a[2 * q] + a[2 * q + 1] * a[2 * q + 1] - K.rate2;
          const double mn = fmax(0.0, P.mu[q] + P.c * gk);
          hn = fmax(hn, fabs(mn - P.mu[q]) / P.c);
          P.mu[q] = mn;
        }
        ++al;
        const bool done = (hn <= eta && conv);
        if (done || al >= K_AL) {
          const double Pv = x[0] * x[1], tm = 0.5 * (P.tg[6] + P.tg[7]);
          const double v8[8] = {x[0] * x[0], x[1] * x[1], Pv * c, Pv * sn, tm + 0.5 * x[2], tm - 0.5 * x[2],
                                clampd(K.rate2 - a[0] * a[0] - a[1] * a[1], 0.0, K.rate2),
                                clampd(K.rate2 - a[2] * a[2] - a[3] * a[3], 0.0, K.rate2)};
#pragma unroll
          for (int i = 0; i < 8; ++i) S.B[(FB_V0 + i) * NBP + bp] = v8[i];
          S.B[(FB_MU0 + 0) * NBP + bp] = 0.0;
          S.B[(FB_MU0 + 1) * NBP + bp] = 0.0;
          S.B[(FB_MU0 + 2) * NBP + bp] = P.mu[0];
          S.B[(FB_MU0 + 3) * NBP + bp] = P.mu[1];
          S.B[FB_C * NBP + bp] = P.c;
#pragma unroll
          for (int r = 0; r < 4; ++r) S.BA[r * NBP + bp] = a[r];
          S.BA[4 * NBP + bp] = v8[0];
          S.BA[5 * NBP + bp] = v8[1];
          S.BA[6 * NBP + bp] = v8[4];
          S.BA[7 * NBP + bp] = v8[5];
          acc_nw += (unsigned long long)newton;
          acc_al += (unsigned long long)al;
          acc_cap += done ? 0ull : 1ull;
          bp = -1;
        } else {
          if (hn > 0.25 * hprev) P.c = fmin(10.0 * P.c, cmax);
          hprev = hn;
          Delta = fmax(Delta, 1e-3);
          itn = 0;
          need_full = true;
        }
      }
    }
  }
}

}  // namespace ucac
