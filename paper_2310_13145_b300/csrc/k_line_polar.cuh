// k_line_polar.cuh -- line x-update per (t, line ij) solved in polar form.
//
// The line subproblem (variables w_i, w_j, wR, wI, theta_i, theta_j and the
// line-limit slacks sigma_ij, sigma_ji; the product equation wR^2 + wI^2 =
// w_i w_j and the angle equation theta_i - theta_j = atan2(wI, wR) of
// Eq. acopf) is parametrised by x = (V_i, V_j, d):
//   w_i = V_i^2, w_j = V_j^2, wR = V_i V_j cos d, wI = V_i V_j sin d,
// which satisfies both equations identically for |d| < pi.  The angle copies
// enter only through d = theta_i - theta_j and their own consensus rows, so
// their common mode has the closed form theta_i + theta_j = t_6 + t_7 and the
// two angle rows contribute rho_va/4 (d - (t_6 - t_7))^2.  The line limits
// keep the slack form of Eq. uc_acopf_ij/ji_limit,
//   h_k = p_k^2 + q_k^2 + sigma_k - rate^2 = 0,  sigma_k >= 0,
// under the augmented Lagrangian mu_k h_k + c/2 h_k^2 with the bounded slacks
// as variables, so the inner objective over v = (V_i, V_j, d, sigma_ij,
// sigma_ji) is smooth and the bound sigma_k >= 0 is met by projection (an
// inequality penalty max(0, .)^2 in x alone has a curvature jump of order c
// at the limit, which stalls the trust-region Newton once c is large).
// This is the same subproblem as the W-form kernel (same feasible set and
// objective, hence the same KKT points); only the coordinates differ.  The
// W-form's upper slack bound sigma_k <= rate^2 is implied by h_k = 0 and is
// dropped: held by an epsilon-active set on a line with almost no flow it
// would pin h_k at the flow's square and make the multiplier oscillate.
// The voltage bounds Vmin <= V <= Vmax are Eq. uc_acopf_w_bound; the angle
// bounds |theta| <= 2 pi of the W-form are never active and are dropped.
//
// Inner solver: the projected Newton method with an epsilon-active set,
// Cholesky (shifted only when not positive definite), a trust radius on x and
// the final-step rule of the W-form kernel, applied to the five variables.
// The objective is quadratic in each slack with curvature c and coupling
// c grad(g_k), so a free slack is eliminated from the Newton system exactly:
// the 3x3 system in x carries c grad(g_k) grad(g_k)^T only for slacks held
// at zero, the slack step follows from the x step, and the x-Hessian drops
// m_k hess(g_k) of a free slack (m_k = mu_k + c h_k vanishes at the slack's
// optimum: this is the Hessian of the problem reduced over the slack).
// Stationarity is tested on the reduced gradient, after which each free
// slack takes its exact step -m_k / c.  A trial step gets a second-order
// correction before the ratio test: free slacks absorb the O(|dx|^2)
// remainder of g_k, and a slack held at zero gets a correction in x along
// grad g_k, so that c/2 h_k^2 sees the linear prediction instead of the
// remainder magnified by c.  An undamped Newton step (unshifted, so the
// Hessian is positive definite and the step descends on the model) of size
// <= 1e-3 (1 + |x|) inside the radius that leaves every free variable inside
// its box is accepted without the ratio test: its model error, O(|d|^3), is
// far below the decrease, and the trial evaluation it saves was most of the
// cost of the late sweeps of a run (1e-2 gains nothing more).
// Precision split (B300's FP64 pipe is 1/64 of its FP32 pipe; it also runs
// the FP32 <-> FP64 conversions, so the FP32 copies are made on the integer
// units: d2f_trunc, f2d_exact): the iterate,
// flows, residuals, gradient and objective are FP64 -- they fix the converged
// point -- while the Hessian and the Newton system are FP32 on lanes whose
// slacks are off zero (condition number ~1e3-1e4, so the direction is
// accurate to ~1e-4 and Newton still converges in a step or two); lanes with
// a slack held at zero (the c grad grad^T term, c up to 1e6 rho) keep the
// FP64 Hessian.  After a final step below 1e-8 the flows and cos/sin are
// updated to first order from the last evaluation, and h_k in FP64 from
// grad g_k (the gradient the slack step was taken from), instead of being
// re-evaluated (the error is the square of the step).  Persistent kernel
// with per-lane work fetching (see k_branch.cuh).
#pragma once
#include "common.cuh"

// 1: the Hessian and the 3x3 Newton system in FP64 on every lane (default
// 0: FP32 on lanes without a held slack, see the precision split above)
#ifndef UCAC_POL_FP64_NEWTON
#define UCAC_POL_FP64_NEWTON 0
#endif

namespace ucac {

// FP64 <-> T (float or double) for the Newton system of type T; the FP32
// conversions run on the integer units (see d2f_trunc, f2d_exact)
template <typename T>
__device__ __forceinline__ T to_t(double x) {
  if constexpr (sizeof(T) == 4)
    return d2f_trunc(x);
  else
    return x;
}
template <typename T>
__device__ __forceinline__ double to_d(T x) {
  if constexpr (sizeof(T) == 4)
    return f2d_exact(x);
  else
    return x;
}

// a_r = q_r V'^2 + V_i V_j E_r with E_r = ga_r cos d + ka_r sin d and V' =
// V_i for the from-end rows r = 0, 1 and V_j for the to-end rows r = 2, 3.
// Within each end the coefficients pair up, (ga_1, ka_1) = (-ka_0, ga_0) and
// (ga_3, ka_3) = (ka_2, -ga_2), so with Ed_r = dE_r/dd only E and Ed of rows 0
// and 2 are formed: E_1 = -Ed_0, Ed_1 = E_0, E_3 = Ed_2, Ed_3 = -E_2.  ga[e],
// ka[e] hold the coefficients of row 2e.  FP32 copies of q, ga, ka for the
// mixed-precision Hessian sit in shared memory (f[j * fs]: q_0..q_3, ga_0,
// ga_1, ka_0, ka_1), so they cost neither registers nor per-evaluation
// conversions on the FP64 pipe
struct PolK {
  double q[4], ga[2], ka[2];
  double rate2, lo0, hi0, lo1, hi1;
  const float *f;
  int fs;
  __device__ __forceinline__ float fq(int r) const { return f[r * fs]; }
  __device__ __forceinline__ float fga(int e) const { return f[(4 + e) * fs]; }
  __device__ __forceinline__ float fka(int e) const { return f[(6 + e) * fs]; }
  // FP32 copies of the voltage bounds (truncated; f[(8 + j) * fs]: lo0, hi0,
  // lo1, hi1), for the common step's near-bound prefilter
  __device__ __forceinline__ float flo(int i) const { return f[(8 + 2 * i) * fs]; }
  __device__ __forceinline__ float fhi(int i) const { return f[(9 + 2 * i) * fs]; }
};

// E_r and Ed_r of the four flow rows from those of rows 0 and 2 (T = double
// or float; the negations fold into the consuming operations)
template <typename T>
__device__ __forceinline__ void pol_angle_terms(T ga0, T ka0, T ga2, T ka2, T c, T s, T (&E)[4], T (&Ed)[4]) {
  E[0] = ga0 * c + ka0 * s;
  Ed[0] = ka0 * c - ga0 * s;
  E[2] = ga2 * c + ka2 * s;
  Ed[2] = ka2 * c - ga2 * s;
  E[1] = -Ed[0];
  Ed[1] = E[0];
  E[3] = Ed[2];
  Ed[3] = -E[2];
}

struct PolP {
  // row targets: t_0..t_5, then the angle rows' difference t_6 - t_7 and
  // mean (t_6 + t_7) / 2 (each formed once per solve)
  double tg[8];
  double rpq, rva;
  float frpq, frva;  // FP32 copies for the Hessian
  double mu[2];  // line-limit multipliers (ij, ji)
  double c, ic;  // penalty and its reciprocal
};

// last full evaluation: flows, their gradients (FP32: used only for the
// first-order update after a tiny step), cos/sin, the point, the limit
// gradients grad(g_k) in FP32 and the multiplier estimates m_k = mu_k + c h_k.
// A free slack is eliminated from the Newton system exactly, so grad g_k
// reaches the x iterates only where a slack is held at zero, a variable is
// near a bound or a trust-region step is modelled: there pol_iter forms it
// in FP64 from the point (pol_dg64).  Elsewhere it enters only the free
// slacks' step and the first-order h_k of a finish after a tiny step, where
// the FP32 copy's ~1e-7 relative error times the step is far below the
// tolerances.
struct PolLast {
  double a[4], c, s, v[5];
  double m[2], h[2];
  float fdg[2][3];
  float da[4][3];
  bool lim;  // a slack is held at zero: the FP64 Hessian is in use
};

constexpr int POL_NV = 5;  // V_i, V_j, d, sigma_ij, sigma_ji

__device__ __forceinline__ double pol_lo(const PolK &K, int i) {
  return i == 0 ? K.lo0 : (i == 1 ? K.lo1 : (i == 2 ? -3.14159265358979 : 0.0));
}
__device__ __forceinline__ double pol_hi(const PolK &K, int i) {
  return i == 0 ? K.hi0 : (i == 1 ? K.hi1 : (i == 2 ? 3.14159265358979 : INFINITY));
}
// projection of variable i onto its bounds (a slack has only its lower
// bound); the same values as fmin(fmax(x, lo), hi) and fmax(x, 0)
__device__ __forceinline__ double pol_clamp(const PolK &K, int i, double x) {
  if (i < 3) {
    long long k = dkey(x);
    const long long kl = dkey(pol_lo(K, i)), kh = dkey(pol_hi(K, i));
    k = k < kl ? kl : k;
    k = k > kh ? kh : k;
    return dunkey(k);
  }
  return __double_as_longlong(x) > 0 ? x : 0.0;
}

// 2 x and x / 2 of a positive normal double (V_i, V_j: the voltage bounds
// are validated positive; rho_va) by one integer addition on the exponent
// field of its high word, off the FP64 pipe (exact)
__device__ __forceinline__ double twice_pos(double x) {
  return __hiloint2double(__double2hiint(x) + (1 << 20), __double2loint(x));
}
__device__ __forceinline__ double half_pos(double x) {
  return __hiloint2double(__double2hiint(x) - (1 << 20), __double2loint(x));
}

// cos d and sin d for |d| <= pi: d = k/256 + r with |r| <= 1/512 (+ 1e-6)
// (r exact), cos(k/256) and sin(k/256) from the table, cos r and sin r from
// their Taylor series to r^4 and r^3 (truncation below 2.5e-16 and 8e-20),
// then the angle-sum formulas.  About 10 FP64 operations against 25 for
// the library sincos.  k is the integer nearest to 256 d rounded from d's
// truncated FP32 copy (the 1.5 * 2^23 shift on the FP32 pipe; its value
// sits in the shifted sum's low mantissa bits), so no FP64 rounding or
// conversion runs; it can miss the nearest integer only where 256 d lies
// within 1e-4 of a half-integer, which |r| <= 1/512 + 1e-6 covers.  The
// index is clamped on the integer units, so every read is in bounds (a NaN
// angle gives NaN)
__device__ __forceinline__ void pol_cossin(double d, double &c, double &s) {
  const float sh = __fadd_rn(__fmul_rn(d2f_trunc(d), (float)TRIG_N), 12582912.0f);
  const float kf = __fsub_rn(sh, 12582912.0f);  // k itself (|k| <= 805 for |d| <= pi)
  int k = (int)(__float_as_uint(sh) & 0x7fffffu) - 0x400000;
  k = k < -TRIG_K ? -TRIG_K : (k > TRIG_K ? TRIG_K : k);
  const double r = fma(-f2d_exact(kf), 1.0 / TRIG_N, d);
  const double r2 = r * r;
  const double sr = fma(r * r2, -1.0 / 6.0, r);
  const double cr = fma(r2, fma(r2, 1.0 / 24.0, -0.5), 1.0);
  const double2 t = g_trig[k + TRIG_K];
  c = fma(t.x, cr, -(t.y * sr));
  s = fma(t.y, cr, t.x * sr);
}

// objective (and flows, cos/sin) at v.  Slacks in free_mask are first set
// to max(0, ht_k - g_k(x)), so that h_k takes its predicted value ht_k (the
// second-order correction of a trial step: without it the c/2 h_k^2 term
// sees the O(|dx|^2) remainder of g_k magnified by c)
__device__ __forceinline__ double pol_obj(const PolK &K, const PolP &P, double (&v)[POL_NV], double (&a)[4],
                                          double &c, double &s, const double (&ht)[2], int free_mask) {
  const double Vi = v[0], Vj = v[1], d = v[2];
  pol_cossin(d, c, s);
  const double Pv = Vi * Vj, Vi2 = Vi * Vi, Vj2 = Vj * Vj;
  double E[4], Ed[4], spe = 0.0;  // spe = sum_r rho_pq (a_r - t_r)^2
  pol_angle_terms(K.ga[0], K.ka[0], K.ga[1], K.ka[1], c, s, E, Ed);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = K.q[r] * (r < 2 ? Vi2 : Vj2) + Pv * E[r];
    const double e = a[r] - P.tg[r];
    spe = fma(P.rpq * e, e, spe);
  }
  const double ewi = Vi2 - P.tg[4], ewj = Vj2 - P.tg[5], et = d - P.tg[6];
  double f = 0.5 * spe + 0.5 * P.rva * (ewi * ewi + ewj * ewj) + 0.25 * P.rva * et * et;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double g = fma(a[2 * k], a[2 * k], fma(a[2 * k + 1], a[2 * k + 1], -K.rate2));
    if ((free_mask >> k) & 1) v[3 + k] = fmax(ht[k] - g, 0.0);
    const double h = g + v[3 + k];
    f += h * (P.mu[k] + 0.5 * P.c * h);
  }
  return f;
}

// objective, reduced x-gradient gx (FP64; the slack terms m_k grad g_k are
// left out -- pol_iter adds them where a slack is held at its bound) and the
// x-Hessian without the c grad grad^T terms (FP32 Hf, or FP64 Hd when a slack
// is held at zero) at v; fills L.  The gradients come from sums over the
// rows, with grad a_r = (2 q_r V_i [r < 2] + V_j E_r, V_i E_r + 2 q_r V_j
// [r >= 2], V_i V_j Ed_r):
//   gx = (2 V_i (pe_0 q_0 + pe_1 q_1) + V_j sum pe_r E_r,
//         2 V_j (pe_2 q_2 + pe_3 q_3) + V_i sum pe_r E_r, V_i V_j sum pe_r Ed_r)
//        + (angle/voltage rows), pe_r = rho_pq (a_r - t_r);
//   grad g_0 = (4 V_i A_q + 2 V_j A_E, 2 V_i A_E, 2 V_i V_j A_Ed) and
//   grad g_1 = (2 V_j A_E, 4 V_j A_q + 2 V_i A_E, 2 V_i V_j A_Ed) with the
//   end's sums A_E = sum a_r E_r, A_Ed = sum a_r Ed_r, A_q = sum a_r q_r.
// With m_k = mu_k + c h_k the x-Hessian is
//   sum_r (w_r grad a_r grad a_r^T + u_r hess a_r) + (angle/voltage rows)
//   + sum_k c grad g_k grad g_k^T,
// w_r = rho_pq + 2 m_k, u_r = rho_pq (a_r - t_r) + 2 m_k a_r (k = r / 2).
__device__ __forceinline__ void pol_full(const PolK &K, const PolP &P, double (&v)[POL_NV], double (&gx)[3],
                                         float (&Hf)[6], double (&Hd)[6], PolLast &L, const double (&ht)[2],
                                         int free_mask) {
  const double Vi = v[0], Vj = v[1], d = v[2];
  double s, c;
  pol_cossin(d, c, s);
  L.c = c;
  L.s = s;
#pragma unroll
  for (int i = 0; i < POL_NV; ++i) L.v[i] = v[i];
  const double Pv = Vi * Vj, Vi2 = Vi * Vi, Vj2 = Vj * Vj;
  // (the FP32 copies are truncated on the integer units: d2f_trunc)
  const float fVi = d2f_trunc(Vi), fVj = d2f_trunc(Vj), fP = fVi * fVj;
  const double Vi2x = twice_pos(Vi), Vj2x = twice_pos(Vj);
  double E[4], Ed[4], pe[4];
  float fE[4], fEd[4];
  // FP32 gradient of the flow (for the FP32 Hessian and the first-order
  // finish) from FP32 cos/sin and constants: two conversions per
  // evaluation, the products on the FP32 pipe
  const float fc = d2f_trunc(c), fs = d2f_trunc(s);
  pol_angle_terms(K.ga[0], K.ka[0], K.ga[1], K.ka[1], c, s, E, Ed);
  pol_angle_terms(K.fga(0), K.fka(0), K.fga(1), K.fka(1), fc, fs, fE, fEd);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const double a = K.q[r] * (r < 2 ? Vi2 : Vj2) + Pv * E[r];
    L.a[r] = a;
    pe[r] = P.rpq * (a - P.tg[r]);
    L.da[r][0] = r < 2 ? 2.0f * K.fq(r) * fVi + fVj * fE[r] : fVj * fE[r];
    L.da[r][1] = r < 2 ? fVi * fE[r] : 2.0f * K.fq(r) * fVj + fVi * fE[r];
    L.da[r][2] = fP * fEd[r];
  }
  const double ewi = Vi2 - P.tg[4], ewj = Vj2 - P.tg[5], et = d - P.tg[6];
  double mhk[2];
  bool lim = false;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r0 = 2 * k, r1 = 2 * k + 1;
    // (two FMAs: the square of the end's q-row flow enters with -rate^2)
    const double g = fma(L.a[r0], L.a[r0], fma(L.a[r1], L.a[r1], -K.rate2));
    if ((free_mask >> k) & 1) {  // second-order correction of a trial point (see pol_obj)
      v[3 + k] = fmax(ht[k] - g, 0.0);
      L.v[3 + k] = v[3 + k];
    }
    const double sk = v[3 + k];
    const double h = g + sk;
    const double m = P.mu[k] + P.c * h;
    L.m[k] = m;
    L.h[k] = h;
    // grad g_k = 2 sum_r a_r grad a_r over the end's two rows, in FP32 from
    // the FP32 flow gradients
    const float fa0 = d2f_trunc(L.a[r0]), fa1 = d2f_trunc(L.a[r1]);
#pragma unroll
    for (int i = 0; i < 3; ++i) L.fdg[k][i] = 2.0f * (fa0 * L.da[r0][i] + fa1 * L.da[r1][i]);
    // a free slack's optimum has m_k = 0, so the Newton model takes the
    // reduced x-Hessian there; m_k hess g_k stays only for a slack that may
    // be held at zero
    // (sk >= 0: compared on its bit pattern, on the integer units)
    const bool held = __double_as_longlong(sk) <= __double_as_longlong(1e-6) && __double_as_longlong(m) > 0;
    mhk[k] = held ? m : 0.0;
    lim = lim || held;
  }
  {
    double SE = pe[0] * E[0], SEd = pe[0] * Ed[0];
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      SE = fma(pe[r], E[r], SE);
      SEd = fma(pe[r], Ed[r], SEd);
    }
    const double Sq0 = fma(pe[0], K.q[0], pe[1] * K.q[1]), Sq1 = fma(pe[2], K.q[2], pe[3] * K.q[3]);
    // (2 V_i Sq0 + 2 rho_va (V_i^2 - t_4) V_i as 2 V_i (Sq0 + rho_va (V_i^2 - t_4)))
    gx[0] = fma(Vi2x, fma(P.rva, ewi, Sq0), Vj * SE);
    gx[1] = fma(Vj2x, fma(P.rva, ewj, Sq1), Vi * SE);
    gx[2] = fma(Pv, SEd, half_pos(P.rva) * et);
  }
  // (UCAC_POL_FP64_NEWTON = 1 builds the all-FP64 Hessian and Newton system
  // on every lane, the same model: the A/B reference of the precision split)
  lim = lim || UCAC_POL_FP64_NEWTON;
  L.lim = lim;
  // packed symmetric index: 0:(0,0) 1:(0,1) 2:(0,2) 3:(1,1) 4:(1,2) 5:(2,2)
  const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
  if (!lim) {
    // no slack held: the row weights are w_r = rho_pq, u_r = rho_pq (a_r - t_r)
    const float rva = P.frva, fw = P.frpq;
#pragma unroll
    for (int q = 0; q < 6; ++q) Hf[q] = 0.0f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float fu = d2f_trunc(pe[r]);
      const float d2[6] = {r < 2 ? 2.0f * K.fq(r) : 0.0f, fE[r], fVj * fEd[r], r < 2 ? 0.0f : 2.0f * K.fq(r),
                           fVi * fEd[r], -fP * fE[r]};
#pragma unroll
      for (int q = 0; q < 6; ++q) Hf[q] += fw * L.da[r][pi_[q]] * L.da[r][pj_[q]] + fu * d2[q];
    }
    Hf[0] += rva * (4.0f * fVi * fVi + 2.0f * d2f_trunc(ewi));
    Hf[3] += rva * (4.0f * fVj * fVj + 2.0f * d2f_trunc(ewj));
    Hf[5] += 0.5f * rva;
  } else {
    double w[4], u[4], da[4][3];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double mh = mhk[r >> 1];
      w[r] = P.rpq + 2.0 * mh;
      u[r] = pe[r] + 2.0 * mh * L.a[r];
      da[r][0] = r < 2 ? fma(K.q[r], Vi2x, Vj * E[r]) : Vj * E[r];
      da[r][1] = r < 2 ? Vi * E[r] : fma(K.q[r], Vj2x, Vi * E[r]);
      da[r][2] = Pv * Ed[r];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) Hd[q] = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const double d2[6] = {r < 2 ? 2.0 * K.q[r] : 0.0, E[r], Vj * Ed[r], r < 2 ? 0.0 : 2.0 * K.q[r], Vi * Ed[r],
                            -Pv * E[r]};
#pragma unroll
      for (int q = 0; q < 6; ++q) Hd[q] += w[r] * da[r][pi_[q]] * da[r][pj_[q]] + u[r] * d2[q];
    }
    Hd[0] += P.rva * (4.0 * Vi * Vi + 2.0 * ewi);
    Hd[3] += P.rva * (4.0 * Vj * Vj + 2.0 * ewj);
    Hd[5] += 0.5 * P.rva;
  }
}

// FP64 gradients of the limit functions at the last evaluation point:
//   grad g_0 = (4 V_i A_q + 2 V_j A_E, 2 V_i A_E, 2 V_i V_j A_Ed),
//   grad g_1 = (2 V_j A_E, 4 V_j A_q + 2 V_i A_E, 2 V_i V_j A_Ed),
// with the end's sums A_E = sum a_r E_r, A_Ed = sum a_r Ed_r, A_q = sum a_r q_r
__device__ __forceinline__ void pol_dg64(const PolK &K, const PolLast &L, double (&dg)[2][3]) {
  const double Vi = L.v[0], Vj = L.v[1];
  const double Pv = Vi * Vj, Vi2x = 2.0 * Vi, Vj2x = 2.0 * Vj;
  double E[4], Ed[4];
  pol_angle_terms(K.ga[0], K.ka[0], K.ga[1], K.ka[1], L.c, L.s, E, Ed);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r0 = 2 * k, r1 = 2 * k + 1;
    const double AE = fma(L.a[r0], E[r0], L.a[r1] * E[r1]);
    const double AEd = fma(L.a[r0], Ed[r0], L.a[r1] * Ed[r1]);
    const double Aq = fma(L.a[r0], K.q[r0], L.a[r1] * K.q[r1]);
    if (k == 0) {
      dg[0][0] = fma(2.0 * Vi2x, Aq, Vj2x * AE);
      dg[0][1] = Vi2x * AE;
    } else {
      dg[1][0] = Vj2x * AE;
      dg[1][1] = fma(2.0 * Vj2x, Aq, Vi2x * AE);
    }
    dg[k][2] = 2.0 * Pv * AEd;
  }
}

// objective at the point of the last evaluation, from its flows and h_k
// (formed only where a ratio test needs it: a trial step, a held slack's step)
__device__ __forceinline__ double pol_f(const PolP &P, const PolLast &L) {
  double spe = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const double e = L.a[r] - P.tg[r];
    spe = fma(P.rpq * e, e, spe);
  }
  const double ewi = L.v[0] * L.v[0] - P.tg[4], ewj = L.v[1] * L.v[1] - P.tg[5];
  const double et = L.v[2] - P.tg[6];
  double f = 0.5 * spe + 0.5 * P.rva * (ewi * ewi + ewj * ewj) + 0.25 * P.rva * et * et;
#pragma unroll
  for (int k = 0; k < 2; ++k) f += L.h[k] * (P.mu[k] + 0.5 * P.c * L.h[k]);
  return f;
}

// a pivot's square root L = sqrt(s) and its reciprocal 1/L; in FP32 both
// from the hardware reciprocal square root (2 ulp: far below the FP32
// Newton system's own error), in FP64 exact
__device__ __forceinline__ void piv_root(float s, float &L, float &iL) {
  iL = rsqrtf(s);
  L = s * iL;
}
__device__ __forceinline__ void piv_root(double s, double &L, double &iL) {
  L = sqrt(s);
  iL = 1.0 / L;
}

// masked 3x3 Cholesky solve (packed symmetric A), T = float or double
template <typename T>
__device__ __forceinline__ bool chol3p(const T (&A)[6], T (&b)[3]) {
  const T s0 = A[0];
  if (!(s0 > T(0))) return false;
  T L00, i0;
  piv_root(s0, L00, i0);
  const T L10 = A[1] * i0, L20 = A[2] * i0;
  const T s1 = A[3] - L10 * L10;
  if (!(s1 > T(0))) return false;
  T L11, i1;
  piv_root(s1, L11, i1);
  const T L21 = (A[4] - L20 * L10) * i1;
  const T s2 = A[5] - L20 * L20 - L21 * L21;
  if (!(s2 > T(0))) return false;
  T L22, i2;
  piv_root(s2, L22, i2);
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


// A pending trial point: evaluated in full at the next trip, then accepted or
// rejected by the ratio test against the model decrease pred.  The record is
// read only on the trial path, so it lives in shared memory, one column per
// lane (field f of a lane's record at rec[32 f]): the point, the predicted
// h_k, pred, the step's scale and its largest x component.
enum { TR_V = 0, TR_HT = 5, TR_PRED = 7, TR_SCALE = 8, TR_SMAX = 9, TR_N = 10 };
enum { NI_TRIAL = 3, NI_FULL = 4 };

// The common Newton iteration of a lane with no slack held at zero (FP32
// Hessian H): no variable within 1e-6 of a bound, the unshifted system
// factorises, no variable is pushed across a bound it sits at, and the step
// is the stop step or lies in the box and the trust region.  Its arithmetic
// is that of pol_iter in this case, except that the free slacks' step takes
// grad g_k . d_x from the FP32 gradients (the slacks do not enter the
// reduced x-system, so the x iterates are the same).  Any other case
// returns NI_FULL with nothing written, and the caller runs pol_iter, which
// forms grad g_k in FP64.
__device__ __forceinline__ int pol_fast(const PolK &K, const PolP &P, double (&v)[POL_NV], const double (&gx)[3],
                                        const PolLast &L, const float (&H)[6], double Delta, double omega,
                                        bool &accepted, int &counted) {
  const long long b6 = __double_as_longlong(1e-6), ABS = 0x7fffffffffffffffLL;
  long long bx = 0;
  // near-bound prefilter (a variable within 1e-6 of a bound hands the step
  // to pol_iter): for V_i, V_j and d in FP32 from truncated copies, whose
  // difference is within two FP32 ulps (< 5e-7 for |x| < 4) of the exact
  // distance, so the 1.5e-6 test is conservative; for a slack its value is
  // its distance (compared on the bit patterns).  With omega < 1e-6 a
  // variable beyond that margin cannot meet the stationarity test through
  // its bound distance, so no FP64 bound distance is formed here
  bool edge = __double_as_longlong(omega) >= b6;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long b = __double_as_longlong(v[i]) & ABS;
    bx = b > bx ? b : bx;
    const float fv = d2f_trunc(v[i]);
    const float flo = i < 2 ? K.flo(i) : -3.14159265f, fhi = i < 2 ? K.fhi(i) : 3.14159265f;
    edge = edge || (fv - flo <= 1.5e-6f) || (fhi - fv <= 1.5e-6f);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
    edge = edge || (__double_as_longlong(v[3 + k]) <= b6 && __double_as_longlong(L.m[k]) > 0);
  if (edge) return NI_FULL;
  const double xmax = __longlong_as_double(bx);
  // stationarity on the reduced gradient, the free slacks' exact step
  bool stat = true;
  const long long bom = __double_as_longlong(omega);
#pragma unroll
  for (int i = 0; i < 3; ++i) stat = stat && (__double_as_longlong(gx[i]) & ABS) <= bom;
  double sn[2];
  bool sok = true;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    sn[k] = v[3 + k] - L.m[k] * P.ic;
    const long long b = __double_as_longlong(sn[k]);
    sok = sok && (b >= 0 || b == (long long)0x8000000000000000ULL);
  }
  accepted = false;
  counted = 0;
  if (stat && sok) {
    v[3] = sn[0];
    v[4] = sn[1];
    return NI_CONV;
  }
  float y[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = to_t<float>(-gx[i]);
  if (!chol3p(H, y)) return NI_FULL;
  double d[POL_NV];
  long long bn = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    d[i] = to_d<float>(y[i]);
    const long long b = __double_as_longlong(d[i]) & ABS;
    bn = b > bn ? b : bn;
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float gd = L.fdg[k][0] * y[0] + L.fdg[k][1] * y[1] + L.fdg[k][2] * y[2];
    d[3 + k] = -L.m[k] * P.ic - f2d_exact(gd);
  }
  // the second pass of pol_iter: no x variable sits within 1e-6 of a bound
  // here, but a slack may (with m_k <= 0); one that the step pushes below
  // zero is fixed there by pol_iter
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (le_nn(v[3 + k], 1e-6) && dkey(d[3 + k]) < dkey(-v[3 + k])) return NI_FULL;
  double vn[POL_NV];
#pragma unroll
  for (int i = 0; i < POL_NV; ++i) vn[i] = v[i] + d[i];
  // the step thresholds 1e-9 (1 + |x|) and 1e-3 (1 + |x|) in FP32 (a step
  // within ~1e-7 relative of one is decided either way)
  const float fx1 = 1.0f + d2f_trunc(xmax);
  const double dn = __longlong_as_double(bn);
  if (le_nn(dn, f2d_exact(1e-9f * fx1))) {
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) v[i] = pol_clamp(K, i, vn[i]);
    counted = 1;
    return NI_CONV;
  }
  // the new point in the box, tested on the integer units (dkey order)
  bool inside = __double_as_longlong(vn[3]) >= 0 && __double_as_longlong(vn[4]) >= 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long kv = dkey(vn[i]);
    inside = inside && kv >= dkey(pol_lo(K, i)) && kv <= dkey(pol_hi(K, i));
  }
  if (inside && le_nn(dn, f2d_exact(1e-3f * fx1)) && le_nn(dn, Delta)) {
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) v[i] = pol_clamp(K, i, vn[i]);
    counted = 1;
    accepted = true;
    return NI_CONT;
  }
  return NI_FULL;
}

// one projected Newton iteration over v = (V_i, V_j, d, sigma_ij, sigma_ji)
// with the x-Hessian H of type T (see newton_iter of the W-form kernel for
// the steps); free slacks are eliminated from the Newton system exactly
template <typename T>
__device__ __forceinline__ int pol_iter(const PolK &K, const PolP &P, double (&v)[POL_NV], double &f,
                                        const double (&gx)[3], const PolLast &L, const T (&H)[6], double &Delta,
                                        double omega, bool &accepted, int &counted, double *trp,
                                        bool &nearb) {
  accepted = false;
  counted = 0;
  const double c = P.c;
  // gx is the reduced x-gradient; the full gradient gr over v adds
  // m_k grad g_k to it -- formed only near a bound and for the model of a
  // trust-region step
  double gr[POL_NV];
  gr[3] = L.m[0];
  gr[4] = L.m[1];
  // FP64 grad g_k (this is the path of the solves pol_fast hands over: a
  // variable near a bound, a held slack, a shifted or second-pass system,
  // a trust-region step)
  double dg[2][3];
  pol_dg64(K, L, dg);
  auto full_grad = [&]() {
#pragma unroll
    for (int i = 0; i < 3; ++i) gr[i] = fma(L.m[0], dg[0][i], fma(L.m[1], dg[1][i], gx[i]));
  };
  double xmax = 0.0, dlo[POL_NV], dhi[POL_NV];
  T hmax = T(0);
  // a variable can only be epsilon-active within 1e-6 of a bound (epsilon
  // <= 1e-6), so the epsilon estimate is skipped when none is that close.
  // v lies in its box, so dlo, dhi >= 0 and their order is the signed order
  // of their bit patterns: the test runs on the integer units (a negative
  // or NaN operand can only make it pass, which is the safe side)
  bool near = false, prox = false;  // prox: an x variable within 1e-6 of a bound
  const long long b6 = __double_as_longlong(1e-6), ABS = 0x7fffffffffffffffLL;
  long long bx = 0;
#pragma unroll
  for (int i = 0; i < POL_NV; ++i) {
    dlo[i] = v[i] - pol_lo(K, i);
    dhi[i] = i < 3 ? pol_hi(K, i) - v[i] : INFINITY;  // a slack has no upper bound
    if (i < 3) {
      const long long b = __double_as_longlong(v[i]) & ABS;
      bx = b > bx ? b : bx;
      const T h = hq(H, i, i);
      hmax = hmax > h ? hmax : h;
      prox = prox || __double_as_longlong(dlo[i]) <= b6 || __double_as_longlong(dhi[i]) <= b6;
    } else {
      near = near || (__double_as_longlong(dlo[i]) <= b6 && __double_as_longlong(gr[i]) > 0);
    }
  }
  xmax = __longlong_as_double(bx);  // max |x_i| (order of non-negative doubles = order of their bits)
  nearb = prox || near;
  if (prox) {
    full_grad();
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const long long bg = __double_as_longlong(gr[i]);
      near = near || (__double_as_longlong(dlo[i]) <= b6 && bg > 0) || (__double_as_longlong(dhi[i]) <= b6 && bg < 0);
    }
  }
  bool act[POL_NV];
  double d[POL_NV];
#pragma unroll
  for (int i = 0; i < POL_NV; ++i) {
    act[i] = false;
    d[i] = 0.0;
  }
  if (near) {
    if (!prox) full_grad();
    // epsilon: largest clamped diagonal Newton step, in T
    T epst = T(0);
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) {
      T di;
      if (i < 3) {
        const T h = hq(H, i, i);
        di = (h > T(0)) ? (T)gr[i] / h : (T)gr[i];
      } else {
        di = (T)(gr[i] * P.ic);
      }
      const T st = (-di < (T)-dlo[i]) ? (T)-dlo[i] : ((-di > (T)dhi[i]) ? (T)dhi[i] : -di);
      const T ast = st < T(0) ? -st : st;
      epst = epst > ast ? epst : ast;
    }
    const double eps = fmin((double)epst, 1e-6);
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) {
      if (dlo[i] <= eps && gr[i] > 0.0) {
        act[i] = true;
        d[i] = -dlo[i] * 1.000001;  // onto the bound (clamped below)
      } else if (dhi[i] <= eps && gr[i] < 0.0) {
        act[i] = true;
        d[i] = dhi[i] * 1.000001;
      }
    }
  }
  // stationarity on the reduced gradient (free slacks eliminated: their
  // m_k grad g_k leaves the x-gradient); at a stationary x each free slack
  // takes its exact step -m_k / c (the objective is quadratic in it) -- m_k
  // itself carries c times the rounding of h_k and never reaches omega
  // (|P(v - g) - v| <= omega holds when |g| <= omega or the bound that -g
  // points at is within omega)
  // (compares of non-negative doubles on their bit patterns, as above)
  double rg[3];
  bool stat = true;
  const long long bom = __double_as_longlong(omega);
#pragma unroll
  for (int i = 0; i < 3; ++i) rg[i] = gx[i];
  if (near) {  // a slack held at its bound keeps its m_k grad g_k
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (act[3 + k]) rg[i] = fma(L.m[k], dg[k][i], rg[i]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const long long br = __double_as_longlong(rg[i]);
    const long long bd = __double_as_longlong(br > 0 ? dlo[i] : dhi[i]);
    stat = stat && ((br & ABS) <= bom || bd <= bom);
  }
  double sn[2];
  bool sok = true;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    sn[k] = v[3 + k];
    if (act[3 + k]) {
      stat = stat && fabs(clampd(v[3 + k] - L.m[k], 0.0, INFINITY) - v[3 + k]) <= omega;
    } else {
      sn[k] = v[3 + k] - L.m[k] * P.ic;
      const long long b = __double_as_longlong(sn[k]);
      sok = sok && (b >= 0 || b == (long long)0x8000000000000000ULL);  // sn >= 0 (-0 included)
    }
  }
  if (stat && sok) {
    v[3] = sn[0];
    v[4] = sn[1];
    return NI_CONV;
  }
  // 3x3 system in x: H plus c grad g_k grad g_k^T of the slacks held at a
  // bound; a free slack's row gives d_sigma_k = -m_k / c - grad g_k . d_x,
  // which turns its m_k grad g_k out of the right-hand side.  Second pass: a
  // free variable that sits at a bound (within 1e-6) and that the Newton step
  // pushes across it is fixed there, and the system is solved again on the
  // rest -- the gradient-based active set misses such a variable when the
  // coupling to the others, not its own gradient, drives it outward, and the
  // projected step would then not be a descent direction of the model
  const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
  long long bn = 0;
  T lm = T(0);
  for (int pass = 0;; ++pass) {
    T Hr[6], rb[3];
    const bool sheld = act[3] || act[4];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      Hr[q] = H[q];
      if (sheld) {
        double add = 0.0;
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (act[3 + k]) add += c * dg[k][pi_[q]] * dg[k][pj_[q]];
        Hr[q] += (T)add;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double r = -rg[i];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (act[3 + k]) r -= c * dg[k][i] * d[3 + k];
      rb[i] = to_t<T>(r);
    }
    T y[3];
    lm = T(0);
    bool ok = false;
    for (int tries = 0; tries < 40; ++tries) {
      T A[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int i = pi_[q], j = pj_[q];
        A[q] = (act[i] || act[j]) ? ((i == j) ? T(1) : T(0)) : Hr[q];
        if (i == j && !act[i]) A[q] += lm;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        T r = rb[i];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          if (act[j]) r -= hq(Hr, i, j) * (T)d[j];
        y[i] = act[i] ? (T)d[i] : r;
      }
      if (chol3p(A, y)) {
        ok = true;
        break;
      }
      lm = (lm == T(0)) ? T(1e-10) * (hmax > T(0) ? hmax : T(1)) : T(10) * lm;
    }
    if (!ok) return NI_STOP;
    bn = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (!act[i]) d[i] = to_d<T>(y[i]);
      const long long b = __double_as_longlong(d[i]) & ABS;
      bn = b > bn ? b : bn;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (!act[3 + k]) d[3 + k] = -L.m[k] * P.ic - (dg[k][0] * d[0] + dg[k][1] * d[1] + dg[k][2] * d[2]);
    if (pass > 0) break;
    bool again = false;
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) {
      if (act[i]) continue;
      const bool lo_at = le_nn(dlo[i], 1e-6) && dkey(d[i]) < dkey(-dlo[i]);
      const bool hi_at = le_nn(dhi[i], 1e-6) && dkey(d[i]) > dkey(dhi[i]);
      if (lo_at || hi_at) {
        act[i] = true;
        d[i] = lo_at ? -dlo[i] * 1.000001 : dhi[i] * 1.000001;  // onto the bound (clamped below)
        again = true;
        if (i >= 3) {  // a held slack keeps its m_k grad g_k in the reduced gradient
#pragma unroll
          for (int j = 0; j < 3; ++j) rg[j] = fma(L.m[i - 3], dg[i - 3][j], rg[j]);
        }
      }
    }
    if (!again) break;
    if (!near) {  // the model of the step now needs the full gradient
      if (!prox) full_grad();
      near = true;
    }
  }
  const double dn = __longlong_as_double(bn);  // max |d_i| over x
  counted = 1;
  // model decrease of a step sg: -(gr . sg + 1/2 sg^T H5 sg), where
  // sg^T H5 sg = sx^T H sx + sum_k c (grad g_k . sx + s_sigma_k)^2
  auto model = [&](const double (&sg)[POL_NV]) -> double {
    double lin = 0.0;
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) lin += gr[i] * sg[i];
    const T s0 = (T)sg[0], s1 = (T)sg[1], s2 = (T)sg[2];
    const T sHs = s0 * (H[0] * s0 + H[1] * s1 + H[2] * s2) + s1 * (H[1] * s0 + H[3] * s1 + H[4] * s2) +
                  s2 * (H[2] * s0 + H[4] * s1 + H[5] * s2);
    double quad = (double)sHs;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double e = dg[k][0] * sg[0] + dg[k][1] * sg[1] + dg[k][2] * sg[2] + sg[3 + k];
      quad += c * e * e;
    }
    return -(lin + 0.5 * quad);
  };
  if (lm == T(0)) {
    if (le_nn(dn, 1e-9 * (1.0 + xmax))) {
#pragma unroll
      for (int i = 0; i < POL_NV; ++i) v[i] = pol_clamp(K, i, v[i] + d[i]);
      return NI_CONV;
    }
    // d_i in [-dlo_i, dhi_i] with dlo, dhi >= 0: a negative d_i against dlo_i
    // by magnitude, a non-negative one against dhi_i (bit-pattern compares)
    bool inside = true;
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) {
      const long long b = __double_as_longlong(d[i]);
      const bool in = b < 0 ? (b & ABS) <= __double_as_longlong(dlo[i]) : b <= __double_as_longlong(dhi[i]);
      inside = inside && (act[i] || in);
    }
    if (inside && le_nn(dn, 1e-3 * (1.0 + xmax)) && le_nn(dn, Delta)) {
#pragma unroll
      for (int i = 0; i < POL_NV; ++i) v[i] = pol_clamp(K, i, v[i] + d[i]);
      accepted = true;
      return NI_CONT;
    }
  }
  const double scale = le_nn(dn, Delta) ? 1.0 : Delta / dn;
  double vt[POL_NV], sg[POL_NV], smax = 0.0;
#pragma unroll
  for (int i = 0; i < POL_NV; ++i) {
    vt[i] = pol_clamp(K, i, v[i] + scale * d[i]);
    sg[i] = vt[i] - v[i];
    if (i < 3) smax = fmax(smax, fabs(sg[i]));
  }
  full_grad();
  const double pred = model(sg);
  // predicted h_k of the trial step; free slacks absorb the remainder of
  // g_k exactly, a slack held at zero gets the correction
  // dx = -sum_k alpha_k grad g_k (Gram system of the held gradients) that
  // restores the linear prediction of its g_k to second order
  double ht[2];
  int free_mask = 0, nheld = 0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    ht[k] = L.h[k] + dg[k][0] * sg[0] + dg[k][1] * sg[1] + dg[k][2] * sg[2] + sg[3 + k];
    if (act[3 + k]) ++nheld; else free_mask |= 1 << k;
  }
  f = pol_f(P, L);  // the ratio test's baseline: the objective at v
  if (nheld == 0) {
    // the trial point becomes the next trip's evaluation point: every lane
    // of the warp then runs one full evaluation per trip, and the ratio test
    // follows it (a rejection re-evaluates the current point)
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) trp[32 * (TR_V + i)] = vt[i];
    trp[32 * TR_HT] = ht[0];
    trp[32 * (TR_HT + 1)] = ht[1];
    trp[32 * TR_PRED] = pred;
    trp[32 * TR_SCALE] = scale;
    trp[32 * TR_SMAX] = smax;
    return NI_TRIAL;
  }
  double at[4], ct, stn;
  double ft = pol_obj(K, P, vt, at, ct, stn, ht, free_mask);
  {
    double r[2], G[3];
#pragma unroll
    for (int k = 0; k < 2; ++k)
      r[k] = act[3 + k] ? (at[2 * k] * at[2 * k] + at[2 * k + 1] * at[2 * k + 1] - K.rate2 + vt[3 + k]) - ht[k] : 0.0;
    G[0] = dg[0][0] * dg[0][0] + dg[0][1] * dg[0][1] + dg[0][2] * dg[0][2];
    G[1] = dg[0][0] * dg[1][0] + dg[0][1] * dg[1][1] + dg[0][2] * dg[1][2];
    G[2] = dg[1][0] * dg[1][0] + dg[1][1] * dg[1][1] + dg[1][2] * dg[1][2];
    double al0 = 0.0, al1 = 0.0;
    if (nheld == 2) {
      const double det = G[0] * G[2] - G[1] * G[1];
      if (det > 1e-12 * G[0] * G[2]) {
        al0 = (G[2] * r[0] - G[1] * r[1]) / det;
        al1 = (G[0] * r[1] - G[1] * r[0]) / det;
      }
    } else if (act[3]) {
      al0 = G[0] > 0.0 ? r[0] / G[0] : 0.0;
    } else {
      al1 = G[2] > 0.0 ? r[1] / G[2] : 0.0;
    }
    double vc[POL_NV];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      vc[i] = clampd(vt[i] - al0 * dg[0][i] - al1 * dg[1][i], pol_lo(K, i), pol_hi(K, i));
    vc[3] = vt[3];
    vc[4] = vt[4];
    double ac[4], cc, sc;
    const double fc = pol_obj(K, P, vc, ac, cc, sc, ht, free_mask);
    if (fc < ft) {
      ft = fc;
#pragma unroll
      for (int i = 0; i < POL_NV; ++i) vt[i] = vc[i];
    }
  }
  const double ared = f - ft;
  if (pred > 0.0 && ared >= 1e-4 * pred) {
#pragma unroll
    for (int i = 0; i < POL_NV; ++i) v[i] = vt[i];
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

// starting point of line-period `it`: V_i, V_j and 1 / c from the kernel's
// own copy (the last solve's values, or sqrt(w) clamped to the voltage band
// after create or import), d = theta_i - theta_j of the stored iterate
// clamped to [-pi, pi], and the slacks projected onto sigma >= 0
__device__ __forceinline__ void pol_start(const Dev &S, long long it, double (&v)[POL_NV], double &ic) {
  const long long NBP = S.NBP;
  v[0] = S.LV[it];
  v[1] = S.LV[NBP + it];
  ic = S.LV[2 * NBP + it];
  // (the clamps on the integer units: dkey order, as in pol_clamp; a NaN's
  // key lies beyond both infinities, so a NaN angle difference starts at
  // -pi or pi by the sign of its pattern)
  long long kd = dkey(S.B[(FB_V0 + 4) * NBP + it] - S.B[(FB_V0 + 5) * NBP + it]);
  const long long kl = dkey(-3.14159265358979), kh = dkey(3.14159265358979);
  kd = kd < kl ? kl : (kd > kh ? kh : kd);
  v[2] = dunkey(kd);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    // positive patterns up to +inf pass, everything else (negative values,
    // -0, any NaN) starts at 0: the same values as fmax(sigma, 0)
    const double sk = S.B[(FB_V0 + 6 + k) * NBP + it];
    const long long b = __double_as_longlong(sk);
    v[3 + k] = (b > 0 && b <= 0x7ff0000000000000LL) ? sk : 0.0;
  }
}

// Finish ring: a lane whose solve is done records what the outputs need
// (flows, FP32 flow gradients and the last step for the first-order update,
// cos/sin, V_i, V_j, d, the angle targets, item and slots) and the warp
// writes the outputs of 32 records at a time with every lane active.  Per
// warp POL_QF records in dynamic shared memory, laid out for all warps of
// the block as doubles [warp][12][QF], floats [warp][15][QF], ints
// [warp][3][QF]; the record fields:
//   doubles 0-3 flows a_r, 4 cos, 5 sin, 6 V_i, 7 V_j, 8 d, 9 step in d,
//     10 the angle targets' mean (t_6 + t_7) / 2, 11 1 / c
//   floats 0-11 grad a_r (FP32, r * 3 + i), 12-14 the step in x (FP32)
//   ints 0 item, 1-2 slots of the from / to end
constexpr int POL_QF = 64;
constexpr int POL_FD = 12, POL_FF = 15, POL_FI = 3;
__host__ __device__ constexpr size_t pol_dyn_smem(int bs) {
  return (size_t)(bs / 32) * POL_QF * (POL_FD * sizeof(double) + POL_FF * sizeof(float) + POL_FI * sizeof(int));
}

// outputs of finish record sl: flows to first order after the final step,
// the W-form iterate (w_i, w_j, wR, wI, theta_i, theta_j) and the line-end
// rows (the slacks, multipliers and penalty are written by the lane itself)
__device__ __forceinline__ void pol_finish_out(const Dev &S, const double *fd, const float *ff, const int *fi,
                                               int sl, unsigned G) {
  const long long NBP = S.NBP, NEP = S.NEP;
  const unsigned fw = (unsigned)fi[sl];
  const long long bp = fw & 0x7fffffffu, lef = fi[POL_QF + sl], let = fi[2 * POL_QF + sl];
  // a flagged solve (see k_line_polar) gets this sweep's mark and joins the
  // next sweep's list (one atomic per warp and flush)
  const bool hard = (fw >> 31) != 0u;
  {
    const unsigned am = __activemask(), hm = __ballot_sync(am, hard);
    if (hm) {
      const int lane = threadIdx.x & 31, leader = __ffs(hm) - 1, nxt = (int)((G + 1u) & 1u);
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&S.pctl[1 + nxt], (unsigned long long)__popc(hm));
      base = __shfl_sync(am, base, leader);
      if (hard) {
        S.pgen[bp] = G + 2u;
        S.plist[(long long)nxt * NBP + (long long)base + __popc(hm & ((1u << lane) - 1u))] = (int)bp;
      }
    }
  }
  const float fx0 = ff[12 * POL_QF + sl], fx1 = ff[13 * POL_QF + sl], fx2 = ff[14 * POL_QF + sl];
  double a[4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
    a[r] = fd[r * POL_QF + sl] + f2d_exact(ff[(3 * r) * POL_QF + sl] * fx0 + ff[(3 * r + 1) * POL_QF + sl] * fx1 +
                                           ff[(3 * r + 2) * POL_QF + sl] * fx2);
  const double c0 = fd[4 * POL_QF + sl], s0 = fd[5 * POL_QF + sl], dx2 = fd[9 * POL_QF + sl];
  const double c = c0 - s0 * dx2, sn = s0 + c0 * dx2;
  const double Vi = fd[6 * POL_QF + sl], Vj = fd[7 * POL_QF + sl], d = fd[8 * POL_QF + sl];
  const double Pv = Vi * Vj, tm = fd[10 * POL_QF + sl];
  const double v6[6] = {Vi * Vi, Vj * Vj, Pv * c, Pv * sn, tm + 0.5 * d, tm - 0.5 * d};
#pragma unroll
  for (int i = 0; i < 6; ++i) S.B[(FB_V0 + i) * NBP + bp] = v6[i];
  S.LV[bp] = Vi;
  S.LV[NBP + bp] = Vj;
  S.LV[2 * NBP + bp] = fd[11 * POL_QF + sl];
#pragma unroll
  for (int r = 0; r < 4; ++r) S.EA[erow_u(r) * NEP + (erow_end(r) ? let : lef)] = a[r];
  S.EA[2 * NEP + lef] = v6[0];
  S.EA[2 * NEP + let] = v6[1];
  S.EA[3 * NEP + lef] = v6[4];
  S.EA[3 * NEP + let] = v6[5];
}

template <int BS>
__global__ void __launch_bounds__(BS) k_line_polar(Dev S) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  __shared__ float kf[12][BS];  // FP32 copies of the lane's line constants and voltage bounds
  // Per-warp ring of prepared starts (item, instance, v, 1 / c).  Lanes that
  // finish a solve take their next item from the ring; when it runs short,
  // the warp fetches 32 items at once and all 32 lanes prepare one each, so
  // the start's square roots and division run with every lane active
  // instead of with the ~1/3 of the lanes that finish in a given trip.  In
  // the last 2 x (resident threads) items the warp fetches only what its
  // lanes need, so that no warp holds a backlog while others run dry.
  constexpr int QN = 64;
  __shared__ double qv[BS / 32][POL_NV + 1][QN];
  __shared__ long long qit[BS / 32][QN];
  __shared__ int qk[BS / 32][QN];
  int qhead = 0, qcount = 0;  // warp-uniform
  bool drained = false;       // warp-uniform: the work counter has passed NBP
  extern __shared__ double pol_dsm[];
  double *frd = pol_dsm + (size_t)wib * POL_FD * POL_QF;
  float *frf = (float *)(pol_dsm + (size_t)(BS / 32) * POL_FD * POL_QF) + (size_t)wib * POL_FF * POL_QF;
  int *fri = (int *)(pol_dsm + (size_t)(BS / 32) * POL_FD * POL_QF) + (size_t)(BS / 32) * POL_FF * POL_QF +
             (size_t)wib * POL_FI * POL_QF;
  __shared__ int ftail[BS / 32];  // records pushed by each warp (monotone)
  int fhead = 0;                  // warp-uniform: records written out
  if (lane == 0) ftail[wib] = 0;
  __syncwarp();
  const long long NBP = S.NBP, NL = S.NL, NEP = S.NEP;
  const long long tail = 2LL * gridDim.x * BS;
  // Order of the work: first the line-periods the previous sweep flagged
  // (a solve that had a variable near a bound or a slack held at zero: the
  // rarer, divergent paths of the solver), from its list, so that they
  // share warps with each other; then every other line-period in index
  // order.  Each solve is independent, so the order changes no result.
  // The list is the one the previous sweep wrote; a line-period is on it
  // exactly when its mark pgen is G + 1, and one that this sweep has already
  // taken from the list and flagged again carries G + 2: the second phase
  // skips both (G changes only when the last warp retires).
  const unsigned G = (unsigned)S.pctl[3];
  // warp-uniform: 0 the listed items, then 1 the rest; 2 the rest when the
  // list is empty (no mark can then equal G + 1 or G + 2, and none is read)
  int phase = S.pctl[1 + (G & 1u)] > 0ull ? 0 : 2;
  const double eta = S.prm.eta;
  const int K_N = S.prm.K_N, K_AL = S.prm.K_AL;
  bool active = true;
  long long bp = -1;  // item
  // per-lane values used only where a solve starts or ends, kept in shared
  // memory (one column per lane) to spare registers: the slots of the
  // item's from / to end, the multiplier loop's previous |h| and penalty
  // cap, and the statistics accumulated for the current instance
  __shared__ long long lsl[BS / 32][2][32];
  __shared__ double lal[BS / 32][2][32];
  __shared__ unsigned long long lst[BS / 32][4][32];
  long long &lef = lsl[wib][0][lane], &let = lsl[wib][1][lane];
  double &hprev = lal[wib][0][lane], &cmax = lal[wib][1][lane];
  unsigned long long &acc_nw = lst[wib][0][lane], &acc_al = lst[wib][1][lane], &acc_cap = lst[wib][2][lane],
                     &acc_w = lst[wib][3][lane];
  lef = let = 0;
  hprev = INFINITY;
  cmax = 0.0;
  int k = 0, itn = 0, al = 0, newton = 0;
  // per-lane statistics, flushed to the instance's counters when the lane
  // moves to another instance or retires (consecutive items mostly share one)
  int acc_k = -1;
  acc_nw = acc_al = acc_cap = acc_w = 0;
  auto flush = [&]() {
    if (acc_k >= 0) {
      unsigned long long *st = (unsigned long long *)(S.bstat + (long long)acc_k * 3);
      atomicAdd(&st[0], acc_nw);
      atomicAdd(&st[1], acc_al);
      if (acc_cap) atomicAdd(&st[2], acc_cap);
      if (acc_w) atomicAdd(&S.wstat[acc_k], acc_w);
    }
    acc_nw = acc_al = acc_cap = acc_w = 0;
  };
  bool need_full = false, trial = false;
  bool hard = false;  // the current solve met a bound or held a slack: flagged for the next sweep
  // a solve that ends with a non-tiny last step is evaluated once more at its
  // final point (at the next trip's single call site, with the rest of the
  // warp) and then finished from that evaluation: 1 converged, 2 stopped
  int fin_pend = 0;
  __shared__ double trs[BS / 32][TR_N][32];  // the lanes' trial records
  double *trp = &trs[wib][0][lane];
  double f = 0.0, Delta = 1.0, omega = 0.0;
  double v[POL_NV], gx[3], Hd[6];
  float Hf[6];
  PolLast L;
  PolK K;
  K.f = &kf[0][threadIdx.x];
  K.fs = BS;
  PolP P;
  while (true) {
    const bool want = active && bp < 0;
    const unsigned m = __ballot_sync(FULL, want);
    if (m) {
      const int nw = __popc(m);
      for (int fetch = 0; fetch < 2 && qcount < nw && !drained; ++fetch) {
        __syncwarp();
        unsigned long long base = 0;
        int nb = 0;
        long long it = -1;
        int ki = 0;
        if (phase == 0) {
          const int par = (int)(G & 1u);
          // the flagged line-periods of the previous sweep, from its list
          if (lane == 0) base = atomicAdd(&S.pctl[0], 32ull);
          base = __shfl_sync(FULL, base, 0);
          const long long left = (long long)S.pctl[1 + par] - (long long)base;
          const int got = left <= 0 ? 0 : (left < 32 ? (int)left : 32);
          if (left <= 32) phase = 1;
          if (lane < got && chk_(S, (long long)base + lane < NBP, 1)) {
            it = S.plist[(long long)par * NBP + (long long)base + lane];
            if (!chk_(S, it >= 0 && it < NBP, 2)) it = -1;
          }
        } else {
          if (lane == 0) {
            const unsigned long long cur = *(volatile unsigned long long *)S.bp_counter;
            nb = ((long long)cur + tail < NBP) ? 32 : nw - qcount;
            base = atomicAdd(S.bp_counter, (unsigned long long)nb);
          }
          base = __shfl_sync(FULL, base, 0);
          nb = __shfl_sync(FULL, nb, 0);
          const long long left = NBP - (long long)base;
          const int got = left <= 0 ? 0 : (left < nb ? (int)left : nb);
          if (left <= nb) drained = true;
          // (a line-period on the list was taken in the first phase)
          if (lane < got) {
            it = (long long)base + lane;
            if (phase == 1) {
              const unsigned mk = S.pgen[it];
              if (mk == G + 1u || mk == G + 2u) it = -1;
            }
          }
        }
        // the lines of a converged instance are skipped: the fetched items
        // that remain are packed into the ring
        if (it >= 0) {
          ki = find_instance(S, it);
          if (!chk_(S, ki >= 0 && ki < S.K && it >= (long long)S.inst[ki].bpo, 3)) it = -1;
          else if (inst_done(S, ki)) it = -1;
        }
        const unsigned vm = __ballot_sync(FULL, it >= 0);
        if (it >= 0) {
          double vs[POL_NV], ic;
          pol_start(S, it, vs, ic);
          const int sl = (qhead + qcount + __popc(vm & ((1u << lane) - 1u))) & (QN - 1);
          qit[wib][sl] = it;
          qk[wib][sl] = ki;
#pragma unroll
          for (int i = 0; i < POL_NV; ++i) qv[wib][i][sl] = vs[i];
          qv[wib][POL_NV][sl] = ic;
        }
        qcount += __popc(vm);
        __syncwarp();
      }
      if (want) {
        const int r = __popc(m & ((1u << lane) - 1u));
        if (r >= qcount) {
          // the ring is empty: retire once the counter has passed NBP, else
          // wait for the next fetch (skipped items can leave a fetch short)
          if (drained) {
            active = false;
            flush();
          }
        } else {
          const int sl = (qhead + r) & (QN - 1);
          bp = qit[wib][sl];
          k = qk[wib][sl];
#pragma unroll
          for (int i = 0; i < POL_NV; ++i) v[i] = qv[wib][i][sl];
          P.ic = qv[wib][POL_NV][sl];
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
          K.q[0] = Gii;  K.q[1] = -Bii; K.q[2] = Gjj;  K.q[3] = -Bjj;
          K.ga[0] = Gij; K.ka[0] = Bij;  K.ga[1] = Gji; K.ka[1] = -Bji;
#pragma unroll
          for (int j = 0; j < 8; ++j) kf[j][threadIdx.x] = S.BCF[j * NL + lg];
          K.rate2 = S.BC[BC_RATE2 * NL + lg];
          K.lo0 = S.BC[(BC_VB + 0) * NL + lg];
          K.hi0 = S.BC[(BC_VB + 1) * NL + lg];
          K.lo1 = S.BC[(BC_VB + 2) * NL + lg];
          K.hi1 = S.BC[(BC_VB + 3) * NL + lg];
          kf[8][threadIdx.x] = d2f_trunc(K.lo0);
          kf[9][threadIdx.x] = d2f_trunc(K.hi0);
          kf[10][threadIdx.x] = d2f_trunc(K.lo1);
          kf[11][threadIdx.x] = d2f_trunc(K.hi1);
          line_ends(S, I, t, lg, lef, let);
          if (!chk_(S, lef >= 0 && lef < NEP && let >= 0 && let < NEP, 4)) lef = let = 0;
#pragma unroll
          for (int r8 = 0; r8 < 8; ++r8) P.tg[r8] = S.ET[erow_u(r8) * NEP + (erow_end(r8) ? let : lef)];
          {
            const double t6 = P.tg[6], t7 = P.tg[7];
            P.tg[6] = t6 - t7;
            P.tg[7] = 0.5 * (t6 + t7);
          }
          P.rpq = I.rpq;
          P.rva = I.rva;
          P.frpq = I.frpq;
          P.frva = I.frva;
          P.mu[0] = S.B[(FB_MU0 + 2) * NBP + bp];
          P.mu[1] = S.B[(FB_MU0 + 3) * NBP + bp];
          P.c = S.B[FB_C * NBP + bp];
          if (S.warm && S.prop[bp] != 0.0f) {
            // learned warm start: the MLP kernel of this sweep chose the
            // network's proposal over the plain start and left its changes
            // of V_i, V_j, d; the Newton solve that follows is the same
            v[0] = pol_clamp(K, 0, v[0] + (double)S.prop[1 * NBP + bp]);
            v[1] = pol_clamp(K, 1, v[1] + (double)S.prop[2 * NBP + bp]);
            v[2] = pol_clamp(K, 2, v[2] + (double)S.prop[3 * NBP + bp]);
            ++acc_w;
          }
          omega = I.omega;
          cmax = I.cmax;
          hprev = INFINITY;
          Delta = 1.0;
          itn = al = newton = 0;
          need_full = true;
          trial = false;
          hard = false;
        }
      }
      const int used = nw < qcount ? nw : qcount;
      qhead = (qhead + used) & (QN - 1);
      qcount -= used;
    }
    if (__ballot_sync(FULL, active) == 0) {
      __syncwarp();
      if (lane < ftail[wib] - fhead) pol_finish_out(S, frd, frf, fri, (fhead + lane) & (POL_QF - 1), G);
      __syncwarp();
      // the last warp to retire makes this sweep's flags and list the next
      // sweep's, and clears the count of the buffer it will write
      if (lane == 0) {
        const unsigned long long nwarps = (unsigned long long)gridDim.x * (BS / 32);
        if (atomicAdd(&S.pctl[4], 1ull) == nwarps - 1ull) {
          S.pctl[1 + (G & 1u)] = 0ull;
          S.pctl[3] = (unsigned long long)(G + 1u);
          S.pctl[4] = 0ull;
        }
      }
      break;
    }
    if (active && bp >= 0) {
      // one full evaluation per trip: at a pending trial point (then the
      // ratio test), else at the current point when it moved
      int out = NI_CONT;
      bool step_now = true;
      if (need_full) {
        // one call site for every lane: the point is the trial point or the
        // current point (two call sites would split the warp between copies)
        double tv[POL_NV], tht[2];
#pragma unroll
        for (int i = 0; i < POL_NV; ++i) tv[i] = trial ? trp[32 * (TR_V + i)] : v[i];
        tht[0] = trial ? trp[32 * TR_HT] : 0.0;
        tht[1] = trial ? trp[32 * (TR_HT + 1)] : 0.0;
        pol_full(K, P, tv, gx, Hf, Hd, L, tht, trial ? 3 : 0);
        if (trial) {
          trial = false;
          const double fe = pol_f(P, L);
          const double ared = f - fe;
          const double pred = trp[32 * TR_PRED], smax = trp[32 * TR_SMAX];
          if (pred > 0.0 && ared >= 1e-4 * pred) {
#pragma unroll
            for (int i = 0; i < POL_NV; ++i) v[i] = tv[i];
            f = fe;
            if (ared >= 0.75 * pred && trp[32 * TR_SCALE] < 1.0) Delta = 2.0 * Delta;
          } else {
            // rejected: the evaluation describes the trial point, so the
            // current point is evaluated again at the next trip
            Delta = 0.25 * smax;
            step_now = false;
            if (Delta <= 1e-15 * (1.0 + fmax(fmax(fabs(v[0]), fabs(v[1])), fabs(v[2])))) out = NI_STOP;
          }
        }
      }
      need_full = !step_now;
      if (fin_pend) {
        step_now = false;
        need_full = false;
        out = NI_STOP;  // (the finish takes conv from fin_pend)
      }
      if (step_now) {
        bool accepted;
        int counted;
        bool nearb;
        if (L.lim) {
          out = pol_iter<double>(K, P, v, f, gx, L, Hd, Delta, omega, accepted, counted, trp, nearb);
        } else {
          out = pol_fast(K, P, v, gx, L, Hf, Delta, omega, accepted, counted);
          nearb = false;
          if (out == NI_FULL) out = pol_iter<float>(K, P, v, f, gx, L, Hf, Delta, omega, accepted, counted, trp, nearb);
        }
        hard = hard || nearb || L.lim;
        newton += counted;
        if (out == NI_TRIAL) {
          trial = true;
          need_full = true;
          out = NI_CONT;
        } else {
          need_full = accepted;
        }
      }
      ++itn;
      if (out != NI_CONT || itn >= K_N) {
        trial = false;
        const bool conv = fin_pend ? fin_pend == 1 : (out == NI_CONV);
        // flows, cos/sin and h_k at v: first order from the last evaluation
        // when the last step is tiny (h_k in FP64 from grad g_k, so that it
        // matches the slack step taken from the same gradient); otherwise v
        // is evaluated at the next trip and the solve finishes from there
        // (the flows and cos/sin themselves are formed from the base values
        // ab, cb, sb and the step fx, dxs by the finish ring: with dx <= 1e-8
        // the FP32 product carries ~1e-15 absolute error)
        const double dx0 = v[0] - L.v[0], dx1 = v[1] - L.v[1], dx2 = v[2] - L.v[2];
        const long long b8 = __double_as_longlong(1e-8);
        const bool tiny = abs_bits(dx0) <= b8 && abs_bits(dx1) <= b8 && abs_bits(dx2) <= b8;
        if (!tiny) {
          fin_pend = conv ? 1 : 2;
          need_full = true;
        } else {
          fin_pend = 0;
          double ab[4], cb, sb, dxs, h[2];
          float fx[3];
          {
#pragma unroll
            for (int r = 0; r < 4; ++r) ab[r] = L.a[r];
            cb = L.c;
            sb = L.s;
            fx[0] = d2f_trunc(dx0);
            fx[1] = d2f_trunc(dx1);
            fx[2] = d2f_trunc(dx2);
            dxs = dx2;
#pragma unroll
            for (int q = 0; q < 2; ++q)
              h[q] = L.h[q] + f2d_exact(L.fdg[q][0] * fx[0] + L.fdg[q][1] * fx[1] + L.fdg[q][2] * fx[2]) +
                     (v[3 + q] - L.v[3 + q]);
          }
          // equality multiplier step on h_k = p_k^2 + q_k^2 + sigma_k - rate^2
          long long bh = 0;
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const long long b = abs_bits(h[q]);
            bh = b > bh ? b : bh;
            P.mu[q] += P.c * h[q];
          }
          const double hn = __longlong_as_double(bh);  // max |h_k|
          ++al;
          const bool done = le_nn(hn, eta) && conv;
          if (done || al >= K_AL) {
            S.B[(FB_V0 + 6) * NBP + bp] = v[3];
            S.B[(FB_V0 + 7) * NBP + bp] = v[4];
            S.B[(FB_MU0 + 0) * NBP + bp] = 0.0;
            S.B[(FB_MU0 + 1) * NBP + bp] = 0.0;
            S.B[(FB_MU0 + 2) * NBP + bp] = P.mu[0];
            S.B[(FB_MU0 + 3) * NBP + bp] = P.mu[1];
            S.B[FB_C * NBP + bp] = P.c;
            {
              const int sl = atomicAdd(&ftail[wib], 1) & (POL_QF - 1);
#pragma unroll
              for (int r = 0; r < 4; ++r) frd[r * POL_QF + sl] = ab[r];
              frd[4 * POL_QF + sl] = cb;
              frd[5 * POL_QF + sl] = sb;
              frd[6 * POL_QF + sl] = v[0];
              frd[7 * POL_QF + sl] = v[1];
              frd[8 * POL_QF + sl] = v[2];
              frd[9 * POL_QF + sl] = dxs;
              frd[10 * POL_QF + sl] = P.tg[7];
              frd[11 * POL_QF + sl] = P.ic;
#pragma unroll
              for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int i = 0; i < 3; ++i) frf[(3 * r + i) * POL_QF + sl] = L.da[r][i];
              frf[12 * POL_QF + sl] = fx[0];
              frf[13 * POL_QF + sl] = fx[1];
              frf[14 * POL_QF + sl] = fx[2];
              fri[sl] = (int)((unsigned)bp | (hard ? 0x80000000u : 0u));
              fri[POL_QF + sl] = (int)lef;
              fri[2 * POL_QF + sl] = (int)let;
            }
            acc_nw += (unsigned long long)newton;
            acc_al += (unsigned long long)al;
            acc_cap += done ? 0ull : 1ull;
            S.lcount[bp] = (unsigned short)min(newton, 65535);  // (saturated)
            S.lcount[NBP + bp] = (unsigned short)min(al, 65535);
            bp = -1;
          } else {
            if (hn > 0.25 * hprev) {
              P.c = fmin(10.0 * P.c, cmax);
              P.ic = 1.0 / P.c;
            }
            hprev = hn;
            Delta = fmax(Delta, 1e-3);
            itn = 0;
            need_full = true;
          }
        }
      }
    }
    // the outputs of 32 finish records, with every lane active
    __syncwarp();
    if (ftail[wib] - fhead >= 32) {
      pol_finish_out(S, frd, frf, fri, (fhead + lane) & (POL_QF - 1), G);
      fhead += 32;
      __syncwarp();
    }
  }
}

}  // namespace ucac
