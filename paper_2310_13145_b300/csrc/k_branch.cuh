// k_branch.cuh -- line x-update per (t, line ij) (Eq. step:opf for the line
// component; the line subproblems the paper solves with a batched
// bound-constrained Newton solver for up to 32 variables, Sec. IV-A).
//
// Variables v = (w_i, w_j, wR, wI, theta_i, theta_j, sigma_ij, sigma_ji) with
// box bounds (Eq. uc_acopf_w_bound for w; |wR|,|wI| <= Vmax_i Vmax_j;
// |theta| <= 2 pi; 0 <= sigma <= rate^2).  Flows are linear in v (the four
// flow equations of Eq. acopf, the second pair read as the j->i direction).
// Equalities (Eq. acopf):
//   h0 = wR^2 + wI^2 - w_i w_j        h1 = theta_i - theta_j - atan2(wI, wR)
//   h2 = p_ij^2 + q_ij^2 + sigma_ij - rate^2,  h3 = same for ji.
// Objective: sum over the 8 consensus rows of rho/2 (a_r - t_r)^2 plus
// mu^T h + c/2 |h|^2, minimised by an augmented-Lagrangian loop (mu += c h,
// c x10 when |h| fell by less than 4x, stop when |h|_inf <= eta) around a
// projected Newton method with an epsilon-active set and a trust radius on
// the step (see br_inner).  The multipliers mu and the penalty c persist per
// (t, line) across sweeps, as does v (the warm start).
//
// B300 mapping: a persistent kernel.  Every lane owns one line solve at a
// time; each pass of the main loop performs one Newton iteration for every
// lane (so the warp executes the same instructions whatever the phase of
// each solve), and a lane whose solve has finished fetches the next
// branch-period from a global counter (warp-aggregated atomic).  Lanes thus
// never wait for the slowest solve of their warp, which is what idles half of
// a statically mapped warp: iteration counts differ from solve to solve.  The
// 8x8 Hessian, its Cholesky factor and all vectors are indexed only by
// compile-time constants (fully unrolled loops, the active set applied by
// masking), so they stay in registers.  The kernel is bound by the FP64 pipe,
// not memory: its loads/stores are a few hundred bytes per solve.
#pragma once
#include "common.cuh"

namespace ucac {

struct BrK {
  double Gii, Bii, Gij, Bij, Gjj, Bjj, Gji, Bji, rate2;
  double lo[8], hi[8];
};

struct BrP {
  double tg[8];
  double rpq, rva;
  double mu[4];
  double c;
};

__device__ __forceinline__ void br_flows(const BrK &K, const double (&v)[8], double (&a)[4]) {
  a[0] = K.Gii * v[0] + K.Gij * v[2] + K.Bij * v[3];
  a[1] = -K.Bii * v[0] - K.Bij * v[2] + K.Gij * v[3];
  a[2] = K.Gjj * v[1] + K.Gji * v[2] - K.Bji * v[3];
  a[3] = -K.Bjj * v[1] - K.Bji * v[2] - K.Gji * v[3];
}

__device__ __forceinline__ void br_cons(const BrK &K, const double (&v)[8], const double (&a)[4], double (&h)[4]) {
  h[0] = v[2] * v[2] + v[3] * v[3] - v[0] * v[1];
  h[1] = v[4] - v[5] - atan2(v[3], v[2]);
  h[2] = a[0] * a[0] + a[1] * a[1] + v[6] - K.rate2;
  h[3] = a[2] * a[2] + a[3] * a[3] + v[7] - K.rate2;
}

__device__ __forceinline__ double br_phi(const BrK &K, const BrP &P, const double (&v)[8]) {
  double a[4], h[4];
  br_flows(K, v, a);
  br_cons(K, v, a, h);
  double f = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) f += 0.5 * P.rpq * (a[r] - P.tg[r]) * (a[r] - P.tg[r]);
  f += 0.5 * P.rva * ((v[0] - P.tg[4]) * (v[0] - P.tg[4]) + (v[1] - P.tg[5]) * (v[1] - P.tg[5]) +
                      (v[4] - P.tg[6]) * (v[4] - P.tg[6]) + (v[5] - P.tg[7]) * (v[5] - P.tg[7]));
#pragma unroll
  for (int k = 0; k < 4; ++k) f += P.mu[k] * h[k] + 0.5 * P.c * h[k] * h[k];
  return f;
}

// gradient and (symmetric) Hessian of the inner objective, exploiting the
// sparsity of the flow and constraint gradients
__device__ __forceinline__ void br_derivs(const BrK &K, const BrP &P, const double (&v)[8], double (&g)[8],
                                          double (&H)[8][8]) {
  double a[4], h[4];
  br_flows(K, v, a);
  br_cons(K, v, a, h);
  // flow gradients restricted to (w_i, wR, wI) and (w_j, wR, wI)
  const double Pi0 = K.Gii, Pi2 = K.Gij, Pi3 = K.Bij;     // d p_ij
  const double Qi0 = -K.Bii, Qi2 = -K.Bij, Qi3 = K.Gij;   // d q_ij
  const double Pj1 = K.Gjj, Pj2 = K.Gji, Pj3 = -K.Bji;    // d p_ji
  const double Qj1 = -K.Bjj, Qj2 = -K.Bji, Qj3 = -K.Gji;  // d q_ji
  double lam[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) lam[k] = P.mu[k] + P.c * h[k];
  const double r2 = v[2] * v[2] + v[3] * v[3];
  const double ir2 = (r2 > 1e-300) ? 1.0 / r2 : 0.0;
  // constraint gradients (nonzero entries)
  const double dh0_0 = -v[1], dh0_1 = -v[0], dh0_2 = 2.0 * v[2], dh0_3 = 2.0 * v[3];
  const double dh1_2 = v[3] * ir2, dh1_3 = -v[2] * ir2;  // dh1_4 = 1, dh1_5 = -1
  const double dh2_0 = 2.0 * (a[0] * Pi0 + a[1] * Qi0), dh2_2 = 2.0 * (a[0] * Pi2 + a[1] * Qi2),
               dh2_3 = 2.0 * (a[0] * Pi3 + a[1] * Qi3);  // dh2_6 = 1
  const double dh3_1 = 2.0 * (a[2] * Pj1 + a[3] * Qj1), dh3_2 = 2.0 * (a[2] * Pj2 + a[3] * Qj2),
               dh3_3 = 2.0 * (a[2] * Pj3 + a[3] * Qj3);  // dh3_7 = 1
  // gradient
  const double e0 = P.rpq * (a[0] - P.tg[0]), e1 = P.rpq * (a[1] - P.tg[1]);
  const double e2 = P.rpq * (a[2] - P.tg[2]), e3 = P.rpq * (a[3] - P.tg[3]);
  g[0] = e0 * Pi0 + e1 * Qi0 + P.rva * (v[0] - P.tg[4]) + lam[0] * dh0_0 + lam[2] * dh2_0;
  g[1] = e2 * Pj1 + e3 * Qj1 + P.rva * (v[1] - P.tg[5]) + lam[0] * dh0_1 + lam[3] * dh3_1;
  g[2] = e0 * Pi2 + e1 * Qi2 + e2 * Pj2 + e3 * Qj2 + lam[0] * dh0_2 + lam[1] * dh1_2 + lam[2] * dh2_2 +
         lam[3] * dh3_2;
  g[3] = e0 * Pi3 + e1 * Qi3 + e2 * Pj3 + e3 * Qj3 + lam[0] * dh0_3 + lam[1] * dh1_3 + lam[2] * dh2_3 +
         lam[3] * dh3_3;
  g[4] = P.rva * (v[4] - P.tg[6]) + lam[1];
  g[5] = P.rva * (v[5] - P.tg[7]) - lam[1];
  g[6] = lam[2];
  g[7] = lam[3];
  // Hessian: (rho_pq + 2 lam2) (P P^T + Q Q^T)_ij + (rho_pq + 2 lam3) (..)_ji
  //          + rho_va diag(0,1,4,5) + sum_k c dh_k dh_k^T + lam0 d2h0 + lam1 d2h1
  const double wi = P.rpq + 2.0 * lam[2], wj = P.rpq + 2.0 * lam[3], c = P.c;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) H[i][j] = 0.0;
  // ij flow block on (0,2,3)
  H[0][0] += wi * (Pi0 * Pi0 + Qi0 * Qi0);
  H[0][2] += wi * (Pi0 * Pi2 + Qi0 * Qi2);
  H[0][3] += wi * (Pi0 * Pi3 + Qi0 * Qi3);
  H[2][2] += wi * (Pi2 * Pi2 + Qi2 * Qi2);
  H[2][3] += wi * (Pi2 * Pi3 + Qi2 * Qi3);
  H[3][3] += wi * (Pi3 * Pi3 + Qi3 * Qi3);
  // ji flow block on (1,2,3)
  H[1][1] += wj * (Pj1 * Pj1 + Qj1 * Qj1);
  H[1][2] += wj * (Pj1 * Pj2 + Qj1 * Qj2);
  H[1][3] += wj * (Pj1 * Pj3 + Qj1 * Qj3);
  H[2][2] += wj * (Pj2 * Pj2 + Qj2 * Qj2);
  H[2][3] += wj * (Pj2 * Pj3 + Qj2 * Qj3);
  H[3][3] += wj * (Pj3 * Pj3 + Qj3 * Qj3);
  H[0][0] += P.rva;
  H[1][1] += P.rva;
  H[4][4] += P.rva;
  H[5][5] += P.rva;
  // c dh0 dh0^T on (0,1,2,3) and lam0 d2h0
  H[0][0] += c * dh0_0 * dh0_0;
  H[0][1] += c * dh0_0 * dh0_1 - lam[0];
  H[0][2] += c * dh0_0 * dh0_2;
  H[0][3] += c * dh0_0 * dh0_3;
  H[1][1] += c * dh0_1 * dh0_1;
  H[1][2] += c * dh0_1 * dh0_2;
  H[1][3] += c * dh0_1 * dh0_3;
  H[2][2] += c * dh0_2 * dh0_2 + 2.0 * lam[0];
  H[2][3] += c * dh0_2 * dh0_3;
  H[3][3] += c * dh0_3 * dh0_3 + 2.0 * lam[0];
  // c dh1 dh1^T on (2,3,4,5) and lam1 d2h1 on (2,3)
  {
    const double ir4 = ir2 * ir2;
    H[2][2] += c * dh1_2 * dh1_2 + lam[1] * (-2.0 * v[2] * v[3] * ir4);
    H[2][3] += c * dh1_2 * dh1_3 + lam[1] * ((v[2] * v[2] - v[3] * v[3]) * ir4);
    H[3][3] += c * dh1_3 * dh1_3 + lam[1] * (2.0 * v[2] * v[3] * ir4);
    H[2][4] += c * dh1_2;
    H[2][5] -= c * dh1_2;
    H[3][4] += c * dh1_3;
    H[3][5] -= c * dh1_3;
    H[4][4] += c;
    H[4][5] -= c;
    H[5][5] += c;
  }
  // c dh2 dh2^T on (0,2,3,6)
  H[0][0] += c * dh2_0 * dh2_0;
  H[0][2] += c * dh2_0 * dh2_2;
  H[0][3] += c * dh2_0 * dh2_3;
  H[0][6] += c * dh2_0;
  H[2][2] += c * dh2_2 * dh2_2;
  H[2][3] += c * dh2_2 * dh2_3;
  H[2][6] += c * dh2_2;
  H[3][3] += c * dh2_3 * dh2_3;
  H[3][6] += c * dh2_3;
  H[6][6] += c;
  // c dh3 dh3^T on (1,2,3,7)
  H[1][1] += c * dh3_1 * dh3_1;
  H[1][2] += c * dh3_1 * dh3_2;
  H[1][3] += c * dh3_1 * dh3_3;
  H[1][7] += c * dh3_1;
  H[2][2] += c * dh3_2 * dh3_2;
  H[2][3] += c * dh3_2 * dh3_3;
  H[2][7] += c * dh3_2;
  H[3][3] += c * dh3_3 * dh3_3;
  H[3][7] += c * dh3_3;
  H[7][7] += c;
  // symmetrise (upper triangle was filled)
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) H[i][j] = H[j][i];
}

// In-place Cholesky solve of A x = b (A SPD, 8x8, lower factor overwrites A).
// Returns false when a pivot is not positive.
__device__ __forceinline__ bool chol8(double (&A)[8][8], double (&b)[8]) {
  double id[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    double s = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= A[j][k] * A[j][k];
    if (!(s > 0.0)) return false;
    const double d = sqrt(s);
    id[j] = 1.0 / d;
    A[j][j] = d;
#pragma unroll
    for (int i = j + 1; i < 8; ++i) {
      double t = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= A[i][k] * A[j][k];
      A[i][j] = t * id[j];
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    double t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= A[i][k] * b[k];
    b[i] = t * id[i];
  }
#pragma unroll
  for (int i = 7; i >= 0; --i) {
    double t = b[i];
#pragma unroll
    for (int k = i + 1; k < 8; ++k) t -= A[k][i] * b[k];
    b[i] = t * id[i];
  }
  return true;
}

// One iteration of the inner solve (projected Newton with an epsilon-active
// set and a trust radius):
//   1. stationarity |P(v - g) - v|_inf <= omega -> converged;
//   2. active set: within eps of a bound with the gradient pointing out
//      (eps = min(1e-6, diagonally scaled projected-gradient size)); active
//      coordinates move onto their bound;
//   3. Newton step on the free set by Cholesky of H_FF (+ lambda I, lambda =
//      1e-10 max diag H growing x10, only when H_FF is not positive definite);
//   4. an undamped step <= 1e-9 (1 + |v|_inf), or one predicting a decrease
//      <= 1e-12 (1 + |phi|), is taken as the final step -> converged;
//   5. otherwise the step is cut to the radius Delta, projected, and accepted
//      when actual >= 1e-4 x predicted decrease (Delta x2 after a very good
//      radius-limited step, Delta = |s|/4 after a rejection).
enum { NI_CONT = 0, NI_CONV = 1, NI_STOP = 2 };

__device__ __forceinline__ int newton_iter(const BrK &K, const BrP &P, double (&v)[8], double &f,
                                           const double (&g)[8], const double (&H)[8][8], double &Delta,
                                           double omega, bool &accepted, int &counted) {
  accepted = false;
  counted = 0;
  double pg = 0.0, hmax = 0.0, vmax = 0.0, eps = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    pg = fmax(pg, fabs(clampd(v[i] - g[i], K.lo[i], K.hi[i]) - v[i]));
    hmax = fmax(hmax, H[i][i]);
    vmax = fmax(vmax, fabs(v[i]));
    const double di = (H[i][i] > 0.0) ? g[i] / H[i][i] : g[i];
    eps = fmax(eps, fabs(clampd(v[i] - di, K.lo[i], K.hi[i]) - v[i]));
  }
  if (pg <= omega) return NI_CONV;
  eps = fmin(eps, 1e-6);
  bool act[8];
  double d[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    act[i] = false;
    d[i] = 0.0;
    if (v[i] <= K.lo[i] + eps && g[i] > 0.0) {
      act[i] = true;
      d[i] = K.lo[i] - v[i];
    } else if (v[i] >= K.hi[i] - eps && g[i] < 0.0) {
      act[i] = true;
      d[i] = K.hi[i] - v[i];
    }
  }
  double lm = 0.0, x[8];
  bool ok = false;
  for (int tries = 0; tries < 40; ++tries) {
    double A[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      double r = -g[i];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (act[j]) r -= H[i][j] * d[j];
        A[i][j] = (act[i] || act[j]) ? ((i == j) ? 1.0 : 0.0) : H[i][j];
      }
      if (!act[i]) A[i][i] += lm;
      x[i] = act[i] ? d[i] : r;
    }
    if (chol8(A, x)) {
      ok = true;
      break;
    }
    lm = (lm == 0.0) ? 1e-10 * hmax : 10.0 * lm;
  }
  if (!ok) return NI_STOP;
  double dn = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    d[i] = x[i];
    dn = fmax(dn, fabs(d[i]));
  }
  counted = 1;
  if (lm == 0.0) {
    double gd = 0.0, dHd = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      gd += g[i] * d[i];
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < 8; ++j) t += H[i][j] * d[j];
      dHd += d[i] * t;
    }
    const double predN = -(gd + 0.5 * dHd);
    if (dn <= 1e-9 * (1.0 + vmax) || predN <= 1e-12 * (1.0 + fabs(f))) {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = clampd(v[i] + d[i], K.lo[i], K.hi[i]);
      return NI_CONV;
    }
  }
  const double scale = (dn > Delta) ? Delta / dn : 1.0;
  double vt[8], s[8], smax = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    vt[i] = clampd(v[i] + scale * d[i], K.lo[i], K.hi[i]);
    s[i] = vt[i] - v[i];
    smax = fmax(smax, fabs(s[i]));
  }
  double gs = 0.0, sHs = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    gs += g[i] * s[i];
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += H[i][j] * s[j];
    sHs += s[i] * t;
  }
  const double pred = -(gs + 0.5 * sHs);
  const double ft = br_phi(K, P, vt);
  const double ared = f - ft;
  if (pred > 0.0 && ared >= 1e-4 * pred) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = vt[i];
    f = ft;
    accepted = true;
    if (ared >= 0.75 * pred && scale < 1.0) Delta = 2.0 * Delta;
    return NI_CONT;
  }
  Delta = 0.25 * smax;
  if (Delta <= 1e-15 * (1.0 + vmax)) {
    counted = 0;
    return NI_STOP;
  }
  return NI_CONT;
}

__device__ __forceinline__ int find_instance(const Dev &S, long long bp) {
  int lo = 0, hi = S.K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((long long)S.inst[mid].bpo <= bp) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Persistent line kernel.  Per solve (augmented-Lagrangian loop around the
// inner Newton iterations, reading R6):
//   inner solve until converged / stopped / K_N iterations; then mu += c h;
//   finished when |h|_inf <= eta after a converged inner solve (or after K_AL
//   rounds, status "capped"); otherwise c x10 (<= c_max) if |h| fell by less
//   than 4x, Delta >= 1e-3, and a new inner solve starts.
template <int BS>
__global__ void __launch_bounds__(BS) k_branch(Dev S) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long NBP = S.NBP, NL = S.NL, NEP = S.NEP;
  const double eta = S.prm.eta;
  const int K_N = S.prm.K_N, K_AL = S.prm.K_AL;
  bool active = true;
  long long bp = -1, lef = 0, let = 0;  // item, slots of its from / to end
  int k = 0, itn = 0, al = 0, newton = 0;
  bool need_f = false, need_gH = false;
  double f = 0.0, Delta = 1.0, hprev = INFINITY, omega = 0.0, cmax = 0.0;
  double v[8], g[8], H[8][8];
  BrK K;
  BrP P;
  while (true) {
    // ---- refill: lanes without a solve take the next branch-periods
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
          if (!chk_(S, k >= 0 && k < S.K && bp >= (long long)S.inst[k].bpo, 6)) k = 0;
        }
        if (active && inst_done(S, k)) {
          bp = -1;  // a converged instance's line: skipped (the lane fetches again)
        } else if (active) {
          const Inst &I = S.inst[k];
          const int loc = (int)(bp - I.bpo);
          const int t = loc / I.nl, l = loc - t * I.nl;
          const long long lg = (long long)I.lo + l;
          K.Gii = S.BC[(BC_Y0 + 0) * NL + lg];
          K.Bii = S.BC[(BC_Y0 + 1) * NL + lg];
          K.Gij = S.BC[(BC_Y0 + 2) * NL + lg];
          K.Bij = S.BC[(BC_Y0 + 3) * NL + lg];
          K.Gjj = S.BC[(BC_Y0 + 4) * NL + lg];
          K.Bjj = S.BC[(BC_Y0 + 5) * NL + lg];
          K.Gji = S.BC[(BC_Y0 + 6) * NL + lg];
          K.Bji = S.BC[(BC_Y0 + 7) * NL + lg];
          K.rate2 = S.BC[BC_RATE2 * NL + lg];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            K.lo[i] = S.BC[(BC_LO + i) * NL + lg];
            K.hi[i] = S.BC[(BC_HI + i) * NL + lg];
          }
          line_ends(S, I, t, lg, lef, let);
          if (!chk_(S, lef >= 0 && lef < NEP && let >= 0 && let < NEP, 5)) lef = let = 0;
#pragma unroll
          for (int r = 0; r < 8; ++r) P.tg[r] = S.ET[erow_u(r) * NEP + (erow_end(r) ? let : lef)];
          P.rpq = I.rpq;
          P.rva = I.rva;
#pragma unroll
          for (int q = 0; q < 4; ++q) P.mu[q] = S.B[(FB_MU0 + q) * NBP + bp];
          P.c = S.B[FB_C * NBP + bp];
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = clampd(S.B[(FB_V0 + i) * NBP + bp], K.lo[i], K.hi[i]);
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
    if (active && bp >= 0) {
      // ---- one Newton iteration
      if (need_f) f = br_phi(K, P, v);
      if (need_gH) br_derivs(K, P, v, g, H);
      need_f = need_gH = false;
      bool accepted;
      int counted;
      const int out = newton_iter(K, P, v, f, g, H, Delta, omega, accepted, counted);
      newton += counted;
      need_gH = accepted;
      ++itn;
      if (out != NI_CONT || itn >= K_N) {
        // ---- end of an inner solve: multiplier update
        const bool conv = (out == NI_CONV);
        double a[4], h[4];
        br_flows(K, v, a);
        br_cons(K, v, a, h);
        double hn = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          P.mu[q] += P.c * h[q];
          hn = fmax(hn, fabs(h[q]));
        }
        ++al;
        const bool done = (hn <= eta && conv);
        if (done || al >= K_AL) {
#pragma unroll
          for (int i = 0; i < 8; ++i) S.B[(FB_V0 + i) * NBP + bp] = v[i];
#pragma unroll
          for (int q = 0; q < 4; ++q) S.B[(FB_MU0 + q) * NBP + bp] = P.mu[q];
          S.B[FB_C * NBP + bp] = P.c;
#pragma unroll
          for (int r = 0; r < 4; ++r) S.EA[erow_u(r) * NEP + (erow_end(r) ? let : lef)] = a[r];
          S.EA[2 * NEP + lef] = v[0];
          S.EA[2 * NEP + let] = v[1];
          S.EA[3 * NEP + lef] = v[4];
          S.EA[3 * NEP + let] = v[5];
          long long *st = S.bstat + (long long)k * 3;
          atomicAdd((unsigned long long *)&st[0], (unsigned long long)newton);
          atomicAdd((unsigned long long *)&st[1], (unsigned long long)al);
          if (!done) atomicAdd((unsigned long long *)&st[2], 1ull);
          S.lcount[bp] = (unsigned short)min(newton, 65535);  // (saturated)
          S.lcount[NBP + bp] = (unsigned short)min(al, 65535);
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
