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
// B300 mapping: one thread per branch-period; the 8x8 Hessian, its Cholesky
// factor and all vectors are indexed only by compile-time constants (fully
// unrolled loops, the active set applied by masking rather than by
// compacting indices), so they stay in registers.  The kernel is bound by the
// FP64 pipe, not memory: its loads/stores are a few hundred bytes per solve.
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

// Inner solve (the damped projected Newton method described above): returns Newton iterations used;
// conv = true when the stationarity test or the final-step test ended it.
__device__ __forceinline__ int br_inner(const BrK &K, const BrP &P, double (&v)[8], int K_N, double omega,
                                        double &Delta, bool &conv) {
  double g[8], H[8][8];
  double f = br_phi(K, P, v);
  br_derivs(K, P, v, g, H);
  int it = 0;
  conv = false;
  for (; it < K_N; ++it) {
    double pg = 0.0, hmax = 0.0, vmax = 0.0, eps = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      pg = fmax(pg, fabs(clampd(v[i] - g[i], K.lo[i], K.hi[i]) - v[i]));
      hmax = fmax(hmax, H[i][i]);
      vmax = fmax(vmax, fabs(v[i]));
      const double di = (H[i][i] > 0.0) ? g[i] / H[i][i] : g[i];
      eps = fmax(eps, fabs(clampd(v[i] - di, K.lo[i], K.hi[i]) - v[i]));
    }
    if (pg <= omega) {
      conv = true;
      break;
    }
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
    if (!ok) break;
    double dn = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      d[i] = x[i];
      dn = fmax(dn, fabs(d[i]));
    }
    double predN = 0.0;
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
      predN = -(gd + 0.5 * dHd);
      if (dn <= 1e-9 * (1.0 + vmax) || predN <= 1e-12 * (1.0 + fabs(f))) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = clampd(v[i] + d[i], K.lo[i], K.hi[i]);
        conv = true;
        ++it;
        break;
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
      br_derivs(K, P, v, g, H);
      if (ared >= 0.75 * pred && scale < 1.0) Delta = 2.0 * Delta;
    } else {
      Delta = 0.25 * smax;
      if (Delta <= 1e-15 * (1.0 + vmax)) break;
    }
  }
  return it;
}

struct BrResult {
  int newton, al, status;
};

__device__ __forceinline__ BrResult branch_solve(const BrK &K, BrP &P, double (&v)[8], double eta, double omega,
                                                 double c_max, int K_AL, int K_N) {
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = clampd(v[i], K.lo[i], K.hi[i]);
  double hprev = INFINITY, Delta = 1.0;
  BrResult R{0, 0, 1};
  for (int al = 0; al < K_AL;) {
    bool conv = false;
    Delta = fmax(Delta, 1e-3);
    R.newton += br_inner(K, P, v, K_N, omega, Delta, conv);
    double a[4], h[4];
    br_flows(K, v, a);
    br_cons(K, v, a, h);
    double hn = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      P.mu[k] += P.c * h[k];
      hn = fmax(hn, fabs(h[k]));
    }
    ++al;
    R.al = al;
    if (hn <= eta && conv) {
      R.status = 0;
      break;
    }
    if (hn > 0.25 * hprev) P.c = fmin(10.0 * P.c, c_max);
    hprev = hn;
  }
  return R;
}

template <int BS>
__global__ void __launch_bounds__(BS) k_branch(Dev S) {
  const int b = blockIdx.x;
  const int k = S.b_bp.inst[b];
  const Inst I = S.inst[k];
  const long long bp = (long long)S.b_bp.first[b] + threadIdx.x;
  const bool valid = bp < (long long)I.bpo + (long long)I.T * I.nl;
  long long nwt = 0, nal = 0, ncap = 0;
  if (valid) {
    const int loc = (int)(bp - I.bpo);
    const int t = loc / I.nl, l = loc - t * I.nl;
    const long long lg = (long long)I.lo + l, NL = S.NL, NBP = S.NBP;
    BrK K;
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
    BrP P;
#pragma unroll
    for (int r = 0; r < 8; ++r) P.tg[r] = S.BT[r * NBP + bp];
    P.rpq = I.rpq;
    P.rva = I.rva;
#pragma unroll
    for (int q = 0; q < 4; ++q) P.mu[q] = S.B[(FB_MU0 + q) * NBP + bp];
    P.c = S.B[FB_C * NBP + bp];
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = S.B[(FB_V0 + i) * NBP + bp];
    const double rmax = fmax(I.rpq, I.rva);
    const BrResult R = branch_solve(K, P, v, S.prm.eta, S.prm.omega_rel * rmax, S.prm.c_max_rel * rmax,
                                    S.prm.K_AL, S.prm.K_N);
#pragma unroll
    for (int i = 0; i < 8; ++i) S.B[(FB_V0 + i) * NBP + bp] = v[i];
#pragma unroll
    for (int q = 0; q < 4; ++q) S.B[(FB_MU0 + q) * NBP + bp] = P.mu[q];
    S.B[FB_C * NBP + bp] = P.c;
    double a[4];
    br_flows(K, v, a);
#pragma unroll
    for (int r = 0; r < 4; ++r) S.BA[r * NBP + bp] = a[r];
    S.BA[4 * NBP + bp] = v[0];
    S.BA[5 * NBP + bp] = v[1];
    S.BA[6 * NBP + bp] = v[4];
    S.BA[7 * NBP + bp] = v[5];
    nwt = R.newton;
    nal = R.al;
    ncap = (R.status != 0);
  }
  // block sums of the iteration counters (fixed order)
  __shared__ long long sh[3][BS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nwt += __shfl_down_sync(0xffffffffu, nwt, o);
    nal += __shfl_down_sync(0xffffffffu, nal, o);
    ncap += __shfl_down_sync(0xffffffffu, ncap, o);
  }
  if (lane == 0) {
    sh[0][wid] = nwt;
    sh[1][wid] = nal;
    sh[2][wid] = ncap;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    long long s = 0;
    for (int w = 0; w < BS / 32; ++w) s += sh[threadIdx.x][w];
    S.part_bp[(long long)b * 3 + threadIdx.x] = s;
  }
}

}  // namespace ucac
