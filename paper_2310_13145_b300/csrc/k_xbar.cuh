// k_xbar.cuh -- x-bar step (Eq. step:uc_bar, step:opf_bar) fused with the
// z-update (Eq. step:z), the y-update (Eq. step:y), the next sweep's x-step
// targets and the residual partial sums; the per-instance finish kernel
// (residuals, inner stop test, outer update of Eq. step:outer); and the
// target preparation used after create / state import.
//
// Every coupling row has exactly one owner among the x-bar threads (the
// thread that owns the row's x-bar variable), so each row is read and written
// once per sweep by one thread with no atomics:
//   bus thread (t,i):   generator consensus rows gp, gq at (t, g at i), the
//                        temporal-copy row tc at (t+1, g at i), and the four
//                        line rows (p, q, w, theta) of every line end at i;
//   x-bar^UC thread (t,g): duplicate rows on, sd at t and su at t+1, the
//                        bound/ramp rows pl, pu, ql, qu, rd at t and ru at
//                        t+1 (plus su, ru at t = 0 for the thread t = 0).
// Row update (R9, R10): c = a - b; z = -(lambda + y + rho c)/(beta + rho);
// y += rho (c + z); next target (b - z) - y/rho.  A pending outer update
// (lambda <- clip(lambda + beta z), beta <- beta_next) decided by the last
// finish kernel is applied to each row right before its z-update.
#pragma once
#include "common.cuh"

namespace ucac {

struct RowCtx {
  double beta, beta_cur, lam_max;
  bool pend;
};

__device__ __forceinline__ RowCtx row_ctx(const Dev &S, int k) {
  const double *c = S.ctrl + (long long)k * NCTRL;
  RowCtx R;
  R.pend = c[C_PEND] != 0.0;
  R.beta_cur = c[C_BETA];
  R.beta = R.pend ? c[C_BNEXT] : c[C_BETA];
  R.lam_max = S.prm.lam_max;
  return R;
}

// x-step target of a row from its x-bar value b: (b - z) - y/rho, each
// operation rounded separately (the UC dynamic program's inputs depend on it
// bit for bit).
__device__ __forceinline__ double row_target(double b, double z, double y, double rho) {
  return __dsub_rn(__dsub_rn(b, z), __ddiv_rn(y, rho));
}

// x-bar-step target of a row from its x value a: (a + z) + y/rho
__device__ __forceinline__ double row_mtarget(double a, double z, double y, double rho) {
  return (a + z) + y / rho;
}

__device__ __forceinline__ void row_update(double *A, double *Y, double *Z, double *L, double *Tg, long long idx,
                                           double b_new, double b_old, double rho, const RowCtx &R,
                                           double (&q)[NQ]) {
  const double a = A[idx], y = Y[idx], z = Z[idx];
  double lam = L[idx];
  if (R.pend) {
    lam = clampd(lam + R.beta_cur * z, -R.lam_max, R.lam_max);
    L[idx] = lam;
  }
  const double c = a - b_new;
  const double zn = -(lam + y + rho * c) / (R.beta + rho);
  const double yn = y + rho * (c + zn);
  Z[idx] = zn;
  Y[idx] = yn;
  Tg[idx] = row_target(b_new, zn, yn, rho);
  q[Q_SP] += (c + zn) * (c + zn);
  q[Q_SD] += (b_new - b_old) * (b_new - b_old);
  q[Q_SZ] += zn * zn;
  q[Q_INF] = fmax(q[Q_INF], fabs(c));
}

// ------------------------------------------------------------ bus (R8) ----
template <int BS>
__global__ void __launch_bounds__(BS) k_bus(Dev S) {
  const int b = blockIdx.x;
  const int k = S.b_up.inst[b];
  const Inst I = S.inst[k];
  const long long up = (long long)S.b_up.first[b] + threadIdx.x;
  double q[NQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (up < (long long)I.upo + (long long)I.T * I.nb) {
    const int loc = (int)(up - I.upo);
    const int t = loc / I.nb, i = loc - t * I.nb, ig = I.uo + i;
    const long long NGP = S.NGP, NBP = S.NBP, NUP = S.NUP;
    const RowCtx R = row_ctx(S, k);
    const double rpq = I.rpq, rva = I.rva, irpq = 1.0 / rpq;
    const bool last = (t == I.T - 1);
    const int g0 = S.gen_ptr[ig], g1 = S.gen_ptr[ig + 1], e0 = S.inc_ptr[ig], e1 = S.inc_ptr[ig + 1];
    // pass 1: targets m_v, weights W_v and the 2x2 multiplier system
    double M00 = 0.0, M01 = 0.0, M11 = 0.0, r0 = 0.0, r1 = 0.0, mw = 0.0, mth = 0.0;
    for (int e = g0; e < g1; ++e) {
      const long long gp = (long long)I.gpo + (long long)t * I.ng + S.gen_idx[e];
      double num = rpq * row_mtarget(S.GA[GR_GP * NGP + gp], S.GZ[GR_GP * NGP + gp], S.GY[GR_GP * NGP + gp], rpq);
      double W = rpq;
      if (!last) {
        const long long gn = gp + I.ng;
        num += rpq * row_mtarget(S.GA[GR_TC * NGP + gn], S.GZ[GR_TC * NGP + gn], S.GY[GR_TC * NGP + gn], rpq);
        W += rpq;
      }
      M00 += 1.0 / W;
      r0 += num / W;
      M11 += irpq;
      r1 += row_mtarget(S.GA[GR_GQ * NGP + gp], S.GZ[GR_GQ * NGP + gp], S.GY[GR_GQ * NGP + gp], rpq);
    }
    for (int e = e0; e < e1; ++e) {
      const long long bp = (long long)I.bpo + (long long)t * I.nl + S.inc_br[e];
      const int sd = S.inc_side[e];
      const int rp = sd ? 2 : 0, rw = sd ? 5 : 4;
      M00 += irpq;
      r0 -= row_mtarget(S.BA[rp * NBP + bp], S.BZ[rp * NBP + bp], S.BY[rp * NBP + bp], rpq);
      M11 += irpq;
      r1 -= row_mtarget(S.BA[(rp + 1) * NBP + bp], S.BZ[(rp + 1) * NBP + bp], S.BY[(rp + 1) * NBP + bp], rpq);
      mw += row_mtarget(S.BA[rw * NBP + bp], S.BZ[rw * NBP + bp], S.BY[rw * NBP + bp], rva);
      mth += row_mtarget(S.BA[(rw + 2) * NBP + bp], S.BZ[(rw + 2) * NBP + bp], S.BY[(rw + 2) * NBP + bp], rva);
    }
    const int deg = e1 - e0;
    mw /= deg;
    mth /= deg;
    const double Ww = rva * deg, aPw = -S.Gs[ig], aQw = S.Bs[ig];
    M00 += aPw * aPw / Ww;
    M01 += aPw * aQw / Ww;
    M11 += aQw * aQw / Ww;
    r0 += aPw * mw - S.Pd[up];
    r1 += aQw * mw - S.Qd[up];
    double nuP, nuQ;
    if (M01 == 0.0) {
      nuP = (M00 > 0.0) ? r0 / M00 : 0.0;
      nuQ = (M11 > 0.0) ? r1 / M11 : 0.0;
    } else {
      const double det = M00 * M11 - M01 * M01;
      nuP = (M11 * r0 - M01 * r1) / det;
      nuQ = (M00 * r1 - M01 * r0) / det;
    }
    // pass 2: new x-bar values, then the rows they own
    for (int e = g0; e < g1; ++e) {
      const long long gp = (long long)I.gpo + (long long)t * I.ng + S.gen_idx[e];
      const long long gn = gp + I.ng;
      double num = rpq * row_mtarget(S.GA[GR_GP * NGP + gp], S.GZ[GR_GP * NGP + gp], S.GY[GR_GP * NGP + gp], rpq);
      double W = rpq;
      if (!last) {
        num += rpq * row_mtarget(S.GA[GR_TC * NGP + gn], S.GZ[GR_TC * NGP + gn], S.GY[GR_TC * NGP + gn], rpq);
        W += rpq;
      }
      const double pnew = num / W - nuP / W;
      const double qnew = row_mtarget(S.GA[GR_GQ * NGP + gp], S.GZ[GR_GQ * NGP + gp], S.GY[GR_GQ * NGP + gp], rpq) -
                          nuQ * irpq;
      const double pold = S.G[F_PBAR * NGP + gp], qold = S.G[F_QBAR * NGP + gp];
      S.G[F_PBAR * NGP + gp] = pnew;
      S.G[F_QBAR * NGP + gp] = qnew;
      row_update(S.GA + GR_GP * NGP, S.GY + GR_GP * NGP, S.GZ + GR_GP * NGP, S.GL + GR_GP * NGP,
                 S.GT + GR_GP * NGP, gp, pnew, pold, rpq, R, q);
      if (!last)
        row_update(S.GA + GR_TC * NGP, S.GY + GR_TC * NGP, S.GZ + GR_TC * NGP, S.GL + GR_TC * NGP,
                   S.GT + GR_TC * NGP, gn, pnew, pold, rpq, R, q);
      row_update(S.GA + GR_GQ * NGP, S.GY + GR_GQ * NGP, S.GZ + GR_GQ * NGP, S.GL + GR_GQ * NGP,
                 S.GT + GR_GQ * NGP, gp, qnew, qold, rpq, R, q);
    }
    const double wold = S.U[FU_W * NUP + up], thold = S.U[FU_TH * NUP + up];
    const double wnew = mw - (nuP * aPw + nuQ * aQw) / Ww;
    const double thnew = (i == I.ref) ? 0.0 : mth;
    S.U[FU_W * NUP + up] = wnew;
    S.U[FU_TH * NUP + up] = thnew;
    for (int e = e0; e < e1; ++e) {
      const long long bp = (long long)I.bpo + (long long)t * I.nl + S.inc_br[e];
      const int sd = S.inc_side[e];
      const int rp = sd ? 2 : 0, rw = sd ? 5 : 4;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int r = rp + u;
        const double m = row_mtarget(S.BA[r * NBP + bp], S.BZ[r * NBP + bp], S.BY[r * NBP + bp], rpq);
        const double vnew = m + (u == 0 ? nuP : nuQ) * irpq;
        const double vold = S.B[(FB_FB0 + r) * NBP + bp];
        S.B[(FB_FB0 + r) * NBP + bp] = vnew;
        row_update(S.BA + r * NBP, S.BY + r * NBP, S.BZ + r * NBP, S.BL + r * NBP, S.BT + r * NBP, bp, vnew,
                   vold, rpq, R, q);
      }
      row_update(S.BA + rw * NBP, S.BY + rw * NBP, S.BZ + rw * NBP, S.BL + rw * NBP, S.BT + rw * NBP, bp, wnew,
                 wold, rva, R, q);
      row_update(S.BA + (rw + 2) * NBP, S.BY + (rw + 2) * NBP, S.BZ + (rw + 2) * NBP, S.BL + (rw + 2) * NBP,
                 S.BT + (rw + 2) * NBP, bp, thnew, thold, rva, R, q);
    }
  }
  block_reduce_q<BS>(q, S.part_up + (long long)b * NQ);
}

// ------------------------------------------------------ x-bar^UC (R7) -----
// min 1/2 x^T H x - g^T x over [0,1]^n (n = 2 or 3) by enumerating the 3^n
// faces: on each face the free coordinates solve the reduced system (masked
// 3x3 Cholesky); candidates inside the box whose fixed coordinates satisfy
// the KKT sign conditions are kept, least objective wins (fallback: least
// objective among in-box candidates).
__device__ __forceinline__ void boxqp3(int n, const double (&H)[3][3], const double (&gv)[3], double (&x)[3]) {
  double scale = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < n) scale = fmax(scale, fabs(gv[i]));
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (i < n && j < n) scale = fmax(scale, fabs(H[i][j]));
  }
  const double tolx = 1e-12, tolg = 1e-12 * scale;
  double best = INFINITY, bestf = INFINITY;
  double xb[3] = {0.0, 0.0, 0.0}, xf[3] = {0.0, 0.0, 0.0};
  bool have = false, havef = false;
  for (int face = 0; face < 27; ++face) {
    int st[3] = {face % 3, (face / 3) % 3, face / 9};  // 0 free, 1 at 0, 2 at 1
    if (n == 2 && st[2] != 0) continue;
    if (n == 2) st[2] = 1;  // absent coordinate pinned at 0
    double A[3][3], rhs[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const bool fi = (st[i] == 0);
      double r = gv[i];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const bool fj = (st[j] == 0);
        const double xj = (st[j] == 2) ? 1.0 : 0.0;
        if (!fj) r -= H[i][j] * xj;
        A[i][j] = (fi && fj) ? H[i][j] : ((i == j) ? 1.0 : 0.0);
      }
      rhs[i] = fi ? r : ((st[i] == 2) ? 1.0 : 0.0);
    }
    // 3x3 Cholesky
    bool ok = true;
    double L00 = 0, L10 = 0, L11 = 0, L20 = 0, L21 = 0, L22 = 0;
    {
      double s = A[0][0];
      if (!(s > 0.0)) ok = false;
      L00 = sqrt(fmax(s, 0.0));
      L10 = A[1][0] / L00;
      L20 = A[2][0] / L00;
      s = A[1][1] - L10 * L10;
      if (!(s > 0.0)) ok = false;
      L11 = sqrt(fmax(s, 0.0));
      L21 = (A[2][1] - L20 * L10) / L11;
      s = A[2][2] - L20 * L20 - L21 * L21;
      if (!(s > 0.0)) ok = false;
      L22 = sqrt(fmax(s, 0.0));
    }
    if (!ok) continue;
    double y0 = rhs[0] / L00;
    double y1 = (rhs[1] - L10 * y0) / L11;
    double y2 = (rhs[2] - L20 * y0 - L21 * y1) / L22;
    double xc[3];
    xc[2] = y2 / L22;
    xc[1] = (y1 - L21 * xc[2]) / L11;
    xc[0] = (y0 - L10 * xc[1] - L20 * xc[2]) / L00;
    bool inbox = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i >= n) continue;
      if (st[i] != 0) xc[i] = (st[i] == 2) ? 1.0 : 0.0;
      if (xc[i] < -tolx || xc[i] > 1.0 + tolx) inbox = false;
    }
    if (n == 2) xc[2] = 0.0;
    if (!inbox) continue;
    double fval = 0.0, gr[3];
    bool kkt = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i >= n) continue;
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (j < n) t += H[i][j] * xc[j];
      gr[i] = t - gv[i];
      fval += 0.5 * xc[i] * t - gv[i] * xc[i];
      if (st[i] == 1 && gr[i] < -tolg) kkt = false;
      if (st[i] == 2 && gr[i] > tolg) kkt = false;
    }
    if (fval < bestf) {
      bestf = fval;
      xf[0] = xc[0]; xf[1] = xc[1]; xf[2] = xc[2];
      havef = true;
    }
    if (kkt && fval < best) {
      best = fval;
      xb[0] = xc[0]; xb[1] = xc[1]; xb[2] = xc[2];
      have = true;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) x[i] = clampd(have ? xb[i] : (havef ? xf[i] : 0.0), 0.0, 1.0);
}

template <int BS>
__global__ void __launch_bounds__(BS) k_ucbar(Dev S) {
  const int b = blockIdx.x;
  const int k = S.b_gp.inst[b];
  const Inst I = S.inst[k];
  const long long gp = (long long)S.b_gp.first[b] + threadIdx.x;
  double q[NQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (gp < (long long)I.gpo + (long long)I.T * I.ng) {
    const int loc = (int)(gp - I.gpo);
    const int tau = loc / I.ng, g = loc - tau * I.ng, gg = I.go + g;
    const long long NGP = S.NGP;
    const bool has_next = tau < I.T - 1;
    const long long gn = gp + I.ng;
    const RowCtx R = row_ctx(S, k);
    const double rpq = I.rpq, ruc = I.ruc;
    const double Pmin = S.Pmin[gg], Pmax = S.Pmax[gg], Qmin = S.Qmin[gg], Qmax = S.Qmax[gg];
    const double RU = S.RU[gg], RD = S.RD[gg], SU = S.SU[gg], SD = S.SD[gg];
#define MT(r, idx, rho) row_mtarget(S.GA[(r)*NGP + (idx)], S.GZ[(r)*NGP + (idx)], S.GY[(r)*NGP + (idx)], rho)
    double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gv[3] = {0, 0, 0};
    auto addrow = [&](double w, double m, double e0, double e1, double e2) {
      const double e[3] = {e0, e1, e2};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gv[a] += w * m * e[a];
#pragma unroll
        for (int c = 0; c < 3; ++c) H[a][c] += w * e[a] * e[c];
      }
    };
    addrow(ruc, MT(GR_ON, gp, ruc), 1.0, 0.0, 0.0);
    addrow(ruc, MT(GR_SD, gp, ruc), 0.0, 1.0, 0.0);
    addrow(rpq, MT(GR_PL, gp, rpq), Pmin, 0.0, 0.0);
    addrow(rpq, MT(GR_PU, gp, rpq), Pmax, 0.0, 0.0);
    addrow(rpq, MT(GR_QL, gp, rpq), Qmin, 0.0, 0.0);
    addrow(rpq, MT(GR_QU, gp, rpq), Qmax, 0.0, 0.0);
    addrow(rpq, MT(GR_RD, gp, rpq), -RD, -SD, 0.0);
    if (has_next) {
      addrow(ruc, MT(GR_SU, gn, ruc), 0.0, 0.0, 1.0);
      addrow(rpq, MT(GR_RU, gn, rpq), RU, 0.0, SU);
    }
    double x[3];
    boxqp3(has_next ? 3 : 2, H, gv, x);
    // lone block: ubar_su at t = 0 (ubar_on before period 1 is the data u0)
    double su0 = 0.0;
    const double u0 = (double)S.u0[gg];
    if (tau == 0) {
      const double Hs = ruc + rpq * SU * SU;
      const double gs = ruc * MT(GR_SU, gp, ruc) + rpq * SU * (MT(GR_RU, gp, rpq) - RU * u0);
      su0 = clampd(gs / Hs, 0.0, 1.0);
    }
#undef MT
    const double on_old = S.G[F_UBON * NGP + gp], sd_old = S.G[F_UBSD * NGP + gp];
    const double su1_old = has_next ? S.G[F_UBSU * NGP + gn] : 0.0;
    const double su0_old = (tau == 0) ? S.G[F_UBSU * NGP + gp] : 0.0;
    const double on = x[0], sdv = x[1], su1 = x[2];
    S.G[F_UBON * NGP + gp] = on;
    S.G[F_UBSD * NGP + gp] = sdv;
    if (has_next) S.G[F_UBSU * NGP + gn] = su1;
    if (tau == 0) S.G[F_UBSU * NGP + gp] = su0;
#define RU_(r, idx, bn, bo, rho) \
  row_update(S.GA + (r)*NGP, S.GY + (r)*NGP, S.GZ + (r)*NGP, S.GL + (r)*NGP, S.GT + (r)*NGP, idx, bn, bo, rho, R, q)
    RU_(GR_ON, gp, on, on_old, ruc);
    RU_(GR_SD, gp, sdv, sd_old, ruc);
    RU_(GR_PL, gp, Pmin * on, Pmin * on_old, rpq);
    RU_(GR_PU, gp, Pmax * on, Pmax * on_old, rpq);
    RU_(GR_QL, gp, Qmin * on, Qmin * on_old, rpq);
    RU_(GR_QU, gp, Qmax * on, Qmax * on_old, rpq);
    RU_(GR_RD, gp, (-RD * on) - SD * sdv, (-RD * on_old) - SD * sd_old, rpq);
    if (has_next) {
      RU_(GR_SU, gn, su1, su1_old, ruc);
      RU_(GR_RU, gn, RU * on + SU * su1, RU * on_old + SU * su1_old, rpq);
    }
    if (tau == 0) {
      RU_(GR_SU, gp, su0, su0_old, ruc);
      RU_(GR_RU, gp, RU * u0 + SU * su0, RU * u0 + SU * su0_old, rpq);
    }
#undef RU_
    const double p = S.G[F_P * NGP + gp];
    q[Q_OBJ] = S.c2p[gg] * p * p + S.c1p[gg] * p + S.c0[gg] * S.G[F_UON * NGP + gp] +
               S.csu[gg] * S.G[F_USU * NGP + gp] + S.csd[gg] * S.G[F_USD * NGP + gp];
  }
  block_reduce_q<BS>(q, S.part_gp + (long long)b * NQ);
}

// ------------------------------------------------------------ finish -------
// One block per instance: fixed-order reduction of the block partials, the
// residual record, and the inner/outer control of Algorithm 1 (inner stop when
// r_p, r_d <= eps_in or after L_max sweeps; converged when additionally
// z_rms <= eps_out; otherwise schedule lambda <- lambda + beta z and
// beta <- tau beta if |z| > theta |z_prev|).
template <int BS>
__global__ void __launch_bounds__(BS) k_finish(Dev S) {
  const int k = blockIdx.x;
  const Inst I = S.inst[k];
  double q[NQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int bb = I.blk_up0 + threadIdx.x; bb < I.blk_up1; bb += BS) {
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const double v = S.part_up[(long long)bb * NQ + j];
      q[j] = (j == Q_INF) ? fmax(q[j], v) : q[j] + v;
    }
  }
  for (int bb = I.blk_gp0 + threadIdx.x; bb < I.blk_gp1; bb += BS) {
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const double v = S.part_gp[(long long)bb * NQ + j];
      q[j] = (j == Q_INF) ? fmax(q[j], v) : q[j] + v;
    }
  }
  long long st3[3] = {0, 0, 0};
  for (int bb = I.blk_bp0 + threadIdx.x; bb < I.blk_bp1; bb += BS)
#pragma unroll
    for (int j = 0; j < 3; ++j) st3[j] += S.part_bp[(long long)bb * 3 + j];
  __shared__ double out[NQ];
  block_reduce_q<BS>(q, out);
  __shared__ long long sst[3][BS];
#pragma unroll
  for (int j = 0; j < 3; ++j) sst[j][threadIdx.x] = st3[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    long long nw = 0, na = 0, nc = 0;
    for (int j = 0; j < BS; ++j) {
      nw += sst[0][j];
      na += sst[1][j];
      nc += sst[2][j];
    }
    const Params &P = S.prm;
    double *c = S.ctrl + (long long)k * NCTRL;
    double *r = S.res + (long long)k * NRES;
    long long *s = S.stat + (long long)k * 4;
    const double m = (double)I.m_rows;
    const double rp = sqrt(out[Q_SP] / m), rd = sqrt(out[Q_SD] / m), zn = sqrt(out[Q_SZ]);
    const double zr = sqrt(out[Q_SZ] / m);
    r[R_RP] = rp;
    r[R_RD] = rd;
    r[R_ZN] = zn;
    r[R_ZRMS] = zr;
    r[R_INF] = out[Q_INF];
    r[R_OBJ] = out[Q_OBJ];
    s[0] += 1;
    s[1] = nw;
    s[2] = na;
    s[3] = nc;
    if (c[C_PEND] != 0.0) {
      c[C_BETA] = c[C_BNEXT];
      c[C_PEND] = 0.0;
    }
    const bool finite = isfinite(rp) && isfinite(rd) && isfinite(zn);
    r[R_STATUS] = finite ? (c[C_DONE] != 0.0 ? 1.0 : 0.0) : -5.0;
    c[C_LIN] += 1.0;
    const bool inner_ok = (rp <= P.eps_in) && (rd <= P.eps_in);
    if (inner_ok || c[C_LIN] >= (double)P.L_max) {
      if (inner_ok && zr <= P.eps_out) {
        c[C_DONE] = 1.0;
        if (finite) r[R_STATUS] = 1.0;
      } else {
        const double bnext = (c[C_ZPREV] >= 0.0 && zn > P.theta * c[C_ZPREV]) ? P.tau * c[C_BETA] : c[C_BETA];
        c[C_PEND] = 1.0;
        c[C_BNEXT] = bnext;
        c[C_ZPREV] = zn;
        c[C_KOUT] += 1.0;
        c[C_LIN] = 0.0;
      }
    }
  }
}

// ----------------------------------------------------------- targets ------
// x-step targets of every row from the current x-bar, z and y (after create
// or import).  One thread per gen-period and per branch-period.
template <int BS>
__global__ void __launch_bounds__(BS) k_prep_gen(Dev S) {
  const int b = blockIdx.x;
  const int k = S.b_gp.inst[b];
  const Inst I = S.inst[k];
  const long long gp = (long long)S.b_gp.first[b] + threadIdx.x;
  if (gp >= (long long)I.gpo + (long long)I.T * I.ng) return;
  const int loc = (int)(gp - I.gpo);
  const int t = loc / I.ng, g = loc - t * I.ng, gg = I.go + g;
  const long long NGP = S.NGP;
  const double on = S.G[F_UBON * NGP + gp], su = S.G[F_UBSU * NGP + gp], sd = S.G[F_UBSD * NGP + gp];
  const double on_prev = (t > 0) ? S.G[F_UBON * NGP + gp - I.ng] : (double)S.u0[gg];
  double bv[NGR];
  bv[GR_ON] = on;
  bv[GR_SU] = su;
  bv[GR_SD] = sd;
  bv[GR_PL] = S.Pmin[gg] * on;
  bv[GR_PU] = S.Pmax[gg] * on;
  bv[GR_QL] = S.Qmin[gg] * on;
  bv[GR_QU] = S.Qmax[gg] * on;
  bv[GR_RD] = (-S.RD[gg] * on) - S.SD[gg] * sd;
  bv[GR_RU] = S.RU[gg] * on_prev + S.SU[gg] * su;
  bv[GR_GP] = S.G[F_PBAR * NGP + gp];
  bv[GR_GQ] = S.G[F_QBAR * NGP + gp];
  bv[GR_TC] = (t > 0) ? S.G[F_PBAR * NGP + gp - I.ng] : 0.0;
#pragma unroll
  for (int r = 0; r < NGR; ++r) {
    const double rho = (r <= GR_SD) ? I.ruc : I.rpq;
    S.GT[r * NGP + gp] = row_target(bv[r], S.GZ[r * NGP + gp], S.GY[r * NGP + gp], rho);
  }
}

template <int BS>
__global__ void __launch_bounds__(BS) k_prep_branch(Dev S) {
  const int b = blockIdx.x;
  const int k = S.b_bp.inst[b];
  const Inst I = S.inst[k];
  const long long bp = (long long)S.b_bp.first[b] + threadIdx.x;
  if (bp >= (long long)I.bpo + (long long)I.T * I.nl) return;
  const int loc = (int)(bp - I.bpo);
  const int t = loc / I.nl, l = loc - t * I.nl;
  const long long NBP = S.NBP, NUP = S.NUP, lg = (long long)I.lo + l;
  const long long uf = (long long)I.upo + (long long)t * I.nb + S.bf[lg];
  const long long ut = (long long)I.upo + (long long)t * I.nb + S.bt[lg];
  double bv[8];
#pragma unroll
  for (int r = 0; r < 4; ++r) bv[r] = S.B[(FB_FB0 + r) * NBP + bp];
  bv[4] = S.U[FU_W * NUP + uf];
  bv[5] = S.U[FU_W * NUP + ut];
  bv[6] = S.U[FU_TH * NUP + uf];
  bv[7] = S.U[FU_TH * NUP + ut];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const double rho = (r < 4) ? I.rpq : I.rva;
    S.BT[r * NBP + bp] = row_target(bv[r], S.BZ[r * NBP + bp], S.BY[r * NBP + bp], rho);
  }
}

}  // namespace ucac
