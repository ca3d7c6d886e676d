// k_gen.cuh -- generator x-update per (t, g) (Eq. step:opf for the generator
// component, with the UC coupling rows of Eq. pg_lo .. ramp_up).
//
// Variables p in [0, Pmax], q in [min(0,Qmin), Qmax], phat in [0, Pmax] (the
// generator's copy of p_{t-1}; the period-0 output p0 is data) and six slacks
// s >= 0.  Objective: c2' p^2 + c1' p + rho/2 sum_r (a_r - t_r)^2 over the
// rows pl, pu, ql, qu, rd, ru, gp, gq, tc, with targets t_r = b_r - z_r -
// y_r/rho written by the x-bar kernels.  Each slack appears in one row, so
// minimising it out leaves rho/2 min(0, .)^2 or rho/2 max(0, .)^2 terms:
// a convex C^1 piecewise quadratic.  q separates from (p, phat).
//
// Exact solution by enumerating pieces: the p-terms have three regimes
// (split at t_pl, t_pu), the ramp terms three regimes in d = p - phat (split
// at t_rd, t_ru).  The global minimiser lies in some closed cell and is the
// box-constrained minimiser of that cell's quadratic, so the candidate whose
// point lies in its own cell (least violation, to absorb rounding) is the
// answer.  The piece of the previous iterate is tried first (near convergence
// it is the answer, so one piece is solved instead of nine), then its
// neighbours, up to the first whose candidate lies in its own cell.  Pure FP64
// register arithmetic, one thread per gen-period.
#pragma once
#include "common.cuh"

namespace ucac {

__device__ __forceinline__ double dist_interval(double x, double lo, double hi) {
  return fmax(fmax(lo - x, x - hi), 0.0);
}

// regime r of a pair of breakpoints (lo side term "below", hi side term "above")
// r = 0: x < min(bl, bh); r = 1: between; r = 2: x > max(bl, bh).
// Active flags: below-term (x < bl) and above-term (x > bh).
__device__ __forceinline__ void regime(int r, double bl, double bh, int &act_lo, int &act_hi, double &ilo,
                                       double &ihi) {
  const double mn = fmin(bl, bh), mx = fmax(bl, bh);
  if (r == 0) {
    act_lo = 1; act_hi = 0; ilo = -INFINITY; ihi = mn;
  } else if (r == 1) {
    const int both = bl > bh;
    act_lo = both; act_hi = both; ilo = mn; ihi = mx;
  } else {
    act_lo = 0; act_hi = 1; ilo = mx; ihi = INFINITY;
  }
}

struct GenOut {
  double p, q, ph, s[6];
};

__device__ __forceinline__ GenOut gen_solve(double c2p, double c1p, double rho, double pmax, double qlo,
                                            double qhi, double p0, bool has_prev, const double (&tg)[9],
                                            double p_prev, double ph_prev) {
  const double t_pl = tg[0], t_pu = tg[1], t_ql = tg[2], t_qu = tg[3], t_rd = tg[4], t_ru = tg[5];
  const double t_gp = tg[6], t_gq = tg[7], t_tc = tg[8];
  GenOut o;
  // ---- q: root of rho[(q - t_gq) + min(0, q - t_ql) + max(0, q - t_qu)] on
  // [qlo, qhi].  D is increasing and linear between its breakpoints t_ql,
  // t_qu, so its sign at the two breakpoints picks the piece that holds the
  // unconstrained root, and that root clamped to [qlo, qhi] is the root on
  // the interval.  The piece's root divides by its slope k = 1, 2 or 3
  // (k = 3 only when the targets cross, t_ql > t_qu)
  {
    auto D = [&](double q) { return (q - t_gq) + fmin(q - t_ql, 0.0) + fmax(q - t_qu, 0.0); };
    const int r = D(fmin(t_ql, t_qu)) >= 0.0 ? 0 : (D(fmax(t_ql, t_qu)) >= 0.0 ? 1 : 2);
    int al, ah;
    double ilo, ihi;
    regime(r, t_ql, t_qu, al, ah, ilo, ihi);
    const double num = t_gq + (al ? t_ql : 0.0) + (ah ? t_qu : 0.0);
    const int k = 1 + al + ah;
    o.q = clampd(k == 1 ? num : (k == 2 ? 0.5 * num : num / 3.0), qlo, qhi);
  }
  // ---- (p, phat): candidate of piece (i, j) and its distance from its cell
  auto piece = [&](int i, int j, double &pc, double &phc) -> double {
    int apl, apu, ard, aru;
    double plo, phi, dlo, dhi;
    regime(i, t_pl, t_pu, apl, apu, plo, phi);
    regime(j, t_rd, t_ru, ard, aru, dlo, dhi);
    // d/dp of the p-terms: alpha p - beta; d/dd of the ramp terms: gamma d - delta
    const double alpha = 2.0 * c2p + rho * (1.0 + apl + apu);
    const double beta = -c1p + rho * (t_gp + (apl ? t_pl : 0.0) + (apu ? t_pu : 0.0));
    const double gamma = rho * (ard + aru);
    const double delta = rho * ((ard ? t_rd : 0.0) + (aru ? t_ru : 0.0));
    if (!has_prev) {
      phc = p0;
      pc = clampd((beta + delta + gamma * p0) / (alpha + gamma), 0.0, pmax);
    } else {
      // minimise 1/2 x^T H x - r^T x over [0,pmax]^2, x = (p, phat)
      const double h11 = alpha + gamma, h12 = -gamma, h22 = rho + gamma;
      const double r1 = beta + delta, r2 = rho * t_tc - delta;
      const double idet = 1.0 / (h11 * h22 - h12 * h12);
      pc = (h22 * r1 - h12 * r2) * idet;
      phc = (h11 * r2 - h12 * r1) * idet;
      if (!(pc >= 0.0 && pc <= pmax && phc >= 0.0 && phc <= pmax)) {
        // minimum on the boundary: best of the four clamped edge minimisers
        const double ih11 = 1.0 / h11, ih22 = 1.0 / h22;
        double bq = INFINITY, bp = 0.0, bph = 0.0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          double xp, xh;
          if (e < 2) {
            xp = (e == 0) ? 0.0 : pmax;
            xh = clampd((r2 - h12 * xp) * ih22, 0.0, pmax);
          } else {
            xh = (e == 2) ? 0.0 : pmax;
            xp = clampd((r1 - h12 * xh) * ih11, 0.0, pmax);
          }
          const double qv = 0.5 * (h11 * xp * xp + 2.0 * h12 * xp * xh + h22 * xh * xh) - r1 * xp - r2 * xh;
          if (qv < bq) {
            bq = qv;
            bp = xp;
            bph = xh;
          }
        }
        pc = bp;
        phc = bph;
      }
    }
    return dist_interval(pc, plo, phi) + dist_interval(pc - phc, dlo, dhi);
  };
  auto regime_of = [](double v, double bl, double bh) { return v < fmin(bl, bh) ? 0 : (v > fmax(bl, bh) ? 2 : 1); };
  double p = 0.0, ph = p0;
  // the previous iterate's piece first: near convergence it is the answer
  const double tol = 1e-13 * (1.0 + fmax(fmax(fabs(t_pl), fabs(t_pu)), fmax(fabs(t_rd), fabs(t_ru))));
  const int i0 = regime_of(p_prev, t_pl, t_pu), j0 = regime_of(p_prev - ph_prev, t_rd, t_ru);
  double best = piece(i0, j0, p, ph);
  if (best > tol) {
    // the other eight, the previous piece's neighbours first (offsets
    // modulo 3: one regime over in d, then in p, then both); a piece whose
    // candidate lies in its own cell within tol is the minimiser, as for the
    // first one, so the search stops there (else the least violation wins)
#pragma unroll 1
    for (int q = 1; q < 9; ++q) {
      const int oi = q < 3 ? 0 : (q < 5 ? q - 2 : (q - 5) / 2 + 1), oj = q < 3 ? q : (q < 5 ? 0 : (q - 5) % 2 + 1);
      int i = i0 + oi, j = j0 + oj;
      i = i >= 3 ? i - 3 : i;
      j = j >= 3 ? j - 3 : j;
      double pc, phc;
      const double viol = piece(i, j, pc, phc);
      if (viol < best) {
        best = viol;
        p = pc;
        ph = phc;
      }
      if (best <= tol) break;
    }
  }
  o.p = p;
  o.ph = ph;
  const double d = p - ph;
  o.s[0] = fmax(p - t_pl, 0.0);
  o.s[1] = fmax(t_pu - p, 0.0);
  o.s[2] = fmax(o.q - t_ql, 0.0);
  o.s[3] = fmax(t_qu - o.q, 0.0);
  o.s[4] = fmax(d - t_rd, 0.0);
  o.s[5] = fmax(t_ru - d, 0.0);
  return o;
}

template <int BS>
__global__ void __launch_bounds__(BS) k_gen(Dev S) {
  const int gr = warp_granule<BS>(S.g_gp.n);
  if (gr < 0) return;
  const int k = S.g_gp.inst[gr];
  if (inst_done(S, k)) return;
  const Inst I = S.inst[k];
  const long long gp = (long long)S.g_gp.first[gr] + (threadIdx.x & 31);
  if (gp >= (long long)I.gpo + (long long)I.T * I.ng) return;
  const int loc = (int)(gp - I.gpo);
  const int t = loc / I.ng, g = loc - t * I.ng, gg = I.go + g;
  const long long NGP = S.NGP;
  double tg[9];
  const int rows[9] = {GR_PL, GR_PU, GR_QL, GR_QU, GR_RD, GR_RU, GR_GP, GR_GQ, GR_TC};
#pragma unroll
  for (int r = 0; r < 9; ++r) tg[r] = S.GT[rows[r] * NGP + gp];
  if (t == 0) tg[8] = 0.0;
  const GenOut o = gen_solve(S.c2p[gg], S.c1p[gg], I.rpq, S.Pmax[gg], S.qlo[gg], S.qhi[gg], S.p0[gg], t > 0, tg,
                             S.G[F_P * NGP + gp], S.G[F_PH * NGP + gp]);
  S.G[F_P * NGP + gp] = o.p;
  S.G[F_Q * NGP + gp] = o.q;
  S.G[F_PH * NGP + gp] = o.ph;
#pragma unroll
  for (int r = 0; r < 6; ++r) S.G[(F_SPL + r) * NGP + gp] = o.s[r];
  const double d = o.p - o.ph;
  S.GA[GR_PL * NGP + gp] = o.p - o.s[0];
  S.GA[GR_PU * NGP + gp] = o.p + o.s[1];
  S.GA[GR_QL * NGP + gp] = o.q - o.s[2];
  S.GA[GR_QU * NGP + gp] = o.q + o.s[3];
  S.GA[GR_RD * NGP + gp] = d - o.s[4];
  S.GA[GR_RU * NGP + gp] = d + o.s[5];
  S.GA[GR_GP * NGP + gp] = o.p;
  S.GA[GR_GQ * NGP + gp] = o.q;
  S.GA[GR_TC * NGP + gp] = (t > 0) ? o.ph : 0.0;
}

}  // namespace ucac
