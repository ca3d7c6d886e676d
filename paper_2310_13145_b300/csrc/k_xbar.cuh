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
#include "dword.cuh"

// resident blocks of 128 threads per SM requested for the bus kernel (its
// register cap: 6 gives 80 registers, the fastest of 4 to 8 measured with
// the current double-word conversions; 76 bytes of spills)
#ifndef UCAC_BUS_MINB
#define UCAC_BUS_MINB 6
#endif
// resident blocks of 256 threads per SM requested for the UC box-QP kernel
// (its register cap: 3 gives 80 registers and 24 warps per SM, 168 bytes
// of spills, the fastest of 2, 3 and 4 measured: 0.119 -> 0.113 ms against
// the uncapped 124 registers)
#ifndef UCAC_UCBAR_MINB
#define UCAC_UCBAR_MINB 3
#endif

namespace ucac {

struct RowCtx {
  double beta_cur, lam_max;
  bool pend;
};

__device__ __forceinline__ RowCtx row_ctx(const Dev &S, int k) {
  const double *c = S.ctrl + (long long)k * NCTRL;
  RowCtx R;
  R.pend = c[C_PEND] != 0.0;
  R.beta_cur = c[C_BETA];
  R.lam_max = S.prm.lam_max;
  return R;
}

// Per-family constants of the row update: rho, 1/rho and -1/(beta + rho),
// taken from the instance record, so that no row-update thread divides (a
// division costs the FP64 pipe about as much as ten multiply-adds, and the
// pipe is the bottleneck).
struct Fam {
  double rho, irho, nbr;
};

__device__ __forceinline__ Fam fam_pq(const Inst &I) { return Fam{I.rpq, I.irpq, I.nbpq}; }
__device__ __forceinline__ Fam fam_va(const Inst &I) { return Fam{I.rva, I.irva, I.nbva}; }
__device__ __forceinline__ Fam fam_uc(const Inst &I) { return Fam{I.ruc, I.iruc, I.nbuc}; }

// x-step target of a UC duplicate row from its x-bar value b: (b - z) - y/rho
// with each operation rounded separately and a true division -- the UC
// dynamic program's inputs depend on it bit for bit.
__device__ __forceinline__ double row_target_exact(double b, double z, double y, double rho) {
  return __dsub_rn(__dsub_rn(b, z), __ddiv_rn(y, rho));
}

// The sum w = z + y * (1/rho) of a row, kept beside its targets: the x-step
// target of a row other than the UC duplicates is b - w, the x-bar-step
// target m = a + w (one addition each instead of an addition and a
// multiply-add).  Explicitly rounded, so that the sweep kernels and the
// target preparation after an import produce the same bits.
__device__ __forceinline__ double row_w(double z, double y, double irho) { return __fma_rn(y, irho, z); }
__device__ __forceinline__ double row_target_w(double b, double w) { return __dsub_rn(b, w); }

// Explicitly rounded operations: the x-bar kernels spell out every multiply,
// add and fused multiply-add, so that no template instantiation (block size)
// can contract or reorder them differently -- results are bit-identical
// whatever launch configuration the autotuner picks.
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }

// x-bar-step target of a row from its x value a and its w = z + y/rho
__device__ __forceinline__ double row_mtarget(double a, double w) { return add_(a, w); }

// the outer update of one row, lambda <- clip(lambda + beta z) (Eq. step:outer)
__device__ __forceinline__ double outer_lambda(double lam, double z, const RowCtx &R) {
  return clampd(fma_(R.beta_cur, z, lam), -R.lam_max, R.lam_max);
}

// ------------------------------------------------------------ bus (R8) ----
// The bus kernel's row algebra runs in double-word arithmetic on the FP32
// pipe (dword.cuh).  B300's FP64 unit takes 16 cycles per warp instruction,
// and in FP64 each coupling row cost ~17 such instructions, which held the
// kernel at a quarter of the HBM bandwidth.  The loads enter as double-words
// truncated on the integer units; the row's z and y are rounded once to FP64
// for the state, and its w = z + y/rho and next x-step target b - w are then
// formed from those FP64 values by the explicitly rounded FP64 operations of
// the target preparation (row_w, row_target_w), so that a run resumed from an
// exported state reproduces them bit for bit.  The x-bar step's targets
// a + w and their sums over the bus stay FP64 too (pass 1: two additions per
// row); the 2x2 multiplier solve, the new x-bar values, z, y and the
// residual sums are double-words, accurate to ~2^-46 relative per operation.
__device__ __forceinline__ dw W_(double x) { return dw_from_d(x); }

struct FamW {
  dw rho, nbr;
  double irho;
};
__device__ __forceinline__ FamW fam_w(const Fam &F) { return FamW{W_(F.rho), W_(F.nbr), F.irho}; }

// residual partials of one bus thread: sums of squares of the primal
// residual, of the x-bar change and of z, and the largest |c| (as a
// magnitude ih + il)
struct QAcc {
  dw sp, sd, sz;
  float ih, il;
};
__device__ __forceinline__ void qacc_inf(QAcc &Q, dw c) {
  const float ah = fabsf(c.h), al = c.h < 0.0f ? -c.l : c.l;
  if (ah > Q.ih || (ah == Q.ih && al > Q.il)) {
    Q.ih = ah;
    Q.il = al;
  }
}

// the row update from its loaded inputs a, y, lambda and the new x-bar value
// b (double-word; bd its stored FP64 value), stored: z, y, w and the next
// target (R9, R10: c = a - b; z = -(lambda + y + rho c)/(beta + rho);
// y += rho (c + z)); SD: accumulate (b - b_old)^2 here
__device__ __forceinline__ void row_dw(double *Y, double *Z, double *Tg, double *Wr, long long idx, dw a, dw y,
                                       dw lam, dw b, double bd, dw bold, const FamW &F, QAcc &Q, bool sd) {
  const dw c = dw_sub(a, b);
  const dw z = dw_mul(dw_fma(F.rho, c, dw_add(lam, y)), F.nbr);
  const dw cz = dw_add(c, z);
  const dw yn = dw_fma(F.rho, cz, y);
  Q.sp = dw_fma(cz, cz, Q.sp);
  // (rows whose square the caller adds once, the w and theta rows of the
  // line ends, pass sd = false: warp-uniform there, it skips the 26
  // operations of a zero square, which would leave Q.sd unchanged)
  if (sd) {
    const dw db = dw_sub(b, bold);
    Q.sd = dw_fma(db, db, Q.sd);
  }
  Q.sz = dw_fma(z, z, Q.sz);
  qacc_inf(Q, c);
  const double zd = dw_to_d(z), yd = dw_to_d(yn);
  const double w = row_w(zd, yd, F.irho);
  Z[idx] = zd;
  Y[idx] = yd;
  Wr[idx] = w;
  Tg[idx] = row_target_w(bd, w);
}

// x-bar-step target a + w of a row, from its FP64 x value and w
__device__ __forceinline__ dw row_mtarget_dw(double a, double w) { return dw_add(W_(a), W_(w)); }

// One warp per (period, block of 32 buses in the instance's degree order):
// the lanes' j-th incident line ends are adjacent slots, so every load and
// store of a line-end row is one coalesced 256-byte access; the lanes of a
// block have (nearly) equal degrees, which keeps the warp converged.
template <int BS>
__global__ void __launch_bounds__(BS, (UCAC_BUS_MINB * 128) / BS) k_bus(Dev S) {
  const int gr = warp_granule<BS>(S.g_up.n);
  if (gr < 0) return;
  const int k = S.g_up.inst[gr];
  if (inst_done(S, k)) return;  // (warp-uniform: a granule is one instance)
  const Inst I = S.inst[k];
  const int tb = S.g_up.first[gr];  // t * nblk + block
  const int t = tb / I.nblk, blk = tb - t * I.nblk;
  const int lane = threadIdx.x & 31, pos = blk * 32 + lane;
  QAcc Q{dw_make(0.0f), dw_make(0.0f), dw_make(0.0f), 0.0f, 0.0f};
  if (pos < I.nb) {
    const int i0 = S.bus_order[I.uo + pos];
    const int i = chk_(S, i0 >= 0 && i0 < I.nb, 10) ? i0 : 0, ig = I.uo + i;
    const long long up = (long long)I.upo + (long long)t * I.nb + i;
    const long long NGP = S.NGP, NEP = S.NEP, NUP = S.NUP;
    const long long e0 = I.eo + (long long)t * I.spp + S.blk_off[I.bo + blk] + lane;  // slot 0 of this bus
    const RowCtx R = row_ctx(S, k);
    const FamW Fpq = fam_w(fam_pq(I)), Fva = fam_w(fam_va(I));
    const dw irpq = W_(I.irpq);
    const bool last = (t == I.T - 1);
    const int d0 = S.inc_ptr[ig + 1] - S.inc_ptr[ig];
    const int deg = chk_(S, e0 >= 0 && (d0 == 0 || e0 + 32LL * (d0 - 1) < NEP), 11) ? d0 : 0;
    const int g0 = S.gen_ptr[ig], g1r = S.gen_ptr[ig + 1];
    const int g1 = chk_(S, g0 >= 0 && g1r >= g0 && g1r <= S.NGEN, 12) ? g1r : g0;
    // pass 1: targets m_v and the right-hand side of the 2x2 multiplier
    // system (its matrix is constant between penalty changes: k_prep_bus).
    // Its sums stay FP64 (two additions per line-end row): in double-words
    // each would take two conversions and two sums, and the kernel's issue
    // slots, not its FP64 pipe, are the scarcer resource (0.338 -> 0.322 ms)
    double r0d = 0.0, r1d = 0.0, mwd = 0.0, mthd = 0.0;
    for (int e = g0; e < g1; ++e) {
      const int gl = S.gen_idx[e];
      if (!chk_(S, gl >= 0 && gl < I.ng, 13)) continue;
      const long long gp = (long long)I.gpo + (long long)t * I.ng + gl;
      double m = row_mtarget(S.GA[GR_GP * NGP + gp], S.GW[GR_GP * NGP + gp]);
      if (!last) {
        const long long gn = gp + I.ng;
        m = mul_(0.5, add_(m, row_mtarget(S.GA[GR_TC * NGP + gn], S.GW[GR_TC * NGP + gn])));
      }
      r0d = add_(r0d, m);
      r1d = add_(r1d, row_mtarget(S.GA[GR_GQ * NGP + gp], S.GW[GR_GQ * NGP + gp]));
    }
    // (the p, q x-bar-step targets are parked in the target slots for pass
    // 2, which overwrites them with the next x-step targets)
#pragma unroll 4
    for (int j = 0; j < deg; ++j) {
      const long long e = e0 + 32LL * j;
      const double mp = row_mtarget(S.EA[e], S.EW[e]);
      const double mq = row_mtarget(S.EA[NEP + e], S.EW[NEP + e]);
      S.ET[e] = mp;
      S.ET[NEP + e] = mq;
      r0d = sub_(r0d, mp);
      r1d = sub_(r1d, mq);
      mwd = add_(mwd, row_mtarget(S.EA[2 * NEP + e], S.EW[2 * NEP + e]));
      mthd = add_(mthd, row_mtarget(S.EA[3 * NEP + e], S.EW[3 * NEP + e]));
    }
    dw r0 = W_(r0d), r1 = W_(r1d), mw = W_(mwd), mth = W_(mthd);
    const float fdeg = (float)deg;
    const dw ideg = W_(S.ideg[ig]);
    mw = dw_mul(mw, ideg);
    mth = dw_mul(mth, ideg);
    const dw iWw = dw_mul(W_(Fva.irho), ideg), aPw = W_(-S.Gs[ig]), aQw = W_(S.Bs[ig]);
    r0 = dw_sub(dw_fma(aPw, mw, r0), W_(S.Pd[up]));
    r1 = dw_sub(dw_fma(aQw, mw, r1), W_(S.Qd[up]));
    const double *cf = S.bus_nu + (last ? 3 * S.NB : 0);
    const dw c0 = W_(cf[ig]), c1 = W_(cf[S.NB + ig]), c2 = W_(cf[2 * S.NB + ig]);
    const dw nuP = dw_fma(c0, r0, dw_neg(dw_mul(c1, r1)));
    const dw nuQ = dw_fma(c2, r1, dw_neg(dw_mul(c1, r0)));
    // a pending outer update first, over every row this thread owns: a
    // separate pass in the few sweeps that carry one, so that the row
    // updates below hold no multiplier clip
    if (R.pend) {
      for (int e = g0; e < g1; ++e) {
        const int gl = S.gen_idx[e];
        if (!chk_(S, gl >= 0 && gl < I.ng, 13)) continue;
        const long long gp = (long long)I.gpo + (long long)t * I.ng + gl;
        const long long r0i = GR_GP * NGP + gp, r1i = GR_TC * NGP + gp + I.ng, r2i = GR_GQ * NGP + gp;
        S.GL[r0i] = outer_lambda(S.GL[r0i], S.GZ[r0i], R);
        if (!last) S.GL[r1i] = outer_lambda(S.GL[r1i], S.GZ[r1i], R);
        S.GL[r2i] = outer_lambda(S.GL[r2i], S.GZ[r2i], R);
      }
      for (int j = 0; j < deg; ++j)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long eu = u * NEP + e0 + 32LL * j;
          S.EL[eu] = outer_lambda(S.EL[eu], S.EZ[eu], R);
        }
    }
    // pass 2: new x-bar values, then the rows they own
    for (int e = g0; e < g1; ++e) {
      const int gl = S.gen_idx[e];
      if (!chk_(S, gl >= 0 && gl < I.ng, 13)) continue;
      const long long gp = (long long)I.gpo + (long long)t * I.ng + gl;
      const long long gn = gp + I.ng;
      dw m = row_mtarget_dw(S.GA[GR_GP * NGP + gp], S.GW[GR_GP * NGP + gp]);
      dw iW = irpq;
      if (!last) {
        m = dw_pow2(dw_add(m, row_mtarget_dw(S.GA[GR_TC * NGP + gn], S.GW[GR_TC * NGP + gn])), 0.5f);
        iW = dw_pow2(irpq, 0.5f);
      }
      const dw pnew = dw_fma(dw_neg(nuP), iW, m);
      const dw qnew = dw_fma(dw_neg(nuQ), irpq, row_mtarget_dw(S.GA[GR_GQ * NGP + gp], S.GW[GR_GQ * NGP + gp]));
      const dw pold = W_(S.G[F_PBAR * NGP + gp]), qold = W_(S.G[F_QBAR * NGP + gp]);
      const double pnd = dw_to_d(pnew), qnd = dw_to_d(qnew);
      S.G[F_PBAR * NGP + gp] = pnd;
      S.G[F_QBAR * NGP + gp] = qnd;
      // rows gp (t), tc (t + 1, absent in the last period) and gq (t)
#pragma unroll 1
      for (int u = 0; u < 3; ++u) {
        if (u == 1 && last) continue;
        const long long ri = (u == 0 ? GR_GP * NGP + gp : (u == 1 ? GR_TC * NGP + gn : GR_GQ * NGP + gp));
        const bool isq = u == 2;
        row_dw(S.GY, S.GZ, S.GT, S.GW, ri, W_(S.GA[ri]), W_(S.GY[ri]), W_(S.GL[ri]), isq ? qnew : pnew,
               isq ? qnd : pnd, isq ? qold : pold, Fpq, Q, true);
      }
    }
    const dw wold = W_(S.U[FU_W * NUP + up]), thold = W_(S.U[FU_TH * NUP + up]);
    const dw wnew = dw_sub(mw, dw_mul(dw_fma(nuP, aPw, dw_mul(nuQ, aQw)), iWw));
    const dw thnew = (i == I.ref) ? dw_make(0.0f) : mth;
    const double wnd = dw_to_d(wnew), thnd = dw_to_d(thnew);
    S.U[FU_W * NUP + up] = wnd;
    S.U[FU_TH * NUP + up] = thnd;
    // every incident w (theta) row has the bus's w (theta) as its x-bar:
    // their x-bar changes enter the dual residual as deg times one square
    const dw dwv = dw_sub(wnew, wold), dth = dw_sub(thnew, thold);
    Q.sd = dw_fma(dw_mul_f(dwv, fdeg), dwv, Q.sd);
    Q.sd = dw_fma(dw_mul_f(dth, fdeg), dth, Q.sd);
    for (int j = 0; j < deg; ++j) {
      const long long e = e0 + 32LL * j;
      // every input of the line end's four rows is loaded before any of
      // its stores (for all the compiler knows a store may alias a later
      // load, so a load placed after a store would cost a round trip of
      // its own): one memory round trip per line end instead of six
      double a[4], y[4], lam[4], mt[2], bo[2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = S.EA[u * NEP + e];
        y[u] = S.EY[u * NEP + e];
        lam[u] = S.EL[u * NEP + e];
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mt[u] = S.ET[u * NEP + e];  // (the x-bar-step target parked by pass 1)
        bo[u] = S.EFB[u * NEP + e];
      }
      const dw vp = dw_fma(nuP, irpq, W_(mt[0])), vq = dw_fma(nuQ, irpq, W_(mt[1]));
      const double vpd = dw_to_d(vp), vqd = dw_to_d(vq);
      S.EFB[e] = vpd;
      S.EFB[NEP + e] = vqd;
      // the rows p, q (x-bar: the line end's new flow copies) and w, theta
      // (x-bar: the bus's w and theta), one body for the four
#pragma unroll 1
      for (int u = 0; u < 4; ++u) {
        const double au = u == 0 ? a[0] : (u == 1 ? a[1] : (u == 2 ? a[2] : a[3]));
        const double yu = u == 0 ? y[0] : (u == 1 ? y[1] : (u == 2 ? y[2] : y[3]));
        const double lu = u == 0 ? lam[0] : (u == 1 ? lam[1] : (u == 2 ? lam[2] : lam[3]));
        const dw bu = u == 0 ? vp : (u == 1 ? vq : (u == 2 ? wnew : thnew));
        const double bud = u == 0 ? vpd : (u == 1 ? vqd : (u == 2 ? wnd : thnd));
        const dw bold = u == 0 ? W_(bo[0]) : (u == 1 ? W_(bo[1]) : bu);
        row_dw(S.EY, S.EZ, S.ET, S.EW, u * NEP + e, W_(au), W_(yu), W_(lu), bu, bud, bold, u < 2 ? Fpq : Fva, Q,
               u < 2);
      }
    }
  }
  double q[NQ] = {dw_to_d(Q.sp), dw_to_d(Q.sd), dw_to_d(Q.sz), dw_to_d(dw{Q.ih, Q.il}), 0.0};
  warp_reduce_q(q, S.part_up + (long long)gr * NQ);
}

// ------------------------------------------------------ x-bar^UC (R7) -----
// min 1/2 x^T H x - g^T x over [0,1]^n (n = 2 or 3): a face fixes each
// coordinate free, at 0 or at 1; on a face the free coordinates solve the
// reduced system (masked 3x3 Cholesky).  A face's point is the answer when it
// lies in the box and the fixed coordinates satisfy the KKT sign conditions
// (the minimiser is unique: H is positive definite).  The face of the previous
// iterate is tried first -- near convergence it is almost always the answer,
// so one face is solved instead of 27; otherwise every face is enumerated and
// the KKT-consistent candidate of least objective is kept (fallback: least
// objective among in-box candidates).
// H of the box QP of generator gg, the same for every period but the last
// (has_next: the su, ru rows of the next period); constant between penalty
// changes.  Rows and weights as listed in k_ucbar.
__device__ __forceinline__ void uc_box_h(const Dev &S, int gg, double rpq, double ruc, bool has_next,
                                         double (&H)[3][3]) {
  const double Pmin = S.Pmin[gg], Pmax = S.Pmax[gg], Qmin = S.Qmin[gg], Qmax = S.Qmax[gg];
  const double RU = S.RU[gg], RD = S.RD[gg], SU = S.SU[gg], SD = S.SD[gg];
  H[0][0] = ruc + rpq * (Pmin * Pmin + Pmax * Pmax + Qmin * Qmin + Qmax * Qmax + RD * RD);
  H[0][1] = rpq * (RD * SD);
  H[1][1] = ruc + rpq * (SD * SD);
  H[0][2] = H[1][2] = H[2][2] = 0.0;
  if (has_next) {
    H[0][0] += rpq * (RU * RU);
    H[0][2] = rpq * (RU * SU);
    H[2][2] = ruc + rpq * (SU * SU);
  }
  H[1][0] = H[0][1];
  H[2][0] = H[0][2];
  H[2][1] = H[1][2];
}

// entries of the inverse table: [variant][free mask][packed (0,0) (0,1)
// (0,2) (1,1) (1,2) (2,2)], each a [NGEN] array
constexpr int UC_HINV_N = 2 * 8 * 6;

struct FaceRes {
  double x[3], f;
  bool inbox, kkt;
  int next[3];  // block principal pivoting: the face to try next
};

// Hv: the generator's inverse table for its variant (k_prep_ucbar), entry
// (mask, q) at Hv[(6 mask + q) NGEN]
__device__ __forceinline__ FaceRes solve_face(int n, const int (&st)[3], const double (&H)[3][3],
                                              const double (&gv)[3], double tolx, double tolg, const double *Hv,
                                              long long NGEN) {
  FaceRes R;
  // free rows: r_i = g_i - sum over the fixed j of H_ij x_j; the free block's
  // inverse (zero outside the block) maps them to the free coordinates
  double rhs[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double r = gv[i];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (st[j] != 0) r -= H[i][j] * ((st[j] == 2) ? 1.0 : 0.0);
    rhs[i] = (st[i] == 0) ? r : 0.0;
  }
  const int mask = (st[0] == 0 ? 1 : 0) | (st[1] == 0 ? 2 : 0) | (st[2] == 0 ? 4 : 0);
  const double *hv = Hv + (long long)mask * 6 * NGEN;
  double Hi[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) Hi[q] = hv[q * NGEN];
  R.x[0] = Hi[0] * rhs[0] + Hi[1] * rhs[1] + Hi[2] * rhs[2];
  R.x[1] = Hi[1] * rhs[0] + Hi[3] * rhs[1] + Hi[4] * rhs[2];
  R.x[2] = Hi[2] * rhs[0] + Hi[4] * rhs[1] + Hi[5] * rhs[2];
  R.inbox = true;
  R.kkt = true;
  R.f = 0.0;
  // (box and sign tests on the integer units, see dkey)
  const long long klo = dkey(-tolx), khi = dkey(1.0 + tolx);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R.next[i] = st[i];
    if (i >= n) continue;
    if (st[i] != 0) R.x[i] = (st[i] == 2) ? 1.0 : 0.0;
    const long long kx = dkey(R.x[i]);
    if (!(kx >= klo && kx <= khi)) R.inbox = false;  // (a NaN's key lies outside)
    if (st[i] == 0 && kx < klo) R.next[i] = 1;       // left the box: fix at the bound crossed
    if (st[i] == 0 && kx > khi) R.next[i] = 2;
  }
  if (n == 2) R.x[2] = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i >= n) continue;
    double t = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (j < n) t += H[i][j] * R.x[j];
    const double gr = t - gv[i];
    R.f += 0.5 * R.x[i] * t - gv[i] * R.x[i];
    if (st[i] == 1 && dkey(gr) < dkey(-tolg)) {
      R.kkt = false;
      R.next[i] = 0;  // the gradient pulls it off its bound: free it
    }
    if (st[i] == 2 && dkey(gr) > dkey(tolg)) {
      R.kkt = false;
      R.next[i] = 0;
    }
  }
  return R;
}

__device__ __forceinline__ void boxqp3(int n, const double (&H)[3][3], const double (&gv)[3], const double (&x0)[3],
                                       double (&x)[3], const double *Hv, long long NGEN) {
  long long bs = 0;  // max |gv_i|, |H_ij| by bit pattern
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i < n) bs = abs_bits(gv[i]) > bs ? abs_bits(gv[i]) : bs;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (i < n && j < n) bs = abs_bits(H[i][j]) > bs ? abs_bits(H[i][j]) : bs;
  }
  const double tolx = 1e-12, tolg = 1e-12 * __longlong_as_double(bs);
  {
    // the previous iterate's face, then up to three block-principal-pivoting
    // steps from it: H is positive definite, so a face whose point is in the
    // box with KKT-consistent signs holds the unique minimiser
    int st[3];
    const long long k0 = dkey(0.0), k1 = dkey(1.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) st[i] = (i >= n) ? 1 : (dkey(x0[i]) <= k0 ? 1 : (dkey(x0[i]) >= k1 ? 2 : 0));
    for (int it = 0; it < 4; ++it) {
      const FaceRes R = solve_face(n, st, H, gv, tolx, tolg, Hv, NGEN);
      if (R.inbox && R.kkt) {
#pragma unroll
        for (int i = 0; i < 3; ++i) x[i] = clampd(R.x[i], 0.0, 1.0);
        return;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) st[i] = R.next[i];
    }
  }
  double best = INFINITY, bestf = INFINITY;
  double xb[3] = {0.0, 0.0, 0.0}, xf[3] = {0.0, 0.0, 0.0};
  bool have = false, havef = false;
  for (int face = 0; face < 27; ++face) {
    int st[3] = {face % 3, (face / 3) % 3, face / 9};
    if (n == 2 && st[2] != 0) continue;
    if (n == 2) st[2] = 1;  // absent coordinate pinned at 0
    const FaceRes R = solve_face(n, st, H, gv, tolx, tolg, Hv, NGEN);
    if (!R.inbox) continue;
    if (R.f < bestf) {
      bestf = R.f;
      xf[0] = R.x[0]; xf[1] = R.x[1]; xf[2] = R.x[2];
      havef = true;
    }
    if (R.kkt && R.f < best) {
      best = R.f;
      xb[0] = R.x[0]; xb[1] = R.x[1]; xb[2] = R.x[2];
      have = true;
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) x[i] = clampd(have ? xb[i] : (havef ? xf[i] : 0.0), 0.0, 1.0);
}

template <int BS>
__global__ void __launch_bounds__(BS, (UCAC_UCBAR_MINB * 256) / BS) k_ucbar(Dev S) {
  const int gr = warp_granule<BS>(S.g_gp.n);
  if (gr < 0) return;
  const int k = S.g_gp.inst[gr];
  if (inst_done(S, k)) return;  // (warp-uniform)
  const Inst I = S.inst[k];
  const long long gp = (long long)S.g_gp.first[gr] + (threadIdx.x & 31);
  double q[NQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (gp < (long long)I.gpo + (long long)I.T * I.ng) {
    const int loc = (int)(gp - I.gpo);
    const int tau = loc / I.ng, g = loc - tau * I.ng, gg = I.go + g;
    const long long NGP = S.NGP;
    const bool has_next = tau < I.T - 1;
    const long long gn = gp + I.ng;
    const RowCtx R = row_ctx(S, k);
    const Fam Fpq = fam_pq(I), Fuc = fam_uc(I);
    const double rpq = I.rpq, ruc = I.ruc;
    const double Pmin = S.Pmin[gg], Pmax = S.Pmax[gg], Qmin = S.Qmin[gg], Qmax = S.Qmax[gg];
    const double RU = S.RU[gg], RD = S.RD[gg], SU = S.SU[gg], SD = S.SD[gg];
#define MT(r, idx, F) row_mtarget(S.GA[(r)*NGP + (idx)], S.GW[(r)*NGP + (idx)])
    // H and gv of the box QP in (u_on, u_sd, u_su at t+1): row r with weight
    // w_r, x-bar-step target m_r and coefficients e_r over the three adds
    // w_r e_r e_r^T to H and w_r m_r e_r to gv.  The rows are
    //   on (ruc; 1, 0, 0), sd (ruc; 0, 1, 0), pl, pu, ql, qu (rpq; Pmin,
    //   Pmax, Qmin, Qmax, 0, 0), rd (rpq; -RD, -SD, 0), and with a next
    //   period su (ruc; 0, 0, 1), ru (rpq; RU, 0, SU);
    // only the nonzero products are formed (the FP64 pipe bounds the kernel).
    const double m_on = MT(GR_ON, gp, Fuc), m_sd = MT(GR_SD, gp, Fuc);
    const double m_pl = MT(GR_PL, gp, Fpq), m_pu = MT(GR_PU, gp, Fpq);
    const double m_ql = MT(GR_QL, gp, Fpq), m_qu = MT(GR_QU, gp, Fpq), m_rd = MT(GR_RD, gp, Fpq);
    double H[3][3], gv[3];
    uc_box_h(S, gg, rpq, ruc, has_next, H);
    gv[0] = ruc * m_on + rpq * (m_pl * Pmin + m_pu * Pmax + m_ql * Qmin + m_qu * Qmax - m_rd * RD);
    gv[1] = ruc * m_sd - rpq * (m_rd * SD);
    gv[2] = 0.0;
    if (has_next) {
      const double m_su = MT(GR_SU, gn, Fuc), m_ru = MT(GR_RU, gn, Fpq);
      gv[0] += rpq * (m_ru * RU);
      gv[2] = ruc * m_su + rpq * (m_ru * SU);
    }
    const double on_old = S.G[F_UBON * NGP + gp], sd_old = S.G[F_UBSD * NGP + gp];
    const double su1_old = has_next ? S.G[F_UBSU * NGP + gn] : 0.0;
    const double su0_old = (tau == 0) ? S.G[F_UBSU * NGP + gp] : 0.0;
    const double x0[3] = {on_old, sd_old, su1_old};
    double x[3];
    boxqp3(has_next ? 3 : 2, H, gv, x0, x, S.uc_hinv + (has_next ? 0LL : 48LL * S.NGEN) + gg, S.NGEN);
    // lone block: ubar_su at t = 0 (ubar_on before period 1 is the data u0)
    double su0 = 0.0;
    const double u0 = (double)S.u0[gg];
    if (tau == 0) {
      const double Hs = ruc + rpq * SU * SU;
      const double gs = ruc * MT(GR_SU, gp, Fuc) + rpq * SU * (MT(GR_RU, gp, Fpq) - RU * u0);
      su0 = clampd(gs / Hs, 0.0, 1.0);
    }
#undef MT
    const double on = x[0], sdv = x[1], su1 = x[2];
    S.G[F_UBON * NGP + gp] = on;
    S.G[F_UBSD * NGP + gp] = sdv;
    if (has_next) S.G[F_UBSU * NGP + gn] = su1;
    if (tau == 0) S.G[F_UBSU * NGP + gp] = su0;
    // the rows: one loop body (double-word row algebra, as in the bus
    // kernel; w and the next target in FP64 from the stored z, y, the UC
    // duplicates' target by row_target_exact), the pending outer update a
    // warp-uniform branch.  Row u: on, sd, pl, pu, ql, qu, rd at t; su, ru at
    // t + 1 (with a next period); su, ru at t = 0 (thread t = 0 only)
    const FamW Wpq = fam_w(Fpq), Wuc = fam_w(Fuc);
    QAcc Q{dw_make(0.0f), dw_make(0.0f), dw_make(0.0f), 0.0f, 0.0f};
#pragma unroll 1
    for (int u = 0; u < 11; ++u) {
      if ((u == 7 || u == 8) && !has_next) continue;
      if (u >= 9 && tau != 0) break;
      int r;
      double bn, bo;
      switch (u) {
        case 0: r = GR_ON; bn = on; bo = on_old; break;
        case 1: r = GR_SD; bn = sdv; bo = sd_old; break;
        case 2: r = GR_PL; bn = Pmin * on; bo = Pmin * on_old; break;
        case 3: r = GR_PU; bn = Pmax * on; bo = Pmax * on_old; break;
        case 4: r = GR_QL; bn = Qmin * on; bo = Qmin * on_old; break;
        case 5: r = GR_QU; bn = Qmax * on; bo = Qmax * on_old; break;
        case 6: r = GR_RD; bn = (-RD * on) - SD * sdv; bo = (-RD * on_old) - SD * sd_old; break;
        case 7: r = GR_SU; bn = su1; bo = su1_old; break;
        case 8: r = GR_RU; bn = RU * on + SU * su1; bo = RU * on_old + SU * su1_old; break;
        case 9: r = GR_SU; bn = su0; bo = su0_old; break;
        default: r = GR_RU; bn = RU * u0 + SU * su0; bo = RU * u0 + SU * su0_old; break;
      }
      const bool uc = r <= GR_SD || r == GR_SU;  // the duplicate rows (rho_uc, exact target)
      const long long ri = (long long)r * NGP + ((u == 7 || u == 8) ? gn : gp);
      double lam = S.GL[ri];
      if (R.pend) {
        lam = outer_lambda(lam, S.GZ[ri], R);
        S.GL[ri] = lam;
      }
      const FamW &F = uc ? Wuc : Wpq;
      const dw b = W_(bn);
      const dw c = dw_sub(W_(S.GA[ri]), b);
      const dw y = W_(S.GY[ri]);
      const dw z = dw_mul(dw_fma(F.rho, c, dw_add(W_(lam), y)), F.nbr);
      const dw cz = dw_add(c, z);
      const dw yn = dw_fma(F.rho, cz, y);
      const dw db = dw_sub(b, W_(bo));
      Q.sp = dw_fma(cz, cz, Q.sp);
      Q.sd = dw_fma(db, db, Q.sd);
      Q.sz = dw_fma(z, z, Q.sz);
      qacc_inf(Q, c);
      const double zd = dw_to_d(z), yd = dw_to_d(yn);
      const double w = row_w(zd, yd, F.irho);
      S.GZ[ri] = zd;
      S.GY[ri] = yd;
      S.GW[ri] = w;
      S.GT[ri] = uc ? row_target_exact(bn, zd, yd, ruc) : row_target_w(bn, w);
    }
    q[Q_SP] = dw_to_d(Q.sp);
    q[Q_SD] = dw_to_d(Q.sd);
    q[Q_SZ] = dw_to_d(Q.sz);
    q[Q_INF] = dw_to_d(dw{Q.ih, Q.il});
    const double p = S.G[F_P * NGP + gp];
    q[Q_OBJ] = S.c2p[gg] * p * p + S.c1p[gg] * p + S.c0[gg] * S.G[F_UON * NGP + gp] +
               S.csu[gg] * S.G[F_USU * NGP + gp] + S.csd[gg] * S.G[F_USD * NGP + gp];
  }
  warp_reduce_q(q, S.part_gp + (long long)gr * NQ);
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
  if (inst_done(S, k)) return;  // converged earlier: the record stays
  const Inst I = S.inst[k];
  double q[NQ] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int up1 = chk_(S, I.gran_up0 >= 0 && I.gran_up1 <= S.g_up.n, 40) ? I.gran_up1 : I.gran_up0;
  const int gp1 = chk_(S, I.gran_gp0 >= 0 && I.gran_gp1 <= S.g_gp.n, 41) ? I.gran_gp1 : I.gran_gp0;
  for (int bb = I.gran_up0 + threadIdx.x; bb < up1; bb += BS) {
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const double v = S.part_up[(long long)bb * NQ + j];
      q[j] = (j == Q_INF) ? fmax(q[j], v) : q[j] + v;
    }
  }
  for (int bb = I.gran_gp0 + threadIdx.x; bb < gp1; bb += BS) {
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const double v = S.part_gp[(long long)bb * NQ + j];
      q[j] = (j == Q_INF) ? fmax(q[j], v) : q[j] + v;
    }
  }
  __shared__ double out[NQ];
  block_reduce_q<BS>(q, out);
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long nw = S.bstat[(long long)k * 3], na = S.bstat[(long long)k * 3 + 1];
    const long long nc = S.bstat[(long long)k * 3 + 2];
    const Params &P = S.prm;
    double *c = S.ctrl + (long long)k * NCTRL;
    double *r = S.res + (long long)k * NRES;
    long long *s = S.stat + (long long)k * 6;
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
    s[4] += nw;
    s[5] += na;
    if (c[C_PEND] != 0.0) {
      c[C_BETA] = c[C_BNEXT];
      c[C_PEND] = 0.0;
    }
    // failure detection: a non-finite residual, a residual past the
    // divergence bound, or (when asked for) a line solve stopped on a cap;
    // the instance then takes no further sweep (stop flag 2)
    const bool finite = isfinite(rp) && isfinite(rd) && isfinite(zn);
    double st = 0.0;
    if (!finite)
      st = (double)UCAC_E_NAN;
    else if (rp > P.div_bound || rd > P.div_bound)
      st = (double)UCAC_E_DIVERGED;
    else if (P.stop_on_cap && nc > 0)
      st = (double)UCAC_E_NEWTON_MAXIT;
    r[R_STATUS] = st;
    r[R_RCHG] = 0.0;
    if (st < 0.0) {
      c[C_DONE] = 2.0;
      return;
    }
    c[C_LIN] += 1.0;
    const bool inner_ok = (rp <= P.eps_in) && (rd <= P.eps_in);
    if (inner_ok || c[C_LIN] >= (double)P.L_max) {
      if (inner_ok && zr <= P.eps_out) {
        c[C_DONE] = 1.0;
        r[R_STATUS] = 1.0;
      } else {
        const double bnext = (c[C_ZPREV] >= 0.0 && zn > P.theta * c[C_ZPREV]) ? P.tau * c[C_BETA] : c[C_BETA];
        c[C_PEND] = 1.0;
        c[C_BNEXT] = bnext;
        c[C_ZPREV] = zn;
        c[C_KOUT] += 1.0;
        c[C_LIN] = 0.0;
      }
    }
    // adaptive penalty by residual balancing (Sec. V names adaptive rules as
    // the way past the penalty sensitivity): every rho_every sweeps, all
    // three penalties grow by rho_tau when r_p > rho_mu r_d and shrink by it
    // when r_d > rho_mu r_p, at most 6 net steps either way from the
    // penalties of create (unbounded, the rule can run away: r_d shrinks as
    // the penalty grows); the sweep's target preparation then rewrites the
    // x-step targets with the new penalties
    if (P.rho_every > 0 && c[C_DONE] == 0.0) {
      c[C_RCNT] += 1.0;
      if (c[C_RCNT] >= (double)P.rho_every) {
        c[C_RCNT] = 0.0;
        const int up = (rp > P.rho_mu * rd && c[C_RLOG] < 6.0) ? 1 : ((rd > P.rho_mu * rp && c[C_RLOG] > -6.0) ? -1 : 0);
        const double sc = up > 0 ? P.rho_tau : (up < 0 ? 1.0 / P.rho_tau : 1.0);
        if (up != 0) {
          c[C_RLOG] += (double)up;
          c[C_RPQ] *= sc;
          c[C_RVA] *= sc;
          c[C_RUC] *= sc;
          Inst *Iw = const_cast<Inst *>(S.inst) + k;
          Iw->rpq = c[C_RPQ];
          Iw->rva = c[C_RVA];
          Iw->ruc = c[C_RUC];
          r[R_RCHG] = 1.0;
        }
      }
    }
    inst_derive(*(const_cast<Inst *>(S.inst) + k), c, S.prm.omega_rel, S.prm.c_max_rel);
  }
}

// instance penalties and their derived constants from the control record
// (after a state import)
__global__ void k_sync_rho(Dev S, int k) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double *c = S.ctrl + (long long)k * NCTRL;
    Inst *Iw = const_cast<Inst *>(S.inst) + k;
    Iw->rpq = c[C_RPQ];
    Iw->rva = c[C_RVA];
    Iw->ruc = c[C_RUC];
    inst_derive(*Iw, c, S.prm.omega_rel, S.prm.c_max_rel);
  }
}

// ----------------------------------------------------------- targets ------
// x-step targets of every row from the current x-bar, z and y (after create
// or import, and after an adaptive-penalty change: changed_only limits the
// pass to instances whose penalties changed in this sweep).  One thread per
// gen-period and per branch-period.
template <int BS>
__global__ void __launch_bounds__(BS) k_prep_gen(Dev S, int changed_only) {
  const int gr = warp_granule<BS>(S.g_gp.n);
  if (gr < 0) return;
  const int k = S.g_gp.inst[gr];
  if (changed_only && S.res[(long long)k * NRES + R_RCHG] == 0.0) return;
  const Inst I = S.inst[k];
  const long long gp = (long long)S.g_gp.first[gr] + (threadIdx.x & 31);
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
  const double irpq = I.irpq, iruc = I.iruc;
#pragma unroll
  for (int r = 0; r < NGR; ++r) {
    const double z = S.GZ[r * NGP + gp], y = S.GY[r * NGP + gp];
    const double w = row_w(z, y, (r <= GR_SD) ? iruc : irpq);
    S.GW[r * NGP + gp] = w;
    S.GT[r * NGP + gp] = (r <= GR_SD) ? row_target_exact(bv[r], z, y, I.ruc) : row_target_w(bv[r], w);
  }
}

template <int BS>
__global__ void __launch_bounds__(BS) k_prep_branch(Dev S, int changed_only) {
  const int gr = warp_granule<BS>(S.g_bp.n);
  if (gr < 0) return;
  const int k = S.g_bp.inst[gr];
  if (changed_only && S.res[(long long)k * NRES + R_RCHG] == 0.0) return;
  const Inst I = S.inst[k];
  const long long bp = (long long)S.g_bp.first[gr] + (threadIdx.x & 31);
  if (bp >= (long long)I.bpo + (long long)I.T * I.nl) return;
  const int loc = (int)(bp - I.bpo);
  const int t = loc / I.nl, l = loc - t * I.nl;
  const long long NEP = S.NEP, NUP = S.NUP, lg = (long long)I.lo + l;
  const long long uf = (long long)I.upo + (long long)t * I.nb + S.bf[lg];
  const long long ut = (long long)I.upo + (long long)t * I.nb + S.bt[lg];
  long long ef, et;
  line_ends(S, I, t, lg, ef, et);
  if (!chk_(S, ef >= 0 && ef < S.NEP && et >= 0 && et < S.NEP, 50)) ef = et = 0;
  double bv[8];
#pragma unroll
  for (int r = 0; r < 4; ++r) bv[r] = S.EFB[erow_u(r) * NEP + (erow_end(r) ? et : ef)];
  bv[4] = S.U[FU_W * NUP + uf];
  bv[5] = S.U[FU_W * NUP + ut];
  bv[6] = S.U[FU_TH * NUP + uf];
  bv[7] = S.U[FU_TH * NUP + ut];
  const double irpq = I.irpq, irva = I.irva;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const long long e = erow_u(r) * NEP + (erow_end(r) ? et : ef);
    const double w = row_w(S.EZ[e], S.EY[e], (r < 4) ? irpq : irva);
    S.EW[e] = w;
    S.ET[e] = row_target_w(bv[r], w);
  }
  if (!changed_only) {
    // the polar line kernel's V_i, V_j and 1/c from the state: sqrt(w)
    // clamped to the voltage band
    const long long NBP = S.NBP, NL = S.NL;
    S.LV[bp] = clampd(sqrt(fmax(S.B[(FB_V0 + 0) * NBP + bp], 0.0)), S.BC[(BC_VB + 0) * NL + lg],
                      S.BC[(BC_VB + 1) * NL + lg]);
    S.LV[NBP + bp] = clampd(sqrt(fmax(S.B[(FB_V0 + 1) * NBP + bp], 0.0)), S.BC[(BC_VB + 2) * NL + lg],
                            S.BC[(BC_VB + 3) * NL + lg]);
    S.LV[2 * NBP + bp] = 1.0 / S.B[FB_C * NBP + bp];
  }
}

// Coefficients of the bus multiplier solve (R8).  The 2x2 system M nu = r
// of bus i has
//   M_PP = sum_g W_g^-1 + deg/rho_pq + Gs^2/(deg rho_va),
//   M_QQ = n_g/rho_pq + deg/rho_pq + Bs^2/(deg rho_va),
//   M_PQ = -Gs Bs/(deg rho_va),
// with W_g = 2 rho_pq for a generator whose p row is averaged with the next
// period's temporal-copy row (every period but the last) and rho_pq in the
// last; so M depends on the penalties and the bus alone.  Its inverse is
// formed here, after create, import and each penalty change, as
// nu_P = c0 r_P - c1 r_Q, nu_Q = c2 r_Q - c1 r_P: [kind][c0, c1, c2][NB],
// kind 0 for t < T - 1 and 1 for t = T - 1.  One thread per bus of
// instance blockIdx.y.
template <int BS>
__global__ void __launch_bounds__(BS) k_prep_bus(Dev S, int changed_only) {
  const int k = blockIdx.y;
  if (changed_only && S.res[(long long)k * NRES + R_RCHG] == 0.0) return;
  const Inst I = S.inst[k];
  const int i = blockIdx.x * BS + threadIdx.x;
  if (i >= I.nb) return;
  const int ig = I.uo + i;
  const double ngen = (double)(S.gen_ptr[ig + 1] - S.gen_ptr[ig]);
  const double fdeg = (double)(S.inc_ptr[ig + 1] - S.inc_ptr[ig]);
  const double irpq = I.irpq, iWw = I.irva * S.ideg[ig], aPw = -S.Gs[ig], aQw = S.Bs[ig];
  for (int kind = 0; kind < 2; ++kind) {
    const double M00 = (kind ? ngen : 0.5 * ngen) * irpq + fdeg * irpq + aPw * aPw * iWw;
    const double M11 = ngen * irpq + fdeg * irpq + aQw * aQw * iWw;
    const double M01 = aPw * aQw * iWw;
    double c0, c1, c2;
    if (M01 == 0.0) {
      c0 = M00 > 0.0 ? 1.0 / M00 : 0.0;
      c1 = 0.0;
      c2 = M11 > 0.0 ? 1.0 / M11 : 0.0;
    } else {
      const double idet = 1.0 / (M00 * M11 - M01 * M01);
      c0 = M11 * idet;
      c1 = M01 * idet;
      c2 = M00 * idet;
    }
    double *cf = S.bus_nu + (long long)kind * 3 * S.NB;
    cf[ig] = c0;
    cf[S.NB + ig] = c1;
    cf[2 * S.NB + ig] = c2;
  }
}

// The UC box QPs' free-block inverses: for each generator of instance
// blockIdx.y, each variant (0: a next period, coordinates on, sd, su; 1: the
// last period, on and sd only) and each mask of free coordinates, the
// inverse of H restricted to the free coordinates (zero outside the block;
// masks that free the absent coordinate of variant 1 stay zero).  H is
// positive definite, so every principal block is invertible.  Formed after
// create, import and each penalty change; one thread per generator.
template <int BS>
__global__ void __launch_bounds__(BS) k_prep_ucbar(Dev S, int changed_only) {
  const int k = blockIdx.y;
  if (changed_only && S.res[(long long)k * NRES + R_RCHG] == 0.0) return;
  const Inst I = S.inst[k];
  const int g = blockIdx.x * BS + threadIdx.x;
  if (g >= I.ng) return;
  const int gg = I.go + g;
  const long long NG = S.NGEN;
  const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
  for (int var = 0; var < 2; ++var) {
    double H[3][3];
    uc_box_h(S, gg, I.rpq, I.ruc, var == 0, H);
    for (int mask = 0; mask < 8; ++mask) {
      double Hi[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
      int f[3], m = 0;
      for (int i = 0; i < 3; ++i)
        if ((mask >> i) & 1) f[m++] = i;
      if (!(var == 1 && (mask & 4))) {
        if (m == 1) {
          Hi[f[0]][f[0]] = 1.0 / H[f[0]][f[0]];
        } else if (m == 2) {
          const double a = H[f[0]][f[0]], b = H[f[0]][f[1]], c = H[f[1]][f[1]];
          const double id = 1.0 / (a * c - b * b);
          Hi[f[0]][f[0]] = c * id;
          Hi[f[0]][f[1]] = Hi[f[1]][f[0]] = -b * id;
          Hi[f[1]][f[1]] = a * id;
        } else if (m == 3) {
          // cofactors of the symmetric 3x3 block
          const double C00 = H[1][1] * H[2][2] - H[1][2] * H[1][2];
          const double C01 = H[0][2] * H[1][2] - H[0][1] * H[2][2];
          const double C02 = H[0][1] * H[1][2] - H[1][1] * H[0][2];
          const double C11 = H[0][0] * H[2][2] - H[0][2] * H[0][2];
          const double C12 = H[0][1] * H[0][2] - H[0][0] * H[1][2];
          const double C22 = H[0][0] * H[1][1] - H[0][1] * H[0][1];
          const double id = 1.0 / (H[0][0] * C00 + H[0][1] * C01 + H[0][2] * C02);
          Hi[0][0] = C00 * id;
          Hi[0][1] = Hi[1][0] = C01 * id;
          Hi[0][2] = Hi[2][0] = C02 * id;
          Hi[1][1] = C11 * id;
          Hi[1][2] = Hi[2][1] = C12 * id;
          Hi[2][2] = C22 * id;
        }
      }
      double *out = S.uc_hinv + ((long long)var * 8 + mask) * 6 * NG + gg;
      for (int q = 0; q < 6; ++q) out[q * NG] = Hi[pi_[q]][pj_[q]];
    }
  }
}

// The line flows of instance k's solution as one [t * nl + l][4] block
// (p_ij, q_ij, p_ji, q_ji: the x values of the four flow rows), gathered from
// the line-end slots for a single copy to the host.
template <int BS>
__global__ void __launch_bounds__(BS) k_solution_flows(Dev S, int k, double *pf) {
  const Inst I = S.inst[k];
  const long long n = (long long)I.T * I.nl;
  const long long loc = (long long)blockIdx.x * BS + threadIdx.x;
  if (loc >= n) return;
  const int t = (int)(loc / I.nl), l = (int)(loc - (long long)t * I.nl);
  long long ef, et;
  line_ends(S, I, t, (long long)I.lo + l, ef, et);
  if (!chk_(S, ef >= 0 && ef < S.NEP && et >= 0 && et < S.NEP, 52)) ef = et = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) pf[loc * 4 + r] = S.EA[erow_u(r) * S.NEP + (erow_end(r) ? et : ef)];
}

// Line-end rows of instance k between the slot layout and the canonical
// [r][t * nl + l] order of the state vector (dir 0: slots -> canon, 1: back).
// arr is a [4][NEP] (or [2][NEP] for the x-bar of p, q) slot array; rows r
// of the canonical block follow erow_u / erow_end (nrows = 8 or 4).
template <int BS>
__global__ void __launch_bounds__(BS) k_edge_canon(Dev S, int k, int dir, double *arr, int nrows, double *canon) {
  const Inst I = S.inst[k];
  const long long n = (long long)I.T * I.nl;
  const long long loc = (long long)blockIdx.x * BS + threadIdx.x;
  if (loc >= n) return;
  const int t = (int)(loc / I.nl), l = (int)(loc - (long long)t * I.nl);
  long long ef, et;
  line_ends(S, I, t, (long long)I.lo + l, ef, et);
  if (!chk_(S, ef >= 0 && ef < S.NEP && et >= 0 && et < S.NEP, 53)) ef = et = 0;
  for (int r = 0; r < nrows; ++r) {
    const long long e = erow_u(r) * S.NEP + (erow_end(r) ? et : ef);
    if (dir == 0)
      canon[(long long)r * n + loc] = arr[e];
    else
      arr[e] = canon[(long long)r * n + loc];
  }
}

}  // namespace ucac
