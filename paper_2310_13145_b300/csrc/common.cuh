// common.cuh -- device-side layout shared by the sweep kernels.
//
// All instances of a handle are concatenated: every per-(period, component)
// array is a structure of arrays over the global item index
//   gen-period     gp = inst.gpo + t * inst.ng + g
//   branch-period  bp = inst.bpo + t * inst.nl + l
//   bus-period     up = inst.upo + t * inst.nb + i
// so one launch covers a whole batch and consecutive threads touch
// consecutive addresses.  The coupling rows of the line ends (p, q, w, theta
// of one end of a line, owned by the bus at that end) are stored in a slot
// layout instead: per instance and period, the buses in degree order are cut
// into blocks of 32 (one warp of the bus kernel), and block b owns W_b slots
// per lane (W_b = its largest degree), slot j of lane l at
//   e = inst.eo + t * inst.spp + blk_off[b] + 32 j + l,
// so the bus kernel's loads of its j-th incident line end are one contiguous
// 256-byte line per warp; the line kernels find their two ends through
// eslot[side][line].  Each warp handles one granule of 32 consecutive
// items of one instance (granule tables never straddle two instances), so
// residual partial sums are per warp and per instance, and the block size of
// a launch changes neither the work split nor any result: it is free to be
// tuned (fixed-order warp partials, fixed-order final sum).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ucac {

// Coupling rows per (t, g) (Eq. uc_duplicate .. ramp_up and the generator
// consensus rows) and per (t, line) (flows, w, theta consensus rows).
enum { GR_ON, GR_SU, GR_SD, GR_PL, GR_PU, GR_QL, GR_QU, GR_RD, GR_RU, GR_GP, GR_GQ, GR_TC, NGR };
enum { NBR = 8 };
// generator-period fields
enum { F_P, F_Q, F_PH, F_SPL, F_SPU, F_SQL, F_SQU, F_SRD, F_SRU, F_UON, F_USU, F_USD, F_PBAR, F_QBAR,
       F_UBON, F_UBSU, F_UBSD, NGF };
// branch-period fields
enum { FB_V0 = 0, FB_MU0 = 8, FB_C = 12, FB_FB0 = 13, NBF = 17 };
// bus-period fields
enum { FU_W, FU_TH, NUF };
// per-instance control scalars
// (C_RPQ..C_RUC: the current penalties, C_RCNT: sweeps since the last
// adaptive-penalty check, C_RLOG: net doublings so far, kept in [-6, 6];
// part of the canonical state)
enum { C_BETA, C_ZPREV, C_LIN, C_KOUT, C_PEND, C_BNEXT, C_DONE, C_RPQ, C_RVA, C_RUC, C_RCNT, C_RLOG, NCTRL };
// residual record
// (R_RCHG: the penalties changed at the end of this sweep)
enum { R_RP, R_RD, R_ZN, R_ZRMS, R_INF, R_OBJ, R_STATUS, R_RCHG, NRES };
// block partial quantities of the x-bar kernels
enum { Q_SP, Q_SD, Q_SZ, Q_INF, Q_OBJ, NQ };
// branch constant table [BC_N][NL]
// (BC_VB: Vmin_i, Vmax_i, Vmin_j, Vmax_j for the polar line solver)
enum { BC_Y0 = 0, BC_RATE2 = 8, BC_LO = 9, BC_HI = 17, BC_VB = 25, BC_N = 29 };

struct Inst {
  int nb, nl, ng, T, ref;
  int go, gpo, lo, bpo, uo, upo;
  long long eo;    // first line-end slot of the instance
  int spp, nblk, bo;  // slots per period, bus blocks per period, first bus block (global)
  int m_rows;
  int gran_gen0, gran_gen1, gran_gp0, gran_gp1, gran_bp0, gran_bp1, gran_up0, gran_up1;
  double rpq, rva, ruc;
  // constants of the next sweep's x-bar row updates: 1/rho of each family,
  // and -1/(beta + rho) with the beta its z-updates use (the scheduled
  // beta_next while an outer update is pending); set by inst_derive whenever
  // a penalty, beta or the pending flag changes, so that no row-update
  // thread divides (the sign is folded in: -(x/(beta + rho)) rounds to the
  // same value as x * (-1/(beta + rho)) with no separate negation)
  double irpq, irva, iruc, nbpq, nbva, nbuc;
  // the line solves' stationarity tolerance omega_rel max(rho) and penalty
  // cap c_max_rel max(rho), and FP32 copies of rho_pq, rho_va (Hessian)
  double omega, cmax;
  float frpq, frva;
};

// the derived constants of I from its penalties and control record c (the
// host at create and the device after each sweep compute the same IEEE
// quotients, so the bits do not depend on where they were formed)
__host__ __device__ inline void inst_derive(Inst &I, const double *c, double omega_rel, double c_max_rel) {
  const double rmax = fmax(I.rpq, I.rva);
  I.omega = omega_rel * rmax;
  I.cmax = c_max_rel * rmax;
  I.frpq = (float)I.rpq;
  I.frva = (float)I.rva;
  const double beta = c[C_PEND] != 0.0 ? c[C_BNEXT] : c[C_BETA];
  I.irpq = 1.0 / I.rpq;
  I.irva = 1.0 / I.rva;
  I.iruc = 1.0 / I.ruc;
  I.nbpq = -1.0 / (beta + I.rpq);
  I.nbva = -1.0 / (beta + I.rva);
  I.nbuc = -1.0 / (beta + I.ruc);
}

struct Params {
  double eps_in, eps_out, tau, theta, beta0, lam_max, eta, omega_rel, c_init_rel, c_max_rel;
  double rho_mu, rho_tau;
  int K_AL, K_N, L_max, line_form, uc_relax, rho_every, stop_on_cap;
  double div_bound;
};

constexpr int GRAN = 32;  // items per granule (one warp)

// cos(k / TRIG_N), sin(k / TRIG_N) for k = -TRIG_K..TRIG_K (|k / TRIG_N| <=
// pi + 1/TRIG_N, 25.8 KB), filled from the host's libm when a handle is
// created (the same values on every device and handle)
constexpr int TRIG_N = 256;
constexpr int TRIG_K = 805;
__device__ double2 g_trig[2 * TRIG_K + 1];

struct Granules {
  int n;
  const int *inst;   // instance of each granule
  const int *first;  // global index of the granule's first item
};

struct Dev {
  int K;
  const Inst *inst;
  Params prm;
  // generator constants [NGEN]
  const double *c2p, *c1p, *c0, *csu, *csd, *Pmin, *Pmax, *Qmin, *Qmax, *qlo, *qhi, *RU, *RD, *SU, *SD, *p0;
  const int *TU, *TD, *u0, *K0;
  // generator-period state [NGF][NGP], rows [NGR][NGP]
  long long NGP;
  double *G, *GA, *GY, *GZ, *GL, *GT, *GW;
  // branch constants [BC_N][NL]
  long long NL;
  const double *BC;
  // FP32 copies of the polar line constants [8][NL]: q_r (Gii, -Bii, Gjj,
  // -Bjj), then ga, ka of the from end (Gij, Bij) and the to end (Gji, -Bji)
  // as ga_0, ga_1, ka_0, ka_1
  const float *BCF;
  const int *bf, *bt;  // local bus index of the from / to end
  // branch-period state [FB_FB0][NBP] (the x-bar values of the flow rows
  // live with the line-end rows)
  long long NBP;
  double *B;
  // the polar line kernel's own copy of V_i, V_j and 1/c of each
  // line-period [3][NBP] (not part of the state: formed from B by the target
  // preparation after create and import, then written by each solve, so
  // that a solve starts without two square roots and a division)
  double *LV;
  // line-end rows in the slot layout: [4][NEP] (p, q, w, theta of the end)
  // for x values, y, z, lambda and x-step targets; x-bar of p, q [2][NEP]
  long long NEP;
  double *EA, *EY, *EZ, *EL, *ET, *EFB, *EW;
  const int *eslot;             // [2][NL]: slot of the from / to end within its period
  const int *blk_off, *blk_w;   // per bus block: slot offset within the period, width
  // buses
  long long NB;
  const double *Gs, *Bs, *ideg, *vmid;  // shunt, 1/degree, middle of the voltage band
  double *bus_nu;  // [2][3][NB]: multiplier-solve coefficients per period kind (k_prep_bus)
  // UC box QPs: the inverse of the free block of H for each free-coordinate
  // mask, [variant (0: a next period, 1: the last)][mask][6 packed][NGEN]
  // (k_prep_ucbar)
  double *uc_hinv;
  long long NGEN;
  // per line-period, its last solve's Newton iterations [0][NBP] and
  // multiplier rounds [1][NBP] (the device counters behind the histograms)
  unsigned short *lcount;
  int *chk;  // first failed index check (UCAC_CHECK builds; 0 = none)
  const int *inc_ptr;            // CSR row pointers over global buses (degree)
  const int *gen_ptr, *gen_idx;  // CSR over global buses; generator index local
  const int *bus_order;                    // [NB] per instance: local buses sorted by (degree, generators)
  long long NUP;
  const double *Pd, *Qd;
  double *U;  // [NUF][NUP]
  // control and records
  double *ctrl;       // [K][NCTRL]
  double *res;        // [K][NRES]
  long long *stat;    // [K][6]: sweeps, newton, al, capped (last sweep), newton, al (all sweeps)
  double *part_up;    // [granules of bus-periods][NQ]
  double *part_gp;    // [granules of gen-periods][NQ]
  long long *bstat;   // [K][3]: Newton iterations, AL rounds, capped solves (line kernel, per sweep)
  // learned warm start: the start of each line-period's solve [4][NBP]
  // written by the MLP kernel of the same sweep (1 when the network's
  // proposal is taken, then its changes of V_i, V_j, d from the plain start),
  // enabled flag, and the count of line solves started from it [K]
  const float *prop;
  int warm;
  unsigned long long *wstat;
  unsigned long long *bp_counter;  // work counter of the persistent line kernel
  // order of the polar line kernel's work: pctl[0] counter of the listed
  // items, [1 + b] count of list b, [3] the sweep generation G (sweeps of
  // the line kernel since create or import), [4] warps retired; the lists
  // plist[b][NBP] of the line-periods a sweep flagged (sweep G writes list
  // (G + 1) & 1, reads list G & 1), and per line-period the generation mark
  // pgen = G + 2 of the last sweep G that flagged it
  unsigned long long *pctl;
  unsigned *pgen;
  int *plist;
  // UC dynamic-program scratch: stage costs, cost-to-go, decisions
  double *dpL;        // [4][T][ng] per instance, instance slice at 4*gpo
  double *dpC;        // [2][T+1][ng] per instance, slice at 2*(gpo+go)
  unsigned char *dpD; // [2][T][ng] per instance, slice at 2*gpo
  Granules g_gen, g_gp, g_bp, g_up;
};

__device__ __forceinline__ double clampd(double x, double lo, double hi) { return fmin(fmax(x, lo), hi); }

// Compares and clamps on the integer units.  B300's FP64 pipe also runs
// FP64 compares and min/max, at the FP64 rate; the signed 64-bit key below
// orders non-NaN doubles like their values (a negative double's magnitude
// bits are flipped), so the same decisions cost only integer operations.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 ? b ^ 0x7fffffffffffffffLL : b;
}
__device__ __forceinline__ double dunkey(long long k) { return __longlong_as_double(k < 0 ? k ^ 0x7fffffffffffffffLL : k); }
// x <= y for a non-negative y: the bit patterns compare the same way (a
// negative x, -0 included, has a negative pattern)
__device__ __forceinline__ bool le_nn(double x, double y) { return __double_as_longlong(x) <= __double_as_longlong(y); }
// max |x_i| of non-negative magnitudes, by bit pattern
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }

// FP64 <-> FP32 conversions on the integer units (the FP64 pipe also runs
// the hardware conversions, at the FP64 rate).  d2f_trunc keeps the top 24
// significant bits of a magnitude in [2^-126, 2^128) (truncation, within one
// FP32 ulp of the rounded value), returns a signed zero below that range and
// a NaN above it (infinities and NaNs included).  f2d_exact widens a normal
// float exactly; a subnormal float becomes a signed zero.
__device__ __forceinline__ float d2f_trunc(double x) {
  // the 32 bits from bit 29 up hold the exponent's low 9 bits above the top
  // 23 fraction bits; adding 2^30 = 2^32 - (896 << 23) modulo 2^32 rebiases
  // the exponent, exactly for biased exponents 897..1150 (the range tests
  // compare the magnitude's high word)
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), a = hi & 0x7fffffffu, sg = hi & 0x80000000u;
  const unsigned f = sg | ((unsigned)(b >> 29) + 0x40000000u);
  return __uint_as_float(a < 0x38100000u ? sg : (a < 0x47f00000u ? f : (sg | 0x7fc00000u)));
}
__device__ __forceinline__ double f2d_exact(float x) {
  // a >> 3 holds the exponent field above the top 20 fraction bits: one
  // addition of 896 << 20 rebiases it
  const unsigned u = __float_as_uint(x);
  const unsigned a = u & 0x7fffffffu, sg = u & 0x80000000u;
  const bool z = a < 0x00800000u;
  return __hiloint2double((int)(z ? sg : (sg | ((a >> 3) + (896u << 20)))), (int)(z ? 0u : (u << 29)));
}


// Index checks.  A UCAC_CHECK=1 build tests every index that the sweep
// kernels take from a table (line-end slots, generator and bus orders, work
// lists, instance lookups) against the extent of the buffer it addresses,
// before the access it guards.  A failed test records its site in S.chk
// (the first one wins) and the guarded access is skipped -- no trap, no
// early exit past a warp-collective -- so the host reads the site after the
// sweep (ucac_iterate fails with UCAC_E_CUDA naming it).  In the default
// build chk_ is the constant true and the tests compile away.
#ifndef UCAC_CHECK
#define UCAC_CHECK 0
#endif
__device__ __forceinline__ bool chk_(const Dev &S, bool ok, int site) {
#if UCAC_CHECK
  if (!ok) atomicCAS(S.chk, 0, site);
  return ok;
#else
  (void)S;
  (void)ok;
  (void)site;
  return true;
#endif
}

// Algorithm 1 stops an instance once it has converged: after the finish
// kernel sets its done flag, no kernel of a later sweep touches the
// instance, so its iterate, residual record and counters stay those of the
// sweep that converged (the other instances of a batch go on)
__device__ __forceinline__ bool inst_done(const Dev &S, int k) {
  return S.ctrl[(long long)k * NCTRL + C_DONE] != 0.0;
}

// slots of the from / to end of line lg at period t of instance I
__device__ __forceinline__ void line_ends(const Dev &S, const Inst &I, int t, long long lg, long long &ef,
                                          long long &et) {
  const long long base = I.eo + (long long)t * I.spp;
  ef = base + S.eslot[lg];
  et = base + S.eslot[S.NL + lg];
}

// canonical line row r (p_ij, q_ij, p_ji, q_ji, w_i, w_j, theta_i, theta_j)
// -> row type u (p, q, w, theta) at its end and the end (0 from, 1 to)
__host__ __device__ __forceinline__ int erow_u(int r) { return r < 4 ? (r & 1) : (r < 6 ? 2 : 3); }
__host__ __device__ __forceinline__ int erow_end(int r) { return r < 4 ? (r >> 1) : (r & 1); }

// granule of the calling warp (uniform across the warp), or -1
template <int BS>
__device__ __forceinline__ int warp_granule(int n) {
  const int gr = blockIdx.x * (BS / 32) + (threadIdx.x >> 5);
  return gr < n ? gr : -1;
}

// deterministic warp reduction of the NQ partials; lanes 0, 8, 16 and 24
// write the sums Q_SP, Q_SD, Q_SZ and Q_OBJ, lane 0 the maximum Q_INF.  The
// four sums share one transposed tree: in the first round a lane keeps two
// of them and passes the other two to its partner, in the second one, so
// the four take 6 FP64 additions per warp instead of 20.  The maximum runs
// on the bit patterns (the partials are non-negative, and non-negative
// doubles order like their bit patterns), on the integer units.
__device__ __forceinline__ void warp_reduce_q(const double (&q)[NQ], double *out) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  // first exchange: lanes 0-15 keep SP and SD, lanes 16-31 SZ and OBJ
  const double a = __dadd_rn(h16 ? q[Q_SZ] : q[Q_SP], __shfl_xor_sync(FULL, h16 ? q[Q_SP] : q[Q_SZ], 16));
  const double b = __dadd_rn(h16 ? q[Q_OBJ] : q[Q_SD], __shfl_xor_sync(FULL, h16 ? q[Q_SD] : q[Q_OBJ], 16));
  // second exchange: of each half, lanes with bit 3 clear keep a, the others b
  double v = __dadd_rn(h8 ? b : a, __shfl_xor_sync(FULL, h8 ? a : b, 8));
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(FULL, v, o));
  long long m = __double_as_longlong(q[Q_INF]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(FULL, m, o);
    m = w > m ? w : m;
  }
  if ((lane & 7) == 0) out[lane == 0 ? Q_SP : (lane == 8 ? Q_SD : (lane == 16 ? Q_SZ : Q_OBJ))] = v;
  if (lane == 0) out[Q_INF] = __longlong_as_double(m);
}

// deterministic block reduction of NQ doubles (sums, except Q_INF = max)
template <int BS>
__device__ __forceinline__ void block_reduce_q(double (&q)[NQ], double *out) {
  __shared__ double sh[NQ][BS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    double v = q[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double w = __shfl_down_sync(0xffffffffu, v, o);
      v = (k == Q_INF) ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int k = threadIdx.x;
    double v = sh[k][0];
    for (int w = 1; w < BS / 32; ++w) v = (k == Q_INF) ? fmax(v, sh[k][w]) : v + sh[k][w];
    out[k] = v;
  }
}

}  // namespace ucac
