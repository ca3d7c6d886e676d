// k_ucdp.cuh -- UC subproblem per generator by dynamic programming
// (Sec. III-B, Algorithm 2).
//
// One thread per generator.  Consecutive generators of an instance sit at
// consecutive addresses of every [T][n_gen] array, so each of the thread's
// per-period loads is coalesced across the warp.  The stage-cost table
// L_t(a,b), the cost-to-go c_{t,s} and the stay/switch decisions live in a
// global scratch laid out [entry][t][g] (coalesced, L2-resident at the
// sizes of interest).  The backward pass is a serial O(T * T_min) chain per
// generator; all 32 lanes of a warp run 32 generators' chains side by side,
// so the FP64 pipe is never issued with idle lanes in the serial part.
//
// Bit-exactness: the stage cost is evaluated with explicitly rounded FP64
// operations (no contraction into FMAs) in this order
//   e_k = u_k - tau_k;  q = ((e_on*e_on) + (e_su*e_su)) + (e_sd*e_sd)
//   L = ((c0*b + csu*su) + csd*sd) + (0.5*rho)*q
// and the switch cost as (L(s,1-s) + sum_{t'} L(1-s,1-s) ascending) + c_next,
// with "stay" chosen when c_stay <= c_switch (Algorithm 2's rule), so the
// decisions equal those of any implementation using the same order.
#pragma once
#include "common.cuh"

namespace ucac {

// The linear parts c0*b + csu*su + csd*sd of the four stage costs, entry
// ab = a*2+b ((b, su, sd) = (0,0,0), (1,1,0), (0,0,1), (1,0,0)); they
// depend on the generator only, so they are formed once, in the order the
// rule at the top of this file fixes.
__device__ __forceinline__ void uc_lin4(double c0, double csu, double csd, double (&lin)[4]) {
  const double b[4] = {0.0, 1.0, 0.0, 1.0}, su[4] = {0.0, 1.0, 0.0, 0.0}, sd[4] = {0.0, 0.0, 1.0, 0.0};
#pragma unroll
  for (int ab = 0; ab < 4; ++ab)
    lin[ab] = __dadd_rn(__dadd_rn(__dmul_rn(c0, b[ab]), __dmul_rn(csu, su[ab])), __dmul_rn(csd, sd[ab]));
}

// The four stage costs of period t, entry ab = a*2+b at L[(ab*T + t)*st],
// the values of the rule at the top of this file: with b, su, sd in {0, 1}
// each e = b - tau is
// -tau (0 - tau is exact) or 1 - tau, and e*e does not depend on e's sign,
// so the six squares are formed once and shared; each q keeps the rule's
// summation order.
__device__ __forceinline__ void uc_stage4(int T, int t, long long st, double ton, double tsu, double tsd,
                                          const double (&lin)[4], double hr, double *L) {
  const double on0 = __dmul_rn(ton, ton), su0 = __dmul_rn(tsu, tsu), sd0 = __dmul_rn(tsd, tsd);
  const double eon = __dsub_rn(1.0, ton), esu = __dsub_rn(1.0, tsu), esd = __dsub_rn(1.0, tsd);
  const double on1 = __dmul_rn(eon, eon), su1 = __dmul_rn(esu, esu), sd1 = __dmul_rn(esd, esd);
  const double a00 = __dadd_rn(on0, su0);
  const double q[4] = {__dadd_rn(a00, sd0), __dadd_rn(__dadd_rn(on1, su1), sd0), __dadd_rn(a00, sd1),
                       __dadd_rn(__dadd_rn(on1, su0), sd0)};
#pragma unroll
  for (int ab = 0; ab < 4; ++ab) L[(ab * T + t) * st] = __dadd_rn(lin[ab], __dmul_rn(hr, q[ab]));
}

// Backward pass and forward reconstruction of Algorithm 2 from the
// stage-cost table L (element stride `st` between periods; C, D scratch with
// the same stride).  Writes u^on_t (0/1) through `uon` and returns c_{1,u0}.
template <typename WriteU>
__device__ __forceinline__ double uc_dp_tab(int T, int TU, int TD, int u0, int K0, long long st, const double *L,
                                            double *C, unsigned char *D, WriteU uon) {
#define LTAB(t1, a, b) L[(((a)*2 + (b)) * T + ((t1)-1)) * st]
#define CTAB(t1, s) C[((s) * (T + 1) + ((t1)-1)) * st]
#define DTAB(t1, s) D[((s)*T + ((t1)-1)) * st]
  CTAB(T + 1, 0) = 0.0;
  CTAB(T + 1, 1) = 0.0;
  for (int t = T; t >= K0 + 1; --t) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int ns = 1 - s;
      const double stay = __dadd_rn(LTAB(t, s, s), CTAB(t + 1, s));
      const int Tm = ns ? TU : TD;
      const int e = min(t + Tm - 1, T);
      double sw = LTAB(t, s, ns);
      for (int tp = t + 1; tp <= e; ++tp) sw = __dadd_rn(sw, LTAB(tp, ns, ns));
      sw = __dadd_rn(sw, CTAB(e + 1, ns));
      const bool keep = stay <= sw;
      CTAB(t, s) = keep ? stay : sw;
      DTAB(t, s) = keep ? 0 : 1;
    }
  }
  double cost;
  if (K0 > 0) {
    double acc = LTAB(1, u0, u0);
    for (int t = 2; t <= K0; ++t) acc = __dadd_rn(acc, LTAB(t, u0, u0));
    cost = __dadd_rn(acc, CTAB(K0 + 1, u0));
  } else {
    cost = CTAB(1, u0);
  }
  for (int t = 1; t <= K0; ++t) uon(t - 1, u0);
  int s = u0, t = K0 + 1;
  while (t <= T) {
    if (DTAB(t, s) == 0) {
      uon(t - 1, s);
      t += 1;
    } else {
      const int ns = 1 - s;
      const int e = min(t + (ns ? TU : TD) - 1, T);
      for (int k = t; k <= e; ++k) uon(k - 1, ns);
      s = ns;
      t = e + 1;
    }
  }
#undef LTAB
#undef CTAB
#undef DTAB
  return cost;
}

// DP for one generator on one thread.  tau_* point at period 0 of the
// generator's column (element stride `st` between periods); L/C/D are
// scratch columns with element stride `stt` (st when not given).
template <typename WriteU>
__device__ __forceinline__ double uc_dp(int T, int TU, int TD, int u0, int K0, double c0, double csu, double csd,
                                        double hr, const double *tau_on, const double *tau_su,
                                        const double *tau_sd, long long st, double *L, double *C,
                                        unsigned char *D, WriteU uon, long long stt = -1) {
  if (stt < 0) stt = st;
  double lin[4];
  uc_lin4(c0, csu, csd, lin);
  for (int t = 0; t < T; ++t) uc_stage4(T, t, stt, tau_on[t * st], tau_su[t * st], tau_sd[t * st], lin, hr, L);
  return uc_dp_tab(T, TU, TD, u0, K0, stt, L, C, D, uon);
}

// In-sweep x^UC step: reads the duplicate-row targets tau = ubar - z - y/rho
// (written by the x-bar^UC kernel of the previous sweep), writes u_on/u_su/
// u_sd and the x-side values of the three duplicate rows.
//
// The tables are the thread's own: with sm_T > 0 (every instance has
// T <= sm_T, and the launch gave BS * ucdp_smem_per_thread(sm_T) bytes of
// dynamic shared memory) they sit in a shared-memory column per thread
// (stride BS), so that the backward chain, which reads each step what the
// step before wrote, waits on shared memory instead of an L2 round trip;
// otherwise in the global scratch.  The arithmetic is the same either way.
__host__ __device__ constexpr size_t ucdp_smem_per_thread(int T) {
  return (size_t)(6 * T + 2) * sizeof(double) + (size_t)2 * T;
}

template <int BS>
__global__ void __launch_bounds__(BS) k_ucdp(Dev S, int sm_T) {
  extern __shared__ double ucdp_sm[];
  const int gr = warp_granule<BS>(S.g_gen.n);
  if (gr < 0) return;
  const int k = S.g_gen.inst[gr];
  if (inst_done(S, k)) return;
  const Inst I = S.inst[k];
  const int gg = S.g_gen.first[gr] + (threadIdx.x & 31);
  if (gg >= I.go + I.ng) return;
  const int g = gg - I.go, ng = I.ng, T = I.T;
  const long long NGP = S.NGP;
  const long long base = (long long)I.gpo + g;
  const double hr = __dmul_rn(0.5, I.ruc);
  const int TU = max(S.TU[gg], 1), TD = max(S.TD[gg], 1), u0 = S.u0[gg];
  const int K0 = min(max(S.K0[gg], 0), T);
  const bool sm = sm_T > 0 && chk_(S, T <= sm_T, 60);
  double *L = sm ? ucdp_sm + threadIdx.x : S.dpL + 4LL * I.gpo + g;
  double *C = sm ? ucdp_sm + (size_t)BS * 4 * sm_T + threadIdx.x : S.dpC + 2LL * (I.gpo + I.go) + g;
  unsigned char *D = sm ? (unsigned char *)(ucdp_sm + (size_t)BS * (6 * sm_T + 2)) + threadIdx.x
                        : S.dpD + 2LL * I.gpo + g;
  const long long st = sm ? BS : ng;
  if (S.prm.uc_relax) {
    // box relaxation of Eq. set:UC (first phase of the UC warm start): each
    // row minimises c u + rho/2 (u - tau)^2 over [0, 1]
    const double c[3] = {S.c0[gg], S.csu[gg], S.csd[gg]};
    const int fl[3] = {F_UON, F_USU, F_USD}, rw[3] = {GR_ON, GR_SU, GR_SD};
    for (int t = 0; t < T; ++t) {
      const long long i = base + (long long)t * ng;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double u = clampd(__dsub_rn(S.GT[rw[q] * NGP + i], __ddiv_rn(c[q], I.ruc)), 0.0, 1.0);
        S.G[fl[q] * NGP + i] = u;
        S.GA[rw[q] * NGP + i] = u;
      }
    }
    return;
  }
  double *uon_a = S.G + (long long)F_UON * NGP + base;
  uc_dp(T, TU, TD, u0, K0, S.c0[gg], S.csu[gg], S.csd[gg], hr, S.GT + GR_ON * NGP + base,
        S.GT + GR_SU * NGP + base, S.GT + GR_SD * NGP + base, (long long)ng, L, C, D,
        [&](int t, int u) { uon_a[(long long)t * ng] = (double)u; }, st);
  int prev = u0;
  for (int t = 0; t < T; ++t) {
    const long long i = base + (long long)t * ng;
    const int u = (int)S.G[F_UON * NGP + i];
    const double su = (u > prev) ? 1.0 : 0.0, sd = (prev > u) ? 1.0 : 0.0;
    S.G[F_USU * NGP + i] = su;
    S.G[F_USD * NGP + i] = sd;
    S.GA[GR_ON * NGP + i] = (double)u;
    S.GA[GR_SU * NGP + i] = su;
    S.GA[GR_SD * NGP + i] = sd;
    prev = u;
  }
}

// Second phase of the UC warm start, one thread per generator: marks
// m_t = [p_{t,g} >= p_frac Pmin_g], then Algorithm 2 with zero costs on the
// targets (m_t, m_t > m_{t-1}, m_{t-1} > m_t) -- the feasible schedule
// nearest to the marks -- into u_on / u_su / u_sd.  The duplicate-row
// targets are used as scratch (the state is re-imported afterwards).
template <int BS>
__global__ void __launch_bounds__(BS) k_uc_round(Dev S, double p_frac) {
  const int gr = warp_granule<BS>(S.g_gen.n);
  if (gr < 0) return;
  const int k = S.g_gen.inst[gr];
  const Inst I = S.inst[k];
  const int gg = S.g_gen.first[gr] + (threadIdx.x & 31);
  if (gg >= I.go + I.ng) return;
  const int g = gg - I.go, ng = I.ng, T = I.T;
  const long long NGP = S.NGP, base = (long long)I.gpo + g;
  const int TU = max(S.TU[gg], 1), TD = max(S.TD[gg], 1), u0 = S.u0[gg];
  const int K0 = min(max(S.K0[gg], 0), T);
  int prev = u0;
  for (int t = 0; t < T; ++t) {
    const long long i = base + (long long)t * ng;
    const int m = S.G[F_P * NGP + i] >= p_frac * S.Pmin[gg] ? 1 : 0;
    S.GT[GR_ON * NGP + i] = (double)m;
    S.GT[GR_SU * NGP + i] = (m > prev) ? 1.0 : 0.0;
    S.GT[GR_SD * NGP + i] = (prev > m) ? 1.0 : 0.0;
    prev = m;
  }
  double *L = S.dpL + 4LL * I.gpo + g;
  double *C = S.dpC + 2LL * (I.gpo + I.go) + g;
  unsigned char *D = S.dpD + 2LL * I.gpo + g;
  double *uon_a = S.G + (long long)F_UON * NGP + base;
  uc_dp(T, TU, TD, u0, K0, 0.0, 0.0, 0.0, 0.5, S.GT + GR_ON * NGP + base, S.GT + GR_SU * NGP + base,
        S.GT + GR_SD * NGP + base, (long long)ng, L, C, D, [&](int t, int u) { uon_a[(long long)t * ng] = (double)u; });
  prev = u0;
  for (int t = 0; t < T; ++t) {
    const long long i = base + (long long)t * ng;
    const int u = (int)S.G[F_UON * NGP + i];
    S.G[F_USU * NGP + i] = (u > prev) ? 1.0 : 0.0;
    S.G[F_USD * NGP + i] = (prev > u) ? 1.0 : 0.0;
    prev = u;
  }
}

// Standalone DP over [T][n_gen] device arrays, one warp per generator, for
// fleets too small to fill the GPU with one thread each: the lanes form the
// 4T stage costs in parallel into shared memory (per warp L [4][T], C
// [2][T+1] doubles, then D [2][T] bytes after the four warps' doubles) and
// lane 0 runs the serial backward pass and the reconstruction on them (the
// same operations in the same order as the thread-per-generator kernel, so
// the same bits).  Blocks of 4 warps; dynamic shared memory
// ucdp_warp_smem(T).
__host__ __device__ constexpr size_t ucdp_warp_smem(int T) {
  return 4 * (6 * (size_t)T + 2) * sizeof(double) + 4 * 2 * (size_t)T;
}

__global__ void __launch_bounds__(128) k_ucdp_warp(int ng, int T, double rho, const double *tau_on,
                                                   const double *tau_su, const double *tau_sd, const double *c0,
                                                   const double *csu, const double *csd, const int *TU,
                                                   const int *TD, const int *u0, const int *K0, int8_t *u_on,
                                                   double *cost) {
  extern __shared__ double dp_sm[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * 4 + w;
  if (g >= ng) return;  // (warp-uniform)
  double *L = dp_sm + (size_t)w * (6 * T + 2);
  double *C = L + 4 * T;
  unsigned char *D = (unsigned char *)(dp_sm + 4 * (6 * (size_t)T + 2)) + (size_t)w * 2 * T;
  const double hr = __dmul_rn(0.5, rho);
  double lin[4];
  uc_lin4(c0[g], csu[g], csd[g], lin);
  for (int t = lane; t < T; t += 32) {
    const long long i = (long long)t * ng + g;
    uc_stage4(T, t, 1, tau_on[i], tau_su[i], tau_sd[i], lin, hr, L);
  }
  __syncwarp();
  if (lane != 0) return;
  int8_t *uo = u_on + g;
  cost[g] = uc_dp_tab(T, max(TU[g], 1), max(TD[g], 1), u0[g] ? 1 : 0, min(max(K0[g], 0), T), 1, L, C, D,
                      [&](int t, int u) { uo[(long long)t * ng] = (int8_t)u; });
}

// Standalone DP over [T][n_gen] device arrays (one thread per generator).
__global__ void __launch_bounds__(128) k_ucdp_standalone(int ng, int T, double rho, const double *tau_on,
                                                         const double *tau_su, const double *tau_sd,
                                                         const double *c0, const double *csu, const double *csd,
                                                         const int *TU, const int *TD, const int *u0,
                                                         const int *K0, int8_t *u_on, double *cost, double *L,
                                                         double *C, unsigned char *D) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  const double hr = __dmul_rn(0.5, rho);
  int8_t *uo = u_on + g;
  cost[g] = uc_dp(T, max(TU[g], 1), max(TD[g], 1), u0[g] ? 1 : 0, min(max(K0[g], 0), T), c0[g], csu[g], csd[g], hr,
                  tau_on + g, tau_su + g, tau_sd + g, (long long)ng, L + g, C + g, D + g,
                  [&](int t, int u) { uo[(long long)t * ng] = (int8_t)u; });
}

}  // namespace ucac
