// k_cold.cuh -- the cold start of Sec. IV-A, formed on the device after the
// constants are uploaded: every bus at the middle of its voltage band with
// zero angles, every unit on at half its capacity with its reactive output at
// the middle of its range, the line variables and flows of that point, the
// line-limit slacks and the initial line penalty.  Each operation is rounded
// as written (explicit intrinsics, no contraction), so the values are those
// of the same formulas in plain IEEE double arithmetic.  The state arena is
// zeroed before these kernels run; fields they do not write start at zero.
#pragma once
#include "common.cuh"

namespace ucac {

// generator-periods (warp granules): p, q, phat, u_on and the x-bar copies
template <int BS>
__global__ void __launch_bounds__(BS) k_cold_gen(Dev S) {
  const int gr = warp_granule<BS>(S.g_gp.n);
  if (gr < 0) return;
  const int k = S.g_gp.inst[gr];
  const Inst I = S.inst[k];
  const long long gp = (long long)S.g_gp.first[gr] + (threadIdx.x & 31);
  if (gp >= (long long)I.gpo + (long long)I.T * I.ng) return;
  const int loc = (int)(gp - I.gpo);
  const int t = loc / I.ng, g = loc - t * I.ng, gg = I.go + g;
  const long long NGP = S.NGP;
  const double p = __dmul_rn(0.5, S.Pmax[gg]), q = __dmul_rn(0.5, __dadd_rn(S.qlo[gg], S.qhi[gg]));
  S.G[F_P * NGP + gp] = p;
  S.G[F_Q * NGP + gp] = q;
  S.G[F_PH * NGP + gp] = t > 0 ? p : S.p0[gg];  // phat before period 0 is the data p0
  S.G[F_UON * NGP + gp] = 1.0;
  S.G[F_PBAR * NGP + gp] = p;
  S.G[F_QBAR * NGP + gp] = q;
  S.G[F_UBON * NGP + gp] = 1.0;
}

// bus-periods of instance blockIdx.y: w = V^2 (theta stays 0)
template <int BS>
__global__ void __launch_bounds__(BS) k_cold_bus(Dev S) {
  const int k = blockIdx.y;
  const Inst I = S.inst[k];
  const long long loc = (long long)blockIdx.x * BS + threadIdx.x;
  if (loc >= (long long)I.T * I.nb) return;
  const int i = (int)(loc % I.nb);
  const double V = S.vmid[I.uo + i];
  S.U[FU_W * S.NUP + I.upo + loc] = __dmul_rn(V, V);
}

// line-periods (warp granules): the W-form line variables
// (w_i, w_j, wR, wI, theta_i, theta_j, s_ij, s_ji) of the flat point, the
// penalty c = c_init_rel max(rho_pq, rho_va), and the x-bar of the four flow
// rows (the flows of that point) in the line-end slots
template <int BS>
__global__ void __launch_bounds__(BS) k_cold_branch(Dev S) {
  const int gr = warp_granule<BS>(S.g_bp.n);
  if (gr < 0) return;
  const int k = S.g_bp.inst[gr];
  const Inst I = S.inst[k];
  const long long bp = (long long)S.g_bp.first[gr] + (threadIdx.x & 31);
  if (bp >= (long long)I.bpo + (long long)I.T * I.nl) return;
  const int loc = (int)(bp - I.bpo);
  const int t = loc / I.nl, l = loc - t * I.nl;
  const long long NL = S.NL, NBP = S.NBP, NEP = S.NEP, lg = (long long)I.lo + l;
  const double Vi = S.vmid[I.uo + S.bf[lg]], Vj = S.vmid[I.uo + S.bt[lg]];
  double v[8] = {__dmul_rn(Vi, Vi), __dmul_rn(Vj, Vj), __dmul_rn(Vi, Vj), 0.0, 0.0, 0.0, 0.0, 0.0};
  double Y[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) Y[q] = S.BC[(BC_Y0 + q) * NL + lg];
  // Y = (Gii, Bii + b/2, Gij, Bij, Gjj, Bjj + b/2, Gji, Bji); flows of rows
  // p_ij, q_ij, p_ji, q_ji in the W form, summed left to right
  const double a0 = __dadd_rn(__dadd_rn(__dmul_rn(Y[0], v[0]), __dmul_rn(Y[2], v[2])), __dmul_rn(Y[3], v[3]));
  const double a1 = __dadd_rn(__dsub_rn(__dmul_rn(-Y[1], v[0]), __dmul_rn(Y[3], v[2])), __dmul_rn(Y[2], v[3]));
  const double a2 = __dsub_rn(__dadd_rn(__dmul_rn(Y[4], v[1]), __dmul_rn(Y[6], v[2])), __dmul_rn(Y[7], v[3]));
  const double a3 = __dsub_rn(__dsub_rn(__dmul_rn(-Y[5], v[1]), __dmul_rn(Y[7], v[2])), __dmul_rn(Y[6], v[3]));
  const double rate2 = S.BC[BC_RATE2 * NL + lg];
  v[6] = fmin(fmax(__dsub_rn(__dsub_rn(rate2, __dmul_rn(a0, a0)), __dmul_rn(a1, a1)), 0.0), rate2);
  v[7] = fmin(fmax(__dsub_rn(__dsub_rn(rate2, __dmul_rn(a2, a2)), __dmul_rn(a3, a3)), 0.0), rate2);
#pragma unroll
  for (int q = 0; q < 8; ++q) S.B[(FB_V0 + q) * NBP + bp] = v[q];
  S.B[FB_C * NBP + bp] = __dmul_rn(S.prm.c_init_rel, fmax(I.rpq, I.rva));
  long long ef, et;
  line_ends(S, I, t, lg, ef, et);
  if (!chk_(S, ef >= 0 && ef < S.NEP && et >= 0 && et < S.NEP, 51)) ef = et = 0;
  const double a[4] = {a0, a1, a2, a3};
#pragma unroll
  for (int r = 0; r < 4; ++r) S.EFB[erow_u(r) * NEP + (erow_end(r) ? et : ef)] = a[r];
}

}  // namespace ucac
