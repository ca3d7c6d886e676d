// k_mlp.cuh -- learned warm start of the line subproblems: a 12-64-64-6 MLP
// (SiLU) that proposes the change of each line's iterate from its features.
//
// Inference runs on the 5th-generation tensor cores: tiles of 128 rows, BF16
// operands staged in shared memory in the canonical K-major layout (8 x 16 B
// core matrices, no swizzle), FP32 accumulators in tensor memory, one
// tcgen05.mma per 16-deep K chunk issued by one thread, completion through
// tcgen05.commit on an mbarrier, accumulators read back with tcgen05.ld for
// the bias + SiLU epilogue, whose BF16 output is the next layer's A operand.
// Training runs in FP32 on the SIMT pipes (forward, backward with fixed-order
// weight-gradient sums, Adam), small enough that its cost does not matter.
//
// Features of line l at period t, from the state the line kernel starts from
// (iterate x0 = (w_i, w_j, wR, wI, theta_i, theta_j), targets t_r, series
// admittance y = g + j b of the line):
//   f0..f2  sqrt(w_i), sqrt(w_j), theta_i - theta_j
//   f3, f4  g / |y|, b / |y|   (direction of the line's admittance)
//   f5..f11 r / s, with the residual r = ((t_p,q - a(x0)) / |y| for the four
//           flow rows, t_wi - w_i, t_wj - w_j, (t_thi - t_thj) - (theta_i -
//           theta_j)) and s = |r|
// and the network predicts (x1 - x0) / s in the W coordinates, so that its
// output scales with the residual (the change of the solution is linear in
// the change of the targets to first order).
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"

namespace ucac {

constexpr int MLP_IN = 12, MLP_H = 64, MLP_OUT = 6;
// flat FP32 parameter vector: W1 [H][IN], b1 [H], W2 [H][H], b2 [H], W3 [OUT][H], b3 [OUT]
constexpr int MLP_OW1 = 0, MLP_OB1 = MLP_OW1 + MLP_H * MLP_IN, MLP_OW2 = MLP_OB1 + MLP_H,
              MLP_OB2 = MLP_OW2 + MLP_H * MLP_H, MLP_OW3 = MLP_OB2 + MLP_H, MLP_OB3 = MLP_OW3 + MLP_OUT * MLP_H,
              MLP_NPARAM = MLP_OB3 + MLP_OUT;
// packed inference weights in the canonical layout: BF16 W1 [64 x 16] (K
// padded; columns 12, 13 hold b1 as a BF16 pair hi + lo), W2 [64 x 64], W3
// [16 x 64] (N padded), B2 [64 x 16] (b2 as a pair in columns 12, 13, zero
// elsewhere), then FP32 b1, b2, b3 (16).  The feature tile carries ones in
// columns 12, 13, so layer 1 adds b1 inside its MMA and an extra 16-deep
// MMA of the feature tile against B2 adds b2 to layer 2 (to ~2^-16 of the
// bias: BF16 hi + lo)
constexpr int MLP_PK_W1 = 0, MLP_PK_W2 = 2048, MLP_PK_W3 = 2048 + 8192, MLP_PK_B2 = 2048 + 8192 + 2048,
              MLP_PK_B = MLP_PK_B2 + 2048, MLP_PACK_BYTES = MLP_PK_B + 4 * (64 + 64 + 16);

// byte offset of element (row, k) of a K-major operand with KG 8-element K
// groups: core matrix (row / 8, k / 8) is 128 contiguous bytes, 16 per row
__host__ __device__ __forceinline__ int canon_off(int row, int k, int KG) {
  return (((row >> 3) * KG + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// ---------------------------------------------------------------- features
// Features of line-period (t, l) of instance I and the scale s; false when
// the residual vanishes (the network then proposes no change).  The flows
// and the residuals' subtractions are FP64 (the residual is a small
// difference of O(1) values); the rest of the features, which the network
// takes in BF16, is FP32 unless EXACT (the feature API, whose scale s is
// compared with FP64 definitions).  aflow (may be NULL) receives the flows
// and the line-limit values g_k = p_k^2 + q_k^2 - rate^2 (formed in FP64:
// the difference is small against its terms) as aflow[4], aflow[5].
template <bool EXACT>
__device__ __forceinline__ bool line_features(const Dev &S, const Inst &I, long long bp, int t, int l,
                                              float (&f)[MLP_IN], double &s, float *aflow = nullptr) {
  if (!EXACT) {
    const long long NBP = S.NBP, NL = S.NL, NEP = S.NEP, lg = (long long)I.lo + l;
    const double wi = S.B[(FB_V0 + 0) * NBP + bp], wj = S.B[(FB_V0 + 1) * NBP + bp];
    const double wR = S.B[(FB_V0 + 2) * NBP + bp], wI = S.B[(FB_V0 + 3) * NBP + bp];
    const double thi = S.B[(FB_V0 + 4) * NBP + bp], thj = S.B[(FB_V0 + 5) * NBP + bp];
    double Y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) Y[q] = S.BC[(BC_Y0 + q) * NL + lg];
    const double a[4] = {Y[0] * wi + Y[2] * wR + Y[3] * wI, -Y[1] * wi - Y[3] * wR + Y[2] * wI,
                         Y[4] * wj + Y[6] * wR - Y[7] * wI, -Y[5] * wj - Y[7] * wR - Y[6] * wI};
    long long ef, et;
    line_ends(S, I, t, lg, ef, et);
    if (!chk_(S, ef >= 0 && ef < S.NEP && et >= 0 && et < S.NEP, 30)) ef = et = 0;
    double tg[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) tg[r] = S.ET[erow_u(r) * NEP + (erow_end(r) ? et : ef)];
    if (aflow) {
#pragma unroll
      for (int r = 0; r < 4; ++r) aflow[r] = (float)a[r];
      const double rate2 = S.BC[BC_RATE2 * NL + lg];
      aflow[4] = (float)(a[0] * a[0] + a[1] * a[1] - rate2);
      aflow[5] = (float)(a[2] * a[2] + a[3] * a[3] - rate2);
    }
    const float g = (float)Y[2], b = (float)Y[3], iym = rsqrtf(g * g + b * b);
    float res[7];
#pragma unroll
    for (int r = 0; r < 4; ++r) res[r] = (float)(tg[r] - a[r]) * iym;
    res[4] = (float)(tg[4] - wi);
    res[5] = (float)(tg[5] - wj);
    const double dth = thi - thj;
    res[6] = (float)((tg[6] - tg[7]) - dth);
    float n2 = 0.0f;
#pragma unroll
    for (int r = 0; r < 7; ++r) n2 = fmaf(res[r], res[r], n2);
    const float sf = sqrtf(n2);
    s = (double)sf;
    f[0] = sqrtf(fmaxf((float)wi, 0.0f));
    f[1] = sqrtf(fmaxf((float)wj, 0.0f));
    f[2] = (float)dth;
    f[3] = -g * iym;  // g / |y| (Y_ij = -y)
    f[4] = -b * iym;  // b / |y|
    if (!(sf > 1e-30f)) {
#pragma unroll
      for (int r = 0; r < 7; ++r) f[5 + r] = 0.0f;
      return false;
    }
    const float is = __frcp_rn(sf);
#pragma unroll
    for (int r = 0; r < 7; ++r) f[5 + r] = res[r] * is;
    return true;
  }
  const long long NBP = S.NBP, NL = S.NL, NEP = S.NEP, lg = (long long)I.lo + l;
  const double wi = S.B[(FB_V0 + 0) * NBP + bp], wj = S.B[(FB_V0 + 1) * NBP + bp];
  const double wR = S.B[(FB_V0 + 2) * NBP + bp], wI = S.B[(FB_V0 + 3) * NBP + bp];
  const double thi = S.B[(FB_V0 + 4) * NBP + bp], thj = S.B[(FB_V0 + 5) * NBP + bp];
  double Y[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) Y[q] = S.BC[(BC_Y0 + q) * NL + lg];
  // flows of the W-form iterate (linear in w_i, w_j, wR, wI)
  const double a[4] = {Y[0] * wi + Y[2] * wR + Y[3] * wI, -Y[1] * wi - Y[3] * wR + Y[2] * wI,
                       Y[4] * wj + Y[6] * wR - Y[7] * wI, -Y[5] * wj - Y[7] * wR - Y[6] * wI};
  long long ef, et;
  line_ends(S, I, t, lg, ef, et);
  if (!chk_(S, ef >= 0 && ef < S.NEP && et >= 0 && et < S.NEP, 31)) ef = et = 0;
  double tg[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) tg[r] = S.ET[erow_u(r) * NEP + (erow_end(r) ? et : ef)];
  const double ym = sqrt(Y[2] * Y[2] + Y[3] * Y[3]), iym = 1.0 / ym;
  double res[7];
#pragma unroll
  for (int r = 0; r < 4; ++r) res[r] = (tg[r] - a[r]) * iym;
  res[4] = tg[4] - wi;
  res[5] = tg[5] - wj;
  res[6] = (tg[6] - tg[7]) - (thi - thj);
  double n2 = 0.0;
#pragma unroll
  for (int r = 0; r < 7; ++r) n2 += res[r] * res[r];
  s = sqrt(n2);
  f[0] = (float)sqrt(fmax(wi, 0.0));
  f[1] = (float)sqrt(fmax(wj, 0.0));
  f[2] = (float)(thi - thj);
  f[3] = (float)(-Y[2] * iym);  // g / |y| (Y_ij = -y)
  f[4] = (float)(-Y[3] * iym);  // b / |y|
  if (!(s > 1e-300)) {
#pragma unroll
    for (int r = 0; r < 7; ++r) f[5 + r] = 0.0f;
    return false;
  }
  const double is = 1.0 / s;
#pragma unroll
  for (int r = 0; r < 7; ++r) f[5 + r] = (float)(res[r] * is);
  return true;
}

// ------------------------------------------------------ tcgen05 helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets between core matrices, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the mbarrier phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
// inference: z sigma(z) = h + h tanh(h) with h = z / 2, on the hardware
// tanh (relative error ~5e-4, below the BF16 rounding of the activation
// that follows): three instructions instead of an exponential and an IEEE
// division, 128 activations per row
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float silu_fast(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_approx(h), h);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&b);
}

// 8 consecutive K elements of one row as one 16-byte store
__device__ __forceinline__ void st_row8(uint8_t *base, int row, int k0, int KG, const float *v) {
  uint4 q;
  q.x = pack_bf16x2(v[0], v[1]);
  q.y = pack_bf16x2(v[2], v[3]);
  q.z = pack_bf16x2(v[4], v[5]);
  q.w = pack_bf16x2(v[6], v[7]);
  *reinterpret_cast<uint4 *>(base + canon_off(row, k0, KG)) = q;
}

// ------------------------------------------------------ start choice
// Whether the polar line solve of row bp should start from the network's
// proposal, and the proposal as changes (dVi, dVj, dd) of the plain start
// V = sqrt(w), d = theta_i - theta_j.  The test is the sign of the change of
// the line objective (slacks at their minimiser) between the two starts,
// formed in FP32 from differences so that no term cancels: the flows change
// by da_r = q_r d(V'^2) + dP E_r + P' dE_r with dE from the half-angle
// formulas, the residual terms by rho da (e + da/2) with the plain residuals
// e rebuilt from the features f and the scale s, and the line-limit terms
// through the change of h = max(g, -mu/c).  A wrong choice between two
// nearly equal starts costs only Newton steps: the solve polishes either to
// the same tolerance.
__device__ __forceinline__ bool warm_choice(const Dev &S, const Inst &I, long long bp, long long lg,
                                            const float (&f)[16], float s, const float (&af)[6],
                                            const float (&dw)[MLP_OUT], float &dVi, float &dVj, float &dd) {
  const long long NBP = S.NBP, NL = S.NL;
  const float Vi = f[0], Vj = f[1], d = f[2];
  // proposal: w + dw, theta + dtheta, projected on the voltage bounds
  const float lo0 = (float)S.BC[(BC_VB + 0) * NL + lg], hi0 = (float)S.BC[(BC_VB + 1) * NL + lg];
  const float lo1 = (float)S.BC[(BC_VB + 2) * NL + lg], hi1 = (float)S.BC[(BC_VB + 3) * NL + lg];
  const float wim = fmaxf(Vi * Vi + dw[0], 0.0f), wjm = fmaxf(Vj * Vj + dw[1], 0.0f);
  dVi = fminf(fmaxf(Vi + __fdividef(dw[0], Vi + sqrtf(wim)), lo0), hi0) - Vi;
  dVj = fminf(fmaxf(Vj + __fdividef(dw[1], Vj + sqrtf(wjm)), lo1), hi1) - Vj;
  dd = dw[4] - dw[5];
  const float dVi2 = dVi * (2.0f * Vi + dVi), dVj2 = dVj * (2.0f * Vj + dVj);
  const float P = Vi * Vj, dP = dVi * Vj + Vi * dVj + dVi * dVj, Pm = P + dP;
  // cos/sin at the plain start and their changes (hardware sin/cos, ~1e-6
  // absolute; the half-angle sine of a small change from its odd series,
  // which keeps its relative accuracy)
  float sn, c, smid, cmid;
  __sincosf(d, &sn, &c);
  const float hh = 0.5f * dd, hh2 = hh * hh;
  const float shh = fabsf(hh) < 0.25f ? hh * (1.0f - hh2 * (1.0f / 6.0f - hh2 * (1.0f / 120.0f))) : __sinf(hh);
  __sincosf(d + hh, &smid, &cmid);
  const float dc = -2.0f * smid * shh, ds = 2.0f * cmid * shh;
  // FP32 line constants: q_0..q_3, ga, ka of the from and the to end
  float q[4], ga[2], ka[2];
#pragma unroll
  for (int r = 0; r < 4; ++r) q[r] = S.BCF[r * NL + lg];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    ga[e] = S.BCF[(4 + e) * NL + lg];
    ka[e] = S.BCF[(6 + e) * NL + lg];
  }
  float E[4], dE[4];
  {
    const float E0 = ga[0] * c + ka[0] * sn, Ed0 = ka[0] * c - ga[0] * sn;
    const float E2 = ga[1] * c + ka[1] * sn, Ed2 = ka[1] * c - ga[1] * sn;
    const float dE0 = ga[0] * dc + ka[0] * ds, dEd0 = ka[0] * dc - ga[0] * ds;
    const float dE2 = ga[1] * dc + ka[1] * ds, dEd2 = ka[1] * dc - ga[1] * ds;
    E[0] = E0; E[1] = -Ed0; E[2] = E2; E[3] = Ed2;
    dE[0] = dE0; dE[1] = -dEd0; dE[2] = dE2; dE[3] = dEd2;
  }
  const float ym = sqrtf(ga[0] * ga[0] + ka[0] * ka[0]);
  const float rpq = (float)I.rpq, rva = (float)I.rva;
  float da[4], df = 0.0f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    da[r] = q[r] * (r < 2 ? dVi2 : dVj2) + dP * E[r] + Pm * dE[r];
    const float e = -f[5 + r] * s * ym;  // a_r - t_r at the plain start
    df += rpq * da[r] * (e + 0.5f * da[r]);
  }
  const float e4 = -f[9] * s, e5 = -f[10] * s, e6 = -f[11] * s;
  df += 0.5f * rva * (dVi2 * (2.0f * e4 + dVi2) + dVj2 * (2.0f * e5 + dVj2));
  df += 0.25f * rva * dd * (2.0f * e6 + dd);
  const float cpen = (float)S.B[FB_C * NBP + bp];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r0 = 2 * k, r1 = 2 * k + 1;
    const float mu = (float)S.B[(FB_MU0 + 2 + k) * NBP + bp];
    const float gp = af[4 + k];
    const float dg = da[r0] * (2.0f * af[r0] + da[r0]) + da[r1] * (2.0f * af[r1] + da[r1]);
    const float hc = -__fdividef(mu, cpen), hp = fmaxf(gp, hc), hm = fmaxf(gp + dg, hc);
    df += (hm - hp) * (mu + 0.5f * cpen * (hm + hp));
  }
  return df < 0.0f;
}

// ------------------------------------------------------------ inference
struct MlpSmem {
  alignas(128) uint8_t w[MLP_PK_B];  // W1 | W2 | W3 | B2
  float b1[64], b2[64], b3[16];
  alignas(128) uint8_t a1[128 * 16 * 2];
  alignas(128) uint8_t a2[128 * 64 * 2];
  alignas(8) unsigned long long mbar;
  uint32_t tmem;
};

// one 64-column accumulator reused by the three layers (each layer's MMA is
// issued after the previous layer's accumulator has been read back), so six
// CTAs fit in an SM's 512 TMEM columns
constexpr uint32_t MLP_TMEM_COLS = 64;
constexpr int MLP_CTAS_PER_SM = 6;

// One persistent CTA of 4 warps per 128-row tile.  FUSED: features from the
// sweep state, output the proposed change s * y of each line-period's
// iterate into prop [6][NBP]; otherwise features feat [n][12] and raw
// outputs out [n][6].  err is set on a timed-out wait.
template <bool FUSED>
__global__ void __launch_bounds__(128, MLP_CTAS_PER_SM) k_mlp(Dev S, const uint8_t *__restrict__ pack, long long n,
                                             const float *__restrict__ feat, float *__restrict__ out, int *err) {
  __shared__ MlpSmem sm;
  const int tid = threadIdx.x, warp = tid >> 5;
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(pack);
    uint4 *dst = reinterpret_cast<uint4 *>(sm.w);
    for (int i = tid; i < MLP_PACK_BYTES / 16; i += 128) dst[i] = src[i];  // w, b1, b2, b3 are contiguous
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(MLP_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem, mbar = smem_u32(&sm.mbar);
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t sa1 = smem_u32(sm.a1), sa2 = smem_u32(sm.a2), sw = smem_u32(sm.w);
  constexpr uint32_t ID64 = umma_idesc_bf16(128, 64), ID16 = umma_idesc_bf16(128, 16);
  uint32_t phase = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile * 128 < n; tile += gridDim.x) {
    const long long row = tile * 128 + tid;
    float f[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) f[j] = 0.0f;
    double sc = 0.0;
    float af[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    int k = 0;
    long long lgr = 0;
    bool live = row < n;
    if (live) {
      if (FUSED) {
        {
          int lo = 0, hi = S.K - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((long long)S.inst[mid].bpo <= row) lo = mid; else hi = mid - 1;
          }
          k = lo;
        }
        const Inst &I = S.inst[k];
        const int loc = (int)(row - I.bpo), t = loc / I.nl, l = loc - t * I.nl;
        lgr = (long long)I.lo + l;
        float ff[MLP_IN];
        live = line_features<false>(S, I, row, t, l, ff, sc, af);
#pragma unroll
        for (int j = 0; j < MLP_IN; ++j) f[j] = ff[j];
      } else {
#pragma unroll
        for (int j = 0; j < MLP_IN; ++j) f[j] = feat[row * MLP_IN + j];
      }
    }
    f[12] = f[13] = 1.0f;  // the bias columns
    st_row8(sm.a1, tid, 0, 2, f);
    st_row8(sm.a1, tid, 8, 2, f + 8);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- layer 1: D1 = A1 [128 x 16] . W1^T
    if (tid == 0) {
      tc_fence_after();
      umma_bf16(tmem, umma_desc(sa1, 128, 256), umma_desc(sw + MLP_PK_W1, 128, 256), ID64, 0);
      umma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1;
    tc_fence_after();
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16];
      tmem_ld16(tmem + lane_base + 16 * c, z);
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = silu_fast(z[j]);  // (b1 added by the MMA)
      st_row8(sm.a2, tid, 16 * c, 8, z);
      st_row8(sm.a2, tid, 16 * c + 8, 8, z + 8);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- layer 2: D2 = A2 [128 x 64] . W2^T, four 16-deep chunks
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma_bf16(tmem, umma_desc(sa2 + 256 * kk, 128, 1024), umma_desc(sw + MLP_PK_W2 + 256 * kk, 128, 1024),
                  ID64, kk > 0);
      // + b2: the feature tile's ones columns against B2
      umma_bf16(tmem, umma_desc(sa1, 128, 256), umma_desc(sw + MLP_PK_B2, 128, 256), ID64, 1);
      umma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1;
    tc_fence_after();
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float z[16];
      tmem_ld16(tmem + lane_base + 16 * c, z);
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = silu_fast(z[j]);  // (b2 added by the MMA)
      st_row8(sm.a2, tid, 16 * c, 8, z);
      st_row8(sm.a2, tid, 16 * c + 8, 8, z + 8);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- layer 3: D3 = A3 [128 x 64] . W3^T (N padded to 16)
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        umma_bf16(tmem, umma_desc(sa2 + 256 * kk, 128, 1024),
                  umma_desc(sw + MLP_PK_W3 + 256 * kk, 128, 1024), ID16, kk > 0);
      umma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase) && ok;
    phase ^= 1;
    tc_fence_after();
    float y[16];
    tmem_ld16(tmem + lane_base, y);
    if (row < n) {
      if (FUSED) {
        // the start of the line solve: [0] 1 when the proposal is taken,
        // [1..3] its changes of V_i, V_j, d
        float take = 0.0f, dVi = 0.0f, dVj = 0.0f, dd = 0.0f;
        if (live) {
          const float sf = (float)sc;
          float dw[MLP_OUT];
#pragma unroll
          for (int j = 0; j < MLP_OUT; ++j) dw[j] = sf * (y[j] + sm.b3[j]);
          take = warm_choice(S, S.inst[k], row, lgr, f, sf, af, dw, dVi, dVj, dd) ? 1.0f : 0.0f;
        }
        out[row] = take;
        out[n + row] = dVi;
        out[2 * n + row] = dVj;
        out[3 * n + row] = dd;
      } else {
#pragma unroll
        for (int j = 0; j < MLP_OUT; ++j) out[row * MLP_OUT + j] = y[j] + sm.b3[j];
      }
    }
    tc_fence_before();
    if (__syncthreads_or(!ok)) break;
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MLP_TMEM_COLS)
                 : "memory");
  }
}

// FP32 parameters -> packed BF16 canonical operands + FP32 biases
__global__ void k_mlp_pack(const float *__restrict__ P, uint8_t *__restrict__ pack) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(pack + MLP_PK_W1);
  __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(pack + MLP_PK_W2);
  __nv_bfloat16 *w3 = reinterpret_cast<__nv_bfloat16 *>(pack + MLP_PK_W3);
  __nv_bfloat16 *b2 = reinterpret_cast<__nv_bfloat16 *>(pack + MLP_PK_B2);
  float *b = reinterpret_cast<float *>(pack + MLP_PK_B);
  if (i < 64 * 16) {
    const int o = i / 16, k = i % 16;
    // a bias as a BF16 pair: hi = bf16(b), lo = bf16(b - hi)
    auto pair = [&](float bias) -> __nv_bfloat16 {
      const __nv_bfloat16 hi = __float2bfloat16_rn(bias);
      return k == 12 ? hi : __float2bfloat16_rn(bias - __bfloat162float(hi));
    };
    w1[canon_off(o, k, 2) / 2] =
        k < MLP_IN ? __float2bfloat16_rn(P[MLP_OW1 + o * MLP_IN + k]) : (k < 14 ? pair(P[MLP_OB1 + o]) : __float2bfloat16_rn(0.0f));
    b2[canon_off(o, k, 2) / 2] = (k == 12 || k == 13) ? pair(P[MLP_OB2 + o]) : __float2bfloat16_rn(0.0f);
  }
  if (i < 64 * 64) {
    const int o = i / 64, k = i % 64;
    w2[canon_off(o, k, 8) / 2] = __float2bfloat16_rn(P[MLP_OW2 + o * MLP_H + k]);
  }
  if (i < 16 * 64) {
    const int o = i / 64, k = i % 64;
    w3[canon_off(o, k, 8) / 2] = __float2bfloat16_rn(o < MLP_OUT ? P[MLP_OW3 + o * MLP_H + k] : 0.0f);
  }
  if (i < 64) {
    b[i] = P[MLP_OB1 + i];
    b[64 + i] = P[MLP_OB2 + i];
  }
  if (i < 16) b[128 + i] = i < MLP_OUT ? P[MLP_OB3 + i] : 0.0f;
}

// ------------------------------------------------------------- training
__device__ __forceinline__ float silu_grad(float z) {
  const float sg = 1.0f / (1.0f + __expf(-z));
  return sg * (1.0f + z * (1.0f - sg));
}

// forward of one sample per thread; keeps the pre-activations, the output
// error gradient dY = 2 (y - label) / n and the sample's squared error
__global__ void k_mlp_fwd_train(long long n, const float *__restrict__ X, const float *__restrict__ Lb,
                                const float *__restrict__ P, float *__restrict__ Z1, float *__restrict__ Z2,
                                float *__restrict__ dY, float *__restrict__ sq) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  float x[MLP_IN], h1[MLP_H];
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) x[i] = X[b * MLP_IN + i];
  for (int o = 0; o < MLP_H; ++o) {
    float z = P[MLP_OB1 + o];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) z = fmaf(P[MLP_OW1 + o * MLP_IN + i], x[i], z);
    Z1[b * MLP_H + o] = z;
    h1[o] = silu(z);
  }
  float y[MLP_OUT];
#pragma unroll
  for (int j = 0; j < MLP_OUT; ++j) y[j] = P[MLP_OB3 + j];
  for (int o = 0; o < MLP_H; ++o) {
    float z = P[MLP_OB2 + o];
    for (int i = 0; i < MLP_H; ++i) z = fmaf(P[MLP_OW2 + o * MLP_H + i], h1[i], z);
    Z2[b * MLP_H + o] = z;
    const float h = silu(z);
#pragma unroll
    for (int j = 0; j < MLP_OUT; ++j) y[j] = fmaf(P[MLP_OW3 + j * MLP_H + o], h, y[j]);
  }
  float e2 = 0.0f;
  const float g = 2.0f / (float)n;
#pragma unroll
  for (int j = 0; j < MLP_OUT; ++j) {
    const float e = y[j] - Lb[b * MLP_OUT + j];
    dY[b * MLP_OUT + j] = g * e;
    e2 = fmaf(e, e, e2);
  }
  sq[b] = e2;
}

// pre-activation gradients dZ2 = (W3^T dY) * silu'(Z2), dZ1 = (W2^T dZ2) * silu'(Z1)
__global__ void k_mlp_bwd_train(long long n, const float *__restrict__ P, const float *__restrict__ Z1,
                                const float *__restrict__ Z2, const float *__restrict__ dY, float *__restrict__ dZ1,
                                float *__restrict__ dZ2) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  float dy[MLP_OUT], d2[MLP_H];
#pragma unroll
  for (int j = 0; j < MLP_OUT; ++j) dy[j] = dY[b * MLP_OUT + j];
  for (int o = 0; o < MLP_H; ++o) {
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < MLP_OUT; ++j) s = fmaf(P[MLP_OW3 + j * MLP_H + o], dy[j], s);
    d2[o] = s * silu_grad(Z2[b * MLP_H + o]);
    dZ2[b * MLP_H + o] = d2[o];
  }
  for (int i = 0; i < MLP_H; ++i) {
    float s = 0.0f;
    for (int o = 0; o < MLP_H; ++o) s = fmaf(P[MLP_OW2 + o * MLP_H + i], d2[o], s);
    dZ1[b * MLP_H + i] = s * silu_grad(Z1[b * MLP_H + i]);
  }
}

// one thread per parameter: sums over the batch in sample order (fixed)
__global__ void k_mlp_wgrad(long long n, const float *__restrict__ X, const float *__restrict__ Z1,
                            const float *__restrict__ Z2, const float *__restrict__ dZ1,
                            const float *__restrict__ dZ2, const float *__restrict__ dY, float *__restrict__ G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  float s = 0.0f;
  if (p < MLP_OB1) {
    const int o = p / MLP_IN, i = p % MLP_IN;
    for (long long b = 0; b < n; ++b) s = fmaf(dZ1[b * MLP_H + o], X[b * MLP_IN + i], s);
  } else if (p < MLP_OW2) {
    const int o = p - MLP_OB1;
    for (long long b = 0; b < n; ++b) s += dZ1[b * MLP_H + o];
  } else if (p < MLP_OB2) {
    const int o = (p - MLP_OW2) / MLP_H, i = (p - MLP_OW2) % MLP_H;
    for (long long b = 0; b < n; ++b) s = fmaf(dZ2[b * MLP_H + o], silu(Z1[b * MLP_H + i]), s);
  } else if (p < MLP_OW3) {
    const int o = p - MLP_OB2;
    for (long long b = 0; b < n; ++b) s += dZ2[b * MLP_H + o];
  } else if (p < MLP_OB3) {
    const int o = (p - MLP_OW3) / MLP_H, i = (p - MLP_OW3) % MLP_H;
    for (long long b = 0; b < n; ++b) s = fmaf(dY[b * MLP_OUT + o], silu(Z2[b * MLP_H + i]), s);
  } else {
    const int o = p - MLP_OB3;
    for (long long b = 0; b < n; ++b) s += dY[b * MLP_OUT + o];
  }
  G[p] = s;
}

// sum of n values in index order (one block; deterministic), scaled
__global__ void k_sum_fixed(long long n, const float *__restrict__ v, float scale, float *__restrict__ out) {
  __shared__ double part[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += (double)v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += part[i];
    *out = (float)(t * scale);
  }
}

// Adam step (bias-corrected), step >= 1
// (1 - beta) and the bias corrections 1 - beta^step come in from the host,
// computed in FP64 (1.0f - 0.999f in FP32 is off by 1.3e-5 relative)
__global__ void k_mlp_adam(const float *__restrict__ G, float *__restrict__ P, float *__restrict__ M,
                           float *__restrict__ V, float lr, float b1, float b2, float omb1, float omb2, float bc1,
                           float bc2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  const float g = G[p];
  const float m = b1 * M[p] + omb1 * g;
  const float v = b2 * V[p] + omb2 * g * g;
  M[p] = m;
  V[p] = v;
  P[p] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

// features of every line-period of instance k (logging for training)
template <int BS>
__global__ void __launch_bounds__(BS) k_line_features(Dev S, int k, float *__restrict__ feat, double *__restrict__ sc) {
  const Inst I = S.inst[k];
  const long long n = (long long)I.T * I.nl;
  const long long loc = (long long)blockIdx.x * BS + threadIdx.x;
  if (loc >= n) return;
  const int t = (int)(loc / I.nl), l = (int)(loc - (long long)t * I.nl);
  float f[MLP_IN];
  double s;
  line_features<true>(S, I, (long long)I.bpo + loc, t, l, f, s);
#pragma unroll
  for (int j = 0; j < MLP_IN; ++j) feat[loc * MLP_IN + j] = f[j];
  sc[loc] = s;
}

// features of every line-period of the handle (global item order)
template <int BS>
__global__ void __launch_bounds__(BS) k_line_features_all(Dev S, float *__restrict__ feat, double *__restrict__ sc) {
  const long long bp = (long long)blockIdx.x * BS + threadIdx.x;
  if (bp >= S.NBP) return;
  int lo = 0, hi = S.K - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((long long)S.inst[mid].bpo <= bp) lo = mid; else hi = mid - 1;
  }
  const Inst &I = S.inst[lo];
  const int loc = (int)(bp - I.bpo), t = loc / I.nl, l = loc - t * I.nl;
  float f[MLP_IN];
  double s;
  line_features<true>(S, I, bp, t, l, f, s);
#pragma unroll
  for (int j = 0; j < MLP_IN; ++j) feat[bp * MLP_IN + j] = f[j];
  sc[bp] = s;
}

}  // namespace ucac
