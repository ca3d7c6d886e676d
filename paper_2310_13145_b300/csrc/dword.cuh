// dword.cuh -- double-word arithmetic on the FP32 pipe.
//
// B300 executes FP64 at 1/64 of its FP32 rate: an FP64 warp instruction
// holds an SM's FP64 unit for 16 cycles, while the same SM issues four FP32
// warp instructions per cycle.  A value carried as the unevaluated sum
// h + l of two floats (a "double-word", |l| < ulp(h)) holds ~48 significant
// bits, and its operations cost 3-15 FP32 instructions, so evaluations whose
// accuracy needs more than FP32 but far less than FP64's 53 bits run much
// faster this way.  The building blocks are the classical error-free
// transformations, written here from their published definitions:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, 6 operations;
//   Fast2Sum (Dekker 1971): the same for |a| >= |b|, 3 operations;
//   TwoProd with an FMA: p + e = a b exactly, 2 operations;
// and the double-word sum, product and product by a float follow the
// algorithms of Joldes, Muller and Popescu, "Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic" (ACM TOMS 44, 2017):
// relative error a few u^2 (u = 2^-24), at most 16 u^2 = 2^-44 for operands
// straight from dw_from_d (whose low parts reach ulp(h), twice a normalised
// pair's; the product also drops the low parts' product), except the sums,
// whose error is a few u^2 (|x| + |y|) (absolute, as for FP64 operands that
// carry their own rounding).
//
// Every operation is spelled with explicitly rounded intrinsics, so that the
// compiler neither contracts nor reorders it; the same source compiles for
// the host (g++, -ffp-contract=off) and gives the same bits, which is how the
// tests check the device arithmetic.  Conversions to and from FP64 run on the
// integer units (dw_from_d) or as one exact FP64 addition (dw_to_d): the FP64
// pipe also executes the hardware conversions, at the FP64 rate.
#pragma once
#include <stdint.h>
#include <string.h>
#include <math.h>

#if defined(__CUDACC__)
#define DW_HD __host__ __device__ __forceinline__
#else
#define DW_HD inline
#endif

namespace ucac {

struct dw {
  float h, l;
};

DW_HD float dw_fadd(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DW_HD float dw_fsub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DW_HD float dw_fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DW_HD float dw_ffma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
DW_HD uint32_t dw_fbits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}
DW_HD float dw_bitsf(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}
DW_HD uint64_t dw_dbits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}
DW_HD double dw_bitsd(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}
// count of leading zeros of a nonzero 32-bit word
DW_HD int dw_clz(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __clz((int)x);
#else
  return __builtin_clz(x);
#endif
}

// ---------------------------------------------------- error-free sums ----
DW_HD void two_sum(float a, float b, float &s, float &e) {
  s = dw_fadd(a, b);
  const float bb = dw_fsub(s, a);
  e = dw_fadd(dw_fsub(a, dw_fsub(s, bb)), dw_fsub(b, bb));
}
DW_HD void fast_two_sum(float a, float b, float &s, float &e) {
  s = dw_fadd(a, b);
  e = dw_fsub(b, dw_fsub(s, a));
}
DW_HD void two_prod(float a, float b, float &p, float &e) {
  p = dw_fmul(a, b);
  e = dw_ffma(a, b, -p);
}

DW_HD dw dw_make(float h) { return dw{h, 0.0f}; }
DW_HD dw dw_neg(dw x) { return dw{-x.h, -x.l}; }
// x * 2^k for a power of two p = 2^k (exact while no part leaves the range)
DW_HD dw dw_pow2(dw x, float p) { return dw{dw_fmul(x.h, p), dw_fmul(x.l, p)}; }

// x + y (the "sloppy" double-word sum: TwoSum of the high parts, the low
// parts added, one Fast2Sum; 11 operations)
DW_HD dw dw_add(dw x, dw y) {
  float sh, sl, zh, zl;
  two_sum(x.h, y.h, sh, sl);
  const float v = dw_fadd(x.l, y.l);
  const float w = dw_fadd(sl, v);
  fast_two_sum(sh, w, zh, zl);
  return dw{zh, zl};
}
DW_HD dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
// x + b for a float b (10 operations)
DW_HD dw dw_add_f(dw x, float b) {
  float sh, sl, zh, zl;
  two_sum(x.h, b, sh, sl);
  const float v = dw_fadd(x.l, sl);
  fast_two_sum(sh, v, zh, zl);
  return dw{zh, zl};
}
// x * y (TwoProd of the high parts, the cross terms by FMA; 8 operations)
DW_HD dw dw_mul(dw x, dw y) {
  float ch, cl, zh, zl;
  two_prod(x.h, y.h, ch, cl);
  const float t = dw_fmul(x.h, y.l);
  const float c2 = dw_ffma(x.l, y.h, t);
  const float c3 = dw_fadd(cl, c2);
  fast_two_sum(ch, c3, zh, zl);
  return dw{zh, zl};
}
// x * b for a float b (6 operations)
DW_HD dw dw_mul_f(dw x, float b) {
  float ch, cl, zh, zl;
  two_prod(x.h, b, ch, cl);
  const float c3 = dw_ffma(x.l, b, cl);
  fast_two_sum(ch, c3, zh, zl);
  return dw{zh, zl};
}
// x^2 (6 operations)
DW_HD dw dw_sqr(dw x) {
  float ch, cl, zh, zl;
  two_prod(x.h, x.h, ch, cl);
  const float c3 = dw_ffma(dw_fadd(x.h, x.h), x.l, cl);
  fast_two_sum(ch, c3, zh, zl);
  return dw{zh, zl};
}
// x * y + z: the product's high part enters a TwoSum with z's, every other
// term (the product's rounding error, the cross terms, z's low part, the
// TwoSum's error) is collected in one float, then one Fast2Sum (15
// operations; the error of the sum above, relative to |x y| + |z|)
DW_HD dw dw_fma(dw x, dw y, dw z) {
  float ph, pl, sh, sl, zh, zl;
  two_prod(x.h, y.h, ph, pl);
  two_sum(ph, z.h, sh, sl);
  float t = dw_ffma(x.h, y.l, pl);
  t = dw_ffma(x.l, y.h, t);
  t = dw_fadd(t, dw_fadd(z.l, sl));
  fast_two_sum(sh, t, zh, zl);
  return dw{zh, zl};
}

// ---------------------------------------------------------- conversions ---
// FP64 -> double-word on the integer units: h keeps the top 24 significant
// bits of x (truncation), l the next 24 (truncation), so h + l = x to 2^-47
// relative, with l of x's sign (or zero) and |l| < ulp(h).  A magnitude
// below 2^-126 becomes a signed zero, one at or above 2^128 (infinities, NaN)
// a NaN; the low part is kept, as a subnormal float where it falls below
// FP32's normal range, while |x| >= 2^-102 and dropped below that, so the
// error bound is 2^-47 |x| + 2^-126 (the relative bound alone holds for
// |x| >= 2^-102).
DW_HD dw dw_from_d(double x) {
  const uint64_t b = dw_dbits(x);
  const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
  const uint32_t a = bh & 0x7fffffffu, sg = bh & 0x80000000u;  // (the range tests compare a: e = a >> 20)
  // the 32 bits from bit 29 up hold e's low 9 bits above the 23 fraction
  // bits h keeps; adding 2^30 = 2^32 - (896 << 23) modulo 2^32 rebiases the
  // exponent, which is exact in those 9 bits (and leaves bit 31 clear) for
  // 897 <= e <= 1150
  const uint32_t hx = (uint32_t)(b >> 29) + 0x40000000u;
  const bool small = a < 0x38100000u, big = a >= 0x47f00000u;  // e <= 896, e >= 1151
  const float h = dw_bitsf(small ? sg : (big ? (sg | 0x7fc00000u) : (sg | hx)));
  // l: the 24 bits below h's, R = bits 28..5 of bl, are worth R 2^(e - 1070).
  // A float of x's sign with exponent field e - 920 and R's low 23 bits as
  // fraction is worth 2^(e - 1047) + (R mod 2^23) 2^(e - 1070); where R's top
  // bit is clear, subtracting the float 2^(e - 1047) of the same sign leaves
  // R 2^(e - 1070) exactly (both share one exponent), and where it is set
  // that 2^(e - 1047) is R's own top bit
  const uint32_t eb = (sg | (hx & 0x7f800000u)) - (24u << 23);
  const uint32_t fl = eb | ((bl >> 5) & 0x7fffffu);
  const float l0 = dw_fsub(dw_bitsf(fl), dw_bitsf((bl & 0x10000000u) != 0u ? 0u : eb));
  const float l = a - 0x39900000u < 0x0e600000u ? l0 : dw_bitsf(sg);  // 921 <= e <= 1150
  return dw{h, l};
}
// float -> FP64 exactly on the integer units (a subnormal float becomes a
// signed zero; infinities and NaN keep their kind).  With the sign cleared,
// a >> 3 holds the exponent field in bits 27..20 above the top 20 fraction
// bits, so one addition of 896 << 20 rebiases it (1792 << 20 takes the
// field 255 of infinities and NaN to 2047)
DW_HD double dw_f2d(float x) {
  const uint32_t u = dw_fbits(x);
  const uint32_t a = u & 0x7fffffffu, sg = u & 0x80000000u;
  const uint32_t hi = sg | ((a >> 3) + (a >= 0x7f800000u ? (1792u << 20) : (896u << 20)));
  const bool z = a < 0x00800000u;
  return dw_bitsd(((uint64_t)(z ? sg : hi) << 32) | (z ? 0u : (u << 29)));
}
// double-word -> FP64: h + l is exact in FP64 (at most 49 significant bits
// for a normalised pair), so one FP64 addition of the widened parts (a
// subnormal low part is dropped by dw_f2d: an error below 2^-126)
DW_HD double dw_to_d(dw x) {
#if defined(__CUDA_ARCH__)
  return __dadd_rn(dw_f2d(x.h), dw_f2d(x.l));
#else
  return dw_f2d(x.h) + dw_f2d(x.l);
#endif
}

// The operations above applied to FP64 inputs (each converted by
// dw_from_d), for the tests that compare the device arithmetic with the
// host's bit for bit: out[0..3] receive the result's parts as doubles.
//   0: x -> (h, l, dw_to_d, the bit pattern of l as an integer)
//   1: x + y   2: x - y   3: x + (float)y
//   4: x * y   5: x * (float)y   6: x^2   7: x * y + z
DW_HD void dw_probe_op(int op, double x, double y, double z, double *out) {
  const dw a = dw_from_d(x), b = dw_from_d(y), cc = dw_from_d(z);
  const float fy = b.h;
  dw r{0.0f, 0.0f};
  out[2] = 0.0;
  out[3] = 0.0;
  switch (op) {
    case 0: r = a; out[2] = dw_to_d(a); out[3] = (double)dw_fbits(a.l); break;
    case 1: r = dw_add(a, b); break;
    case 2: r = dw_sub(a, b); break;
    case 3: r = dw_add_f(a, fy); break;
    case 4: r = dw_mul(a, b); break;
    case 5: r = dw_mul_f(a, fy); break;
    case 6: r = dw_sqr(a); break;
    case 7: r = dw_fma(a, b, cc); break;
    default: break;
  }
  out[0] = dw_f2d(r.h);
  out[1] = dw_f2d(r.l);
}

}  // namespace ucac
