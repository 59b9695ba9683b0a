// tg_fpconv.cuh -- FP64 <-> FP32 conversions, the double-FP32 ("double-float") numbers and
// their arithmetic, usable on the device and (for the CPU tests) on the host.
//
// Why the conversions are written out: GB300's FP64 pipe issues about two lanes per clock
// per SM (a kernel doing 16 FP64 operations per voxel saturated it at 590 G operations/s),
// 1/64 of the FP32 rate, and it also executes the FP64 <-> FP32 conversion instructions.  A
// streaming kernel that converts each value it reads is then bound by that pipe instead of
// by HBM.  The functions below produce the same results as the conversion instructions
// (round to nearest, ties to even) from integer bit operations and FP32 arithmetic; only
// rare operands (FP32-subnormal results, overflow, infinities, NaN) go to the instruction.
//
// A double-FP32 number hi + lo with |lo| <= ulp(hi) / 2 carries about 48 bits of
// significand.  Its operations are the classical error-free transformations: Knuth's
// two-sum for a + b and the fused multiply-add remainder a * b - fl(a * b) for products.
#pragma once

#include <cstdint>
#include <cstring>
#include <cmath>

#if defined(__CUDACC__)
#define TG_HD __host__ __device__ __forceinline__
#else
#define TG_HD inline
#endif

namespace tg {

namespace fpc {
TG_HD unsigned long long bits64(double x) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
TG_HD double from_bits64(unsigned hi, unsigned lo) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)hi, (int)lo);
#else
  const unsigned long long b = ((unsigned long long)hi << 32) | lo;
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}
TG_HD unsigned bits32(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof u);
  return u;
#endif
}
TG_HD float from_bits32(unsigned u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}
// rounded FP32 operations that the compiler may not contract or reorder
TG_HD float add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  volatile float s = a + b;
  return s;
#endif
}
TG_HD float sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  volatile float s = a - b;
  return s;
#endif
}
TG_HD float mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  volatile float s = a * b;
  return s;
#endif
}
TG_HD float fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}
TG_HD float div(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdiv_rn(a, b);
#else
  volatile float s = a / b;
  return s;
#endif
}
TG_HD float i2f(int d) {   // exact below 2^24, else rounded to nearest
#if defined(__CUDA_ARCH__)
  return __int2float_rn(d);
#else
  return (float)d;
#endif
}
// The conversion instructions, for the rare operands only.  They are kept out of line:
// inlined, the compiler turns the rare branch into predicated code, and predicated-off FP64
// instructions still occupy the FP64 pipe.
#if defined(__CUDACC__)
#define TG_HD_COLD static __host__ __device__ __noinline__
#else
#define TG_HD_COLD static __attribute__((noinline))
#endif
TG_HD_COLD float cvt_f32(double x) {
#if defined(__CUDA_ARCH__)
  return __double2float_rn(x);
#else
  return (float)x;
#endif
}
TG_HD_COLD double cvt_f64(float f) { return (double)f; }
TG_HD_COLD float cvt_tail(double x, float h) {   // fl32(x - h) for the split's rare operands
#if defined(__CUDA_ARCH__)
  return __double2float_rn(x - (double)h);
#else
  return (float)(x - (double)h);
#endif
}
}  // namespace fpc

// FP64 -> FP32, round to nearest even.  Normal FP32 results (2^-126 <= |x| < 2^127) and
// |x| < 2^-150 (which round to a signed zero) take integer operations only.
TG_HD float f32_of(double x) {
  const unsigned long long b = fpc::bits64(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e - 897u < 253u) {
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned t = lo & 0x1FFFFFFFu;   // the 29 bits below FP32's last place
    f += (t > 0x10000000u || (t == 0x10000000u && (f & 1u))) ? 1u : 0u;   // a carry bumps the exponent
    return fpc::from_bits32(f);
  }
  if (e < 873u) return fpc::from_bits32(hi & 0x80000000u);
  return fpc::cvt_f32(x);
}

// FP32 -> FP64 (exact).  Normal numbers and zeros take integer operations only.
TG_HD double f64_of(float f) {
  const unsigned u = fpc::bits32(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e - 1u < 254u)
    return fpc::from_bits64((u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xFFFFFu),
                            u << 29);
  if ((u & 0x7FFFFFFFu) == 0u) return fpc::from_bits64(u, 0u);
  return fpc::cvt_f64(f);
}

namespace fpc {
TG_HD_COLD double scale_slow(double x, double s) { return x * s; }
}  // namespace fpc
using fpc::scale_slow;

// f * s in FP64 for s = 2^k an exact power of two (normal): the exponent field of the
// converted value moved by k where the result stays normal, else an FP64 multiplication
TG_HD double f64_of_scaled(float f, double s) {
  const double x = f64_of(f);
  const unsigned long long b = fpc::bits64(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7FFu);
  const int k = (int)((fpc::bits64(s) >> 52) & 0x7FFu) - 1023;
  if (e != 0 && e != 0x7FF && e + k >= 1 && e + k <= 0x7FE)
    return fpc::from_bits64(hi + ((unsigned)k << 20), (unsigned)b);
  if ((b << 1) == 0ull) return x;   // +-0
  return scale_slow(x, s);
}

struct Df {
  float hi, lo;
};

// x = hi + lo with hi = fl32(x) and lo = fl32(x - hi).  x - hi is the FP64 tail below FP32's
// last place, sign(x) (t - c 2^29) 2^(E - 52) with t the 29 tail bits, c the rounding carry
// and E the exponent: an integer of at most 29 bits times a power of two, so lo is that
// integer rounded to FP32 and scaled exactly (twice rounded only where lo is FP32-subnormal).
TG_HD Df df_split(double x) {
  const unsigned long long b = fpc::bits64(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e - 897u < 253u) {
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const int t = (int)(lo & 0x1FFFFFFFu);
    const bool up = t > 0x10000000 || (t == 0x10000000 && (f & 1u));
    f += up ? 1u : 0u;
    const int d = up ? t - 0x20000000 : t;
    const int sd = (hi & 0x80000000u) ? -d : d;
    const float p2 = fpc::from_bits32((e - 896u) << 23);   // 2^E
    const float r = fpc::mul(fpc::mul(fpc::i2f(sd), 0x1p-52f), p2);
    return {fpc::from_bits32(f), r};
  }
  if (e < 873u) {
    const float z = fpc::from_bits32(hi & 0x80000000u);
    return {z, z};
  }
  const float h = fpc::cvt_f32(x);
  return {h, fpc::cvt_tail(x, h)};
}
inline Df df_split_host(double x) {   // the plain form, for constants set up on the host
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}
// hi + lo rounded to FP64: one FP64 addition of the exactly converted parts
TG_HD double df_value(Df x) { return f64_of(x.hi) + f64_of(x.lo); }

TG_HD Df df_two_sum(float a, float b) {
  const float s = fpc::add(a, b);
  const float bb = fpc::sub(s, a);
  const float e = fpc::add(fpc::sub(a, fpc::sub(s, bb)), fpc::sub(b, bb));
  return {s, e};
}
TG_HD Df df_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = fpc::add(a, b);
  return {s, fpc::sub(b, fpc::sub(s, a))};
}
TG_HD Df df_add(Df x, Df y) {
  Df s = df_two_sum(x.hi, y.hi);
  const Df t = df_two_sum(x.lo, y.lo);
  s = df_fast_two_sum(s.hi, fpc::add(s.lo, t.hi));
  return df_fast_two_sum(s.hi, fpc::add(s.lo, t.lo));
}
// x + y for operands of one sign (no cancellation): one two-sum of the leading parts, the
// tails added in FP32.  Relative error about 2^-46; this shorter ("sloppy") form loses its
// bound only where the operands cancel, which sums of positive coefficients never do.
TG_HD Df df_add_pos(Df x, Df y) {
  const Df s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, fpc::add(s.lo, fpc::add(x.lo, y.lo)));
}
TG_HD Df df_neg(Df x) { return {-x.hi, -x.lo}; }
TG_HD Df df_sub(Df x, Df y) { return df_add(x, df_neg(y)); }
TG_HD Df df_mul(Df x, Df y) {
  const float p = fpc::mul(x.hi, y.hi);
  float e = fpc::fma(x.hi, y.hi, -p);
  e = fpc::fma(x.hi, y.lo, e);
  e = fpc::fma(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
// A compensated sum s + c.  Each addend's leading part enters s through an error-free
// two-sum; that error, the addend's tail and the products' rounding errors (fused
// multiply-add remainders) collect in the FP32 compensation c.  This is the summation and dot
// product of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26,
// 2005) with double-FP32 operands: about 11 FP32 operations per product term against 26 for a
// double-FP32 product and addition, with an error of order 2^-48 of the terms' magnitudes.
struct CSum {
  float s, c;
};
TG_HD void cs_add(CSum& a, Df t) {   // a += t
  const Df q = df_two_sum(a.s, t.hi);
  a.s = q.hi;
  a.c = fpc::add(a.c, fpc::add(q.lo, t.lo));
}
TG_HD void cs_fma(CSum& a, Df x, Df y) {   // a += x y
  const float p = fpc::mul(x.hi, y.hi);
  const float e = fpc::fma(x.hi, y.hi, -p);
  const Df q = df_two_sum(a.s, p);
  a.s = q.hi;
  a.c = fpc::fma(x.hi, y.lo, fpc::fma(x.lo, y.hi, fpc::add(a.c, fpc::add(q.lo, e))));
}
TG_HD Df cs_value(CSum a) { return df_two_sum(a.s, a.c); }
// x - y for values whose difference matters only to 2^-48 of their own size (neighbouring
// nodes of a smooth field): one two-sum of the leading parts, the tails' difference added
TG_HD Df df_sub_near(Df x, Df y) {
  const Df q = df_two_sum(x.hi, -y.hi);
  return df_two_sum(q.hi, fpc::add(q.lo, fpc::sub(x.lo, y.lo)));
}

// x / y: the FP32 quotient, then one correction from the double-FP32 remainder x - q y
TG_HD Df df_div(Df x, Df y) {
  const float q = fpc::div(x.hi, y.hi);
  const Df r = df_sub(x, df_mul(Df{q, 0.0f}, y));
  return df_fast_two_sum(q, fpc::div(r.hi, y.hi));
}
// x / j for a small positive integer j (exact FP32 remainder of the leading part)
TG_HD Df df_div_int(Df x, float j) {
  const float q = fpc::div(x.hi, j);
  const float rem = fpc::fma(-q, j, x.hi);   // x.hi - q j exactly
  return df_fast_two_sum(q, fpc::div(fpc::add(rem, x.lo), j));
}

// expm1(x) for x <= 0 in double-FP32: halve x until |y| <= 1/8, sum the Taylor series
// y (1 + y (1/2 + y (1/6 + y (1/24 + y (1/120 + y R(y)))))), whose terms from y^6 / 720 on
// (below 4e-8 of the sum) form R in FP32 and the rest in double-FP32, then undo each halving
// with expm1(2y) = expm1(y) (2 + expm1(y)), which for y < 0 adds no relative error.
TG_HD Df df_expm1_neg(Df x) {
  int k = 0;
  Df y = x;
  while (y.hi < -0.125f && k < 12) {   // |x| < 2^9 needs at most 12 halvings
    y = {0.5f * y.hi, 0.5f * y.lo};
    ++k;
  }
  // 1/720 + y/5040 + y^2/40320 + y^3/362880 + y^4/3628800 (remainder below 3e-17 relative)
  const float yh = y.hi;
  const float R = fpc::fma(yh, fpc::fma(yh, fpc::fma(yh, fpc::fma(yh, 2.7557319e-7f, 2.7557319e-6f),
                                                     2.4801587e-5f), 1.9841270e-4f),
                           1.3888889e-3f);
  const Df c120 = {0.008333333767950535f, -4.34617203337595e-10f};
  const Df c24 = {0.0416666679084301f, -1.2417634698280722e-09f};
  const Df c6 = {0.1666666716337204f, -4.967053879312289e-09f};
  Df t = df_add(c120, df_mul(y, Df{R, 0.0f}));
  t = df_add(c24, df_mul(y, t));
  t = df_add(c6, df_mul(y, t));
  t = df_add(Df{0.5f, 0.0f}, df_mul(y, t));
  t = df_add(Df{1.0f, 0.0f}, df_mul(y, t));
  Df m = df_mul(y, t);
  for (int q = 0; q < k; ++q) m = df_mul(m, df_add(Df{2.0f, 0.0f}, m));
  return m;
}

// tanh(s) in double-FP32: tanh|s| = -m / (2 + m) with m = expm1(-2|s|), odd in s; 1 where
// |s| >= 17 (1 - tanh 17 < 4e-15).  Relative error about 1e-14.
TG_HD Df df_tanh(Df s) {
  const bool neg = s.hi < 0.0f;
  const Df a = neg ? df_neg(s) : s;
  if (a.hi >= 17.0f) return {neg ? -1.0f : 1.0f, 0.0f};   // (NaN falls through)
  const Df m = df_expm1_neg(Df{-2.0f * a.hi, -2.0f * a.lo});
  const Df t = df_div(df_neg(m), df_add(Df{2.0f, 0.0f}, m));
  return neg ? df_neg(t) : t;
}

}  // namespace tg
