// fe_arith.h -- number types of the apply kernels: double-word arithmetic, the value traits of
// each arithmetic, and the 1D tables (with their even-odd forms).
//
// Number types.  The FP64 path of the library computes in double-word ("double-float")
// arithmetic on the FP32 pipe: a value is an unevaluated sum hi + lo of two floats (Dekker 1971;
// error-free TwoSum/TwoProd as in Joldes, Muller, Popescu, "Tight and rigorous error bounds for
// basic building blocks of double-word arithmetic", ACM TOMS 2017).  GB300 executes FP64 FMAs at
// about 1/70 of its FP32 rate, so this is the arithmetic that lets an FP64-accurate operator get
// near the memory roofline.  The same sweep code is instantiated for `double` (the FP64 pipe,
// kept as a cross-check variant), for `float` (the FP32 path of mixed precision) and for float
// values with 16-bit product operands.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define FE_MAXN 8

// ---------------------------------------------------------------------------------------------
// double-word arithmetic
// ---------------------------------------------------------------------------------------------
struct dw {
  float h, l;
};

// All double-word primitives use the _rn intrinsics so that the compiler never contracts a
// product and a sum into one FMA, which would break the error-free transformations.
__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
// unnormalised accumulator acc + c*v, 10 FP32 operations.  s = acc.h + p with p = fl(c.h v.h); of
// the TwoSum error, acc.h's share t1 = acc.h - (s - bb) is exact (bb = s - acc.h), and p's share
// p - bb plus the product error c.h v.h - p is c.h v.h - bb, one fma (a small value rounded once,
// an error of order 2^-24 ulp(s)).  The low parts and cross products go in float.
// The 12-operation form: exact product error and a full TwoSum, low parts summed in float.
__device__ __forceinline__ dw dw_mac12(dw acc, dw c, dw v) {
  float p = __fmul_rn(c.h, v.h);
  float e = __fmaf_rn(c.h, v.h, -p);
  e = __fmaf_rn(c.h, v.l, e);
  e = __fmaf_rn(c.l, v.h, e);
  dw s = dw_two_sum(acc.h, p);
  return {s.h, __fadd_rn(acc.l, __fadd_rn(s.l, e))};
}
#ifndef FE_MAC_V1
__device__ __forceinline__ dw dw_mac(dw acc, dw c, dw v) {
  const float p = __fmul_rn(c.h, v.h);
  const float s = __fadd_rn(acc.h, p);
  const float bb = __fsub_rn(s, acc.h);
  const float t1 = __fsub_rn(acc.h, __fsub_rn(s, bb));
  const float t2 = __fmaf_rn(c.h, v.h, -bb);
  const float x = __fmaf_rn(c.l, v.h, __fmaf_rn(c.h, v.l, acc.l));
  return {s, __fadd_rn(__fadd_rn(t1, t2), x)};
}
#else
__device__ __forceinline__ dw dw_mac(dw acc, dw c, dw v) { return dw_mac12(acc, c, v); }
#endif
// c*v as an unnormalised pair (the first term of a dot product: no TwoSum with a zero accumulator)
__device__ __forceinline__ dw dw_prod(dw c, dw v) {
  float p = __fmul_rn(c.h, v.h);
  float e = __fmaf_rn(c.h, v.h, -p);
  e = __fmaf_rn(c.h, v.l, e);
  e = __fmaf_rn(c.l, v.h, e);
  return {p, e};
}
__device__ __forceinline__ dw dw_add_keep(dw a, dw b) {
  dw s = dw_two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ dw dw_norm(dw a) { return dw_fast_two_sum(a.h, a.l); }
__device__ __forceinline__ dw dw_add(dw a, dw b) {
  dw s = dw_two_sum(a.h, b.h);
  return dw_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dw dw_mul(dw a, dw b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dw_fast_two_sum(p, e);
}

// Out-of-range paths of the conversions below, kept out of line: inlined, the compiler
// predicates them into every call, and their conversions and FP64 adds then occupy the slow FP64
// pipe even though they never take effect.
static __device__ __noinline__ dw dw_from_double_slow(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

// binary64 -> double-word by bit manipulation on the integer pipe (FP64<->FP32 conversions run
// at the FP64 rate on GB300).  hi = x truncated to 24 significant bits, lo = the remaining 29
// bits rounded to float.  Exact range 2^-74 <= |x| < 2^128; other values take the FP64 path.
__device__ __forceinline__ dw dw_from_double(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  if (e - 949u <= 201u) {
    unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    float hi = __uint_as_float(sign | ((e - 896u) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
    // float of the 29-bit integer m without an int->float conversion (those issue on the slow FP64
    // pipe): low 23 and high 6 bits are exact floats through the 2^23 bias, and the fma rounds
    // m once, as a conversion would
    const unsigned m = (unsigned)b & 0x1FFFFFFFu;
    const float flo = __fsub_rn(__uint_as_float(0x4B000000u | (m & 0x7FFFFFu)), 8388608.0f);
    const float fhi = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 23)), 8388608.0f);
    float lo = __fmul_rn(__fmaf_rn(fhi, 8388608.0f, flo), __uint_as_float((e - 948u) << 23));
    lo = __uint_as_float(__float_as_uint(lo) | sign);
    return {hi, lo};
  }
  return dw_from_double_slow(x);
}
// x * 2^-sh as a double-word: dw_from_double on the scaled exponent (sh from the CTA's largest
// input, see cta_exp_shift in fe_apply_kernel.cuh).  Zero and subnormal x give 0; values that
// the scaling leaves outside the exact range take the FP64 path (out of line).
static __device__ __noinline__ dw dw_from_double_sh_slow(double x, int sh) {
  const double v = scalbn(x, -sh);
  const float hi = __double2float_rn(v);
  return {hi, __double2float_rn(v - (double)hi)};
}
__device__ __forceinline__ dw dw_from_double_sh(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned e0 = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned e = e0 - (unsigned)sh;
  if (e - 949u <= 201u && e0 - 1u < 2046u) {  // finite, normal, in range after the shift
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | ((e - 896u) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
    const unsigned m = (unsigned)b & 0x1FFFFFFFu;
    const float flo = __fsub_rn(__uint_as_float(0x4B000000u | (m & 0x7FFFFFu)), 8388608.0f);
    const float fhi = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 23)), 8388608.0f);
    float lo = __fmul_rn(__fmaf_rn(fhi, 8388608.0f, flo), __uint_as_float((e - 948u) << 23));
    lo = __uint_as_float(__float_as_uint(lo) | sign);
    return {hi, lo};
  }
  if (e0 == 0u) return {0.0f, 0.0f};
  return dw_from_double_sh_slow(x, sh);
}

// x * 2^-sh as a double-word without a branch: exact (as dw_from_double) for
// 2^-74 <= |x| 2^-sh < 2^128; smaller values, zero and subnormals give 0; infinities and NaN give
// NaN.  The callers choose sh so that no scaled value reaches 2^128.
__device__ __forceinline__ dw dw_from_double_ftz(double x, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned e0 = (unsigned)(b >> 52) & 0x7FFu;
  const unsigned e = e0 - (unsigned)sh;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sign | (((e - 896u) & 0xFFu) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
  const unsigned m = (unsigned)b & 0x1FFFFFFFu;
  const float flo = __fsub_rn(__uint_as_float(0x4B000000u | (m & 0x7FFFFFu)), 8388608.0f);
  const float fhi = __fsub_rn(__uint_as_float(0x4B000000u | (m >> 23)), 8388608.0f);
  float lo = __fmul_rn(__fmaf_rn(fhi, 8388608.0f, flo), __uint_as_float(((e - 948u) & 0xFFu) << 23));
  lo = __uint_as_float(__float_as_uint(lo) | sign);
  const bool in = e - 949u <= 201u && e0 != 0u;
  const float nan = __uint_as_float(0x7FC00000u);
  return e0 == 0x7FFu ? dw{nan, nan} : (in ? dw{hi, lo} : dw{0.0f, 0.0f});
}

// float -> binary64 exactly for normal floats by bit manipulation; zero and subnormal -> 0.
__device__ __forceinline__ double f2d_bits(float f) {
  unsigned u = __float_as_uint(f);
  unsigned e = (u >> 23) & 0xFFu;
  if (e - 1u < 254u) {
    unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                           ((unsigned long long)(e + 896u) << 52) |
                           ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
  }
  if (e == 0u) return 0.0;
  return (double)f;  // inf / nan
}
__device__ __forceinline__ double dw_to_double(dw a) { return f2d_bits(a.h) + f2d_bits(a.l); }
static __device__ __noinline__ double dw_to_double_slow(dw a) { return f2d_bits(a.h) + f2d_bits(a.l); }

// binary64 of h + l on the integer and FP32 pipes (no FP64 add): after a TwoSum |l| <= ulp(h)/2,
// so l is at most 2^28 units of 2^(e-52), e the exponent of h; those units, truncated to an
// integer, are added to (or, for opposite signs, subtracted from) the bit pattern of h, whose
// low 29 mantissa bits are zero.  Subtracting from a power of two crosses into the binade below,
// where the unit is half as large.  Result within 2^(e-52) of h + l (about one double ulp).
// Zero and the exponent range outside 2^-75 .. 2^127 take the FP64 path.
__device__ __forceinline__ double dw_to_double_int(dw a) {
  const dw s = dw_two_sum(a.h, a.l);
  const unsigned hb = __float_as_uint(s.h);
  const unsigned e8 = (hb >> 23) & 0xFFu;
  if (s.h == 0.0f) return 0.0;
  if (e8 - 52u > 202u) return dw_to_double_slow(s);
  const unsigned long long dh = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                ((unsigned long long)(e8 + 896u) << 52) |
                                ((unsigned long long)(hb & 0x7FFFFFu) << 29);
  const float v = __fmul_rn(fabsf(s.l), __uint_as_float((306u - e8) << 23));
  const unsigned vb = __float_as_uint(v);
  const int ev = (int)(vb >> 23) - 127;
  const unsigned mv = (vb & 0x7FFFFFu) | 0x800000u;
  const unsigned li = ev >= 23 ? (mv << (ev - 23)) : (ev >= 0 ? (mv >> (23 - ev)) : 0u);
  unsigned long long out;
  if (((hb ^ __float_as_uint(s.l)) & 0x80000000u) == 0u)
    out = dh + li;
  else
    out = dh - ((hb & 0x7FFFFFu) == 0u ? 2ull * li : (unsigned long long)li);
  return __longlong_as_double((long long)out);
}

// (h + l) * 2^sh as binary64: dw_to_double_int, then sh added to the exponent field; results
// that leave the normal binary64 range take the FP64 path (out of line).
static __device__ __noinline__ double dw_to_double_sh_slow(double v, int sh) { return scalbn(v, sh); }
__device__ __forceinline__ double dw_to_double_sh(dw a, int sh) {
  const double v = dw_to_double_int(a);
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
  if (e == 0u || sh == 0) return v;
  if (e != 0x7FFu && (e + (unsigned)sh) - 1u < 2046u)
    return __longlong_as_double((long long)(b + ((unsigned long long)(long long)sh << 52)));
  return dw_to_double_sh_slow(v, sh);
}

// ---------------------------------------------------------------------------------------------
// number traits: value type V, storage type of vectors (SV) and of geometry (GV)
// ---------------------------------------------------------------------------------------------
template <class V>
struct NT;

template <>
struct NT<double> {
  using SV = double;
  using GV = double;
  static constexpr bool LOWP = false;
  __device__ static __forceinline__ double zero() { return 0.0; }
  __device__ static __forceinline__ double mac(double a, double c, double v) { return fma(c, v, a); }
  __device__ static __forceinline__ double mac12(double a, double c, double v) { return fma(c, v, a); }
  __device__ static __forceinline__ double prod(double c, double v) { return c * v; }
  __device__ static __forceinline__ double addk(double a, double b) { return a + b; }
  __device__ static __forceinline__ double subk(double a, double b) { return a - b; }
  __device__ static __forceinline__ double fin(double a) { return a; }
  __device__ static __forceinline__ double keep(double a) { return a; }
  __device__ static __forceinline__ double mul(double a, double b) { return a * b; }
  __device__ static __forceinline__ double add(double a, double b) { return a + b; }
  __device__ static __forceinline__ double sub(double a, double b) { return a - b; }
  __device__ static __forceinline__ double recip(double a) { return 1.0 / a; }
  __device__ static __forceinline__ double neg(double a) { return -a; }
  __device__ static __forceinline__ double load(const double* p) { return __ldg(p); }
  __device__ static __forceinline__ double load_stream(const double* p) { return __ldcs(p); }
  __device__ static __forceinline__ void store(double* p, double v, int = 0) { __stcs(p, v); }
  __device__ static __forceinline__ double to_sv(double v, int = 0) { return v; }
  __device__ static __forceinline__ void store_sv(double* p, double v) { __stcs(p, v); }
  __device__ static __forceinline__ double geo(const double* p) { return __ldcs(p); }
};

template <>
struct NT<float> {
  using SV = float;
  using GV = float;
  static constexpr bool LOWP = false;
  __device__ static __forceinline__ float zero() { return 0.0f; }
  __device__ static __forceinline__ float mac(float a, float c, float v) { return fmaf(c, v, a); }
  __device__ static __forceinline__ float mac12(float a, float c, float v) { return fmaf(c, v, a); }
  __device__ static __forceinline__ float prod(float c, float v) { return c * v; }
  __device__ static __forceinline__ float addk(float a, float b) { return a + b; }
  __device__ static __forceinline__ float subk(float a, float b) { return a - b; }
  __device__ static __forceinline__ float fin(float a) { return a; }
  __device__ static __forceinline__ float keep(float a) { return a; }
  __device__ static __forceinline__ float mul(float a, float b) { return a * b; }
  __device__ static __forceinline__ float add(float a, float b) { return a + b; }
  __device__ static __forceinline__ float sub(float a, float b) { return a - b; }
  __device__ static __forceinline__ float recip(float a) { return 1.0f / a; }
  __device__ static __forceinline__ float neg(float a) { return -a; }
  __device__ static __forceinline__ float load(const float* p) { return __ldg(p); }
  __device__ static __forceinline__ float load_stream(const float* p) { return __ldcs(p); }
  __device__ static __forceinline__ void store(float* p, float v, int = 0) { __stcs(p, v); }
  __device__ static __forceinline__ float to_sv(float v, int = 0) { return v; }
  __device__ static __forceinline__ void store_sv(float* p, float v) { __stcs(p, v); }
  __device__ static __forceinline__ float geo(const float* p) { return __ldcs(p); }
};

// 16-bit contractions with FP32 accumulation (FE_BF16_F32ACC, FE_F16_F32ACC): a value is a float,
// but every operand of a product (inputs, intermediate sweep values, 1D coefficients, metric) is
// rounded to the 16-bit format, so each product is exact in FP32 and only the accumulation is
// FP32.  Vectors are FP32 arrays; the metric is stored in the 16-bit format.
struct bfv {
  float v;
  static constexpr bool BF = true;
};
struct hfv {
  float v;
  static constexpr bool BF = false;
};
template <class W>
struct NT16 {
  using SV = float;
  using GV = unsigned short;  // bits of the 16-bit metric value
  static constexpr bool LOWP = true;
  __device__ static __forceinline__ float rnd(float x) {
    if constexpr (W::BF)
      return __bfloat162float(__float2bfloat16_rn(x));
    else
      return __half2float(__float2half_rn(x));
  }
  __device__ static __forceinline__ W zero() { return {0.0f}; }
  __device__ static __forceinline__ W mac(W a, W c, W x) { return {fmaf(c.v, x.v, a.v)}; }
  __device__ static __forceinline__ W mac12(W a, W c, W x) { return {fmaf(c.v, x.v, a.v)}; }
  __device__ static __forceinline__ W prod(W c, W x) { return {c.v * x.v}; }
  __device__ static __forceinline__ W addk(W a, W b) { return {rnd(a.v + b.v)}; }
  __device__ static __forceinline__ W subk(W a, W b) { return {rnd(a.v - b.v)}; }
  __device__ static __forceinline__ W fin(W a) { return a; }
  __device__ static __forceinline__ W keep(W a) { return {rnd(a.v)}; }
  __device__ static __forceinline__ W mul(W a, W b) { return {a.v * b.v}; }
  __device__ static __forceinline__ W add(W a, W b) { return {a.v + b.v}; }
  __device__ static __forceinline__ W sub(W a, W b) { return {a.v - b.v}; }
  __device__ static __forceinline__ W recip(W a) { return {1.0f / a.v}; }
  __device__ static __forceinline__ W neg(W a) { return {-a.v}; }
  __device__ static __forceinline__ W load(const float* p) { return {rnd(__ldg(p))}; }
  __device__ static __forceinline__ W load_stream(const float* p) { return {rnd(__ldcs(p))}; }
  __device__ static __forceinline__ void store(float* p, W x, int = 0) { __stcs(p, x.v); }
  __device__ static __forceinline__ W geo(const unsigned short* p) {
    const unsigned short b = __ldcs(p);
    if constexpr (W::BF)
      return {__uint_as_float((unsigned)b << 16)};
    else
      return {__half2float(__ushort_as_half(b))};
  }
};

template <>
struct NT<dw> {
  using SV = double;
  using GV = float2;
  static constexpr bool LOWP = false;
  __device__ static __forceinline__ dw zero() { return {0.0f, 0.0f}; }
  __device__ static __forceinline__ dw mac(dw a, dw c, dw v) { return dw_mac(a, c, v); }
  // the 12-operation form, for the geometry terms (their error reaches every output)
  __device__ static __forceinline__ dw mac12(dw a, dw c, dw v) { return dw_mac12(a, c, v); }
  __device__ static __forceinline__ dw prod(dw c, dw v) { return dw_prod(c, v); }
  // unnormalised sums (TwoSum of the high parts, low parts added in float): the error stays at
  // the double-word level of the operands, which is all the following products need
  __device__ static __forceinline__ dw addk(dw a, dw b) { return dw_add_keep(a, b); }
  __device__ static __forceinline__ dw subk(dw a, dw b) { return dw_add_keep(a, {-b.h, -b.l}); }
  __device__ static __forceinline__ dw fin(dw a) { return dw_norm(a); }
  // intermediate results of the sweeps stay unnormalised: |lo| stays below a few ulp(hi), and the
  // next products use lo only in FP32 cross terms (relative effect ~2^-45)
  __device__ static __forceinline__ dw keep(dw a) { return a; }
  __device__ static __forceinline__ dw mul(dw a, dw b) { return dw_mul(a, b); }
  __device__ static __forceinline__ dw add(dw a, dw b) { return dw_add(a, b); }
  __device__ static __forceinline__ dw sub(dw a, dw b) { return dw_add(a, {-b.h, -b.l}); }
  // one Newton step from the float reciprocal: r = r0 + r0 (1 - a r0)
  __device__ static __forceinline__ dw recip(dw a) {
    const float r0 = __frcp_rn(a.h);
    const dw e = dw_add({1.0f, 0.0f}, dw_mul(a, {-r0, 0.0f}));
    return dw_add({r0, 0.0f}, dw_mul({r0, 0.0f}, e));
  }
  __device__ static __forceinline__ dw neg(dw a) { return {-a.h, -a.l}; }
  __device__ static __forceinline__ dw load(const double* p) { return dw_from_double(__ldg(p)); }
  __device__ static __forceinline__ dw load_stream(const double* p) { return dw_from_double(__ldcs(p)); }
  // stores of values computed on inputs scaled by 2^-sh (the CTA's exponent shift)
  __device__ static __forceinline__ void store(double* p, dw v, int sh = 0) {
    __stcs(p, dw_to_double_sh(v, sh));
  }
  // the stored value (binary64) and its store, for sums formed on stored values
  __device__ static __forceinline__ double to_sv(dw v, int sh = 0) { return dw_to_double_sh(v, sh); }
  __device__ static __forceinline__ void store_sv(double* p, double v) { __stcs(p, v); }
  __device__ static __forceinline__ dw geo(const float2* p) {
    float2 g = __ldcs(p);
    return {g.x, g.y};
  }
};
template <>
struct NT<bfv> : NT16<bfv> {};
template <>
struct NT<hfv> : NT16<hfv> {};

// ---------------------------------------------------------------------------------------------
// 1D tables passed by value as kernel parameters (they land in the constant bank and are read
// with compile-time offsets).  Index convention: A[q][i] maps node/point i to point q.
// ---------------------------------------------------------------------------------------------
// Even-odd form of an n x n matrix M with the reflection symmetry M[n-1-q][n-1-r] = sig M[q][r]
// (sig = +1 for V, -1 for D: node and point sets are symmetric about 1/2).  With
// e_r = x_r + x_{n-1-r} and o_r = x_r - x_{n-1-r} (r < n/2), a = sum_r A[q][r] e_r (+ cm[q] x_mid),
// b = sum_r B[q][r] o_r:  (M x)_q = a + b and (M x)_{n-1-q} = sig (a - b); for odd n the middle
// output is sum_r cr[r] e_r + mm x_mid (sig = +1) or sum_r cr[r] o_r (sig = -1).  About half the
// multiply-adds of the plain product.
template <int N, class V>
struct EO {
  static constexpr int H = N / 2;
  V A[H][H];  // (M[q][r] + M[q][n-1-r]) / 2
  V B[H][H];  // (M[q][r] - M[q][n-1-r]) / 2
  V cm[H];    // M[q][mid]   (odd n)
  V cr[H];    // M[mid][r]   (odd n)
  V mm;       // M[mid][mid] (odd n, sig = +1)
};

// Even-odd form of the n x (n-1) matrix B' that maps the n-1 differences d_s = x_{s+1} - x_s of a
// line's nodal values to the derivative at the n Gauss points: B'[q][s] = sum_{r > s} B[q][r],
// B[q][r] = l_r'(s_q) (B x = B' d because the rows of B sum to zero).  B' is even under the
// reflection (q, s) -> (n-1-q, n-2-s); with e_s = d_s + d_{n-2-s}, o_s = d_s - d_{n-2-s}
// (s < (n-1)/2), a = sum_s A[q][s] e_s (+ cm[q] d_mid for even n), b = sum_s B[q][s] o_s:
// output q is a + b and output n-1-q is a - b; for odd n the middle output is sum_s cr[s] e_s.
template <int N, class V>
struct EOB {
  static constexpr int NI = N - 1, HI = NI / 2, HO = N / 2;
  static constexpr int HA = HI > 0 ? HI : 1;
  V A[HO][HA];
  V B[HO][HA];
  V cm[HO];  // B'[q][(n-2)/2]   (even n: the middle difference)
  V cr[HA];  // B'[(n-1)/2][s]   (odd n: the middle output)
};

template <int N, class V>
struct Tab1D {
  V V_[N][N];  // V[q][i]  = l_i(s_q): GLL-node Lagrange basis at Gauss point q      (Sec. 2.3 "V")
  V D_[N][N];  // D[q][r]  = derivative of the Gauss-point Lagrange basis r at s_q (collocation)
  V W_[N];     // Gauss weights on [0,1]
  EO<N, V> eV, eVT, eD, eDT;  // even-odd forms of V, V^T, D, D^T
  EOB<N, V> eB;               // even-odd form of B' (derivative from nodal differences)
};
