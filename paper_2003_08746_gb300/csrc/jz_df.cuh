// Double-float ("FP32 pair") arithmetic for the FP64 form's stage passes.
//
// A value is an unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48
// significant bits (relative precision ~2^-48 against FP64's 2^-53).  On a GB300 the FP64
// pipe retires 2 operations per SM per clock against 128 for FP32, so a double-float
// operation of 6-20 FP32 instructions is still several times cheaper than one FP64
// instruction; the FP64 form's parity bar (1e-12 relative on the state) leaves room for the
// extra rounding (measured by the parity tests).
//
// The building blocks are the error-free transformations of the literature:
//   two_sum       Knuth, The Art of Computer Programming vol. 2, Sec. 4.2.2 (s + e = a + b exactly)
//   fast_two_sum  Dekker (1971), for |a| >= |b|
//   two_prod      the product error by one fused multiply-add (a * b = p + e exactly)
// and the double-word sum, product and quotient built from them as in Dekker (1971) and in
// Joldes, Muller & Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44 (2017): the "sloppy" sum (error relative to |x| + |y|)
// and the product with three fused multiply-adds.  Reciprocal, square root and cube roots are
// one Newton (or third-order) correction, computed in double-float, of an FP32 MUFU seed.
#pragma once

#include <cuda_runtime.h>

namespace jz {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_make(float hi, float lo) { return dfl{hi, lo}; }
__device__ __forceinline__ dfl df_from(float a) { return dfl{a, 0.f}; }
__device__ __forceinline__ dfl df_load(const float2* p, long long i) {
  const float2 v = p[i];
  return dfl{v.x, v.y};
}
__device__ __forceinline__ void df_store(float2* p, long long i, dfl a) { p[i] = make_float2(a.hi, a.lo); }

// s + e = a + b exactly (6 operations)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (3 operations)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ dfl df_norm(float a, float b) {
  dfl r;
  fast_two_sum(a, b, r.hi, r.lo);
  return r;
}

// x + y (11 operations; error <= ~2^-47 (|x| + |y|))
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  return df_norm(s, e);
}
__device__ __forceinline__ dfl df_neg(dfl x) { return dfl{-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
// x + f for an FP32 f (9 operations)
__device__ __forceinline__ dfl df_add_f(dfl x, float f) {
  float s, e;
  two_sum(x.hi, f, s, e);
  return df_norm(s, __fadd_rn(e, x.lo));
}

// x * y (7 operations)
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_norm(p, e);
}
// x * f for an FP32 f (5 operations)
__device__ __forceinline__ dfl df_mul_f(dfl x, float f) {
  const float p = __fmul_rn(x.hi, f);
  float e = __fmaf_rn(x.hi, f, -p);
  e = __fmaf_rn(x.lo, f, e);
  return df_norm(p, e);
}
// x * y + z (15 operations)
__device__ __forceinline__ dfl df_fma(dfl x, dfl y, dfl z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float s, f;
  two_sum(p, z.hi, s, f);
  f = __fadd_rn(f, __fadd_rn(e, z.lo));
  return df_norm(s, f);
}
// Unnormalized ("lazy") forms of the sum, product and fused multiply-add: the same operations
// without the final fast_two_sum.  That step is exact, so the value hi + lo is the one the
// normalized form would give; only |lo| may exceed ulp(hi)/2 (by a few ulp).  A later operation
// that takes such an input still carries lo through its error terms, at a cost of the same order
// as its own rounding (~2^-46 relative).  A chain of them is normalized (df_n) before its value is
// stored, compared, or seeds a reciprocal or root.
__device__ __forceinline__ dfl df_add_l(dfl x, dfl y) {        // 8 operations
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  return dfl{s, __fadd_rn(e, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ dfl df_sub_l(dfl x, dfl y) { return df_add_l(x, dfl{-y.hi, -y.lo}); }
__device__ __forceinline__ dfl df_mul_l(dfl x, dfl y) {        // 4 operations
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return dfl{p, e};
}
__device__ __forceinline__ dfl df_fma_l(dfl x, dfl y, dfl z) {  // 12 operations
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  float s, f;
  two_sum(p, z.hi, s, f);
  return dfl{s, __fadd_rn(f, __fadd_rn(e, z.lo))};
}
__device__ __forceinline__ dfl df_n(dfl x) { return df_norm(x.hi, x.lo); }

// x * 2^k exactly (power-of-two scaling)
__device__ __forceinline__ dfl df_scale(dfl x, float pow2) { return dfl{x.hi * pow2, x.lo * pow2}; }

__device__ __forceinline__ float mufu_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float mufu_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 1/x for 1e-30 < |x| < 1e30 (the arguments here are densities, temperatures and pressure
// sums of order one): seed r ~ 1/x.hi, e = 1 - x r (x r in double-float, then one FP32
// subtraction, exact in its leading part), 1/x = r / (1 - e) ~ r (1 + e + e^2).
__device__ __forceinline__ dfl df_rcp(dfl x) {
  const float r = mufu_rcp(x.hi);
  const dfl p = df_mul_f(x, r);
  const float e = __fsub_rn(__fsub_rn(1.f, p.hi), p.lo);
  return df_norm(r, __fmul_rn(r, __fmaf_rn(e, e, e)));
}
// FP32's exponent range bounds the pair's: below ~1e-30 the low word underflows and the MUFU
// seeds (which flush subnormal arguments to 0) would return Inf.  Such arguments arise only as
// products of round-off noise (strain rates of a quiescent region, ~1e-20 squared); the roots
// below take them through the IEEE FP32 routines, which handle subnormals, with an error that is
// negligible against the terms they enter.
constexpr float kDfTiny = 1e-30f;

// sqrt(x) for x >= 0: seed y ~ x.hi^(-1/2), s = x.hi y, and s + (x - s^2) y / 2 with x - s^2
// formed exactly in its leading part (two_prod of s).  Returns 0 for x = 0.
__device__ __forceinline__ dfl df_sqrt(dfl x) {
  if (!(x.hi > 0.f)) return dfl{0.f, 0.f};
  if (x.hi < kDfTiny) return dfl{sqrtf(x.hi), 0.f};
  const float y = mufu_rsqrt(x.hi);
  const float s = __fmul_rn(x.hi, y);
  const float pp = __fmul_rn(s, s);
  const float pe = __fmaf_rn(s, s, -pp);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, pp), pe), x.lo);
  return df_norm(s, __fmul_rn(__fmul_rn(0.5f, y), r));
}
// x^(1/3) and x^(2/3) for x >= 0: seed z ~ x^(-1/3) from lg2/ex2 and one FP32 Newton step; with
// e = 1 - x z^3 (in
// double-float), x^(-1/3) = z (1 - e)^(-1/3) ~ z (1 + u), u = e (1/3 + 2e/9), the product z u
// kept exactly (two_prod); then x^(2/3) = x x^(-1/3) and x^(1/3) = x^(2/3) x^(-1/3).
__device__ __forceinline__ void df_cbrt_pair(dfl x, dfl& c1, dfl& c2) {
  if (!(x.hi > 0.f)) {
    c1 = dfl{0.f, 0.f};
    c2 = dfl{0.f, 0.f};
    return;
  }
  if (x.hi < kDfTiny) {
    const float t = cbrtf(x.hi);
    c1 = dfl{t, 0.f};
    c2 = dfl{t * t, 0.f};
    return;
  }
  // MUFU seed (~2^-19 for large exponents), one FP32 Newton step to ~2^-23, so that the
  // FP32-rounded correction u below stays ~2^-47 of the result
  const float z0 = mufu_ex2(mufu_lg2(x.hi) * (-1.f / 3.f));
  const float z = __fmaf_rn(z0 * (1.f / 3.f), __fmaf_rn(-x.hi * z0, z0 * z0, 1.f), z0);
  const dfl z2 = df_norm(__fmul_rn(z, z), __fmaf_rn(z, z, -__fmul_rn(z, z)));   // z^2 exactly
  const dfl xz3 = df_mul_f(df_mul(x, z2), z);
  const float e = __fsub_rn(__fsub_rn(1.f, xz3.hi), xz3.lo);
  const float u = e * __fmaf_rn(2.f / 9.f, e, 1.f / 3.f);
  const float zu = __fmul_rn(z, u), zue = __fmaf_rn(z, u, -zu);
  dfl iz = df_norm(z, zu);
  iz = df_norm(iz.hi, __fadd_rn(iz.lo, zue));         // x^(-1/3)
  c2 = df_mul(x, iz);                                 // x^(2/3) = x x^(-1/3)
  c1 = df_mul(c2, iz);                                // x^(1/3) = x^(2/3) x^(-1/3)
}

__device__ __forceinline__ bool df_gt0(dfl a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }
__device__ __forceinline__ bool df_ge(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
__device__ __forceinline__ dfl df_abs(dfl a) { return (a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f)) ? df_neg(a) : a; }
__device__ __forceinline__ dfl df_max(dfl a, dfl b) { return df_ge(a, b) ? a : b; }

// FP64 <-> double-float by integer operations on the IEEE fields, so that conversions stay off
// the FP64 pipe except for one subtraction.  hi is x truncated to 24 significant bits (exact in
// FP64), lo the rest, truncated to FP32 (24 of the remaining 29 bits).  Valid for
// 2^-100 <= |x| < 2^120 and for 0; smaller magnitudes flush to 0.
__device__ __forceinline__ float df_trunc_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned f = __funnelshift_l(lo, hi - (896u << 20), 3);
  const unsigned r = (f & 0x7FFFFFFFu) | (hi & 0x80000000u);
  return __uint_as_float((hi << 1) >= (897u << 21) ? r : (hi & 0x80000000u));
}
__device__ __forceinline__ double df_exact_f64(float f) {      // exact; subnormals flush to 0
  const unsigned b = __float_as_uint(f);
  const unsigned s = b & 0x80000000u, e8 = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e8 == 0) return __hiloint2double((int)s, 0);
  return __hiloint2double((int)(s | ((e8 + 896u) << 20) | (m >> 3)), (int)(m << 29));
}
__device__ __forceinline__ dfl df_of(double x) {
  const float h = df_trunc_f32(x);
  return dfl{h, df_trunc_f32(x - df_exact_f64(h))};
}
__device__ __forceinline__ double df_to_f64(dfl a) { return df_exact_f64(a.hi) + df_exact_f64(a.lo); }

}  // namespace jz
