// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  GB300 runs
// FP32 at 62x its FP64 rate, so FFT stages in this format reach FP64-class
// accuracy (about 1e-14 relative per operation) much faster than in FP64.
// Error-free transformations (Knuth's two-sum, Dekker's fast two-sum, and the
// FMA-based exact product) build the arithmetic:
//   two_sum(a, b):      s = a + b, e = (a - (s - v)) + (b - v) with v = s - a
//   fast_two_sum(a, b): s = a + b, e = b - (s - a)                (|a| >= |b|)
//   two_prod(a, b):     p = a * b, e = fma(a, b, -p)
// Addition is the "sloppy" variant (error bounded by eps (|a| + |b|)), which is
// the bound that FFT error analysis uses anyway.
#pragma once

#include <cuda_runtime.h>

namespace frlap {

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // from a double: for constants only (constexpr, folded at compile time)
  __host__ __device__ constexpr explicit dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr explicit dfl(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// A complex double-float, laid out for Blackwell's paired FP32 instructions: hi holds the
// (real, imaginary) high words and lo the low words, so the two components' identical
// double-float sequences issue as one stream of float2 operations (__fadd2_rn, __fmul2_rn,
// __ffma2_rn).  Each component of a paired operation is rounded exactly as the scalar
// __fadd_rn / __fmul_rn / __fmaf_rn, so the error-free transformations hold per component.
// 16 bytes, as before: [re.hi, im.hi, re.lo, im.lo].
struct cdf {
  float2 hi, lo;
};

// Split a double into hi + lo with integer operations only (GB300's FP64 and conversion
// pipes are narrow): hi keeps the sign, exponent and top 23 fraction bits (truncated),
// lo is the remaining 29 fraction bits rounded to a float, so hi + lo equals d to about
// 2^-47 relative.  Zero, subnormal, huge and non-finite values take the conversion path.
__device__ __forceinline__ dfl df_from(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ffu);  // biased exponent
  if (e < 1023 - 70 || e > 1023 + 120) {  // fast path keeps both parts normal floats
    const float h = __double2float_rn(d);
    return dfl(h, __double2float_rn(d - (double)h));
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long frac = b & 0xfffffffffffffull;
  const unsigned hb = sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(frac >> 29);
  const unsigned low = (unsigned)(frac & 0x1fffffffu);                    // weight 2^(e - 1023 - 52)
  const float scale = __int_as_float((e - 1023 - 52 + 127) << 23);         // 2^(e - 1075), normal here
  const float lo = __uint2float_rn(low) * scale;
  return dfl(__int_as_float((int)hb), sign ? -lo : lo);
}
// hi + lo as a double (widening on the bits measured slower than the conversion instructions here)
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dfl(s, e);
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
// The sum without the closing renormalisation (8 instructions instead of 11): hi + lo is
// still the sloppy sum, but lo may exceed ulp(hi)/2 by a few units.  For a sum that only
// feeds another addition, which renormalises; the inputs may be unnormalised themselves.
__device__ __forceinline__ dfl add_lazy(dfl a, dfl b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  return dfl(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a b + c d with one normalisation: the two leading products are split exactly (FMA), summed
// with two_sum, and the error terms and cross products gathered in one FP32 accumulator
// (19 instructions against 25 for two products and a sum; error about eps^2 (|ab| + |cd|)).
__device__ __forceinline__ dfl df_dot2(dfl a, dfl b, dfl c, dfl d) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float q = __fmul_rn(c.hi, d.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  float f = __fmaf_rn(c.hi, d.hi, -q);
  const float s = __fadd_rn(p, q);
  const float v = __fsub_rn(s, p);
  const float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(q, v));
  e = __fmaf_rn(a.hi, b.lo, e);
  f = __fmaf_rn(c.hi, d.lo, f);
  e = __fmaf_rn(a.lo, b.hi, e);
  f = __fmaf_rn(c.lo, d.hi, f);
  return fast_two_sum(s, __fadd_rn(t, __fadd_rn(e, f)));
}

// df_dot2 without the closing renormalisation (16 instructions), for a product that only
// feeds a sum
__device__ __forceinline__ dfl df_dot2_lazy(dfl a, dfl b, dfl c, dfl d) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float q = __fmul_rn(c.hi, d.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  float f = __fmaf_rn(c.hi, d.hi, -q);
  const float s = __fadd_rn(p, q);
  const float v = __fsub_rn(s, p);
  const float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(q, v));
  e = __fmaf_rn(a.hi, b.lo, e);
  f = __fmaf_rn(c.hi, d.lo, f);
  e = __fmaf_rn(a.lo, b.hi, e);
  f = __fmaf_rn(c.lo, d.hi, f);
  return dfl(s, __fadd_rn(t, __fadd_rn(e, f)));
}

// ---- paired (float2) operations
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a - b as one paired FMA, b * (-1) + a: the product is exact, so it is a - b rounded once
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p_bcast(float v) { return make_float2(v, v); }

__host__ __device__ __forceinline__ cdf make_cdf(dfl re, dfl im) {
  cdf c;
  c.hi = make_float2(re.hi, im.hi);
  c.lo = make_float2(re.lo, im.lo);
  return c;
}
__device__ __forceinline__ dfl cdf_re(cdf a) { return dfl(a.hi.x, a.lo.x); }
__device__ __forceinline__ dfl cdf_im(cdf a) { return dfl(a.hi.y, a.lo.y); }

// two-sum of the high words with the low words folded in: (s, t) with s + t = a + b up to the
// low-word rounding (the "lazy" sum, 8 paired operations)
__device__ __forceinline__ cdf cdf_sum_lazy(cdf a, cdf b) {
  const float2 s = p_add(a.hi, b.hi);
  const float2 v = p_sub(s, a.hi);
  const float2 e = p_add(p_sub(a.hi, p_sub(s, v)), p_sub(b.hi, v));
  cdf r;
  r.hi = s;
  r.lo = p_add(e, p_add(a.lo, b.lo));
  return r;
}
// a - b the same way: two-sum of a.hi and -b.hi, where -b.hi - v = -(b.hi + v) exactly
__device__ __forceinline__ cdf cdf_diff_lazy(cdf a, cdf b) {
  const float2 s = p_sub(a.hi, b.hi);
  const float2 v = p_sub(s, a.hi);
  const float2 e = p_sub(p_sub(a.hi, p_sub(s, v)), p_add(b.hi, v));
  cdf r;
  r.hi = s;
  r.lo = p_add(e, p_sub(a.lo, b.lo));
  return r;
}
// Dekker's fast two-sum on the pair (|hi| >= |lo| per component)
__device__ __forceinline__ cdf cdf_norm(cdf a) {
  const float2 S = p_add(a.hi, a.lo);
  cdf r;
  r.hi = S;
  r.lo = p_sub(a.lo, p_sub(S, a.hi));
  return r;
}

__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return cdf_norm(cdf_sum_lazy(a, b)); }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return cdf_norm(cdf_diff_lazy(a, b)); }
__device__ __forceinline__ cdf add_lazy(cdf a, cdf b) { return cdf_sum_lazy(a, b); }
__device__ __forceinline__ cdf sub_lazy(cdf a, cdf b) { return cdf_diff_lazy(a, b); }

// real double-float times complex: both components' exact products, one normalisation
__device__ __forceinline__ cdf operator*(dfl s, cdf a) {
  const float2 sh = p_bcast(s.hi), sl = p_bcast(s.lo);
  const float2 p = p_mul(sh, a.hi);
  float2 e = p_fma(sh, a.hi, p_neg(p));
  e = p_fma(sh, a.lo, e);
  e = p_fma(sl, a.hi, e);
  cdf r;
  r.hi = p;
  r.lo = e;
  return cdf_norm(r);
}

// The pair (x, y) of a1 b1 + a2 b2, with a1, a2 per-lane real double-floats given as (hi, lo)
// pairs and b1, b2 complex: the leading products split exactly (FMA), summed by two-sum, the
// errors and cross products gathered in one accumulator (as the scalar dot product, 16 paired
// operations before the closing normalisation).
__device__ __forceinline__ cdf cdf_dot2_lazy(float2 a1h, float2 a1l, cdf b1, float2 a2h, float2 a2l, cdf b2) {
  const float2 p = p_mul(a1h, b1.hi);
  const float2 q = p_mul(a2h, b2.hi);
  float2 e = p_fma(a1h, b1.hi, p_neg(p));
  float2 f = p_fma(a2h, b2.hi, p_neg(q));
  const float2 s = p_add(p, q);
  const float2 v = p_sub(s, p);
  const float2 t = p_add(p_sub(p, p_sub(s, v)), p_sub(q, v));
  e = p_fma(a1h, b1.lo, e);
  f = p_fma(a2h, b2.lo, f);
  e = p_fma(a1l, b1.hi, e);
  f = p_fma(a2l, b2.hi, f);
  cdf r;
  r.hi = s;
  r.lo = p_add(t, p_add(e, f));
  return r;
}
// i b = (-b.y, b.x) and i conj(b) = (b.y, b.x)
__device__ __forceinline__ cdf cdf_times_i(cdf b) {
  cdf r;
  r.hi = make_float2(-b.hi.y, b.hi.x);
  r.lo = make_float2(-b.lo.y, b.lo.x);
  return r;
}
__device__ __forceinline__ cdf cdf_swap(cdf b) {
  cdf r;
  r.hi = make_float2(b.hi.y, b.hi.x);
  r.lo = make_float2(b.lo.y, b.lo.x);
  return r;
}
__device__ __forceinline__ cdf cdf_conj(cdf b) {
  cdf r;
  r.hi = make_float2(b.hi.x, -b.hi.y);
  r.lo = make_float2(b.lo.x, -b.lo.y);
  return r;
}
// a b = re(a) (b.x, b.y) + im(a) (-b.y, b.x)
__device__ __forceinline__ cdf cmul_lazy(cdf a, cdf b) {
  return cdf_dot2_lazy(p_bcast(a.hi.x), p_bcast(a.lo.x), b, p_bcast(a.hi.y), p_bcast(a.lo.y), cdf_times_i(b));
}
// a conj(b) = re(a) (b.x, -b.y) + im(a) (b.y, b.x)
__device__ __forceinline__ cdf cmulc_lazy(cdf a, cdf b) {
  return cdf_dot2_lazy(p_bcast(a.hi.x), p_bcast(a.lo.x), cdf_conj(b), p_bcast(a.hi.y), p_bcast(a.lo.y),
                       cdf_swap(b));
}
__device__ __forceinline__ cdf cmul(cdf a, cdf b) { return cdf_norm(cmul_lazy(a, b)); }
__device__ __forceinline__ cdf cmulc(cdf a, cdf b) { return cdf_norm(cmulc_lazy(a, b)); }

}  // namespace frlap
