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

struct cdf {
  dfl x, y;  // real, imaginary
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

__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return cdf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cdf add_lazy(cdf a, cdf b) { return cdf{add_lazy(a.x, b.x), add_lazy(a.y, b.y)}; }
__device__ __forceinline__ cdf sub_lazy(cdf a, cdf b) { return cdf{add_lazy(a.x, -b.x), add_lazy(a.y, -b.y)}; }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return cdf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cdf operator*(dfl s, cdf a) { return cdf{s * a.x, s * a.y}; }
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  return cdf{df_dot2(a.x, b.x, -a.y, b.y), df_dot2(a.x, b.y, a.y, b.x)};
}
// a * conj(b)
__device__ __forceinline__ cdf cmulc(cdf a, cdf b) {
  return cdf{df_dot2(a.x, b.x, a.y, b.y), df_dot2(a.y, b.x, -a.x, b.y)};
}
// products that only feed a sum (the twiddle factors ahead of a DFT kernel)
__device__ __forceinline__ cdf cmul_lazy(cdf a, cdf b) {
  return cdf{df_dot2_lazy(a.x, b.x, -a.y, b.y), df_dot2_lazy(a.x, b.y, a.y, b.x)};
}
__device__ __forceinline__ cdf cmulc_lazy(cdf a, cdf b) {
  return cdf{df_dot2_lazy(a.x, b.x, a.y, b.y), df_dot2_lazy(a.y, b.x, -a.x, b.y)};
}

}  // namespace frlap
