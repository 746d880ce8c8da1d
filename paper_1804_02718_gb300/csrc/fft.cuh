// Shared-memory FFT of one power-of-two line per thread group, used by every
// stage of the circulant-embedding apply and by the symbol generation.
//
// Layout: a CTA holds TL lines in shared memory, each in sline(L) slots with
// element i at slot spad(i); each line of length L = 2^logL
// (16 <= L) is processed by G = L/16 threads ("lanes"), each holding 16 complex
// values in registers per stage.  Stages are Stockham (self-sorting): stage s
// reads x[j + r L/R], multiplies by the twiddles W_{Ns R}^{r k} (k = j mod Ns),
// does a radix-R DFT in registers and writes to (j - k) R + k + r Ns; the
// result is in natural order with no bit reversal.  All reads of a stage
// happen before a barrier and all writes after it, so one buffer suffices.
// Radices: one 2/4/8 stage for the leftover log2 factor, then radix-16 stages.
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / Ptab), m < Ptab, of the
// longest transform on that axis; a length-L transform indexes it with stride
// Ptab / L.  SIGN = -1 is the forward transform, +1 the (unnormalised) inverse.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace frlap {

// Shared-memory index of logical element i of a line: one padding slot after
// every 16 elements, so that the stride-R stores of the early Stockham stages
// and the contiguous loads both spread over the banks.
__host__ __device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
// Slots per line for logical indices 0..L (L itself is used by the real-data transforms).
__host__ __device__ __forceinline__ int sline(int L) { return L + (L >> 4) + 1; }

// cos x (sine = false) or sin x (sine = true) for |x| <= pi by the Taylor series, at compile
// time: 40 terms leave a remainder far below double rounding.
constexpr double taylor_cs(double x, bool sine) {
  double term = sine ? x : 1.0, sum = term;
  for (int k = 1; k < 40; ++k) {
    const double a = sine ? 2.0 * k : 2.0 * k - 1.0, b = sine ? 2.0 * k + 1.0 : 2.0 * k;
    term *= -x * x / (a * b);
    sum += term;
  }
  return sum;
}
// W_32^j = exp(-2 pi i j / 32), j = 0..16, rounded to FP32 (the twiddle tables' sign convention).
// With G = P/32 lanes per line of a P-point table, W_P^{k + j G} = W_P^k W_32^j: the real-data
// splits of the FP32 first and last stages form their per-bin twiddles from one table entry per
// thread and these constants, which the unrolled loops read as constant-bank operands.
struct W32Table {
  float re[17], im[17];
};
constexpr W32Table make_w32_table() {
  W32Table t{};
  for (int j = 0; j <= 16; ++j) {
    const double x = 3.14159265358979323846 * j / 16.0;
    t.re[j] = (float)taylor_cs(x, false);
    t.im[j] = (float)-taylor_cs(x, true);
  }
  return t;
}
static __constant__ W32Table c_w32 = make_w32_table();


template <int SIGN, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a - b;
  a = a + b;
  b = t;
}

// The first-level sums feed only the second level, so they skip the double-float
// renormalisation (add_lazy); the outputs are normalised.
template <int SIGN, typename C>
__device__ __forceinline__ void dft4(C& a, C& b, C& c, C& d) {
  C s0 = add_lazy(a, c), d0 = sub_lazy(a, c), s1 = add_lazy(b, d), d1 = mul_i<SIGN>(sub_lazy(b, d));
  a = s0 + s1;
  c = s0 - s1;
  b = d0 + d1;
  d = d0 - d1;
}

// exp(SIGN * 2 pi i m / 16) for the small set of m used inside the radix-16 kernel
template <int SIGN, typename T>
__device__ __forceinline__ cplx<T> w16(int m) {
  constexpr T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), r2 = T(0.70710678118654752440);
  constexpr T one = T(1.0), zero = T(0.0);
  T re = zero, im = zero;
  switch (m) {
    case 0: re = one; im = zero; break;
    case 1: re = c1; im = s1; break;
    case 2: re = r2; im = r2; break;
    case 3: re = s1; im = c1; break;
    case 4: re = zero; im = one; break;
    case 6: re = -r2; im = r2; break;
    case 9: re = -c1; im = -s1; break;
    default: break;
  }
  return mk<cplx<T>>(re, SIGN < 0 ? -im : im);
}

// radix-2 combine of dft8 after the even (v[0,2,4,6]) and odd (v[1,3,5,7]) length-4 DFTs
template <int SIGN, typename C>
__device__ __forceinline__ void dft8_combine(C* v) {
  using T = real_t<C>;
  constexpr T r2 = T(0.70710678118654752440);
  C o1 = v[3], o2 = v[5], o3 = v[7];
  // W8^1 = (1 + SIGN i)/sqrt2, W8^2 = SIGN i, W8^3 = (-1 + SIGN i)/sqrt2:
  // W8^1 o = r2 (o + SIGN i o), W8^3 o = r2 (SIGN i o - o)
  const C t1 = r2 * (o1 + mul_i<SIGN>(o1));
  const C t3 = r2 * (mul_i<SIGN>(o3) - o3);
  C t2 = mul_i<SIGN>(o2);
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + t1; v[5] = e1 - t1;
  v[2] = e2 + t2; v[6] = e2 - t2;
  v[3] = e3 + t3; v[7] = e3 - t3;
}

template <int SIGN, typename C>
__device__ __forceinline__ void dft8(C* v) {
  // even / odd halves
  dft4<SIGN>(v[0], v[2], v[4], v[6]);
  dft4<SIGN>(v[1], v[3], v[5], v[7]);
  dft8_combine<SIGN>(v);
}

// twiddles by W16^{j2 k1} and the length-4 DFTs over j2 (second half of dft16)
template <int SIGN, typename C>
__device__ __forceinline__ void dft16_tail(C* v) {
  using T = real_t<C>;
  // v[4 k1 + j2] = A_{j2}[k1]; twiddle by W16^{j2 k1}
#pragma unroll
  for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
    for (int j2 = 1; j2 < 4; ++j2) {
      const int m = j2 * k1;
      if (m == 4) v[4 * k1 + j2] = mul_i<SIGN>(v[4 * k1 + j2]);  // W16^4 = SIGN i
      else v[4 * k1 + j2] = cmul_lazy(v[4 * k1 + j2], w16<SIGN, T>(m));  // feeds the second-level sums
    }
  // length-4 DFTs over j2 for each k1: X[k1 + 4 k2]
  C out[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C a = v[4 * k1], b = v[4 * k1 + 1], c = v[4 * k1 + 2], d = v[4 * k1 + 3];
    dft4<SIGN>(a, b, c, d);
    out[k1] = a; out[k1 + 4] = b; out[k1 + 8] = c; out[k1 + 12] = d;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = out[i];
}

template <int SIGN, typename C>
__device__ __forceinline__ void dft16(C* v) {
  // x[4 j1 + j2]: length-4 DFTs over j1 for each j2
#pragma unroll
  for (int j2 = 0; j2 < 4; ++j2) dft4<SIGN>(v[j2], v[4 + j2], v[8 + j2], v[12 + j2]);
  dft16_tail<SIGN>(v);
}

// dft16 of an input whose upper half x[8..15] is zero (the zero-padded first stage)
template <int SIGN, typename C>
__device__ __forceinline__ void dft16_zin(C* v) {
#pragma unroll
  for (int j2 = 0; j2 < 4; ++j2) {
    const C a = v[j2], b = v[4 + j2];
    const C bi = mul_i<SIGN>(b);
    v[j2] = a + b;
    v[4 + j2] = a + bi;
    v[8 + j2] = a - b;
    v[12 + j2] = a - bi;
  }
  dft16_tail<SIGN>(v);
}

// dft8 of an input whose upper half x[4..7] is zero
template <int SIGN, typename C>
__device__ __forceinline__ void dft8_zin(C* v) {
  // even and odd quarter-length DFTs with two nonzero inputs each, then the radix-2 combine of dft8
  const C e0 = v[0], e1 = v[2], o0 = v[1], o1 = v[3];
  const C e1i = mul_i<SIGN>(e1), o1i = mul_i<SIGN>(o1);
  v[0] = e0 + e1; v[2] = e0 + e1i; v[4] = e0 - e1; v[6] = e0 - e1i;
  v[1] = o0 + o1; v[3] = o0 + o1i; v[5] = o0 - o1; v[7] = o0 - o1i;
  dft8_combine<SIGN>(v);
}

template <int R, int SIGN, bool ZIN, typename C>
__device__ __forceinline__ void dftR(C* v) {
  if constexpr (R == 2) dft2<SIGN>(v[0], v[1]);
  else if constexpr (R == 4) dft4<SIGN>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) {
    if constexpr (ZIN) dft8_zin<SIGN>(v); else dft8<SIGN>(v);
  } else {
    if constexpr (ZIN) dft16_zin<SIGN>(v); else dft16<SIGN>(v);
  }
}

// Twiddles W^r, r = 1..15, W = W_{16 Ns}^k, of one radix-16 butterfly, loaded after the
// stage barrier from the table's stage entries (layout: twiddle_entries), so that the 32
// lanes of a warp read consecutive entries.  (Issuing these loads before the barrier was
// measured slower: the extra live registers cost more than the hidden latency.)
template <typename T>
__device__ __forceinline__ void twiddles16(cplx<T>* w, const cplx<T>* __restrict__ tw, int k, int logNs,
                                           int logPtab) {
  const int Ns = 1 << logNs;
  const cplx<T>* st = tw + (1 << logPtab) + 15 * (Ns - 1) - Ns + k;
  if constexpr (std::is_same<T, float>::value) {
    // FP32: six loads, W^{rk} for r = 1, 2, 3, 4, 8, 12, and W^{(r0 + 4 r1) k} = W^{r0 k} W^{4 r1 k}
    // for the nine others (one rounded product of two rounded entries each); the global loads
    // are the first and last FP32 stages' largest L1 cost
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      w[r] = FRLAP_GLD(st + r * Ns);
      w[4 * r] = FRLAP_GLD(st + 4 * r * Ns);
    }
#pragma unroll
    for (int r1 = 1; r1 < 4; ++r1)
#pragma unroll
      for (int r0 = 1; r0 < 4; ++r0) w[r0 + 4 * r1] = cmul(w[r0], w[4 * r1]);
  } else {
#pragma unroll
    for (int r = 1; r < 16; ++r) w[r] = FRLAP_GLD(st + r * Ns);
  }
}

// Barrier between the read and write halves of a stage.  The G = L/16 lanes of a line
// are consecutive threads starting at a multiple of G, so a line of at most 512 points
// (G <= 32) lies inside one warp, and a warp barrier suffices: the other warps of the CTA
// proceed independently.  CTAs are whole warps (the launchers round their size to a
// multiple of 32 threads) and every thread calls the transform, so the full-warp barrier
// is well defined.  A longer line spans G/32 whole warps.  In the FP64 and double-float
// engines such a line synchronises on its own named barrier (1 + its index in the CTA)
// over its G threads when the CTA holds several lines (CTAs hold at most 512 threads, so
// at most 8 such lines and barriers 1..8); this measured 4% faster for the 2048-point
// double-float rows.  FP32 keeps the CTA barrier, which measured faster there.
template <typename T>
__device__ __forceinline__ void line_sync(int logL) {
  if (logL <= 9) {
    __syncwarp();
  } else if (std::is_same<T, float>::value || (int)blockDim.x == (1 << (logL - 4))) {
    __syncthreads();
  } else {
    const int G = 1 << (logL - 4);
    const int id = 1 + (int)(threadIdx.x >> (logL - 4));
    asm volatile("bar.sync %0, %1;" : : "r"(id), "r"(G) : "memory");
  }
}

// One Stockham stage of radix R on a line of length L = 2^logL held in `buf`
// (padded layout, see spad).  ZIN: the input's upper half is zero (first stage of a
// zero-padded forward transform; those elements are not read).  HOUT: only the lower
// half of the output is used later (last stage of a cropped inverse transform).
template <typename T, int R, int SIGN, bool ZIN, bool HOUT>
__device__ __forceinline__ void fft_stage(cplx<T>* buf, int logL, int Ns, int logNs, int lane,
                                          const cplx<T>* __restrict__ tw, int logPtab) {
  using C = cplx<T>;
  constexpr int E = 16, B = E / R;
  constexpr int LOGR = (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : 4;
  const int G = 1 << (logL - 4);
  const int LR = 1 << (logL - LOGR);
  // W_{Ns R}^{r k} = tw[r k Ptab / (Ns R)]
  const int sh = logPtab - logNs - LOGR;
  C v[E];
  // padded addresses: element i sits at i + i/16.  A stride that is a multiple of 16
  // elements keeps the same in-group offset, so address = base + r * (stride * 17/16).
  const bool lr16 = (LR & 15) == 0;
  const int lstep = LR + (LR >> 4);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = lane + b * G;
    const int base = spad(j);
#pragma unroll
    for (int r = 0; r < R; ++r)
      v[b * R + r] = (ZIN && 2 * r >= R) ? czero<C>() : buf[lr16 ? base + r * lstep : spad(j + r * LR)];
  }
  line_sync<T>(logL);
  const bool ns16 = (Ns & 15) == 0;
  const int sstep = Ns + (Ns >> 4);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = lane + b * G;
    const int k = j & (Ns - 1);
    if (Ns > 1) {
      if constexpr (R == 16) {
        C w[16];
        twiddles16<T>(w, tw, k, logNs, logPtab);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[b * R + r] = (SIGN < 0) ? cmul(v[b * R + r], w[r]) : cmulc(v[b * R + r], w[r]);
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C wr = FRLAP_GLD(tw + ((r * k) << sh));
          v[b * R + r] = (SIGN < 0) ? cmul(v[b * R + r], wr) : cmulc(v[b * R + r], wr);
        }
      }
    }
    dftR<R, SIGN, ZIN>(&v[b * R]);
    const int o = (j - k) * R + k;
    const int obase = spad(o);
    // Ns = 1: o is a multiple of R and o + r never crosses a 16-element group (R divides 16)
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (!HOUT || 2 * r < R)
        buf[Ns == 1 ? obase + r : (ns16 ? obase + r * sstep : spad(o + r * Ns))] = v[b * R + r];
  }
  line_sync<T>(logL);
}

// Full transform of the line in `buf` (length 2^logL >= 16).  Every thread of the
// CTA must call this with the same logL (the stages contain barriers, over the CTA for
// logL > 9, else over the warp: a caller that then reads other lines synchronises the
// CTA itself).
// ZIN: the upper half of the input line is zero (its slots are neither read nor
// needed); HOUT: only the lower half of the output is read afterwards (the upper
// half of the buffer is left stale).  The last stage is always radix 16.
template <typename T, int SIGN, bool ZIN_ = false, bool HOUT_ = false>
__device__ __forceinline__ void fft_line(cplx<T>* buf, int logL, int lane, const cplx<T>* __restrict__ tw,
                                         int logPtab) {
  // The pruned first/last stages pay off where arithmetic is the bottleneck (FP64); for
  // FP32 and double-float they only add code (three copies of the radix-16 stage instead
  // of one loop body), which measured slower, so they are used for FP64 only.
  constexpr bool ZIN = ZIN_ && std::is_same<T, double>::value;
  constexpr bool HOUT = HOUT_ && std::is_same<T, double>::value;
  const int rem = logL & 3;
  int logNs = 0;
  if (rem == 1) { fft_stage<T, 2, SIGN, ZIN, false>(buf, logL, 1, 0, lane, tw, logPtab); logNs = 1; }
  else if (rem == 2) { fft_stage<T, 4, SIGN, ZIN, false>(buf, logL, 1, 0, lane, tw, logPtab); logNs = 2; }
  else if (rem == 3) { fft_stage<T, 8, SIGN, ZIN, false>(buf, logL, 1, 0, lane, tw, logPtab); logNs = 3; }
  if constexpr (!ZIN && !HOUT) {
    while (logNs < logL) {
      fft_stage<T, 16, SIGN, false, false>(buf, logL, 1 << logNs, logNs, lane, tw, logPtab);
      logNs += 4;
    }
    return;
  } else {
    if (logNs == 0) {
      // the first stage is radix 16
      if (logL == 4) {
        fft_stage<T, 16, SIGN, ZIN, HOUT>(buf, logL, 1, 0, lane, tw, logPtab);
        return;
      }
      fft_stage<T, 16, SIGN, ZIN, false>(buf, logL, 1, 0, lane, tw, logPtab);
      logNs = 4;
    }
    while (logNs + 4 < logL) {
      fft_stage<T, 16, SIGN, false, false>(buf, logL, 1 << logNs, logNs, lane, tw, logPtab);
      logNs += 4;
    }
    fft_stage<T, 16, SIGN, false, HOUT>(buf, logL, 1 << logNs, logNs, lane, tw, logPtab);
  }
}

// ---------------------------------------------------------------------------------------
// Register-resident transform.  The Stockham stages all read the same element set per
// thread: lane j (of G = L/16) reads x[j + m G], m = 0..15.  So a caller can load that set
// straight from global memory into registers, and after the last stage the thread holds
// X[j + m G] in the same registers: it can multiply, start another
// transform, or store to global memory without a shared-memory round trip.  Only the
// exchanges between stages go through `buf` (padded layout, see spad).
//
// fft_regs: on entry v[m] = x[lane + m G], on exit v[m] = X[lane + m G], m = 0..15.
// sync_first: other threads may still be reading `buf` (a barrier precedes the first
// write).  ZIN: x[L/2..L) is zero (first-stage DFTs take the zero-aware form for FP64).

// Stage order.  REM = log2(L) mod 4 is a template parameter, so each kernel carries only
// the stages its length needs.  The leftover radix-2^REM stage runs last for REM = 1, 2
// (a leading radix-2/4 stage writes with stride 2/4 elements, which conflicts in shared
// memory for 16-byte elements) and first for REM = 3 (measured faster for the 2048-point
// row transforms).  A last stage of any radix R leaves its outputs in the register layout:
// butterfly b of this lane is j = lane + b G (b < B = 16/R), takes x[j + r L/R] = v[b + r B]
// and produces X[j + r L/R], which is again v[b + r B].

// First stage (Ns = 1) of radix R: butterfly b is j = lane + b G with inputs v[b + r B];
// its outputs replace them (v[b + r B] = output r, to go to position j R + r).
template <typename T, int R, int SIGN, bool ZIN>
__device__ __forceinline__ void regs_first_stage(cplx<T>* v) {
  using C = cplx<T>;
  constexpr int B = 16 / R;
  constexpr bool Z = ZIN && !std::is_same<T, float>::value;  // FP32: the zero-aware form measured no faster
#pragma unroll
  for (int b = 0; b < B; ++b) {
    C t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) t[r] = v[b + r * B];
    dftR<R, SIGN, Z>(t);
#pragma unroll
    for (int r = 0; r < R; ++r) v[b + r * B] = t[r];
  }
}

template <typename T, int R>
__device__ __forceinline__ void regs_first_write(cplx<T>* buf, const cplx<T>* v, int lane, int G) {
  constexpr int B = 16 / R;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int ob = spad((lane + b * G) * R);  // j R + r never crosses a 16-element group
#pragma unroll
    for (int r = 0; r < R; ++r) buf[ob + r] = v[b + r * B];
  }
}

// Last stage (Ns = L/R) of radix R: k = j, twiddles W_L^{r j} = tw[(r j) << shift].
template <typename T, int R, int SIGN>
__device__ __forceinline__ void regs_last_stage(cplx<T>* v, int lane, int G, const cplx<T>* __restrict__ tw,
                                                int shift) {
  using C = cplx<T>;
  constexpr int B = 16 / R;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = lane + b * G;
    C t[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      t[r] = v[b + r * B];
      if (r > 0) {
        const C wr = FRLAP_GLD(tw + ((r * j) << shift));
        t[r] = (SIGN < 0) ? cmul_lazy(t[r], wr) : cmulc_lazy(t[r], wr);
      }
    }
    dftR<R, SIGN, false>(t);
#pragma unroll
    for (int r = 0; r < R; ++r) v[b + r * B] = t[r];
  }
}

// v[m] = x[lane + m G] from buf
template <typename T>
__device__ __forceinline__ void regs_read(cplx<T>* v, const cplx<T>* buf, int lane, int G) {
  const bool g16 = (G & 15) == 0;
  const int rbase = spad(lane), rstep = G + (G >> 4);
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = buf[g16 ? rbase + m * rstep : spad(lane + m * G)];
}

// radix-16 stage with Ns = 2^logNs on v: twiddles W_{16 Ns}^{r k}, k = lane mod Ns
template <typename T, int SIGN>
__device__ __forceinline__ void regs_stage16(cplx<T>* v, int lane, int logNs, const cplx<T>* __restrict__ tw,
                                             int logPtab) {
  if (logNs > 0) {
    const int k = lane & ((1 << logNs) - 1);
    cplx<T> w[16];
    twiddles16<T>(w, tw, k, logNs, logPtab);
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = (SIGN < 0) ? cmul_lazy(v[r], w[r]) : cmulc_lazy(v[r], w[r]);
  }
  dft16<SIGN>(v);
}

// outputs of a radix-16 stage with Ns = 2^logNs: element r to (lane - k) 16 + k + r Ns
template <typename T>
__device__ __forceinline__ void regs_write16(cplx<T>* buf, const cplx<T>* v, int lane, int logNs) {
  const int Ns = 1 << logNs;
  const int k = lane & (Ns - 1);
  const int o = (lane - k) * 16 + k;
  const bool ns16 = (Ns & 15) == 0;
  const int obase = spad(o), sstep = Ns + (Ns >> 4);
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[ns16 ? obase + r * sstep : spad(o + r * Ns)] = v[r];
}

template <typename T, int SIGN, bool ZIN, int REM>
__device__ __forceinline__ void fft_regs(cplx<T>* v, cplx<T>* buf, int logL, int lane,
                                         const cplx<T>* __restrict__ tw, int logPtab, bool sync_first) {
  const int G = 1 << (logL - 4);
  if constexpr (REM == 3) {
    regs_first_stage<T, 8, SIGN, ZIN>(v);
    if (sync_first) line_sync<T>(logL);
    regs_first_write<T, 8>(buf, v, lane, G);
    int logNs = 3;
    while (true) {
      line_sync<T>(logL);
      regs_read<T>(v, buf, lane, G);
      regs_stage16<T, SIGN>(v, lane, logNs, tw, logPtab);
      if (logNs + 4 == logL) return;
      line_sync<T>(logL);
      regs_write16<T>(buf, v, lane, logNs);
      logNs += 4;
    }
  } else {
    regs_first_stage<T, 16, SIGN, ZIN>(v);
    if (REM == 0 && logL == 4) return;  // one stage: output r of lane 0 is X[r]
    if (sync_first) line_sync<T>(logL);
    regs_write16<T>(buf, v, lane, 0);
    int logNs = 4;
    while (true) {
      line_sync<T>(logL);
      regs_read<T>(v, buf, lane, G);
      if constexpr (REM != 0) {
        if (logNs + REM == logL) {
          regs_last_stage<T, (1 << REM), SIGN>(v, lane, G, tw, logPtab - logL);
          return;
        }
      }
      regs_stage16<T, SIGN>(v, lane, logNs, tw, logPtab);
      if (logNs + 4 == logL) return;
      line_sync<T>(logL);
      regs_write16<T>(buf, v, lane, logNs);
      logNs += 4;
    }
  }
}

}  // namespace frlap
