// The FFT apply y = A u of the multilevel Toeplitz matrix of eqs. A-2D / A-3D
// through its circulant embedding (the FFT-based product the paper asserts after
// eqs. A-2D and Aj-3D).
//
// Pipeline (P_r = embedding size, H = P_x/2; S1, S2 = workspace spectra):
//   2D: r2c_T  : rows of u (x lines)        -> S1[kx][y]        (pad + real FFT along x, transposed store)
//       colmul : S1[kx][:] lines over y     -> in place         (pad, FFT_y, x lambda, IFFT_y, crop)
//       c2r_T  : S1[kx][y]                  -> rows of y        (inverse real FFT along x, crop)
//   3D: r2c_T  : rows (z,y) of u            -> S1[kx][z][y]
//       c2cT_f : S1[kx][z][:] lines over y  -> S2[kx][ky][z]    (pad, FFT_y, transposed store)
//       colmul : S2[kx][ky][:] lines over z -> in place         (pad, FFT_z, x lambda, IFFT_z, crop)
//       c2cT_i : S2[kx][:][z]               -> S1[kx][z][y]     (IFFT_y, crop)
//       c2r_T  : S1[kx][(z,y)]              -> rows of y
// Every stage reads and writes whole contiguous lines or TL-wide contiguous
// tiles; every global index below is bounded by the line/tile validity tests.
//
// This header holds the kernel and launcher templates; apply_f32.cu, apply_f64.cu and
// apply_dfl.cu instantiate them per engine (three translation units, built in parallel).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fft.cuh"

namespace frlap {

namespace {

// Batched launches: instance b = blockIdx.y reads and writes at these element offsets
// (input, output, symbol) times b, and stops early when skip[b * skip_stride] is set.
struct Batch {
  size_t in = 0, out = 0, lam = 0;
  int skip = 0;
};

#ifdef FRLAP_BOUNDS_CHECK
__global__ void k_bc_register(BcTable t) { g_bc_table = t; }

// The byte ranges one launching call may touch, registered on its stream before its kernels.
struct BcRanges {
  BcTable t = {};
  void add(const void* p, size_t bytes) {
    if (!p || bytes == 0 || t.n >= kBcMaxRanges) return;
    t.lo[t.n] = reinterpret_cast<unsigned long long>(p);
    t.hi[t.n] = t.lo[t.n] + bytes;
    ++t.n;
  }
  cudaError_t commit(cudaStream_t s) const {
    k_bc_register<<<1, 1, 0, s>>>(t);
    return cudaGetLastError();
  }
};
#endif

// Where a middle-stage column finds its multiplier line.  Column index: 2D kx, 3D kx * P_y + ky.
struct LamMap {
  int d;       // 2 or 3
  int logPy;   // 3D: log2 P_y
  int Py;
  int Hx1;     // P_x/2 + 1
  int Hy1;     // P_y/2 + 1
  int Hz1;     // P_z/2 + 1 (3D)
};

// Global loads are issued in unrolled batches before their shared-memory stores, so that
// each thread keeps many loads in flight (the kernels are latency-bound otherwise).

// One line of P = 16 G elements, zero beyond n (or all zero if !valid): lane loads lane + j G.
template <typename C>
__device__ __forceinline__ void load_line(C* buf, const C* __restrict__ src, int lane, int G, int n, bool valid) {
  constexpr int U = sizeof(C) <= 8 ? 16 : 8;
#pragma unroll 1
  for (int j0 = 0; j0 < 16; j0 += U) {
    C t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = lane + (j0 + u) * G;
      t[u] = (valid && i < n) ? FRLAP_GLD(src + i) : czero<C>();
    }
#pragma unroll
    for (int u = 0; u < U; ++u) buf[spad(lane + (j0 + u) * G)] = t[u];
  }
}

// Asynchronous copy of one 8- or 16-byte element from global to shared memory (cp.async;
// with pred false it writes zeros and reads nothing).  The copies of a thread complete at
// cp_async_wait_all(); a CTA barrier after it makes them visible to the other threads.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool pred) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp_async_elem: 4, 8 or 16 bytes");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = pred ? BYTES : 0;
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(sz) : "memory");
  else if constexpr (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(sz) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(sz) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- bulk asynchronous copies completing on an mbarrier (the TMA unit's untiled copy)
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
  // the initialised barrier is visible to the asynchronous proxy that completes its transactions
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// One arrival that also raises the phase's expected transaction count by `bytes`.
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// dst (shared, 16-byte aligned) <- src (global, 16-byte aligned), `bytes` a multiple of 16; the
// bytes count against bar's expected transactions.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Waits until the phase of `bar` with the given parity has completed.  Each try suspends the
// thread for at most about kWaitHintNs; after kWaitTries tries (about a second) it gives up and
// returns false.
constexpr unsigned kWaitHintNs = 1000;
constexpr int kWaitTries = 1 << 20;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  for (int i = 0; i < kWaitTries; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Waits that gave up (one copy per translation unit; wait_collect reads and resets it).
static __device__ unsigned long long g_wait_timeouts = 0ull;

// smem[l][spad(k)] = src[k * ld + line0 + l] for l < TL, k < total / TL (zero past nlines);
// TL is a power of two dividing blockDim.x.  Thread t serves line t mod TL and rows
// k = t / TL + j (blockDim.x / TL), walking its source column with a pointer increment.  Every
// element is an asynchronous copy, so a thread has all of its loads in flight at once and no
// registers hold them; the caller synchronises the CTA.
template <typename C>
__device__ __forceinline__ void load_transposed(C* smem, const C* __restrict__ src, int total, int TL, int LS,
                                                size_t ld, int line0, int nlines) {
  const int logTL = __ffs(TL) - 1;
  const int lt = threadIdx.x & (TL - 1);
  const int kstep = (int)blockDim.x >> logTL;
  const int kend = total >> logTL;
  const bool ok = line0 + lt < nlines;
  C* row = smem + (size_t)lt * LS;
  int k = (int)threadIdx.x >> logTL;
  const C* gp = src + (size_t)k * ld + line0 + lt;
  const size_t gstep = (size_t)kstep * ld;
#pragma unroll 4
  for (; k < kend; k += kstep, gp += gstep) {
    const bool okk = ok && FRLAP_GOK(gp);
    cp_async_elem<(int)sizeof(C)>(&row[spad(k)], okk ? gp : src, okk);
  }
  cp_async_wait_all();
}

// Threads per CTA the apply kernels are compiled for.  FP32 kernels fit 64 registers a thread,
// so 1024-thread CTAs cost them no registers and let the transposed stages hold twice as many
// lines per CTA; the FP64 and double-float kernels need 128 registers (512 threads).
template <typename T>
constexpr int kMaxCta = std::is_same<T, float>::value ? 1024 : 512;

// Shared-memory stride between the transform lines of one first-stage (k_r2c_T) CTA.  Its transposed
// store has a warp read TL lines x 32/TL consecutive bins; for FP32 (16 complex values per 128-byte
// wavefront) the lines are offset by 32/TL slots modulo 16, so that one warp's reads fill whole
// wavefronts: 2047^2 FP32 r2c 20.1 -> 18.2 us per vector.  Lines of at least 512 points only (the
// 256-point rows of 255^3 measured no better); the same offset on the last stage's transposed load
// measured slower (2047^2: 18.2 -> 19.4 us), so it keeps sline.
template <typename T>
__host__ __device__ __forceinline__ int r2c_line_stride(int L, int TL) {
  int s = sline(L);
  if (std::is_same<T, float>::value && TL > 1 && L >= 512) {
    const int want = (32 / TL) & 15;
    s += ((want - s % 16) + 16) % 16;
  }
  return s;
}

// The real-data split of the first and last stages: computed per output element inside the
// transposed store / the transform's register load (one complex product per element, no
// shared-memory write-back), or in place per pair of bins (one product per pair, one more pass
// over shared memory).  Per stage and engine, the faster measured form: the per-element form in
// the forward stage of FP32 and double-float and in the inverse stage of FP32 (2047^2:
// double-float r2c 99 -> 95 us, FP32 c2r 24 -> 22 us); the per-pair form where the extra
// products cost more than the pass (native FP64; the double-float inverse, 75 against 86 us).
template <typename T>
constexpr bool kFusedSplitR2C = !std::is_same<T, double>::value;
template <typename T>
constexpr bool kFusedSplitC2R = std::is_same<T, float>::value;

// The first stage runs as the persistent k_r2c_pf (its input rows' loads overlap the previous
// tile's arithmetic) in the FP64 and double-float engines for transforms of up to 1024 points,
// as measured: double-float 255^3 r2c 235 -> 221 us per 2-vector launch, while the 2048-point
// rows of 2047^2 keep k_r2c_T (71 against 77 us per vector).  FP32 keeps k_r2c_T everywhere: its
// first stage is bound by shared-memory and store throughput, not load latency (persistent form
// at 255^3: 44.7 -> 51.0 us per launch; at 2047^2: 21.3 -> 21.0 us per vector).  -1: never.
template <typename T>
constexpr int kR2CPersistentMaxLogH = std::is_same<T, float>::value ? -1 : 10;
template <typename T>
inline bool use_r2c_pf(int logH, const void* u) {
  return logH <= kR2CPersistentMaxLogH<T> && (reinterpret_cast<uintptr_t>(u) % sizeof(io_t<T>)) == 0;
}
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA

// Multiprocessors of the current device (cached per device).
inline int device_sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

// The rest of the first stage for one tile of TL rows, once each thread holds its row's packed
// samples in v (lane's q = lane + m G, see k_r2c_T): the half-length transform, the real-data
// split and the transposed store of bins 0..H into out[k * ldo + line].
template <typename T, int REM, bool ZIN = true>
__device__ __forceinline__ void r2c_tile(cplx<T>* v, cplx<T>* smem, cplx<T>* __restrict__ out, int nlines, size_t ldo,
                                         int logH, int TL, const cplx<T>* __restrict__ tw, int logP, int line0, int l,
                                         int lane) {
  using C = cplx<T>;
  const int H = 1 << logH, G = H >> 4;
  const int LS = r2c_line_stride<T>(H, TL);
  C* buf = smem + (size_t)l * LS;
  fft_regs<T, -1, ZIN, REM>(v, buf, logH, lane, tw, logP, false);
  line_sync<T>(logH);
#pragma unroll
  for (int m = 0; m < 16; ++m) buf[spad(lane + m * G)] = v[m];
  // The half-length transform Z of the packed samples gives X[k], k = 0..H, by the real-data
  // split: with a = Z[k mod H], b = conj Z[(H-k) mod H], E = (a + b)/2 and O = -i (a - b)/2,
  // X[k] = E + W^k O (W = exp(-2 pi i / 2H)).
  const int logTL = __ffs(TL) - 1;
  // Transposed store: thread t serves line t mod TL of the tile and bins k = t / TL + j G of it
  // (TL G threads), walking its output column with a pointer increment.
  const int lt = threadIdx.x & (TL - 1);
  const bool lt_ok = line0 + lt < nlines;
  const C* trow = smem + (size_t)lt * LS;
  const size_t gstep = (size_t)G * ldo;
  if constexpr (kFusedSplitR2C<T>) {
    // each output of the transposed store computes its own X[k] from the two bins it needs
    // (one product per output, no write-back pass over shared memory)
    __syncthreads();
    if (lt_ok) {
      int k = (int)threadIdx.x >> logTL;
      C* gp = out + (size_t)k * ldo + line0 + lt;
      if constexpr (std::is_same<T, float>::value) {
        // FP32: the thread's bins are k0 + j G, and W^{k0 + j G} = W^{k0} W_32^j (one table load)
        const C w0 = FRLAP_GLD(tw + k);
#pragma unroll
        for (int j = 0; j <= 16; ++j) {
          const int kj = k + j * G;
          if (kj <= H) {
            const C a = trow[spad(kj & (H - 1))];
            const C b = conjg(trow[spad((H - kj) & (H - 1))]);
            const C wk = j == 0 ? w0 : cmul(w0, make_float2(c_w32.re[j], c_w32.im[j]));
            FRLAP_GST(gp + (size_t)j * gstep, halve(a + b) + cmul(wk, halve(mul_i<-1>(a - b))));
          }
        }
      } else {
#pragma unroll 4
        for (; k <= H; k += G, gp += gstep) {
          const C a = trow[spad(k & (H - 1))];
          const C b = conjg(trow[spad((H - k) & (H - 1))]);
          FRLAP_GST(gp, halve(a + b) + cmul(FRLAP_GLD(tw + k), halve(mul_i<-1>(a - b))));
        }
      }
    }
  } else {
    line_sync<T>(logH);
    // in place, one product per pair: X[k] = E + W^k O and X[H-k] = conj(E - W^k O)
    for (int k = lane; k <= H / 2; k += G) {
      const int km = H - k;
      const C a = buf[spad(k)];
      const C b = conjg(buf[spad(km & (H - 1))]);
      const C e = halve(a + b);
      const C t = cmul(FRLAP_GLD(tw + k), halve(mul_i<-1>(a - b)));
      buf[spad(k)] = e + t;
      if (k != km) buf[spad(km)] = conjg(e - t);
    }
    __syncthreads();
    if (lt_ok) {
      int k = (int)threadIdx.x >> logTL;
      C* gp = out + (size_t)k * ldo + line0 + lt;
#pragma unroll 4
      for (; k <= H; k += G, gp += gstep) FRLAP_GST(gp, trow[spad(k)]);
    }
  }
}

// ODD: the row is extended oddly instead of by zeros, to P = 2H = 2(n + 1) points: z_j = x_{j-1} for
// 1 <= j <= n, z_{P-j} = -z_j, z_0 = z_H = 0.  Its DFT is -2i times the row's sine transform (DST-I),
// so the same pipeline applies a multiplier in the sine basis of the box (the tau preconditioner).
template <typename V>
__device__ __forceinline__ V odd_ext(const V* __restrict__ src, int j, int n, int H, bool valid) {
  if (!valid) return V(0);
  if (j >= 1 && j <= n) return FRLAP_GLD(src + (j - 1));
  if (j > H && 2 * H - j - 1 < n) return -FRLAP_GLD(src + (2 * H - j - 1));
  return V(0);
}

template <typename T, int REM, int LOGL = 0, bool ODD = false>
__global__ void __launch_bounds__(kMaxCta<T>, 1) k_r2c_T(const io_t<T>* __restrict__ in, cplx<T>* __restrict__ out, int nlines, int n, int ldi,
                        size_t ldo, int logH, int TL, const cplx<T>* __restrict__ tw, int logP,
                        const int* __restrict__ skip, Batch bt) {
  static_assert(LOGL == 0 || (LOGL & 3) == REM, "REM = LOGL mod 4");
  if constexpr (LOGL > 0) {  // transform length fixed at compile time
    logH = LOGL;
    logP = LOGL + 1;
  }
  {
    const size_t bi = blockIdx.y;
    in += bi * bt.in;
    out += bi * bt.out;
    if (skip) skip += bi * bt.skip;
  }
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  if (skip && FRLAP_GLD(skip)) return;
  const int H = 1 << logH, G = H >> 4;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int line0 = blockIdx.x * TL;
  const int line = line0 + l;
  const bool valid = line < nlines;
  const io_t<T>* src = in + (size_t)(valid ? line : 0) * ldi;
  // packed samples z[q] = x[2q] + i x[2q+1]; lane holds q = lane + m G.  n <= H, so z is zero
  // for q >= H/2 (m >= 8): the upper half of the transform input.
  C v[16];
  if constexpr (ODD) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = lane + m * G;
      v[m] = mk<C>(from_io<T>(odd_ext(src, 2 * q, n, H, valid)), from_io<T>(odd_ext(src, 2 * q + 1, n, H, valid)));
    }
    r2c_tile<T, REM, false>(v, smem, out, nlines, ldo, logH, TL, tw, logP, line0, l, lane);
    return;
  } else {
    // A row that starts on a pair boundary is read one pair (x[2q], x[2q+1]) per load.
    using IO2 = io_pair<T>;
    const bool pair_aligned = (reinterpret_cast<uintptr_t>(src) % sizeof(IO2)) == 0;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = lane + m * G;
      io_t<T> re = io_t<T>(0), im = io_t<T>(0);
      if (m < 8 && valid) {
        if (pair_aligned && 2 * q + 1 < n) {
          const IO2 t = FRLAP_GLD(reinterpret_cast<const IO2*>(src + 2 * q));
          re = t.x;
          im = t.y;
        } else {
          if (2 * q < n) re = FRLAP_GLD(src + 2 * q);
          if (2 * q + 1 < n) im = FRLAP_GLD(src + 2 * q + 1);
        }
      }
      v[m] = mk<C>(from_io<T>(re), from_io<T>(im));
    }
    r2c_tile<T, REM>(v, smem, out, nlines, ldo, logH, TL, tw, logP, line0, l, lane);
  }
}

// Staging area of k_r2c_pf: the TL n elements of a tile's rows (E bytes each), shifted by the
// tile start's offset from a 16-byte boundary (0..16/E - 1 elements), rounded up to 16 bytes;
// then the mbarrier.
template <int E>
__host__ __device__ __forceinline__ int r2c_stage_elems(int TL, int n) {
  constexpr int A = 16 / E;
  return (TL * n + 2 * A - 2) / A * A;
}
// Byte offset of the staging area: after the TL transform lines, rounded up to 16 bytes (an
// FP32 line of sline(H) complex elements is 8 bytes past a 16-byte boundary when TL is odd).
template <typename T>
__host__ __device__ __forceinline__ size_t r2c_stage_offset(int TL, int H) {
  return ((size_t)TL * sline(H) * sizeof(cplx<T>) + 15) & ~(size_t)15;
}
template <typename T>
size_t r2c_pf_smem_bytes(int TL, int H, int n) {
  constexpr int E = (int)sizeof(io_t<T>);
  return r2c_stage_offset<T>(TL, H) + (size_t)r2c_stage_elems<E>(TL, n) * E + 16;
}

// Persistent form of k_r2c_T for rows whose TL rows per tile are contiguous (row stride n).
// CTA c takes the tiles t = c, c + gridDim.x, ... of all instances (t = instance * tiles +
// tile).  A tile's rows reach a shared-memory staging area by one bulk asynchronous copy,
// completing on an mbarrier, that thread 0 issues as soon as every thread holds the previous
// tile's samples in registers: the copy runs during that tile's transform and transposed
// store, so the loads' latency leaves the critical path.  The bulk copy moves the
// 16-byte-aligned interior of the tile's span; the elements before and after it (a span that
// does not start or end on a 16-byte boundary) are element-sized cp.async copies.
template <typename T, int REM, int LOGL = 0>
__global__ void __launch_bounds__(kMaxCta<T>, 1) k_r2c_pf(const io_t<T>* __restrict__ in, cplx<T>* __restrict__ out, int nlines, int n,
                         size_t ldo, int logH, int TL, const cplx<T>* __restrict__ tw, int logP,
                         const int* __restrict__ skip, Batch bt, int ninst) {
  static_assert(LOGL == 0 || (LOGL & 3) == REM, "REM = LOGL mod 4");
  if constexpr (LOGL > 0) {  // transform length fixed at compile time
    logH = LOGL;
    logP = LOGL + 1;
  }
  using C = cplx<T>;
  using IO = io_t<T>;
  constexpr int E = (int)sizeof(IO);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  const int H = 1 << logH, G = H >> 4;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  IO* stage = reinterpret_cast<IO*>(smem_raw + r2c_stage_offset<T>(TL, H));  // 16-byte aligned
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(stage + r2c_stage_elems<E>(TL, n));
  const int ntiles = (nlines + TL - 1) / TL;
  const long long total = (long long)ntiles * ninst;
  // tile t: its instance, first row, and the address of its first element
  auto tile_src = [&](long long t, int& b, int& line0) {
    b = (int)(t / ntiles);
    line0 = (int)(t - (long long)b * ntiles) * TL;
    return in + (size_t)b * bt.in + (size_t)line0 * n;
  };
  // thread 0: start the copies of tile t into the staging area (element j at stage[j + off])
  auto issue = [&](long long t) {
    int b, line0;
    const IO* src = tile_src(t, b, line0);
    if (skip && FRLAP_GLD(skip + (size_t)b * bt.skip)) {  // a skipped instance: nothing to copy
      mbar_arrive_tx(bar, 0u);
      return;
    }
    const int cnt = min(TL, nlines - line0) * n;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    const int off = (int)((a & 15) / E);
    const uintptr_t a1 = (a + 15) & ~(uintptr_t)15, e0 = (a + (uintptr_t)cnt * E) & ~(uintptr_t)15;
    unsigned bytes = e0 > a1 ? (unsigned)(e0 - a1) : 0u;
    const int h = min((int)((a1 - a) / E), cnt);                         // elements before the bulk part
    const int tl0 = bytes ? (int)((e0 - a) / E) : h;                     // first element after it
#ifdef FRLAP_BOUNDS_CHECK
    if (bytes && !bc_ok(reinterpret_cast<const void*>(a1), bytes)) bytes = 0u;
#endif
    for (int j = 0; j < h; ++j) cp_async_elem<E>(stage + j + off, src + j, FRLAP_GOK(src + j));
    for (int j = tl0; j < cnt; ++j) cp_async_elem<E>(stage + j + off, src + j, FRLAP_GOK(src + j));
    mbar_arrive_tx(bar, bytes);
    if (bytes) bulk_g2s(stage + h + off, reinterpret_cast<const void*>(a1), bytes, bar);
  };
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  long long t = blockIdx.x;
  if (threadIdx.x == 0 && t < total) issue(t);
  unsigned parity = 0;
  for (; t < total; t += gridDim.x) {
    cp_async_wait_all();  // thread 0's element copies of this tile
    const bool ok = mbar_wait(bar, parity);
    parity ^= 1;
    if (!__syncthreads_and(ok)) {  // the staging copy did not complete in time: record and stop
      if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1ull);
      return;
    }
    int b, line0;
    const IO* src = tile_src(t, b, line0);
    const bool skipped = skip && FRLAP_GLD(skip + (size_t)b * bt.skip);
    const int off = (int)((reinterpret_cast<uintptr_t>(src) & 15) / E);
    const bool valid = line0 + l < nlines;
    // packed samples z[q] = x[2q] + i x[2q+1] of row line0 + l, as in k_r2c_T
    const IO* row = stage + (size_t)l * n + off;
    const bool pair_aligned = ((l * n + off) & 1) == 0;
    using IO2 = io_pair<T>;
    C v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = lane + m * G;
      IO re = IO(0), im = IO(0);
      if (m < 8 && valid) {
        if (pair_aligned && 2 * q + 1 < n) {
          const IO2 p2 = *reinterpret_cast<const IO2*>(row + 2 * q);
          re = p2.x;
          im = p2.y;
        } else {
          if (2 * q < n) re = row[2 * q];
          if (2 * q + 1 < n) im = row[2 * q + 1];
        }
      }
      v[m] = mk<C>(from_io<T>(re), from_io<T>(im));
    }
    __syncthreads();  // the staging area is free: start the next tile's copy
    if (threadIdx.x == 0 && t + gridDim.x < total) issue(t + gridDim.x);
    if (!skipped)
      r2c_tile<T, REM>(v, smem, out + (size_t)b * bt.out, nlines, ldo, logH, TL, tw, logP, line0, l, lane);
  }
}

template <typename T, int REM, int LOGL = 0, bool ODD = false>
__global__ void __launch_bounds__(kMaxCta<T>, 1) k_c2r_T(const cplx<T>* __restrict__ in, io_t<T>* __restrict__ out, int nlines, int n, size_t ldi,
                        int ldo, int logH, int TL, const cplx<T>* __restrict__ tw, int logP,
                        const int* __restrict__ skip, Batch bt) {
  static_assert(LOGL == 0 || (LOGL & 3) == REM, "REM = LOGL mod 4");
  if constexpr (LOGL > 0) {  // transform length fixed at compile time
    logH = LOGL;
    logP = LOGL + 1;
  }
  {
    const size_t bi = blockIdx.y;
    in += bi * bt.in;
    out += bi * bt.out;
    if (skip) skip += bi * bt.skip;
  }
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  if (skip && FRLAP_GLD(skip)) return;
  const int H = 1 << logH, G = H >> 4;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int line0 = blockIdx.x * TL;
  const int line = line0 + l;
  const int LS = sline(H);
  const int total = TL * (H + 1);
  load_transposed<C>(smem, in, total, TL, LS, ldi, line0, nlines);
  __syncthreads();
  C* buf = smem + (size_t)l * LS;
  // repack: Z[k] = A + i T with A = X[k] + conj X[H-k], T = W^{-k} (X[k] - conj X[H-k]), so that
  // the unnormalised inverse half-length transform gives P (y[2j] + i y[2j+1])
  C v[16];
  if constexpr (kFusedSplitC2R<T>) {
    // straight into the registers the transform starts from (one product per element); the
    // twiddle of bin lane + m G is W^{lane} W_32^m (one table load per thread)
    const C w0 = FRLAP_GLD(tw + lane);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int k = lane + m * G;
      const C xk = buf[spad(k)];
      const C b = conjg(buf[spad(H - k)]);
      const C wk = m == 0 ? w0 : cmul(w0, mk<C>(c_w32.re[m], c_w32.im[m]));
      v[m] = (xk + b) + mul_i<1>(cmulc(xk - b, wk));
    }
  } else {
    // in place, one product per pair; the partner is Z[H-k] = conj(A - i T)
    for (int k = lane; k <= H / 2; k += G) {
      const int km = H - k;
      const C xk = buf[spad(k)];
      const C b = conjg(buf[spad(km)]);
      const C A = xk + b;
      const C iT = mul_i<1>(cmulc(xk - b, FRLAP_GLD(tw + k)));
      buf[spad(k)] = A + iT;
      if (k != km && km != H) buf[spad(km)] = conjg(A - iT);
    }
    line_sync<T>(logH);
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = buf[spad(lane + m * G)];
  }
  fft_regs<T, 1, false, REM>(v, buf, logH, lane, tw, logP, true);
  // v[m] = y[2q] + i y[2q+1] (times P), q = lane + m G; n <= H keeps only m < 8
  if (ODD) {  // the odd extension's row: x_i = y_{i+1}, i < n = H - 1
    if (line < nlines) {
      io_t<T>* dst = out + (size_t)line * ldo;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int q = lane + m * G;
        if (q >= 1 && 2 * q <= n) FRLAP_GST(dst + (2 * q - 1), to_io<T>(re(v[m])));
        if (2 * q + 1 <= n) FRLAP_GST(dst + 2 * q, to_io<T>(im(v[m])));
      }
    }
  } else if (line < nlines) {
    io_t<T>* dst = out + (size_t)line * ldo;
    using IO2 = io_pair<T>;
    const bool pair_aligned = (reinterpret_cast<uintptr_t>(dst) % sizeof(IO2)) == 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int q = lane + m * G;
      if (pair_aligned && 2 * q + 1 < n) {
        IO2 t;
        t.x = to_io<T>(re(v[m]));
        t.y = to_io<T>(im(v[m]));
        FRLAP_GST(reinterpret_cast<IO2*>(dst + 2 * q), t);
      } else {
        if (2 * q < n) FRLAP_GST(dst + 2 * q, to_io<T>(re(v[m])));
        if (2 * q + 1 < n) FRLAP_GST(dst + 2 * q + 1, to_io<T>(im(v[m])));
      }
    }
  }
}

// The middle stage of 2D plans with a P = 16384-point y embedding (n_y up to 8191), as two
// transforms of the longest line length the kernels hold, L = P/2 = 8192 points, split by the
// parity of the frequency.  The column v is zero past n_y <= L, so
//   X[2m]   = sum_{j<L} v_j W_L^{jm}                 (the even half: the L-point DFT of v),
//   X[2m+1] = sum_{j<L} (v_j W_P^j) W_L^{jm}         (the odd half: of v times W_P^j),
// and the inverse, sum_k lambda_k X_k W_P^{-jk} (1/P is part of lambda), is
//   y_j = IDFT_L(lambda_{2m} X[2m])_j + W_P^{-j} IDFT_L(lambda_{2m+1} X[2m+1])_j
// with unnormalised inverse transforms.  ODD = false computes the even half into tmp (same layout
// as the columns); ODD = true the odd half, adds tmp, and writes the column in place.  The
// transforms read the P-point twiddle table: its stage entries W_{16 Ns}^{rk} do not depend on P,
// and the last (radix-2) stage reads every second plain entry.
template <typename T, bool ODD>
__global__ void __launch_bounds__(kMaxCta<T>, 1) k_colmul_split(cplx<T>* __restrict__ data, cplx<T>* __restrict__ tmp,
                                                                int ncols, int n, size_t ld, int TL,
                                                                const T* __restrict__ lam, int Hy1,
                                                                const cplx<T>* __restrict__ tw,
                                                                const int* __restrict__ skip, Batch bt) {
  constexpr int logL = 13, L = 1 << logL, P = 2 * L, G = L >> 4, REM = logL & 3, logPtab = logL + 1;
  {
    const size_t bi = blockIdx.y;
    data += bi * bt.in;
    tmp += bi * bt.out;
    lam += bi * bt.lam;
    if (skip) skip += bi * bt.skip;
  }
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  if (skip && FRLAP_GLD(skip)) return;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int col = blockIdx.x * TL + l;
  const bool valid = col < ncols;
  C* buf = smem + (size_t)l * sline(L);
  C* line = data + (size_t)(valid ? col : 0) * ld;
  C* tline = tmp + (size_t)(valid ? col : 0) * ld;
  // lane holds elements j = lane + m G, m = 0..15 (all of them: n can exceed L/2)
  C v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int j = lane + m * G;
    v[m] = (valid && j < n) ? ld_stream(&line[j]) : czero<C>();
    if constexpr (ODD) v[m] = cmul(v[m], FRLAP_GLD(tw + j));
  }
  fft_regs<T, -1, false, REM>(v, buf, logL, lane, tw, logPtab, false);
  const T* __restrict__ lrow = lam + (size_t)(valid ? col : 0) * Hy1;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int k = 2 * (lane + m * G) + (ODD ? 1 : 0);  // frequency of this output, folded below
    v[m] = ld_stream(&lrow[min(k, P - k)]) * v[m];
  }
  fft_regs<T, 1, false, REM>(v, buf, logL, lane, tw, logPtab, true);
  if (!valid) return;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int j = lane + m * G;
    if (j < n) {
      if constexpr (ODD) FRLAP_GST(line + j, cmulc(v[m], FRLAP_GLD(tw + j)) + FRLAP_GLD(tline + j));
      else FRLAP_GST(tline + j, v[m]);
    }
  }
}

// ODD (see k_r2c_T): the column's entries are the transform's outputs 1 .. n, at offset -1.
template <typename C>
__device__ __forceinline__ void store_line_odd(const C* v, C* __restrict__ data, int ncols, int n, size_t ld,
                                               int logP, int TL) {
  unsigned tid;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
  const int G = 1 << (logP - 4);
  const int lane = (int)tid & (G - 1);
  const int col = (int)blockIdx.x * TL + ((int)tid >> (logP - 4));
  if (col >= ncols) return;
  C* out = data + (size_t)col * ld;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int j = lane + m * G;
    if (j >= 1 && j <= n) FRLAP_GST(out + (j - 1), v[m]);
  }
}

// The cropped output of k_colmul: column blockIdx.x * TL + tid / G, elements lane + m G < n
// (m < 8; n <= P/2).  The thread's column and lane are re-derived from
// the special registers here, not kept live across both transforms (that spilled).
template <typename C>
__device__ __forceinline__ void store_line(const C* v, C* __restrict__ data, int ncols, int n, size_t ld, int logP,
                                           int TL) {
  unsigned tid;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
  const int G = 1 << (logP - 4);
  const int lane = (int)tid & (G - 1);
  const int col = (int)blockIdx.x * TL + ((int)tid >> (logP - 4));
  if (col >= ncols) return;
  C* out = data + (size_t)col * ld;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = lane + m * G;
    if (i < n) FRLAP_GST(out + i, v[m]);
  }
}

// lines of length n (contiguous, stride ld) -> zero-pad to P, FFT, * lambda, IFFT, crop, in place
// LOGP > 0: the line length 2^LOGP is fixed at compile time (the logP / logPtab arguments are
// ignored), so stage spans, lane counts and shared-memory strides fold into constants.
template <typename T, int REM, int LOGP = 0, bool ODD = false>
__global__ void __launch_bounds__(kMaxCta<T>, 1) k_colmul(cplx<T>* __restrict__ data, int ncols, int n, size_t ld, int logP, int TL,
                         const T* __restrict__ lam, LamMap map, const cplx<T>* __restrict__ tw, int logPtab,
                         const int* __restrict__ skip, Batch bt) {
  static_assert(LOGP == 0 || (LOGP & 3) == REM, "k_colmul: REM = LOGP mod 4");
  if constexpr (LOGP > 0) {
    logP = LOGP;
    logPtab = LOGP;
  }
  {
    const size_t bi = blockIdx.y;
    data += bi * bt.in;
    lam += bi * bt.lam;
    if (skip) skip += bi * bt.skip;
  }
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  if (skip && FRLAP_GLD(skip)) return;
  const int P = 1 << logP, G = P >> 4;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int col = blockIdx.x * TL + l;
  const bool valid = col < ncols;
  C* buf = smem + (size_t)l * sline(P);
  C* line = data + (size_t)(valid ? col : 0) * ld;
  // lane holds elements lane + m G; n <= P/2, so m >= 8 is the zero padding (ODD: the column's odd
  // extension to P = 2(n + 1) points, as in k_r2c_T)
  C v[16];
  if constexpr (ODD) {
    const int H = P >> 1;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int j = lane + m * G;
      C x = czero<C>();
      if (valid) {
        if (j >= 1 && j <= n) x = ld_stream(&line[j - 1]);
        else if (j > H && 2 * H - j - 1 < n) x = czero<C>() - ld_stream(&line[2 * H - j - 1]);
      }
      v[m] = x;
    }
  } else {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int i = lane + m * G;
      v[m] = (m < 8 && valid && i < n) ? ld_stream(&line[i]) : czero<C>();
    }
  }
  // line-major symbol: the folded line of this column is contiguous
  auto symbol_row = [&]() -> const T* {
    const int c = valid ? col : 0;
    if (map.d == 2) return lam + (size_t)c * map.Hy1;
    const int kx = c >> map.logPy, ky = c & (map.Py - 1);
    return lam + ((size_t)kx * map.Hy1 + min(ky, map.Py - ky)) * map.Hz1;
  };
  // Forward transform with the zero-input first stage, multiply, inverse transform.  (Double-float
  // once ran the inverse as conj(FFT(conj(.))) to execute a single copy of the stage code, which the
  // instruction cache favoured; with its arithmetic in paired instructions the code is half the size
  // and the two copies measured faster: 255^3 colmul 1.017 -> 0.992 ms.)
  fft_regs<T, -1, !ODD, REM>(v, buf, logP, lane, tw, logPtab, false);
  const T* __restrict__ lrow = symbol_row();
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int k = lane + m * G;
    v[m] = ld_stream(&lrow[min(k, P - k)]) * v[m];
  }
  fft_regs<T, 1, false, REM>(v, buf, logP, lane, tw, logPtab, true);
  if constexpr (ODD) store_line_odd(v, data, ncols, n, ld, logP, TL);
  else store_line(v, data, ncols, n, ld, logP, TL);
}

// The middle stage of the residual apply of double-float plans (apply_launch_b<double, dfl>): the
// forward transform and the symbol product in FP64, then each value split into a double-float pair
// and the inverse transform in double-float.  The column is read as FP64 and written back in place
// as double-float (16 bytes per complex value either way).  Rounding in the forward transform
// reaches the product multiplied by up to lambda_max, so that transform keeps FP64; the inverse
// transform's rounding is relative to the product itself, where double-float's 2^-48 suffices.
template <int REM>
__global__ void __launch_bounds__(kMaxCta<double>, 1)
    k_colmul_hyb(double2* __restrict__ data, int ncols, int n, size_t ld, int logP, int TL,
                 const double* __restrict__ lam, LamMap map, const double2* __restrict__ tw64,
                 const cdf* __restrict__ twdf, const int* __restrict__ skip, Batch bt) {
  {
    const size_t bi = blockIdx.y;
    data += bi * bt.in;
    lam += bi * bt.lam;
    if (skip) skip += bi * bt.skip;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* smem = reinterpret_cast<double2*>(smem_raw);
  if (skip && FRLAP_GLD(skip)) return;
  const int P = 1 << logP, G = P >> 4;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int col = blockIdx.x * TL + l;
  const bool valid = col < ncols;
  double2* buf = smem + (size_t)l * sline(P);
  const double2* line = data + (size_t)(valid ? col : 0) * ld;
  double2 v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int i = lane + m * G;
    v[m] = (m < 8 && valid && i < n) ? ld_stream(&line[i]) : czero<double2>();
  }
  fft_regs<double, -1, true, REM>(v, buf, logP, lane, tw64, logP, false);
  const int c = valid ? col : 0;
  const double* __restrict__ lrow =
      map.d == 2 ? lam + (size_t)c * map.Hy1
                 : lam + ((size_t)(c >> map.logPy) * map.Hy1 + min(c & (map.Py - 1), map.Py - (c & (map.Py - 1)))) *
                             map.Hz1;
  cdf w[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int k = lane + m * G;
    const double2 t = ld_stream(&lrow[min(k, P - k)]) * v[m];
    w[m] = make_cdf(df_from(t.x), df_from(t.y));
  }
  fft_regs<dfl, 1, false, REM>(w, reinterpret_cast<cdf*>(buf), logP, lane, twdf, logP, true);
  store_line(w, reinterpret_cast<cdf*>(data), ncols, n, ld, logP, TL);
}

// groups of contiguous lines of length n -> pad, FFT, transposed store out[g][k][line]
template <typename T, int REM, int LOGL = 0, bool ODD = false>
__global__ void __launch_bounds__(kMaxCta<T>, 1) k_c2cT_fwd(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int nlines, int tiles, int n,
                           size_t gin, int ldi, size_t gout, int ldo, int logP, int TL,
                           const cplx<T>* __restrict__ tw, int logPtab, const int* __restrict__ skip, Batch bt) {
  static_assert(LOGL == 0 || (LOGL & 3) == REM, "REM = LOGL mod 4");
  if constexpr (LOGL > 0) {  // line length fixed at compile time
    logP = LOGL;
    logPtab = LOGL;
  }
  {
    const size_t bi = blockIdx.y;
    in += bi * bt.in;
    out += bi * bt.out;
    if (skip) skip += bi * bt.skip;
  }
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  if (skip && FRLAP_GLD(skip)) return;
  const int P = 1 << logP, G = P >> 4;
  const int g = blockIdx.x / tiles, tile = blockIdx.x % tiles;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int line0 = tile * TL;
  const int line = line0 + l;
  const bool valid = line < nlines;
  const int LS = sline(P);
  C* buf = smem + (size_t)l * LS;
  const C* src = in + g * gin + (size_t)(valid ? line : 0) * ldi;
  C v[16];
  if constexpr (ODD) {  // the line's odd extension to P = 2(n + 1) points (see k_r2c_T)
    const int H = P >> 1;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int j = lane + m * G;
      C x = czero<C>();
      if (valid) {
        if (j >= 1 && j <= n) x = FRLAP_GLD(src + (j - 1));
        else if (j > H && 2 * H - j - 1 < n) x = czero<C>() - FRLAP_GLD(src + (2 * H - j - 1));
      }
      v[m] = x;
    }
  } else {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int i = lane + m * G;
      v[m] = (m < 8 && valid && i < n) ? FRLAP_GLD(src + i) : czero<C>();
    }
  }
  fft_regs<T, -1, !ODD, REM>(v, buf, logP, lane, tw, logPtab, false);
  line_sync<T>(logP);
#pragma unroll
  for (int m = 0; m < 16; ++m) buf[spad(lane + m * G)] = v[m];
  __syncthreads();
  // transposed store: thread t serves line t mod TL and rows k = t / TL + j G
  const int logTL = __ffs(TL) - 1;
  const int lt = threadIdx.x & (TL - 1);
  if (line0 + lt < nlines) {
    const C* trow = smem + (size_t)lt * LS;
    int k = (int)threadIdx.x >> logTL;
    C* gp = out + g * gout + (size_t)k * ldo + line0 + lt;
    const size_t gstep = (size_t)G * ldo;
#pragma unroll 4
    for (; k < P; k += G, gp += gstep) FRLAP_GST(gp, trow[spad(k)]);
  }
}

// transposed in[g][k][line] (k < P) -> IFFT along k, crop to n, store out[g][line][i]
template <typename T, int REM, int LOGL = 0, bool ODD = false>
__global__ void __launch_bounds__(kMaxCta<T>, 1) k_c2cT_inv(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int nlines, int tiles, int n,
                           size_t gin, int ldi, size_t gout, int ldo, int logP, int TL,
                           const cplx<T>* __restrict__ tw, int logPtab, const int* __restrict__ skip, Batch bt) {
  static_assert(LOGL == 0 || (LOGL & 3) == REM, "REM = LOGL mod 4");
  if constexpr (LOGL > 0) {  // line length fixed at compile time
    logP = LOGL;
    logPtab = LOGL;
  }
  {
    const size_t bi = blockIdx.y;
    in += bi * bt.in;
    out += bi * bt.out;
    if (skip) skip += bi * bt.skip;
  }
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  if (skip && FRLAP_GLD(skip)) return;
  const int P = 1 << logP, G = P >> 4;
  const int g = blockIdx.x / tiles, tile = blockIdx.x % tiles;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int line0 = tile * TL;
  const int line = line0 + l;
  const C* src = in + g * gin;
  const int LS = sline(P);
  const int total = TL * P;
  load_transposed<C>(smem, src, total, TL, LS, ldi, line0, nlines);
  __syncthreads();
  C* buf = smem + (size_t)l * LS;
  C v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = buf[spad(lane + m * G)];
  fft_regs<T, 1, false, REM>(v, buf, logP, lane, tw, logPtab, true);
  if (line < nlines) {
    C* dst = out + g * gout + (size_t)line * ldo;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int i = lane + m * G;
      if (ODD) {  // outputs 1 .. n of the odd extension, at offset -1
        if (i >= 1 && i <= n) FRLAP_GST(dst + (i - 1), v[m]);
      } else if (i < n) {
        FRLAP_GST(dst + i, v[m]);
      }
    }
  }
}


// lines of length n (stride ld) -> zero-pad to P, forward FFT, write all P outputs (stride ldo)
template <typename T>
__global__ void __launch_bounds__(kMaxCta<T>, 1)
    k_col_fwd(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int ncols, int n, size_t ld, size_t ldo,
              int logP, int TL, const cplx<T>* __restrict__ tw, int logPtab) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  const int P = 1 << logP, G = P >> 4;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int col = blockIdx.x * TL + l;
  const bool valid = col < ncols;
  C* buf = smem + (size_t)l * sline(P);
  const C* src = in + (size_t)(valid ? col : 0) * ld;
  load_line<C>(buf, src, lane, G, n, valid);
  __syncthreads();
  fft_line<T, -1, true, false>(buf, logP, lane, tw, logPtab);
  if (valid) {
    C* dst = out + (size_t)col * ldo;
    for (int i = lane; i < P; i += G) FRLAP_GST(dst + i, buf[spad(i)]);
  }
}

// lines of P spectrum values (stride ld) -> * multiplier, inverse FFT, crop to n, write (stride ldo)
template <typename T>
__global__ void __launch_bounds__(kMaxCta<T>, 1)
    k_col_mulinv(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int ncols, int n, size_t ld, size_t ldo,
                 int logP, int TL, const T* __restrict__ lam, LamMap map, const cplx<T>* __restrict__ tw,
                 int logPtab) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  const int P = 1 << logP, G = P >> 4;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const int col = blockIdx.x * TL + l;
  const bool valid = col < ncols;
  C* buf = smem + (size_t)l * sline(P);
  const C* src = in + (size_t)(valid ? col : 0) * ld;
  // the multiplier is in natural octant order here (it comes from the learning kernels)
  size_t lam_base;
  int lam_stride;
  if (map.d == 2) {
    lam_base = valid ? col : 0;
    lam_stride = map.Hx1;
  } else {
    const int c = valid ? col : 0;
    const int kx = c >> map.logPy, ky = c & (map.Py - 1);
    lam_base = (size_t)min(ky, map.Py - ky) * map.Hx1 + kx;
    lam_stride = map.Hy1 * map.Hx1;
  }
  for (int k = lane; k < P; k += G) {
    const int kf = min(k, P - k);
    buf[spad(k)] = valid ? FRLAP_GLD(lam + lam_base + (size_t)kf * lam_stride) * FRLAP_GLD(src + k) : czero<C>();
  }
  __syncthreads();
  fft_line<T, 1, false, true>(buf, logP, lane, tw, logPtab);
  if (valid) {
    C* dst = out + (size_t)col * ldo;
    for (int i = lane; i < n; i += G) FRLAP_GST(dst + i, buf[spad(i)]);
  }
}

// Lines per CTA for a line of `len` complex slots: as many as fit in
// `budget` bytes of shared memory and 256 threads (at least one), rounded down to a
// power of two, in whole warps.
// (the apply kernels are compiled for 512 (FP32: 1024) threads per CTA; CTAs of at most 256
// threads measured fastest: more independent CTAs per SM overlap their phases)
int pick_tl(int len, int elem_bytes, int G, int budget, int max_lines, long long lines = 1LL << 40) {
  int tl = budget / (len * elem_bytes);
  tl = tl < 1 ? 1 : tl;
  while (tl > 1 && tl * G > 256) --tl;
  if (tl > max_lines) tl = max_lines;
  // a power of two (the transposed loads and stores index lines by shifts)
  int p2 = 1;
  while (2 * p2 <= tl) p2 *= 2;
  tl = p2;
  // whole warps (the FFT stages of lines shorter than 32 lanes end with a warp barrier)
  const int q = G < 32 ? 32 / G : 1;
  if (tl < q) tl = q;
  // a launch of few lines in all: fewer lines per CTA, so that it still spreads over the SMs
  while (tl > q && (lines + tl - 1) / tl < 2 * 152) tl /= 2;
  return tl;
}

// A tuned choice (> 0) replaces the shared-memory / thread budget; whole warps and the
// spreading of small launches still apply.
int pick_tl_tuned(int tuned, int len, int elem_bytes, int G, int budget, long long lines) {
  if (tuned <= 0) return pick_tl(len, elem_bytes, G, budget, 64, lines);
  int tl = tuned;
  const int q = G < 32 ? 32 / G : 1;
  if (tl < q) tl = q;
  while (tl > q && (lines + tl - 1) / tl < 2 * 152) tl /= 2;
  return tl;
}

template <typename T>
constexpr int engine_index() {
  return std::is_same<T, float>::value ? 0 : (std::is_same<T, double>::value ? 1 : 2);
}

template <typename Kern>
cudaError_t set_smem(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The transform kernels are instantiated per REM = log2(P) mod 4 (the stage sequence is
// then fixed at compile time); f(RemTag<REM>) launches the matching instance.
template <int R>
struct RemTag {
  static constexpr int value = R;
};
template <typename F>
cudaError_t with_rem(int logP, F&& f) {
  switch (logP & 3) {
    case 0: return f(RemTag<0>{});
    case 1: return f(RemTag<1>{});
    case 2: return f(RemTag<2>{});
    default: return f(RemTag<3>{});
  }
}

template <int R, int L>
struct ShapeTag {
  static constexpr int rem = R;
  static constexpr int logp = L;
};
// Transform shapes of the apply stages: with SPEC, every line length the plans allow (2^4 .. 2^13
// points) runs a kernel with the length fixed at compile time; without, the run-time-length
// kernel.  k_colmul is specialised for FP32 and double-float, the other stages for FP32 only
// (the double-float ones are dominated by their arithmetic; their instances would double the
// compile time).
template <typename T, bool SPEC = !std::is_same<T, double>::value, typename F>
cudaError_t with_line_shape(int logP, F&& f) {
  if constexpr (SPEC) {
    switch (logP) {
      case 4: return f(ShapeTag<0, 4>{});
      case 5: return f(ShapeTag<1, 5>{});
      case 6: return f(ShapeTag<2, 6>{});
      case 7: return f(ShapeTag<3, 7>{});
      case 8: return f(ShapeTag<0, 8>{});
      case 9: return f(ShapeTag<1, 9>{});
      case 10: return f(ShapeTag<2, 10>{});
      case 11: return f(ShapeTag<3, 11>{});
      case 12: return f(ShapeTag<0, 12>{});
      case 13: return f(ShapeTag<1, 13>{});
      default: return cudaErrorInvalidValue;  // plan creation admits no longer line
    }
  } else {
    return with_rem(logP, [&](auto t) { return f(ShapeTag<decltype(t)::value, 0>{}); });
  }
}

}  // namespace

// B instances of the same shape: u, y at stride `vstride` elements, workspace at stride
// apply_work_bytes(p), symbols at stride lam_stride (0: all share one), skip flags at
// stride skip_stride ints.
template <typename T>
static const cplx<T>* twiddle_table(const Plan& p, int r) {
  if constexpr (std::is_same<T, double>::value) return p.tw64[r];
  else if constexpr (std::is_same<T, float>::value) return p.tw32[r];
  else return p.twdf[r];
}

template <typename T>
static const T* symbol_table(const Plan& p) {
  if constexpr (std::is_same<T, double>::value) return p.lamL64;
  else if constexpr (std::is_same<T, float>::value) return p.lam32;
  else return p.lamdf;
}

// The first stage as the persistent k_r2c_pf: as many CTAs as fit on the device at once, or one
// per tile if there are fewer tiles.
template <typename T>
cudaError_t launch_r2c_pf(const io_t<T>* u, cplx<T>* S1, int nrows, int nx, size_t ld1, int logH, int tl, size_t sm,
                          const cplx<T>* tw, const int* skip, Batch b_in, int B, cudaStream_t s) {
  if constexpr (kR2CPersistentMaxLogH<T> < 0) {
    return cudaErrorNotSupported;
  } else {
    const int G = 1 << (logH - 4);
    return with_line_shape<T, std::is_same<T, float>::value>(logH, [&](auto tag) {
      constexpr int REM = decltype(tag)::rem, LL = decltype(tag)::logp;
      cudaError_t e = set_smem(k_r2c_pf<T, REM, LL>, sm);
      if (e != cudaSuccess) return e;
      int occ = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_r2c_pf<T, REM, LL>, tl * G, sm);
      if (e != cudaSuccess) return e;
      const long long tiles = (long long)((nrows + tl - 1) / tl) * B;
      const long long slots = (long long)(occ > 0 ? occ : 1) * device_sm_count();
      const int grid = (int)(tiles < slots ? tiles : slots);
      k_r2c_pf<T, REM, LL><<<grid, tl * G, sm, s>>>(u, S1, nrows, nx, ld1, logH, tl, tw, logH + 1, skip, b_in, B);
      return cudaGetLastError();
    });
  }
}

// The hybrid middle stage (k_colmul_hyb), one instance per REM; a template so that only the
// translation unit that runs it compiles it.
template <int UNUSED = 0>
cudaError_t launch_colmul_hyb(double2* data, int ncols, int n, size_t ld, int logP, int tl, const double* lam,
                              LamMap map, const double2* tw64, const cdf* twdf, const int* skip, Batch b, int grid,
                              int B, size_t sm, cudaStream_t s) {
  const int G = 1 << (logP - 4);
  return with_rem(logP, [&](auto tag) {
    constexpr int REM = decltype(tag)::value;
    cudaError_t e = set_smem(k_colmul_hyb<REM>, sm);
    if (e != cudaSuccess) return e;
    k_colmul_hyb<REM><<<dim3(grid, B), tl * G, sm, s>>>(data, ncols, n, ld, logP, tl, lam, map, tw64, twdf, skip, b);
    return cudaGetLastError();
  });
}

// TI: the engine of the inverse transforms (the last stage, the 3D inverse y stage and the middle
// stage's inverse half); TI = T but for the residual apply of double-float plans, <double, dfl>
// (k_colmul_hyb), which plans with the split middle stage do not take.
template <typename T, typename TI = T>
static cudaError_t apply_launch_b(const Plan& p, int B, const io_t<T>* u, io_t<TI>* y, size_t vstride, void* work,
                                  cudaStream_t s, const int* skip, int skip_stride, cudaEvent_t const* ev,
                                  const T* lam_override, size_t lam_stride, bool odd = false) {
  constexpr bool kHyb = !std::is_same<T, TI>::value;
  static_assert(!kHyb || (std::is_same<T, double>::value && std::is_same<TI, dfl>::value),
                "apply_launch_b: the only mixed form is FP64 forward, double-float inverse");
  if (kHyb && (odd || (p.d == 2 && p.P[1] > kMaxLine))) return cudaErrorNotSupported;
  // odd: the pipeline on odd extensions (a multiplier in the sine basis, see k_r2c_T); the FP32
  // engine only, P_r = 2(n_r + 1) on every axis (the callers check)
  if (odd && (!std::is_same<T, float>::value || p.P[1] > kMaxLine)) return cudaErrorNotSupported;
  int stage = 0;
  auto mark = [&]() -> cudaError_t {
    if (ev && ev[stage]) {
      cudaError_t e = cudaEventRecord(ev[stage], s);
      if (e != cudaSuccess) return e;
    }
    ++stage;
    return cudaSuccess;
  };
  using C = cplx<T>;
  const int eb = sizeof(C);
  const int budget = 96 * 1024;
  const int* tuned = p.tl_tuned[engine_index<T>()];
  const C* tw[3];
  for (int r = 0; r < 3; ++r) tw[r] = twiddle_table<T>(p, r);
  using CI = cplx<TI>;
  static_assert(sizeof(CI) == sizeof(C), "apply_launch_b: both engines keep the same bytes per value");
  const int* tunedI = p.tl_tuned[engine_index<TI>()];
  const CI* twI[3];
  for (int r = 0; r < 3; ++r) twI[r] = twiddle_table<TI>(p, r);
  const T* lam = lam_override ? lam_override : symbol_table<T>(p);
  C* S1 = reinterpret_cast<C*>(work);
  C* S2 = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(work) + align256(p.s1_elems * eb));
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const int logPx = p.logP[0], logPy = p.logP[1], logPz = p.logP[2];
  const int Hx = p.P[0] / 2;
  const int nrows = ny * (p.d == 3 ? nz : 1);
  const size_t ld1 = (size_t)nrows;  // S1 k-stride: all (z, y) rows
  // per-instance workspace: S1 and S2 of one apply, in complex elements
  const size_t wstride = apply_work_bytes(p, sizeof(T)) / eb;
#ifdef FRLAP_BOUNDS_CHECK
  {
    BcRanges r;
    const size_t vext = ((size_t)(B - 1) * vstride + p.M) * sizeof(io_t<T>);
    r.add(u, vext);
    r.add(y, vext);
    r.add(work, (size_t)B * apply_work_bytes(p, sizeof(T)));
    r.add(lam, ((size_t)(B - 1) * lam_stride + p.lam_count) * sizeof(T));
    for (int a = 0; a < p.d; ++a) r.add(tw[a], (size_t)twiddle_entries(p.P[a]) * sizeof(C));
    if (kHyb)
      for (int a = 0; a < p.d; ++a) r.add(twI[a], (size_t)twiddle_entries(p.P[a]) * sizeof(CI));
    if (skip) r.add(skip, ((size_t)(B - 1) * skip_stride + 1) * sizeof(int));
    cudaError_t e = r.commit(s);
    if (e != cudaSuccess) return e;
  }
#endif
  if (B > 1) S2 = S1 + align256(p.s1_elems * eb) / eb;
  Batch b_in;   // u -> S1
  b_in.in = vstride;
  b_in.out = wstride;
  b_in.skip = skip_stride;
  Batch b_ws;   // workspace-only stages (+ symbol)
  b_ws.in = wstride;
  b_ws.out = wstride;
  b_ws.lam = lam_stride;
  b_ws.skip = skip_stride;
  Batch b_out;  // S1 -> y
  b_out.in = wstride;
  b_out.out = vstride;
  b_out.skip = skip_stride;

  // ---- stage 1: rows of u -> S1[kx][row]
  if (!odd && use_r2c_pf<T>(logPx - 1, u)) {
    const int G = Hx >> 4;
    const int q = G < 32 ? 32 / G : 1;
    int tl = pick_tl_tuned(tuned[0], sline(Hx), eb, G, budget, (long long)nrows * B);
    while (tl > q && r2c_pf_smem_bytes<T>(tl, Hx, nx) > kMaxSmem) tl /= 2;
    const size_t sm = r2c_pf_smem_bytes<T>(tl, Hx, nx);
    cudaError_t e;
    if ((e = mark()) != cudaSuccess) return e;
    e = launch_r2c_pf<T>(u, S1, nrows, nx, ld1, logPx - 1, tl, sm, tw[0], skip, b_in, B, s);
    if (e != cudaSuccess) return e;
  } else {
    const int G = Hx >> 4;
    const int tl = pick_tl_tuned(tuned[0], sline(Hx), eb, G, budget, (long long)nrows * B);
    const size_t sm = (size_t)tl * r2c_line_stride<T>(Hx, tl) * eb;
    cudaError_t e;
    const int grid = (nrows + tl - 1) / tl;
    if ((e = mark()) != cudaSuccess) return e;
    if constexpr (std::is_same<T, float>::value) {
      if (odd)
        e = with_rem(logPx - 1, [&](auto tag) {
          constexpr int REM = decltype(tag)::value;
          cudaError_t e2 = set_smem(k_r2c_T<T, REM, 0, true>, sm);
          if (e2 != cudaSuccess) return e2;
          k_r2c_T<T, REM, 0, true><<<dim3(grid, B), tl * G, sm, s>>>(u, S1, nrows, nx, nx, ld1, logPx - 1, tl, tw[0],
                                                                      logPx, skip, b_in);
          return cudaGetLastError();
        });
    }
    if (!odd)
      e = with_line_shape<T, std::is_same<T, float>::value>(logPx - 1, [&](auto tag) {
        constexpr int REM = decltype(tag)::rem, LL = decltype(tag)::logp;
        cudaError_t e2 = set_smem(k_r2c_T<T, REM, LL>, sm);
        if (e2 != cudaSuccess) return e2;
        k_r2c_T<T, REM, LL><<<dim3(grid, B), tl * G, sm, s>>>(u, S1, nrows, nx, nx, ld1, logPx - 1, tl, tw[0], logPx, skip, b_in);
        return cudaGetLastError();
      });
    if (e != cudaSuccess) return e;
  }
  LamMap map;
  map.d = p.d;
  map.Hx1 = Hx + 1;
  map.logPy = logPy;
  map.Py = p.P[1];
  map.Hy1 = p.P[1] / 2 + 1;
  map.Hz1 = p.d == 3 ? p.P[2] / 2 + 1 : 1;
  if (p.d == 2 && p.P[1] > kMaxLine) {
    // 16384-point y embedding: the even and the odd half of the middle stage (k_colmul_split)
    constexpr int L = kMaxLine, G = L >> 4;
    const int tl = pick_tl_tuned(tuned[1], sline(L), eb, G, budget, (long long)(Hx + 1) * B);
    const size_t sm = (size_t)tl * sline(L) * eb;
    const int ncols = Hx + 1;
    const int grid = (ncols + tl - 1) / tl;
    Batch b_split = b_ws;  // columns in S1, the even half in S2 (same per-instance stride)
    cudaError_t e;
    if ((e = mark()) != cudaSuccess) return e;
    if constexpr (kHyb) {
      return cudaErrorNotSupported;  // refused above; no split instances in the hybrid's unit
    } else {
      if ((e = set_smem(k_colmul_split<T, false>, sm)) != cudaSuccess) return e;
      if ((e = set_smem(k_colmul_split<T, true>, sm)) != cudaSuccess) return e;
      k_colmul_split<T, false><<<dim3(grid, B), tl * G, sm, s>>>(S1, S2, ncols, ny, ld1, tl, lam, map.Hy1, tw[1],
                                                                skip, b_split);
      k_colmul_split<T, true><<<dim3(grid, B), tl * G, sm, s>>>(S1, S2, ncols, ny, ld1, tl, lam, map.Hy1, tw[1],
                                                               skip, b_split);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  } else if (p.d == 2) {
    const int G = p.P[1] >> 4;
    const int tl = pick_tl_tuned(tuned[1], sline(p.P[1]), eb, G, budget, (long long)(Hx + 1) * B);
    const size_t sm = (size_t)tl * sline(p.P[1]) * eb;
    cudaError_t e;
    const int ncols = Hx + 1;
    const int grid = (ncols + tl - 1) / tl;
    if ((e = mark()) != cudaSuccess) return e;
    if constexpr (kHyb) {
      e = launch_colmul_hyb(reinterpret_cast<double2*>(S1), ncols, ny, ld1, logPy, tl,
                            reinterpret_cast<const double*>(lam), map, reinterpret_cast<const double2*>(tw[1]),
                            reinterpret_cast<const cdf*>(twI[1]), skip, b_ws, grid, B, sm, s);
    } else {
    if constexpr (std::is_same<T, float>::value) {
      if (odd)
        e = with_rem(logPy, [&](auto tag) {
          constexpr int REM = decltype(tag)::value;
          cudaError_t e2 = set_smem(k_colmul<T, REM, 0, true>, sm);
          if (e2 != cudaSuccess) return e2;
          k_colmul<T, REM, 0, true><<<dim3(grid, B), tl * G, sm, s>>>(S1, ncols, ny, ld1, logPy, tl, lam, map, tw[1],
                                                                       logPy, skip, b_ws);
          return cudaGetLastError();
        });
    }
    if (!odd)
      e = with_line_shape<T>(logPy, [&](auto tag) {
        constexpr int REM = decltype(tag)::rem, LP = decltype(tag)::logp;
        cudaError_t e2 = set_smem(k_colmul<T, REM, LP>, sm);
        if (e2 != cudaSuccess) return e2;
        k_colmul<T, REM, LP><<<dim3(grid, B), tl * G, sm, s>>>(S1, ncols, ny, ld1, logPy, tl, lam, map, tw[1], logPy, skip, b_ws);
        return cudaGetLastError();
      });
    }
    if (e != cudaSuccess) return e;
  } else {
    const int Py = p.P[1], Pz = p.P[2];
    // ---- stage 2: S1[kx][z][y] -> FFT_y -> S2[kx][ky][z]
    {
      const int G = Py >> 4;
      const int tl = pick_tl_tuned(tuned[1], sline(Py), eb, G, budget, (long long)nz * (Hx + 1) * B);
      const size_t sm = (size_t)tl * sline(Py) * eb;
      cudaError_t e;
      const int tiles = (nz + tl - 1) / tl;
      const int grid = (Hx + 1) * tiles;
    if ((e = mark()) != cudaSuccess) return e;
    if constexpr (std::is_same<T, float>::value) {
      if (odd)
        e = with_rem(logPy, [&](auto tag) {
          constexpr int REM = decltype(tag)::value;
          cudaError_t e2 = set_smem(k_c2cT_fwd<T, REM, 0, true>, sm);
          if (e2 != cudaSuccess) return e2;
          k_c2cT_fwd<T, REM, 0, true><<<dim3(grid, B), tl * G, sm, s>>>(S1, S2, nz, tiles, ny, (size_t)nz * ny, ny,
                                                                         (size_t)Py * nz, nz, logPy, tl, tw[1], logPy,
                                                                         skip, b_ws);
          return cudaGetLastError();
        });
    }
    if (!odd)
    e = with_line_shape<T, std::is_same<T, float>::value>(logPy, [&](auto tag) {
      constexpr int REM = decltype(tag)::rem, LL = decltype(tag)::logp;
      cudaError_t e2 = set_smem(k_c2cT_fwd<T, REM, LL>, sm);
      if (e2 != cudaSuccess) return e2;
      k_c2cT_fwd<T, REM, LL><<<dim3(grid, B), tl * G, sm, s>>>(S1, S2, nz, tiles, ny, (size_t)nz * ny, ny, (size_t)Py * nz, nz, logPy, tl, tw[1], logPy, skip, b_ws);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    }
    // ---- stage 3: S2[kx][ky][:] -> FFT_z, * lambda, IFFT_z
    {
      const int G = Pz >> 4;
      const int tl = pick_tl_tuned(tuned[2], sline(Pz), eb, G, budget, (long long)(Hx + 1) * Py * B);
      const size_t sm = (size_t)tl * sline(Pz) * eb;
      cudaError_t e;
      const int ncols = (Hx + 1) * Py;
      const int grid = (ncols + tl - 1) / tl;
    if ((e = mark()) != cudaSuccess) return e;
    if constexpr (kHyb) {
      e = launch_colmul_hyb(reinterpret_cast<double2*>(S2), ncols, nz, (size_t)nz, logPz, tl,
                            reinterpret_cast<const double*>(lam), map, reinterpret_cast<const double2*>(tw[2]),
                            reinterpret_cast<const cdf*>(twI[2]), skip, b_ws, grid, B, sm, s);
    } else {
    if constexpr (std::is_same<T, float>::value) {
      if (odd)
        e = with_rem(logPz, [&](auto tag) {
          constexpr int REM = decltype(tag)::value;
          cudaError_t e2 = set_smem(k_colmul<T, REM, 0, true>, sm);
          if (e2 != cudaSuccess) return e2;
          k_colmul<T, REM, 0, true><<<dim3(grid, B), tl * G, sm, s>>>(S2, ncols, nz, (size_t)nz, logPz, tl, lam, map,
                                                                       tw[2], logPz, skip, b_ws);
          return cudaGetLastError();
        });
    }
    if (!odd)
    e = with_line_shape<T>(logPz, [&](auto tag) {
      constexpr int REM = decltype(tag)::rem, LP = decltype(tag)::logp;
      cudaError_t e2 = set_smem(k_colmul<T, REM, LP>, sm);
      if (e2 != cudaSuccess) return e2;
      k_colmul<T, REM, LP><<<dim3(grid, B), tl * G, sm, s>>>(S2, ncols, nz, (size_t)nz, logPz, tl, lam, map, tw[2], logPz, skip, b_ws);
      return cudaGetLastError();
    });
    }
    if (e != cudaSuccess) return e;
    }
    // ---- stage 4: S2[kx][ky][z] -> IFFT_y -> S1[kx][z][y] (engine TI)
    {
      CI* S1i = reinterpret_cast<CI*>(S1);
      CI* S2i = reinterpret_cast<CI*>(S2);
      const int G = Py >> 4;
      const int tl = pick_tl_tuned(tunedI[3], sline(Py), eb, G, budget, (long long)nz * (Hx + 1) * B);
      const size_t sm = (size_t)tl * sline(Py) * eb;
      cudaError_t e;
      const int tiles = (nz + tl - 1) / tl;
      const int grid = (Hx + 1) * tiles;
    if ((e = mark()) != cudaSuccess) return e;
    if constexpr (std::is_same<TI, float>::value) {
      if (odd)
        e = with_rem(logPy, [&](auto tag) {
          constexpr int REM = decltype(tag)::value;
          cudaError_t e2 = set_smem(k_c2cT_inv<TI, REM, 0, true>, sm);
          if (e2 != cudaSuccess) return e2;
          k_c2cT_inv<TI, REM, 0, true><<<dim3(grid, B), tl * G, sm, s>>>(S2i, S1i, nz, tiles, ny, (size_t)Py * nz, nz,
                                                                          (size_t)nz * ny, ny, logPy, tl, twI[1], logPy,
                                                                          skip, b_ws);
          return cudaGetLastError();
        });
    }
    if (!odd)
    e = with_line_shape<TI, std::is_same<TI, float>::value>(logPy, [&](auto tag) {
      constexpr int REM = decltype(tag)::rem, LL = decltype(tag)::logp;
      cudaError_t e2 = set_smem(k_c2cT_inv<TI, REM, LL>, sm);
      if (e2 != cudaSuccess) return e2;
      k_c2cT_inv<TI, REM, LL><<<dim3(grid, B), tl * G, sm, s>>>(S2i, S1i, nz, tiles, ny, (size_t)Py * nz, nz, (size_t)nz * ny, ny, logPy, tl, twI[1], logPy, skip, b_ws);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    }
  }
  // ---- last stage: S1[kx][row] -> rows of y (engine TI)
  {
    const CI* S1i = reinterpret_cast<const CI*>(S1);
    const int G = Hx >> 4;
    const int tl = pick_tl_tuned(tunedI[p.d == 2 ? 2 : 4], sline(Hx), eb, G, budget, (long long)nrows * B);
    const size_t sm = (size_t)tl * sline(Hx) * eb;
    cudaError_t e;
    const int grid = (nrows + tl - 1) / tl;
    if ((e = mark()) != cudaSuccess) return e;
    if constexpr (std::is_same<TI, float>::value) {
      if (odd)
        e = with_rem(logPx - 1, [&](auto tag) {
          constexpr int REM = decltype(tag)::value;
          cudaError_t e2 = set_smem(k_c2r_T<TI, REM, 0, true>, sm);
          if (e2 != cudaSuccess) return e2;
          k_c2r_T<TI, REM, 0, true><<<dim3(grid, B), tl * G, sm, s>>>(S1i, y, nrows, nx, ld1, nx, logPx - 1, tl, twI[0],
                                                                       logPx, skip, b_out);
          return cudaGetLastError();
        });
    }
    if (!odd)
      e = with_line_shape<TI, std::is_same<TI, float>::value>(logPx - 1, [&](auto tag) {
        constexpr int REM = decltype(tag)::rem, LL = decltype(tag)::logp;
        cudaError_t e2 = set_smem(k_c2r_T<TI, REM, LL>, sm);
        if (e2 != cudaSuccess) return e2;
        k_c2r_T<TI, REM, LL><<<dim3(grid, B), tl * G, sm, s>>>(S1i, y, nrows, nx, ld1, nx, logPx - 1, tl, twI[0], logPx, skip, b_out);
        return cudaGetLastError();
      });
    if (e != cudaSuccess) return e;
  }
  return mark();
}

template <typename T>
cudaError_t apply_launch(const Plan& p, const io_t<T>* u, io_t<T>* y, void* work, cudaStream_t s, const int* skip,
                         cudaEvent_t const* ev, const T* lam_override, bool odd) {
  return apply_launch_b<T>(p, 1, u, y, 0, work, s, skip, 0, ev, lam_override, 0, odd);
}

template <typename T>
cudaError_t apply_batch_launch(const Plan& p, int B, const io_t<T>* u, io_t<T>* y, size_t vstride, void* work,
                               cudaStream_t s, const int* skip, int skip_stride, const T* lam, size_t lam_stride,
                               cudaEvent_t const* ev) {
  return apply_launch_b<T>(p, B, u, y, vstride, work, s, skip, skip_stride, ev, lam, lam_stride);
}

// SP = F R^T u on the half spectrum: 2D [kx][ky], 3D [kx][ky][kz] (kx <= P_x/2, full ky, kz).
template <typename T>
cudaError_t spectrum_forward(const Plan& p, const T* u, cplx<T>* SP, void* work, cudaStream_t s) {
  using C = cplx<T>;
  const int eb = sizeof(C);
  const int budget = 96 * 1024;
  const C* tw[3];
  for (int r = 0; r < 3; ++r) tw[r] = twiddle_table<T>(p, r);
#ifdef FRLAP_BOUNDS_CHECK
  {
    BcRanges r;
    r.add(u, p.M * sizeof(T));
    r.add(SP, spectrum_elems(p) * sizeof(C));
    r.add(work, apply_work_bytes(p, sizeof(T)));
    for (int a = 0; a < p.d; ++a) r.add(tw[a], (size_t)twiddle_entries(p.P[a]) * sizeof(C));
    cudaError_t e = r.commit(s);
    if (e != cudaSuccess) return e;
  }
#endif
  C* S1 = reinterpret_cast<C*>(work);
  C* S2 = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(work) + align256(p.s1_elems * eb));
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const int Hx = p.P[0] / 2;
  const int nrows = ny * (p.d == 3 ? nz : 1);
  cudaError_t e;
  {
    const int G = Hx >> 4;
    const int tl = pick_tl(sline(Hx), eb, G, budget, 64);
    const size_t sm = (size_t)tl * r2c_line_stride<T>(Hx, tl) * eb;
    e = with_rem(p.logP[0] - 1, [&](auto tag) {
      constexpr int REM = decltype(tag)::value;
      cudaError_t e2 = set_smem(k_r2c_T<T, REM>, sm);
      if (e2 != cudaSuccess) return e2;
      k_r2c_T<T, REM><<<(nrows + tl - 1) / tl, tl * G, sm, s>>>(u, S1, nrows, nx, nx, (size_t)nrows, p.logP[0] - 1, tl, tw[0], p.logP[0], nullptr, Batch{});
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  const C* lines = S1;
  int ncols = Hx + 1, n = ny, logP = p.logP[1];
  size_t ld = (size_t)nrows;
  const C* twl = tw[1];
  if (p.d == 3) {
    const int Py = p.P[1];
    const int G = Py >> 4;
    const int tl = pick_tl(sline(Py), eb, G, budget, 64);
    const size_t sm = (size_t)tl * sline(Py) * eb;
    const int tiles = (nz + tl - 1) / tl;
    e = with_rem(p.logP[1], [&](auto tag) {
      constexpr int REM = decltype(tag)::value;
      cudaError_t e2 = set_smem(k_c2cT_fwd<T, REM>, sm);
      if (e2 != cudaSuccess) return e2;
      k_c2cT_fwd<T, REM><<<(Hx + 1) * tiles, tl * G, sm, s>>>(S1, S2, nz, tiles, ny, (size_t)nz * ny, ny, (size_t)Py * nz, nz, p.logP[1], tl, tw[1], p.logP[1], nullptr, Batch{});
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    lines = S2;
    ncols = (Hx + 1) * Py;
    n = nz;
    ld = (size_t)nz;
    logP = p.logP[2];
    twl = tw[2];
  }
  const int P = 1 << logP;
  const int G = P >> 4;
  const int tl = pick_tl(sline(P), eb, G, budget, 64);
  const size_t sm = (size_t)tl * sline(P) * eb;
  if ((e = set_smem(k_col_fwd<T>, sm)) != cudaSuccess) return e;
  k_col_fwd<T><<<(ncols + tl - 1) / tl, tl * G, sm, s>>>(lines, SP, ncols, n, ld, (size_t)P, logP, tl, twl, logP);
  return cudaGetLastError();
}

// y = R F^-1 (mult * SP), mult = a symbol octant with the 1/prod(P) factor folded in.
template <typename T>
cudaError_t spectrum_inverse(const Plan& p, const cplx<T>* SP, const T* mult, T* y, void* work, cudaStream_t s) {
  using C = cplx<T>;
  const int eb = sizeof(C);
  const int budget = 96 * 1024;
  const C* tw[3];
  for (int r = 0; r < 3; ++r) tw[r] = twiddle_table<T>(p, r);
#ifdef FRLAP_BOUNDS_CHECK
  {
    BcRanges r;
    r.add(SP, spectrum_elems(p) * sizeof(C));
    r.add(mult, p.lam_count * sizeof(T));
    r.add(y, p.M * sizeof(T));
    r.add(work, apply_work_bytes(p, sizeof(T)));
    for (int a = 0; a < p.d; ++a) r.add(tw[a], (size_t)twiddle_entries(p.P[a]) * sizeof(C));
    cudaError_t e = r.commit(s);
    if (e != cudaSuccess) return e;
  }
#endif
  C* S1 = reinterpret_cast<C*>(work);
  C* S2 = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(work) + align256(p.s1_elems * eb));
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const int Hx = p.P[0] / 2;
  const int nrows = ny * (p.d == 3 ? nz : 1);
  LamMap map;
  map.d = p.d;
  map.Hx1 = Hx + 1;
  map.logPy = p.logP[1];
  map.Py = p.P[1];
  map.Hy1 = p.P[1] / 2 + 1;
  map.Hz1 = p.d == 3 ? p.P[2] / 2 + 1 : 1;
  cudaError_t e;
  {
    const int logP = p.d == 2 ? p.logP[1] : p.logP[2];
    const int P = 1 << logP;
    const int G = P >> 4;
    const int tl = pick_tl(sline(P), eb, G, budget, 64);
    const size_t sm = (size_t)tl * sline(P) * eb;
    if ((e = set_smem(k_col_mulinv<T>, sm)) != cudaSuccess) return e;
    const int ncols = p.d == 2 ? Hx + 1 : (Hx + 1) * p.P[1];
    const int n = p.d == 2 ? ny : nz;
    C* dst = p.d == 2 ? S1 : S2;
    const size_t ldo = p.d == 2 ? (size_t)nrows : (size_t)nz;
    k_col_mulinv<T><<<(ncols + tl - 1) / tl, tl * G, sm, s>>>(SP, dst, ncols, n, (size_t)P, ldo, logP, tl, mult, map,
                                                               p.d == 2 ? tw[1] : tw[2], logP);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (p.d == 3) {
    const int Py = p.P[1];
    const int G = Py >> 4;
    const int tl = pick_tl(sline(Py), eb, G, budget, 64);
    const size_t sm = (size_t)tl * sline(Py) * eb;
    const int tiles = (nz + tl - 1) / tl;
    e = with_rem(p.logP[1], [&](auto tag) {
      constexpr int REM = decltype(tag)::value;
      cudaError_t e2 = set_smem(k_c2cT_inv<T, REM>, sm);
      if (e2 != cudaSuccess) return e2;
      k_c2cT_inv<T, REM><<<(Hx + 1) * tiles, tl * G, sm, s>>>(S2, S1, nz, tiles, ny, (size_t)Py * nz, nz, (size_t)nz * ny, ny, p.logP[1], tl, tw[1], p.logP[1], nullptr, Batch{});
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  {
    const int G = Hx >> 4;
    const int tl = pick_tl(sline(Hx), eb, G, budget, 64);
    const size_t sm = (size_t)tl * sline(Hx) * eb;
    e = with_rem(p.logP[0] - 1, [&](auto tag) {
      constexpr int REM = decltype(tag)::value;
      cudaError_t e2 = set_smem(k_c2r_T<T, REM>, sm);
      if (e2 != cudaSuccess) return e2;
      k_c2r_T<T, REM><<<(nrows + tl - 1) / tl, tl * G, sm, s>>>(S1, y, nrows, nx, (size_t)nrows, nx, p.logP[0] - 1, tl, tw[0], p.logP[0], nullptr, Batch{});
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}


// Lines per CTA candidates of apply stage `st`: powers of two from whole warps up to the
// compiled thread bound (kMaxCta), 64 lines, and 227 KB of shared memory.
template <typename T>
static int stage_line_length(const Plan& p, int st) {
  const int Hx = p.P[0] / 2;
  if (p.d == 2) return st == 1 ? (p.P[1] > kMaxLine ? kMaxLine : p.P[1]) : Hx;
  if (st == 0 || st == 4) return Hx;
  return st == 2 ? p.P[2] : p.P[1];
}

template <typename T>
cudaError_t autotune_engine(Plan& p, int B, io_t<T>* u, io_t<T>* y, void* work, cudaStream_t s) {
  const int ns = p.d == 2 ? 3 : 5;
  const int eng = engine_index<T>();
  const int eb = (int)sizeof(cplx<T>);
  cudaEvent_t ev[6];
  for (int i = 0; i <= ns; ++i) {
    cudaError_t e = cudaEventCreate(&ev[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
      return e;
    }
  }
  cudaError_t e = cudaMemsetAsync(u, 0, (size_t)B * p.M * sizeof(io_t<T>), s);
  for (int st = 0; st < ns && e == cudaSuccess; ++st) {
    const int L = stage_line_length<T>(p, st);
    const int G = L >> 4;
    int best = 0;
    float best_ms = 0.f;
    for (int t = 1; t <= 64 && e == cudaSuccess; t *= 2) {
      const size_t smem = (st == 0 && use_r2c_pf<T>(p.logP[0] - 1, u)) ? r2c_pf_smem_bytes<T>(t, L, p.n[0])
                          : st == 0                                     ? (size_t)t * r2c_line_stride<T>(L, t) * eb
                                                                         : (size_t)t * sline(L) * eb;
      if (t * G > kMaxCta<T> || smem > kMaxSmem) break;
      if (G < 32 && t < 32 / G) continue;
      p.tl_tuned[eng][st] = t;
      float ms = 0.f;
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // one warm-up, two timed
        e = apply_launch_b<T>(p, B, u, y, p.M, work, s, nullptr, 0, ev, nullptr, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[ns]);
        float t_ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, ev[st], ev[st + 1]);
        if (rep > 0) ms += t_ms;
      }
      if (e == cudaSuccess && (best == 0 || ms < best_ms)) {
        best = t;
        best_ms = ms;
      }
    }
    p.tl_tuned[eng][st] = best;
  }
  for (int i = 0; i <= ns; ++i) cudaEventDestroy(ev[i]);
  return e;
}

// The give-up count and the bounds-check state of the including translation unit (every unit that
// includes this header has its own), read and reset.
[[maybe_unused]] static cudaError_t unit_wait_collect(unsigned long long* count) {
  unsigned long long c = 0ull;
  cudaError_t e = cudaMemcpyFromSymbol(&c, g_wait_timeouts, sizeof(c));
  if (e != cudaSuccess) return e;
  const unsigned long long z = 0ull;
  e = cudaMemcpyToSymbol(g_wait_timeouts, &z, sizeof(z));
  *count = c;
  return e;
}

[[maybe_unused]] static cudaError_t unit_bc_collect(unsigned long long* count, unsigned long long* first) {
#ifdef FRLAP_BOUNDS_CHECK
  BcState st;
  cudaError_t e = cudaMemcpyFromSymbol(&st, g_bc_state, sizeof(st));
  if (e != cudaSuccess) return e;
  const BcState z = {0ull, ~0ull};
  e = cudaMemcpyToSymbol(g_bc_state, &z, sizeof(z));
  *count = st.count;
  *first = st.first;
  return e;
#else
  *count = 0ull;
  *first = ~0ull;
  return cudaSuccess;
#endif
}

template <typename T>
cudaError_t wait_collect(unsigned long long* count) {
  return unit_wait_collect(count);
}
template <typename T>
cudaError_t bc_collect(unsigned long long* count, unsigned long long* first) {
  return unit_bc_collect(count, first);
}

}  // namespace frlap
