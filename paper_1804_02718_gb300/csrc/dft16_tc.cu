// Radix-16 DFT stages in two engines, CUDA cores and tensor cores (tcgen05, split TF32), to
// measure whether the tensor-core form of the FFTs' radix-16 stages pays on this GPU.  The apply
// does not use these kernels; frlap_dft16_stages runs them on tiles held on chip.
//
// One tile: 128 rows of 16 complex FP32 values, row r = 16 a + b (a < 8, b < 16).  One stage:
//   x'[a, b][q] = v[a, b][q] W_256^{b q} / 4            (twiddles; the 1/4 keeps the norm)
//   u[a, q][b]  = x'[a, b][q]                            (the exchange between stages)
//   v[a, q][k]  = sum_b u[a, q][b] W_16^{b k}            (a 16-point DFT per row)
// with W_L = exp(-2 pi i / L): the data movement and arithmetic of one Stockham radix-16 stage.
// A kernel loads its tile once, runs `reps` stages on chip and stores the tile.
//
// Tensor-core form.  The 16-point DFT of a row is a product with the real 32 x 32 matrix F of
// the DFT (row x row layout [re0, im0, re1, im1, ...]): D = A F, A the 128 x 32 tile.  TF32
// keeps 10 fraction bits, so both operands are split, x = x_hi + x_lo with x_hi = tf32(x), and
// D = A_hi F_hi + A_lo F_hi + A_hi F_lo (error about 2^-21 relative; A_lo F_lo is below it).
// One tcgen05.mma of kind::tf32 is M = 128, N = 32, K = 8: twelve per stage, accumulated in
// tensor memory (32 columns), read back with tcgen05.ld.  Operands sit in shared memory in the
// no-swizzle K-major layout: 8-row x 16-byte core matrices; the K-adjacent core matrices of A
// are 144 bytes apart (not 128), so that the exchange's stores of one row by 16 threads spread
// over all banks.
#include <cstdint>

#include "common.cuh"
#include "fft.cuh"

namespace frlap {
namespace {

constexpr int kTileRows = 128;
constexpr int kTileFloats = kTileRows * 32;
constexpr int kLboA = 144;                         // bytes between K-adjacent core matrices of A
constexpr int kSboA = 8 * kLboA;                   // bytes between 8-row groups of A
constexpr int kABytes = (kTileRows / 8) * kSboA;   // 18432
constexpr int kLboB = 128, kSboB = 8 * 128;
constexpr int kBBytes = (32 / 8) * kSboB;          // 4096
constexpr int kTcSmem = 2 * kABytes + 2 * kBBytes + 16;
constexpr int kTmemCols = 32;

// Instruction descriptor of kind::tf32: D in F32 (bits 4-5 = 1), A and B in TF32 (bits 7-9 and
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: start address, leading (K) and stride (M/N)
// byte offsets, all in 16-byte units; bits 46-47 = 1 (the Blackwell descriptor version).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ int a_offset(int r, int k) {  // bytes; r < 128, k < 32 (real index)
  return (r >> 3) * kSboA + (k >> 2) * kLboA + (r & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ int b_offset(int n, int k) {  // element (n, k) of F stored N-row, K-major
  return (n >> 3) * kSboB + (k >> 2) * kLboB + (n & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdescTf32), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void ld_row32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait on an mbarrier phase (as the apply's waits: about a second, then false).
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < (1 << 20); ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(1000u)
        : "memory");
    if (done) return true;
  }
  return false;
}

static __device__ unsigned long long g_tc_wait_timeouts = 0ull;

// cos and sin of pi m / 8, m < 16, in double, at compile time (Taylor series on |x| <= pi)
struct Cs16 {
  double c[16], s[16];
};
constexpr Cs16 make_cs16() {
  Cs16 t{};
  for (int m = 0; m < 16; ++m) {
    const int r = m <= 8 ? m : 16 - m;  // x = 2 pi - x' for m > 8: cos x = cos x', sin x = -sin x'
    const double x = 3.14159265358979323846 * r / 8.0;
    t.c[m] = taylor_cs(x, false);
    t.s[m] = m <= 8 ? taylor_cs(x, true) : -taylor_cs(x, true);
  }
  return t;
}
static __constant__ Cs16 c_cs16 = make_cs16();

// W_256^{b q} / 4 for q < 16 (the thread's row twiddles; the 16-point DFT multiplies norms by 4)
__device__ __forceinline__ void row_twiddles(float2* tw, int b) {
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    float s, c;
    sincospif(-(float)(b * q) / 128.0f, &s, &c);
    tw[q] = make_float2(0.25f * c, 0.25f * s);
  }
}

__device__ __forceinline__ void load_row(const float* __restrict__ in, float2* v) {
  const float4* p = reinterpret_cast<const float4*>(in);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 t = p[i];
    v[2 * i] = make_float2(t.x, t.y);
    v[2 * i + 1] = make_float2(t.z, t.w);
  }
}
__device__ __forceinline__ void store_row(float* __restrict__ out, const float2* v) {
  float4* p = reinterpret_cast<float4*>(out);
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
}

// CUDA-core form: the exchange through shared memory (rows padded to 17 values), then the
// register radix-16 DFT of the apply's FFTs.
__global__ void __launch_bounds__(128) k_dft16_cc(const float* __restrict__ in, float* __restrict__ out, int reps) {
  __shared__ float2 s[kTileRows * 17];
  const int m = threadIdx.x, a = m >> 4, b = m & 15;
  const size_t t0 = (size_t)blockIdx.x * kTileFloats + (size_t)m * 32;
  float2 v[16], tw[16];
  load_row(in + t0, v);
  row_twiddles(tw, b);
  for (int rep = 0; rep < reps; ++rep) {
#pragma unroll
    for (int q = 0; q < 16; ++q) s[(a * 16 + q) * 17 + b] = cmul(v[q], tw[q]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = s[m * 17 + k];
    __syncthreads();
    dft16<-1>(v);
  }
  store_row(out + t0, v);
}

// Tensor-core form (one tile per CTA, 4 warps; warp w reads tensor-memory lanes 32w..32w+31).
__global__ void __launch_bounds__(128) k_dft16_tc(const float* __restrict__ in, float* __restrict__ out, int reps) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* a_hi = sm;
  unsigned char* a_lo = sm + kABytes;
  unsigned char* b_hi = sm + 2 * kABytes;
  unsigned char* b_lo = b_hi + kBBytes;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(b_lo + kBBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int m = threadIdx.x, warp = m >> 5, a = m >> 4, b = m & 15;

  // F, split: element (n, k) with n = 2 q + c (output q, c = 0 real / 1 imaginary part) and
  // k = 2 j + d (input j, d likewise); theta = 2 pi j q / 16:
  //   re Y_q = sum_j re x_j cos theta + im x_j sin theta,  im Y_q = sum_j -re x_j sin theta + im x_j cos theta
  for (int e = m; e < 32 * 32; e += kTileRows) {
    const int n = e >> 5, k = e & 31, q = n >> 1, c = n & 1, j = k >> 1, d = k & 1;
    const double sn = c_cs16.s[(j * q) & 15], cs = c_cs16.c[(j * q) & 15];
    const double f = c == 0 ? (d == 0 ? cs : sn) : (d == 0 ? -sn : cs);
    const float fh = tf32_rna((float)f);
    *reinterpret_cast<float*>(b_hi + b_offset(n, k)) = fh;
    *reinterpret_cast<float*>(b_lo + b_offset(n, k)) = (float)(f - (double)fh);
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (m == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t bar_a = smem_addr(bar);
  const uint32_t sa_hi = smem_addr(a_hi), sa_lo = smem_addr(a_lo), sb_hi = smem_addr(b_hi), sb_lo = smem_addr(b_lo);

  const size_t t0 = (size_t)blockIdx.x * kTileFloats + (size_t)m * 32;
  float2 v[16], tw[16];
  load_row(in + t0, v);
  row_twiddles(tw, b);
  bool ok = true;
  int issued = 0;  // stages whose MMAs were issued
  for (int rep = 0; rep < reps; ++rep) {
    // twiddle, split, and the exchange: value q of row (a, b) goes to row (a, q), input b
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float2 x = cmul(v[q], tw[q]);
      const float2 h = make_float2(tf32_rna(x.x), tf32_rna(x.y));
      const int off = a_offset(a * 16 + q, 2 * b);
      *reinterpret_cast<float2*>(a_hi + off) = h;
      *reinterpret_cast<float2*>(a_lo + off) = make_float2(x.x - h.x, x.y - h.y);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc_fence_before();
    if (!__syncthreads_and(ok)) break;
    if (m == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < 4; ++s)
        mma_tf32(tmem, smem_desc(sa_hi + 2 * s * kLboA, kLboA, kSboA), smem_desc(sb_hi + 2 * s * kLboB, kLboB, kSboB),
                 s > 0);
#pragma unroll
      for (int s = 0; s < 4; ++s)
        mma_tf32(tmem, smem_desc(sa_lo + 2 * s * kLboA, kLboA, kSboA), smem_desc(sb_hi + 2 * s * kLboB, kLboB, kSboB), 1);
#pragma unroll
      for (int s = 0; s < 4; ++s)
        mma_tf32(tmem, smem_desc(sa_hi + 2 * s * kLboA, kLboA, kSboA), smem_desc(sb_lo + 2 * s * kLboB, kLboB, kSboB), 1);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_a)
                   : "memory");
    }
    ++issued;
    ok = bar_wait(bar_a, (uint32_t)rep & 1u);
    __syncwarp();  // the warp-wide tcgen05.ld needs its lanes converged after the wait loop
    tc_fence_after();
    float r[32];
    ld_row32(tmem + ((uint32_t)(32 * warp) << 16), r);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = make_float2(r[2 * q], r[2 * q + 1]);
  }
  if (!ok) {
    // a stage's wait gave up: wait (bounded) for its MMAs before the tensor memory is freed
    if (m == 0) atomicAdd(&g_tc_wait_timeouts, 1ull);
    if (issued > 0) bar_wait(bar_a, (uint32_t)(issued - 1) & 1u);
  } else {
    store_row(out + t0, v);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

cudaError_t dft16_stages_launch(int engine, const float* in, float* out, int ntiles, int reps, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (engine == 0) {
    k_dft16_cc<<<ntiles, kTileRows, 0, s>>>(in, out, reps);
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(k_dft16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  k_dft16_tc<<<ntiles, kTileRows, kTcSmem, s>>>(in, out, reps);
  return cudaGetLastError();
}

cudaError_t dft16_wait_collect(unsigned long long* count) {
  unsigned long long c = 0ull;
  cudaError_t e = cudaMemcpyFromSymbol(&c, g_tc_wait_timeouts, sizeof(c));
  if (e != cudaSuccess) return e;
  const unsigned long long z = 0ull;
  e = cudaMemcpyToSymbol(g_tc_wait_timeouts, &z, sizeof(z));
  *count = c;
  return e;
}

}  // namespace frlap
