// Internal definitions shared by the frlap CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <cstring>
#include <type_traits>

#include <string>

#include "../../include/frlap.h"
#include "dfloat.cuh"

namespace frlap {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
frlap_status fail(frlap_status code, const std::string& msg);
frlap_status cuda_fail(cudaError_t e, const char* where);

#define FRLAP_CUDA_TRY(call)                                   \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::frlap::cuda_fail(e_, #call); \
  } while (0)

#define FRLAP_LAUNCH_CHECK(where)                                   \
  do {                                                              \
    cudaError_t e_ = cudaGetLastError();                            \
    if (e_ != cudaSuccess) return ::frlap::cuda_fail(e_, where);    \
  } while (0)

// Upper bound on the passes of the graph-launched solver loops set by frlap_set_loop_pass_limit
// (0: none); a loop's bound is min(its own derived bound, this one).
unsigned loop_pass_limit();
inline unsigned capped_passes(unsigned derived) {
  const unsigned cap = loop_pass_limit();
  return (cap > 0u && cap < derived) ? cap : derived;
}

// ---------------------------------------------------------------- complex
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<dfl> { using type = cdf; };
template <typename T> using cplx = typename cplx_t<T>::type;

#ifdef FRLAP_BOUNDS_CHECK
constexpr int kBcMaxRanges = 12;
// the global byte ranges [lo, hi) the current launch may touch
struct BcTable {
  unsigned long long lo[kBcMaxRanges], hi[kBcMaxRanges];
  int n;
};
// accesses outside every range: how many, and the lowest such address
struct BcState {
  unsigned long long count, first;
};
// One copy per translation unit (file-scope statics): each apply translation unit registers and
// reports its own (apply_impl.cuh).
static __device__ BcTable g_bc_table;
static __device__ BcState g_bc_state = {0ull, ~0ull};

__device__ __forceinline__ bool bc_ok(const void* p, size_t bytes) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  if (g_bc_table.n == 0) return true;  // a translation unit that registers no ranges (symbol generation)
  for (int i = 0; i < g_bc_table.n; ++i)
    if (a >= g_bc_table.lo[i] && a + bytes <= g_bc_table.hi[i]) return true;
  atomicAdd(&g_bc_state.count, 1ull);
  atomicMin(&g_bc_state.first, a);
  return false;
}
template <typename V>
__device__ __forceinline__ V bc_ld(const V* p) {
  V v;
  if (bc_ok(p, sizeof(V))) v = *p;
  else memset(&v, 0, sizeof(V));
  return v;
}
template <typename V>
__device__ __forceinline__ void bc_st(V* p, const V& v) {
  if (bc_ok(p, sizeof(V))) *p = v;
}
#endif

// Load of data a kernel reads once (cache-streaming: evict-first in L1 and L2), so that the
// twiddle tables keep the L1.  8- and 16-byte values: float2 / float4 / double2 / cdf; 4 and 8
// byte scalars.
template <typename V>
__device__ __forceinline__ V ld_stream(const V* p) {
  static_assert(sizeof(V) == 4 || sizeof(V) == 8 || sizeof(V) == 16, "ld_stream: 4, 8 or 16 bytes");
  V r;
#ifdef FRLAP_BOUNDS_CHECK
  if (!bc_ok(p, sizeof(V))) {
    memset(&r, 0, sizeof(V));
    return r;
  }
#endif
  if constexpr (sizeof(V) == 4) {
    const float t = __ldcs(reinterpret_cast<const float*>(p));
    memcpy(&r, &t, 4);
  } else if constexpr (sizeof(V) == 8) {
    const float2 t = __ldcs(reinterpret_cast<const float2*>(p));
    memcpy(&r, &t, 8);
  } else {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    memcpy(&r, &t, 16);
  }
  return r;
}

// ---------------------------------------------------------------- bounds-checked build
// With -DFRLAP_BOUNDS_CHECK every global load and store of the apply kernels goes through
// FRLAP_GLD / FRLAP_GST / FRLAP_GOK, which test the accessed bytes against the buffers the
// launching call registered (apply_impl.cuh: the call's vectors, workspace, symbol, twiddle
// tables and skip flags).  An access outside all of them is counted, its address kept, and
// the access is skipped (a load returns zero): nothing faults.  Without the macro the three
// expand to the plain accesses.
#ifdef FRLAP_BOUNDS_CHECK
#define FRLAP_GLD(p) ::frlap::bc_ld(p)
#define FRLAP_GST(p, v) ::frlap::bc_st((p), (v))
#define FRLAP_GOK(p) ::frlap::bc_ok((p), sizeof(*(p)))
#else
#define FRLAP_GLD(p) (*(p))
#define FRLAP_GST(p, v) (*(p) = (v))
#define FRLAP_GOK(p) true
#endif


// storage type of the real grid vectors and of the symbol for each compute type:
// FP32 and FP64 compute and store in their own type; double-float computes in
// dfl, reads and writes FP64 vectors, and keeps its symbol/twiddles as dfl.
template <typename T> struct io_t_ { using type = T; };
template <> struct io_t_<dfl> { using type = double; };
template <typename T> using io_t = typename io_t_<T>::type;

// two consecutive grid values as one aligned vector (float2 / double2)
template <typename T> using io_pair = typename std::conditional<sizeof(io_t<T>) == 4, float2, double2>::type;

template <typename T> __device__ __forceinline__ T from_io(io_t<T> v) { return v; }
template <> __device__ __forceinline__ dfl from_io<dfl>(double v) { return df_from(v); }
template <typename T> __device__ __forceinline__ io_t<T> to_io(T v) { return v; }
template <> __device__ __forceinline__ double to_io<dfl>(dfl v) { return df_to(v); }

// the real type of a complex type
template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<cdf> { using type = dfl; };
template <typename C> using real_t = typename real_of<C>::type;

__host__ __device__ __forceinline__ float2 make_cplx(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 make_cplx(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ cdf make_cplx(dfl a, dfl b) { return make_cdf(a, b); }
template <typename C> __host__ __device__ __forceinline__ C mk(real_t<C> a, real_t<C> b) { return make_cplx(a, b); }
template <typename C> __host__ __device__ __forceinline__ C czero() {
  using T = real_t<C>;
  return mk<C>(T(0), T(0));
}
// real and imaginary parts
__device__ __forceinline__ float re(float2 a) { return a.x; }
__device__ __forceinline__ float im(float2 a) { return a.y; }
__device__ __forceinline__ double re(double2 a) { return a.x; }
__device__ __forceinline__ double im(double2 a) { return a.y; }
__device__ __forceinline__ dfl re(cdf a) { return cdf_re(a); }
__device__ __forceinline__ dfl im(cdf a) { return cdf_im(a); }
// FP32 complex sums as single paired instructions (each component rounded as the scalar add;
// a - b as b * (-1) + a, whose product is exact)
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return __fmul2_rn(make_float2(s, s), a); }
// Sums that only feed another sum: plain for FP32 / FP64; without the closing renormalisation
// for double-float (dfloat.cuh).
__device__ __forceinline__ float2 add_lazy(float2 a, float2 b) { return a + b; }
__device__ __forceinline__ float2 sub_lazy(float2 a, float2 b) { return a - b; }
__device__ __forceinline__ double2 add_lazy(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 sub_lazy(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// a / 2, exactly (a power-of-two scaling of each component)
__device__ __forceinline__ float2 halve(float2 a) { return __fmul2_rn(a, make_float2(0.5f, 0.5f)); }
__device__ __forceinline__ double2 halve(double2 a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
__device__ __forceinline__ cdf halve(cdf a) {
  cdf r;
  r.hi = p_mul(a.hi, p_bcast(0.5f));
  r.lo = p_mul(a.lo, p_bcast(0.5f));
  return r;
}
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// complex product a*b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// products that only feed a sum: as cmul / cmulc here, unrenormalised for double-float
__device__ __forceinline__ float2 cmul_lazy(float2 a, float2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 cmul_lazy(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 cmulc_lazy(float2 a, float2 b) { return cmulc(a, b); }
__device__ __forceinline__ double2 cmulc_lazy(double2 a, double2 b) { return cmulc(a, b); }
template <typename C> __device__ __forceinline__ C conjg(C a) { a.y = -a.y; return a; }
template <> __device__ __forceinline__ cdf conjg<cdf>(cdf a) { return cdf_conj(a); }
// multiply by -i (forward) or +i (inverse): sign = -1 gives -i*a
template <int SIGN, typename C> __device__ __forceinline__ C mul_i(C a) {
  C r;
  if (SIGN < 0) { r.x = a.y; r.y = -a.x; } else { r.x = -a.y; r.y = a.x; }
  return r;
}
template <int SIGN> __device__ __forceinline__ cdf mul_i_cdf(cdf a) {
  cdf r;
  if (SIGN < 0) {
    r.hi = make_float2(a.hi.y, -a.hi.x);
    r.lo = make_float2(a.lo.y, -a.lo.x);
  } else {
    r.hi = make_float2(-a.hi.y, a.hi.x);
    r.lo = make_float2(-a.lo.y, a.lo.x);
  }
  return r;
}
template <> __device__ __forceinline__ cdf mul_i<-1, cdf>(cdf a) { return mul_i_cdf<-1>(a); }
template <> __device__ __forceinline__ cdf mul_i<1, cdf>(cdf a) { return mul_i_cdf<1>(a); }

// ---------------------------------------------------------------- plan
// Longest FFT line the transform kernels hold (one line of 2^13 points per 2^9 threads); longer
// 2D embeddings (16384 points) split their middle stage into two halves of this length.
constexpr int kMaxLine = 8192;

struct Plan {
  int d;
  int N[3];        // mesh intervals per axis (x, y, z); unused axes = 2
  int n[3];        // interior unknowns per axis n_r = N_r - 1 (unused axes 1)
  int P[3];        // embedding (FFT) sizes per axis (unused axes 1)
  int logP[3];
  int Nmax;
  double alpha, gamma, h, c;
  int prec;        // frlap_prec
  size_t M;        // number of unknowns
  size_t lam_count;            // prod (P_r/2 + 1) over the used axes
  // The symbol octant lambda(kx, ky[, kz]), k_r = 0..P_r/2, with 1/prod(P) folded in.
  // lam64 is in natural order ([ky][kx] / [kz][ky][kx], kx fastest).  The tables the
  // apply's middle stage reads (lamL64, lam32, lamdf and the preconditioner multipliers)
  // are line-major: axes reversed ([kx][ky] / [kx][ky][kz]), so that the folded line of
  // one column is contiguous.
  double* lam64 = nullptr;     // natural order, FP64 (always built)
  double* lamL64 = nullptr;    // line-major, FP64 (always built)
  float* lam32 = nullptr;      // line-major, FP32 (all plans but F64)
  // exp(-2 pi i m / P_r), m < P_r, followed by the radix-16 stage table of
  // twiddle_entries(P_r): see there
  double2* tw64[3] = {nullptr, nullptr, nullptr};
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  cdf* twdf[3] = {nullptr, nullptr, nullptr};      // the same twiddles as double-floats
  dfl* lamdf = nullptr;        // line-major, as double-floats (DF64 plans)
  bool df64 = false;           // FP64-precision vectors are applied with double-float FFTs
  // workspace layout of one apply, in complex elements of the apply precision
  size_t s1_elems = 0, s2_elems = 0;
  cudaStream_t side = nullptr;  // internal stream for captured solver graphs
  // preconditioner multipliers (line-major like lam32, FP32; nullptr until built)
  float* mu_strang = nullptr;   // inverse of the multilevel Strang circulant, embedded like A
  float* mu_learned = nullptr;  // learned Fourier multiplier
  float* mu_tau = nullptr;      // inverse of diag(S A S) in the sine basis S (applied on odd extensions)
  // lines per CTA of each apply stage, per engine (0 FP32, 1 FP64, 2 double-float), set by
  // frlap_plan_autotune; 0 = the built-in choice
  int tl_tuned[3][5] = {};
};

// Bounded waits of the apply kernels on their asynchronous copies (mbarrier phases) that gave up
// since the last call, per engine's translation unit (the counter is reset).  A kernel whose wait
// gives up records it and returns without storing that tile's results.
template <typename T>
cudaError_t wait_collect(unsigned long long* count);

// Bounds-checked builds: accesses outside the registered ranges since the last call, summed per
// engine's translation unit (the counters are reset); ordinary builds report zero.
template <typename T>
cudaError_t bc_collect(unsigned long long* count, unsigned long long* first);
// Bounds-checked builds: registers one 8-double range and probes 8 loads inside it and 5 just past
// it (memory the library owns, so the probes are safe even unchecked); *flagged = accesses flagged.
cudaError_t bc_selftest(unsigned long long* flagged);
// Runs one bounded mbarrier wait that nothing completes; *timeouts = waits that gave up (1 expected).
cudaError_t wait_selftest(unsigned long long* timeouts);
// the residual apply of double-float plans (FP64 forward, double-float inverse transforms; see
// apply_hyb.cu); cudaErrorNotSupported for other plans and for plans with a split middle stage
cudaError_t apply_residual_hyb(const Plan& p, const double* u, double* y, void* work, cudaStream_t s);
cudaError_t hyb_wait_collect(unsigned long long* count);
cudaError_t hyb_bc_collect(unsigned long long* count, unsigned long long* first);
// radix-16 stages on CUDA cores (engine 0) or tensor cores (engine 1); see dft16_tc.cu
cudaError_t dft16_stages_launch(int engine, const float* in, float* out, int ntiles, int reps, cudaStream_t s);
cudaError_t dft16_wait_collect(unsigned long long* count);

// apply pipeline (apply.cu); work must hold apply_work_bytes(plan, sizeof(T)) bytes
// T = compute type (float, double or dfl); vectors are io_t<T>, symbol overrides are T
template <typename T>
// odd: a multiplier lam_override in the sine basis (FP32, P_r = 2(n_r + 1); see k_r2c_T)
cudaError_t apply_launch(const Plan& p, const io_t<T>* u, io_t<T>* y, void* work, cudaStream_t s, const int* skip,
                         cudaEvent_t const* ev = nullptr, const T* lam_override = nullptr, bool odd = false);
// FP64 vectors through the plan's FP64 engine (native double or double-float)
cudaError_t apply64(const Plan& p, const double* u, double* y, void* work, cudaStream_t s, const int* skip,
                    cudaEvent_t const* ev = nullptr);
size_t apply_work_bytes(const Plan& p, int real_bytes);
// times every admissible lines-per-CTA choice of each apply stage on a batch of B zero vectors
// (u, y: B vectors each; work: B apply workspaces) and stores the fastest in p.tl_tuned
template <typename T>
cudaError_t autotune_engine(Plan& p, int B, io_t<T>* u, io_t<T>* y, void* work, cudaStream_t s);
// B same-shape instances in one launch per stage (see apply.cu)
template <typename T>
cudaError_t apply_batch_launch(const Plan& p, int B, const io_t<T>* u, io_t<T>* y, size_t vstride, void* work,
                               cudaStream_t s, const int* skip, int skip_stride, const T* lam, size_t lam_stride,
                               cudaEvent_t const* ev = nullptr);
// forward half spectrum F R^T u (2D [kx][ky], 3D [kx][ky][kz]) and its multiplied inverse; same workspace as apply
size_t spectrum_elems(const Plan& p);
template <typename T>
cudaError_t spectrum_forward(const Plan& p, const T* u, cplx<T>* SP, void* work, cudaStream_t s);
template <typename T>
cudaError_t spectrum_inverse(const Plan& p, const cplx<T>* SP, const T* mult, T* y, void* work, cudaStream_t s);

// coefficient / symbol generation (coeffs.cu)
cudaError_t coeffs_launch(int d, double alpha, double gamma, double h, int Nmax, double* coef, void* scratch,
                          cudaStream_t s);
size_t coeffs_scratch_bytes(int d, int Nmax);
cudaError_t symbol_launch(const Plan& p, const double* coef, double* lam_oct, cudaStream_t s);
// the sine-basis preconditioner of sigma I + s A from the plan's mu_tau (built), into mu_b
// (lam_count floats, line-major like mu_tau)
cudaError_t shifted_tau_launch(const Plan& p, double sigma, double s, float* mu_b, cudaStream_t st);
// the generator t_k = -c a_k (k_r <= n_r - 1, zero elsewhere) on the octant, natural order
cudaError_t generator_octant_launch(const Plan& p, const double* coef, double* lam_oct, cudaStream_t s);
// Entries of an FP64 / double-float twiddle table for embedding size P (a power of two >= 32).
// [0, P): W_P^m = exp(-2 pi i m / P).  Then, for Ns = 1, 2, 4, ..., P/16, the twiddles of a
// radix-16 Stockham stage with Ns: W_{16 Ns}^{r k} (r = 1..15, k < Ns) at
// P + 15 (Ns - 1) + (r - 1) Ns + k, so a warp's 32 consecutive k of one r are 32 consecutive
// entries (one load over a few cache lines instead of one line per lane).  The stage entries
// are copies of plain entries (W_{16 Ns}^{r k} = W_P^{r k P / (16 Ns)}), so both give the same bits.
inline int twiddle_entries(int P) { return P + 15 * (P / 8 - 1); }
// fills tw64 and tw32 (twiddle_entries(P) entries each; tw32 may be null)
cudaError_t twiddle_launch(int P, double2* tw64, float2* tw32, cudaStream_t s);
cudaError_t scale_symbol_launch(double* lam64, float* lam32, size_t n, double s, cudaStream_t st);
// dst (line-major, converted to To) = s * oct (natural order); To = double, float or dfl
template <typename To>
cudaError_t line_symbol_launch(const Plan& p, const double* oct, To* dst, double s, cudaStream_t st);
cudaError_t to_df_launch(const double* src, dfl* dst, size_t n, cudaStream_t st);
cudaError_t to_cdf_launch(const double2* src, cdf* dst, size_t n, cudaStream_t st);
// even DFT of the octant along every axis (used for both the operator and preconditioner symbols)
cudaError_t symbol_axes_launch(const Plan& p, double* lam_oct, cudaStream_t s);

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// True if the byte ranges [a, a + bytes) and [b, b + bytes) share any byte.
inline bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}
// Bytes of one grid vector of the plan in the element type of its apply (float for F32 plans,
// double otherwise).
inline size_t vector_bytes(const Plan& p, bool f32) { return p.M * (f32 ? sizeof(float) : sizeof(double)); }

}  // namespace frlap

// the opaque handle of the C ABI is the plan itself
struct frlap_plan : public frlap::Plan {};
