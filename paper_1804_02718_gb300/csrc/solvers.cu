// Device-resident conjugate gradients around the FFT apply (Sec. 5.3: each linear
// system is solved by CG with the FFT-based product), its use inside an FP64
// iterative-refinement loop with FP32 inner solves, and the semi-implicit
// Allen-Cahn step.
//
// The operator of every solve is B v = sigma v + s A v (Poisson: sigma = 0, s = 1;
// Allen-Cahn: sigma = 1, s = tau eps^2).  All CG scalars live on the device; each
// kernel reads a `done` flag first and does nothing once the iteration has
// stopped, so the host launches iterations in chunks and looks at the flag only
// between chunks.  Inner products are accumulated in FP64 with a fixed
// reduction order (per-block partials, then the last block to finish sums them
// in block order), so results are deterministic.
#include <math.h>

#include <type_traits>

#include <vector>

#include "common.cuh"

namespace frlap {

namespace {

constexpr int kBlocks = 2 * 152;  // grid of the vector kernels: two CTAs per SM (four measured slower)
constexpr int kThreads = 512;
// grid for n elements: two CTAs per SM, fewer for short vectors (the reductions use gridDim.x)
inline unsigned vgrid(size_t n) {
  const size_t b = (n + kThreads - 1) / kThreads;
  return (unsigned)(b < 1 ? 1 : (b > (size_t)kBlocks ? (size_t)kBlocks : b));
}

struct CgState {
  double rr;        // r . r
  double rz;        // r . z (z = M^-1 r; equals rr without a preconditioner)
  double pq;        // p . B p
  double alpha, beta;
  double tol2;      // (rtol ||f||)^2
  double fnorm2;
  double sigma, s;  // operator B = sigma I + s A
  int done;
  int status;       // frlap_status of the iteration
  int iters;
  unsigned counter; // last-block ticket for the reductions
  unsigned passes;  // loop passes of the graph-launched iterations
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Two block sums, then the last block to arrive reduces all partials in block order.
// Returns true in thread 0 of the last block, with the totals in *ta, *tb.
__device__ __forceinline__ bool grid_sum2(double a, double b, double* partials, unsigned* counter, double* ta,
                                          double* tb) {
  __shared__ double red[32];
  __shared__ bool is_last;
  const double sa = block_sum(a, red);
  __syncthreads();
  const double sb = block_sum(b, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = sa;
    partials[gridDim.x + blockIdx.x] = sb;
    __threadfence();
    is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  double va = 0.0, vb = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    va += *((volatile double*)&partials[i]);
    vb += *((volatile double*)&partials[gridDim.x + i]);
  }
  __syncthreads();
  const double xa = block_sum(va, red);
  __syncthreads();
  const double xb = block_sum(vb, red);
  if (threadIdx.x == 0) {
    *ta = xa;
    *tb = xb;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

#define GRID_STRIDE(i, n) \
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// The vector kernels of an iteration give each thread kU elements per pass, one grid apart (so each
// warp's accesses stay coalesced), and load all of them before any arithmetic: with one element per
// pass a warp had one or two loads in flight, and these kernels ran at 1-2 TB/s, latency-bound.
// Inside, the u-th element of the pass is i = base + u * gstride (valid while i < n).
constexpr int kU = 4;
// Element arithmetic and per-thread partial sums of the iteration kernels: FP32 for FP32 vectors (the
// inner solves of iterative refinement, which aim at 1e-4), FP64 otherwise; the block and grid sums are
// FP64 either way.  FP64 arithmetic and FP32-FP64 conversions run far below the FP32 rate here, and in
// FP64 they made the FP32 update kernel 3x slower than its memory traffic.
template <typename T>
using acc_t = typename std::conditional<sizeof(T) == 4, float, double>::type;
#define GRID_STRIDE_U(base, n)                                                                              \
  for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x, gstride = (size_t)gridDim.x * blockDim.x; \
       base < (n); base += kU * gstride)

// r = f - (sigma x + s q) (q = A x when use_x); rr = r.r, fnorm2 = f.f; sets tol2, done; r32 (may be
// null): an FP32 copy of r for the preconditioner
template <typename T>
__global__ void k_cg_init(const T* __restrict__ f, const T* __restrict__ x, const T* __restrict__ q, T* r, size_t n,
                          double* partials, CgState* S, double rtol, int use_x, float* __restrict__ r32) {
  double a = 0.0, b = 0.0;
  const double sg = S->sigma, sc = S->s;
  GRID_STRIDE(i, n) {
    const double fi = (double)f[i];
    double ri = fi;
    if (use_x) ri = fi - (sg * (double)x[i] + sc * (double)q[i]);
    const T rt = (T)ri;
    r[i] = rt;
    if (r32) r32[i] = (float)rt;
    a += (double)rt * (double)rt;
    b += fi * fi;
  }
  double ta, tb;
  if (grid_sum2(a, b, partials, &S->counter, &ta, &tb)) {
    S->rr = ta;
    S->fnorm2 = tb;
    S->tol2 = rtol * rtol * tb;
    S->iters = 0;
    S->status = FRLAP_OK;
    S->done = 0;
    if (!isfinite(ta) || !isfinite(tb)) {
      S->status = FRLAP_ENAN;
      S->done = 1;
    } else if (ta <= S->tol2) {
      S->done = 1;
    }
  }
}

// p = z (the preconditioner output zp, or r itself), rz = r.z
template <typename T, typename TP>
__global__ void k_pcg_start(const T* __restrict__ r, const TP* __restrict__ zp, T* p, size_t n, double* partials,
                            CgState* S) {
  using A = acc_t<T>;
  A a = 0;
  GRID_STRIDE_U(b0, n) {
    T rv[kU], zv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        rv[u] = r[i];
        zv[u] = zp ? (T)zp[i] : rv[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        p[i] = zv[u];
        a += (A)rv[u] * (A)zv[u];
      }
    }
  }
  double ta, tb;
  if (grid_sum2((double)a, 0.0, partials, &S->counter, &ta, &tb)) {
    S->rz = ta;
    if (zp && !(ta > 0.0) && !S->done) {
      S->status = isfinite(ta) ? FRLAP_EBREAKDOWN : FRLAP_ENAN;
      S->done = 1;
    }
  }
}

// q <- sigma p + s q ; pq = p . q ; alpha = rz / pq (breakdown if pq <= 0)
template <typename T>
__global__ void k_cg_pq(const T* __restrict__ p, T* q, size_t n, double* partials, CgState* S) {
  if (S->done) return;
  using A = acc_t<T>;
  const A sg = (A)S->sigma, sc = (A)S->s;
  const bool plain = S->sigma == 0.0 && S->s == 1.0;  // B = A (the Poisson problem): q is already B p
  A a = 0;
  GRID_STRIDE_U(b0, n) {
    T pv[kU], qv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        pv[u] = p[i];
        qv[u] = q[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        const A pi = (A)pv[u];
        T qi = qv[u];
        if (!plain) {
          qi = (T)(sg * pi + sc * (A)qi);
          q[i] = qi;
        }
        a += pi * (A)qi;
      }
    }
  }
  double ta, tb;
  if (grid_sum2((double)a, 0.0, partials, &S->counter, &ta, &tb)) {
    S->pq = ta;
    if (!(ta > 0.0) || !isfinite(ta)) {
      S->status = isfinite(ta) ? FRLAP_EBREAKDOWN : FRLAP_ENAN;
      S->done = 1;
    } else {
      S->alpha = S->rz / ta;
    }
  }
}

// x += alpha p ; r -= alpha q ; rr = r.r ; convergence test.  Without a preconditioner also
// beta = rr_new / rr_old (z = r).  With one, beta is formed after the preconditioner solve.
// r32 (may be null): an FP32 copy of the new r for the preconditioner
template <typename T>
__global__ void k_cg_update(T* x, T* r, const T* __restrict__ p, const T* __restrict__ q, size_t n,
                            double* partials, CgState* S, int maxit, int precond, float* __restrict__ r32) {
  if (S->done) return;
  using A = acc_t<T>;
  const A al = (A)S->alpha;
  A a = 0;
  GRID_STRIDE_U(b0, n) {
    T xv[kU], rv[kU], pv[kU], qv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        xv[u] = x[i];
        rv[u] = r[i];
        pv[u] = p[i];
        qv[u] = q[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        x[i] = (T)((A)xv[u] + al * (A)pv[u]);
        const T ri = (T)((A)rv[u] - al * (A)qv[u]);
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        a += (A)ri * (A)ri;
      }
    }
  }
  double ta, tb;
  if (grid_sum2((double)a, 0.0, partials, &S->counter, &ta, &tb)) {
    if (!precond) {
      S->beta = ta / S->rz;
      S->rz = ta;
    }
    S->rr = ta;
    S->iters += 1;
    if (!isfinite(ta)) {
      S->status = FRLAP_ENAN;
      S->done = 1;
    } else if (ta <= S->tol2) {
      S->done = 1;
    } else if (S->iters >= maxit) {
      S->status = FRLAP_ENOCONV;
      S->done = 1;
    }
  }
}

// after z = M^-1 r (the preconditioner output zp): rz_new = r.z, zq = z.q;
// flexible (Polak-Ribiere) beta = z.(r_new - r_old) / rz_old = -alpha zq / rz_old
template <typename T, typename TP>
__global__ void k_pcg_beta(const T* __restrict__ r, const TP* __restrict__ zp, const T* __restrict__ q, size_t n,
                           double* partials, CgState* S) {
  if (S->done) return;
  using A = acc_t<T>;
  A a = 0, b = 0;
  GRID_STRIDE_U(b0, n) {
    T zv[kU], rv[kU], qv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        zv[u] = (T)zp[i];
        rv[u] = r[i];
        qv[u] = q[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        a += (A)rv[u] * (A)zv[u];
        b += (A)zv[u] * (A)qv[u];
      }
    }
  }
  double ta, tb;
  if (grid_sum2((double)a, (double)b, partials, &S->counter, &ta, &tb)) {
    if (!(ta > 0.0) || !isfinite(ta)) {
      S->status = isfinite(ta) ? FRLAP_EBREAKDOWN : FRLAP_ENAN;
      S->done = 1;
    } else {
      S->beta = -S->alpha * tb / S->rz;
      S->rz = ta;
    }
  }
}

// p = z + beta p (z: the preconditioner output, or r itself)
template <typename T, typename TZ>
__global__ void k_cg_dir(const TZ* __restrict__ z, T* p, size_t n, const CgState* S) {
  if (S->done) return;
  using A = acc_t<T>;
  const A b = (A)S->beta;
  GRID_STRIDE_U(b0, n) {
    TZ zv[kU];
    T pv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) {
        zv[u] = z[i];
        pv[u] = p[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < n) p[i] = (T)((A)zv[u] + b * (A)pv[u]);
    }
  }
}


__global__ void k_set_state(CgState* S, double sigma, double s) {
  S->sigma = sigma;
  S->s = s;
  S->counter = 0u;
  S->done = 0;
  S->status = FRLAP_OK;
  S->iters = 0;
  S->passes = 0u;
}

// loop control of the graph-launched CG: another pass while the solve runs (bounded)
__global__ void k_cg_control(CgState* S, unsigned max_passes, cudaGraphConditionalHandle h) {
  const unsigned c = S->passes + 1u;
  S->passes = c;
  cudaGraphSetConditional(h, (!S->done && c < max_passes) ? 1u : 0u);
}

// true residual norms: out[0] = ||f - (sigma x + s q)||^2, out[1] = ||f||^2
__global__ void k_resid(const double* __restrict__ f, const double* __restrict__ x, const double* __restrict__ q,
                        size_t n, double sigma, double s, double* partials, unsigned* counter, double* out,
                        double* rvec, double* rnorm_scale) {
  double a = 0.0, b = 0.0;
  GRID_STRIDE(i, n) {
    const double ri = f[i] - (sigma * x[i] + s * q[i]);
    if (rvec) rvec[i] = ri;
    a += ri * ri;
    b += f[i] * f[i];
  }
  double ta, tb;
  if (grid_sum2(a, b, partials, counter, &ta, &tb)) {
    out[0] = ta;
    out[1] = tb;
    if (rnorm_scale) *rnorm_scale = sqrt(ta);
  }
}

// r32 = r / scale (FP32 right-hand side of an inner solve), d32 = 0
__global__ void k_to_f32(const double* __restrict__ r, const double* scale, float* r32, float* d32, size_t n) {
  const double sc = *scale;
  const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    r32[i] = (float)(r[i] * inv);
    d32[i] = 0.0f;
  }
}

// x += scale * d32
__global__ void k_correct(double* x, const float* __restrict__ d32, const double* scale, size_t n) {
  const double sc = *scale;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] += sc * (double)d32[i];
}

// Crank-Nicolson right-hand side of the paper's model for ubar = u + 1 (eqs. AC-1, AC-2):
// ubar - tau/2 A ubar - tau delta^-alpha u (u^2 - 1), u = ubar - 1
__global__ void k_cn_rhs(const double* __restrict__ ub, const double* __restrict__ aub, double* rhs, size_t n,
                         double tau, double kdel) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double b = ub[i], u = b - 1.0;
    rhs[i] = b - 0.5 * tau * aub[i] - tau * kdel * u * (u * u - 1.0);
  }
}

// out = scale * sum x, by one CTA in a fixed order (deterministic)
__global__ void k_sum_one_block(const double* __restrict__ x, size_t n, double scale, double* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) v += x[i];
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) *out = scale * t;
}

// *out = max_i |x_i| as the bit pattern of a non-negative double (whose unsigned order is the
// numeric order), or the pattern of a quiet NaN if any x_i is not finite; *out must start at 0.
// No squares are formed, so no value of x can overflow it.
__global__ void k_maxabs(const double* __restrict__ x, size_t n, unsigned long long* out) {
  double m = 0.0;
  bool bad = false;
  GRID_STRIDE(i, n) {
    const double v = fabs(x[i]);
    bad |= !isfinite(v);
    m = v > m ? v : m;
  }
  unsigned long long b = bad ? 0x7ff8000000000000ull : (unsigned long long)__double_as_longlong(m);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_down_sync(0xffffffffu, b, o);
    b = t > b ? t : b;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

// dst = 2^e src (exact in FP64 away from overflow and subnormals; dst may equal src)
__global__ void k_scale_pow2(const double* src, double* dst, size_t n, int e) {
  GRID_STRIDE(i, n) dst[i] = ldexp(src[i], e);
}

// Allen-Cahn right-hand side u + tau (u - u^3)
__global__ void k_ac_rhs(const double* __restrict__ u, double* rhs, size_t n, double tau) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = u[i];
    rhs[i] = v + tau * (v - v * v * v);
  }
}

size_t vec_bytes(const Plan& p, int eb) { return align256(p.M * (size_t)eb); }

}  // namespace

// the apply of a CG in precision T: FP32 vectors through the FP32 engine, FP64
// vectors through the plan's FP64 engine (native or double-float)
template <typename T>
static cudaError_t apply_T(const Plan& p, const T* u, T* y, void* work, cudaStream_t s, const int* skip) {
  if constexpr (sizeof(T) == 8) return apply64(p, u, y, work, s, skip);
  else return apply_launch<float>(p, u, y, work, s, skip);
}

// The residuals f - B x that restart a solve or decide its convergence.  The iterations may run
// on double-float (48-bit products, 5.6x faster than native FP64), but a residual computed with it
// carries the forward transforms' rounding times up to lambda_max (about 5e-15 lambda_max ||x||),
// which at 2047^2 already sits near 1e-10 ||f||.  So the forward transforms of a residual run in
// native FP64: on double-float plans the hybrid apply (FP64 forward, double-float inverse
// transforms, apply_hyb.cu), as accurate as native FP64 near a solution and 1.7x faster; native FP64
// throughout on F64 plans and on plans with a split middle stage.  A restart from such a residual
// removes the recurrence's drift, as in iterative refinement.
template <typename T>
static cudaError_t apply_residual(const Plan& p, const T* u, T* y, void* work, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    if (p.df64) {
      const cudaError_t e = apply_residual_hyb(p, u, y, work, s);
      if (e != cudaErrorNotSupported) return e;
    }
    return apply_launch<double>(p, u, y, work, s, nullptr);
  } else {
    return apply_launch<float>(p, u, y, work, s, nullptr);
  }
}

// workspace of one (P)CG solve in precision T:
// [apply work T][apply work FP32 (precond, T = double)][r][p][q][z][r32][z32][partials][state]
size_t cg_work_bytes(const Plan& p, int eb) {
  size_t b = apply_work_bytes(p, eb) + 4 * vec_bytes(p, eb) + 2 * vec_bytes(p, 4) +
             align256(2 * kBlocks * sizeof(double)) + align256(sizeof(CgState));
  if (eb == 8) b += apply_work_bytes(p, 4);
  return b;
}

struct CgBufs {
  void* awork;
  void* awork32;
  void* r;
  void* p;
  void* q;
  void* z;
  float* r32;
  float* z32;
  double* partials;
  CgState* S;
};

static CgBufs carve(const Plan& p, void* work, int eb) {
  CgBufs b;
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  b.awork = w;
  w += apply_work_bytes(p, eb);
  b.awork32 = nullptr;
  if (eb == 8) {
    b.awork32 = w;
    w += apply_work_bytes(p, 4);
  }
  b.r = w;
  w += vec_bytes(p, eb);
  b.p = w;
  w += vec_bytes(p, eb);
  b.q = w;
  w += vec_bytes(p, eb);
  b.z = w;
  w += vec_bytes(p, eb);
  b.r32 = reinterpret_cast<float*>(w);
  w += vec_bytes(p, 4);
  b.z32 = reinterpret_cast<float*>(w);
  w += vec_bytes(p, 4);
  b.partials = reinterpret_cast<double*>(w);
  w += align256(2 * kBlocks * sizeof(double));
  b.S = reinterpret_cast<CgState*>(w);
  return b;
}

// z32 = M^-1 r: one FP32 apply with the preconditioner symbol mu (skipped once done); odd: mu is a
// multiplier in the sine basis (applied on odd extensions)
template <typename T>
static cudaError_t precondition(const Plan& p, const CgBufs& b, const float* mu, bool odd, cudaStream_t st) {
  const float* src;
  if constexpr (sizeof(T) == 8) {
    src = b.r32;  // written with r by k_cg_init / k_cg_update
    return apply_launch<float>(p, src, b.z32, b.awork32, st, &b.S->done, nullptr, mu, odd);
  } else {
    src = reinterpret_cast<const float*>(b.r);
    return apply_launch<float>(p, src, b.z32, b.awork, st, &b.S->done, nullptr, mu, odd);
  }
}

// (Flexible) PCG on B x = f, B = sigma I + s A, in precision T; x holds x0 on entry.
// mu = FP32 preconditioner symbol (octant) or nullptr for plain CG.
template <typename T>
static frlap_status run_cg(const Plan& p, const T* f, T* x, double sigma, double s, double rtol, int maxit,
                           int use_x0, const float* mu, bool odd, void* work, cudaStream_t st, CgState* hS,
                           T* snap = nullptr, int nsnap = 0) {
  const CgBufs b = carve(p, work, sizeof(T));
  T* r = reinterpret_cast<T*>(b.r);
  T* pv = reinterpret_cast<T*>(b.p);
  T* q = reinterpret_cast<T*>(b.q);
  CgState* S = b.S;
  const size_t n = p.M;
  k_set_state<<<1, 1, 0, st>>>(S, sigma, s);
  FRLAP_LAUNCH_CHECK("k_set_state");
  if (use_x0) {
    // use_x0 = 1: the plan's engine; 2: native FP64 (a restart, which must see the true residual)
    cudaError_t e = use_x0 == 2 ? apply_residual<T>(p, x, q, b.awork, st) : apply_T<T>(p, x, q, b.awork, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "apply (initial residual)");
  }
  float* r32 = (mu && sizeof(T) == 8) ? b.r32 : nullptr;  // FP64 solves hand the preconditioner an FP32 r
  k_cg_init<T><<<vgrid(n), kThreads, 0, st>>>(f, x, q, r, n, b.partials, S, rtol, use_x0, r32);
  FRLAP_LAUNCH_CHECK("k_cg_init");
  if (mu) {
    cudaError_t e = precondition<T>(p, b, mu, odd, st);
    if (e != cudaSuccess) return cuda_fail(e, "preconditioner");
    k_pcg_start<T, float><<<vgrid(n), kThreads, 0, st>>>(r, b.z32, pv, n, b.partials, S);
  } else {
    k_pcg_start<T, T><<<vgrid(n), kThreads, 0, st>>>(r, nullptr, pv, n, b.partials, S);
  }
  FRLAP_LAUNCH_CHECK("k_pcg_start");
  if (snap && nsnap > 0) FRLAP_CUDA_TRY(cudaMemcpyAsync(snap, x, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  const int* done = &S->done;
  // one iteration on stream `ss`; the snapshot copy (training pairs) needs the host's count
  auto iteration = [&](cudaStream_t ss, int it) -> cudaError_t {
    cudaError_t e = apply_T<T>(p, pv, q, b.awork, ss, done);
    if (e != cudaSuccess) return e;
    k_cg_pq<T><<<vgrid(n), kThreads, 0, ss>>>(pv, q, n, b.partials, S);
    k_cg_update<T><<<vgrid(n), kThreads, 0, ss>>>(x, r, pv, q, n, b.partials, S, maxit, mu != nullptr, r32);
    if (snap && it + 1 < nsnap) {
      e = cudaMemcpyAsync(snap + (size_t)(it + 1) * n, x, n * sizeof(T), cudaMemcpyDeviceToDevice, ss);
      if (e != cudaSuccess) return e;
    }
    if (mu) {
      e = precondition<T>(p, b, mu, odd, ss);
      if (e != cudaSuccess) return e;
      k_pcg_beta<T, float><<<vgrid(n), kThreads, 0, ss>>>(r, b.z32, q, n, b.partials, S);
      k_cg_dir<T, float><<<vgrid(n), kThreads, 0, ss>>>(b.z32, pv, n, S);
    } else {
      k_cg_dir<T, T><<<vgrid(n), kThreads, 0, ss>>>(r, pv, n, S);
    }
    return cudaGetLastError();
  };
  // The first iterations run as plain launches; when the solve goes on (and takes no
  // snapshots), the rest runs as one CUDA-graph launch: a conditional WHILE node whose body
  // is one iteration plus k_cg_control, which ends the loop once the update kernel has set
  // `done` (converged, breakdown or maxit), and after at most maxit + 2 passes regardless.
  const int chunk = 8;
  int launched = 0;
  while (true) {
    for (int c = 0; c < chunk; ++c) {
      cudaError_t e = iteration(st, launched + c);
      if (e != cudaSuccess) return cuda_fail(e, "CG iteration");
    }
    launched += chunk;
    FRLAP_CUDA_TRY(cudaMemcpyAsync(hS, S, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    FRLAP_CUDA_TRY(cudaStreamSynchronize(st));
    if (hS->done) return FRLAP_OK;
    if (launched > maxit + chunk) return FRLAP_OK;  // cannot happen: the update kernel stops at maxit
    if (!snap) break;
  }
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  cudaGraphConditionalHandle h;
  if (e == cudaSuccess) e = cudaGraphCreate(&graph, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t eb = iteration(cs, launched);
    if (eb == cudaSuccess) {
      k_cg_control<<<1, 1, 0, cs>>>(S, capped_passes((unsigned)maxit + 2u), h);
      eb = cudaGetLastError();
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (eb != cudaSuccess) e = eb;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hS, S, sizeof(CgState), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_fail(e, "graph-launched CG iterations");
  if (!hS->done) {  // the loop ran out of passes (a limit set by frlap_set_loop_pass_limit)
    hS->status = FRLAP_ETIMEOUT;
    hS->done = 1;
  }
  return FRLAP_OK;
}

// true relative residual ||f - B x|| / ||f|| in FP64 (uses the apply work and q buffer)
// (zero_x: x is known to be zero, so A x = 0 needs no apply)
static frlap_status true_residual(const Plan& p, const double* f, const double* x, double sigma, double s,
                                  void* work, cudaStream_t st, double* relres, double* rvec,
                                  double* rnorm_dev, bool native = true, bool zero_x = false) {
  const CgBufs b = carve(p, work, 8);
  double* q = reinterpret_cast<double*>(b.q);
  CgState* S = b.S;
  // the reduction ticket must start at zero (this workspace may not have run a CG yet)
  FRLAP_CUDA_TRY(cudaMemsetAsync(&S->counter, 0, sizeof(unsigned), st));
  cudaError_t e = zero_x   ? cudaMemsetAsync(q, 0, p.M * sizeof(double), st)
                  : native ? apply_residual<double>(p, x, q, b.awork, st)
                           : apply64(p, x, q, b.awork, st, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "apply (true residual)");
  double* out = &S->alpha;  // reuse two scalar slots (alpha, beta) for the norms
  k_resid<<<vgrid(p.M), kThreads, 0, st>>>(f, x, q, p.M, sigma, s, b.partials, &S->counter, out, rvec, rnorm_dev);
  FRLAP_LAUNCH_CHECK("k_resid");
  double h[2];
  FRLAP_CUDA_TRY(cudaMemcpyAsync(h, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  FRLAP_CUDA_TRY(cudaStreamSynchronize(st));
  *relres = (h[1] > 0.0) ? sqrt(h[0] / h[1]) : 0.0;
  return FRLAP_OK;
}

// r = f - A x (r may be null) and ||r|| / ||f||, with the apply that decides convergence
frlap_status residual_impl(const Plan& p, const double* f, const double* x, double* r, double* relres, void* work,
                           cudaStream_t st) {
  return true_residual(p, f, x, 0.0, 1.0, work, st, relres, r, nullptr, true);
}

// E[j] <- xs - E[j]
__global__ void k_err_from_snap(double* E, const double* __restrict__ xs, size_t n) {
  GRID_STRIDE(i, n) E[i] = xs[i] - E[i];
}

frlap_status cg_pairs_impl(const Plan& p, const double* f, int K, double rtol, double* E, double* R, int* npairs,
                           void* work, cudaStream_t st) {
  CgBufs b = carve(p, work, 8);
  double* x = reinterpret_cast<double*>(b.z);  // the solution lives in the (unused) z buffer
  FRLAP_CUDA_TRY(cudaMemsetAsync(x, 0, p.M * sizeof(double), st));
  CgState hS;
  frlap_status rc = run_cg<double>(p, f, x, 0.0, 1.0, rtol, 1000000, 0, nullptr, false, work, st, &hS, E, K);
  if (rc != FRLAP_OK) return rc;
  if (hS.status != FRLAP_OK) return fail((frlap_status)hS.status, "CG for the training pairs stopped early");
  // x_0 .. x_{iters-1}: the last iterate is the solution itself (zero error) and is left out
  const int np = hS.iters < K ? hS.iters : K;
  for (int j = 0; j < np; ++j) {
    double* Ej = E + (size_t)j * p.M;
    k_err_from_snap<<<vgrid(p.M), kThreads, 0, st>>>(Ej, x, p.M);
    FRLAP_LAUNCH_CHECK("k_err_from_snap");
    cudaError_t e = apply64(p, Ej, R + (size_t)j * p.M, b.awork, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "apply (training pairs)");
  }
  FRLAP_CUDA_TRY(cudaStreamSynchronize(st));
  if (npairs) *npairs = np;
  return FRLAP_OK;
}

size_t ir_work_bytes(const Plan& p) {
  // FP64 CG state (for the outer residual) + FP32 CG workspace + r64 + r32, d32
  return cg_work_bytes(p, 8) + cg_work_bytes(p, 4) + vec_bytes(p, 8) + 2 * vec_bytes(p, 4) + 256;
}

// CG workspace, two vectors (right-hand side, A ubar) and a slot for the mass of the Crank-Nicolson model
// CG workspace, two FP64 vectors, the shifted sine-basis multiplier (FP32 octant), the mass slot
size_t ac_work_bytes(const Plan& p) {
  return cg_work_bytes(p, 8) + 2 * vec_bytes(p, 8) + align256(p.lam_count * sizeof(float)) + 256;
}

// Workspace of frlap_pcg_solve: the CG or refinement workspace, and on double-float plans the
// scaled right-hand side (one FP64 vector) behind it.
static size_t pcg_base_bytes(const Plan& p) {
  if (p.prec == FRLAP_MIXED || p.prec == FRLAP_MIXED_DF64) return ir_work_bytes(p);
  return cg_work_bytes(p, p.prec == FRLAP_F32 ? 4 : 8);
}
size_t pcg_work_bytes(const Plan& p) { return pcg_base_bytes(p) + (p.df64 ? vec_bytes(p, 8) : 0); }

static frlap_status pcg_solve_core(const Plan& p, const double* f, double* x, double rtol, int maxit, int solver,
                                   const float* mu, double inner_rtol, int* iters, double* relres, void* work,
                                   cudaStream_t st, bool x0_zero);

// max |f_i| and max |x0_i| first (one synchronisation): a zero x0 needs no apply for the initial
// residual (r = f), and on double-float plans, which keep FP32's exponent range, the system is
// solved for 2^-e f with 2^e the power of two at or below max |f_i| (and x0 scaled alike), and x
// is scaled back: every scaling is by a power of two, exact in FP64, so the solve is the same up
// to the double-float range it now stays inside.
frlap_status pcg_solve_impl(const Plan& p, const double* f, double* x, double rtol, int maxit, int solver,
                            const float* mu, double inner_rtol, int* iters, double* relres, void* work,
                            cudaStream_t st) {
  const CgBufs b = carve(p, work, 8);
  unsigned long long* slot = reinterpret_cast<unsigned long long*>(&b.S->alpha);  // alpha, beta: two slots
  FRLAP_CUDA_TRY(cudaMemsetAsync(slot, 0, 2 * sizeof(unsigned long long), st));
  k_maxabs<<<vgrid(p.M), kThreads, 0, st>>>(f, p.M, slot);
  k_maxabs<<<vgrid(p.M), kThreads, 0, st>>>(x, p.M, slot + 1);
  FRLAP_LAUNCH_CHECK("k_maxabs");
  unsigned long long bits[2] = {0ull, 0ull};
  FRLAP_CUDA_TRY(cudaMemcpyAsync(bits, slot, sizeof(bits), cudaMemcpyDeviceToHost, st));
  FRLAP_CUDA_TRY(cudaStreamSynchronize(st));
  double fmax = 0.0, xmax = 0.0;
  memcpy(&fmax, &bits[0], sizeof(fmax));
  memcpy(&xmax, &bits[1], sizeof(xmax));
  const bool x0_zero = xmax == 0.0;  // false for a non-finite x0 (its pattern is a NaN)
  if (!p.df64)
    return pcg_solve_core(p, f, x, rtol, maxit, solver, mu, inner_rtol, iters, relres, work, st, x0_zero);
  if (!isfinite(fmax)) return fail(FRLAP_ENAN, "non-finite value in the right-hand side");
  const int e = fmax > 0.0 ? ilogb(fmax) : 0;
  if (e == 0)
    return pcg_solve_core(p, f, x, rtol, maxit, solver, mu, inner_rtol, iters, relres, work, st, x0_zero);
  double* fs = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(work) + pcg_base_bytes(p));
  k_scale_pow2<<<vgrid(p.M), kThreads, 0, st>>>(f, fs, p.M, -e);
  if (!x0_zero) k_scale_pow2<<<vgrid(p.M), kThreads, 0, st>>>(x, x, p.M, -e);
  FRLAP_LAUNCH_CHECK("k_scale_pow2");
  const frlap_status rc = pcg_solve_core(p, fs, x, rtol, maxit, solver, mu, inner_rtol, iters, relres, work, st,
                                         x0_zero);
  k_scale_pow2<<<vgrid(p.M), kThreads, 0, st>>>(x, x, p.M, e);
  cudaError_t ce = cudaGetLastError();
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "k_scale_pow2 (solution)");
  return rc;
}

static frlap_status pcg_solve_core(const Plan& p, const double* f, double* x, double rtol, int maxit, int solver,
                                   const float* mu, double inner_rtol, int* iters, double* relres, void* work,
                                   cudaStream_t st, bool x0_zero) {
  CgState hS;
  const bool odd = mu != nullptr && mu == p.mu_tau;  // the sine-basis multiplier runs on odd extensions
  if (solver == FRLAP_SOLVE_CG) {
    // CG, then the true residual; if rounding left the true residual above rtol while the
    // recursive one met it, restart from the current x (at most 4 restarts, within maxit).
    // A restart aims at rtol / 10: it starts from the native FP64 residual, so its own
    // recursive residual going well below rtol carries the true one below rtol too.
    int total = 0;
    double rel = 0.0;
    frlap_status rc = FRLAP_OK;
    for (int restart = 0; restart < 5; ++restart) {
      const double rt = restart == 0 ? rtol : 0.1 * rtol;
      const int use_x0 = restart > 0 ? 2 : x0_zero ? 0 : 1;
      rc = run_cg<double>(p, f, x, 0.0, 1.0, rt, maxit - total, use_x0, mu, odd, work, st, &hS);
      if (rc != FRLAP_OK) return rc;
      total += hS.iters;
      rc = true_residual(p, f, x, 0.0, 1.0, work, st, &rel, nullptr, nullptr);
      if (rc != FRLAP_OK) return rc;
      if (hS.status != FRLAP_OK || rel <= rtol || total >= maxit || hS.iters == 0) break;
    }
    if (iters) *iters = total;
    if (relres) *relres = rel;
    if (hS.status != FRLAP_OK) return fail((frlap_status)hS.status, "CG stopped early (see status code)");
    if (!(rel <= rtol)) return fail(FRLAP_ENOCONV, "true residual above rtol (rounding floor of the apply)");
    return FRLAP_OK;
  }
  // iterative refinement: x <- x + ||r|| * CG32(A, r/||r||)
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  void* work64 = w;
  w += cg_work_bytes(p, 8);
  void* work32 = w;
  w += cg_work_bytes(p, 4);
  double* r64 = reinterpret_cast<double*>(w);
  w += vec_bytes(p, 8);
  float* r32 = reinterpret_cast<float*>(w);
  w += vec_bytes(p, 4);
  float* d32 = reinterpret_cast<float*>(w);
  w += vec_bytes(p, 4);
  double* rnorm = reinterpret_cast<double*>(w);
  int total = 0;
  double rel = 0.0;
  const int max_outer = 60;
  // Outer residuals use the plan's FP64-side engine while far from rtol; from 1e-6 on (and to
  // decide convergence) the native FP64 engine computes them.
  double prev = 1.0;
  for (int outer = 0; outer <= max_outer; ++outer) {
    const bool native = prev <= 1e-6;
    frlap_status rc = true_residual(p, f, x, 0.0, 1.0, work64, st, &rel, r64, rnorm, native, outer == 0 && x0_zero);
    if (rc == FRLAP_OK && !native && rel <= 1e-6)
      rc = true_residual(p, f, x, 0.0, 1.0, work64, st, &rel, r64, rnorm, true);
    if (rc != FRLAP_OK) return rc;
    prev = rel;
    if (!isfinite(rel)) return fail(FRLAP_ENAN, "non-finite residual in iterative refinement");
    if (rel <= rtol || outer == max_outer || total >= maxit) break;
    k_to_f32<<<vgrid(p.M), kThreads, 0, st>>>(r64, rnorm, r32, d32, p.M);
    FRLAP_LAUNCH_CHECK("k_to_f32");
    rc = run_cg<float>(p, r32, d32, 0.0, 1.0, inner_rtol, maxit - total, 0, mu, odd, work32, st, &hS);
    if (rc != FRLAP_OK) return rc;
    total += hS.iters;
    if (hS.status == FRLAP_ENAN) return fail(FRLAP_ENAN, "non-finite value in the FP32 inner solve");
    k_correct<<<vgrid(p.M), kThreads, 0, st>>>(x, d32, rnorm, p.M);
    FRLAP_LAUNCH_CHECK("k_correct");
  }
  if (iters) *iters = total;
  if (relres) *relres = rel;
  if (!(rel <= rtol)) return fail(FRLAP_ENOCONV, "iterative refinement did not reach rtol");
  return FRLAP_OK;
}

// The paper's model (eqs. AC-1, AC-2; Crank-Nicolson in time, Sec. 5.4) for ubar = u + 1: per step
// rhs = (I - tau/2 A) ubar - tau delta^-alpha f(ubar - 1), then (I + tau/2 A) ubar' = rhs by CG from
// ubar; h_mass[step] = h^d sum ubar' if h_mass is given.
frlap_status allen_cahn_cn_impl(const Plan& p, double* ub, double tau, double delta, int nsteps, double rtol,
                                int* iters, double* h_mass, void* work, cudaStream_t st) {
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  void* cgw = w;
  w += cg_work_bytes(p, 8);
  double* rhs = reinterpret_cast<double*>(w);
  w += vec_bytes(p, 8);
  double* aub = reinterpret_cast<double*>(w);
  w += vec_bytes(p, 8);
  float* mu_b = reinterpret_cast<float*>(w);
  w += align256(p.lam_count * sizeof(float));
  double* dmass = reinterpret_cast<double*>(w);
  const float* mu = nullptr;
  if (p.mu_tau) {  // (I + tau/2 A) preconditioned in the sine basis
    FRLAP_CUDA_TRY(shifted_tau_launch(p, 1.0, 0.5 * tau, mu_b, st));
    mu = mu_b;
  }
  const CgBufs b = carve(p, cgw, 8);  // its apply workspace is free between the solves
  const double kdel = pow(delta, -p.alpha);
  const double hd = pow(p.h, (double)p.d);
  int total = 0;
  CgState hS;
  for (int step = 0; step < nsteps; ++step) {
    cudaError_t e = apply64(p, ub, aub, b.awork, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "apply (Crank-Nicolson right-hand side)");
    k_cn_rhs<<<vgrid(p.M), kThreads, 0, st>>>(ub, aub, rhs, p.M, tau, kdel);
    FRLAP_LAUNCH_CHECK("k_cn_rhs");
    frlap_status rc = run_cg<double>(p, rhs, ub, 1.0, 0.5 * tau, rtol, 100000, 1, mu, mu != nullptr, cgw, st, &hS);
    if (rc != FRLAP_OK) return rc;
    total += hS.iters;
    if (hS.status != FRLAP_OK) {
      if (iters) *iters = total;
      return fail((frlap_status)hS.status, "Allen-Cahn (Crank-Nicolson) CG solve stopped early");
    }
    if (h_mass) {
      k_sum_one_block<<<1, 1024, 0, st>>>(ub, p.M, hd, dmass);
      FRLAP_LAUNCH_CHECK("k_sum_one_block");
      FRLAP_CUDA_TRY(cudaMemcpyAsync(h_mass + step, dmass, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
  }
  if (h_mass) FRLAP_CUDA_TRY(cudaStreamSynchronize(st));
  if (iters) *iters = total;
  return FRLAP_OK;
}

frlap_status allen_cahn_impl(const Plan& p, double* u, double tau, double eps, int nsteps, double rtol,
                             int* iters, void* work, cudaStream_t st) {
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  void* cgw = w;
  w += cg_work_bytes(p, 8);
  double* rhs = reinterpret_cast<double*>(w);
  w += vec_bytes(p, 8);
  w += vec_bytes(p, 8);
  float* mu_b = reinterpret_cast<float*>(w);
  const float* mu = nullptr;
  if (p.mu_tau) {  // (I + tau eps^2 A) preconditioned in the sine basis
    FRLAP_CUDA_TRY(shifted_tau_launch(p, 1.0, tau * eps * eps, mu_b, st));
    mu = mu_b;
  }
  int total = 0;
  CgState hS;
  for (int step = 0; step < nsteps; ++step) {
    k_ac_rhs<<<vgrid(p.M), kThreads, 0, st>>>(u, rhs, p.M, tau);
    FRLAP_LAUNCH_CHECK("k_ac_rhs");
    frlap_status rc = run_cg<double>(p, rhs, u, 1.0, tau * eps * eps, rtol, 100000, 1, mu, mu != nullptr, cgw, st,
                                     &hS);
    if (rc != FRLAP_OK) return rc;
    total += hS.iters;
    if (hS.status != FRLAP_OK) {
      if (iters) *iters = total;
      return fail((frlap_status)hS.status, "Allen-Cahn CG solve stopped early");
    }
  }
  if (iters) *iters = total;
  return FRLAP_OK;
}

}  // namespace frlap
