// Coefficients a_k of the scheme (Sec. 2 eqs. amn, a00; Sec. 4 a_mns, a000), the
// real symbol of their circulant embedding, and FFT twiddle tables; all in FP64
// on the device.
//
// Quadrature (the paper leaves it open): every element integral
// w_k = int_{[k,k+1]^d} |xi|^-p dxi (h = 1, p = d + alpha - gamma) with k != 0 is a
// tensor Gauss-Legendre sum whose order falls with the element's distance from
// the singular point xi = 0; the origin element and the far field are reduced
// by splitting the cube into d pyramids (on each, one coordinate is the largest),
// which integrates the radial variable in closed form and leaves a smooth
// (d-1)-dimensional integral.  Gauss-Legendre nodes are computed on the device by
// Newton's method on the three-term Legendre recurrence.
#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "fft.cuh"

namespace frlap {

namespace {

// orders used by the element rule and by the pyramid integrals
constexpr int kNumQ = 6;
__constant__ int c_q[kNumQ] = {4, 5, 8, 14, 20, 32};
constexpr int kQTotal = 83;

// nodes on [0,1] and weights summing to 1, one thread per node
__global__ void k_gauss(double* nodes, double* weights) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kQTotal) return;
  int qi = 0;
  int off[kNumQ + 1] = {0, 4, 9, 17, 31, 51, 83};
  while (t >= off[qi + 1]) ++qi;
  const int q = c_q[qi];
  const int i = t - off[qi];
  double x = cos(M_PI * (i + 0.75) / (q + 0.5));
  double dP = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= q; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dP = q * (x * p1 - p0) / (x * x - 1.0);
    const double dx = p1 / dP;
    x -= dx;
    if (fabs(dx) < 1e-17) break;
  }
  {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= q; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dP = q * (x * p1 - p0) / (x * x - 1.0);
  }
  nodes[t] = 0.5 * (1.0 - x);
  weights[t] = 1.0 / ((1.0 - x * x) * dP * dP);  // (2/((1-x^2)P'^2)) / 2
}

__device__ __forceinline__ int q_index(int dist) {
  // Gauss-Legendre order for an element whose lower corner has max-norm dist >= 1;
  // the error decays like (2 dist)^(-2q)
  if (dist <= 2) return 4;   // 20 points
  if (dist <= 6) return 3;   // 14
  if (dist <= 24) return 2;  // 8
  if (dist <= 96) return 1;  // 5
  return 0;                  // 4
}

template <int D>
__global__ void k_element_weights(double* w, int N, double p, const double* __restrict__ gn,
                                  const double* __restrict__ gw) {
  const size_t total = (D == 2) ? (size_t)N * N : (size_t)N * N * N;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int k[3];
  size_t rest = e;
  for (int r = 0; r < D; ++r) {
    k[r] = (int)(rest % N);
    rest /= N;
  }
  // |xi|^-p and the tensor rule are symmetric under permutations of the coordinates, so
  // w_k = w_{sorted k}: only elements with k[0] <= k[1] (<= k[2]) are integrated here, and
  // k_fill_permuted copies them to the others (2D: half, 3D: a sixth of the work).
  for (int r = 0; r + 1 < D; ++r)
    if (k[r] > k[r + 1]) return;
  int dist = k[D - 1];
  if (dist == 0) return;  // origin element: k_pyramid
  const int qi = q_index(dist);
  int off[kNumQ + 1] = {0, 4, 9, 17, 31, 51, 83};
  const int q = off[qi + 1] - off[qi];
  const double* xn = gn + off[qi];
  const double* xw = gw + off[qi];
  const double mp = -0.5 * p;
  double acc = 0.0;
  if (D == 2) {
    for (int i = 0; i < q; ++i) {
      const double a = k[0] + xn[i];
      double s = 0.0;
      for (int j = 0; j < q; ++j) {
        const double b = k[1] + xn[j];
        s += xw[j] * pow(a * a + b * b, mp);
      }
      acc += xw[i] * s;
    }
  } else {
    for (int i = 0; i < q; ++i) {
      const double a = k[0] + xn[i];
      double s1 = 0.0;
      for (int j = 0; j < q; ++j) {
        const double b = k[1] + xn[j];
        const double ab = a * a + b * b;
        double s2 = 0.0;
        for (int l = 0; l < q; ++l) {
          const double c = k[2] + xn[l];
          s2 += xw[l] * pow(ab + c * c, mp);
        }
        s1 += xw[j] * s2;
      }
      acc += xw[i] * s1;
    }
  }
  w[e] = acc;
}

// w[e] = w[index of the sorted coordinates of element e], for every element whose coordinates are
// not in ascending order (k_element_weights integrated only the sorted ones)
template <int D>
__global__ void k_fill_permuted(double* w, int N) {
  const size_t total = (D == 2) ? (size_t)N * N : (size_t)N * N * N;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  int k[3] = {0, 0, 0};
  size_t rest = e;
  for (int r = 0; r < D; ++r) {
    k[r] = (int)(rest % N);
    rest /= N;
  }
  bool sorted = true;
  for (int r = 0; r + 1 < D; ++r) sorted = sorted && k[r] <= k[r + 1];
  if (sorted) return;
  // sort ascending (at most three entries)
  for (int i = 0; i < D; ++i)
    for (int j = 0; j + 1 < D - i; ++j)
      if (k[j] > k[j + 1]) {
        const int t = k[j];
        k[j] = k[j + 1];
        k[j + 1] = t;
      }
  size_t src = 0, stride = 1;
  for (int r = 0; r < D; ++r) {
    src += (size_t)k[r] * stride;
    stride *= N;
  }
  w[e] = w[src];
}

// pyramid reductions: out[0] = w_0 = d/(d-p) int_{[0,1]^(d-1)} (1+|s|^2)^(-p/2),
// out[1] = W_D2 = d N^-alpha / alpha int_{[0,1]^(d-1)} (1+|s|^2)^(-(d+alpha)/2)   (h = 1)
__global__ void k_pyramid(int d, double p, double alpha, int N, const double* __restrict__ gn,
                          const double* __restrict__ gw, double* out, double* w) {
  const int off = 51;  // offset of the 32-point rule in the node table
  const int q = 32;
  const int cnt = (d == 2) ? q : q * q;
  double s0 = 0.0, s1 = 0.0;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    double r2 = 1.0, wt;
    if (d == 2) {
      r2 += gn[off + t] * gn[off + t];
      wt = gw[off + t];
    } else {
      const int i = t / q, j = t % q;
      r2 += gn[off + i] * gn[off + i] + gn[off + j] * gn[off + j];
      wt = gw[off + i] * gw[off + j];
    }
    s0 += wt * pow(r2, -0.5 * p);
    s1 += wt * pow(r2, -0.5 * (d + alpha));
  }
  __shared__ double r0[256], r1[256];
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      r0[threadIdx.x] += r0[threadIdx.x + st];
      r1[threadIdx.x] += r1[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = d / (d - p) * r0[0];
    out[1] = d * pow((double)N, -alpha) / alpha * r1[0];
    w[0] = out[0];
  }
}

// a_k for k != 0 (scaled by h^-alpha) and the block partial sums of 2^(d-sigma) a_k
template <int D>
__global__ void k_assemble(const double* __restrict__ w, int N, double gamma, double hscale,
                           const double* __restrict__ pyr, double* coef, double* partial) {
  const int N1 = N + 1;
  const size_t total = (D == 2) ? (size_t)N1 * N1 : (size_t)N1 * N1 * N1;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (e < total) {
    int k[3] = {0, 0, 0};
    size_t rest = e;
    for (int r = 0; r < D; ++r) {
      k[r] = (int)(rest % N1);
      rest /= N1;
    }
    int ksum = 0, sigma = 0;
    double k2 = 0.0;
    for (int r = 0; r < D; ++r) {
      ksum += k[r];
      sigma += (k[r] == 0);
      k2 += (double)k[r] * k[r];
    }
    if (ksum > 0) {
      // W(T_k): elements k - e, e in {0,1}^D, inside [0, N-1]^D
      double WT = 0.0;
      for (int m = 0; m < (1 << D); ++m) {
        bool ok = true;
        size_t idx = 0, stride = 1;
        for (int r = 0; r < D; ++r) {
          const int kr = k[r] - ((m >> r) & 1);
          ok = ok && kr >= 0 && kr <= N - 1;
          idx += (size_t)(kr < 0 ? 0 : kr) * stride;
          stride *= N;
        }
        if (ok) WT += w[idx];
      }
      // origin correction: (c^gamma_k - 1) w_0 on the vertices of the origin element
      double kappa = 0.0;
      if (gamma == 2.0) {
        bool unit = true;
        for (int r = 0; r < D; ++r) unit = unit && k[r] <= 1;
        if (unit) kappa = (ksum == 1) ? ((D == 2) ? 1.0 : 5.0 / 3.0) : -1.0;
      }
      const double a = ldexp(1.0, sigma - D) / pow(k2, 0.5 * gamma) * (WT + kappa * pyr[0]);
      coef[e] = a * hscale;
      contrib = ldexp(a, D - sigma);
    }
  }
  // block reduction of the a_0 terms (h = 1 units)
  __shared__ double red[256];
  red[threadIdx.x] = contrib;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// a_0 = -(sum of partials) - 2^d W_D2, scaled; one block, fixed summation order
__global__ void k_diag(const double* __restrict__ partial, int nparts, int d, const double* __restrict__ pyr,
                       double hscale, double* coef) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) coef[0] = (-red[0] - ldexp(pyr[1], d)) * hscale;
}

// symbol octant initialisation: t_k = -c a_k for k_r <= n_r - 1, 0 elsewhere in [0, P_r/2]
__global__ void k_sym_init(const double* __restrict__ coef, int Nmax, int d, int nx, int ny, int nz, int Hx1,
                           int Hy1, int Hz1, double c, double* lam) {
  const size_t total = (size_t)Hx1 * Hy1 * Hz1;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int kx = (int)(e % Hx1);
  const int ky = (int)((e / Hx1) % Hy1);
  const int kz = (int)(e / ((size_t)Hx1 * Hy1));
  double v = 0.0;
  if (kx <= nx - 1 && ky <= ny - 1 && kz <= nz - 1) {
    const size_t N1 = (size_t)Nmax + 1;
    const size_t ci = (d == 2) ? (size_t)ky * N1 + kx : ((size_t)kz * N1 + ky) * N1 + kx;
    v = -c * coef[ci];
  }
  lam[e] = v;
}

// even DFT along one axis of the octant: for every line (stride `stride`, P/2+1 entries)
// g(j) = sum_{k = -P/2+1}^{P/2} t(|k|) e^{-2 pi i j k / P}, j = 0..P/2 (real, since t is even)
__global__ void __launch_bounds__(512) k_sym_axis(double* lam, size_t nlines, int logP, size_t stride, size_t inner, int TL,
                           const double2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* smem = reinterpret_cast<double2*>(smem_raw);
  const int P = 1 << logP, G = P >> 4, H = P / 2;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const size_t line = (size_t)blockIdx.x * TL + l;
  const bool valid = line < nlines;
  // line index -> base offset: lines enumerate (outer, inner) with `inner` lines per outer slab
  const size_t li = valid ? line : 0;
  const size_t base = (li / inner) * inner * (size_t)(H + 1) + (li % inner);
  double2* buf = smem + (size_t)l * sline(P);
  for (int j = lane; j < P; j += G) {
    const int kf = min(j, P - j);
    buf[spad(j)] = make_double2(valid ? lam[base + (size_t)kf * stride] : 0.0, 0.0);
  }
  __syncthreads();
  fft_line<double, -1>(buf, logP, lane, tw, logP);
  if (valid)
    for (int j = lane; j <= H; j += G) lam[base + (size_t)j * stride] = buf[spad(j)].x;
}

// k_sym_axis for P = 2 L points with L = 8192, the longest line the FFT kernels hold: one line per
// CTA, split by output parity.  With t the P-periodic even extension of the line's generator,
//   g(2m)   = sum_{k<L} (t_k + t_{k+L}) W_L^{km},
//   g(2m+1) = sum_{k<L} (t_k - t_{k+L}) W_P^k W_L^{km},
// two L-point transforms (the P-point table serves them, see fft_line).  The line's P/2 + 1 input
// values are first copied to shared memory, since the outputs overwrite them in place.
__global__ void __launch_bounds__(512) k_sym_axis_split(double* lam, size_t nlines, size_t stride, size_t inner,
                                                        const double2* __restrict__ tw) {
  constexpr int logL = 13, L = 1 << logL, P = 2 * L, H = L, G = L >> 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  double* t = reinterpret_cast<double*>(smem_raw + (size_t)sline(L) * sizeof(double2));  // t_0 .. t_{P/2}
  const int lane = threadIdx.x;
  const size_t line = blockIdx.x;
  if (line >= nlines) return;
  const size_t base = (line / inner) * inner * (size_t)(H + 1) + (line % inner);
  for (int j = lane; j <= H; j += G) t[j] = lam[base + (size_t)j * stride];
  __syncthreads();
  for (int parity = 0; parity < 2; ++parity) {
    for (int k = lane; k < L; k += G) {
      // t_{k + L} = t_{P - k - L} = t_{L - k} by the even extension (k + L <= P - 1)
      const double a = t[k], b = t[L - k];
      buf[spad(k)] = parity == 0 ? make_double2(a + b, 0.0) : cmul(make_double2(a - b, 0.0), tw[k]);
    }
    __syncthreads();
    fft_line<double, -1>(buf, logL, lane, tw, logL + 1);
    // outputs j = 2m + parity <= P/2, m < L
    for (int m = lane; m < L; m += G) {
      const int j = 2 * m + parity;
      if (j <= H) lam[base + (size_t)j * stride] = buf[spad(m)].x;
    }
    __syncthreads();
  }
}

__global__ void k_scale_copy(double* lam64, float* lam32, size_t n, double s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = lam64[i] * s;
  lam64[i] = v;
  if (lam32) lam32[i] = (float)v;
}

__global__ void k_twiddle(int P, double2* tw64, float2* tw32) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= P) return;
  double s, c;
  sincospi(2.0 * m / P, &s, &c);
  tw64[m] = make_double2(c, -s);
  if (tw32) tw32[m] = make_float2((float)c, (float)-s);
}

// radix-16 stage entries of the table (layout: twiddle_entries), gathered from its first P
__global__ void k_twiddle_stage(int P, int logP, double2* tw64, float2* tw32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 15 * (P / 8 - 1)) return;
  int logNs = 0;
  while (15 * ((2 << logNs) - 1) <= i) ++logNs;
  const int Ns = 1 << logNs, off = i - 15 * (Ns - 1);
  const int r = off / Ns + 1, k = off % Ns;
  const double2 w = tw64[(r * k) << (logP - logNs - 4)];
  tw64[P + i] = w;
  if (tw32) tw32[P + i] = make_float2((float)w.x, (float)w.y);
}

}  // namespace

size_t coeffs_scratch_bytes(int d, int Nmax) {
  const size_t nel = (d == 2) ? (size_t)Nmax * Nmax : (size_t)Nmax * Nmax * Nmax;
  const size_t N1 = (size_t)Nmax + 1;
  const size_t nco = (d == 2) ? N1 * N1 : N1 * N1 * N1;
  const size_t nparts = (nco + 255) / 256;
  return align256(nel * 8) + align256(nparts * 8) + align256(2 * kQTotal * 8) + 256;
}

cudaError_t coeffs_launch(int d, double alpha, double gamma, double h, int N, double* coef, void* scratch,
                          cudaStream_t s) {
  unsigned char* sp = reinterpret_cast<unsigned char*>(scratch);
  const size_t nel = (d == 2) ? (size_t)N * N : (size_t)N * N * N;
  const size_t N1 = (size_t)N + 1;
  const size_t nco = (d == 2) ? N1 * N1 : N1 * N1 * N1;
  const int nparts = (int)((nco + 255) / 256);
  double* w = reinterpret_cast<double*>(sp);
  sp += align256(nel * 8);
  double* partial = reinterpret_cast<double*>(sp);
  sp += align256((size_t)nparts * 8);
  double* gn = reinterpret_cast<double*>(sp);
  double* gw = gn + kQTotal;
  sp += align256(2 * kQTotal * 8);
  double* pyr = reinterpret_cast<double*>(sp);
  const double p = d + alpha - gamma;
  const double hscale = pow(h, -alpha);
  k_gauss<<<1, 128, 0, s>>>(gn, gw);
  const int bs = 256;
  const unsigned gridw = (unsigned)((nel + bs - 1) / bs);
  if (d == 2) {
    k_element_weights<2><<<gridw, bs, 0, s>>>(w, N, p, gn, gw);
    k_fill_permuted<2><<<gridw, bs, 0, s>>>(w, N);
  } else {
    k_element_weights<3><<<gridw, bs, 0, s>>>(w, N, p, gn, gw);
    k_fill_permuted<3><<<gridw, bs, 0, s>>>(w, N);
  }
  k_pyramid<<<1, 256, 0, s>>>(d, p, alpha, N, gn, gw, pyr, w);
  if (d == 2) k_assemble<2><<<nparts, 256, 0, s>>>(w, N, gamma, hscale, pyr, coef, partial);
  else k_assemble<3><<<nparts, 256, 0, s>>>(w, N, gamma, hscale, pyr, coef, partial);
  k_diag<<<1, 256, 0, s>>>(partial, nparts, d, pyr, hscale, coef);
  return cudaGetLastError();
}

cudaError_t twiddle_launch(int P, double2* tw64, float2* tw32, cudaStream_t s) {
  k_twiddle<<<(P + 255) / 256, 256, 0, s>>>(P, tw64, tw32);
  int logP = 0;
  while ((1 << logP) < P) ++logP;
  const int nst = twiddle_entries(P) - P;
  k_twiddle_stage<<<(nst + 255) / 256, 256, 0, s>>>(P, logP, tw64, tw32);
  return cudaGetLastError();
}

cudaError_t generator_octant_launch(const Plan& p, const double* coef, double* lam, cudaStream_t s) {
  const int Hx1 = p.P[0] / 2 + 1, Hy1 = p.P[1] / 2 + 1, Hz1 = (p.d == 3) ? p.P[2] / 2 + 1 : 1;
  const size_t total = (size_t)Hx1 * Hy1 * Hz1;
  k_sym_init<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(coef, p.Nmax, p.d, p.n[0], p.n[1],
                                                             p.d == 3 ? p.n[2] : 1, Hx1, Hy1, Hz1, p.c, lam);
  return cudaGetLastError();
}

cudaError_t symbol_launch(const Plan& p, const double* coef, double* lam, cudaStream_t s) {
  cudaError_t e = generator_octant_launch(p, coef, lam, s);
  if (e != cudaSuccess) return e;
  return symbol_axes_launch(p, lam, s);
}

cudaError_t symbol_axes_launch(const Plan& p, double* lam, cudaStream_t s) {
  const int Hx1 = p.P[0] / 2 + 1, Hy1 = p.P[1] / 2 + 1, Hz1 = (p.d == 3) ? p.P[2] / 2 + 1 : 1;
  const size_t total = (size_t)Hx1 * Hy1 * Hz1;
  cudaError_t e;
  const int H1[3] = {Hx1, Hy1, Hz1};
  for (int r = 0; r < p.d; ++r) {
    const int P = p.P[r];
    const int logP = p.logP[r];
    if (P > kMaxLine) {  // two half-length transforms per line (k_sym_axis_split)
      size_t stride = 1;
      for (int q = 0; q < r; ++q) stride *= H1[q];
      const size_t nlines = total / H1[r];
      const size_t sm = (size_t)sline(kMaxLine) * 16 + (size_t)(P / 2 + 1) * 8;
      e = cudaFuncSetAttribute(k_sym_axis_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      k_sym_axis_split<<<(unsigned)nlines, kMaxLine / 16, sm, s>>>(lam, nlines, stride, stride, p.tw64[r]);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      continue;
    }
    const int G = P >> 4;
    int tl = (48 * 1024) / (sline(P) * 16);
    if (tl < 1) tl = 1;
    while (tl > 1 && tl * G > 512) --tl;
    if (G < 32) tl = tl < 32 / G ? 32 / G : tl - tl % (32 / G);  // whole warps (see line_sync)
    // lines along axis r: stride = product of H1 of faster axes; inner = that same product
    size_t stride = 1;
    for (int q = 0; q < r; ++q) stride *= H1[q];
    const size_t nlines = total / H1[r];
    const size_t sm = (size_t)tl * sline(P) * 16;
    e = cudaFuncSetAttribute(k_sym_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((nlines + tl - 1) / tl);
    k_sym_axis<<<grid, tl * G, sm, s>>>(lam, nlines, logP, stride, stride, tl, p.tw64[r]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace frlap

namespace frlap {
namespace {
__global__ void k_to_df(const double* __restrict__ src, dfl* dst, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = df_from(src[i]);
}
}  // namespace

namespace {
__global__ void k_to_cdf(const double2* __restrict__ src, cdf* dst, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_cdf(df_from(src[i].x), df_from(src[i].y));
}
}  // namespace

// double-float copy of a complex table (twiddles), n values, in the paired layout of cdf
cudaError_t to_cdf_launch(const double2* src, cdf* dst, size_t n, cudaStream_t st) {
  k_to_cdf<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

// double-float copies of a symbol (n values)
cudaError_t to_df_launch(const double* src, dfl* dst, size_t n, cudaStream_t st) {
  k_to_df<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t scale_symbol_launch(double* lam64, float* lam32, size_t n, double s, cudaStream_t st) {
  k_scale_copy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(lam64, lam32, n, s);
  return cudaGetLastError();
}

namespace {
template <typename To>
__device__ __forceinline__ To from_double(double v) {
  if constexpr (std::is_same<To, dfl>::value) return df_from(v);
  else return (To)v;
}

// natural octant [A][Bm][Cx] (Cx fastest) -> line-major [Cx][Bm][A] (A fastest), times s
template <typename To>
__global__ void k_oct_to_line(const double* __restrict__ oct, To* __restrict__ dst, size_t n, int A, int Bm, int Cx,
                              double s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = (int)(i % A);
  const size_t r = i / A;
  const int b = (int)(r % Bm), c = (int)(r / Bm);
  dst[i] = from_double<To>(oct[((size_t)a * Bm + b) * Cx + c] * s);
}
}  // namespace

template <typename To>
cudaError_t line_symbol_launch(const Plan& p, const double* oct, To* dst, double s, cudaStream_t st) {
  const int Hx1 = p.P[0] / 2 + 1, Hy1 = p.P[1] / 2 + 1;
  const int A = (p.d == 3) ? p.P[2] / 2 + 1 : Hy1, Bm = (p.d == 3) ? Hy1 : 1;
  const size_t n = p.lam_count;
  k_oct_to_line<To><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(oct, dst, n, A, Bm, Hx1, s);
  return cudaGetLastError();
}
template cudaError_t line_symbol_launch<double>(const Plan&, const double*, double*, double, cudaStream_t);
template cudaError_t line_symbol_launch<float>(const Plan&, const double*, float*, double, cudaStream_t);
template cudaError_t line_symbol_launch<dfl>(const Plan&, const double*, dfl*, double, cudaStream_t);
}  // namespace frlap
