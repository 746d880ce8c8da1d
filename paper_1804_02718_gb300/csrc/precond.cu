// Preconditioner symbols for the PCG solves.
//
// Strang circulant.  The multilevel Strang circulant S of A keeps, along every
// axis, the Toeplitz entry of offset min(j, n_r - j) in its first column.  Its
// eigenvalues are the size-n_r DFTs of that column (real, as the column is even),
// and S^-1 is again a multilevel circulant: its first column g is the inverse DFT
// of 1/lambda_S.  Read as a Toeplitz matrix (entry g[(i - j) mod n] at offset i - j),
// S^-1 is applied exactly like A: g is embedded in the same P_r-point circulant
// and its octant symbol is stored, so a preconditioner solve costs one FP32
// apply and needs no FFT of the (generally odd) length n_r.  The size-n_r DFTs
// of the set-up are direct O(n_r) sums per output in FP64.
//
// Sine-basis (tau) preconditioner.  The multilevel DST-I S (orthonormal sine modes of the box,
// which vanish on its boundary like u) diagonalises the "tau" matrix algebra; the member closest to A
// in the Frobenius norm is S diag(S A S) S, and its inverse M = S diag(S A S)^-1 S is the
// preconditioner.  The diagonal is separable: with t the generator (t_d = -c a_d) and, per axis,
//   C[k][d] = m_d / (n + 1) * ((n - d) cos(a_k d) + sin(a_k (d + 1)) / sin a_k),  a_k = pi k / (n + 1),
// (m_0 = 1, m_d = 2 otherwise; the closed form of sum_i s_k(i) s_k(i + d) over the two signs of d),
// diag(S A S)[k] = sum_d t_d prod_r C_r[k_r][d_r].  Each axis transform is one complex DFT of
// P = 2(n + 1) points per line (k_tau_axis), so the set-up costs about two symbol transforms.  M is
// applied as a multiplier on odd extensions to P points through the apply pipeline (its DFT is the
// DST), one FP32 apply per iteration, and needs P_r = 2 N_r on every axis.
#include <math.h>

#include "common.cuh"
#include "fft.cuh"

namespace frlap {

namespace {

// first column of the Strang circulant: s[j] = -c a[min(j_r, n_r - j_r)], j in [0, n)^d, x fastest
__global__ void k_strang_col(const double* __restrict__ coef, int Nmax, int d, int nx, int ny, int nz, double c,
                             double* s) {
  const size_t total = (size_t)nx * ny * nz;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int jx = (int)(e % nx), jy = (int)((e / nx) % ny), jz = (int)(e / ((size_t)nx * ny));
  const int kx = min(jx, nx - jx), ky = min(jy, ny - jy), kz = min(jz, nz - jz);
  const size_t N1 = (size_t)Nmax + 1;
  const size_t ci = (d == 2) ? (size_t)ky * N1 + kx : ((size_t)kz * N1 + ky) * N1 + kx;
  s[e] = -c * coef[ci];
}

// out[j] = scale * sum_{k < n} in[k] cos(2 pi j k / n) along one axis, in place, one line per CTA
__global__ void k_even_dft(double* data, int n, size_t stride, size_t inner, double scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* line = reinterpret_cast<double*>(smem_raw);
  double* ctab = line + n;
  const size_t li = blockIdx.x;
  const size_t base = (li / inner) * inner * (size_t)n + (li % inner);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    line[k] = data[base + (size_t)k * stride];
    ctab[k] = cospi(2.0 * k / n);
  }
  __syncthreads();
  double outv[8];
  int cnt = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double acc = 0.0;
    int m = 0;
    for (int k = 0; k < n; ++k) {
      acc = fma(line[k], ctab[m], acc);
      m += j;
      if (m >= n) m -= n;
    }
    if (cnt < 8) outv[cnt] = acc * scale;
    ++cnt;
  }
  __syncthreads();
  cnt = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    if (cnt < 8) data[base + (size_t)j * stride] = outv[cnt];
    ++cnt;
  }
}

// v <- 1 / v ; counts entries that are not positive (their modes are dropped: inverse set to 0)
__global__ void k_invert(double* v, size_t n, unsigned* bad) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = v[i];
    if (!(x > 0.0) || !isfinite(x)) {
      atomicAdd(bad, 1u);
      v[i] = 0.0;
    } else {
      v[i] = 1.0 / x;
    }
  }
}

// octant fill: oct[k] = g[k] for k_r <= n_r - 1 (inside the octant), 0 elsewhere
__global__ void k_oct_from_grid(const double* __restrict__ g, int nx, int ny, int nz, int Hx1, int Hy1, int Hz1,
                                double* oct) {
  const size_t total = (size_t)Hx1 * Hy1 * Hz1;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int kx = (int)(e % Hx1), ky = (int)((e / Hx1) % Hy1), kz = (int)(e / ((size_t)Hx1 * Hy1));
  double v = 0.0;
  if (kx < nx && ky < ny && kz < nz) v = g[((size_t)kz * ny + ky) * nx + kx];
  oct[e] = v;
}

__global__ void k_scale_to_f32(const double* __restrict__ src, float* dst, size_t n, double s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)(src[i] * s);
}

}  // namespace

cudaError_t scale_to_f32_launch(const double* src, float* dst, size_t n, double s, cudaStream_t st) {
  k_scale_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n, s);
  return cudaGetLastError();
}

size_t strang_scratch_bytes(const Plan& p) {
  const size_t N1 = (size_t)p.Nmax + 1;
  const size_t ncoef = (p.d == 2) ? N1 * N1 : N1 * N1 * N1;
  return align256(ncoef * 8) + align256(coeffs_scratch_bytes(p.d, p.Nmax)) + align256(p.M * 8) +
         align256(p.lam_count * 8) + 256;
}

// Builds plan->mu_strang (FP32 octant, 1/prod(P) folded in).  Returns the number of
// non-positive Strang eigenvalues through *bad_host (0 for this operator: A is strictly
// diagonally dominant, and so is its Strang circulant).
cudaError_t strang_build(Plan& p, void* scratch, cudaStream_t s, unsigned* bad_host) {
  unsigned char* w = reinterpret_cast<unsigned char*>(scratch);
  const size_t N1 = (size_t)p.Nmax + 1;
  const size_t ncoef = (p.d == 2) ? N1 * N1 : N1 * N1 * N1;
  double* coef = reinterpret_cast<double*>(w);
  w += align256(ncoef * 8);
  void* cscratch = w;
  w += align256(coeffs_scratch_bytes(p.d, p.Nmax));
  double* grid = reinterpret_cast<double*>(w);
  w += align256(p.M * 8);
  double* oct = reinterpret_cast<double*>(w);
  w += align256(p.lam_count * 8);
  unsigned* bad = reinterpret_cast<unsigned*>(w);
  cudaError_t e = coeffs_launch(p.d, p.alpha, p.gamma, p.h, p.Nmax, coef, cscratch, s);
  if (e != cudaSuccess) return e;
  const int nx = p.n[0], ny = p.n[1], nz = (p.d == 3) ? p.n[2] : 1;
  k_strang_col<<<(unsigned)((p.M + 255) / 256), 256, 0, s>>>(coef, p.Nmax, p.d, nx, ny, nz, p.c, grid);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nn[3] = {nx, ny, nz};
  // forward: lambda_S = DFT_n of the column; then 1/lambda_S; then g = inverse DFT (scale 1/n per axis)
  for (int pass = 0; pass < 2; ++pass) {
    size_t stride = 1;
    for (int r = 0; r < p.d; ++r) {
      const int n = nn[r];
      const size_t nlines = p.M / n;
      const size_t sm = 2 * (size_t)n * sizeof(double);
      e = cudaFuncSetAttribute(k_even_dft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      const int threads = n <= 256 ? 256 : 512;
      const double scale = pass == 0 ? 1.0 : 1.0 / n;
      k_even_dft<<<(unsigned)nlines, threads, sm, s>>>(grid, n, stride, stride, scale);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      stride *= n;
    }
    if (pass == 0) {
      if ((e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
      k_invert<<<2 * 152, 256, 0, s>>>(grid, p.M, bad);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  const int Hx1 = p.P[0] / 2 + 1, Hy1 = p.P[1] / 2 + 1, Hz1 = (p.d == 3) ? p.P[2] / 2 + 1 : 1;
  k_oct_from_grid<<<(unsigned)((p.lam_count + 255) / 256), 256, 0, s>>>(grid, nx, ny, nz, Hx1, Hy1, Hz1, oct);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = symbol_axes_launch(p, oct, s)) != cudaSuccess) return e;
  double scale = 1.0;
  for (int r = 0; r < p.d; ++r) scale /= (double)p.P[r];
  if ((e = line_symbol_launch<float>(p, oct, p.mu_strang, scale, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(bad_host, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

namespace {

// One axis of diag(S A S): for each line v_d (d = 0 .. n-1, stored at entries 0 .. n-1 of the octant
// line), out_k = sum_d C[k][d] v_d for k = 1 .. n, stored at entries 1 .. n (entries 0 and n + 1 = P/2
// become 0).  With w1_d = m_d (n - d) v_d and w2_{d+1} = m_d v_d, one P-point DFT F of w1 + i w2 gives
// the cosine sums A_k = Re DFT(w1)_k and the sine sums B_k = -Im DFT(w2)_k (separated by F_k and
// conj F_{P-k}); out_k = (A_k + B_k / sin a_k) / (n + 1).  TL lines per CTA of P/16 threads each, in
// whole warps (the FFT helpers end their short-line stages with warp barriers).
__global__ void __launch_bounds__(512) k_tau_axis(double* oct, size_t nlines, int logP, size_t stride, size_t inner,
                                                  int n, int TL, const double2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = 1 << logP, G = P >> 4, H = P / 2;
  const int l = threadIdx.x / G, lane = threadIdx.x % G;
  const size_t line = (size_t)blockIdx.x * TL + l;
  const bool valid = line < nlines;
  double2* buf = reinterpret_cast<double2*>(smem_raw) + (size_t)l * sline(P);
  const size_t li = valid ? line : 0;
  const size_t base = (li / inner) * inner * (size_t)(H + 1) + (li % inner);
  for (int j = lane; j < P; j += G) {
    const double w1 = (valid && j < n) ? (j == 0 ? 1.0 : 2.0) * (double)(n - j) * oct[base + (size_t)j * stride] : 0.0;
    const double w2 = (valid && j >= 1 && j <= n) ? (j == 1 ? 1.0 : 2.0) * oct[base + (size_t)(j - 1) * stride] : 0.0;
    buf[spad(j)] = make_double2(w1, w2);
  }
  __syncthreads();
  fft_line<double, -1>(buf, logP, lane, tw, logP);
  __syncthreads();
  if (!valid) return;
  for (int k = lane; k <= H; k += G) {
    double out = 0.0;
    if (k >= 1 && k <= n) {
      const double2 f = buf[spad(k)], g = buf[spad(P - k)];
      const double A = 0.5 * (f.x + g.x);  // Re of (F_k + conj F_{P-k}) / 2
      const double B = 0.5 * (f.x - g.x);  // -Im of (F_k - conj F_{P-k}) / 2i
      out = (A + B / sinpi((double)k / (n + 1))) / (n + 1);
    }
    oct[base + (size_t)k * stride] = out;
  }
}

// mu = 1 / diag(S A S) on the modes k_r = 1 .. n_r (0 elsewhere); counts non-positive entries.
// 2D: Hy1 = total / Hx1 and nz = 0 (no z axis).
__global__ void k_tau_invert(double* oct, size_t total, int Hx1, int Hy1, int nx, int ny, int nz, unsigned* bad) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int kx = (int)(i % Hx1), ky = (int)((i / Hx1) % Hy1), kz = (int)(i / ((size_t)Hx1 * Hy1));
  double v = 0.0;
  if (kx >= 1 && kx <= nx && ky >= 1 && ky <= ny && (nz == 0 ? kz == 0 : (kz >= 1 && kz <= nz))) {
    const double t = oct[i];
    if (t > 0.0) v = 1.0 / t;
    else atomicAdd(bad, 1u);
  }
  oct[i] = v;
}

}  // namespace

namespace {
// mu_b = scale / (sigma + s tau) from mu = scale / tau (0 stays 0): the sine-basis preconditioner of
// sigma I + s A, whose diagonal in the sine basis is sigma + s diag(S A S)
__global__ void k_tau_shift(const float* __restrict__ mu, float* __restrict__ mu_b, size_t n, double scale,
                            double sigma, double s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m = mu[i];
  mu_b[i] = m == 0.0 ? 0.0f : (float)(scale * m / (sigma * m + s * scale));
}
}  // namespace

cudaError_t shifted_tau_launch(const Plan& p, double sigma, double s, float* mu_b, cudaStream_t st) {
  double scale = 1.0;
  for (int r = 0; r < p.d; ++r) scale /= (double)p.P[r];
  k_tau_shift<<<(unsigned)((p.lam_count + 255) / 256), 256, 0, st>>>(p.mu_tau, mu_b, p.lam_count, scale, sigma, s);
  return cudaGetLastError();
}

size_t tau_scratch_bytes(const Plan& p) {
  const size_t N1 = (size_t)p.Nmax + 1;
  const size_t ncoef = (p.d == 2) ? N1 * N1 : N1 * N1 * N1;
  return align256(ncoef * 8) + align256(coeffs_scratch_bytes(p.d, p.Nmax)) + align256(p.lam_count * 8) + 256;
}

// Builds plan->mu_tau (line-major FP32, the 1/prod(P) of the apply pipeline folded in).  Needs
// P_r = 2 N_r <= 8192 on every axis (the caller checks).  *bad_host: entries of diag(S A S) that are not
// positive (none for a symmetric positive definite A: each is a Rayleigh quotient of A).
cudaError_t tau_build(Plan& p, void* scratch, cudaStream_t s, unsigned* bad_host) {
  unsigned char* w = reinterpret_cast<unsigned char*>(scratch);
  const size_t N1 = (size_t)p.Nmax + 1;
  const size_t ncoef = (p.d == 2) ? N1 * N1 : N1 * N1 * N1;
  double* coef = reinterpret_cast<double*>(w);
  w += align256(ncoef * 8);
  void* cscratch = w;
  w += align256(coeffs_scratch_bytes(p.d, p.Nmax));
  double* oct = reinterpret_cast<double*>(w);
  w += align256(p.lam_count * 8);
  unsigned* bad = reinterpret_cast<unsigned*>(w);
  cudaError_t e = coeffs_launch(p.d, p.alpha, p.gamma, p.h, p.Nmax, coef, cscratch, s);
  if (e != cudaSuccess) return e;
  if ((e = generator_octant_launch(p, coef, oct, s)) != cudaSuccess) return e;
  const int Hx1 = p.P[0] / 2 + 1, Hy1 = p.P[1] / 2 + 1, Hz1 = p.d == 3 ? p.P[2] / 2 + 1 : 1;
  const int H1[3] = {Hx1, Hy1, Hz1};
  const size_t total = (size_t)Hx1 * Hy1 * Hz1;
  for (int r = 0; r < p.d; ++r) {
    size_t stride = 1;
    for (int q = 0; q < r; ++q) stride *= H1[q];
    const size_t nlines = total / H1[r];
    const int G = p.P[r] / 16;
    const int tl = G < 32 ? 32 / G : 1;
    const size_t sm = (size_t)tl * sline(p.P[r]) * sizeof(double2);
    if ((e = cudaFuncSetAttribute(k_tau_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
      return e;
    k_tau_axis<<<(unsigned)((nlines + tl - 1) / tl), tl * G, sm, s>>>(oct, nlines, p.logP[r], stride, stride, p.n[r],
                                                                     tl, p.tw64[r]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  k_tau_invert<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(oct, total, Hx1, Hy1, p.n[0], p.n[1],
                                                               p.d == 3 ? p.n[2] : 0, bad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double scale = 1.0;
  for (int r = 0; r < p.d; ++r) scale /= (double)p.P[r];
  if ((e = line_symbol_launch<float>(p, oct, p.mu_tau, scale, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(bad_host, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace frlap
