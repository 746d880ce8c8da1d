// The learned Fourier-multiplier preconditioner: a per-frequency MLP over
// (alpha, kappa_x, kappa_y, kappa_z), kappa_r = k_r / (P_r/2) on the symbol octant,
// two tanh layers of 64 units, output s; multiplier m(k) = exp(s(k)) / lambda(k)
// (lambda = A's embedding symbol, so a zero network is the inverse-embedding
// preconditioner).  M^-1 r = R F^-1 (m . F R^T r).
//
// Training pairs (r_b, e_b = A^-1 r_b) come from the plain CG solver.  The loss is
// the relative A-norm error of z_b = M^-1 r_b as an approximation of e_b:
//   L = mean_b ||e_b - z_b||_A^2 / ||e_b||_A^2 = mean_b (1 - 2 a_b / c_b + b_b / c_b),
//   a = r.z,  b = z.Az,  c = r.e.
// (For the untrained network M A >= I, with most eigenvalues at 1, so the loss pins the
// overall scale of M; a per-pair scale-free form let bands of frequencies rescale
// independently and spread the spectrum of M A.)
// With ^ the P-point DFT of a zero-padded field, R = r^, W = (Az)^:
//   dL/dm(k) = mean_b [ -(2/c) |R(k)|^2 + (1/c) 2 Re(conj(W(k)) R(k)) ] / prod(P),
// summed over the mirror images of each octant entry, and dL/ds(k) = dL/dm(k) m(k);
// the network gradient follows by backpropagation.
// Spectra and residuals are FP64; the network is FP32 (weights, activations),
// its gradient is reduced in FP64.
#include <math.h>

#include "common.cuh"

namespace frlap {

namespace {

constexpr int HID = FRLAP_MLP_HIDDEN;
constexpr int NF = FRLAP_MLP_NFEAT;
constexpr int NPAR = FRLAP_MLP_NPARAM;
// parameter offsets (W1 [HID][NF], b1, W2 [HID][HID] (out, in), b2, w3, b3)
constexpr int OW1 = 0, OB1 = OW1 + HID * NF, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + HID;
static_assert(OB3 + 1 == NPAR, "parameter layout");

struct Oct {
  int d;
  int Hx1, Hy1, Hz1;  // octant extents
  float ix, iy, iz;   // 1 / (P_r / 2)
  float alpha;
};

__device__ __forceinline__ void features(const Oct& o, size_t f, float* phi) {
  const int kx = (int)(f % o.Hx1);
  const int ky = (int)((f / o.Hx1) % o.Hy1);
  const int kz = (int)(f / ((size_t)o.Hx1 * o.Hy1));
  phi[0] = o.alpha;
  phi[1] = kx * o.ix;
  phi[2] = ky * o.iy;
  phi[3] = (o.d == 3) ? kz * o.iz : 0.0f;
}

// m(f) = exp(s(f)) / lambda(f); optional caches of the two hidden layers for backprop
__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ params, Oct o, const double* __restrict__ lam,
                                                 double lamscale, size_t F, double* m, double* m_scaled,
                                                 double mscale, float* h1c, float* h2c) {
  __shared__ float W[NPAR];
  for (int i = threadIdx.x; i < NPAR; i += blockDim.x) W[i] = params[i];
  __syncthreads();
  const size_t f = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  float phi[NF];
  features(o, f, phi);
  float h1[HID];
#pragma unroll
  for (int h = 0; h < HID; ++h) {
    float a = W[OB1 + h];
#pragma unroll
    for (int j = 0; j < NF; ++j) a = fmaf(W[OW1 + h * NF + j], phi[j], a);
    h1[h] = tanhf(a);
    if (h1c) h1c[f * HID + h] = h1[h];
  }
  float s = W[OB3];
  for (int q = 0; q < HID; ++q) {
    float a = W[OB2 + q];
#pragma unroll
    for (int i = 0; i < HID; ++i) a = fmaf(W[OW2 + q * HID + i], h1[i], a);
    const float h2 = tanhf(a);
    if (h2c) h2c[f * HID + q] = h2;
    s = fmaf(W[OW3 + q], h2, s);
  }
  const double l = lam[f] * lamscale;
  const double mv = (l > 0.0) ? exp((double)s) / l : 0.0;
  m[f] = mv;
  if (m_scaled) m_scaled[f] = mv * mscale;
}

// per-block partial gradients of sum_f g_s(f) s(f), g_s = g_m * m; 64 entries per block, 256 threads
constexpr int BENT = 64;
__global__ void __launch_bounds__(256) k_mlp_bwd(const float* __restrict__ params, Oct o,
                                                 const double* __restrict__ g_m, const double* __restrict__ m,
                                                 const float* __restrict__ h1c, const float* __restrict__ h2c,
                                                 size_t F, float* partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* W2 = reinterpret_cast<float*>(smem_raw);  // [HID][HID]
  float* sh1 = W2 + HID * HID;                      // [BENT][HID]
  float* sh2 = sh1 + BENT * HID;
  float* sga2 = sh2 + BENT * HID;
  float* sga1 = sga2 + BENT * HID;
  float* sphi = sga1 + BENT * HID;                  // [BENT][NF]
  float* sgs = sphi + BENT * NF;                    // [BENT]
  for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) W2[i] = params[OW2 + i];
  const size_t f0 = (size_t)blockIdx.x * BENT;
  // load caches and per-entry output gradient
  for (int i = threadIdx.x; i < BENT * HID; i += blockDim.x) {
    const int e = i / HID, h = i % HID;
    const size_t f = f0 + e;
    const bool v = f < F;
    sh1[i] = v ? h1c[f * HID + h] : 0.0f;
    sh2[i] = v ? h2c[f * HID + h] : 0.0f;
  }
  for (int e = threadIdx.x; e < BENT; e += blockDim.x) {
    const size_t f = f0 + e;
    float phi[NF];
    features(o, f < F ? f : 0, phi);
    for (int j = 0; j < NF; ++j) sphi[e * NF + j] = phi[j];
    sgs[e] = (f < F) ? (float)(g_m[f] * m[f]) : 0.0f;
  }
  __syncthreads();
  // g_a2[e][q] = g_s[e] w3[q] (1 - h2^2)
  for (int i = threadIdx.x; i < BENT * HID; i += blockDim.x) {
    const int e = i / HID, q = i % HID;
    const float h2 = sh2[i];
    sga2[i] = sgs[e] * params[OW3 + q] * (1.0f - h2 * h2);
  }
  __syncthreads();
  // g_a1[e][h] = (sum_q W2[q][h] g_a2[e][q]) (1 - h1^2)
  for (int i = threadIdx.x; i < BENT * HID; i += blockDim.x) {
    const int e = i / HID, h = i % HID;
    float a = 0.0f;
    for (int q = 0; q < HID; ++q) a = fmaf(W2[q * HID + h], sga2[e * HID + q], a);
    const float h1 = sh1[i];
    sga1[i] = a * (1.0f - h1 * h1);
  }
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * NPAR;
  for (int p = threadIdx.x; p < NPAR; p += blockDim.x) {
    float acc = 0.0f;
    if (p < OB1) {  // W1[h][j]
      const int h = p / NF, j = p % NF;
      for (int e = 0; e < BENT; ++e) acc = fmaf(sga1[e * HID + h], sphi[e * NF + j], acc);
    } else if (p < OW2) {  // b1
      const int h = p - OB1;
      for (int e = 0; e < BENT; ++e) acc += sga1[e * HID + h];
    } else if (p < OB2) {  // W2[q][i]
      const int q = (p - OW2) / HID, i = (p - OW2) % HID;
      for (int e = 0; e < BENT; ++e) acc = fmaf(sga2[e * HID + q], sh1[e * HID + i], acc);
    } else if (p < OW3) {  // b2
      const int q = p - OB2;
      for (int e = 0; e < BENT; ++e) acc += sga2[e * HID + q];
    } else if (p < OB3) {  // w3
      const int q = p - OW3;
      for (int e = 0; e < BENT; ++e) acc = fmaf(sgs[e], sh2[e * HID + q], acc);
    } else {  // b3
      for (int e = 0; e < BENT; ++e) acc += sgs[e];
    }
    out[p] = acc;
  }
}

// grad[p] = sum over blocks of the partials (FP64 accumulation, fixed order)
__global__ void k_param_reduce(const float* __restrict__ partial, int nblocks, float* grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPAR) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) acc += (double)partial[(size_t)b * NPAR + p];
  grad[p] = (float)acc;
}

__device__ __forceinline__ double bsum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// one block: out[0] = r.z, out[1] = z.w, out[2] = r.e
__global__ void k_dots3(const double* __restrict__ r, const double* __restrict__ z, const double* __restrict__ w,
                        const double* __restrict__ e, size_t n, double* out) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double ri = r[i], zi = z[i];
    a += ri * zi;
    b += zi * w[i];
    c += ri * e[i];
  }
  const double ta = bsum(a, red);
  const double tb = bsum(b, red);
  const double tc = bsum(c, red);
  if (threadIdx.x == 0) {
    out[0] = ta;
    out[1] = tb;
    out[2] = tc;
  }
}

// g_m[f] += (x weight) * sum over the y (z) mirror images of
//           [ -(2/c) |R|^2 + (1/c) 2 Re(conj(W) R) ] / (B prod(P))
__global__ void k_grad_accum(const double2* __restrict__ SR, const double2* __restrict__ SW, Oct o, int Py, int Pz,
                             const double* __restrict__ dots, int B, double invP, double* g_m) {
  const size_t F = (size_t)o.Hx1 * o.Hy1 * o.Hz1;
  const size_t f = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int kx = (int)(f % o.Hx1);
  const int ky = (int)((f / o.Hx1) % o.Hy1);
  const int kz = (int)(f / ((size_t)o.Hx1 * o.Hy1));
  const int ny_img = (ky == 0 || 2 * ky == Py) ? 1 : 2;
  const int nz_img = (o.d == 2) ? 1 : ((kz == 0 || 2 * kz == Pz) ? 1 : 2);
  const double c = dots[2];
  if (!(c > 0.0)) return;  // degenerate pair (zero error): no contribution
  const double ca = -2.0 / c, cb = 2.0 / c;
  double acc = 0.0;
  for (int i = 0; i < ny_img; ++i) {
    const int yy = i == 0 ? ky : Py - ky;
    for (int j = 0; j < nz_img; ++j) {
      const int zz = j == 0 ? kz : Pz - kz;
      const size_t idx = (o.d == 2) ? (size_t)kx * Py + yy : ((size_t)kx * Py + yy) * Pz + zz;
      const double2 rv = SR[idx], wv = SW[idx];
      acc += ca * (rv.x * rv.x + rv.y * rv.y) + cb * (wv.x * rv.x + wv.y * rv.y);
    }
  }
  const double wx = (kx == 0 || kx == o.Hx1 - 1) ? 1.0 : 2.0;
  g_m[f] += wx * acc * invP / B;
}

__global__ void k_loss(const double* __restrict__ dots, int B, double* loss) {
  double L = 0.0;
  for (int i = 0; i < B; ++i) {
    const double a = dots[3 * i], b = dots[3 * i + 1], c = dots[3 * i + 2];
    if (c > 0.0) L += (1.0 - 2.0 * a / c + b / c) / B;
  }
  *loss = L;
}

__global__ void k_adam(float* p, const float* __restrict__ g, float* m1, float* m2, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

Oct make_oct(const Plan& p) {
  Oct o;
  o.d = p.d;
  o.Hx1 = p.P[0] / 2 + 1;
  o.Hy1 = p.P[1] / 2 + 1;
  o.Hz1 = (p.d == 3) ? p.P[2] / 2 + 1 : 1;
  o.ix = 2.0f / p.P[0];
  o.iy = 2.0f / p.P[1];
  o.iz = (p.d == 3) ? 2.0f / p.P[2] : 0.0f;
  o.alpha = (float)p.alpha;
  return o;
}

double prodP(const Plan& p) {
  double s = 1.0;
  for (int r = 0; r < p.d; ++r) s *= (double)p.P[r];
  return s;
}

struct LearnBufs {
  void* awork;
  double2* SR;
  double2* SD;
  double* z;
  double* w;
  double* m;
  double* ms;
  double* gm;
  float* h1;
  float* h2;
  float* partial;
  double* norms;
};

LearnBufs carve_learn(const Plan& p, void* work, int B) {
  LearnBufs b;
  const size_t F = p.lam_count;
  const size_t nblk = (F + BENT - 1) / BENT;
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  b.awork = w;
  w += apply_work_bytes(p, 8);
  b.SR = reinterpret_cast<double2*>(w);
  w += align256(spectrum_elems(p) * 16);
  b.SD = reinterpret_cast<double2*>(w);
  w += align256(spectrum_elems(p) * 16);
  b.z = reinterpret_cast<double*>(w);
  w += align256(p.M * 8);
  b.w = reinterpret_cast<double*>(w);
  w += align256(p.M * 8);
  b.m = reinterpret_cast<double*>(w);
  w += align256(F * 8);
  b.ms = reinterpret_cast<double*>(w);
  w += align256(F * 8);
  b.gm = reinterpret_cast<double*>(w);
  w += align256(F * 8);
  b.h1 = reinterpret_cast<float*>(w);
  w += align256(F * HID * 4);
  b.h2 = reinterpret_cast<float*>(w);
  w += align256(F * HID * 4);
  b.partial = reinterpret_cast<float*>(w);
  w += align256(nblk * NPAR * 4);
  b.norms = reinterpret_cast<double*>(w);
  (void)B;
  return b;
}

}  // namespace

size_t learn_work_bytes(const Plan& p, int B) {
  const size_t F = p.lam_count;
  const size_t nblk = (F + BENT - 1) / BENT;
  return apply_work_bytes(p, 8) + 2 * align256(spectrum_elems(p) * 16) + 2 * align256(p.M * 8) +
         3 * align256(F * 8) + 2 * align256(F * HID * 4) + align256(nblk * NPAR * 4) + align256((size_t)3 * B * 8) +
         256;
}

cudaError_t mlp_multiplier_launch(const Plan& p, const float* params, double* m, cudaStream_t s) {
  const Oct o = make_oct(p);
  const size_t F = p.lam_count;
  k_mlp_fwd<<<(unsigned)((F + 127) / 128), 128, 0, s>>>(params, o, p.lam64, prodP(p), F, m, nullptr, 1.0, nullptr,
                                                        nullptr);
  return cudaGetLastError();
}

cudaError_t learn_grad_launch(const Plan& p, const float* params, const double* r, const double* e, int B,
                              float* grad, double* loss, void* work, cudaStream_t s) {
  const LearnBufs b = carve_learn(p, work, B);
  const Oct o = make_oct(p);
  const size_t F = p.lam_count;
  const double PP = prodP(p);
  cudaError_t err;
  k_mlp_fwd<<<(unsigned)((F + 127) / 128), 128, 0, s>>>(params, o, p.lam64, PP, F, b.m, b.ms, 1.0 / PP, b.h1, b.h2);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(b.gm, 0, F * sizeof(double), s)) != cudaSuccess) return err;
  const int Py = p.P[1], Pz = (p.d == 3) ? p.P[2] : 1;
  for (int i = 0; i < B; ++i) {
    const double* ri = r + (size_t)i * p.M;
    const double* ei = e + (size_t)i * p.M;
    if ((err = spectrum_forward<double>(p, ri, b.SR, b.awork, s)) != cudaSuccess) return err;
    if ((err = spectrum_inverse<double>(p, b.SR, b.ms, b.z, b.awork, s)) != cudaSuccess) return err;
    if ((err = apply_launch<double>(p, b.z, b.w, b.awork, s, nullptr)) != cudaSuccess) return err;
    if ((err = spectrum_forward<double>(p, b.w, b.SD, b.awork, s)) != cudaSuccess) return err;
    k_dots3<<<1, 1024, 0, s>>>(ri, b.z, b.w, ei, p.M, b.norms + 3 * i);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    k_grad_accum<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(b.SR, b.SD, o, Py, Pz, b.norms + 3 * i, B, 1.0 / PP,
                                                            b.gm);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  k_loss<<<1, 1, 0, s>>>(b.norms, B, loss);
  const int nblk = (int)((F + BENT - 1) / BENT);
  const size_t sm = (size_t)(HID * HID + 4 * BENT * HID + BENT * NF + BENT) * sizeof(float);
  if ((err = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
    return err;
  k_mlp_bwd<<<nblk, 256, sm, s>>>(params, o, b.gm, b.m, b.h1, b.h2, F, b.partial);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  k_param_reduce<<<(NPAR + 255) / 256, 256, 0, s>>>(b.partial, nblk, grad);
  return cudaGetLastError();
}

cudaError_t adam_launch(float* p, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                        int t, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m1, m2, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace frlap
