// C-ABI entry points of libfrlap (declared in include/frlap.h).
#include <math.h>
#include <stdio.h>

#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace frlap {

static thread_local std::string g_last_error;
static std::atomic<unsigned> g_pass_limit{0u};

unsigned loop_pass_limit() { return g_pass_limit.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

frlap_status fail(frlap_status code, const std::string& msg) {
  set_error(msg);
  return code;
}

frlap_status cuda_fail(cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  set_error(m);
  return FRLAP_ECUDA;
}

size_t cg_work_bytes(const Plan& p, int eb);
size_t ir_work_bytes(const Plan& p);
size_t pcg_work_bytes(const Plan& p);
size_t ac_work_bytes(const Plan& p);
frlap_status pcg_solve_impl(const Plan& p, const double* f, double* x, double rtol, int maxit, int solver,
                            const float* mu, double inner_rtol, int* iters, double* relres, void* work,
                            cudaStream_t st);
frlap_status residual_impl(const Plan& p, const double* f, const double* x, double* r, double* relres, void* work,
                           cudaStream_t st);
size_t strang_scratch_bytes(const Plan& p);
size_t learn_work_bytes(const Plan& p, int B);
cudaError_t mlp_multiplier_launch(const Plan& p, const float* params, double* m, cudaStream_t s);
cudaError_t learn_grad_launch(const Plan& p, const float* params, const double* r, const double* e, int B,
                              float* grad, double* loss, void* work, cudaStream_t s);
cudaError_t adam_launch(float* p, const float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                        int t, cudaStream_t s);
size_t ac_batch_work_bytes(int nb, const frlap_plan* const* plans);
frlap_status ac_batch_impl(int nb, const frlap_plan* const* plans, double* const* u, double tau, double eps,
                           int nsteps, double rtol, int maxit, int* iters_out, int* status_out, void* work,
                           cudaStream_t user);
frlap_status cg_pairs_impl(const Plan& p, const double* f, int K, double rtol, double* E, double* R, int* npairs,
                           void* work, cudaStream_t st);
cudaError_t strang_build(Plan& p, void* scratch, cudaStream_t s, unsigned* bad_host);
size_t tau_scratch_bytes(const Plan& p);
cudaError_t tau_build(Plan& p, void* scratch, cudaStream_t s, unsigned* bad_host);
cudaError_t scale_to_f32_launch(const double* src, float* dst, size_t n, double s, cudaStream_t st);
frlap_status allen_cahn_cn_impl(const Plan& p, double* ub, double tau, double delta, int nsteps, double rtol,
                                int* iters, double* h_mass, void* work, cudaStream_t st);
frlap_status allen_cahn_impl(const Plan& p, double* u, double tau, double eps, int nsteps, double rtol,
                             int* iters, void* work, cudaStream_t st);

static double c_dalpha_host(int d, double alpha) {
  return pow(2.0, alpha - 1.0) * alpha * tgamma((d + alpha) / 2.0) /
         (pow(M_PI, d / 2.0) * tgamma(1.0 - alpha / 2.0));
}

static frlap_status check_params(int d, double alpha, double gamma, double h, const int* N) {
  if (d != 2 && d != 3) return fail(FRLAP_EINVAL, "d must be 2 or 3");
  if (!(alpha > 0.0 && alpha < 2.0)) return fail(FRLAP_EINVAL, "alpha must lie in (0, 2)");
  if (!(gamma > alpha && gamma <= 2.0)) return fail(FRLAP_EINVAL, "gamma must lie in (alpha, 2]");
  if (!(h > 0.0) || !isfinite(h)) return fail(FRLAP_EINVAL, "h must be positive and finite");
  if (!N) return fail(FRLAP_EINVAL, "N is NULL");
  // 2D: N <= 8192 (embeddings of up to 16384 points; the 16384-point middle stage runs as two
  // 8192-point halves, the rows as 8192-point half-length transforms); 3D: N <= 1024
  const int Nlim = (d == 2) ? 8192 : 1024;
  for (int r = 0; r < d; ++r)
    if (N[r] < 2 || N[r] > Nlim) return fail(FRLAP_EINVAL, "each N[r] must lie in [2, 8192] (2D) or [2, 1024] (3D)");
  return FRLAP_OK;
}

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace frlap

using namespace frlap;

extern "C" {

const char* frlap_last_error(void) { return g_last_error.c_str(); }

frlap_status frlap_async_wait_report(unsigned long long* timeouts) {
  if (!timeouts) return fail(FRLAP_EINVAL, "timeouts is NULL");
  unsigned long long total = 0ull;
  cudaError_t (*collect[3])(unsigned long long*) = {wait_collect<float>, wait_collect<double>, wait_collect<dfl>};
  for (auto fn : collect) {
    unsigned long long c = 0ull;
    FRLAP_CUDA_TRY(fn(&c));
    total += c;
  }
  for (auto fn : {dft16_wait_collect, hyb_wait_collect}) {
    unsigned long long c = 0ull;
    FRLAP_CUDA_TRY(fn(&c));
    total += c;
  }
  *timeouts = total;
  return FRLAP_OK;
}

frlap_status frlap_dft16_stages(int engine, const float* d_in, float* d_out, int ntiles, int reps, void* stream) {
  if (engine != 0 && engine != 1) return fail(FRLAP_EINVAL, "engine must be 0 (CUDA cores) or 1 (tensor cores)");
  if (ntiles < 0 || ntiles > (1 << 24)) return fail(FRLAP_EINVAL, "ntiles must be in [0, 2^24]");
  if (reps < 0 || reps > (1 << 16)) return fail(FRLAP_EINVAL, "reps must be in [0, 65536]");
  if (ntiles == 0) return FRLAP_OK;
  if (!d_in || !d_out) return fail(FRLAP_EINVAL, "d_in and d_out must not be NULL");
  if (reinterpret_cast<uintptr_t>(d_in) % 16 || reinterpret_cast<uintptr_t>(d_out) % 16)
    return fail(FRLAP_EINVAL, "d_in and d_out must be 16-byte aligned");
  const size_t bytes = (size_t)ntiles * 4096 * sizeof(float);
  if (d_in != d_out && ranges_overlap(d_in, d_out, bytes))
    return fail(FRLAP_EINVAL, "d_in and d_out must be equal or not overlap");
  FRLAP_CUDA_TRY(dft16_stages_launch(engine, d_in, d_out, ntiles, reps, static_cast<cudaStream_t>(stream)));
  return FRLAP_OK;
}

frlap_status frlap_async_wait_selftest(unsigned long long* timeouts) {
  if (!timeouts) return fail(FRLAP_EINVAL, "timeouts is NULL");
  FRLAP_CUDA_TRY(wait_selftest(timeouts));
  return FRLAP_OK;
}

frlap_status frlap_bounds_check_report(int* enabled, unsigned long long* violations,
                                       unsigned long long* first_address) {
  if (!violations) return fail(FRLAP_EINVAL, "violations is NULL");
  unsigned long long total = 0ull, first = ~0ull;
  cudaError_t (*collect[4])(unsigned long long*, unsigned long long*) = {bc_collect<float>, bc_collect<double>,
                                                                         bc_collect<dfl>, hyb_bc_collect};
  for (auto fn : collect) {
    unsigned long long c = 0ull, f = ~0ull;
    FRLAP_CUDA_TRY(fn(&c, &f));
    total += c;
    if (f < first) first = f;
  }
#ifdef FRLAP_BOUNDS_CHECK
  if (enabled) *enabled = 1;
#else
  if (enabled) *enabled = 0;
#endif
  *violations = total;
  if (first_address) *first_address = total ? first : 0ull;
  return FRLAP_OK;
}

frlap_status frlap_bounds_check_selftest(unsigned long long* flagged) {
  if (!flagged) return fail(FRLAP_EINVAL, "flagged is NULL");
#ifdef FRLAP_BOUNDS_CHECK
  FRLAP_CUDA_TRY(bc_selftest(flagged));
  return FRLAP_OK;
#else
  *flagged = 0ull;
  return fail(FRLAP_EINVAL, "not a bounds-checked build (compile with -DFRLAP_BOUNDS_CHECK)");
#endif
}

frlap_status frlap_set_loop_pass_limit(unsigned max_passes) {
  g_pass_limit.store(max_passes, std::memory_order_relaxed);
  return FRLAP_OK;
}

frlap_status frlap_c_dalpha(int d, double alpha, double* out) {
  if (d != 2 && d != 3) return fail(FRLAP_EINVAL, "d must be 2 or 3");
  if (!(alpha > 0.0 && alpha < 2.0)) return fail(FRLAP_EINVAL, "alpha must lie in (0, 2)");
  if (!out) return fail(FRLAP_EINVAL, "out is NULL");
  *out = c_dalpha_host(d, alpha);
  return FRLAP_OK;
}

frlap_status frlap_coeffs(int d, double alpha, double gamma, double h, const int* N, double* d_coeffs,
                          void* stream) {
  frlap_status rc = check_params(d, alpha, gamma, h, N);
  if (rc != FRLAP_OK) return rc;
  if (!d_coeffs) return fail(FRLAP_EINVAL, "d_coeffs is NULL");
  int Nmax = 0;
  for (int r = 0; r < d; ++r) Nmax = N[r] > Nmax ? N[r] : Nmax;
  cudaStream_t s = (cudaStream_t)stream;
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, coeffs_scratch_bytes(d, Nmax), s);
  if (e != cudaSuccess) return fail(FRLAP_ENOMEM, "frlap_coeffs: scratch allocation failed");
  e = coeffs_launch(d, alpha, gamma, h, Nmax, d_coeffs, scratch, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_coeffs kernels");
  if (e2 != cudaSuccess) return cuda_fail(e2, "frlap_coeffs free");
  return FRLAP_OK;
}

frlap_status frlap_plan_destroy(frlap_plan* plan) {
  if (!plan) return FRLAP_OK;
  cudaFree(plan->lam64);
  cudaFree(plan->lamL64);
  cudaFree(plan->lam32);
  cudaFree(plan->mu_strang);
  cudaFree(plan->mu_learned);
  cudaFree(plan->mu_tau);
  cudaFree(plan->lamdf);
  for (int r = 0; r < 3; ++r) {
    cudaFree(plan->tw64[r]);
    cudaFree(plan->tw32[r]);
    cudaFree(plan->twdf[r]);
  }
  if (plan->side) cudaStreamDestroy(plan->side);
  delete plan;
  return FRLAP_OK;
}

frlap_status frlap_plan_create(int d, double alpha, double gamma, double h, const int* N, int prec,
                               void* stream, frlap_plan** out) {
  frlap_status rc = check_params(d, alpha, gamma, h, N);
  if (rc != FRLAP_OK) return rc;
  if (!out) return fail(FRLAP_EINVAL, "out is NULL");
  if (prec < FRLAP_F64 || prec > FRLAP_MIXED_DF64) return fail(FRLAP_EINVAL, "unknown precision");
  *out = nullptr;
  frlap_plan* p = new (std::nothrow) frlap_plan();
  if (!p) return fail(FRLAP_ENOMEM, "host allocation failed");
  p->d = d;
  p->alpha = alpha;
  p->gamma = gamma;
  p->h = h;
  p->prec = prec;
  p->df64 = (prec == FRLAP_DF64 || prec == FRLAP_MIXED_DF64);
  p->c = c_dalpha_host(d, alpha);
  p->Nmax = 0;
  p->M = 1;
  p->lam_count = 1;
  for (int r = 0; r < 3; ++r) {
    if (r < d) {
      p->N[r] = N[r];
      p->n[r] = N[r] - 1;
      int Pr = 1 << ilog2(2 * p->n[r] - 1);
      if (Pr < 32) Pr = 32;
      p->P[r] = Pr;
      p->logP[r] = ilog2(Pr);
      p->Nmax = N[r] > p->Nmax ? N[r] : p->Nmax;
      p->M *= (size_t)p->n[r];
      p->lam_count *= (size_t)(Pr / 2 + 1);
    } else {
      p->N[r] = 2;
      p->n[r] = 1;
      p->P[r] = 1;
      p->logP[r] = 0;
    }
  }
  const int Hx1 = p->P[0] / 2 + 1;
  const size_t nrows = (size_t)p->n[1] * (d == 3 ? p->n[2] : 1);
  p->s1_elems = (size_t)Hx1 * nrows;
  // 3D: the transposed y spectra; 2D with a 16384-point y embedding: the even half of the split
  // middle stage (same layout as S1)
  p->s2_elems = (d == 3) ? (size_t)Hx1 * p->P[1] * p->n[2] : (p->P[1] > kMaxLine ? p->s1_elems : 0);

  cudaStream_t s = (cudaStream_t)stream;
  double* coef = nullptr;
  void* scratch = nullptr;
  const size_t N1 = (size_t)p->Nmax + 1;
  const size_t ncoef = (d == 2) ? N1 * N1 : N1 * N1 * N1;
  auto cleanup = [&](frlap_status code, const std::string& msg) {
    cudaStreamSynchronize(s);
    if (coef) cudaFree(coef);
    if (scratch) cudaFree(scratch);
    frlap_plan_destroy(p);
    return fail(code, msg);
  };
  if (cudaMalloc(&coef, ncoef * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&scratch, coeffs_scratch_bytes(d, p->Nmax)) != cudaSuccess ||
      cudaMalloc(&p->lam64, p->lam_count * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&p->lamL64, p->lam_count * sizeof(double)) != cudaSuccess)
    return cleanup(FRLAP_ENOMEM, "plan allocation failed");
  if (prec != FRLAP_F64 && cudaMalloc(&p->lam32, p->lam_count * sizeof(float)) != cudaSuccess)
    return cleanup(FRLAP_ENOMEM, "plan allocation failed");
  for (int r = 0; r < d; ++r) {
    const int ntw = twiddle_entries(p->P[r]);
    if (cudaMalloc(&p->tw64[r], ntw * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&p->tw32[r], ntw * sizeof(float2)) != cudaSuccess)
      return cleanup(FRLAP_ENOMEM, "plan allocation failed");
    cudaError_t e = twiddle_launch(p->P[r], p->tw64[r], p->tw32[r], s);
    if (e != cudaSuccess) return cleanup(FRLAP_ECUDA, std::string("twiddles: ") + cudaGetErrorString(e));
    if (p->df64) {
      if (cudaMalloc(&p->twdf[r], ntw * sizeof(cdf)) != cudaSuccess)
        return cleanup(FRLAP_ENOMEM, "plan allocation failed");
      e = to_cdf_launch(p->tw64[r], p->twdf[r], (size_t)ntw, s);
      if (e != cudaSuccess) return cleanup(FRLAP_ECUDA, std::string("twiddles: ") + cudaGetErrorString(e));
    }
  }
  cudaError_t e = coeffs_launch(d, alpha, gamma, h, p->Nmax, coef, scratch, s);
  if (e != cudaSuccess) return cleanup(FRLAP_ECUDA, std::string("coefficients: ") + cudaGetErrorString(e));
  e = symbol_launch(*p, coef, p->lam64, s);
  if (e != cudaSuccess) return cleanup(FRLAP_ECUDA, std::string("symbol: ") + cudaGetErrorString(e));
  double scale = 1.0;
  for (int r = 0; r < d; ++r) scale /= (double)p->P[r];
  e = scale_symbol_launch(p->lam64, nullptr, p->lam_count, scale, s);
  if (e != cudaSuccess) return cleanup(FRLAP_ECUDA, std::string("symbol scale: ") + cudaGetErrorString(e));
  e = line_symbol_launch<double>(*p, p->lam64, p->lamL64, 1.0, s);
  if (e == cudaSuccess && p->lam32) e = line_symbol_launch<float>(*p, p->lam64, p->lam32, 1.0, s);
  if (e != cudaSuccess) return cleanup(FRLAP_ECUDA, std::string("symbol copy: ") + cudaGetErrorString(e));
  if (p->df64) {
    if (cudaMalloc(&p->lamdf, p->lam_count * sizeof(dfl)) != cudaSuccess)
      return cleanup(FRLAP_ENOMEM, "plan allocation failed");
    e = line_symbol_launch<dfl>(*p, p->lam64, p->lamdf, 1.0, s);
    if (e != cudaSuccess) return cleanup(FRLAP_ECUDA, std::string("symbol copy: ") + cudaGetErrorString(e));
  }
  e = cudaStreamSynchronize(s);
  cudaFree(coef);
  cudaFree(scratch);
  coef = nullptr;
  scratch = nullptr;
  if (e != cudaSuccess) {
    frlap_plan_destroy(p);
    return cuda_fail(e, "plan creation");
  }
  *out = p;
  return FRLAP_OK;
}

size_t frlap_workspace_bytes(const frlap_plan* plan, int op) {
  if (!plan) return 0;
  const int eb = (plan->prec == FRLAP_F32) ? 4 : 8;
  switch (op) {
    case FRLAP_OP_APPLY: {
      size_t b = apply_work_bytes(*plan, eb);
      if (plan->prec != FRLAP_F32) b = apply_work_bytes(*plan, 8);
      return b;
    }
    case FRLAP_OP_PCG:
      return pcg_work_bytes(*plan);
    case FRLAP_OP_AC:
      return ac_work_bytes(*plan);
    default:
      return 0;
  }
}

frlap_status frlap_plan_shape(const frlap_plan* plan, int* n, int* P) {
  if (!plan) return fail(FRLAP_EINVAL, "plan is NULL");
  for (int r = 0; r < plan->d; ++r) {
    if (n) n[r] = plan->n[r];
    if (P) P[r] = plan->P[r];
  }
  return FRLAP_OK;
}

frlap_status frlap_plan_symbol(const frlap_plan* plan, double* d_lambda, void* stream) {
  if (!plan || !d_lambda) return fail(FRLAP_EINVAL, "plan or d_lambda is NULL");
  FRLAP_CUDA_TRY(cudaMemcpyAsync(d_lambda, plan->lam64, plan->lam_count * sizeof(double),
                                 cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return FRLAP_OK;
}

static frlap_status check_work(void* d_work) {
  if (!d_work) return fail(FRLAP_EWORKSPACE, "d_work is NULL");
  if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0) return fail(FRLAP_EWORKSPACE, "d_work is not 256-byte aligned");
  return FRLAP_OK;
}

frlap_status frlap_apply(const frlap_plan* plan, const void* d_u, void* d_y, void* d_work, void* stream) {
  if (!plan || !d_u || !d_y) return fail(FRLAP_EINVAL, "plan, d_u or d_y is NULL");
  if (ranges_overlap(d_u, d_y, vector_bytes(*plan, plan->prec == FRLAP_F32)))
    return fail(FRLAP_EINVAL, "d_u and d_y must not overlap");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  cudaError_t e;
  if (plan->prec == FRLAP_F32)
    e = apply_launch<float>(*plan, (const float*)d_u, (float*)d_y, d_work, (cudaStream_t)stream, nullptr);
  else
    e = apply64(*plan, (const double*)d_u, (double*)d_y, d_work, (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_apply");
  return FRLAP_OK;
}

int frlap_apply_nstages(const frlap_plan* plan) { return plan ? (plan->d == 2 ? 3 : 5) : 0; }

size_t frlap_apply_batch_workspace_bytes(const frlap_plan* plan, int nbatch) {
  if (!plan || nbatch < 1) return 0;
  return (size_t)nbatch * frlap_workspace_bytes(plan, FRLAP_OP_APPLY);
}

frlap_status frlap_apply_batch(const frlap_plan* plan, int nbatch, const void* d_u, void* d_y, void* d_work,
                               void* stream, void* const* events) {
  if (!plan || !d_u || !d_y) return fail(FRLAP_EINVAL, "plan, d_u or d_y is NULL");
  if (nbatch < 1 || nbatch > 65535) return fail(FRLAP_EINVAL, "nbatch must be in 1..65535");
  const size_t bytes = (size_t)nbatch * plan->M * (plan->prec == FRLAP_F32 ? 4 : 8);
  const uintptr_t u0 = reinterpret_cast<uintptr_t>(d_u), y0 = reinterpret_cast<uintptr_t>(d_y);
  if (u0 < y0 + bytes && y0 < u0 + bytes) return fail(FRLAP_EINVAL, "d_u and d_y must not overlap");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  cudaEvent_t const* ev = reinterpret_cast<cudaEvent_t const*>(events);
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (plan->prec == FRLAP_F32)
    e = apply_batch_launch<float>(*plan, nbatch, (const float*)d_u, (float*)d_y, plan->M, d_work, s, nullptr, 0,
                                  nullptr, 0, ev);
  else if (plan->df64)
    e = apply_batch_launch<dfl>(*plan, nbatch, (const double*)d_u, (double*)d_y, plan->M, d_work, s, nullptr, 0,
                                nullptr, 0, ev);
  else
    e = apply_batch_launch<double>(*plan, nbatch, (const double*)d_u, (double*)d_y, plan->M, d_work, s, nullptr, 0,
                                   nullptr, 0, ev);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_apply_batch");
  return FRLAP_OK;
}

size_t frlap_autotune_workspace_bytes(const frlap_plan* plan, int nbatch) {
  if (!plan || nbatch < 1) return 0;
  return 2 * align256((size_t)nbatch * plan->M * 8) + (size_t)nbatch * apply_work_bytes(*plan, 8);
}

frlap_status frlap_plan_autotune(frlap_plan* plan, int nbatch, void* d_work, void* stream, int* chosen) {
  if (!plan) return fail(FRLAP_EINVAL, "plan is NULL");
  if (nbatch < 1 || nbatch > 65535) return fail(FRLAP_EINVAL, "nbatch must be in 1..65535");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  unsigned char* w = reinterpret_cast<unsigned char*>(d_work);
  void* u = w;
  void* y = w + align256((size_t)nbatch * plan->M * 8);
  void* work = w + 2 * align256((size_t)nbatch * plan->M * 8);
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  const int p = plan->prec;
  if (p == FRLAP_F64 || p == FRLAP_MIXED)
    e = autotune_engine<double>(*plan, nbatch, (double*)u, (double*)y, work, s);
  else if (p == FRLAP_DF64 || p == FRLAP_MIXED_DF64)
    e = autotune_engine<dfl>(*plan, nbatch, (double*)u, (double*)y, work, s);
  if (e == cudaSuccess && p != FRLAP_F64 && p != FRLAP_DF64)
    e = autotune_engine<float>(*plan, nbatch, (float*)u, (float*)y, work, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_plan_autotune");
  if (chosen) {
    const int e64 = plan->df64 ? 2 : 1;
    for (int st = 0; st < 5; ++st) {
      chosen[st] = plan->tl_tuned[e64][st];
      chosen[5 + st] = plan->tl_tuned[0][st];
    }
  }
  return FRLAP_OK;
}

// Host-buffer batch: two device slots, each holding `chunk` input and output vectors and the
// batched apply workspace of one chunk (the slots compute on two streams).
static size_t host_slot_bytes(const frlap_plan* plan, int chunk) {
  const size_t vb = (size_t)chunk * plan->M * (plan->prec == FRLAP_F32 ? 4 : 8);
  return 2 * align256(vb) + align256(frlap_apply_batch_workspace_bytes(plan, chunk));
}

// device slots of frlap_apply_host (input, output and apply workspace for one chunk each): three, so that
// the copy in of chunk c+2 and the copy out of chunk c-1 overlap the apply of chunk c
constexpr int kHostSlots = 3;

size_t frlap_apply_host_workspace_bytes(const frlap_plan* plan, int chunk) {
  if (!plan || chunk < 1) return 0;
  return kHostSlots * host_slot_bytes(plan, chunk);
}

frlap_status frlap_apply_host(const frlap_plan* plan, int nbatch, int chunk, const void* h_u, void* h_y,
                              void* d_work, void* stream) {
  if (!plan || !h_u || !h_y) return fail(FRLAP_EINVAL, "plan, h_u or h_y is NULL");
  if (nbatch < 1 || chunk < 1 || chunk > 65535) return fail(FRLAP_EINVAL, "need nbatch >= 1 and chunk in 1..65535");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  const size_t eb = plan->prec == FRLAP_F32 ? 4 : 8;
  const size_t vbytes = plan->M * eb;
  if (ranges_overlap(h_u, h_y, (size_t)nbatch * vbytes)) return fail(FRLAP_EINVAL, "h_u and h_y must not overlap");
  unsigned char* w = reinterpret_cast<unsigned char*>(d_work);
  unsigned char* du[kHostSlots];
  unsigned char* dy[kHostSlots];
  void* awork[kHostSlots];
  for (int k = 0; k < kHostSlots; ++k) {
    du[k] = w + k * host_slot_bytes(plan, chunk);
    dy[k] = du[k] + align256((size_t)chunk * vbytes);
    awork[k] = dy[k] + align256((size_t)chunk * vbytes);
  }
  const cudaStream_t cs = (cudaStream_t)stream;
  // Chunk boundaries: with chunks of more than one vector the first and the last chunk hold one vector,
  // so the pipeline fills (first copy in) and drains (last copy out) at the cost of one vector's copy.
  std::vector<int> c0, cn;  // first vector and count of each chunk
  {
    int v = 0;
    const bool ends = chunk > 1 && nbatch > 2;
    if (ends) {
      c0.push_back(0);
      cn.push_back(1);
      v = 1;
    }
    while (v < nbatch) {
      int nb = nbatch - v < chunk ? nbatch - v : chunk;
      if (ends && v + nb == nbatch && nb > 1) --nb;  // leave one vector for the last chunk
      c0.push_back(v);
      cn.push_back(nb);
      v += nb;
    }
  }
  const int nchunks = (int)c0.size();
  // chunk c uses slot c mod kHostSlots and computes on comp[c mod 2] (comp[0] = the caller's stream): the
  // kernels of consecutive chunks overlap, filling each other's last partial wave
  cudaStream_t sin = nullptr, sout = nullptr, c1 = nullptr;
  // in[k]: slot k's input has arrived; done[k]: slot k's apply finished; out[k]: slot k's output copied
  cudaEvent_t in[kHostSlots] = {}, done[kHostSlots] = {}, out[kHostSlots] = {};
  cudaError_t e = cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c1, cudaStreamNonBlocking);
  const cudaStream_t comp[2] = {cs, c1};
  for (int k = 0; k < kHostSlots && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&out[k], cudaEventDisableTiming);
  }
  // the internal streams start after the caller's earlier work on `stream`
  if (e == cudaSuccess) e = cudaEventRecord(done[0], cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, done[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, done[0], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c1, done[0], 0);
  auto copy_in = [&](int c) -> cudaError_t {
    const int k = c % kHostSlots;
    const int nb = cn[c];
    cudaError_t r = cudaSuccess;
    if (c >= kHostSlots) r = cudaStreamWaitEvent(sin, done[k], 0);  // slot k's previous apply has read its input
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(du[k], static_cast<const unsigned char*>(h_u) + (size_t)c0[c] * vbytes,
                          (size_t)nb * vbytes, cudaMemcpyHostToDevice, sin);
    if (r == cudaSuccess) r = cudaEventRecord(in[k], sin);
    return r;
  };
  for (int c = 0; c < kHostSlots - 1 && c < nchunks && e == cudaSuccess; ++c) e = copy_in(c);
  for (int c = 0; c < nchunks && e == cudaSuccess; ++c) {
    const int k = c % kHostSlots;
    const int nb = cn[c];
    if (c + kHostSlots - 1 < nchunks) e = copy_in(c + kHostSlots - 1);
    const cudaStream_t ks = comp[c & 1];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, in[k], 0);
    if (e == cudaSuccess && c >= kHostSlots) e = cudaStreamWaitEvent(ks, out[k], 0);  // slot k's output copied out
    if (e == cudaSuccess) {
      if (plan->prec == FRLAP_F32)
        e = apply_batch_launch<float>(*plan, nb, (const float*)du[k], (float*)dy[k], plan->M, awork[k], ks, nullptr,
                                      0, nullptr, 0);
      else if (plan->df64)
        e = apply_batch_launch<dfl>(*plan, nb, (const double*)du[k], (double*)dy[k], plan->M, awork[k], ks, nullptr,
                                    0, nullptr, 0);
      else
        e = apply_batch_launch<double>(*plan, nb, (const double*)du[k], (double*)dy[k], plan->M, awork[k], ks,
                                       nullptr, 0, nullptr, 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(done[k], ks);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, done[k], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<unsigned char*>(h_y) + (size_t)c0[c] * vbytes, dy[k], (size_t)nb * vbytes,
                          cudaMemcpyDeviceToHost, sout);
    if (e == cudaSuccess) e = cudaEventRecord(out[k], sout);
  }
  // `stream` ends after the last copy out; then wait for everything
  for (int k = 0; k < kHostSlots && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(cs, out[k], 0);
  cudaError_t es = cudaStreamSynchronize(cs);
  if (e == cudaSuccess) e = es;
  if (sin) cudaStreamSynchronize(sin);
  if (sout) cudaStreamSynchronize(sout);
  if (c1) cudaStreamSynchronize(c1);
  for (int k = 0; k < kHostSlots; ++k) {
    if (in[k]) cudaEventDestroy(in[k]);
    if (done[k]) cudaEventDestroy(done[k]);
    if (out[k]) cudaEventDestroy(out[k]);
  }
  if (sin) cudaStreamDestroy(sin);
  if (sout) cudaStreamDestroy(sout);
  if (c1) cudaStreamDestroy(c1);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_apply_host");
  return FRLAP_OK;
}

frlap_status frlap_apply_profiled(const frlap_plan* plan, const void* d_u, void* d_y, void* d_work, void* stream,
                                  void* const* events) {
  if (!plan || !d_u || !d_y || !events) return fail(FRLAP_EINVAL, "plan, d_u, d_y or events is NULL");
  if (ranges_overlap(d_u, d_y, vector_bytes(*plan, plan->prec == FRLAP_F32)))
    return fail(FRLAP_EINVAL, "d_u and d_y must not overlap");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  cudaEvent_t const* ev = reinterpret_cast<cudaEvent_t const*>(events);
  cudaError_t e;
  if (plan->prec == FRLAP_F32)
    e = apply_launch<float>(*plan, (const float*)d_u, (float*)d_y, d_work, (cudaStream_t)stream, nullptr, ev);
  else
    e = apply64(*plan, (const double*)d_u, (double*)d_y, d_work, (cudaStream_t)stream, nullptr, ev);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_apply_profiled");
  return FRLAP_OK;
}

frlap_status frlap_apply_f32(const frlap_plan* plan, const float* d_u, float* d_y, void* d_work, void* stream) {
  if (!plan || !d_u || !d_y) return fail(FRLAP_EINVAL, "plan, d_u or d_y is NULL");
  if (plan->prec == FRLAP_F64) return fail(FRLAP_EINVAL, "frlap_apply_f32 needs an F32 or MIXED plan");
  if (ranges_overlap(d_u, d_y, vector_bytes(*plan, true))) return fail(FRLAP_EINVAL, "d_u and d_y must not overlap");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  cudaError_t e = apply_launch<float>(*plan, d_u, d_y, d_work, (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_apply_f32");
  return FRLAP_OK;
}

frlap_status frlap_pcg_solve(const frlap_plan* plan, const double* d_f, double* d_x, double rtol, int maxit,
                             int solver, int precond, double inner_rtol, int* iters, double* relres, void* d_work,
                             void* stream) {
  if (!plan || !d_f || !d_x) return fail(FRLAP_EINVAL, "plan, d_f or d_x is NULL");
  const float* mu = nullptr;
  if (precond == FRLAP_PRECOND_STRANG) {
    if (!plan->mu_strang) return fail(FRLAP_EINVAL, "Strang preconditioner not built (frlap_precond_strang)");
    mu = plan->mu_strang;
  } else if (precond == FRLAP_PRECOND_LEARNED) {
    if (!plan->mu_learned) return fail(FRLAP_EINVAL, "no learned multiplier set (frlap_precond_set_symbol)");
    mu = plan->mu_learned;
  } else if (precond == FRLAP_PRECOND_TAU) {
    if (!plan->mu_tau) return fail(FRLAP_EINVAL, "sine-basis preconditioner not built (frlap_precond_tau)");
    mu = plan->mu_tau;
  } else if (precond != FRLAP_PRECOND_NONE) {
    return fail(FRLAP_EINVAL, "unknown preconditioner");
  }
  if (!(rtol > 0.0) || maxit < 1) return fail(FRLAP_EINVAL, "need rtol > 0 and maxit >= 1");
  if (solver == FRLAP_SOLVE_CG && plan->prec == FRLAP_F32)
    return fail(FRLAP_EINVAL, "FP64 CG needs an F64 or MIXED plan");
  if (solver == FRLAP_SOLVE_IR && plan->prec != FRLAP_MIXED && plan->prec != FRLAP_MIXED_DF64)
    return fail(FRLAP_EINVAL, "iterative refinement needs a MIXED or MIXED_DF64 plan");
  if (solver != FRLAP_SOLVE_CG && solver != FRLAP_SOLVE_IR) return fail(FRLAP_EINVAL, "unknown solver");
  if (solver == FRLAP_SOLVE_IR && !(inner_rtol > 0.0 && inner_rtol < 1.0))
    return fail(FRLAP_EINVAL, "inner_rtol must lie in (0, 1)");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  return pcg_solve_impl(*plan, d_f, d_x, rtol, maxit, solver, mu, inner_rtol, iters, relres, d_work,
                        (cudaStream_t)stream);
}

frlap_status frlap_residual(const frlap_plan* plan, const double* d_f, const double* d_x, double* d_r,
                            double* relres, void* d_work, void* stream) {
  if (!plan || !d_f || !d_x || !relres) return fail(FRLAP_EINVAL, "plan, d_f, d_x or relres is NULL");
  if (plan->prec == FRLAP_F32) return fail(FRLAP_EINVAL, "the residual needs an F64, MIXED or double-float plan");
  const size_t vb = vector_bytes(*plan, false);
  if (d_r && (ranges_overlap(d_r, d_f, vb) || ranges_overlap(d_r, d_x, vb)))
    return fail(FRLAP_EINVAL, "d_r must not overlap d_f or d_x");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  return residual_impl(*plan, d_f, d_x, d_r, relres, d_work, (cudaStream_t)stream);
}

frlap_status frlap_precond_strang(frlap_plan* plan, int* n_nonpositive, void* stream) {
  if (!plan) return fail(FRLAP_EINVAL, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (!plan->mu_strang && cudaMalloc(&plan->mu_strang, plan->lam_count * sizeof(float)) != cudaSuccess)
    return fail(FRLAP_ENOMEM, "Strang symbol allocation failed");
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, strang_scratch_bytes(*plan), s) != cudaSuccess)
    return fail(FRLAP_ENOMEM, "Strang scratch allocation failed");
  unsigned bad = 0;
  cudaError_t e = strang_build(*plan, scratch, s, &bad);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_precond_strang");
  if (n_nonpositive) *n_nonpositive = (int)bad;
  return FRLAP_OK;
}

frlap_status frlap_precond_tau(frlap_plan* plan, int* n_nonpositive, void* stream) {
  if (!plan) return fail(FRLAP_EINVAL, "plan is NULL");
  for (int r = 0; r < plan->d; ++r)
    if (plan->P[r] != 2 * plan->N[r] || plan->P[r] > kMaxLine)
      return fail(FRLAP_EINVAL, "the sine-basis preconditioner needs every N[r] a power of two of at least 16 "
                                "(and at most 4096)");
  cudaStream_t s = (cudaStream_t)stream;
  if (!plan->mu_tau && cudaMalloc(&plan->mu_tau, plan->lam_count * sizeof(float)) != cudaSuccess)
    return fail(FRLAP_ENOMEM, "sine-basis multiplier allocation failed");
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, tau_scratch_bytes(*plan), s) != cudaSuccess)
    return fail(FRLAP_ENOMEM, "sine-basis scratch allocation failed");
  unsigned bad = 0;
  cudaError_t e = tau_build(*plan, scratch, s, &bad);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_precond_tau");
  if (n_nonpositive) *n_nonpositive = (int)bad;
  return FRLAP_OK;
}

frlap_status frlap_precond_apply(const frlap_plan* plan, int precond, const float* d_r, float* d_z, void* d_work,
                                 void* stream) {
  if (!plan || !d_r || !d_z) return fail(FRLAP_EINVAL, "plan, d_r or d_z is NULL");
  if (ranges_overlap(d_r, d_z, vector_bytes(*plan, true))) return fail(FRLAP_EINVAL, "d_r and d_z must not overlap");
  const float* mu = precond == FRLAP_PRECOND_STRANG    ? plan->mu_strang
                    : precond == FRLAP_PRECOND_LEARNED ? plan->mu_learned
                    : precond == FRLAP_PRECOND_TAU     ? plan->mu_tau
                                                       : nullptr;
  if (!mu) return fail(FRLAP_EINVAL, "preconditioner not available on this plan");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  cudaError_t e = apply_launch<float>(*plan, d_r, d_z, d_work, (cudaStream_t)stream, nullptr, nullptr, mu,
                                      precond == FRLAP_PRECOND_TAU);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_precond_apply");
  return FRLAP_OK;
}

frlap_status frlap_mlp_multiplier(const frlap_plan* plan, const float* d_params, double* d_m, void* stream) {
  if (!plan || !d_params || !d_m) return fail(FRLAP_EINVAL, "plan, d_params or d_m is NULL");
  cudaError_t e = mlp_multiplier_launch(*plan, d_params, d_m, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_mlp_multiplier");
  return FRLAP_OK;
}

size_t frlap_learn_workspace_bytes(const frlap_plan* plan, int B) {
  if (!plan || B < 1) return 0;
  return learn_work_bytes(*plan, B);
}

frlap_status frlap_learn_grad(const frlap_plan* plan, const float* d_params, const double* d_r, const double* d_e,
                              int B, float* d_grad, double* d_loss, void* d_work, void* stream) {
  if (!plan || !d_params || !d_r || !d_e || !d_grad || !d_loss) return fail(FRLAP_EINVAL, "NULL argument");
  if (B < 1) return fail(FRLAP_EINVAL, "B must be >= 1");
  if (plan->prec == FRLAP_F32) return fail(FRLAP_EINVAL, "training needs an F64 or MIXED plan (FP64 spectra)");
  for (int r = 0; r < plan->d; ++r)
    if (plan->P[r] > kMaxLine)
      return fail(FRLAP_EINVAL, "training spectra need embeddings of at most 8192 points per axis (2D N <= 4096)");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  cudaError_t e = learn_grad_launch(*plan, d_params, d_r, d_e, B, d_grad, d_loss, d_work, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_learn_grad");
  return FRLAP_OK;
}

frlap_status frlap_adam_step(float* d_params, const float* d_grad, float* d_m1, float* d_m2, int n, float lr,
                             float beta1, float beta2, float eps, int t, void* stream) {
  if (!d_params || !d_grad || !d_m1 || !d_m2 || n < 1 || t < 1) return fail(FRLAP_EINVAL, "bad Adam arguments");
  cudaError_t e = adam_launch(d_params, d_grad, d_m1, d_m2, n, lr, beta1, beta2, eps, t, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_adam_step");
  return FRLAP_OK;
}

frlap_status frlap_cg_pairs(const frlap_plan* plan, const double* d_f, int K, double rtol, double* d_E, double* d_R,
                            int* npairs, void* d_work, void* stream) {
  if (!plan || !d_f || !d_E || !d_R || K < 1 || !(rtol > 0.0)) return fail(FRLAP_EINVAL, "bad arguments");
  if (plan->prec == FRLAP_F32) return fail(FRLAP_EINVAL, "training pairs need an F64 or MIXED plan");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  return cg_pairs_impl(*plan, d_f, K, rtol, d_E, d_R, npairs, d_work, (cudaStream_t)stream);
}

size_t frlap_allen_cahn_batch_workspace_bytes(int nbatch, const frlap_plan* const* plans) {
  if (nbatch < 1 || !plans) return 0;
  for (int i = 0; i < nbatch; ++i)
    if (!plans[i]) return 0;
  return ac_batch_work_bytes(nbatch, plans);
}

frlap_status frlap_allen_cahn_batch(int nbatch, const frlap_plan* const* plans, double* const* d_u, double tau,
                                    double eps, int nsteps, double rtol, int maxit, int* iters, int* status,
                                    void* d_work, void* stream) {
  if (nbatch < 1 || !plans || !d_u) return fail(FRLAP_EINVAL, "need nbatch >= 1, plans and d_u");
  for (int i = 0; i < nbatch; ++i) {
    if (!plans[i] || !d_u[i]) return fail(FRLAP_EINVAL, "NULL plan or d_u entry");
    if (plans[i]->prec == FRLAP_F32) return fail(FRLAP_EINVAL, "Allen-Cahn batch needs F64 or MIXED plans");
  }
  if (!(tau > 0.0) || !(eps > 0.0) || nsteps < 0 || !(rtol > 0.0) || maxit < 1)
    return fail(FRLAP_EINVAL, "need tau > 0, eps > 0, nsteps >= 0, rtol > 0, maxit >= 1");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  return ac_batch_impl(nbatch, plans, d_u, tau, eps, nsteps, rtol, maxit, iters, status, d_work,
                       (cudaStream_t)stream);
}

frlap_status frlap_precond_set_symbol(frlap_plan* plan, const double* d_m, void* stream) {
  if (!plan || !d_m) return fail(FRLAP_EINVAL, "plan or d_m is NULL");
  if (!plan->mu_learned && cudaMalloc(&plan->mu_learned, plan->lam_count * sizeof(float)) != cudaSuccess)
    return fail(FRLAP_ENOMEM, "multiplier allocation failed");
  double scale = 1.0;
  for (int r = 0; r < plan->d; ++r) scale /= (double)plan->P[r];
  cudaError_t e = line_symbol_launch<float>(*plan, d_m, plan->mu_learned, scale, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_precond_set_symbol");
  return FRLAP_OK;
}

frlap_status frlap_allen_cahn_step(const frlap_plan* plan, double* d_u, double tau, double eps, int nsteps,
                                   double rtol, int* iters, void* d_work, void* stream) {
  if (!plan || !d_u) return fail(FRLAP_EINVAL, "plan or d_u is NULL");
  if (plan->prec == FRLAP_F32) return fail(FRLAP_EINVAL, "Allen-Cahn steps need an F64 or MIXED plan");
  if (!(tau > 0.0) || !(eps > 0.0) || nsteps < 0 || !(rtol > 0.0))
    return fail(FRLAP_EINVAL, "need tau > 0, eps > 0, nsteps >= 0, rtol > 0");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  return allen_cahn_impl(*plan, d_u, tau, eps, nsteps, rtol, iters, d_work, (cudaStream_t)stream);
}

frlap_status frlap_allen_cahn_cn(const frlap_plan* plan, double* d_ubar, double tau, double delta, int nsteps,
                                 double rtol, int* iters, double* h_mass, void* d_work, void* stream) {
  if (!plan || !d_ubar) return fail(FRLAP_EINVAL, "plan or d_ubar is NULL");
  if (plan->prec == FRLAP_F32) return fail(FRLAP_EINVAL, "Allen-Cahn steps need an F64, DF64 or MIXED plan");
  if (!(tau > 0.0) || !(delta > 0.0) || nsteps < 0 || !(rtol > 0.0))
    return fail(FRLAP_EINVAL, "need tau > 0, delta > 0, nsteps >= 0, rtol > 0");
  frlap_status rc = check_work(d_work);
  if (rc != FRLAP_OK) return rc;
  return allen_cahn_cn_impl(*plan, d_ubar, tau, delta, nsteps, rtol, iters, h_mass, d_work, (cudaStream_t)stream);
}

}  // extern "C"
