// Many semi-implicit Allen-Cahn instances in one CUDA-graph launch.
//
// Every instance i (its own plan: alpha, grid) advances nsteps steps of
//   (I + tau eps^2 A_i) u^{n+1} = u^n + tau (u^n - (u^n)^3),
// each step solved by CG to ||r|| <= rtol ||rhs|| (at most maxit iterations), the
// first from x0 = 0 and every later one from the previous step's solution.  Instances of the same shape form a group whose vectors are
// stacked, so each kernel below handles a whole group (blockIdx.y = instance).
//
// Control flow lives on the device.  The graph is one conditional WHILE node whose
// body runs one CG iteration for every instance that is still solving, then an
// `advance` kernel that, for each instance whose solve has just ended, copies the
// solution into u and sets up the next step (or marks the instance finished),
// then a kernel that keeps the loop going while any instance is unfinished.  The
// loop count is bounded: each solve stops after maxit iterations, and the control
// kernel also stops the loop after nsteps * (maxit + 2) + 8 passes (or the lower limit set by
// frlap_set_loop_pass_limit), reporting FRLAP_ETIMEOUT.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace frlap {

namespace {

constexpr int kAcBlocks = 32;  // blocks per instance for the vector kernels
constexpr int kAcThreads = 256;

struct AcState {
  double rr, pq, alpha, beta, tol2;
  int done;      // the current solve has ended (converged or maxit)
  int fresh;     // no solve has run yet (u^0 is current)
  int finished;  // all steps done
  int step;      // completed steps
  int iters;     // CG iterations of the current solve
  int iters_total;
  int status;    // FRLAP_ENOCONV if some solve hit maxit
  unsigned counter;
  int pad_;
};
static_assert(sizeof(AcState) % sizeof(int) == 0, "state stride in ints");

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

// per-instance reduction over the instance's blocks; true in thread 0 of its last block
__device__ __forceinline__ bool inst_sum(double v, double* partials, unsigned* counter, double* total) {
  __shared__ double red[32];
  __shared__ bool last;
  const double s = bsum(v, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += *((volatile double*)&partials[i]);
  const double tot = bsum(t, red);
  if (threadIdx.x == 0) {
    *total = tot;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

#define INST_LOOP(i, n) for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)
// The iteration kernels take kU elements per thread and pass, one grid apart, all loaded before any
// arithmetic (several loads in flight per warp; see the CG kernels); the u-th is base + u * gstride.
constexpr int kU = 4;
#define INST_LOOP_U(base, n)                                                                                 \
  for (size_t base = (size_t)blockIdx.x * blockDim.x + threadIdx.x, gstride = (size_t)gridDim.x * blockDim.x; \
       base < (n); base += kU * gstride)

// two per-instance sums (partial arrays pa, pb); true in thread 0 of the instance's last block
__device__ __forceinline__ bool inst_sum2(double a, double b, double* pa, double* pb, unsigned* counter,
                                          double* ta, double* tb) {
  __shared__ double red[32];
  __shared__ bool last;
  const double sa = bsum(a, red);
  const double sb = bsum(b, red);
  if (threadIdx.x == 0) {
    pa[blockIdx.x] = sa;
    pb[blockIdx.x] = sb;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  double xa = 0.0, xb = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    xa += *((volatile double*)&pa[i]);
    xb += *((volatile double*)&pb[i]);
  }
  const double va = bsum(xa, red);
  const double vb = bsum(xb, red);
  if (threadIdx.x == 0) {
    *ta = va;
    *tb = vb;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

// Start of a solve.  The first step: rhs = u + tau (u - u^3), x = 0, r = p = rhs.  After a solve:
// u <- x, and the next step starts from x = u^{n+1} itself (warm start).  Its initial residual
// needs no apply: the finished solve's recursive residual is r = rhs_old - B x, so
// rhs_new - B x = rhs_new - rhs_old + r, with rhs_old recomputed from the old u.
__global__ void k_ac_advance(double* u, double* x, double* r, double* p, size_t M, size_t vs, AcState* S,
                             double* partials, double* partials2, int nsteps, double tau, double rtol) {
  const int b = blockIdx.y;
  AcState* st = S + b;
  if (!st->done || st->finished) return;
  const bool fresh = st->fresh != 0;
  const bool last_step = !fresh && st->step + 1 >= nsteps;
  u += b * vs;
  x += b * vs;
  r += b * vs;
  p += b * vs;
  double acc_r = 0.0, acc_h = 0.0;
  INST_LOOP(i, M) {
    if (fresh) {
      const double v = u[i];
      const double rh = v + tau * (v - v * v * v);
      x[i] = 0.0;
      r[i] = rh;
      p[i] = rh;
      acc_r += rh * rh;
      acc_h += rh * rh;
    } else {
      const double uo = u[i], v = x[i];
      u[i] = v;
      if (!last_step) {
        const double rh_old = uo + tau * (uo - uo * uo * uo);
        const double rh = v + tau * (v - v * v * v);
        const double r0 = rh - rh_old + r[i];
        r[i] = r0;
        p[i] = r0;
        acc_r += r0 * r0;
        acc_h += rh * rh;
      }
    }
  }
  double tot_r, tot_h;
  if (inst_sum2(acc_r, acc_h, partials + (size_t)b * gridDim.x, partials2 + (size_t)b * gridDim.x, &st->counter,
                &tot_r, &tot_h)) {
    if (!fresh) st->step += 1;
    st->fresh = 0;
    if (st->step >= nsteps) {
      st->finished = 1;
    } else {
      st->rr = tot_r;
      st->tol2 = rtol * rtol * tot_h;
      st->iters = 0;
      st->done = (tot_r <= st->tol2) ? 1 : 0;
    }
  }
}

// q <- p + s q ; pq ; alpha
__global__ void k_ac_pq(const double* __restrict__ p, double* q, size_t M, size_t vs, AcState* S, double* partials,
                        double s) {
  const int b = blockIdx.y;
  AcState* st = S + b;
  if (st->done) return;
  p += b * vs;
  q += b * vs;
  double acc = 0.0;
  INST_LOOP_U(b0, M) {
    double pv[kU], qv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < M) {
        pv[u] = p[i];
        qv[u] = q[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < M) {
        const double qi = pv[u] + s * qv[u];
        q[i] = qi;
        acc += pv[u] * qi;
      }
    }
  }
  double tot;
  if (inst_sum(acc, partials + (size_t)b * gridDim.x, &st->counter, &tot)) {
    st->pq = tot;
    if (!(tot > 0.0) || !isfinite(tot)) {
      st->status = isfinite(tot) ? FRLAP_EBREAKDOWN : FRLAP_ENAN;
      st->done = 1;
    } else {
      st->alpha = st->rr / tot;
    }
  }
}

// x += alpha p ; r -= alpha q ; convergence / maxit ; beta
__global__ void k_ac_update(double* x, double* r, const double* __restrict__ p, const double* __restrict__ q, size_t M,
                            size_t vs, AcState* S, double* partials, int maxit) {
  const int b = blockIdx.y;
  AcState* st = S + b;
  if (st->done) return;
  x += b * vs;
  r += b * vs;
  p += b * vs;
  q += b * vs;
  const double al = st->alpha;
  double acc = 0.0;
  INST_LOOP_U(b0, M) {
    double xv[kU], rv[kU], pv[kU], qv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < M) {
        xv[u] = x[i];
        rv[u] = r[i];
        pv[u] = p[i];
        qv[u] = q[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < M) {
        x[i] = xv[u] + al * pv[u];
        const double ri = rv[u] - al * qv[u];
        r[i] = ri;
        acc += ri * ri;
      }
    }
  }
  double tot;
  if (inst_sum(acc, partials + (size_t)b * gridDim.x, &st->counter, &tot)) {
    st->beta = tot / st->rr;
    st->rr = tot;
    st->iters += 1;
    st->iters_total += 1;
    if (!isfinite(tot)) {
      st->status = FRLAP_ENAN;
      st->done = 1;
    } else if (tot <= st->tol2) {
      st->done = 1;
    } else if (st->iters >= maxit) {
      st->status = FRLAP_ENOCONV;
      st->done = 1;
    }
  }
}

__global__ void k_ac_dir(const double* __restrict__ r, double* p, size_t M, size_t vs, const AcState* S) {
  const int b = blockIdx.y;
  if (S[b].done) return;
  r += b * vs;
  p += b * vs;
  const double be = S[b].beta;
  INST_LOOP_U(b0, M) {
    double rv[kU], pv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < M) {
        rv[u] = r[i];
        pv[u] = p[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const size_t i = b0 + u * gstride;
      if (i < M) p[i] = rv[u] + be * pv[u];
    }
  }
}

// keep looping while an instance is unfinished; bounded by max_passes
__global__ void k_ac_control(const AcState* S, int n, unsigned* passes, unsigned max_passes, int* timeout,
                             cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!S[i].finished) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned c = *passes + 1u;
    *passes = c;
    int go = any;
    if (go && c >= max_passes) {
      *timeout = 1;
      go = 0;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

__global__ void k_ac_reset(AcState* S, int n, unsigned* passes, int* timeout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *passes = 0u;
    *timeout = 0;
  }
  if (i >= n) return;
  AcState s = {};
  s.done = 1;
  s.fresh = 1;
  S[i] = s;
}

struct Group {
  const Plan* plan;     // shape representative
  std::vector<int> idx; // instances (indices into the caller's arrays)
  size_t M, vs, work_stride;  // unknowns per instance, stride between stacked instances
  double* lam;          // [B][lam_count]
  double* u;            // [B][M] each: u, x, r, p, q
  double* x;
  double* r;
  double* p;
  double* q;
  void* awork;          // [B][apply work]
  double* partials;     // [B][kAcBlocks]
  double* partials2;    // [B][kAcBlocks] (the second sum of k_ac_advance)
  AcState* S;           // points into the global state array
};

bool same_shape(const Plan& a, const Plan& b) {
  if (a.d != b.d || a.df64 != b.df64) return false;
  for (int r = 0; r < a.d; ++r)
    if (a.n[r] != b.n[r] || a.P[r] != b.P[r]) return false;
  return true;
}

std::vector<Group> make_groups(int nb, const frlap_plan* const* plans) {
  std::vector<Group> g;
  for (int i = 0; i < nb; ++i) {
    bool placed = false;
    for (auto& gr : g)
      if (same_shape(*gr.plan, *plans[i])) {
        gr.idx.push_back(i);
        placed = true;
        break;
      }
    if (!placed) {
      Group ng{};
      ng.plan = plans[i];
      ng.idx.push_back(i);
      g.push_back(ng);
    }
  }
  return g;
}

// the group's batched apply through its FP64 engine; lam holds the stacked symbols in that engine's type
cudaError_t batch_apply(const Plan& p, int B, const double* u, double* y, size_t vs, void* work, cudaStream_t s,
                        const int* skip, int skip_stride, const double* lam, size_t lam_stride) {
  if (p.df64)
    return apply_batch_launch<dfl>(p, B, u, y, vs, work, s, skip, skip_stride, reinterpret_cast<const dfl*>(lam),
                                   lam_stride);
  return apply_batch_launch<double>(p, B, u, y, vs, work, s, skip, skip_stride, lam, lam_stride);
}

size_t group_bytes(const Group& g) {
  const Plan& p = *g.plan;
  const size_t B = g.idx.size();
  return B * (align256(p.lam_count * 8) + 5 * align256(p.M * 8) + apply_work_bytes(p, 8) +
              2 * align256(kAcBlocks * sizeof(double)));
}

}  // namespace

size_t ac_batch_work_bytes(int nb, const frlap_plan* const* plans) {
  size_t b = align256((size_t)nb * sizeof(AcState)) + 512;
  for (auto& g : make_groups(nb, plans)) b += group_bytes(g);
  return b;
}

frlap_status ac_batch_impl(int nb, const frlap_plan* const* plans, double* const* u, double tau, double eps,
                           int nsteps, double rtol, int maxit, int* iters_out, int* status_out, void* work,
                           cudaStream_t user) {
  std::vector<Group> groups = make_groups(nb, plans);
  unsigned char* w = reinterpret_cast<unsigned char*>(work);
  AcState* S_all = reinterpret_cast<AcState*>(w);
  w += align256((size_t)nb * sizeof(AcState));
  unsigned* passes = reinterpret_cast<unsigned*>(w);
  int* timeout = reinterpret_cast<int*>(w + 256);
  w += 512;
  int soff = 0;
  for (auto& g : groups) {
    const Plan& p = *g.plan;
    const size_t B = g.idx.size();
    g.M = p.M;
    g.work_stride = apply_work_bytes(p, 8);
    g.lam = reinterpret_cast<double*>(w);
    w += B * align256(p.lam_count * 8);
    double* vecs = reinterpret_cast<double*>(w);
    const size_t vs = align256(p.M * 8) / 8;  // stride between instances in doubles
    g.u = vecs;
    g.x = vecs + 1 * B * vs;
    g.r = vecs + 2 * B * vs;
    g.p = vecs + 3 * B * vs;
    g.q = vecs + 4 * B * vs;
    g.vs = vs;
    w += 5 * B * align256(p.M * 8);
    g.awork = w;
    w += B * g.work_stride;
    g.partials = reinterpret_cast<double*>(w);
    w += B * align256(kAcBlocks * sizeof(double));
    g.partials2 = reinterpret_cast<double*>(w);
    w += B * align256(kAcBlocks * sizeof(double));
    g.S = S_all + soff;
    soff += (int)B;
  }
  // the graph runs on its own stream, ordered after the caller's work
  cudaStream_t s;
  FRLAP_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t ev0, ev1;
  cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  frlap_status rc = FRLAP_OK;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaStreamDestroy(s);
  };
  do {
    cudaError_t e;
    if ((e = cudaEventRecord(ev0, user)) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev0, 0)) != cudaSuccess) {
      rc = cuda_fail(e, "stream ordering");
      break;
    }
    // stage the inputs and symbols
    for (auto& g : groups) {
      const Plan& p = *g.plan;
      for (size_t k = 0; k < g.idx.size() && e == cudaSuccess; ++k) {
        const frlap_plan* pi = plans[g.idx[k]];
        e = cudaMemcpyAsync(g.u + k * g.vs, u[g.idx[k]], p.M * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(g.lam + k * (align256(p.lam_count * 8) / 8),
                              p.df64 ? static_cast<const void*>(pi->lamdf) : static_cast<const void*>(pi->lamL64),
                              p.lam_count * 8, cudaMemcpyDeviceToDevice, s);
      }
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "staging copies");
      break;
    }
    k_ac_reset<<<(nb + 255) / 256, 256, 0, s>>>(S_all, nb, passes, timeout);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      rc = cuda_fail(e, "k_ac_reset");
      break;
    }
    // set the kernel attributes before capture (the first apply does it)
    for (auto& g : groups) {
      const Plan& p = *g.plan;
      e = batch_apply(p, (int)g.idx.size(), g.p, g.q, g.vs, g.awork, s, &g.S[0].done,
                      (int)(sizeof(AcState) / sizeof(int)), g.lam, align256(p.lam_count * 8) / 8);
      if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "batched apply");
      break;
    }
    // graph: one WHILE node
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
      rc = cuda_fail(e, "graph creation");
      break;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np)) != cudaSuccess) {
      rc = cuda_fail(e, "conditional node");
      break;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess) {
      rc = cuda_fail(e, "begin capture");
      break;
    }
    const double sc = tau * eps * eps;
    const int sstride = (int)(sizeof(AcState) / sizeof(int));
    for (auto& g : groups) {
      const Plan& p = *g.plan;
      const int B = (int)g.idx.size();
      batch_apply(p, B, g.p, g.q, g.vs, g.awork, s, &g.S[0].done, sstride, g.lam, align256(p.lam_count * 8) / 8);
      const dim3 grid(kAcBlocks, B);
      k_ac_pq<<<grid, kAcThreads, 0, s>>>(g.p, g.q, g.M, g.vs, g.S, g.partials, sc);
      k_ac_update<<<grid, kAcThreads, 0, s>>>(g.x, g.r, g.p, g.q, g.M, g.vs, g.S, g.partials, maxit);
      k_ac_dir<<<grid, kAcThreads, 0, s>>>(g.r, g.p, g.M, g.vs, g.S);
      k_ac_advance<<<grid, kAcThreads, 0, s>>>(g.u, g.x, g.r, g.p, g.M, g.vs, g.S, g.partials, g.partials2, nsteps,
                                                tau, rtol);
    }
    const unsigned max_passes = capped_passes((unsigned)nsteps * (unsigned)(maxit + 2) + 8u);
    k_ac_control<<<1, 256, 0, s>>>(S_all, nb, passes, max_passes, timeout, h);
    cudaGraph_t captured = nullptr;
    cudaError_t ecap = cudaGetLastError();
    e = cudaStreamEndCapture(s, &captured);
    if (ecap != cudaSuccess || e != cudaSuccess) {
      rc = cuda_fail(ecap != cudaSuccess ? ecap : e, "capture of the loop body");
      break;
    }
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
      rc = cuda_fail(e, "graph instantiation");
      break;
    }
    if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) {
      rc = cuda_fail(e, "graph launch");
      break;
    }
    // results back to the caller's buffers
    for (auto& g : groups) {
      const Plan& p = *g.plan;
      for (size_t k = 0; k < g.idx.size() && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(u[g.idx[k]], g.u + k * g.vs, p.M * 8, cudaMemcpyDeviceToDevice, s);
    }
    std::vector<AcState> hs(nb);
    int hto = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), S_all, nb * sizeof(AcState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hto, timeout, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "Allen-Cahn batch");
      break;
    }
    // report per caller index
    int off = 0;
    for (auto& g : groups) {
      for (size_t k = 0; k < g.idx.size(); ++k) {
        const AcState& st = hs[off + k];
        if (iters_out) iters_out[g.idx[k]] = st.iters_total;
        if (status_out) status_out[g.idx[k]] = st.status;
        if (st.status != FRLAP_OK && rc == FRLAP_OK) rc = fail((frlap_status)st.status, "an instance's solve stopped early");
      }
      off += (int)g.idx.size();
    }
    if (hto) rc = fail(FRLAP_ETIMEOUT, "Allen-Cahn batch loop reached its pass limit");
    if ((e = cudaEventRecord(ev1, s)) == cudaSuccess) e = cudaStreamWaitEvent(user, ev1, 0);
    if (e != cudaSuccess && rc == FRLAP_OK) rc = cuda_fail(e, "stream ordering");
  } while (false);
  cleanup();
  return rc;
}

}  // namespace frlap
