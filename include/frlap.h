/*
 * frlap -- GB300 (sm_103a) library for the finite-difference integral fractional
 * Laplacian of Duo & Zhang, "Accurate numerical methods for two and three
 * dimensional integral fractional Laplacian with applications" (arXiv:1804.02718).
 *
 * The operator: on the box Omega = prod_r (a_r, a_r + N_r h) with u = 0 outside,
 * the scheme of eq. fLh-2D (2D) / eq. fLh-3D (3D) is the matrix-vector product
 * y = A u with the symmetric multilevel Toeplitz matrix A[i,j] = -c_{d,alpha} a_{|i-j|}
 * (eqs. A-2D, Aj, A-3D, Aj-3D); a_k are the coefficients of eqs. amn, a00
 * (2D) and a_mns, a000 (3D); c_{d,alpha} is the constant of Sec. 1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - d is 2 or 3.  N[r] (r = 0 is x, 1 is y, 2 is z) is the number of mesh
 *    intervals along axis r, 2 <= N[r] <= 8192 (2D) or 1024 (3D), so there are n_r = N[r] - 1 interior
 *    unknowns along axis r.  The grid vector u is stored x fastest: a C-order
 *    array [n_z][n_y][n_x] (3D) or [n_y][n_x] (2D), as in eq. product / A3D.
 *    h > 0 is the mesh size; the coefficient table uses N_max = max_r N[r]
 *    (the paper's L = N_max h is the longest side).
 *  - 0 < alpha < 2 and alpha < gamma <= 2 (gamma = 2 is the paper's default;
 *    Sec. 5 uses it throughout).
 *  - Every pointer named d_* is a DEVICE pointer owned by the caller; the
 *    library never frees it.  Pointers to host scalars (iters, relres) are
 *    host pointers.  `stream` is a cudaStream_t (NULL = legacy default stream);
 *    all work is enqueued on it and entry points return without waiting,
 *    except where a host scalar output is written (they synchronise `stream`).
 *  - Only the set-up calls frlap_plan_create and frlap_coeffs allocate device
 *    memory (frlap_coeffs: stream-ordered scratch, freed before it returns);
 *    the scratch every other call needs is the caller's d_work buffer of at
 *    least frlap_workspace_bytes() bytes, 256-byte aligned.
 *  - Errors are reported by the return code; frlap_last_error() gives a
 *    message for the calling thread.  No C++ exception crosses this boundary.
 *    Invalid arguments return FRLAP_EINVAL before anything is enqueued.
 */
#ifndef FRLAP_H
#define FRLAP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FRLAP_OK = 0,
  FRLAP_EINVAL = 1,      /* bad argument (d, alpha, gamma, h, N, sizes, null pointers) */
  FRLAP_ENOMEM = 2,      /* device allocation in frlap_plan_create failed */
  FRLAP_EWORKSPACE = 3,  /* d_work is NULL or misaligned */
  FRLAP_ECUDA = 4,       /* a CUDA runtime call or kernel launch failed */
  FRLAP_ENOCONV = 5,     /* iterative solver hit maxit before reaching rtol */
  FRLAP_EBREAKDOWN = 6,  /* CG breakdown: p^T A p <= 0 or non-finite */
  FRLAP_ENAN = 7,        /* non-finite value in the right-hand side or iterate */
  FRLAP_ETIMEOUT = 8     /* a bounded device-side wait expired */
} frlap_status;

/* Arithmetic of the FFT apply.  F64: IEEE double everywhere.  F32: single
 * precision FFT stages and symbol.  MIXED: a plan that holds both, so
 * that the iterative-refinement solver can run FP32 inner applies and FP64
 * outer residuals (coefficients and symbol are always generated in FP64).
 * DF64: FP64 vectors in memory, FFT stages in double-float arithmetic (pairs
 * of FP32 numbers, about 48 significant bits), which GB300 runs several times
 * faster than FP64 at an accuracy within the FP64 tolerance of the apply.
 * Double-float keeps FP32's exponent range: the FFT stages hold values up to
 * about 3.4e38 (larger ones become infinite) and lose low-order bits below
 * about 1e-31 (FP32's smallest normal number is 1.2e-38 and the low word sits
 * 2^-24 below the high one).  A DF64 apply is therefore accurate to the FP64
 * tolerance for inputs with 1e-25 <~ max|u_i| and lambda_max max|u_i| <~ 1e35;
 * outside that range use an F64 plan.  frlap_pcg_solve scales the system by the
 * power of two at or below 1/max|f_i| before its double-float iterations (an
 * exact scaling, undone on the solution), so its solves have no such limit; it
 * returns FRLAP_ENAN if the right-hand side itself is not finite.
 * MIXED_DF64: MIXED with the FP64 side computed as in DF64.
 * In frlap_pcg_solve the iterations use the plan's engine, but the residuals
 * f - A x that restart a CG solve or decide convergence (the final check, and
 * the refinement residuals from 1e-6 relative on) are computed with the native
 * FP64 engine: double-float rounding, about 5e-15 lambda_max ||x||, would
 * otherwise set a residual floor near 1e-10 ||f|| at 2047^2. */
typedef enum { FRLAP_F64 = 0, FRLAP_F32 = 1, FRLAP_MIXED = 2, FRLAP_DF64 = 3, FRLAP_MIXED_DF64 = 4 } frlap_prec;

/* Which scratch size frlap_workspace_bytes reports. */
typedef enum { FRLAP_OP_APPLY = 0, FRLAP_OP_PCG = 1, FRLAP_OP_AC = 2 } frlap_op;

/* Solver variants of frlap_pcg_solve. */
typedef enum {
  FRLAP_SOLVE_CG = 0,      /* plain FP64 conjugate gradients (Sec. 5.3: CG with the FFT product) */
  FRLAP_SOLVE_IR = 1       /* FP64 iterative refinement around FP32 CG (MIXED plans) */
} frlap_solver;

/* Preconditioners of frlap_pcg_solve.  Each is a multiplier applied through the
 * apply pipeline (one FP32 apply per iteration), so the outer FP64 iteration is
 * flexible (Polak-Ribiere) PCG: in the Fourier basis of A's circulant embedding
 * (Strang, learned) or in the sine basis of the box (tau). */
typedef enum {
  FRLAP_PRECOND_NONE = 0,
  FRLAP_PRECOND_STRANG = 1,   /* inverse of the multilevel Strang circulant (built by frlap_precond_strang) */
  FRLAP_PRECOND_LEARNED = 2,  /* a multiplier set by frlap_precond_set_symbol (e.g. the learned MLP's) */
  FRLAP_PRECOND_TAU = 3       /* S diag(S A S)^-1 S, S the multilevel DST-I (built by frlap_precond_tau) */
} frlap_precond;

typedef struct frlap_plan frlap_plan;

/* c_{d,alpha} = 2^(alpha-1) alpha Gamma((d+alpha)/2) / (pi^(d/2) Gamma(1-alpha/2))
 * (Sec. 1, the normalisation constant of eq. fL-nD).  Host-only, no device work.
 * Returns FRLAP_EINVAL unless d in {2,3} and 0 < alpha < 2. */
frlap_status frlap_c_dalpha(int d, double alpha, double* out);

/* The coefficients a_k of the scheme, k in [0, N_max]^d, in FP64, for mesh size h:
 *   a_k = 2^sigma(k) / (2^d |h k|^gamma) * (int_{T_k} |xi|^(gamma-d-alpha) dxi + kappa_k w_0)  (k != 0)
 *   a_0 = - sum_{k != 0} 2^(d - sigma(k)) a_k - 2^d int_{D_2} |xi|^-(d+alpha) dxi
 * (Sec. 2 eqs. amn, a00; Sec. 4 a_mns, a000), sigma(k) = number of zero
 * components of k, T_k = the elements of (0, N_max h)^d having h k as a vertex,
 * kappa_k the origin correction (gamma = 2: +1 in 2D / +5/3 in 3D on unit axis
 * offsets, -1 on the other vertices of the origin element, including (1,1,1); gamma < 2: 0).
 * Output d_coeffs: (N_max+1)^d doubles, C-order with the x offset fastest.
 * Computed entirely on the device (quadrature, assembly, reduction for a_0). */
frlap_status frlap_coeffs(int d, double alpha, double gamma, double h, const int* N,
                          double* d_coeffs, void* stream);

/* Create a plan: coefficients, the real symbol lambda of the circulant
 * embedding of A (size P_r = max(32, next power of two >= 2 n_r - 1) per axis,
 * stored as its (P_r/2+1)-per-axis octant, 1/prod(P_r) folded in), FFT
 * twiddle tables.  Allocates the plan's device memory (set-up call).
 * `*out` receives the plan; destroy it with frlap_plan_destroy. */
frlap_status frlap_plan_create(int d, double alpha, double gamma, double h, const int* N, int prec,
                               void* stream, frlap_plan** out);
frlap_status frlap_plan_destroy(frlap_plan* plan);

/* Bytes of caller-provided scratch needed by `op` on this plan (0 on a NULL plan). */
size_t frlap_workspace_bytes(const frlap_plan* plan, int op);

/* Interior sizes n_r and embedding sizes P_r of a plan (either may be NULL). */
frlap_status frlap_plan_shape(const frlap_plan* plan, int* n, int* P);

/* Copy the symbol octant (prod_r (P_r/2+1) doubles, x fastest, including the
 * 1/prod(P_r) factor) into d_lambda.  For tests and for building preconditioners. */
frlap_status frlap_plan_symbol(const frlap_plan* plan, double* d_lambda, void* stream);

/* y = A u on the interior nodes (eq. product / A3D), computed by the FFT of
 * the circulant embedding: zero-pad u to P_r per axis, forward real-to-complex
 * FFT along x, complex FFTs along y (and z), multiply by lambda, inverse FFTs,
 * keep the first n_r entries per axis.  d_u, d_y: prod(n_r) elements of double
 * (F64, MIXED, DF64 and MIXED_DF64 plans) or float (F32 plans); they must not overlap. */
frlap_status frlap_apply(const frlap_plan* plan, const void* d_u, void* d_y, void* d_work, void* stream);

/* Number of kernel stages of one apply (2D: 3, 3D: 5): pad + real FFT along x,
 * the FFT/multiply stages along y (and z), inverse real FFT along x + crop. */
int frlap_apply_nstages(const frlap_plan* plan);

/* nbatch products y_b = A u_b (b = 0..nbatch-1) of the same plan, each as in
 * frlap_apply, with one kernel launch per stage for the whole batch: the
 * instances fill the GPU together instead of one after another.  Many
 * right-hand sides or time levels of one operator are the use (the paper applies
 * A once per CG iteration and time step, Secs. 5.3-5.4).
 * d_u, d_y: nbatch vectors of prod(n_r) elements each, back to back, of the
 * element type frlap_apply takes for the plan; the two ranges must not overlap.
 * d_work: frlap_apply_batch_workspace_bytes(plan, nbatch) bytes, 256-byte aligned.
 * events: NULL, or frlap_apply_nstages(plan) + 1 cudaEvent_t recorded on `stream`
 * before each stage and after the last (NULL entries are skipped).
 * 1 <= nbatch <= 65535, else FRLAP_EINVAL. */
size_t frlap_apply_batch_workspace_bytes(const frlap_plan* plan, int nbatch);
frlap_status frlap_apply_batch(const frlap_plan* plan, int nbatch, const void* d_u, void* d_y, void* d_work,
                               void* stream, void* const* events);

/* frlap_apply_batch from and to HOST buffers: y_b = A u_b for b = 0..nbatch-1, with
 * h_u, h_y in host memory (nbatch vectors back to back, element type as in
 * frlap_apply).  The batch moves in chunks of `chunk` vectors through three device
 * slots: the copies in of chunks i+1 and i+2 and the copy out of chunk i-1 run on
 * internal streams while chunk i is applied, and consecutive chunks compute on
 * `stream` and on an internal stream, so their kernels may overlap.  When chunk > 1
 * and nbatch > 2 the first and the last chunk hold one vector, so that filling and
 * draining the pipeline costs one vector's copy.  For the copies to overlap, h_u and
 * h_y must be pinned (page-locked); pageable buffers give the same result with
 * serialised copies.  h_u and h_y must not overlap.  d_work:
 * frlap_apply_host_workspace_bytes(plan, chunk) bytes, 256-byte aligned.
 * Synchronises `stream`: h_y is complete on return.  1 <= chunk <= 65535,
 * nbatch >= 1, else FRLAP_EINVAL. */
/* Autotuner of the apply's launch shapes.  For each stage of the apply, and for each
 * engine the plan uses (FP32, and FP64 or double-float), times every admissible
 * number of FFT lines per CTA (powers of two up to 512 threads and 227 KB of shared
 * memory) on a batch of nbatch zero vectors, and keeps the fastest in the plan;
 * later applies, batched applies, solves and Allen-Cahn runs on the plan use it.
 * The stages are timed independently (one launch each), so the search is exact
 * per stage.  d_work: frlap_autotune_workspace_bytes(plan, nbatch) bytes, 256-byte
 * aligned; chosen (may be NULL): 10 ints, the FP64-side choices of stages 0..4, then
 * the FP32 ones (0 where a stage or engine does not exist).  Synchronises stream;
 * not to be called while another thread uses the plan.  1 <= nbatch <= 65535. */
size_t frlap_autotune_workspace_bytes(const frlap_plan* plan, int nbatch);
frlap_status frlap_plan_autotune(frlap_plan* plan, int nbatch, void* d_work, void* stream, int* chosen);

size_t frlap_apply_host_workspace_bytes(const frlap_plan* plan, int chunk);
frlap_status frlap_apply_host(const frlap_plan* plan, int nbatch, int chunk, const void* h_u, void* h_y,
                              void* d_work, void* stream);

/* frlap_apply with timing marks: events[i] (a cudaEvent_t, or NULL to skip) is
 * recorded on `stream` just before stage i, events[nstages] after the last
 * stage.  The caller creates the events; the array must hold nstages+1 entries. */
frlap_status frlap_apply_profiled(const frlap_plan* plan, const void* d_u, void* d_y, void* d_work, void* stream,
                                  void* const* events);

/* Size of the device array behind frlap_apply_noalloc: 32 MiB. */
#define FRLAP_NOALLOC_MAX_BYTES (32u << 20)

/* frlap_apply for callers that must not allocate device memory at call time:
 * code inside a host framework that owns the GPU's memory and forbids
 * cudaMalloc, and latency-bound loops that cannot afford the device-wide
 * synchronisation a cudaMalloc/cudaFree implies.  The paper has no counterpart;
 * this is a library convenience.  Same product, arguments and result as
 * frlap_apply, but the scratch is a fixed library-owned device array of
 * FRLAP_NOALLOC_MAX_BYTES, reserved on every GPU that loads the library until
 * the process exits.  The call allocates nothing.
 *  - Limit: plans whose frlap_workspace_bytes(plan, FRLAP_OP_APPLY) exceeds
 *    FRLAP_NOALLOC_MAX_BYTES are rejected with FRLAP_EINVAL and a message.
 *    In interior unknowns per axis (n = N - 1) for square and cubic grids:
 *    2D FP64-class plans (F64, MIXED, DF64, MIXED_DF64) n <= 1024, 2D F32 n <= 2047,
 *    3D FP64-class n <= 64, 3D F32 n <= 93.
 *  - The first call on a device looks up the array's device address on the
 *    current device and caches it for the process; make that first call before
 *    any stream capture.  cudaDeviceReset on a device invalidates the cached
 *    address: do not call this entry point on that device afterwards.
 *  - All calls on a device share the array: two calls whose GPU work overlaps
 *    (unordered streams) race and give wrong results.  Calls ordered on one
 *    stream are safe; no state carries over from one call to the next. */
frlap_status frlap_apply_noalloc(const frlap_plan* plan, const void* d_u, void* d_y, void* stream);

/* Same product in FP32 on a MIXED plan (float in, float out). */
frlap_status frlap_apply_f32(const frlap_plan* plan, const float* d_u, float* d_y, void* d_work, void* stream);

/* Solve A x = f (the fractional Poisson problem eqs. Poisson, BCP, discretised
 * by the scheme) by conjugate gradients with the FFT product (Sec. 5.3).
 * d_f, d_x: prod(n_r) doubles; d_x holds the initial guess on entry and the
 * solution on exit.  Stops when ||f - A x||_2 <= rtol ||f||_2 (recursive
 * residual, then confirmed with a true FP64 residual), or after maxit iterations.
 * solver = FRLAP_SOLVE_CG (any plan but F32) or FRLAP_SOLVE_IR (MIXED plans: FP32 CG
 * inner solves to inner_rtol, FP64 outer residual and update).  precond =
 * frlap_precond (applied in FP32 inside the CG iteration: flexible PCG).
 * *iters (may be NULL) receives the CG iterations (IR: total inner iterations),
 * *relres (may be NULL) the final true relative residual.  Synchronises stream.
 * Returns FRLAP_ENOCONV if rtol was not reached. */
frlap_status frlap_pcg_solve(const frlap_plan* plan, const double* d_f, double* d_x, double rtol, int maxit,
                             int solver, int precond, double inner_rtol, int* iters, double* relres, void* d_work,
                             void* stream);

/* r = f - A x and ||r||_2 / ||f||_2 in FP64: the true relative residual that decides frlap_pcg_solve's
 * convergence (the paper solves its systems by CG, Sec. 5.3), with the same apply.  F64 and MIXED plans: the native FP64 apply.
 * Double-float plans: forward transforms and symbol product in FP64, inverse transforms in
 * double-float.  The forward transforms' rounding reaches A x multiplied by up to lambda_max, the
 * inverse ones' only relative to A x itself; so near a solution (||A x|| far below lambda_max ||x||)
 * this is as accurate as native FP64 and about 1.7x faster (2D plans with a 16384-point y embedding
 * use native FP64).  Far from a solution it is as accurate as the double-float apply.
 * d_f, d_x: device FP64 vectors of the plan's unknowns (x-fastest); d_r: device, the residual, or NULL
 * for the norm only (must not overlap d_f or d_x); d_work: frlap_workspace_bytes(plan, FRLAP_OP_PCG).
 * Synchronises `stream` to return *relres.  FRLAP_EINVAL: NULL plan, d_f, d_x or relres, an F32 plan,
 * overlapping d_r, or a NULL workspace. */
frlap_status frlap_residual(const frlap_plan* plan, const double* d_f, const double* d_x, double* d_r,
                            double* relres, void* d_work, void* stream);

/* Build the Strang-circulant preconditioner of the plan (set-up call: allocates
 * the symbol and temporary scratch).  The Strang circulant S keeps, along each
 * axis, the Toeplitz entry of offset min(j, n_r - j) in its first column; its
 * inverse is a multilevel circulant, applied through A's embedding.  Its
 * eigenvalues are positive for this operator (A is strictly diagonally
 * dominant); non-positive ones would be dropped and are counted in
 * *n_nonpositive (may be NULL).  Synchronises stream. */
frlap_status frlap_precond_strang(frlap_plan* plan, int* n_nonpositive, void* stream);

/* Build the sine-basis ("tau") preconditioner of the plan (set-up call: allocates the
 * multiplier and temporary scratch).  S, the orthonormal multilevel DST-I, holds the sine
 * modes of the box, which vanish on its boundary as u does; M = S diag(S A S)^-1 S is the
 * inverse of the member of the algebra S diagonalises that is closest to A in the
 * Frobenius norm.  diag(S A S) is computed from the coefficients by one P-point DFT per
 * line and axis; M is applied on odd extensions of the vector to P = 2 N_r points per
 * axis (whose DFT is the DST) through the apply pipeline, one FP32 apply per iteration.
 * Needs every N[r] a power of two of at least 16 (so that P_r = 2 N_r; 2D N[r] <= 4096),
 * else FRLAP_EINVAL.  Entries of diag(S A S) are Rayleigh quotients of A, positive for this
 * operator; non-positive ones would be dropped and are counted in *n_nonpositive (may be
 * NULL).  Synchronises stream. */
frlap_status frlap_precond_tau(frlap_plan* plan, int* n_nonpositive, void* stream);

/* z = M^-1 r for one of the plan's preconditioners, in FP32 (r, z: prod(n_r)
 * floats, not overlapping; d_work: frlap_workspace_bytes(plan, FRLAP_OP_APPLY)). */
frlap_status frlap_precond_apply(const frlap_plan* plan, int precond, const float* d_r, float* d_z, void* d_work,
                                 void* stream);

/* Install a preconditioner multiplier m (octant layout of frlap_plan_symbol:
 * prod_r (P_r/2+1) doubles, x fastest) as FRLAP_PRECOND_LEARNED: M^-1 r =
 * restrict(IDFT(m * DFT(zero-padded r))) with the 1/prod(P_r) factor applied
 * by the library.  m must be positive for M to be SPD.  The plan keeps an FP32
 * copy (allocated on the first call). */
frlap_status frlap_precond_set_symbol(frlap_plan* plan, const double* d_m, void* stream);

/* nsteps semi-implicit steps of the fractional Allen-Cahn equation
 * u_t = -eps^2 (-Delta)^{alpha/2} u + u - u^3 with u = 0 outside the box:
 * (I + tau eps^2 A) u^{n+1} = u^n + tau (u^n - (u^n)^3), each solved by CG
 * from u^n to relative residual rtol (the paper's model, eqs. AC-1/AC-2, steps
 * with Crank-Nicolson and CG; this is the semi-implicit form of the same
 * space discretisation).  When the plan's sine-basis preconditioner is built
 * (frlap_precond_tau), each solve is PCG with S diag(1 + tau eps^2 S A S)^-1 S.
 * d_u: prod(n_r) doubles, updated in place.  *iters (may be NULL): total CG
 * iterations.  Synchronises stream. */
frlap_status frlap_allen_cahn_step(const frlap_plan* plan, double* d_u, double tau, double eps, int nsteps,
                                   double rtol, int* iters, void* d_work, void* stream);

/* nsteps Crank-Nicolson steps of the paper's own fractional Allen-Cahn model (eqs.
 * AC-1, AC-2, Sec. 5.4): u_t = -(-Delta)^{alpha/2} u - delta^{-alpha} u (u^2 - 1) on the
 * box, u = -1 outside.  The unknown is ubar = u + 1, which vanishes outside (the
 * fractional Laplacian of a constant is zero).  Each step solves
 *   (I + tau/2 A) ubar^{n+1} = (I - tau/2 A) ubar^n - tau delta^{-alpha} u^n ((u^n)^2 - 1)
 * by CG from ubar^n to relative residual rtol (the reaction term taken at t_n: the
 * paper states Crank-Nicolson with one CG solve per step but not how the reaction
 * enters; with the plan's sine-basis preconditioner built (frlap_precond_tau), PCG with
 * S diag(1 + tau/2 S A S)^-1 S).  d_ubar: prod(n_r) doubles, updated in place.  h_mass (host, may be NULL):
 * nsteps doubles, h^d sum ubar after each step (the bubbles' area or volume).
 * *iters (may be NULL): total CG iterations.  d_work: frlap_workspace_bytes(plan,
 * FRLAP_OP_AC) bytes.  Synchronises stream.  F32 plans are refused (FRLAP_EINVAL). */
frlap_status frlap_allen_cahn_cn(const frlap_plan* plan, double* d_ubar, double tau, double delta, int nsteps,
                                 double rtol, int* iters, double* h_mass, void* d_work, void* stream);

/* ---- learned preconditioner (an extension; the paper has no learned part) ----
 * A per-frequency MLP on the symbol octant: features (alpha, kappa_x, kappa_y,
 * kappa_z), kappa_r = k_r / (P_r/2) (kappa_z = 0 in 2D), two tanh layers of
 * FRLAP_MLP_HIDDEN units, scalar output s; multiplier m(k) = exp(s(k)) / lambda(k)
 * with lambda the symbol of A's embedding (a zero network gives m = 1/lambda).
 * Parameters: FRLAP_MLP_NPARAM floats, in order W1[64][4], b1[64], W2[64][64]
 * (out, in), b2[64], w3[64], b3[1]. */
#define FRLAP_MLP_HIDDEN 64
#define FRLAP_MLP_NFEAT 4
#define FRLAP_MLP_NPARAM 4545

/* m on the plan's octant (prod_r (P_r/2+1) doubles, x fastest); pass it to
 * frlap_precond_set_symbol to use it in frlap_pcg_solve. */
frlap_status frlap_mlp_multiplier(const frlap_plan* plan, const float* d_params, double* d_m, void* stream);

/* Scratch for frlap_learn_grad with a batch of B pairs. */
size_t frlap_learn_workspace_bytes(const frlap_plan* plan, int B);

/* Preconditioner loss over B pairs (d_r, d_e: B consecutive grid vectors of
 * doubles, e_b = A^-1 r_b) and its gradient with respect to the parameters.
 * With z_b = M^-1 r_b, the loss is the A-norm error left by the best multiple
 * of z_b (one preconditioned steepest-descent step; PCG is unchanged when M is
 * scaled, so the loss is scale-free):
 *   L = mean_b [1 - (r_b.z_b)^2 / ((z_b.A z_b)(r_b.e_b))],  r_b.e_b = ||e_b||_A^2.
 * d_grad (FRLAP_MLP_NPARAM floats, overwritten), d_loss (one double on the
 * device).  FP64 spectra, FP32 network.  Plans with an embedding of more than
 * 8192 points along an axis (2D N[r] > 4096) are refused with FRLAP_EINVAL. */
frlap_status frlap_learn_grad(const frlap_plan* plan, const float* d_params, const double* d_r, const double* d_e,
                              int B, float* d_grad, double* d_loss, void* d_work, void* stream);

/* One Adam step (step counter t >= 1) on n parameters, in place. */
frlap_status frlap_adam_step(float* d_params, const float* d_grad, float* d_m1, float* d_m2, int n, float lr,
                             float beta1, float beta2, float eps, int t, void* stream);

/* Training pairs from the plain FP64 CG solver: run CG on A x = f from x0 = 0 to
 * rtol and snapshot the iterates x_0 = 0, x_1, ...; on return d_E[j] = x* - x_j
 * and d_R[j] = A d_E[j] (= f - A x_j), j < *npairs = min(iterations, K): the
 * final iterate (zero error) is left out.  Each pair is prod(n_r) doubles.
 * d_work: frlap_workspace_bytes(plan, FRLAP_OP_PCG).  Synchronises stream. */
frlap_status frlap_cg_pairs(const frlap_plan* plan, const double* d_f, int K, double rtol, double* d_E, double* d_R,
                            int* npairs, void* d_work, void* stream);

/* Batched Allen-Cahn: nbatch instances (each its own plan: alpha and grid; F64 or
 * MIXED plans) advance nsteps semi-implicit steps each, all in one CUDA-graph
 * launch with on-device control: one conditional WHILE node whose body runs one CG
 * iteration for every instance still solving, then moves each instance whose solve
 * has ended to its next step.  Each step solves (I + tau eps^2 A_i) v =
 * u + tau (u - u^3) by CG to ||r|| <= rtol ||rhs|| or maxit iterations, the first
 * step from v = 0 and every later one from the previous step's solution (its initial
 * residual follows from the finished solve's residual, with no extra apply).
 * Instances of equal shape share one launch per kernel.  d_u[i]: instance i's
 * grid vector (doubles), updated in place.  iters[i], status[i] (host arrays, may
 * be NULL): total CG iterations and frlap_status per instance.  The loop is bounded
 * (nsteps * (maxit + 2) + 8 passes, or frlap_set_loop_pass_limit's lower cap;
 * FRLAP_ETIMEOUT past that).  d_work:
 * frlap_allen_cahn_batch_workspace_bytes bytes.  Synchronises stream. */
size_t frlap_allen_cahn_batch_workspace_bytes(int nbatch, const frlap_plan* const* plans);
frlap_status frlap_allen_cahn_batch(int nbatch, const frlap_plan* const* plans, double* const* d_u, double tau,
                                    double eps, int nsteps, double rtol, int maxit, int* iters, int* status,
                                    void* d_work, void* stream);

/* Process-wide cap on the passes of the graph-launched loops: the conditional WHILE
 * node of frlap_pcg_solve's CG (after its first 8 iterations) and of
 * frlap_allen_cahn_batch.  Each loop stops after min(its own bound, max_passes)
 * passes; a loop that stops there with work left returns FRLAP_ETIMEOUT, leaving
 * the context usable.  0 (the default) keeps the loops' own bounds.  For callers
 * that want a hard bound on the GPU time of one call, and for tests of the
 * time-out path.  The paper has no counterpart. */
frlap_status frlap_set_loop_pass_limit(unsigned max_passes);

/* The first apply stage of the FP64 and double-float engines stages its input rows in shared
 * memory by bulk asynchronous copies and waits for each on an mbarrier.  Every such wait is
 * bounded (about a second); a wait that gives up is counted, and that kernel returns without
 * storing its remaining tiles (the call's result is then wrong).  frlap_async_wait_report returns
 * in *timeouts the count since the previous report (summed over the engines and the tensor-core
 * waits of frlap_dft16_stages, then reset).
 * Synchronises the device.  A tool for tests and health checks; the paper has no counterpart. */
frlap_status frlap_async_wait_report(unsigned long long* timeouts);
/* The give-up path of that wait: one warp waits on an mbarrier phase that nothing completes (no
 * arrival, no copy in flight) until the bound runs out (about a second) and records it.  Returns in
 * *timeouts the waits that gave up (1 expected; the counter is reset before and after), leaving the
 * context usable.  Synchronises the device.  For tests. */
frlap_status frlap_async_wait_selftest(unsigned long long* timeouts);

/* Radix-16 FFT stages in two engines, to measure the tensor-core form of the stages the apply's
 * transforms are made of (the apply itself runs them on CUDA cores).  Textbook FFT arithmetic, not
 * from the paper, which only states that the Toeplitz products are computed by FFT (Sec. 2 after
 * eq. product, Sec. 4 after eq. A3D).
 * Data: ntiles tiles of 128 rows x 16 complex FP32 values (re, im interleaved; 4096 floats, 16 KB
 * per tile), row r = 16 a + b (a < 8, b < 16).  Each tile is loaded once, then `reps` stages run
 * on chip, each
 *   x'[a,b][q] = v[a,b][q] W_256^{bq} / 4;  v[a,q][k] = sum_b x'[a,b][q] W_16^{bk}   (W_L = exp(-2 pi i/L)),
 * i.e. twiddles (scaled so that a stage keeps the norm), the transposing exchange of a Stockham stage
 * and a 16-point DFT per row; then the
 * tile is stored to d_out.  engine 0: CUDA cores (shared-memory exchange, register radix-16
 * butterflies, as in the apply); engine 1: tensor cores (tcgen05.mma kind::tf32, the DFT as a real
 * 32 x 32 matrix product with both operands split into TF32 high and low parts, three products
 * accumulated in FP32 in tensor memory; relative error about 1e-6 per stage).  d_in, d_out: device,
 * 16-byte aligned, equal (in place) or not overlapping; 0 <= ntiles <= 2^24, 0 <= reps <= 65536.
 * Asynchronous on `stream`.  A stage whose tensor-core completion wait gives up (about a second)
 * leaves its tile unwritten and counts in frlap_async_wait_report.  FRLAP_EINVAL on bad arguments,
 * FRLAP_ECUDA on a launch error. */
frlap_status frlap_dft16_stages(int engine, const float* d_in, float* d_out, int ntiles, int reps, void* stream);

/* Bounds-checked builds (compiled with -DFRLAP_BOUNDS_CHECK; the package's build script makes
 * them as libfrlap_bc.so).  There every global load and store of the apply kernels is first tested
 * against the buffers its call registered (the call's vectors, workspace, symbol, twiddle tables and
 * skip flags); an access outside all of them is not performed (a load gives zero) but counted.
 * frlap_bounds_check_report returns in *violations the count since the previous report (summed
 * over the FP32, FP64 and double-float kernels, then reset) and in *first_address (may be NULL) the
 * lowest such address; *enabled (may be NULL) is 1 in a checked build, 0 otherwise (where
 * *violations is always 0).  Synchronises the device.  A tool for tests, standing in for a memory
 * checker; the paper has no counterpart. */
frlap_status frlap_bounds_check_report(int* enabled, unsigned long long* violations, unsigned long long* first_address);

/* Checked builds only: probes the checker itself on library-owned memory (8 loads inside a
 * registered range, 5 just past it, which the checks must skip) and returns in *flagged the
 * accesses it flagged: 5 when it works.  FRLAP_EINVAL in ordinary builds. */
frlap_status frlap_bounds_check_selftest(unsigned long long* flagged);

/* The message for the last error on the calling thread ("" if none). */
const char* frlap_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FRLAP_H */
