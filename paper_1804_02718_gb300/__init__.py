"""GB300 (sm_103a) library for the Duo & Zhang finite-difference integral fractional Laplacian.

The compute path is the CUDA library libfrlap.so (C ABI in include/frlap.h); this
package is its thin Python binding.  Build the library with
`paper_1804_02718_gb300.build.build()` (nvcc, sm_103a); every call raises if it
is missing -- there is no CPU fallback.
"""
from ._binding import (  # noqa: F401
    FRLAP_F32, FRLAP_F64, FRLAP_MIXED, FRLAP_DF64, FRLAP_MIXED_DF64, FRLAP_OP_AC, FRLAP_OP_APPLY, FRLAP_OP_PCG, FRLAP_SOLVE_CG,
    FRLAP_SOLVE_IR, FRLAP_PRECOND_NONE, FRLAP_PRECOND_STRANG, FRLAP_PRECOND_LEARNED, FRLAP_PRECOND_TAU, LIB_PATH, STATUS, FrlapError, Plan, frlap_allen_cahn_step, frlap_apply, frlap_apply_f32,
    frlap_apply_nstages, frlap_apply_profiled, frlap_apply_noalloc, NOALLOC_MAX_BYTES,
    frlap_apply_batch, frlap_apply_batch_workspace_bytes, frlap_apply_host, frlap_apply_host_workspace_bytes,
    frlap_plan_autotune, frlap_allen_cahn_cn,
    frlap_c_dalpha, frlap_coeffs, frlap_pcg_solve, frlap_precond_strang, frlap_precond_tau, frlap_precond_set_symbol, frlap_precond_apply,
    frlap_mlp_multiplier, frlap_learn_workspace_bytes, frlap_learn_grad, frlap_adam_step, frlap_cg_pairs, MLP_NPARAM,
    frlap_allen_cahn_batch, frlap_allen_cahn_batch_workspace_bytes, frlap_plan_create, frlap_plan_destroy,
    frlap_workspace_bytes, frlap_set_loop_pass_limit, frlap_bounds_check_report, frlap_bounds_check_selftest,
    frlap_async_wait_report, frlap_async_wait_selftest, frlap_dft16_stages, frlap_residual, lib,
)
