// The residual apply of double-float plans: FP64 forward transforms and symbol product, double-float
// inverse transforms (apply_launch_b<double, dfl>, kernels in apply_impl.cuh).  Its own translation
// unit, compiled beside the engines' ones.
//
// A residual f - A x near a solution is small against lambda_max ||x||.  The forward transforms'
// rounding (relative to ||x||) reaches A x multiplied by up to lambda_max, as in any FFT product, so
// those transforms stay in FP64; the inverse transforms' rounding is relative to the product they
// transform, the size of A x itself, so double-float's 2^-48 keeps it far below the forward part.
// The result is then as accurate as the all-FP64 apply near a solution, at the cost of the FP64
// forward half only.
#include "apply_impl.cuh"

namespace frlap {

cudaError_t apply_residual_hyb(const Plan& p, const double* u, double* y, void* work, cudaStream_t s) {
  if (!p.df64) return cudaErrorNotSupported;
  return apply_launch_b<double, dfl>(p, 1, u, y, 0, work, s, nullptr, 0, nullptr, nullptr, 0, false);
}

cudaError_t hyb_wait_collect(unsigned long long* count) { return unit_wait_collect(count); }
cudaError_t hyb_bc_collect(unsigned long long* count, unsigned long long* first) {
  return unit_bc_collect(count, first);
}

}  // namespace frlap
