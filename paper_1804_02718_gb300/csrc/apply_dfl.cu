// Double-float instances of the FFT apply (kernels and launchers in apply_impl.cuh).
#include "apply_impl.cuh"

namespace frlap {

template cudaError_t apply_batch_launch<dfl>(const Plan&, int, const double*, double*, size_t, void*, cudaStream_t,
                                             const int*, int, const dfl*, size_t, cudaEvent_t const*);
template cudaError_t apply_launch<dfl>(const Plan&, const double*, double*, void*, cudaStream_t, const int*,
                                       cudaEvent_t const*, const dfl*, bool);

template cudaError_t autotune_engine<dfl>(Plan&, int, double*, double*, void*, cudaStream_t);

template cudaError_t bc_collect<dfl>(unsigned long long*, unsigned long long*);
template cudaError_t wait_collect<dfl>(unsigned long long*);

}  // namespace frlap
