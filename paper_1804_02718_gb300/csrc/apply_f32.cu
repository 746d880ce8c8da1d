// FP32 instances of the FFT apply (kernels and launchers in apply_impl.cuh).
#include "apply_impl.cuh"

namespace frlap {

template cudaError_t apply_batch_launch<float>(const Plan&, int, const float*, float*, size_t, void*, cudaStream_t,
                                               const int*, int, const float*, size_t, cudaEvent_t const*);
template cudaError_t apply_launch<float>(const Plan&, const float*, float*, void*, cudaStream_t, const int*,
                                         cudaEvent_t const*, const float*, bool);

template cudaError_t autotune_engine<float>(Plan&, int, float*, float*, void*, cudaStream_t);

template cudaError_t bc_collect<float>(unsigned long long*, unsigned long long*);
template cudaError_t wait_collect<float>(unsigned long long*);

}  // namespace frlap
