// frlap_apply_noalloc: the FFT apply for callers that cannot allocate device
// memory, with its scratch in a fixed, library-owned device array.
//
// The array below is reserved on every GPU that loads this library, for the
// life of the process.  In host code its name is only a host-side stand-in, so
// the device address is looked up once per device with cudaGetSymbolAddress
// (with that device current) and cached; the first call on a device does that
// look-up.  The cached address belongs to the device's current context: after
// cudaDeviceReset on a device the array is re-created, possibly elsewhere, so this
// entry point must not be called on that device again in the same process.
// All calls on a device share the one array: calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on it.
// Nothing needs clearing between calls: the first apply stage writes every
// scratch entry that a later stage reads.
#include <mutex>

#include "common.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FRLAP_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

using namespace frlap;

extern "C" frlap_status frlap_apply_noalloc(const frlap_plan* plan, const void* d_u, void* d_y, void* stream) {
  if (!plan || !d_u || !d_y) return fail(FRLAP_EINVAL, "plan, d_u or d_y is NULL");
  const bool f32 = plan->prec == FRLAP_F32;
  if (ranges_overlap(d_u, d_y, vector_bytes(*plan, f32))) return fail(FRLAP_EINVAL, "d_u and d_y must not overlap");
  const size_t need = apply_work_bytes(*plan, f32 ? 4 : 8);
  if (need > (size_t)FRLAP_NOALLOC_MAX_BYTES)
    return fail(FRLAP_EINVAL, "frlap_apply_noalloc: this grid needs " + std::to_string(need) +
                                  " bytes of scratch, more than the " + std::to_string((size_t)FRLAP_NOALLOC_MAX_BYTES) +
                                  "-byte static buffer; use frlap_apply with a caller workspace");
  int dev = -1;
  FRLAP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(FRLAP_EINVAL, "device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* addr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
      g_scratch_addr[dev] = addr;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaError_t e;
  if (f32)
    e = apply_launch<float>(*plan, (const float*)d_u, (float*)d_y, scratch, (cudaStream_t)stream, nullptr);
  else
    e = apply64(*plan, (const double*)d_u, (double*)d_y, scratch, (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "frlap_apply_noalloc");
  return FRLAP_OK;
}
