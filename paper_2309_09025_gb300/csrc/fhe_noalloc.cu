// fhe_noalloc.cu -- bootstrapping entry point that allocates no memory.
//
// fhe_pbs_batch keeps the ciphertexts extracted between blind rotation and key
// switching in the key handle's workspace.  fhe_pbs_batch_noalloc runs the
// same kernels (exact CUDA-core variant) but takes that scratch from a fixed
// array compiled into the library, so a call performs no cudaMalloc, cudaFree
// or other allocation.
#include <cuda_runtime.h>

#include <mutex>

#include "fhe_internal.cuh"

// Scratch for the extracted LWE_z ciphertexts: L x count x (kN + 1) words.
// Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[FHE_PBS_NOALLOC_MAX_WORDS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t *g_scratch_ptr[kMaxDevices];  // device address of the array, per device
bool g_scratch_ready[kMaxDevices];

// Resolve the array's device address on the current device (once per device).
// In host code `g_noalloc_scratch` only names a host-side stand-in; kernels
// must be given the address returned here.
int scratch_for_current_device(uint32_t **out) {
  int dev = 0;
  FHE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FHE_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ready[dev]) {
    void *p = nullptr;
    FHE_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    g_scratch_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  return FHE_OK;
}
}  // namespace

extern "C" int fhe_pbs_batch_noalloc(const fhe_keys *K, const uint32_t *ct_in, size_t count,
                                     const fhe_lut *lut, uint32_t *ct_out, void *stream) {
  if (!K || !lut || (count && (!ct_in || !ct_out)) || lut->N != K->P.N || lut->groups != 1u)
    return FHE_EINVAL;
  if (lut->L == 0u) return FHE_EINVAL;
  if (!count) return FHE_OK;
  // L * count * (kN + 1) <= the array's size, checked by division so that no
  // product can wrap for a huge count
  const uint64_t per_ct = (uint64_t)lut->L * K->P.big_words();
  if ((uint64_t)count > (uint64_t)FHE_PBS_NOALLOC_MAX_WORDS / per_ct) return FHE_EINVAL;
  int dev = 0;
  FHE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != K->device) return FHE_EINVAL;
  uint32_t *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  return fhe::pbs_exact_into(K, ct_in, count, lut, ct_out, scratch, (cudaStream_t)stream);
}
