// fhe_pbs_tc.cu -- tensor-core (tcgen05) variant of the blind rotation.
#include <cuda_runtime.h>

#include "fhe_internal.cuh"

namespace fhe {
int pbs_tc(fhe_keys *K, const uint32_t *ct_in, size_t count, const fhe_lut *lut,
           uint32_t *ct_out, cudaStream_t st) {
  (void)K; (void)ct_in; (void)count; (void)lut; (void)ct_out; (void)st;
  return FHE_EUNSUPPORTED;
}
}  // namespace fhe
