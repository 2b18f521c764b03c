// Tensor-core (tcgen05) screen for the top-k network path.
#include <cuda_runtime.h>

#include "internal.cuh"
#include "topk_common.cuh"

namespace gmgm {

size_t topk_tc_scratch_bytes(int64_t, int, gmgm_prec) { return 0; }

cudaError_t launch_screen_tc(gmgm_handle*, int64_t, int, const void*, int, int64_t, const double*, gmgm_prec,
                             int32_t*, float*, float*, void*) {
  return cudaErrorNotSupported;
}

}  // namespace gmgm
