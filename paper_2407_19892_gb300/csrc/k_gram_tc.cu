// Tensor-core (tcgen05) Gram.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace gmgm {

int gram_tc_splits(gmgm_handle*, const gmgm_matrix*) { return 1; }

cudaError_t launch_gram_tc(gmgm_handle*, const gmgm_matrix*, gmgm_prec, double*, int64_t, int, float*, int) {
  return cudaErrorNotSupported;
}

}  // namespace gmgm
