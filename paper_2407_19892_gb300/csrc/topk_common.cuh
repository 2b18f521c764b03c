// Shared pieces of the top-k network path: candidate-list size, list update,
// and the launchers implemented across k_topk.cu / k_topk_tc.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gmgm.h"

struct gmgm_handle;

namespace gmgm {

constexpr int kC = 32;  // candidate slots per row in every screen

// Offer (|value| v, column j) to a row's unsorted candidate list of kC
// slots.  While the list fills, every offer is taken; afterwards an offer
// replaces the current minimum only if strictly larger, so at any time every
// column not in the list has a screened value <= minv.
__device__ __forceinline__ void list_offer(float* lv, int* li, int& cnt, float& minv, int& minpos, float v, int j) {
  if (cnt < kC) {
    lv[cnt] = v;
    li[cnt] = j;
    ++cnt;
    if (cnt == kC) {
      minv = lv[0];
      minpos = 0;
      for (int c = 1; c < kC; ++c)
        if (lv[c] < minv) minv = lv[c], minpos = c;
    }
    return;
  }
  if (v > minv) {
    lv[minpos] = v;
    li[minpos] = j;
    minv = lv[0];
    minpos = 0;
    for (int c = 1; c < kC; ++c)
      if (lv[c] < minv) minv = lv[c], minpos = c;
  }
}

// |screen - exact| <= screen_unit(prec, r) * sum_k |psi_k V_ik| max_j |V_jk|
double screen_unit(gmgm_prec prec, int r);

// rescore + certify m rows (all rows, or rows[] with m or a device-side
// count); candidate layout by nl and lstride as in rescore_kernel
void launch_rescore(cudaStream_t s, int64_t d, int r, const void* V, int v64, int64_t ldv, const double* psi, int k,
                    const int* rows, const int* count_dev, const int32_t* cidx, const float* cval,
                    const float* thr, int nl, int64_t lstride, int64_t m, const unsigned* colmax_bits, double u,
                    int32_t* idx, float* val, int64_t orow0, int* flag_list, int* flag_count, unsigned* err_bits);

// tensor-core screens: BF16 over all rows; 3xBF16 over m listed rows in ncs
// column slices (candidate arrays hold ncs * m list pairs)
size_t topk_tc_scratch_bytes(int64_t d, int r, gmgm_prec prec);
int screen_tc_slices(int64_t m, int num_sms, int64_t cap_rows);
// (the rows [row0, row0 + m) of Psi, listed in `rows`, or every row when
// rows is null)
cudaError_t launch_screen_tc(gmgm_handle* h, int64_t d, int r, const void* V, int v64, int64_t ldv,
                             const double* psi, gmgm_prec prec, int32_t* cidx, float* cval, float* thr,
                             void* scratch, int64_t row0, int64_t m, const int* rows,
                             unsigned long long* tiles_run);  // (may be null) += B tiles multiplied
cudaError_t launch_screen_tc_repair(gmgm_handle* h, int64_t d, int r, const void* V, int v64, int64_t ldv,
                                    const double* psi, const int* rows, int m, int ncs, int32_t* cidx, float* cval,
                                    float* thr, void* scratch);

}  // namespace gmgm
