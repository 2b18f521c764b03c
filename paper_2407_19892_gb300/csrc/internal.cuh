// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "gmgm.h"

struct gmgm_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  // device status word (OR of GMGM_DEV_* bits) + grid-barrier words
  int* d_status = nullptr;
  unsigned* d_barrier = nullptr;  // [0] = arrivals in the current launch, [2] = abort flag
  // lazily grown scratch arena
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  std::string last_error;
};

namespace gmgm {

// Set the handle's message and return `code`.
int fail(gmgm_handle* h, int code, const std::string& msg);

// Count kernel launches issued by the library (process-wide diagnostic).
void note_launch(int n = 1);

// Ensure the scratch arena holds at least `bytes`; returns GMGM_OK or an
// error (the arena is synchronised and re-allocated when it grows).
int ensure_scratch(gmgm_handle* h, size_t bytes);

// Bump allocator over the scratch arena (256-byte aligned slices).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
  static size_t round(size_t n) { return (n + 255) & ~size_t(255); }
};

// Check a CUDA call; on failure record the message and return GMGM_E_CUDA.
#define GMGM_CUDA_TRY(h, call)                                               \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      return ::gmgm::fail((h), GMGM_E_CUDA,                                  \
                          std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

// ---- kernel launchers (return cudaError_t of the launch) ----

cudaError_t launch_preprocess(gmgm_handle* h, int64_t n, int64_t p, const float* counts,
                              int64_t ldc, float* x_out, int64_t ldx, uint16_t* xt_hi,
                              uint16_t* xt_lo, int64_t ld_t, double* colsum_scratch,
                              double* colmean_out);

// throughput probes: kind 0 FP64 FMA (flop/s), 1 special-function unit
// (reciprocal + base-2 logarithm operations/s)
int peak_probe(gmgm_handle* h, int kind, long long iters, double* rate);

// preprocessing of a CSR count matrix straight into the BF16 planes of X^T
size_t preprocess_csr_scratch_bytes(int64_t p);
cudaError_t launch_preprocess_csr(gmgm_handle* h, int64_t n, int64_t p, const int64_t* indptr, const int32_t* indices,
                                  const float* data, uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t,
                                  double* colmean_out);

// row-split preprocessing: column sums of log1p over a row block, and the
// centring of a row block by given column sums over n_total rows
cudaError_t launch_colsum_log1p(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc,
                                double* colsum, int accumulate);
cudaError_t launch_centre(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc,
                          const double* colsum, int64_t n_total, float* x_out, int64_t ldx, uint16_t* xt_hi,
                          uint16_t* xt_lo, int64_t ld_t);

cudaError_t launch_gram_fp32(gmgm_handle* h, const gmgm_matrix* m, int side, double* S,
                             int64_t lds, int accumulate, float* partials, int splits);
int gram_fp32_splits(gmgm_handle* h, const gmgm_matrix* m, int side);
size_t gram_fp32_scratch_bytes(int64_t dS, int splits);

cudaError_t launch_gram_tc(gmgm_handle* h, const gmgm_matrix* m, gmgm_prec prec, double* S,
                           int64_t lds, int accumulate, float* partials, int splits);
int gram_tc_splits(gmgm_handle* h, const gmgm_matrix* m);
size_t gram_tc_scratch_bytes(gmgm_handle* h, const gmgm_matrix* m);

// FP64 eigendecomposition of S: the nval largest eigenvalues (descending)
// and eigenvectors for the nvec largest, or for the ascending eigenvalue
// indices vlist[0..nvec) (device) when vlist is given
size_t eig_scratch_bytes(int64_t d, int32_t nval, int32_t nvec);
cudaError_t launch_eig(gmgm_handle* h, int64_t d, const double* S, int64_t lds, int32_t nval, double* evals,
                       const int* vlist, int32_t nvec, double* evecs, int64_t ldv, void* scratch);

cudaError_t launch_lift(gmgm_handle* h, const gmgm_matrix* m, int32_t r, const double* W,
                        int64_t ldw, const double* E, float* U, int64_t ldu, float* wscr);
// tensor-core lift from the BF16 planes of X^T (r <= 64)
bool lift_tc_eligible(const gmgm_matrix* m, int32_t r);
size_t lift_tc_scratch_bytes(const gmgm_matrix* m);
cudaError_t launch_lift_tc(gmgm_handle* h, const gmgm_matrix* m, int32_t r, const double* W, int64_t ldw,
                           const double* E, float* U, int64_t ldu, void* scratch);

// rank-based scores (Nonparanormal Skeptic / COCA) of a count matrix
int skeptic_rows(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, float* z, int64_t ldz,
                 uint16_t* hi, uint16_t* lo, int64_t ld_t, int32_t* ranks, int64_t ldr);
int skeptic_cols(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, float* z, int64_t ldz,
                 uint16_t* hi, uint16_t* lo, int64_t ld_t, int32_t* ranks, int64_t ldr);

// global top-n edges from per-row top-k lists
size_t topn_scratch_bytes(int64_t d, int32_t k, int64_t n);
int topn_run(gmgm_handle* h, int64_t d, int32_t k, const int32_t* idx, const float* val, int64_t n, int32_t* io,
             int32_t* jo, float* vo, int64_t* count_out, int* certified_out);

struct SolveDesc;  // defined in k_solve.cu
size_t solve_scratch_bytes(const gmgm_problem* p);
cudaError_t launch_solve(gmgm_handle* h, const gmgm_problem* p, const double* const* init,
                         const gmgm_solve_opts* o, double* const* out, void* scratch,
                         gmgm_solve_stats* d_stats);

size_t mlp_scratch_bytes(int batch, int64_t steps);
cudaError_t launch_features(gmgm_handle* h, const double* E0, int r0, const double* E1, int r1, float* out);
cudaError_t launch_targets(gmgm_handle* h, const double* E0, int r0, const double* E1, int r1, const double* l0,
                           const double* l1, float* out);
cudaError_t mlp_forward(gmgm_handle* h, const float* P, const float* X, int B, float* out, void* scratch);
cudaError_t mlp_loss_grad(gmgm_handle* h, const float* P, const float* X, const float* T, int B, float* G,
                          float* loss_dev, void* scratch);
cudaError_t mlp_train(gmgm_handle* h, float* P, float* adam, const float* X, const float* T, int n,
                      const gmgm_train_opts* o, float* loss_dev, void* scratch);
cudaError_t warmstart_infer(gmgm_handle* h, const float* P, const double* E0, int r0, const double* E1, int r1,
                            double eps, double* l0, double* l1, void* scratch);

size_t topk_scratch_bytes(int64_t d, int32_t r, int32_t k, gmgm_prec prec);
// rows [row0, row0 + m) of Psi (m < 0: every row); idx, val hold m x k
int topk_run(gmgm_handle* h, int64_t d, int32_t r, const void* V, int v_fp64, int64_t ldv,
             const double* psi, int32_t k, gmgm_prec prec, int32_t* idx, float* val,
             void* scratch, gmgm_topk_stats* st, int64_t row0 = 0, int64_t m = -1);
// V square (r == d) with orthonormal columns: Psi = c I + V diag(psi - c) V^T
// with c = min psi; the network is that of the columns with psi > c
size_t topk_ortho_scratch_bytes(int64_t d, int32_t r, int32_t k, gmgm_prec prec);
// the network of W diag(psi) W^T for W the eigenvectors of S (full rank),
// eigenvectors formed only for the eigenvalues whose psi exceeds min psi
size_t topk_gram_scratch_bytes(int64_t d, int32_t k, gmgm_prec prec);
int topk_run_gram(gmgm_handle* h, int64_t d, const double* S, int64_t lds, const double* psi, int32_t k,
                  gmgm_prec prec, int32_t* idx, float* val, void* scratch, gmgm_topk_stats* st);
int topk_run_ortho(gmgm_handle* h, int64_t d, int32_t r, const void* V, int v_fp64, int64_t ldv,
                   const double* psi, int32_t k, gmgm_prec prec, int32_t* idx, float* val,
                   void* scratch, gmgm_topk_stats* st);

}  // namespace gmgm
