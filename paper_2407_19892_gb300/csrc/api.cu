// C-ABI entry points: argument checks, scratch management and dispatch.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <string>

#include "device.cuh"
#include "internal.cuh"

namespace gmgm {

int fail(gmgm_handle* h, int code, const std::string& msg) {
  if (h) h->last_error = msg;
  return code;
}

static std::atomic<unsigned long long> g_launches{0};

void note_launch(int n) { g_launches.fetch_add(static_cast<unsigned long long>(n), std::memory_order_relaxed); }

// Host-side fault injection: GMGM_FAULT holds a comma-separated list of
// injected failures ("alloc": a scratch allocation that has to grow fails).
// The failure is produced on the host; nothing is faulted on the device.
bool fault_injected(const char* what) {
  const char* f = std::getenv("GMGM_FAULT");
  return f && std::strstr(f, what);
}

// A bounded wait on a device word that nothing sets: after `spins` polls
// the TIMEOUT status bit is set and the kernel returns (the path every
// spinning kernel takes when a wait gives up).
__global__ void probe_wait_kernel(const unsigned* flag, long long spins, int* status) {
  if (threadIdx.x != 0) return;
  const volatile unsigned* f = flag;
  for (long long i = 0; i < spins; ++i) {
    if (*f != 0u) return;
    __nanosleep(100);
  }
  set_status(status, GMGM_DEV_TIMEOUT);
}

int ensure_scratch(gmgm_handle* h, size_t bytes) {
  if (bytes <= h->scratch_bytes) return GMGM_OK;
  if (fault_injected("alloc")) return fail(h, GMGM_E_NOMEM, "scratch allocation failed (injected: GMGM_FAULT=alloc)");
  if (h->scratch) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_bytes = 0;
  }
  size_t want = bytes + (bytes >> 3);
  cudaError_t e = cudaMalloc(&h->scratch, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, GMGM_E_NOMEM, std::string("scratch cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->scratch_bytes = want;
  return GMGM_OK;
}

}  // namespace gmgm

using gmgm::fail;

extern "C" {

const char* gmgm_version(void) { return "gmgm 0.1 sm_103a"; }

uint64_t gmgm_kernel_launches(void) { return gmgm::g_launches.load(std::memory_order_relaxed); }

int gmgm_create(gmgm_handle** out, int device, void* stream) {
  if (!out) return GMGM_E_ARG;
  *out = nullptr;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return GMGM_E_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GMGM_E_CUDA;
  }
  gmgm_handle* h = new gmgm_handle();
  h->device = device;
  h->stream = static_cast<cudaStream_t>(stream);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&h->d_status, 64) != cudaSuccess ||
      cudaMalloc(&h->d_barrier, 64) != cudaSuccess ||
      cudaMemset(h->d_status, 0, 64) != cudaSuccess ||
      cudaMemset(h->d_barrier, 0, 64) != cudaSuccess) {
    cudaGetLastError();
    if (h->d_status) cudaFree(h->d_status);
    if (h->d_barrier) cudaFree(h->d_barrier);
    delete h;
    cudaSetDevice(cur);
    return GMGM_E_CUDA;
  }
  cudaSetDevice(cur);
  *out = h;
  return GMGM_OK;
}

int gmgm_destroy(gmgm_handle* h) {
  if (!h) return GMGM_E_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->scratch) cudaFree(h->scratch);
  cudaFree(h->d_status);
  cudaFree(h->d_barrier);
  cudaSetDevice(cur);
  delete h;
  return GMGM_OK;
}

int gmgm_set_stream(gmgm_handle* h, void* stream) {
  if (!h) return GMGM_E_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return GMGM_OK;
}

const char* gmgm_last_error(const gmgm_handle* h) { return h ? h->last_error.c_str() : "null handle"; }

int gmgm_device_status(gmgm_handle* h) {
  if (!h) return GMGM_E_ARG;
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  GMGM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  int st = 0;
  GMGM_CUDA_TRY(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  GMGM_CUDA_TRY(h, cudaMemset(h->d_status, 0, sizeof(int)));
  return st;
}

int gmgm_probe_wait(gmgm_handle* h, int64_t spins) {
  if (!h) return GMGM_E_ARG;
  if (spins < 1 || spins > (int64_t(1) << 20)) return fail(h, GMGM_E_ARG, "gmgm_probe_wait: need 1 <= spins <= 2^20");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  unsigned* flag = h->d_barrier + 8;  // a word no kernel writes
  GMGM_CUDA_TRY(h, cudaMemsetAsync(flag, 0, sizeof(unsigned), h->stream));
  gmgm::probe_wait_kernel<<<1, 32, 0, h->stream>>>(flag, spins, h->d_status);
  GMGM_CUDA_TRY(h, cudaGetLastError());
  return GMGM_OK;
}

int gmgm_preprocess(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc,
                    float* x_out, int64_t ldx, uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t,
                    double* colmean_out) {
  if (!h) return GMGM_E_ARG;
  if (n < 2 || p < 1 || !counts || (!x_out && !xt_hi) || ldc < p || (x_out && ldx < p))
    return fail(h, GMGM_E_ARG, "gmgm_preprocess: need n >= 2, p >= 1, ldc, ldx >= p, counts and x_out or the planes");
  if ((const void*)counts == (const void*)x_out && ldc != ldx)
    return fail(h, GMGM_E_ARG, "gmgm_preprocess: in-place needs ldx == ldc");
  if ((xt_hi == nullptr) != (xt_lo == nullptr))
    return fail(h, GMGM_E_ARG, "gmgm_preprocess: xt_hi and xt_lo must both be set or both NULL");
  if (xt_hi && (ld_t < n || ld_t % 64 != 0 || ((uintptr_t)xt_hi % 16) || ((uintptr_t)xt_lo % 16)))
    return fail(h, GMGM_E_ARG, "gmgm_preprocess: ld_t must be >= n, a multiple of 64, 16-byte aligned xt");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, size_t(p) * sizeof(double) + 256);
  if (rc) return rc;
  GMGM_CUDA_TRY(h, gmgm::launch_preprocess(h, n, p, counts, ldc, x_out, ldx, xt_hi, xt_lo, ld_t,
                                           static_cast<double*>(h->scratch), colmean_out));
  return GMGM_OK;
}

int gmgm_skeptic(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, int axis, float* z_out,
                 int64_t ldz, uint16_t* zt_hi, uint16_t* zt_lo, int64_t ld_t, int32_t* ranks_out, int64_t ldr) {
  if (!h) return GMGM_E_ARG;
  if (n < 1 || p < 1 || n > (int64_t(1) << 31) - 2 || p > (int64_t(1) << 31) - 2 || !counts || ldc < p)
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: need 1 <= n, p < 2^31, ldc >= p, non-null counts");
  if (axis != GMGM_AXIS_ROWS && axis != GMGM_AXIS_COLS)
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: axis must be GMGM_AXIS_ROWS or GMGM_AXIS_COLS");
  if (!z_out && !zt_hi && !ranks_out) return fail(h, GMGM_E_ARG, "gmgm_skeptic: no output requested");
  if ((z_out && ldz < p) || (ranks_out && ldr < p))
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: ldz, ldr must be >= p");
  if ((zt_hi == nullptr) != (zt_lo == nullptr))
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: zt_hi and zt_lo must both be set or both NULL");
  if (zt_hi && (ld_t < n || ld_t % 64 != 0 || ((uintptr_t)zt_hi % 16) || ((uintptr_t)zt_lo % 16)))
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: ld_t must be >= n, a multiple of 64, 16-byte aligned planes");
  if (axis == GMGM_AXIS_ROWS && zt_hi && !z_out)
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: GMGM_AXIS_ROWS writes the planes from z_out; pass z_out");
  if ((const void*)z_out == (const void*)counts)
    return fail(h, GMGM_E_ARG, "gmgm_skeptic: z_out must not alias counts");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  if (axis == GMGM_AXIS_ROWS)
    return gmgm::skeptic_rows(h, n, p, counts, ldc, z_out, ldz, zt_hi, zt_lo, ld_t, ranks_out, ldr);
  return gmgm::skeptic_cols(h, n, p, counts, ldc, z_out, ldz, zt_hi, zt_lo, ld_t, ranks_out, ldr);
}

int gmgm_gram(gmgm_handle* h, const gmgm_matrix* m, int side, gmgm_prec prec, double* S,
              int64_t lds, int accumulate) {
  if (!h) return GMGM_E_ARG;
  if (!m || !S || m->batch < 1 || m->rows < 1 || m->cols < 1)
    return fail(h, GMGM_E_ARG, "gmgm_gram: null argument or empty shape");
  if (side != GMGM_SIDE_COLS && side != GMGM_SIDE_ROWS)
    return fail(h, GMGM_E_ARG, "gmgm_gram: side must be GMGM_SIDE_COLS or GMGM_SIDE_ROWS");
  const int64_t dS = side == GMGM_SIDE_COLS ? m->cols : m->rows;
  if (lds < dS) return fail(h, GMGM_E_ARG, "gmgm_gram: lds < size of S");
  if (dS > 65536) return fail(h, GMGM_E_ARG, "gmgm_gram: S larger than 65536 x 65536");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  if (prec == GMGM_FP32) {
    if (!m->x || m->ld < m->cols || (m->batch > 1 && m->batch_stride < m->rows * m->ld))
      return fail(h, GMGM_E_ARG, "gmgm_gram: FP32 needs x, ld >= cols, batch_stride >= rows*ld");
    int splits = gmgm::gram_fp32_splits(h, m, side);
    int rc = gmgm::ensure_scratch(h, gmgm::gram_fp32_scratch_bytes(dS, splits));
    if (rc) return rc;
    GMGM_CUDA_TRY(h, gmgm::launch_gram_fp32(h, m, side, S, lds, accumulate,
                                            static_cast<float*>(h->scratch), splits));
    return GMGM_OK;
  }
  if (prec == GMGM_BF16 || prec == GMGM_BF16X3) {
    if (side != GMGM_SIDE_COLS || m->batch != 1)
      return fail(h, GMGM_E_ARG, "gmgm_gram: tensor-core Gram supports side COLS, batch 1");
    if (!m->xt_hi || (prec == GMGM_BF16X3 && !m->xt_lo) || m->ld_t < m->rows || m->ld_t % 64)
      return fail(h, GMGM_E_ARG, "gmgm_gram: BF16 needs xt_hi (+ xt_lo for BF16X3), ld_t >= rows, % 64");
    if (((uintptr_t)m->xt_hi % 16) || (m->xt_lo && ((uintptr_t)m->xt_lo % 16)))
      return fail(h, GMGM_E_ARG, "gmgm_gram: xt buffers must be 16-byte aligned");
    int splits = gmgm::gram_tc_splits(h, m);
    int rc = gmgm::ensure_scratch(h, gmgm::gram_tc_scratch_bytes(h, m));
    if (rc) return rc;
    GMGM_CUDA_TRY(h, gmgm::launch_gram_tc(h, m, prec, S, lds, accumulate,
                                          static_cast<float*>(h->scratch), splits));
    return GMGM_OK;
  }
  return fail(h, GMGM_E_ARG, "gmgm_gram: unsupported precision");
}

int gmgm_spectra(gmgm_handle* h, int64_t d, const double* S, int64_t lds, int32_t r,
                 double* evals, int32_t rv, double* evecs, int64_t ldv) {
  if (!h) return GMGM_E_ARG;
  if (d < 1 || d > 8192 || r < 1 || r > d || !S || !evals || lds < d)
    return fail(h, GMGM_E_ARG, "gmgm_spectra: need 1 <= r <= d <= 8192, lds >= d");
  if (rv < 0 || rv > r || (rv > 0) != (evecs != nullptr) || (rv > 0 && ldv < rv))
    return fail(h, GMGM_E_ARG, "gmgm_spectra: need 0 <= rv <= r, evecs non-null iff rv > 0, ldv >= rv");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, gmgm::eig_scratch_bytes(d, r, rv));
  if (rc) return rc;
  GMGM_CUDA_TRY(h, gmgm::launch_eig(h, d, S, lds, r, evals, nullptr, rv, evecs, ldv, h->scratch));
  return GMGM_OK;
}

int gmgm_lift(gmgm_handle* h, const gmgm_matrix* m, int32_t r, const double* W, int64_t ldw,
              const double* E, float* U, int64_t ldu) {
  if (!h) return GMGM_E_ARG;
  if (!m || m->batch != 1 || m->rows < 1 || m->cols < 1)
    return fail(h, GMGM_E_ARG, "gmgm_lift: need one matrix");
  if (r < 1 || r > 256 || r > m->cols || !W || !E || !U || ldw < r || ldu < r)
    return fail(h, GMGM_E_ARG, "gmgm_lift: need 1 <= r <= min(256, cols), ldw, ldu >= r");
  if ((m->xt_hi != nullptr) != (m->xt_lo != nullptr))
    return fail(h, GMGM_E_ARG, "gmgm_lift: xt_hi and xt_lo must both be set or both be NULL");
  if (m->xt_hi && (m->ld_t < m->rows || m->ld_t % 64 != 0))
    return fail(h, GMGM_E_ARG, "gmgm_lift: need ld_t >= rows, ld_t % 64 == 0 with the BF16 planes");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  if (gmgm::lift_tc_eligible(m, r)) {
    int rc = gmgm::ensure_scratch(h, gmgm::lift_tc_scratch_bytes(m));
    if (rc) return rc;
    GMGM_CUDA_TRY(h, gmgm::launch_lift_tc(h, m, r, W, ldw, E, U, ldu, h->scratch));
    return GMGM_OK;
  }
  if (!m->x || m->ld < m->cols)
    return fail(h, GMGM_E_ARG, "gmgm_lift: need the FP32 matrix (or its BF16 planes with r <= 64)");
  int rc = gmgm::ensure_scratch(h, size_t(m->cols) * ((r + 63) / 64) * 64 * sizeof(float) + 256);
  if (rc) return rc;
  GMGM_CUDA_TRY(h, gmgm::launch_lift(h, m, r, W, ldw, E, U, ldu, static_cast<float*>(h->scratch)));
  return GMGM_OK;
}

int gmgm_eigsolve(gmgm_handle* h, const gmgm_problem* p, const double* const* init,
                  const gmgm_solve_opts* o, double* const* lambda_out, gmgm_solve_stats* stats) {
  if (!h) return GMGM_E_ARG;
  if (!p || !lambda_out) return fail(h, GMGM_E_ARG, "gmgm_eigsolve: null problem or output");
  if (p->n_axes < 1 || p->n_axes > GMGM_MAX_AXES || p->n_modalities < 1 ||
      p->n_modalities > GMGM_MAX_MODALITIES)
    return fail(h, GMGM_E_ARG, "gmgm_eigsolve: bad axis or modality count");
  int64_t total = 0;
  for (int a = 0; a < p->n_axes; ++a) {
    if (p->r[a] < 1 || !p->E[a] || !lambda_out[a] || (init && !init[a]))
      return fail(h, GMGM_E_ARG, "gmgm_eigsolve: bad rank or null pointer for an axis");
    total += p->r[a];
  }
  if (total > 16384) return fail(h, GMGM_E_ARG, "gmgm_eigsolve: sum of ranks > 16384");
  int used[GMGM_MAX_AXES] = {0, 0, 0, 0};
  for (int g = 0; g < p->n_modalities; ++g) {
    int k = p->mod_n_axes[g];
    if (k < 1 || k > GMGM_MAX_AXES) return fail(h, GMGM_E_ARG, "gmgm_eigsolve: bad modality size");
    int64_t pts = 1;
    int seen = 0;
    for (int q = 0; q < k; ++q) {
      int a = p->mod_axes[g][q];
      if (a < 0 || a >= p->n_axes || (seen & (1 << a)))
        return fail(h, GMGM_E_ARG, "gmgm_eigsolve: bad or repeated axis in a modality");
      seen |= 1 << a;
      used[a] = 1;
      pts *= p->r[a];
    }
    if (pts > (int64_t(1) << 31)) return fail(h, GMGM_E_ARG, "gmgm_eigsolve: grid too large");
  }
  for (int a = 0; a < p->n_axes; ++a)
    if (!used[a]) return fail(h, GMGM_E_ARG, "gmgm_eigsolve: an axis is in no modality");
  gmgm_solve_opts opt = {1e-9, 200, 200, 1, 1, 0.0};
  if (o) {
    opt = *o;
    if (opt.tol <= 0) opt.tol = 1e-9;
    if (opt.max_newton <= 0) opt.max_newton = 200;
    if (opt.max_cg <= 0) opt.max_cg = 200;
  }
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  size_t need = gmgm::solve_scratch_bytes(p) + sizeof(gmgm_solve_stats) + 512;
  int rc = gmgm::ensure_scratch(h, need);
  if (rc) return rc;
  gmgm_solve_stats* d_stats = reinterpret_cast<gmgm_solve_stats*>(
      static_cast<char*>(h->scratch) + gmgm::Carve::round(gmgm::solve_scratch_bytes(p)));
  GMGM_CUDA_TRY(h, gmgm::launch_solve(h, p, init, &opt, lambda_out, h->scratch, d_stats));
  if (stats) {
    GMGM_CUDA_TRY(h, cudaMemcpyAsync(stats, d_stats, sizeof(gmgm_solve_stats),
                                     cudaMemcpyDeviceToHost, h->stream));
    GMGM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (stats->status != GMGM_OK)
      return fail(h, stats->status, "gmgm_eigsolve: device solve did not reach tolerance");
  }
  return GMGM_OK;
}

// ---- learned warm start ----------------------------------------------------

static int ws_check_axes(gmgm_handle* h, const double* E0, int32_t r0, const double* E1, int32_t r1,
                         const char* who) {
  if (!E0 || !E1 || r0 < 2 || r1 < 2)
    return fail(h, GMGM_E_ARG, std::string(who) + ": need two axes with ranks >= 2");
  return GMGM_OK;
}

int gmgm_warmstart_features(gmgm_handle* h, const double* E0, int32_t r0, const double* E1, int32_t r1,
                            float* feats) {
  if (!h) return GMGM_E_ARG;
  int rc = ws_check_axes(h, E0, r0, E1, r1, "gmgm_warmstart_features");
  if (rc) return rc;
  if (!feats) return fail(h, GMGM_E_ARG, "gmgm_warmstart_features: null output");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  GMGM_CUDA_TRY(h, gmgm::launch_features(h, E0, r0, E1, r1, feats));
  return GMGM_OK;
}

int gmgm_warmstart_targets(gmgm_handle* h, const double* E0, int32_t r0, const double* E1, int32_t r1,
                           const double* lam0, const double* lam1, float* targets) {
  if (!h) return GMGM_E_ARG;
  int rc = ws_check_axes(h, E0, r0, E1, r1, "gmgm_warmstart_targets");
  if (rc) return rc;
  if (!lam0 || !lam1 || !targets) return fail(h, GMGM_E_ARG, "gmgm_warmstart_targets: null argument");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  GMGM_CUDA_TRY(h, gmgm::launch_targets(h, E0, r0, E1, r1, lam0, lam1, targets));
  return GMGM_OK;
}

int gmgm_mlp_forward(gmgm_handle* h, const float* params, const float* feats, int32_t n, float* out) {
  if (!h) return GMGM_E_ARG;
  if (!params || !feats || !out || n < 1 || n > (1 << 20))
    return fail(h, GMGM_E_ARG, "gmgm_mlp_forward: need buffers and 1 <= n <= 2^20");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, gmgm::mlp_scratch_bytes(n, 0));
  if (rc) return rc;
  GMGM_CUDA_TRY(h, gmgm::mlp_forward(h, params, feats, n, out, h->scratch));
  return GMGM_OK;
}

int gmgm_mlp_loss_grad(gmgm_handle* h, const float* params, const float* feats, const float* targets, int32_t n,
                       float* grad, float* loss) {
  if (!h) return GMGM_E_ARG;
  if (!params || !feats || !targets || n < 1 || n > (1 << 20))
    return fail(h, GMGM_E_ARG, "gmgm_mlp_loss_grad: need buffers and 1 <= n <= 2^20");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  const size_t need = gmgm::mlp_scratch_bytes(n, 0);
  int rc = gmgm::ensure_scratch(h, need + 512);
  if (rc) return rc;
  float* loss_dev = reinterpret_cast<float*>(static_cast<char*>(h->scratch) + gmgm::Carve::round(need));
  GMGM_CUDA_TRY(h, gmgm::mlp_loss_grad(h, params, feats, targets, n, grad, loss_dev, h->scratch));
  if (loss) {
    GMGM_CUDA_TRY(h, cudaMemcpyAsync(loss, loss_dev, 4, cudaMemcpyDeviceToHost, h->stream));
    GMGM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return GMGM_OK;
}

int gmgm_warmstart_train(gmgm_handle* h, float* params, float* adam_state, const float* feats, const float* targets,
                         int32_t n, const gmgm_train_opts* opts, float* final_loss) {
  if (!h) return GMGM_E_ARG;
  if (!params || !adam_state || !feats || !targets || !opts || n < 1 || n > (1 << 20) || opts->steps < 0 ||
      opts->steps > (1 << 24) || opts->batch < 1 || !(opts->lr > 0.f))
    return fail(h, GMGM_E_ARG, "gmgm_warmstart_train: bad buffers or options");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  const int B = opts->batch < n ? opts->batch : n;
  const size_t need = gmgm::mlp_scratch_bytes(B, opts->steps);
  int rc = gmgm::ensure_scratch(h, need + 512);
  if (rc) return rc;
  float* loss_dev = reinterpret_cast<float*>(static_cast<char*>(h->scratch) + gmgm::Carve::round(need));
  GMGM_CUDA_TRY(h, gmgm::mlp_train(h, params, adam_state, feats, targets, n, opts, loss_dev, h->scratch));
  if (final_loss) {
    GMGM_CUDA_TRY(h, cudaMemcpyAsync(final_loss, loss_dev, 4, cudaMemcpyDeviceToHost, h->stream));
    GMGM_CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return GMGM_OK;
}

int gmgm_warmstart_infer(gmgm_handle* h, const float* params, const double* E0, int32_t r0, const double* E1,
                         int32_t r1, double eps, double* lam0_out, double* lam1_out) {
  if (!h) return GMGM_E_ARG;
  int rc = ws_check_axes(h, E0, r0, E1, r1, "gmgm_warmstart_infer");
  if (rc) return rc;
  if (!params || !lam0_out || !lam1_out) return fail(h, GMGM_E_ARG, "gmgm_warmstart_infer: null argument");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  rc = gmgm::ensure_scratch(h, gmgm::mlp_scratch_bytes(1, 0));
  if (rc) return rc;
  GMGM_CUDA_TRY(h, gmgm::warmstart_infer(h, params, E0, r0, E1, r1, eps > 0 ? eps : 0.0, lam0_out, lam1_out,
                                         h->scratch));
  return GMGM_OK;
}

int gmgm_topk_network(gmgm_handle* h, int64_t d, int32_t r, const void* V, int v_fp64,
                      int64_t ldv, const double* psi, int32_t k, gmgm_prec prec, uint32_t flags,
                      int32_t* idx_out, float* val_out, gmgm_topk_stats* stats) {
  if (!h) return GMGM_E_ARG;
  if (d < 2 || r < 1 || !V || !psi || !idx_out || !val_out || ldv < r)
    return fail(h, GMGM_E_ARG, "gmgm_topk_network: need d >= 2, r >= 1, ldv >= r, non-null buffers");
  if (k < 1 || k > 32 || k >= d) return fail(h, GMGM_E_ARG, "gmgm_topk_network: need 1 <= k <= 32, k < d");
  if (d > (int64_t(1) << 31) - 1) return fail(h, GMGM_E_ARG, "gmgm_topk_network: d >= 2^31");
  if (r > 4096) return fail(h, GMGM_E_ARG, "gmgm_topk_network: r > 4096");
  if (prec != GMGM_FP32 && prec != GMGM_BF16)
    return fail(h, GMGM_E_ARG, "gmgm_topk_network: prec must be FP32 or BF16");
  if (flags & ~GMGM_TOPK_ORTHO) return fail(h, GMGM_E_ARG, "gmgm_topk_network: unknown flags");
  if ((flags & GMGM_TOPK_ORTHO) && r != d)
    return fail(h, GMGM_E_ARG, "gmgm_topk_network: GMGM_TOPK_ORTHO needs a square V (r == d)");
  if (prec != GMGM_FP32 && r > 64 && !(flags & GMGM_TOPK_ORTHO))
    return fail(h, GMGM_E_ARG, "gmgm_topk_network: tensor-core screen supports r <= 64");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  if (flags & GMGM_TOPK_ORTHO) {
    int rc = gmgm::ensure_scratch(h, gmgm::topk_ortho_scratch_bytes(d, r, k, prec));
    if (rc) return rc;
    return gmgm::topk_run_ortho(h, d, r, V, v_fp64, ldv, psi, k, prec, idx_out, val_out, h->scratch, stats);
  }
  int rc = gmgm::ensure_scratch(h, gmgm::topk_scratch_bytes(d, r, k, prec));
  if (rc) return rc;
  return gmgm::topk_run(h, d, r, V, v_fp64, ldv, psi, k, prec, idx_out, val_out, h->scratch, stats);
}

int gmgm_topk_network_rows(gmgm_handle* h, int64_t d, int32_t r, const void* V, int v_fp64, int64_t ldv,
                           const double* psi, int32_t k, gmgm_prec prec, int64_t row0, int64_t m,
                           int32_t* idx_out, float* val_out, gmgm_topk_stats* stats) {
  if (!h) return GMGM_E_ARG;
  if (d < 2 || r < 1 || !V || !psi || !idx_out || !val_out || ldv < r)
    return fail(h, GMGM_E_ARG, "gmgm_topk_network_rows: need d >= 2, r >= 1, ldv >= r, non-null buffers");
  if (k < 1 || k > 32 || k >= d) return fail(h, GMGM_E_ARG, "gmgm_topk_network_rows: need 1 <= k <= 32, k < d");
  if (d > (int64_t(1) << 31) - 1 || r > 4096) return fail(h, GMGM_E_ARG, "gmgm_topk_network_rows: d >= 2^31 or r > 4096");
  if (row0 < 0 || m < 1 || row0 + m > d) return fail(h, GMGM_E_ARG, "gmgm_topk_network_rows: need 0 <= row0, m >= 1, row0 + m <= d");
  if (prec != GMGM_FP32 && prec != GMGM_BF16)
    return fail(h, GMGM_E_ARG, "gmgm_topk_network_rows: prec must be FP32 or BF16");
  if (prec != GMGM_FP32 && r > 64) return fail(h, GMGM_E_ARG, "gmgm_topk_network_rows: tensor-core screen supports r <= 64");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, gmgm::topk_scratch_bytes(d, r, k, prec));
  if (rc) return rc;
  return gmgm::topk_run(h, d, r, V, v_fp64, ldv, psi, k, prec, idx_out, val_out, h->scratch, stats, row0, m);
}

int gmgm_peak_probe(gmgm_handle* h, int kind, int64_t iters, double* rate) {
  if (!h) return GMGM_E_ARG;
  if ((kind != GMGM_PROBE_FP64 && kind != GMGM_PROBE_SFU) || iters < 1 || iters > (int64_t(1) << 24) || !rate)
    return fail(h, GMGM_E_ARG, "gmgm_peak_probe: kind FP64 or SFU, 1 <= iters <= 2^24, non-null rate");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, 256);
  if (rc) return rc;
  return gmgm::peak_probe(h, kind, iters, rate);
}

int gmgm_preprocess_csr(gmgm_handle* h, int64_t n, int64_t p, const int64_t* indptr, const int32_t* indices,
                        const float* data, uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t, double* colmean_out) {
  if (!h) return GMGM_E_ARG;
  if (n < 1 || p < 1 || p > 16384 || n > (int64_t(1) << 31) - 1 || !indptr || !indices || !data || !xt_hi ||
      !xt_lo)
    return fail(h, GMGM_E_ARG, "gmgm_preprocess_csr: need n >= 1, 1 <= p <= 16384, non-null buffers");
  if (ld_t < n || ld_t % 64 != 0 || ((uintptr_t)xt_hi % 16) || ((uintptr_t)xt_lo % 16))
    return fail(h, GMGM_E_ARG, "gmgm_preprocess_csr: ld_t must be >= n, a multiple of 64, 16-byte aligned planes");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, gmgm::preprocess_csr_scratch_bytes(p));
  if (rc) return rc;
  GMGM_CUDA_TRY(h, gmgm::launch_preprocess_csr(h, n, p, indptr, indices, data, xt_hi, xt_lo, ld_t, colmean_out));
  return GMGM_OK;
}

int gmgm_colsum_log1p(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, double* colsum,
                      int accumulate) {
  if (!h) return GMGM_E_ARG;
  if (n < 1 || p < 1 || !counts || !colsum || ldc < p)
    return fail(h, GMGM_E_ARG, "gmgm_colsum_log1p: need n, p >= 1, ldc >= p, non-null buffers");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  GMGM_CUDA_TRY(h, gmgm::launch_colsum_log1p(h, n, p, counts, ldc, colsum, accumulate));
  return GMGM_OK;
}

int gmgm_centre(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, const double* colsum,
                int64_t n_total, float* x_out, int64_t ldx, uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t) {
  if (!h) return GMGM_E_ARG;
  if (n < 1 || p < 1 || n_total < n || !counts || !colsum || !x_out || ldc < p || ldx < p)
    return fail(h, GMGM_E_ARG, "gmgm_centre: need 1 <= n <= n_total, p >= 1, ldc, ldx >= p, non-null buffers");
  if ((const void*)counts == (const void*)x_out && ldc != ldx)
    return fail(h, GMGM_E_ARG, "gmgm_centre: in-place needs ldx == ldc");
  if ((xt_hi == nullptr) != (xt_lo == nullptr))
    return fail(h, GMGM_E_ARG, "gmgm_centre: xt_hi and xt_lo must both be set or both NULL");
  if (xt_hi && (ld_t < n || ld_t % 64 != 0 || ((uintptr_t)xt_hi % 16) || ((uintptr_t)xt_lo % 16)))
    return fail(h, GMGM_E_ARG, "gmgm_centre: ld_t must be >= n, a multiple of 64, 16-byte aligned xt");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  GMGM_CUDA_TRY(h, gmgm::launch_centre(h, n, p, counts, ldc, colsum, n_total, x_out, ldx, xt_hi, xt_lo, ld_t));
  return GMGM_OK;
}

int gmgm_topn_edges(gmgm_handle* h, int64_t d, int32_t k, const int32_t* idx, const float* val, int64_t n,
                    int32_t* i_out, int32_t* j_out, float* v_out, int64_t* count, int* certified) {
  if (!h) return GMGM_E_ARG;
  if (d < 2 || d > (int64_t(1) << 31) - 1 || k < 1 || k >= d || !idx || !val || !i_out || !j_out || !v_out ||
      !count || !certified)
    return fail(h, GMGM_E_ARG, "gmgm_topn_edges: need 2 <= d < 2^31, 1 <= k < d, non-null buffers");
  if (n < 1 || n > d * int64_t(k) || n > (int64_t(1) << 30))
    return fail(h, GMGM_E_ARG, "gmgm_topn_edges: need 1 <= n <= d k, n <= 2^30");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, gmgm::topn_scratch_bytes(d, k, n));
  if (rc) return rc;
  return gmgm::topn_run(h, d, k, idx, val, n, i_out, j_out, v_out, count, certified);
}

int gmgm_topk_network_gram(gmgm_handle* h, int64_t d, const double* S, int64_t lds, const double* psi,
                           int32_t k, gmgm_prec prec, int32_t* idx_out, float* val_out, gmgm_topk_stats* stats) {
  if (!h) return GMGM_E_ARG;
  if (d < 2 || d > 8192 || !S || !psi || !idx_out || !val_out || lds < d)
    return fail(h, GMGM_E_ARG, "gmgm_topk_network_gram: need 2 <= d <= 8192, lds >= d, non-null buffers");
  if (k < 1 || k > 32 || k >= d) return fail(h, GMGM_E_ARG, "gmgm_topk_network_gram: need 1 <= k <= 32, k < d");
  if (prec != GMGM_FP32 && prec != GMGM_BF16)
    return fail(h, GMGM_E_ARG, "gmgm_topk_network_gram: prec must be FP32 or BF16");
  GMGM_CUDA_TRY(h, cudaSetDevice(h->device));
  int rc = gmgm::ensure_scratch(h, gmgm::topk_gram_scratch_bytes(d, k, prec));
  if (rc) return rc;
  return gmgm::topk_run_gram(h, d, S, lds, psi, k, prec, idx_out, val_out, h->scratch, stats);
}

}  // extern "C"
