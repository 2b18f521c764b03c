/*
 * gmgm.h -- C ABI of the GB300 (sm_103a) implementation of the improved
 * multi-axis Gaussian graphical model fit ("GmGM", arXiv 2407.19892).
 *
 * The model (Introduction; Eq. of Section "The model"): data tensors that
 * share axes are drawn from a Kronecker-sum-structured (singular) normal,
 * precision  Psi_1 (+) Psi_2 (+) ... ; one sparse graph Psi_l per axis is the
 * output.  Algorithm 1 (appendix "The algorithm") fits it in four steps, each
 * an entry point here:
 *
 *   gmgm_gram          S_l = mat_l[D] mat_l[D]^T         (Section "Algorithm")
 *   gmgm_spectra       top-r eigenpairs of S_l           (Theorem 1; Alg. 1)
 *   gmgm_lift          singular vectors of the large axis through the small
 *                      Gram (Section "Algorithm": the eigenvectors of S_l are
 *                      the singular vectors of mat_l[D])
 *   gmgm_eigsolve      eigenvalues Lam_l of the MLE      (Proposition on the
 *                      eigenvalue gradient; existence lemma; Alg. 1 loop)
 *   gmgm_topk_network  thresh(V_l Lam_l V_l^T) fused     (Alg. 1 last loop;
 *                      appendix "Computational complexity": threshold while
 *                      recomposing, O(n_l) memory)
 *
 * plus gmgm_preprocess (log1p + column centring of counts, with the BF16
 * hi/lo split of the transpose that the tensor-core Gram reads).
 *
 * Conventions shared by every entry point:
 *  - Pointers documented "device" must be device memory of the handle's
 *    device; "host" pointers are ordinary host memory.  The caller owns every
 *    input and output buffer.  The library owns only scratch memory, which it
 *    allocates lazily inside the handle and frees in gmgm_destroy.
 *  - Matrices are row-major with an explicit leading dimension (elements).
 *  - Work is enqueued on the handle's stream and the call returns without
 *    synchronising, unless a host-side stats pointer is passed (documented
 *    per call), in which case the call synchronises the stream to fill it.
 *  - Return value: GMGM_OK or a negative gmgm_status.  Argument errors are
 *    detected on the host before anything is enqueued (GMGM_E_ARG; nothing
 *    is modified).  Errors found on the device (non-finite values, solver not
 *    converged, spin-wait timeout) set bits of a device status word that
 *    gmgm_device_status() returns after synchronising.  gmgm_last_error()
 *    gives a message for the last failure.  Invalid input is never silently
 *    repaired, and there is no CPU fallback.
 */
#ifndef GMGM_H_
#define GMGM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmgm_handle gmgm_handle;

typedef enum {
  GMGM_OK = 0,
  GMGM_E_ARG = -1,            /* invalid argument (host-detected) */
  GMGM_E_CUDA = -2,           /* a CUDA runtime call failed */
  GMGM_E_NOMEM = -3,          /* scratch allocation failed */
  GMGM_E_NONFINITE = -4,      /* NaN/Inf met on the device */
  GMGM_E_NOT_CONVERGED = -5,  /* eigenvalue solve hit its iteration cap */
  GMGM_E_INFEASIBLE = -6,     /* no feasible step (all s > 0 lost) */
  GMGM_E_CAND_OVERFLOW = -7,  /* top-k screen could not certify a row */
  GMGM_E_TIMEOUT = -8         /* a bounded device spin-wait gave up */
} gmgm_status;

/* Device status word bits (gmgm_device_status returns their OR, or 0). */
#define GMGM_DEV_NONFINITE 0x1
#define GMGM_DEV_NOT_CONVERGED 0x2
#define GMGM_DEV_INFEASIBLE 0x4
#define GMGM_DEV_CAND_OVERFLOW 0x8
#define GMGM_DEV_TIMEOUT 0x10
#define GMGM_DEV_NOT_COUNTS 0x20  /* gmgm_skeptic met a value that is not a
                                     count (negative, fractional, > 2^24,
                                     NaN or Inf); gmgm_preprocess_csr an entry
                                     that is negative or non-finite, or a
                                     column index out of range or out of
                                     order */

typedef enum {
  GMGM_FP32 = 0,   /* FP32 SIMT arithmetic (the plain comparator form) */
  GMGM_BF16 = 1,   /* BF16 tensor-core products, FP32 accumulation */
  GMGM_BF16X3 = 2, /* 3xBF16 split products (hi*hi + hi*lo + lo*hi), FP32 acc. */
  GMGM_FP64 = 3
} gmgm_prec;

/* ---- handle ------------------------------------------------------------ */

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *h receives the
 * handle.  Returns GMGM_E_CUDA if the device cannot be selected. */
int gmgm_create(gmgm_handle** h, int device, void* cuda_stream);

/* Synchronise the handle's stream, free its scratch memory and the handle. */
int gmgm_destroy(gmgm_handle* h);

/* Re-bind the handle to another stream of the same device. */
int gmgm_set_stream(gmgm_handle* h, void* cuda_stream);

/* Message for the last non-OK return on this handle ("" if none).  The
 * string is owned by the handle and valid until the next call on it. */
const char* gmgm_last_error(const gmgm_handle* h);

/* Synchronise the handle's stream, then return and clear the device status
 * word (an OR of GMGM_DEV_* bits; 0 = no device-side error).  A negative
 * value is a gmgm_status for a failed synchronisation. */
int gmgm_device_status(gmgm_handle* h);

/* Failure-detection check: one kernel polls a device word that nothing
 * sets, `spins` times (1 <= spins <= 2^20, about 100 ns apart), then sets
 * GMGM_DEV_TIMEOUT and returns, the path every spinning kernel of the
 * library takes when a bounded wait gives up.  Enqueued on the handle's
 * stream; read the bit with gmgm_device_status.  The handle stays usable.
 * Errors: GMGM_E_ARG for spins out of range.
 *
 * Host-side fault injection: with the environment variable GMGM_FAULT
 * containing "alloc", every call whose scratch has to grow returns
 * GMGM_E_NOMEM instead of allocating (nothing is faulted on the device). */
int gmgm_probe_wait(gmgm_handle* h, int64_t spins);

/* Throughput probes for roofline denominators no library measures here
 * (not part of the paper): GMGM_PROBE_FP64 runs independent FP64 FMA chains
 * on every SM and returns FP64 flop/s; GMGM_PROBE_SFU runs chains of one
 * approximate reciprocal and one approximate base-2 logarithm per step (the
 * special-function work of one grid term of the eigenvalue solve) and
 * returns special-function operations/s.  `iters` steps per chain
 * (1..2^24); synchronises the stream.  Errors: GMGM_E_ARG. */
#define GMGM_PROBE_FP64 0
#define GMGM_PROBE_SFU 1
int gmgm_peak_probe(gmgm_handle* h, int kind, int64_t iters, double* rate);

/* Library version string, e.g. "gmgm 0.1 sm_103a". */
const char* gmgm_version(void);

/* Number of CUDA kernels this library has launched in this process, over
 * all handles (a diagnostic for benchmarks; not synchronising). */
uint64_t gmgm_kernel_launches(void);

/* ---- preprocessing ------------------------------------------------------ */

/* X = log1p(counts) - column means, for an n x p count matrix (cells x genes).
 *   counts  device, n x p FP32, leading dimension ldc >= p.
 *   x_out   device, n x p FP32, leading dimension ldx >= p; may alias counts
 *           (then ldx must equal ldc).  May be NULL when xt_hi, xt_lo are
 *           given: only the BF16 planes are written (the tensor-core Gram and
 *           lift read nothing else), saving the n p FP32 stores.
 *   xt_hi, xt_lo  device, optional (both NULL or both set): the BF16 split of
 *           X^T, p x ld_t row-major (gene-major), hi = bf16(x),
 *           lo = bf16(x - hi); columns n..ld_t-1 are written as zero.
 *           ld_t >= n and a multiple of 64 (the tensor-core K tile).
 *   colmean_out  device, optional, p FP64 column means of log1p(counts).
 * The paper's own transform is the Nonparanormal Skeptic (Section "The
 * model"); the log1p + centring used here is the transform of the scRNA-like
 * workloads.  Errors: GMGM_E_ARG for n < 2, p < 1, bad strides/alignment. */
int gmgm_preprocess(gmgm_handle* h, int64_t n, int64_t p,
                    const float* counts, int64_t ldc,
                    float* x_out, int64_t ldx,
                    uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t,
                    double* colmean_out);

/* ---- rank-based statistics (Nonparanormal Skeptic, COCA form) ---------- */

#define GMGM_AXIS_ROWS 0  /* rank each row across its p entries (cells x genes:
                             the cell axis, each cell over its genes) */
#define GMGM_AXIS_COLS 1  /* rank each column across the n rows (the gene
                             axis, each gene over the cells) */

/* Normal scores of the ranks of a count matrix along one axis (Section "The
 * model": the Gaussian-copula assumption and the Nonparanormal Skeptic;
 * Section "Algorithm": the COCA form, ranks mapped to a normal distribution
 * before the Gram; the worked example of the appendix "Preserving input
 * sparsity" fixes the conventions).  Along GMGM_AXIS_ROWS each row of the
 * n x p matrix is ranked across its p entries; along GMGM_AXIS_COLS each
 * column across its n entries.  The rank of an entry is 1 + the number of
 * strictly smaller entries of its row (column), so ties take the lowest
 * rank of their group; rank k of N entries maps to the score
 * Phi^-1(k / (N + 1)), evaluated in FP64 and rounded to FP32.  The axis'
 * Gram is then the Gram of the scores (S_genes = Z^T Z for the column
 * scores Z; the cell axis through the dual Gram of the row scores), with
 * no re-centring.
 *   counts     device, n x p FP32, leading dimension ldc >= p: counts, i.e.
 *              non-negative integers <= 2^24 (ranks come from counting, not
 *              sorting).  Any other value sets GMGM_DEV_NOT_COUNTS in the
 *              device status word and leaves the outputs undefined.
 *   z_out      device, optional, n x p FP32 scores (ldz >= p); required with
 *              the planes along GMGM_AXIS_ROWS (they are written from it).
 *   zt_hi, zt_lo  device, optional (both or neither): the BF16 split of
 *              Z^T, p x ld_t (ld_t >= n, a multiple of 64; columns n..ld_t-1
 *              zero), the layout gmgm_gram and gmgm_lift read.
 *   ranks_out  device, optional, n x p int32 ranks (ldr >= p).
 * Work: GMGM_AXIS_COLS reads the counts three times (per-column maxima, read
 * back to size one histogram per column; histograms; scores) and
 * synchronises the stream once; GMGM_AXIS_ROWS reads them once (one warp
 * per row, a shared-memory histogram of the values below 1024; a larger
 * value is ranked by counting the larger entries of its row).
 * Errors: GMGM_E_ARG (shapes, strides, no output, missing z_out),
 * GMGM_E_NOMEM; device bit GMGM_DEV_NOT_COUNTS. */
int gmgm_skeptic(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, int axis,
                 float* z_out, int64_t ldz, uint16_t* zt_hi, uint16_t* zt_lo, int64_t ld_t,
                 int32_t* ranks_out, int64_t ldr);

/* The preprocessing of a sparse count matrix without its dense form (the
 * appendix "Preserving input sparsity": a transformed matrix with the
 * input's sparsity plus a rank-one term).  log1p keeps zeros at zero and the
 * centring subtracts the rank-one 1 mu^T, so X = log1p(C) - 1 mu^T: the
 * column means mu come from the non-zeros, and the BF16 hi/lo planes of X^T
 * are written tile by tile (each tile starts at -mu, the rank-one term, and
 * the rows' non-zeros are scattered over it).  The dense counts and the
 * dense FP32 X are never formed; gmgm_gram (BF16 / BF16X3) and gmgm_lift
 * read the planes.
 *   indptr   device, n + 1 int64 row offsets; indices device, int32 column
 *            indices, strictly ascending within a row; data device, FP32
 *            counts (finite, >= 0).  An entry breaking these is left out
 *            and sets GMGM_DEV_NOT_COUNTS.
 *   xt_hi, xt_lo  device, p x ld_t BF16 (ld_t >= n, a multiple of 64;
 *            cells n..ld_t-1 written as zero).
 *   colmean_out  device, optional, p FP64 column means of log1p(C).
 * 1 <= p <= 16384.  Errors: GMGM_E_ARG. */
int gmgm_preprocess_csr(gmgm_handle* h, int64_t n, int64_t p, const int64_t* indptr, const int32_t* indices,
                        const float* data, uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t, double* colmean_out);

/* The preprocessing of a matrix whose rows (cells) are split over several
 * calls or processes (the cell-sharded fit: S_genes = X^T X is a sum over
 * row blocks, Section "Algorithm"), in two steps with an exchange between:
 *   gmgm_colsum_log1p   FP64 column sums of log1p(counts) over this row
 *                       block (n x p, device), written to (accumulate = 0)
 *                       or added to (accumulate = 1) colsum (device, p);
 *   gmgm_centre         X = log1p(counts) - colsum / n_total for this row
 *                       block, with the optional BF16 split of X^T exactly
 *                       as gmgm_preprocess (ld_t >= n, a multiple of 64;
 *                       columns n..ld_t-1 zero).  colsum holds the sums over
 *                       all n_total rows (summed over the blocks by the
 *                       caller).
 * gmgm_preprocess is the two steps on one block (n_total = n).
 * Errors: GMGM_E_ARG (shapes, strides, n_total < n). */
int gmgm_colsum_log1p(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, double* colsum,
                      int accumulate);
int gmgm_centre(gmgm_handle* h, int64_t n, int64_t p, const float* counts, int64_t ldc, const double* colsum,
                int64_t n_total, float* x_out, int64_t ldx, uint16_t* xt_hi, uint16_t* xt_lo, int64_t ld_t);

/* ---- step 1: Gram ------------------------------------------------------- */

/* A batch of equally shaped matrices X_b (rows x cols), b < batch. */
typedef struct {
  int64_t batch;          /* >= 1 */
  int64_t rows, cols;     /* shape of each X_b */
  int64_t ld;             /* row stride of X_b in elements (>= cols) */
  int64_t batch_stride;   /* elements from X_b to X_{b+1} */
  const float* x;         /* device FP32 data (used by GMGM_FP32) */
  const uint16_t* xt_hi;  /* device BF16 hi split of X^T: cols x ld_t
                             (used by GMGM_BF16 / GMGM_BF16X3; batch == 1) */
  const uint16_t* xt_lo;  /* device BF16 lo split (GMGM_BF16X3) */
  int64_t ld_t;           /* leading dimension of xt_* (>= rows, % 64 == 0) */
} gmgm_matrix;

#define GMGM_SIDE_COLS 0  /* S = sum_b X_b^T X_b  (cols x cols) */
#define GMGM_SIDE_ROWS 1  /* S = sum_b X_b X_b^T  (rows x rows) */

/* Axis Gram S_l = mat_l[D] mat_l[D]^T (Notation section; Section
 * "Algorithm" for the sum over modalities = Gram of the concatenation).
 * For a matrix (cells x genes) S_genes = X^T X is side GMGM_SIDE_COLS; for a
 * 3-axis tensor T (d0 x d1 x d2, row-major) the three Grams are
 *   axis 0: one matrix d0 x (d1 d2), side ROWS;
 *   axis 1: batch d0 of d1 x d2 slices, side ROWS;
 *   axis 2: one matrix (d0 d1) x d2, side COLS.
 * S is written (accumulate = 0) or added to (accumulate = 1), FP64, device,
 * leading dimension lds; both triangles are written.  Partial sums are
 * formed in `prec` arithmetic and combined in FP64.  GMGM_SIDE_ROWS supports
 * GMGM_FP32 only.  Errors: GMGM_E_ARG (shape/stride/precision). */
/* Why one matrix per call rather than a list of labelled tensors: every
 * axis Gram of a tensor is the Gram of a matricization, and each of those
 * is one strided matrix or one batch of equally strided slices (the three
 * forms above), so the tensor bookkeeping (which index is which axis, which
 * modalities share it) stays with the caller, and the sum over modalities
 * or over row blocks of cells (a sharded fit) is `accumulate`.  A tensor of
 * order four or more is reached the same way: its axis-l matricization is a
 * batch of (product of the leading extents) slices of d_l x (product of the
 * trailing extents); only the batch form's single level of batching is
 * built in, so the caller loops over the outer indices with accumulate = 1. */
int gmgm_gram(gmgm_handle* h, const gmgm_matrix* m, int side, gmgm_prec prec,
              double* S, int64_t lds, int accumulate);

/* ---- step 2: spectra ---------------------------------------------------- */

/* Eigendecomposition of a symmetric FP64 matrix S (d x d, device, leading
 * dimension lds; only the lower triangle is read) on the GPU: Householder
 * tridiagonalisation, bisection for the eigenvalues, inverse iteration with
 * re-orthogonalisation of close clusters for the vectors, and the
 * back-transformation.  The first three run in double-float arithmetic
 * (pairs of FP32 numbers, about 48 significant bits) on a copy of S scaled
 * by a power of two; eigenvalues agree with an FP64 LAPACK solve to about
 * 1e-14 of the largest, eigenvector residuals |S w - lambda w| likewise.
 * Theorem 1: the top-r eigenvectors of S_l are those of the MLE Psi_l.
 *   evals  device, r FP64, the r largest eigenvalues, descending.
 *   rv     0 <= rv <= r: eigenvectors are formed for the rv largest
 *          eigenvalues only (the back-transformation is O(d^2) per vector).
 *   evecs  device, d x rv FP64 row-major (column c is the eigenvector of
 *          evals[c]), leading dimension ldv >= rv; NULL iff rv = 0.
 * 1 <= r <= d <= 8192.  Eigenvector signs are arbitrary.  The call uses a
 * cooperative launch.  Errors: GMGM_E_ARG, GMGM_E_CUDA; device TIMEOUT bit
 * if a grid barrier gave up. */
int gmgm_spectra(gmgm_handle* h, int64_t d, const double* S, int64_t lds,
                 int32_t r, double* evals, int32_t rv, double* evecs,
                 int64_t ldv);

/* Dual lift (Section "Algorithm": eigenvectors of S_l are singular vectors
 * of mat_l[D]; Algorithm 1 takes the top-r left singular vectors): for the
 * matrix X (rows x cols) and the top-r eigenpairs (W, E) of X^T X,
 * U = X W diag(E)^-1/2 are the top-r eigenvectors of X X^T.
 *   m      one matrix (batch 1).  With its BF16 split of X^T (m->xt_hi and
 *          m->xt_lo, cols x ld_t, as gmgm_preprocess writes it) and r <= 64
 *          the product runs on the tensor cores from the two planes
 *          (3xBF16 products, the FP32 accumulation drained every 128
 *          columns of X; error about 1e-6 of max |U|); otherwise from the
 *          FP32 matrix m->x on the FP32 pipe.
 *   W      device, cols x r FP64 row-major, leading dimension ldw.
 *   E      device, r FP64, all > 0.
 *   U      device, rows x r FP32 row-major, leading dimension ldu >= r.
 * 1 <= r <= 256.  Errors: GMGM_E_ARG (batch != 1, shapes, only one of the
 * planes given, ld_t < rows or not a multiple of 64, no FP32 matrix where
 * the tensor-core form does not apply). */
int gmgm_lift(gmgm_handle* h, const gmgm_matrix* m, int32_t r,
              const double* W, int64_t ldw, const double* E,
              float* U, int64_t ldu);

/* ---- step 3: eigenvalue solve ------------------------------------------- */

#define GMGM_MAX_AXES 4
#define GMGM_MAX_MODALITIES 4

/* The eigenvalue problem: per-axis spectra E_l (descending, > 0) and the
 * modalities, each a list of axis indices in tensor order.  Objective
 * (twice the NLL, constants dropped):
 *   f(Lam) = sum_l E_l . Lam_l - sum_gamma sum_{grid of gamma} log s,
 *   s(i_1, i_2, ...) = sum_{l in gamma} lam_{l, i_l},
 * over the box lam_l,i >= eps_l. */
typedef struct {
  int32_t n_axes;                     /* 1..GMGM_MAX_AXES */
  int32_t r[GMGM_MAX_AXES];           /* ranks r_l >= 1 */
  const double* E[GMGM_MAX_AXES];     /* device, r_l FP64 each */
  double eps[GMGM_MAX_AXES];          /* box; <= 0 selects the default:
                                         1e-10 * max over modalities of
                                         sum_l max_i 1/E_l,i (same for all l) */
  int32_t n_modalities;               /* 1..GMGM_MAX_MODALITIES */
  int32_t mod_n_axes[GMGM_MAX_MODALITIES];
  int32_t mod_axes[GMGM_MAX_MODALITIES][GMGM_MAX_AXES];
} gmgm_problem;

typedef struct {
  double tol;           /* relative projected-KKT target, max_i |P(g)_i|/E_i
                           (<= 0: 1e-9) */
  int32_t max_newton;   /* Newton iteration cap (<= 0: 200) */
  int32_t max_cg;       /* CG iterations per Newton step (<= 0: 200) */
  int32_t fp32_phase;   /* 1: iterate in FP32 (Kahan/FP64 partials) until
                           rel. KKT <= 1e-5, then FP64; 0: FP64 throughout */
  int32_t gauge;        /* 1: apply the gauge convention (flat shift, single
                           modality with equal traces): every axis but the
                           first gets min = eps.  0: leave as solved. */
  double trace_rtol;    /* with gauge = 1 and one modality: traces that agree
                           within this relative tolerance are made exactly
                           equal before the solve (each axis' spectrum
                           scaled by the mean trace over its own, a change
                           of at most trace_rtol relative), so the flat
                           shift is exact.  Full-rank axes of one tensor
                           have equal traces in exact arithmetic; spectra
                           from FP32 Grams differ by ~1e-7.  0: 1e-6;
                           < 0: off (only traces equal to 1e-9 count). */
} gmgm_solve_opts;

typedef struct {
  int32_t status;       /* GMGM_OK, GMGM_E_NOT_CONVERGED, ... */
  int32_t newton_iters;
  int32_t cg_iters;     /* total Hessian-vector products */
  int32_t grid_passes;  /* total passes over the Kronecker-sum grids */
  int32_t n_active;     /* coordinates at their bound */
  int32_t fp64_iters;   /* Newton iterations run in FP64 */
  double rel_kkt;       /* final FP64 relative projected-KKT residual */
  double objective;     /* final f(Lam), FP64 */
} gmgm_solve_stats;

/* Solve for the eigenvalues Lam_l of the MLE (Proposition on the gradient:
 * g_l,i = E_l,i - sum_{gamma containing l} sum_{other indices} 1/s; the
 * existence lemma's box Lam_l >= eps_l).  One persistent single-CTA kernel
 * runs a projected Newton method (Bertsekas' active set; conjugate gradients
 * on the free set with Hessian-vector products computed as grid reductions;
 * Armijo search along the projection arc) and the final KKT check in FP64.
 *   init        host array of n_axes device pointers (r_l FP64 each) for the
 *               starting point, or NULL for Algorithm 1's Lam^0 = 1/E.
 *   lambda_out  host array of n_axes device pointers (r_l FP64 each).
 *   stats       host, optional; if non-NULL the call synchronises and fills
 *               it (and returns its status).
 * Sizes: sum_l r_l <= 16384; every modality grid <= 2^31 points.
 * Every E_l,i must be positive and finite (f has no minimiser when some
 * E_l,i <= 0, i.e. X lacks full rank on that axis): otherwise lambda_out is
 * NaN, no iteration runs and the status is GMGM_E_INFEASIBLE (a zero or
 * negative value) or GMGM_E_NONFINITE (a NaN or Inf).
 * Errors: GMGM_E_ARG; device bits NOT_CONVERGED / INFEASIBLE / NONFINITE. */
int gmgm_eigsolve(gmgm_handle* h, const gmgm_problem* p,
                  const double* const* init, const gmgm_solve_opts* opts,
                  double* const* lambda_out, gmgm_solve_stats* stats);

/* The same eigenvalue solve for callers that cannot allocate device memory
 * at call time (a host whose own allocator has reserved the device, a
 * latency-critical loop that cannot afford cudaMalloc's implicit device
 * synchronisation, a plugin with a fixed memory budget).  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *   - No handle, no allocation: the solver's working vectors, status word
 *     and statistics live in one fixed device array inside the library
 *     (about 0.5 MB), which every device that loads the library holds until
 *     the process exits.  The call makes no cudaMalloc/cudaFree.
 *   - Runs on the calling thread's current device and on `cuda_stream`
 *     (a cudaStream_t, NULL = legacy default stream).  The first call on a
 *     device looks up the array's device address (a one-time, non-allocating
 *     runtime query); make that first call before any stream capture.
 *   - Limit: sum_l r_l <= 4096.  Larger problems, and every argument error
 *     of gmgm_eigsolve, return GMGM_E_ARG before anything is enqueued.
 *   - All calls share the one array and it keeps the last call's contents:
 *     calls that may overlap on the GPU (different streams, or different
 *     host threads) race and must be serialised by the caller.
 *   - Arguments as gmgm_eigsolve.  `stats` (host, optional): if non-NULL the
 *     call synchronises the stream, fills it and returns its status.
 *     Otherwise device-detected problems are only visible in the returned
 *     lambda values (the status word is private to this entry point).
 *   - The array's device address is looked up on every call (a lookup, not
 *     an allocation), so the entry point stays valid after a device reset
 *     reloads the module. */
int gmgm_eigsolve_static(const gmgm_problem* p, const double* const* init,
                         const gmgm_solve_opts* opts, double* const* lambda_out,
                         gmgm_solve_stats* stats, void* cuda_stream);

/* ---- learned warm start of the eigenvalue solve ------------------------- */
/* Not part of the paper: Algorithm 1 starts the solve at Lam^0 = 1/E.  A
 * small network predicts the start instead; the solve then runs to the same
 * tolerance, so the prediction changes the iteration count, never the result
 * (and a non-finite prediction falls back to 1/E).  Two-axis problems only.
 *
 * Features (132 FP32): for each axis, the interpolated log E at 64 evenly
 * spaced rank positions minus log(mean E); then log(r_0)/8, log(r_1)/8,
 * log tr E_0 - log tr E_1, log E_0[0] - log E_1[0].
 * Targets (128 FP32): for each axis, the interpolated log(lam_i E_i) at the
 * same 64 positions.
 * Network: 132 -> 256 -> 256 -> 128, ReLU hidden layers, linear output, MSE.
 * Parameters: one FP32 vector of GMGM_MLP_PARAMS values, in order
 * W1 [256][132], b1 [256], W2 [256][256], b2 [256], W3 [128][256], b3 [128]. */
#define GMGM_MLP_IN 132
#define GMGM_MLP_HIDDEN 256
#define GMGM_MLP_OUT 128
#define GMGM_MLP_PARAMS (256 * 132 + 256 + 256 * 256 + 256 + 128 * 256 + 128)

typedef struct {
  int32_t steps;   /* Adam steps */
  int32_t batch;   /* mini-batch size (capped at n) */
  float lr, beta1, beta2, eps;
  uint64_t seed;   /* mini-batch order (seeded shuffles on the host) */
} gmgm_train_opts;

/* Features of a two-axis problem (E_0: r_0, E_1: r_1, device FP64,
 * descending, > 0) into `feats` (device, 132 FP32). */
int gmgm_warmstart_features(gmgm_handle* h, const double* E0, int32_t r0,
                            const double* E1, int32_t r1, float* feats);

/* Targets of a solved problem (lam_0, lam_1 device FP64) into `targets`
 * (device, 128 FP32). */
int gmgm_warmstart_targets(gmgm_handle* h, const double* E0, int32_t r0,
                           const double* E1, int32_t r1, const double* lam0,
                           const double* lam1, float* targets);

/* Network output for n feature rows (device n x 132) into `out` (device
 * n x 128). */
int gmgm_mlp_forward(gmgm_handle* h, const float* params, const float* feats,
                     int32_t n, float* out);

/* MSE loss of n rows and its gradient w.r.t. the parameters (device,
 * GMGM_MLP_PARAMS floats; may be NULL).  `loss` (host, optional): if given the
 * call synchronises and stores the loss. */
int gmgm_mlp_loss_grad(gmgm_handle* h, const float* params, const float* feats,
                       const float* targets, int32_t n, float* grad, float* loss);

/* Train in place with Adam: `params` (device, in/out), `adam_state` (device,
 * 2 * GMGM_MLP_PARAMS floats, zero for a fresh start), n rows of features and
 * targets (device).  `final_loss` (host, optional): loss of the last
 * mini-batch (synchronises). */
int gmgm_warmstart_train(gmgm_handle* h, float* params, float* adam_state,
                         const float* feats, const float* targets, int32_t n,
                         const gmgm_train_opts* opts, float* final_loss);

/* Predicted start lam_0 (r_0), lam_1 (r_1) (device FP64) for the solve's
 * `init`: lam_i = exp(interpolated prediction) / E_i, at least `eps`. */
int gmgm_warmstart_infer(gmgm_handle* h, const float* params, const double* E0,
                         int32_t r0, const double* E1, int32_t r1, double eps,
                         double* lam0_out, double* lam1_out);

/* ---- step 4: recomposition + per-row top-k ------------------------------ */

typedef struct {
  int64_t rows_uncertified;  /* rows the first screen did not certify */
  int64_t rows_exact;        /* rows that ended in the exact FP64 scan */
  int64_t candidates;        /* candidate slots per row used by the screen */
  double screen_ms;          /* device time of the first screen */
  double rescore_ms;         /* device time of rescoring (+ repair) */
  double screen_err_ratio;   /* max over candidates of |screened - exact| /
                                the screen's error bound (<= 1 expected) */
  int64_t screen_tiles;      /* GMGM_BF16: 128 x 256 tiles the first screen
                                multiplied (sampling pass included) */
  int64_t screen_tiles_dense; /* GMGM_BF16: tiles of one dense sweep
                                 (row blocks x column tiles) */
} gmgm_topk_stats;

/* Per-row top-k of Psi = V diag(psi) V^T without forming Psi (Algorithm 1:
 * thresh_{n_l}[V_l Lam_l V_l^T], "threshold simultaneously with
 * recomposition").  Readings: an edge's strength is |Psi_ij|; the diagonal
 * is excluded; each row keeps its own k edges; equal magnitudes are ordered
 * by the lower column index.
 *   V       device, d x r row-major, FP32 (v_fp64 = 0) or FP64 (v_fp64 = 1),
 *           leading dimension ldv >= r.
 *   psi     device, r FP64 eigenvalues.
 *   k       1 <= k <= 32 and k < d.
 *   prec    screen arithmetic: GMGM_FP32 (SIMT) or GMGM_BF16 (tcgen05 tensor
 *           cores, r <= 64); any other value is GMGM_E_ARG.
 *   flags   0, or GMGM_TOPK_ORTHO: V is square (r == d) with orthonormal
 *           columns (the full eigenvector matrix of an axis at full rank).
 *           Then Psi = c I + V diag(psi - c) V^T with c = min psi, and the
 *           off-diagonal entries depend only on the columns with psi > c
 *           (the identifiability appendix's diagonal shift, exact when
 *           V V^T = I): the network is computed from those columns alone,
 *           and when there are none every off-diagonal entry is 0 (each row
 *           takes the k lowest columns j != i by the tie rule, values 0).
 *           The caller guarantees the orthonormality; it is not checked.
 *           With r - (columns dropped) > 64 a BF16 request screens in FP32.
 *   idx_out device, d x k int32: column indices, by |Psi_ij| descending.
 *   val_out device, d x k FP32: the signed Psi_ij from V (as given) and
 *           psi, rounded to FP32 (computed in double-float for an FP32 V,
 *           in FP64 for an FP64 V).
 *   stats   host, optional; if non-NULL the call synchronises and fills it.
 * Exactness: every row's screen is certified with a rigorous error bound of
 * the screen arithmetic (the k-th exact value must beat the best excluded
 * screened value plus the bound, rounded up); rows that fail are rescreened
 * with split products (after a BF16 screen) and, failing again, recomputed
 * in FP64, so idx_out is
 * the exact top-k of the given V and psi.  Candidates are ranked by values
 * exact to about 2^-46 of sum_q |V_iq psi_q V_jq|: entries closer than that
 * may be ordered either way (equal values by the lower column).
 * Errors: GMGM_E_ARG. */
#define GMGM_TOPK_ORTHO 1u

/* One V serves both the screen and the rescoring (no separate FP64 copy for
 * rescoring): the screen rounds V to its own arithmetic internally, and the
 * rescoring reads V as given (an FP64 V is rescored in FP64, an FP32 V in
 * double-float from its exact FP32 values), so the lists are exact for the
 * V the caller passed and a second copy would only duplicate memory. */
int gmgm_topk_network(gmgm_handle* h, int64_t d, int32_t r,
                      const void* V, int v_fp64, int64_t ldv,
                      const double* psi, int32_t k, gmgm_prec prec,
                      uint32_t flags, int32_t* idx_out, float* val_out,
                      gmgm_topk_stats* stats);

/* The rows [row0, row0 + m) of the network of gmgm_topk_network (the same
 * V diag(psi) V^T, every column screened, the same readings, precision and
 * certification): what one process of a row-sharded fit computes for the
 * rows it owns, with V the full (all-gathered) vectors.
 *   idx_out, val_out  device, m x k: row row0 + t of Psi in row t.
 * 0 <= row0, 1 <= m, row0 + m <= d; other arguments as gmgm_topk_network
 * (flags 0).  Errors: GMGM_E_ARG. */
int gmgm_topk_network_rows(gmgm_handle* h, int64_t d, int32_t r, const void* V, int v_fp64, int64_t ldv,
                           const double* psi, int32_t k, gmgm_prec prec, int64_t row0, int64_t m,
                           int32_t* idx_out, float* val_out, gmgm_topk_stats* stats);

/* The network of a full-rank axis straight from its Gram: Psi = W diag(psi)
 * W^T with W the d x d orthonormal eigenvectors of S (psi[j] pairs with the
 * j-th largest eigenvalue of S; the axis' full spectrum).  As for
 * GMGM_TOPK_ORTHO, Psi = c I + W diag(psi - c) W^T with c = min psi, and
 * the off-diagonal entries depend only on the eigenvectors whose psi
 * exceeds c: only those are formed (tridiagonalisation of S, bisection and
 * inverse iteration for those eigenvalues, back-transformation), then the
 * network follows as in gmgm_topk_network; with none, every off-diagonal
 * entry is 0 and each row takes the k lowest columns j != i (values 0).
 * Eigenvalues of S closer than 1e-7 ||S|| whose psi fall on both sides of
 * c are a boundary case: their vectors are orthogonalised within the formed
 * set only.
 *   S     device, d x d FP64 (lower triangle read), leading dimension lds.
 *   psi   device, d FP64.
 *   k, prec, idx_out, val_out, stats: as gmgm_topk_network.
 * 2 <= d <= 8192.  Errors: GMGM_E_ARG, GMGM_E_CUDA. */
int gmgm_topk_network_gram(gmgm_handle* h, int64_t d, const double* S,
                           int64_t lds, const double* psi, int32_t k,
                           gmgm_prec prec, int32_t* idx_out, float* val_out,
                           gmgm_topk_stats* stats);

/* Global top-n edges of an axis (Algorithm 1's last loop with the global
 * threshold thresh_{n_l}; the appendix "Computational complexity" keeps the
 * n_l strongest edges with a heap of size n_l), derived from its per-row
 * top-k lists (as gmgm_topk_network writes them): the union of the lists as
 * unordered pairs (i < j, the value listed by the lower row i when both
 * rows list the pair), its n strongest by |value| descending, ties by (i, j)
 * ascending.  The result is the global top-n of the network exactly when
 * every row's k-th magnitude lies strictly below the n-th selected magnitude
 * (no row can then hold an edge that strong outside its own list), or every
 * list holds all d - 1 columns; *certified reports this.  A row whose list
 * reaches that magnitude may hide more: rerun its rows with a larger k.
 *   idx, val   device, d x k int32 / FP32 per-row lists (a list entry j < 0
 *              or j == i is ignored).
 *   n          1 <= n <= d k, n <= 2^30.
 *   i_out, j_out, v_out  device, n int32 / int32 / FP32: the edges, by
 *              |value| descending then (i, j).
 *   count      host: the edges written (< n when the union holds fewer
 *              distinct pairs; then *certified = 0).
 *   certified  host: 1 if the edges are the network's global top-n.
 * Synchronises the stream.  Errors: GMGM_E_ARG, GMGM_E_NOMEM,
 * GMGM_E_CAND_OVERFLOW (more pairs tie at the n-th magnitude than the
 * selection holds: at least 2n + 2 and 2^22). */
int gmgm_topn_edges(gmgm_handle* h, int64_t d, int32_t k, const int32_t* idx, const float* val, int64_t n,
                    int32_t* i_out, int32_t* j_out, float* v_out, int64_t* count, int* certified);

#ifdef __cplusplus
}
#endif

#endif /* GMGM_H_ */
