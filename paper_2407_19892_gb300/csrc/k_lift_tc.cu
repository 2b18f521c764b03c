// Dual lift on the tensor cores, sm_103a: U = X W_r diag(E_r)^-1/2 (rows x
// r, FP32), the top-r left singular vectors of X from the right ones
// (Section "Algorithm": the eigenvectors of the small Gram are the right
// singular vectors of X; Algorithm 1 takes the top-r of them).
//
// The operands are the BF16 hi/lo planes of X^T that the preprocessing
// writes for the Gram (gene-major, cells contiguous), read here as an
// MN-major A operand: D[128 cells x 64] = A[128 cells x K genes] B^T with
// B = (W_r diag(E_r)^-1/2)^T (64 x K, K-major, zero beyond r and beyond the
// genes) split into three BF16 planes b0 + b1 + b2 (exact to ~2^-27), and
// five products x_hi (b0 + b1 + b2) + x_lo (b0 + b1): what is left is the
// planes' own representation of X (hi + lo, 16 significant bits, ~2^-18
// relative) and the dropped x_lo b2 (~2^-27).  The tensor core's FP32
// accumulation runs over kLDrain x 64 genes at a time; each partial is
// drained from TMEM into FP32 registers, so the accumulation error does
// not grow with the gene count.
//
// Work item: a block of 256 cells (two M = 128 tiles sharing every B
// chunk).  Persistent, one CTA per SM, warp-specialised:
//   warp 0      TMA producer: per 64-gene chunk four 64 x 64 boxes of each
//               plane (128-byte swizzle, one 128-byte row per gene) and the
//               chunk of B, into a 2-stage ring;
//   warp 1      MMA issuer: per chunk and tile 4 K steps x 5 products,
//               M = 128, N = 64, accumulators in TMEM (2 buffers x 2 tiles
//               x 64 columns);
//   warps 2-9   epilogue: one thread per cell row, tcgen05.ld of the drained
//               partial (64 columns) added to registers; the r outputs are
//               stored once per block.
// HBM-bound: the two planes are read once (4 bytes per cell and gene).
// Every wait is bounded (GMGM_DEV_TIMEOUT on expiry, TMEM freed on exit).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace gmgm {
namespace {

constexpr int kLM = 128;                      // MMA M: cells per tile
constexpr int kLTiles = 2;                    // tiles per work item (share B)
constexpr int kLBlock = kLM * kLTiles;        // cells per work item
constexpr int kLN = 64;                       // MMA N: r padded
constexpr int kLK = 64;                       // genes per chunk (one 128-byte row)
constexpr int kLStages = 2;
constexpr int kLDrain = 2;                    // chunks per accumulator drain (128 genes)
constexpr int kLEpiWarps = 8;
constexpr int kLThreads = 64 + 32 * kLEpiWarps;
constexpr int kABox = 64 * kLK * 2;           // one box: 64 cells x 64 genes (8 KB)
constexpr int kAPlane = kLBlock * kLK * 2;    // 32 KB: four boxes
constexpr int kBPlane = kLN * kLK * 2;        // 8 KB
constexpr int kBPlanes = 3;                   // B = b0 + b1 + b2
constexpr int kLStage = 2 * kAPlane + kBPlanes * kBPlane;
constexpr int kLTmemCols = 2 * kLTiles * kLN;  // 256
constexpr long long kLSpin = 1ll << 23;

struct __align__(8) LBars {
  uint64_t full[kLStages];
  uint64_t empty[kLStages];
  uint64_t accf[2];
  uint64_t acce[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

constexpr size_t kLSmem = 1024 + size_t(kLStages) * kLStage + sizeof(LBars);

__device__ __forceinline__ bool l_aborted(LBars* bs) { return *reinterpret_cast<volatile int*>(&bs->abort) != 0; }
__device__ __forceinline__ void l_abort(LBars* bs, int* status) {
  atomicExch(&bs->abort, 1);
  set_status(status, GMGM_DEV_TIMEOUT);
}

// lbo / sbo: byte strides of the MN-major A operand between its 64-cell
// groups (one TMA box apart) and between its 8-gene groups (one swizzle
// atom apart).
__global__ void __launch_bounds__(kLThreads, 1)
    lift_tc_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                   const __grid_constant__ CUtensorMap tB0, const __grid_constant__ CUtensorMap tB1,
                   const __grid_constant__ CUtensorMap tB2, int64_t n,
                   int nkc, int r, float* __restrict__ U, int64_t ldu, uint32_t lbo, uint32_t sbo,
                   int* __restrict__ status) {
  extern __shared__ uint8_t lsm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(lsm_raw) + 1023) & ~uintptr_t(1023));
  LBars* bs = reinterpret_cast<LBars*>(smem + kLStages * kLStage);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kLStages; ++s) tc::mbar_init(&bs->full[s], 1), tc::mbar_init(&bs->empty[s], 1);
    for (int b = 0; b < 2; ++b) tc::mbar_init(&bs->accf[b], 1), tc::mbar_init(&bs->acce[b], kLEpiWarps);
    tc::mbar_init(&bs->done, 1);
    bs->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tAh);
    tc::prefetch_tmap(&tAl);
    tc::prefetch_tmap(&tB0);
    tc::prefetch_tmap(&tB1);
    tc::prefetch_tmap(&tB2);
  }
  if (warp == 1) tc::tmem_alloc(&bs->tmem_base, kLTmemCols);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = bs->tmem_base;
  const int64_t nblk = (n + kLBlock - 1) / kLBlock;
  const int ndrain = (nkc + kLDrain - 1) / kLDrain;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      long long issued = 0;
      for (int64_t blk = blockIdx.x; blk < nblk && !l_aborted(bs); blk += gridDim.x) {
        const int x0 = int(blk * kLBlock);
        for (int kc = 0; kc < nkc; ++kc, ++issued) {
          const int s = int(issued % kLStages);
          const uint32_t k = uint32_t(issued / kLStages);
          if (!tc::mbar_wait(&bs->empty[s], (k & 1) ^ 1, kLSpin)) {
            l_abort(bs, status);
            break;
          }
          uint8_t* st = smem + s * kLStage;
          tc::mbar_arrive_expect_tx(&bs->full[s], kLStage);
#pragma unroll
          for (int j = 0; j < kLBlock / 64; ++j) {
            tc::tma_load_2d(st + j * kABox, &tAh, &bs->full[s], x0 + j * 64, kc * kLK);
            tc::tma_load_2d(st + kAPlane + j * kABox, &tAl, &bs->full[s], x0 + j * 64, kc * kLK);
          }
          tc::tma_load_2d(st + 2 * kAPlane, &tB0, &bs->full[s], kc * kLK, 0);
          tc::tma_load_2d(st + 2 * kAPlane + kBPlane, &tB1, &bs->full[s], kc * kLK, 0);
          tc::tma_load_2d(st + 2 * kAPlane + 2 * kBPlane, &tB2, &bs->full[s], kc * kLK, 0);
        }
      }
      if (l_aborted(bs))
        for (long long x = issued > kLStages ? issued - kLStages : 0; x < issued; ++x)
          tc::mbar_wait(&bs->full[x % kLStages], uint32_t(x / kLStages) & 1, kLSpin);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = tc::idesc_bf16_f32_amn(kLM, kLN);
      long long used = 0, accu = 0;
      for (int64_t blk = blockIdx.x; blk < nblk && !l_aborted(bs); blk += gridDim.x) {
        int b = 0;
        for (int kc = 0; kc < nkc; ++kc, ++used) {
          const int s = int(used % kLStages);
          if (kc % kLDrain == 0) {
            b = int(accu & 1);
            if (!tc::mbar_wait(&bs->acce[b], (uint32_t(accu >> 1) & 1) ^ 1, kLSpin)) {
              l_abort(bs, status);
              break;
            }
          }
          if (!tc::mbar_wait(&bs->full[s], uint32_t(used / kLStages) & 1, kLSpin)) {
            l_abort(bs, status);
            break;
          }
          tc::fence_after_sync();
          const uint32_t base = tc::smem_u32(smem + s * kLStage);
          const uint32_t b0 = base + 2 * kAPlane, b1 = b0 + kBPlane, b2 = b1 + kBPlane;
#pragma unroll
          for (int t = 0; t < kLTiles; ++t) {
            const uint32_t d = tmem + uint32_t(b * kLTiles * kLN + t * kLN);
            const uint32_t ah = base + t * 2 * kABox, al = ah + kAPlane;
#pragma unroll
            for (int ks = 0; ks < kLK / 16; ++ks) {
              const uint32_t acc = (kc % kLDrain == 0 && ks == 0) ? 0u : 1u;
              const uint64_t xh = tc::sdesc_mn128(ah + ks * 2048, lbo, sbo), xl = tc::sdesc_mn128(al + ks * 2048, lbo, sbo);
              // smallest products first
              tc::mma_bf16(d, xl, tc::sdesc_k128(b1 + ks * 32), idesc, acc);
              tc::mma_bf16(d, xh, tc::sdesc_k128(b2 + ks * 32), idesc, 1u);
              tc::mma_bf16(d, xh, tc::sdesc_k128(b1 + ks * 32), idesc, 1u);
              tc::mma_bf16(d, xl, tc::sdesc_k128(b0 + ks * 32), idesc, 1u);
              tc::mma_bf16(d, xh, tc::sdesc_k128(b0 + ks * 32), idesc, 1u);
            }
          }
          tc::mma_commit(&bs->empty[s]);
          if (kc % kLDrain == kLDrain - 1 || kc == nkc - 1) {
            tc::mma_commit(&bs->accf[b]);
            ++accu;
          }
        }
      }
      tc::mma_commit(&bs->done);
      tc::mbar_wait(&bs->done, 0, kLSpin);
    }
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;
    const int t = ew >> 2;      // tile of the work item
    const int q = warp & 3;     // TMEM lane quarter this warp may access
    const int row_local = q * 32 + lane;
    long long accu = 0;
    bool ok = true;
    for (int64_t blk = blockIdx.x; blk < nblk && ok; blk += gridDim.x) {
      float acc[kLN];
#pragma unroll
      for (int c = 0; c < kLN; ++c) acc[c] = 0.f;
      for (int dr = 0; dr < ndrain; ++dr, ++accu) {
        const int b = int(accu & 1);
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&bs->accf[b], uint32_t(accu >> 1) & 1, kLSpin))) {
          if (lane == 0) l_abort(bs, status);
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(b * kLTiles * kLN + t * kLN);
        uint32_t v0[32], v1[32];
        __syncwarp();
        tc::tmem_ld_32x32b_x32(taddr, v0);
        tc::tmem_ld_32x32b_x32(taddr + 32, v1);
        tc::tmem_ld_wait();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bs->acce[b]);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          acc[c] += __uint_as_float(v0[c]);
          acc[32 + c] += __uint_as_float(v1[c]);
        }
      }
      if (!ok || __any_sync(0xffffffffu, l_aborted(bs))) break;
      const int64_t row = blk * kLBlock + t * kLM + row_local;
      if (row < n) {
        float* dst = U + row * ldu;
#pragma unroll
        for (int c = 0; c < kLN; ++c)
          if (c < r) dst[c] = acc[c];
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kLTmemCols);
  }
}

// B = (W_r diag(E_r)^-1/2)^T in three BF16 planes b0 + b1 + b2 (each the
// rounding of what the previous ones leave, in FP64): kLN rows x kpad
// genes, zero beyond r rows and beyond p genes.
__global__ void lift_b_kernel(const double* __restrict__ W, int64_t ldw, const double* __restrict__ E, int64_t p,
                              int r, int64_t kpad, __nv_bfloat16* __restrict__ B0, __nv_bfloat16* __restrict__ B1,
                              __nv_bfloat16* __restrict__ B2) {
  const int64_t total = int64_t(kLN) * kpad;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = e / kpad, g = e - c * kpad;
    double x = (c < r && g < p) ? W[g * ldw + c] / sqrt(E[c]) : 0.0;
    const __nv_bfloat16 v0 = __float2bfloat16_rn(float(x));
    x -= double(__bfloat162float(v0));
    const __nv_bfloat16 v1 = __float2bfloat16_rn(float(x));
    x -= double(__bfloat162float(v1));
    B0[e] = v0;
    B1[e] = v1;
    B2[e] = __float2bfloat16_rn(float(x));
  }
}

typedef CUresult (*LEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

LEncodeFn l_encode() {
  static LEncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<LEncodeFn>(p);
  }
  return fn;
}

// rows x cols bf16 row-major (leading dimension ld elements), 64 x 64 boxes
bool lmap(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld) {
  LEncodeFn fn = l_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(ld) * 2};
  cuuint32_t box[2] = {64u, 64u};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool lift_tc_eligible(const gmgm_matrix* m, int32_t r) {
  return m->xt_hi && m->xt_lo && r <= kLN && m->ld_t >= m->rows && m->ld_t % 64 == 0 &&
         m->rows <= (int64_t(1) << 30) && m->cols <= (int64_t(1) << 30);
}

size_t lift_tc_scratch_bytes(const gmgm_matrix* m) {
  const int64_t kpad = (m->cols + kLK - 1) / kLK * kLK;
  return kBPlanes * Carve::round(size_t(kLN) * kpad * 2) + 1024;
}

cudaError_t launch_lift_tc(gmgm_handle* h, const gmgm_matrix* m, int32_t r, const double* W, int64_t ldw,
                           const double* E, float* U, int64_t ldu, void* scratch) {
  const int64_t p = m->cols, n = m->rows;
  const int64_t kpad = (p + kLK - 1) / kLK * kLK;
  Carve c(scratch);
  __nv_bfloat16* B0 = c.take<__nv_bfloat16>(size_t(kLN) * kpad);
  __nv_bfloat16* B1 = c.take<__nv_bfloat16>(size_t(kLN) * kpad);
  __nv_bfloat16* B2 = c.take<__nv_bfloat16>(size_t(kLN) * kpad);
  {
    const int64_t total = int64_t(kLN) * kpad;
    const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, int64_t(h->num_sms) * 8));
    lift_b_kernel<<<blocks, 256, 0, h->stream>>>(W, ldw, E, p, r, kpad, B0, B1, B2);
  }
  CUtensorMap ah, al, b0, b1, b2;
  if (!lmap(&ah, m->xt_hi, p, m->ld_t, m->ld_t) || !lmap(&al, m->xt_lo, p, m->ld_t, m->ld_t) ||
      !lmap(&b0, B0, kLN, kpad, kpad) || !lmap(&b1, B1, kLN, kpad, kpad) || !lmap(&b2, B2, kLN, kpad, kpad))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(lift_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kLSmem));
  if (e != cudaSuccess) return e;
  const int64_t nblk = (n + kLBlock - 1) / kLBlock;
  const int grid = int(std::min<int64_t>(nblk, h->num_sms));
  lift_tc_kernel<<<grid, kLThreads, kLSmem, h->stream>>>(ah, al, b0, b1, b2, n, int(kpad / kLK), r, U, ldu,
                                                         uint32_t(kABox), 1024u, h->d_status);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace gmgm
