// Tensor-core Gram S = X^T X (cells x genes X, the small gene axis), sm_103a.
//
// Operands are the BF16 planes of X^T written by the preprocessing kernel
// (gene-major, K = cells contiguous): x = hi + lo.  3xBF16 forms
// hi.hi^T + hi.lo^T + lo.hi^T (the dropped lo.lo^T is below 2^-16 of each
// product); plain BF16 forms hi.hi^T only.
//
// Work item = (output tile 128 genes x 256 genes of the upper triangle,
// K split: every nsplit-th drain block of the cells, so all CTAs sweep the
// cells together and share each slice of the planes through L2).  The tensor
// core's FP32 accumulation is kept short: the accumulator is drained every
// kSub K blocks (1024 cells) into a running tile owned by the CTA, kept as
// double-float (FP32 hi + lo, exact TwoSum; ~2^-48 relative) so the drains
// run on the FP32 pipe.  The accumulation's rounding error grows with the
// length of a block (measured at 1M cells x 2000 genes against an FP64 Gram
// of the same X: 3.7e-5 of max|S| with 2048-cell blocks, 1.85e-5 with 1024,
// 9.7e-6 with 512; the FP32 SIMT Gram reaches 3.2e-5).  Persistent CTAs,
// warp-specialised:
//   warp 0      TMA producer: per K block the A (128 rows) and B (256 rows)
//               slices of hi (and lo) into a 2-stage ring;
//   warp 1      MMA issuer: tcgen05.mma M=128 N=256 K=16, FP32 accumulator
//               in TMEM (double-buffered, 2 x 256 columns);
//   warps 2-5   epilogue: tcgen05.ld each drained accumulator and add it to
//               the item's running tile; a second kernel sums the K splits
//               in FP64 and writes both triangles of S.
// Every wait is bounded (GMGM_DEV_TIMEOUT on expiry, TMEM freed on exit).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace gmgm {
namespace {

constexpr int kGM = 128;                     // tile rows (genes a)
constexpr int kGN = 256;                     // tile cols (genes b)
constexpr int kSub = 16;                     // 64-cell K blocks per accumulator drain
constexpr int kGStages = 2;
constexpr int kGThreads = 64 + 128;
constexpr int kABytes = kGM * 128;           // 16 KB per plane
constexpr int kBBytes = kGN * 128;           // 32 KB per plane
constexpr int kStageBytes = 2 * (kABytes + kBBytes);
constexpr long long kGSpin = 1ll << 23;
constexpr int kPaceWindow = 2;               // drains a CTA may run ahead of the slowest

struct __align__(8) GBars {
  uint64_t full[kGStages];
  uint64_t empty[kGStages];
  uint64_t accf[2];
  uint64_t acce[2];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

constexpr size_t kGSmem = 1024 + size_t(kGStages) * kStageBytes + sizeof(GBars);

__device__ __forceinline__ bool g_aborted(GBars* bs) { return *reinterpret_cast<volatile int*>(&bs->abort) != 0; }
__device__ __forceinline__ void g_abort(GBars* bs, int* status) {
  atomicExch(&bs->abort, 1);
  set_status(status, GMGM_DEV_TIMEOUT);
}

// (hi, lo) += x in double-float: hi + lo carries the running sum to ~2^-48
// relative (TwoSum: the rounding error of hi + x is exact in FP32), on the
// FP32 pipe (GB300's FP64 rate would bound the drains).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err;
}

// tiles: list of (row tile, col tile) of the upper triangle; nprod: 1 (BF16)
// or 3 (3xBF16).
__global__ void __launch_bounds__(kGThreads, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                   const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                   const int2* __restrict__ tiles, int ntiles, int nkb_total, int nsplit, int nprod,
                   float2* __restrict__ part, unsigned* __restrict__ pace, int* __restrict__ status) {
  extern __shared__ uint8_t gsm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  GBars* bs = reinterpret_cast<GBars*>(smem + kGStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) tc::mbar_init(&bs->full[s], 1), tc::mbar_init(&bs->empty[s], 1);
    for (int b = 0; b < 2; ++b) tc::mbar_init(&bs->accf[b], 1), tc::mbar_init(&bs->acce[b], 4);
    tc::mbar_init(&bs->done, 1);
    bs->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc(&bs->tmem_base, 512);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = bs->tmem_base;
  // item w = (K split ch, tile ti); split ch takes the drain blocks ch,
  // ch + nsplit, ... so every CTA sweeps the cells in the same order and the
  // current slice of the X^T planes is read from L2 by all tiles
  const int items = ntiles * nsplit;
  const int kstride = nsplit * kSub;
  const uint32_t stage_tx = uint32_t(nprod == 3 ? kStageBytes : kABytes + kBBytes);

  if (warp == 0) {
    if (lane == 0) {
      long long issued = 0;
      for (int w = blockIdx.x; w < items && !g_aborted(bs); w += gridDim.x) {
        const int ch = w / ntiles, ti = w - ch * ntiles;
        const int2 tl = tiles[ti];
        for (int sb = ch * kSub; sb < nkb_total && !g_aborted(bs); sb += kstride) {
          if (pace) {
            // pacing (one item per co-resident CTA): start drain q once every
            // CTA has started drain q - kPaceWindow, so the CTAs sweep the
            // cells within an L2-sized window and share the planes' reads
            const int q = (sb - ch * kSub) / kstride;
            atomicAdd(pace + q, 1u);
            if (q >= kPaceWindow) {
              const volatile unsigned* pw = pace + (q - kPaceWindow);
              long long spins = 0;
              while (*pw < gridDim.x) {
                if (g_aborted(bs) || ++spins > kGSpin) {
                  g_abort(bs, status);
                  break;
                }
                __nanosleep(64);
              }
              if (g_aborted(bs)) break;
            }
          }
          const int se = min(nkb_total, sb + kSub);
          for (int kb = sb; kb < se; ++kb, ++issued) {
            const int s = int(issued % kGStages);
            const uint32_t k = uint32_t(issued / kGStages);
            if (!tc::mbar_wait(&bs->empty[s], (k & 1) ^ 1, kGSpin)) {
              g_abort(bs, status);
              break;
            }
            uint8_t* st = smem + s * kStageBytes;
            tc::mbar_arrive_expect_tx(&bs->full[s], stage_tx);
            tc::tma_load_2d(st, &tAh, &bs->full[s], kb * 64, tl.x * kGM);
            tc::tma_load_2d(st + 2 * kABytes, &tBh, &bs->full[s], kb * 64, tl.y * kGN);
            if (nprod == 3) {
              tc::tma_load_2d(st + kABytes, &tAl, &bs->full[s], kb * 64, tl.x * kGM);
              tc::tma_load_2d(st + 2 * kABytes + kBBytes, &tBl, &bs->full[s], kb * 64, tl.y * kGN);
            }
          }
        }
      }
      if (g_aborted(bs))
        for (long long x = issued > kGStages ? issued - kGStages : 0; x < issued; ++x)
          tc::mbar_wait(&bs->full[x % kGStages], uint32_t(x / kGStages) & 1, kGSpin);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kGM, kGN);
      long long used = 0, accu = 0;
      for (int w = blockIdx.x; w < items && !g_aborted(bs); w += gridDim.x) {
        const int ch = w / ntiles;
        for (int sb = ch * kSub; sb < nkb_total && !g_aborted(bs); sb += kstride, ++accu) {
          const int b = int(accu & 1);
          if (!tc::mbar_wait(&bs->acce[b], (uint32_t(accu >> 1) & 1) ^ 1, kGSpin)) {
            g_abort(bs, status);
            break;
          }
          tc::fence_after_sync();
          const uint32_t d = tmem + uint32_t(b * kGN);
          bool first = true;
          const int se = min(nkb_total, sb + kSub);
          for (int kb = sb; kb < se; ++kb, ++used) {
            const int s = int(used % kGStages);
            if (!tc::mbar_wait(&bs->full[s], uint32_t(used / kGStages) & 1, kGSpin)) {
              g_abort(bs, status);
              break;
            }
            tc::fence_after_sync();
            const uint32_t st = tc::smem_u32(smem + s * kStageBytes);
            const uint32_t ah = st, al = st + kABytes, bh = st + 2 * kABytes, bl = bh + kBBytes;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              tc::mma_bf16(d, tc::sdesc_k128(ah + ks * 32), tc::sdesc_k128(bh + ks * 32), idesc, first ? 0u : 1u);
              first = false;
              if (nprod == 3) {
                tc::mma_bf16(d, tc::sdesc_k128(ah + ks * 32), tc::sdesc_k128(bl + ks * 32), idesc, 1u);
                tc::mma_bf16(d, tc::sdesc_k128(al + ks * 32), tc::sdesc_k128(bh + ks * 32), idesc, 1u);
              }
            }
            tc::mma_commit(&bs->empty[s]);
          }
          if (g_aborted(bs)) break;
          tc::mma_commit(&bs->accf[b]);
        }
      }
      tc::mma_commit(&bs->done);
      tc::mbar_wait(&bs->done, 0, kGSpin);
    }
  } else {
    // epilogue: thread = one tile row (TMEM lane), 256 FP32 columns
    const int q = warp & 3;
    const int row = q * 32 + lane;
    long long accu = 0;
    for (int w = blockIdx.x; w < items && !g_aborted(bs); w += gridDim.x) {
      const int ch = w / ntiles;
      float4* dst = reinterpret_cast<float4*>(part + (int64_t(w) * kGM + row) * kGN);
      for (int sb = ch * kSub; sb < nkb_total && !g_aborted(bs); sb += kstride, ++accu) {
        const int b = int(accu & 1);
        if (!tc::mbar_wait(&bs->accf[b], uint32_t(accu >> 1) & 1, kGSpin)) {
          g_abort(bs, status);
          break;
        }
        tc::fence_after_sync();
        const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(b * kGN);
        const bool init = sb == ch * kSub;
#pragma unroll 1
        for (int c = 0; c < kGN / 32; ++c) {
          uint32_t r[32];
          __syncwarp();
          tc::tmem_ld_32x32b_x32(taddr + c * 32, r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float x0 = __uint_as_float(r[2 * e]), x1 = __uint_as_float(r[2 * e + 1]);
            float4 v;  // (hi, lo) of two columns
            if (init) {
              v = make_float4(x0, 0.f, x1, 0.f);
            } else {
              v = dst[c * 16 + e];
              two_sum_acc(v.x, v.y, x0);
              two_sum_acc(v.z, v.w, x1);
            }
            dst[c * 16 + e] = v;
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bs->acce[b]);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 512);
  }
}

// S[a][c] = sum over K splits of the partial tile holding (min, max), each a
// double-float (hi, lo) pair, summed in FP64.
__global__ void gram_tc_combine_kernel(const float2* __restrict__ part, const int* __restrict__ tile_of, int ntn,
                                       int ntiles, int nsplit, int64_t p, double* __restrict__ S, int64_t lds,
                                       int accumulate) {
  const int64_t a = int64_t(blockIdx.y) * blockDim.y + threadIdx.y;
  const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a >= p || c >= p) return;
  const int64_t lo = min(a, c), hi = max(a, c);
  const int ti = tile_of[(lo / kGM) * ntn + hi / kGN];
  const int64_t off = (lo % kGM) * kGN + hi % kGN;
  double s = 0.0;
  for (int ch = 0; ch < nsplit; ++ch) {
    const float2 hl = part[(int64_t(ch) * ntiles + ti) * (kGM * kGN) + off];
    s += double(hl.x) + double(hl.y);
  }
  if (accumulate)
    S[a * lds + c] += s;
  else
    S[a * lds + c] = s;
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn g_encode() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

// X^T plane: p rows x ld_t bf16 (row-major), box boxrows x 64
bool gmap(CUtensorMap* m, const void* base, int64_t p, int64_t ld_t, int boxrows) {
  EncodeFn fn = g_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {cuuint64_t(ld_t), cuuint64_t(p)};
  cuuint64_t strides[1] = {cuuint64_t(ld_t) * 2};
  cuuint32_t box[2] = {64u, cuuint32_t(boxrows)};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct GramPlan {
  int ntm, ntn, ntiles, nkb, nsplit;
};

GramPlan plan(const gmgm_matrix* m, int num_sms) {
  GramPlan g;
  const int64_t p = m->cols;
  g.ntm = int((p + kGM - 1) / kGM);
  g.ntn = int((p + kGN - 1) / kGN);
  g.ntiles = 0;
  for (int nt = 0; nt < g.ntn; ++nt)
    for (int mt = 0; mt < g.ntm; ++mt)
      if (int64_t(nt) * kGN + kGN - 1 >= int64_t(mt) * kGM) ++g.ntiles;
  g.nkb = int(m->ld_t / 64);
  // K splits per tile: enough work items to cover the SMs, each split at
  // least one drain long
  g.nsplit = std::max(1, std::min((num_sms + g.ntiles / 2) / g.ntiles, (g.nkb + kSub - 1) / kSub));
  return g;
}

}  // namespace

int gram_tc_splits(gmgm_handle* h, const gmgm_matrix* m) { return plan(m, h->num_sms).nsplit; }

size_t gram_tc_scratch_bytes(gmgm_handle* h, const gmgm_matrix* m) {
  GramPlan g = plan(m, h->num_sms);
  return Carve::round(size_t(g.nsplit) * g.ntiles * kGM * kGN * 8) + Carve::round(size_t(g.ntiles) * 8) +
         Carve::round(size_t(g.ntm) * g.ntn * 4) + Carve::round((size_t(g.nkb) + 2) * 4) + 4096;
}

cudaError_t launch_gram_tc(gmgm_handle* h, const gmgm_matrix* m, gmgm_prec prec, double* S, int64_t lds,
                           int accumulate, float* scratch, int /*splits*/) {
  GramPlan g = plan(m, h->num_sms);
  Carve c(scratch);
  float2* part = c.take<float2>(size_t(g.nsplit) * g.ntiles * kGM * kGN);
  int2* tiles = c.take<int2>(g.ntiles);
  int* tile_of = c.take<int>(size_t(g.ntm) * g.ntn);
  unsigned* pace = c.take<unsigned>(size_t(g.nkb) + 2);
  // tile list (host-built, small) and its inverse map
  std::vector<int2> ht;
  std::vector<int> hof(size_t(g.ntm) * g.ntn, -1);
  for (int nt = 0; nt < g.ntn; ++nt)
    for (int mt = 0; mt < g.ntm; ++mt)
      if (int64_t(nt) * kGN + kGN - 1 >= int64_t(mt) * kGM) {
        hof[size_t(mt) * g.ntn + nt] = int(ht.size());
        ht.push_back(make_int2(mt, nt));
      }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(tiles, ht.data(), ht.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(tile_of, hof.data(), hof.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream)) !=
      cudaSuccess)
    return e;
  // the host vectors must outlive the async copies
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return e;
  const int nprod = prec == GMGM_BF16X3 ? 3 : 1;
  CUtensorMap ah, al, bh, bl;
  const void* lo = m->xt_lo ? m->xt_lo : m->xt_hi;
  if (!gmap(&ah, m->xt_hi, m->cols, m->ld_t, kGM) || !gmap(&al, lo, m->cols, m->ld_t, kGM) ||
      !gmap(&bh, m->xt_hi, m->cols, m->ld_t, kGN) || !gmap(&bl, lo, m->cols, m->ld_t, kGN))
    return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kGSmem))) !=
      cudaSuccess)
    return e;
  const int items = g.ntiles * g.nsplit;
  const int grid = std::min(items, h->num_sms);
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram_tc_kernel, kGThreads, kGSmem)) != cudaSuccess)
    return e;
  if (items <= h->num_sms && per_sm >= 1) {
    // one item per CTA, all co-resident (cooperative launch): paced sweep
    const int kstride = g.nsplit * kSub;
    const int nq = (g.nkb + kstride - 1) / kstride + 1;
    if ((e = cudaMemsetAsync(pace, 0, size_t(nq) * sizeof(unsigned), h->stream)) != cudaSuccess) return e;
    const int2* tl = tiles;
    int nt = g.ntiles, nkb = g.nkb, ns = g.nsplit, np = nprod;
    int* status = h->d_status;
    void* args[] = {&ah, &al, &bh, &bl, &tl, &nt, &nkb, &ns, &np, &part, &pace, &status};
    if ((e = cudaLaunchCooperativeKernel((void*)gram_tc_kernel, dim3(grid), dim3(kGThreads), args, kGSmem,
                                         h->stream)) != cudaSuccess)
      return e;
  } else {
    gram_tc_kernel<<<grid, kGThreads, kGSmem, h->stream>>>(ah, al, bh, bl, tiles, g.ntiles, g.nkb, g.nsplit, nprod,
                                                           part, nullptr, h->d_status);
  }
  dim3 cb(32, 8), cg(unsigned((m->cols + 31) / 32), unsigned((m->cols + 7) / 8));
  gram_tc_combine_kernel<<<cg, cb, 0, h->stream>>>(part, tile_of, g.ntn, g.ntiles, g.nsplit, m->cols, S, lds,
                                                   accumulate);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace gmgm
