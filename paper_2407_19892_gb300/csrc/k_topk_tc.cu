// Tensor-core screens for the per-row top-k of Psi = V diag(psi) V^T
// (Algorithm 1: threshold simultaneously with recomposition), sm_103a.
//
// One kernel template, two instances:
//   main screen    BF16 operands (one product per K step), 128 x 256 tiles,
//                  over every row;
//   repair screen  3xBF16 split products (hi.hi + hi.lo + lo.hi: ~120x
//                  tighter error bound), 128 x 128 tiles, over the rows the
//                  main screen could not certify.
// Persistent, warp-specialised, one CTA per SM:
//   warp 0      TMA producer: the CTA's 128 A rows once per row block, then
//               every B tile into a 3-stage shared-memory ring;
//   warp 1      MMA issuer (one thread): per B tile D[128 x TN] = A B^T
//               (K = 64 in four K=16 steps), FP32 in TMEM, double-buffered;
//   warps 2-9   epilogue: two threads per row (one per half of the tile's
//               columns), each owning a kC-slot candidate list; tcgen05.ld.red
//               (sm_103a) brings 32 columns at a time together with their
//               largest magnitude, so a chunk costs one compare against the
//               list's threshold.
// A chunk that beats its row's threshold is merged by the whole warp: the
// owning lane stages its 32 values in shared memory, each lane takes one,
// and the winners enter the row's list, which is kept sorted over the lanes
// (lane c holds slot c; a ballot finds each winner's position and the lanes
// below it shift down one slot).  The threshold of a (row, half) list is the
// larger of its own minimum and its partner's (each list publishes its
// minimum in shared memory once full); a stale read only admits more
// candidates.
// Threshold floor (main screen, long sweeps): a sampling pass over every
// 16th B tile first keeps, per (row, half), the 6 largest 32-column chunk
// maxima in registers (a branch-free insert per chunk); the 6th of them is a
// floor below which the full sweep offers nothing.  About 6 x 16 columns of
// the half lie above it, so a list fills with values that mostly stay: the
// inserts of a random-order sweep (about kC ln(n / kC) per list) drop to
// about kC ln 3.  Every column left out of a row's two lists has a screened
// value <= the larger of the floor and the final minima.  Each row gets
// 2 kC candidates and two thresholds; the rescore keeps the kC largest
// screened values and folds the largest dropped one into the row's
// certification threshold.  All CTAs sweep the B tiles in the same order (L2
// reuse).  Every wait is bounded; on timeout the kernel records
// GMGM_DEV_TIMEOUT and leaves after freeing its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"
#include "topk_common.cuh"

namespace gmgm {
namespace {

constexpr int kTM = 128;                     // rows per row block (MMA M)
constexpr int kKP = 64;                      // padded K (bf16 elements, one 128-byte row)
constexpr int kMaxStages = 4;                // B-tile ring depth at most
constexpr size_t kSmemCap = 232448;          // dynamic shared memory per CTA
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kATile = kTM * kKP * 2;        // 16 KB per plane
constexpr int kLists = 2 * kTM;              // (row, half) lists per CTA
constexpr unsigned kFull = 0xffffffffu;
constexpr long long kSpin = 1ll << 23;       // polls per bounded wait
constexpr int kSampK = 6;                    // chunk maxima kept by the sampling pass
constexpr int kSampMinTiles = 128;           // shortest slice that takes a sampling pass

// Sampling-pass tiles of the slice [t0, t1): every SAMP-th tile, when the
// slice is long enough for a floor to pay.
template <int SAMP>
__host__ __device__ __forceinline__ int sample_tiles(int t0, int t1) {
  return (SAMP > 0 && t1 - t0 >= kSampMinTiles) ? (t1 - t0 + SAMP - 1) / SAMP : 0;
}

// B tile of step u of a work item: the ns sampled tiles, then the slice.
template <int SAMP>
__device__ __forceinline__ int tile_of(int u, int ns, int t0) {
  return u < ns ? t0 + u * SAMP : t0 + (u - ns);
}

struct __align__(8) Bars {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t accf[2];
  uint64_t acce[2];
  uint64_t afull;
  uint64_t aempty;
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

// TN columns per B tile; NP products per K step (1: BF16, 3: split).  The B
// ring takes as many stages (up to kMaxStages) as the shared memory left
// over holds.
template <int TN, int NP>
struct Screen {
  static constexpr int kTN = TN;
  static constexpr int kChunks = TN / 64;                 // 32-column chunks per half
  static constexpr int kPlanes = NP == 3 ? 2 : 1;         // hi (+ lo)
  static constexpr int kBTile = TN * kKP * 2;             // per plane
  static constexpr int kTmemCols = 2 * TN;
  // lists (values, columns), published minima, one 32-value staging row per epilogue warp
  static constexpr size_t kLists_ = size_t(2) * kC * kLists * 4 + size_t(kLists) * 8 + size_t(kEpiWarps) * 32 * 4;
  static constexpr size_t kFixed = 1024 /*align slack*/ + size_t(kPlanes) * kATile + kLists_ + sizeof(Bars);
  static constexpr int kStages = int((kSmemCap - kFixed) / (size_t(kPlanes) * kBTile)) < kMaxStages
                                     ? int((kSmemCap - kFixed) / (size_t(kPlanes) * kBTile))
                                     : kMaxStages;
  static_assert(kStages >= 2, "B-tile ring");
};

template <class S>
constexpr size_t smem_bytes() {
  return S::kFixed + size_t(S::kStages) * S::kPlanes * S::kBTile;
}

__device__ __forceinline__ void raise_abort(Bars* bs, int* status) {
  atomicExch(&bs->abort, 1);
  set_status(status, GMGM_DEV_TIMEOUT);
}

__device__ __forceinline__ bool aborted(Bars* bs) { return *reinterpret_cast<volatile int*>(&bs->abort) != 0; }

__device__ __forceinline__ float partner_min(const volatile unsigned long long* partner, unsigned tag) {
  const unsigned long long pv = *partner;
  return unsigned(pv >> 32) == tag ? __uint_as_float(unsigned(pv)) : -1.f;
}

// Warp-cooperative insert into one (row, half) list.  The list is sorted in
// descending order over the lanes: lane c holds slot c (value lv[Lr * kC +
// c], column li[...]), empty slots hold -1, so slot 31 is the list's minimum
// once it is full and -1 before.  Every lane offers at most one magnitude x
// (column jx; -1 offers nothing); those above `thr` are inserted one by one
// in lane order (a ballot finds the insertion position, the lanes below it
// shift down one slot and the last slot falls out).  Returns the new
// minimum.  Called by the whole warp.
__device__ __forceinline__ float coop_insert(float* lv, int* li, int Lr, int lane, float x, int jx, float thr) {
  float lval = lv[Lr * kC + lane];
  int lidx = li[Lr * kC + lane];
  unsigned w = __ballot_sync(kFull, x > thr);
  while (w) {
    const int e = __ffs(w) - 1;
    w &= w - 1;
    const float v = __shfl_sync(kFull, x, e);
    const int j = __shfl_sync(kFull, jx, e);
    if (v <= __shfl_sync(kFull, lval, 31)) continue;  // below the list's minimum by now (warp-uniform)
    const int pos = __popc(__ballot_sync(kFull, lval >= v));
    const float uv = __shfl_up_sync(kFull, lval, 1);
    const int ui = __shfl_up_sync(kFull, lidx, 1);
    if (lane > pos) lval = uv, lidx = ui;
    if (lane == pos) lval = v, lidx = j;
  }
  lv[Lr * kC + lane] = lval;
  li[Lr * kC + lane] = lidx;
  return __shfl_sync(kFull, lval, 31);
}

// Epilogue warp: wait for accumulator buffer accu & 1, pull this warp's lane
// quarter of the half's columns in one round trip, and hand the buffer back
// to the MMA warp.  mx[c] = max |r[c][e]| over chunk c, reduced by the
// tensor-memory load itself (tcgen05.ld.red).  False (abort raised) when the
// wait gives up.
template <class S>
__device__ __forceinline__ bool take_tile(Bars* bs, uint32_t tmem, int q, int half, long long accu, int lane,
                                          int* status, uint32_t (&r)[S::kChunks][32], float (&mx)[S::kChunks]) {
  const int b = int(accu & 1);
  if (!__all_sync(kFull, tc::mbar_wait(&bs->accf[b], uint32_t(accu >> 1) & 1, kSpin))) {
    if (lane == 0) raise_abort(bs, status);
    return false;
  }
  tc::fence_after_sync();
  const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(b * S::kTN + half * (S::kTN / 2));
  __syncwarp();
#pragma unroll
  for (int c = 0; c < S::kChunks; ++c) tc::tmem_ld_red_absmax_32x32b_x32(taddr + c * 32, r[c], mx[c]);
  tc::tmem_ld_wait();
  tc::fence_before_sync();
  __syncwarp();
  if (lane == 0) tc::mbar_arrive(&bs->acce[b]);
  return true;
}

// m rows of A (hi, lo planes) against n rows of B (hi, lo planes), the B
// tiles split into ncs column slices; work item = (row block, slice).  Row p
// of A is row rows[p] of Psi (p itself when rows is null); slice cs writes
// its two lists of row p to cand_*[cs * m + p][2 kC] and their thresholds to
// thr_out[cs * m + p][2].  SAMP > 0: sampling pass over every SAMP-th tile
// of a long slice first (threshold floor).
template <int TN, int NP, int SAMP>
__global__ void __launch_bounds__(kThreads, 1)
    screen_tc_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                     const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int m, int n,
                     int ncs, const int* __restrict__ rows, int32_t* __restrict__ cand_idx,
                     float* __restrict__ cand_val, float* __restrict__ thr_out, int* __restrict__ status,
                     unsigned long long* __restrict__ tiles_run) {
  using S = Screen<TN, NP>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                                  // [kPlanes][kATile]
  uint8_t* sB = sA + S::kPlanes * kATile;              // [kStages][kPlanes][kBTile]
  float* lv = reinterpret_cast<float*>(sB + S::kStages * S::kPlanes * S::kBTile);  // [kLists][kC]
  int* li = reinterpret_cast<int*>(lv + kC * kLists);                              // [kLists][kC]
  unsigned long long* pubs = reinterpret_cast<unsigned long long*>(li + kC * kLists);  // [kLists] (tag, minimum)
  uint32_t* stage_all = reinterpret_cast<uint32_t*>(pubs + kLists);              // [kEpiWarps][32]
  Bars* bs = reinterpret_cast<Bars*>(stage_all + kEpiWarps * 32);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S::kStages; ++s) tc::mbar_init(&bs->full[s], 1), tc::mbar_init(&bs->empty[s], 1);
    for (int b = 0; b < 2; ++b) tc::mbar_init(&bs->accf[b], 1), tc::mbar_init(&bs->acce[b], kEpiWarps);
    tc::mbar_init(&bs->afull, 1);
    tc::mbar_init(&bs->aempty, 1);
    tc::mbar_init(&bs->done, 1);
    bs->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmAh);
    tc::prefetch_tmap(&tmBh);
    if (NP == 3) {
      tc::prefetch_tmap(&tmAl);
      tc::prefetch_tmap(&tmBl);
    }
  }
  for (int L = threadIdx.x; L < kLists; L += blockDim.x) pubs[L] = ~0ull;  // no row block yet
  if (warp == 1) tc::tmem_alloc(&bs->tmem_base, S::kTmemCols);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = bs->tmem_base;
  const int nrb = (m + kTM - 1) / kTM;
  const int ntiles = (n + TN - 1) / TN;
  const int items = nrb * ncs;
  const int per_slice = (ntiles + ncs - 1) / ncs;  // B tiles per column slice

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      long long issued = 0;
      int rbi = 0;
      for (int w = blockIdx.x; w < items && !aborted(bs); w += gridDim.x, ++rbi) {
        const int rb = w / ncs, cs = w - rb * ncs;
        const int t0 = cs * per_slice, t1 = min(ntiles, t0 + per_slice);
        if (!tc::mbar_wait(&bs->aempty, (rbi & 1) ^ 1, kSpin)) {
          raise_abort(bs, status);
          break;
        }
        tc::mbar_arrive_expect_tx(&bs->afull, S::kPlanes * kATile);
        tc::tma_load_2d(sA, &tmAh, &bs->afull, 0, rb * kTM);
        if (NP == 3) tc::tma_load_2d(sA + kATile, &tmAl, &bs->afull, 0, rb * kTM);
        const int ns = sample_tiles<SAMP>(t0, t1);
        for (int u = 0; u < ns + (t1 - t0); ++u, ++issued) {
          const int t = tile_of<SAMP>(u, ns, t0);
          const int s = int(issued % S::kStages);
          const uint32_t k = uint32_t(issued / S::kStages);
          if (!tc::mbar_wait(&bs->empty[s], (k & 1) ^ 1, kSpin)) {
            raise_abort(bs, status);
            break;
          }
          uint8_t* dst = sB + s * S::kPlanes * S::kBTile;
          tc::mbar_arrive_expect_tx(&bs->full[s], S::kPlanes * S::kBTile);
          tc::tma_load_2d(dst, &tmBh, &bs->full[s], 0, t * TN);
          if (NP == 3) tc::tma_load_2d(dst + S::kBTile, &tmBl, &bs->full[s], 0, t * TN);
        }
        if (aborted(bs)) break;
      }
      if (aborted(bs)) {
        // let the loads already in flight land before the CTA can exit
        for (long long x = issued > S::kStages ? issued - S::kStages : 0; x < issued; ++x)
          tc::mbar_wait(&bs->full[x % S::kStages], uint32_t(x / S::kStages) & 1, kSpin);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = tc::idesc_bf16_f32(kTM, TN);
      const uint32_t ah = tc::smem_u32(sA), al = ah + kATile;
      long long used = 0, accu = 0;
      int rbi = 0;
      for (int w = blockIdx.x; w < items && !aborted(bs); w += gridDim.x, ++rbi) {
        const int cs = w % ncs;
        const int t0 = cs * per_slice, t1 = min(ntiles, t0 + per_slice);
        if (!tc::mbar_wait(&bs->afull, rbi & 1, kSpin)) {
          raise_abort(bs, status);
          break;
        }
        const int nsteps = sample_tiles<SAMP>(t0, t1) + (t1 - t0);
        for (int u = 0; u < nsteps; ++u, ++used, ++accu) {
          const int s = int(used % S::kStages);
          const int b = int(accu & 1);
          if (!tc::mbar_wait(&bs->full[s], uint32_t(used / S::kStages) & 1, kSpin) ||
              !tc::mbar_wait(&bs->acce[b], (uint32_t(accu >> 1) & 1) ^ 1, kSpin)) {
            raise_abort(bs, status);
            break;
          }
          tc::fence_after_sync();
          const uint32_t bh = tc::smem_u32(sB + s * S::kPlanes * S::kBTile), bl = bh + S::kBTile;
          const uint32_t d = tmem + uint32_t(b * TN);
#pragma unroll
          for (int ks = 0; ks < kKP / 16; ++ks) {  // K = 64 always: the padding columns are exact zeros
            tc::mma_bf16(d, tc::sdesc_k128(ah + ks * 32), tc::sdesc_k128(bh + ks * 32), idesc, ks > 0);
            if (NP == 3) {
              tc::mma_bf16(d, tc::sdesc_k128(ah + ks * 32), tc::sdesc_k128(bl + ks * 32), idesc, 1u);
              tc::mma_bf16(d, tc::sdesc_k128(al + ks * 32), tc::sdesc_k128(bh + ks * 32), idesc, 1u);
            }
          }
          tc::mma_commit(&bs->accf[b]);  // the epilogue's hand-off first: it is on the critical chain
          tc::mma_commit(&bs->empty[s]);
        }
        tc::mma_commit(&bs->aempty);
      }
      // drain: every MMA issued so far has completed once `done` fires
      tc::mma_commit(&bs->done);
      tc::mbar_wait(&bs->done, 0, kSpin);
      if (tiles_run) atomicAdd(tiles_run, static_cast<unsigned long long>(used));
    }
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;
    const int half = ew >> 2;  // half of the tile's columns (warp-uniform)
    const int q = warp & 3;    // TMEM lane quarter this warp may access
    const int row_local = q * 32 + lane;
    const int Lw = half * kTM + q * 32;  // list of lane 0 of this warp
    const int L = Lw + lane;
    unsigned long long* mine = pubs + L;
    const volatile unsigned long long* partner = pubs + (1 - half) * kTM + row_local;
    uint32_t* stg = stage_all + ew * 32;
    long long accu = 0;
    for (int w = blockIdx.x; w < items; w += gridDim.x) {
      if (__any_sync(kFull, aborted(bs))) break;
      const int rb = w / ncs, cs = w - rb * ncs;
      const int t0 = cs * per_slice, t1 = min(ntiles, t0 + per_slice);
      const int p = rb * kTM + row_local;                      // row of A
      const int self = p < m ? (rows ? rows[p] : p) : -1;     // its column in Psi
      const int64_t out = int64_t(cs) * m + p;                 // its list pair
      const unsigned tag = unsigned(w);
#pragma unroll 4
      for (int x = 0; x < 32; ++x) lv[(Lw + x) * kC + lane] = -1.f, li[(Lw + x) * kC + lane] = -1;  // the warp's lists
      float minv = -1.f;  // this lane's list minimum (-1 until full)
      bool ok = true;
      const int ns = sample_tiles<SAMP>(t0, t1);
      float floor_v = -1.f;  // no floor until a sampling pass has run
      if (SAMP > 0 && ns > 0) {
        float top[kSampK];   // largest chunk maxima so far, descending
#pragma unroll
        for (int x = 0; x < kSampK; ++x) top[x] = -1.f;
        for (int u = 0; u < ns; ++u, ++accu) {
          uint32_t r[S::kChunks][32];
          float cm[S::kChunks];
          ok = take_tile<S>(bs, tmem, q, half, accu, lane, status, r, cm);
          if (!ok) break;
          const int j0 = (t0 + u * SAMP) * TN + half * (TN / 2);
#pragma unroll
          for (int c = 0; c < S::kChunks; ++c) {
            float mx = cm[c];
            const int se = self - (j0 + c * 32);
            if (se >= 0 && se < 32) {  // the row's own column is no edge
              mx = 0.f;
#pragma unroll
              for (int e = 0; e < 32; ++e) mx = e == se ? mx : fmaxf(mx, fabsf(__uint_as_float(r[c][e])));
            }
#pragma unroll
            for (int x = 0; x < kSampK; ++x) {  // branch-free insert
              const float hi = fmaxf(top[x], mx);
              mx = fminf(top[x], mx);
              top[x] = hi;
            }
          }
        }
        floor_v = top[kSampK - 1];
      }
      __syncwarp();
      float thr = fmaxf(floor_v, minv);
      for (int t = t0; ok && t < t1; ++t, ++accu) {
        uint32_t r[S::kChunks][32];
        float cm[S::kChunks];
        ok = take_tile<S>(bs, tmem, q, half, accu, lane, status, r, cm);
        if (!ok) break;
        const int j0 = t * TN + half * (TN / 2);  // warp-uniform
        thr = fmaxf(thr, partner_min(partner, tag));
#pragma unroll
        for (int c = 0; c < S::kChunks; ++c) {
          // (the chunk holding a row's own column always passes: the insert drops that column)
          unsigned hm = __ballot_sync(kFull, cm[c] > thr);
          while (hm) {  // lanes whose chunk c beats their threshold, one at a time
            const int h = __ffs(hm) - 1;
            hm &= hm - 1;
            if (lane == h) {
#pragma unroll
              for (int k = 0; k < 8; ++k)
                reinterpret_cast<uint4*>(stg)[k] =
                    make_uint4(r[c][4 * k], r[c][4 * k + 1], r[c][4 * k + 2], r[c][4 * k + 3]);
            }
            __syncwarp();
            const int j = j0 + c * 32 + lane;
            const int self_h = __shfl_sync(kFull, self, h);  // (every lane takes part in each shuffle)
            const float thr_h = __shfl_sync(kFull, thr, h);
            const float x = (j < n && j != self_h) ? fabsf(__uint_as_float(stg[lane])) : -1.f;
            const float mnew = coop_insert(lv, li, Lw + h, lane, x, j, thr_h);
            __syncwarp();
            if (lane == h) {
              minv = mnew;
              thr = fmaxf(thr, mnew);
              *reinterpret_cast<volatile unsigned long long*>(mine) =
                  (static_cast<unsigned long long>(tag) << 32) | __float_as_uint(mnew);  // for the partner
            }
          }
        }
      }
      if (!ok || __any_sync(kFull, aborted(bs))) break;
      __syncwarp();
      for (int x = 0; x < 32; ++x) {  // the warp's lists, one coalesced row of kC slots each
        const int px = rb * kTM + q * 32 + x;
        if (px < m) {
          const int64_t o = (int64_t(cs) * m + px) * (2 * kC) + half * kC + lane;
          cand_idx[o] = li[(Lw + x) * kC + lane];
          cand_val[o] = lv[(Lw + x) * kC + lane];
        }
      }
      if (p < m) thr_out[out * 2 + half] = fmaxf(floor_v, minv);  // -1: no floor and the list never full
      __syncwarp();
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, S::kTmemCols);
  }
}

// Operands of the screens, rows x 64 bf16 row-major, K zero-padded.
__device__ __forceinline__ double vload(const void* V, int v64, int64_t idx) {
  return v64 ? static_cast<const double*>(V)[idx] : double(static_cast<const float*>(V)[idx]);
}

// Main screen: A = bf16(V psi), B = bf16(V).
__global__ void prep_tc_kernel(const void* V, int v64, int64_t ldv, const double* __restrict__ psi, int64_t n, int r,
                               __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ B) {
  const int64_t total = n * kKP;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / kKP;
    const int k = int(e - i * kKP);
    const double v = k < r ? vload(V, v64, i * ldv + k) : 0.0;
    A[e] = __float2bfloat16_rn(k < r ? float(v * psi[k]) : 0.f);
    B[e] = __float2bfloat16_rn(float(v));
  }
}

// Repair screen, split planes x = hi + lo (hi = bf16(x), lo = bf16(x - hi)):
// A for the listed rows (x = V_ik psi_k), and lo of B (x = V_ik; hi is the
// main screen's B).
__global__ void prep_split_kernel(const void* V, int v64, int64_t ldv, const double* __restrict__ psi, int64_t n, int r,
                                  const int* __restrict__ rows, int64_t m, const __nv_bfloat16* __restrict__ Bh,
                                  __nv_bfloat16* __restrict__ Bl, __nv_bfloat16* __restrict__ Ah,
                                  __nv_bfloat16* __restrict__ Al) {
  const int64_t nb = n * kKP, total = nb + m * kKP;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    if (e < nb) {
      const int64_t i = e / kKP;
      const int k = int(e - i * kKP);
      const float x = k < r ? float(vload(V, v64, i * ldv + k)) : 0.f;
      Bl[e] = __float2bfloat16_rn(x - __bfloat162float(Bh[e]));
    } else {
      const int64_t f = e - nb, p = f / kKP;
      const int k = int(f - p * kKP);
      const double x = k < r ? vload(V, v64, int64_t(rows[p]) * ldv + k) * psi[k] : 0.0;
      const __nv_bfloat16 hi = __float2bfloat16_rn(float(x));
      Ah[f] = hi;
      Al[f] = __float2bfloat16_rn(float(x - double(__bfloat162float(hi))));
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// rows x 64 bf16, row-major; box boxrows x 64 (one 128-byte swizzle span)
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int boxrows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cuuint64_t(kKP), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(kKP) * 2};
  cuuint32_t box[2] = {cuuint32_t(kKP), cuuint32_t(boxrows)};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TN, int NP, int SAMP>
cudaError_t run_screen(gmgm_handle* h, const void* ah, const void* al, int m, const void* bh, const void* bl, int n,
                       int ncs, const int* rows, int r, int32_t* cidx, float* cval, float* thr,
                       unsigned long long* tiles_run = nullptr) {
  CUtensorMap mah, mal, mbh, mbl;
  if (!make_map(&mah, ah, m, kTM) || !make_map(&mbh, bh, n, TN)) return cudaErrorInvalidValue;
  mal = mah;
  mbl = mbh;
  if (NP == 3 && (!make_map(&mal, al, m, kTM) || !make_map(&mbl, bl, n, TN))) return cudaErrorInvalidValue;
  auto kern = screen_tc_kernel<TN, NP, SAMP>;
  const size_t smem = smem_bytes<Screen<TN, NP>>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const int items = int((m + kTM - 1) / kTM) * ncs;
  const int grid = std::min(items, h->num_sms);
  kern<<<grid, kThreads, smem, h->stream>>>(mah, mal, mbh, mbl, m, n, ncs, rows, cidx, cval, thr, h->d_status,
                                            tiles_run);
  return cudaGetLastError();
}

// main: TN 256, one product, stash, sampling pass over every 16th tile;
// repair: TN 128, split products
using MainScreen = Screen<256, 1>;
using RepairScreen = Screen<128, 3>;
static_assert(smem_bytes<MainScreen>() <= kSmemCap && smem_bytes<RepairScreen>() <= kSmemCap, "shared memory");

}  // namespace

size_t topk_tc_scratch_bytes(int64_t d, int r, gmgm_prec prec) {
  if (prec != GMGM_BF16) return 0;
  // main A, B; repair lo of B, hi and lo of A (at most d listed rows)
  return Carve::round(size_t(d) * kKP * 2) * 5 + 1024;
}

int screen_tc_slices(int64_t m, int num_sms, int64_t cap_rows) {
  const int64_t nrb = (m + kTM - 1) / kTM;
  int64_t ncs = std::max<int64_t>(1, num_sms / std::max<int64_t>(1, nrb));
  ncs = std::min<int64_t>(ncs, 8);
  ncs = std::min<int64_t>(ncs, std::max<int64_t>(1, cap_rows / std::max<int64_t>(1, m)));
  return int(ncs);
}

cudaError_t launch_screen_tc(gmgm_handle* h, int64_t d, int r, const void* V, int v64, int64_t ldv, const double* psi,
                             gmgm_prec prec, int32_t* cidx, float* cval, float* thr, void* scratch, int64_t row0,
                             int64_t m, const int* rows, unsigned long long* tiles_run) {
  if (prec != GMGM_BF16 || r > kKP || d > (int64_t(1) << 30)) return cudaErrorNotSupported;
  Carve c(scratch);
  __nv_bfloat16* A = c.take<__nv_bfloat16>(size_t(d) * kKP);
  __nv_bfloat16* B = c.take<__nv_bfloat16>(size_t(d) * kKP);
  {
    const int64_t total = d * kKP;
    const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, int64_t(h->num_sms) * 16));
    prep_tc_kernel<<<blocks, 256, 0, h->stream>>>(V, v64, ldv, psi, d, r, A, B);
  }
  note_launch(2);
  // rows [row0, row0 + m): their A rows are contiguous from row row0
  return run_screen<256, 1, 16>(h, A + row0 * kKP, nullptr, int(m), B, nullptr, int(d), 1, rows, r, cidx, cval,
                                      thr, tiles_run);
}

cudaError_t launch_screen_tc_repair(gmgm_handle* h, int64_t d, int r, const void* V, int v64, int64_t ldv,
                                    const double* psi, const int* rows, int m, int ncs, int32_t* cidx, float* cval,
                                    float* thr, void* scratch) {
  if (r > kKP || d > (int64_t(1) << 30) || m < 1) return cudaErrorNotSupported;
  Carve c(scratch);
  c.take<__nv_bfloat16>(size_t(d) * kKP);  // main A (not used here)
  const __nv_bfloat16* Bh = c.take<__nv_bfloat16>(size_t(d) * kKP);
  __nv_bfloat16* Bl = c.take<__nv_bfloat16>(size_t(d) * kKP);
  __nv_bfloat16* Ah = c.take<__nv_bfloat16>(size_t(d) * kKP);
  __nv_bfloat16* Al = c.take<__nv_bfloat16>(size_t(d) * kKP);
  {
    const int64_t total = (d + m) * kKP;
    const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, int64_t(h->num_sms) * 16));
    prep_split_kernel<<<blocks, 256, 0, h->stream>>>(V, v64, ldv, psi, d, r, rows, m, Bh, Bl, Ah, Al);
  }
  note_launch(2);
  return run_screen<128, 3, 0>(h, Ah, Al, m, Bh, Bl, int(d), ncs, rows, r, cidx, cval, thr);
}

}  // namespace gmgm
