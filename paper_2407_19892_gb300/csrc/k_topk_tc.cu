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
//               every B tile into a shared-memory ring;
//   warp 1      MMA issuer (one thread): per B tile D[128 x TN] = A B^T
//               (K = 64 in four K=16 steps), FP32 in TMEM, double-buffered;
//   warps 2-9   screening: two threads per row (one per half of the tile's
//               columns); tcgen05.ld.red (sm_103a) brings 32 columns at a
//               time together with their largest magnitude, so a chunk costs
//               one compare against its row's threshold, and a chunk that
//               beats it is copied (32 values) into the warp's queue in
//               shared memory;
//   warps 10-11 merging: each owns the (row, half) candidate lists of one
//               half and takes up to 32 queued chunks at a time, one per
//               lane, so 32 lists take their winners in parallel; it
//               publishes each list's minimum, and the screening threads
//               read their own and their partner's (the other half of the
//               row) as their threshold.
// The screening warps hand the accumulator back to the MMA right after
// loading it, and a chunk with winners costs them one copy, not a merge:
// the accumulator hand-off no longer waits on list updates, whose cost is
// about the same for 1 or 32 chunks.  A stale threshold only lets more
// chunks through.
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
constexpr int kInsWarps = 2;                 // list-merging warps, one per half of the tile's columns
constexpr int kThreads = 64 + 32 * (kEpiWarps + kInsWarps);
constexpr int kQ = 32;                       // queued hit chunks per epilogue warp (a power of two, >= 32)
constexpr int kQStride = 36;                 // words per queued chunk (32 values, 16-byte aligned rows)
constexpr int kQEnd = -1, kQDone = -2;       // queue entries that close a work item / the launch
constexpr int kATile = kTM * kKP * 2;        // 16 KB per plane
constexpr int kLists = 2 * kTM;              // (row, half) lists per CTA
constexpr unsigned kFull = 0xffffffffu;
constexpr long long kSpin = 1ll << 23;       // polls per bounded wait
constexpr int kSampK = 6;                    // chunk maxima kept by the sampling pass
constexpr int kSampMinTiles = 128;           // shortest slice that takes a sampling pass

// Release store / acquire load of a shared-memory word (CTA scope): the
// queue positions that hand hit chunks from the screening warps to the
// merging warps.
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(tc::smem_u32(p)) : "memory");
  return v;
}

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
  // lists (values, columns, slot-major), per list its count, minimum and
  // the minimum's slot, the published minima, and per epilogue warp a queue
  // of kQ hit chunks (values, (first column | lane) word, threshold) with its
  // two positions
  static constexpr size_t kLists_ = size_t(2) * kC * kLists * 4 + size_t(3) * kLists * 4 + size_t(kLists) * 8 +
                                    size_t(kEpiWarps) * (size_t(kQ) * (kQStride + 2) * 4 + 2 * 4);
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

// A list's published minimum for work item `tag` (-1 while it is not full or
// still shows an earlier item).
__device__ __forceinline__ float list_min(const volatile unsigned long long* pub, unsigned tag) {
  const unsigned long long pv = *pub;
  return unsigned(pv >> 32) == tag ? __uint_as_float(unsigned(pv)) : -1.f;
}

// One (row, half) list, slot-major (slot c of list L at [c * kLists + L]),
// unsorted: it fills, then an offer above its minimum replaces the minimum
// and a rescan of the 32 slots finds the next.  `cnt`, `minv` and `minp`
// live in shared memory between offers.  One lane per list.
__device__ __forceinline__ void list_offer(float* lv, int* li, int L, int& cnt, float& minv, int& minp, float v,
                                           int j) {
  if (cnt < kC) {
    lv[cnt * kLists + L] = v;
    li[cnt * kLists + L] = j;
    if (++cnt < kC) return;
  } else {
    if (v <= minv) return;
    lv[minp * kLists + L] = v;
    li[minp * kLists + L] = j;
  }
  minv = lv[L];
  minp = 0;
#pragma unroll 8
  for (int c = 1; c < kC; ++c) {
    const float x = lv[c * kLists + L];
    if (x < minv) minv = x, minp = c;
  }
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
  float* lv = reinterpret_cast<float*>(sB + S::kStages * S::kPlanes * S::kBTile);  // [kC][kLists]
  int* li = reinterpret_cast<int*>(lv + kC * kLists);                              // [kC][kLists]
  int* lcnt = reinterpret_cast<int*>(li + kC * kLists);                           // [kLists]
  float* lmin = reinterpret_cast<float*>(lcnt + kLists);                          // [kLists]
  int* lminp = reinterpret_cast<int*>(lmin + kLists);                             // [kLists]
  unsigned long long* pubs = reinterpret_cast<unsigned long long*>(lminp + kLists);  // [kLists] (tag, minimum)
  uint32_t* qval_all = reinterpret_cast<uint32_t*>(pubs + kLists);               // [kEpiWarps][kQ][kQStride]
  int* qmeta_all = reinterpret_cast<int*>(qval_all + kEpiWarps * kQ * kQStride); // [kEpiWarps][kQ]
  float* qthr_all = reinterpret_cast<float*>(qmeta_all + kEpiWarps * kQ);        // [kEpiWarps][kQ]
  int* qpos = reinterpret_cast<int*>(qthr_all + kEpiWarps * kQ);                 // [kEpiWarps][2]: tail, head
  Bars* bs = reinterpret_cast<Bars*>(qpos + kEpiWarps * 2);
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
  for (int L = threadIdx.x; L < kLists; L += blockDim.x)
    pubs[L] = ~0ull, lcnt[L] = 0, lmin[L] = -1.f, lminp[L] = 0;  // empty lists, no row block yet
  for (int x = threadIdx.x; x < kEpiWarps * 2; x += blockDim.x) qpos[x] = 0;
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
  } else if (warp < 2 + kEpiWarps) {
    // ---------------- epilogue ----------------
    // Screens each tile's chunks against the row's threshold and queues the
    // chunks that beat it for the merging warp of its half.
    const int ew = warp - 2;
    const int half = ew >> 2;  // half of the tile's columns (warp-uniform)
    const int q = warp & 3;    // TMEM lane quarter this warp may access
    const int row_local = q * 32 + lane;
    const int L = half * kTM + row_local;
    const volatile unsigned long long* own = pubs + L;
    const volatile unsigned long long* partner = pubs + (1 - half) * kTM + row_local;
    uint32_t* qval = qval_all + ew * kQ * kQStride;
    int* qmeta = qmeta_all + ew * kQ;
    float* qthr = qthr_all + ew * kQ;
    int* qtail = qpos + ew * 2;
    const int* qhead = qpos + ew * 2 + 1;
    const unsigned lt = (1u << lane) - 1u;
    int tail = 0, head_seen = 0, published = 0;
    bool ok = true;
    auto publish = [&]() {  // the entries written so far become visible to the merging warp
      __syncwarp();
      if (lane == 0) st_release(qtail, tail);
      published = tail;
    };
    // room for `need` more entries; false (abort raised) when the wait gives up
    auto room = [&](int need) -> bool {
      if (tail + need - head_seen <= kQ) return true;
      if (published != tail) publish();
      const uint64_t t0 = tc::globaltimer_ns();
      for (;;) {
        head_seen = __shfl_sync(kFull, lane == 0 ? ld_acquire(qhead) : 0, 0);
        if (tail + need - head_seen <= kQ) return true;
        if (__any_sync(kFull, aborted(bs)) || tc::globaltimer_ns() - t0 > tc::kWaitLimitNs) {
          if (lane == 0) raise_abort(bs, status);
          return false;
        }
      }
    };
    long long accu = 0;
    for (int w = blockIdx.x; w < items && ok; w += gridDim.x) {
      if (__any_sync(kFull, aborted(bs))) break;
      const int cs = w % ncs;
      const int t0 = cs * per_slice, t1 = min(ntiles, t0 + per_slice);
      const unsigned tag = unsigned(w);
      const int ns = sample_tiles<SAMP>(t0, t1);
      float floor_v = -1.f;  // no floor until a sampling pass has run
      if (SAMP > 0 && ns > 0) {
        const int p = (w / ncs) * kTM + row_local;
        const int self = p < m ? (rows ? rows[p] : p) : -1;  // its column in Psi
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
      float thr = floor_v;
      for (int t = t0; ok && t < t1; ++t, ++accu) {
        uint32_t r[S::kChunks][32];
        float cm[S::kChunks];
        ok = take_tile<S>(bs, tmem, q, half, accu, lane, status, r, cm);
        if (!ok) break;
        // the previous tile's chunks are published only now, once this tile's
        // accumulator is back with the MMA (off the hand-off's critical path)
        if (published != tail) publish();
        const int j0 = t * TN + half * (TN / 2);  // warp-uniform
        if ((t & 31) == 0)  // the lists' minima move slowly: every 32nd tile is often enough
          thr = fmaxf(thr, fmaxf(list_min(own, tag), list_min(partner, tag)));
#pragma unroll
        for (int c = 0; c < S::kChunks; ++c) {
          // (the chunk holding a row's own column always passes: the merge drops that column)
          const bool hit = cm[c] > thr;
          const unsigned hm = __ballot_sync(kFull, hit);
          if (hm) {
            const int cnt = __popc(hm);
            if (!room(cnt)) {
              ok = false;
              break;
            }
            if (hit) {
              const int slot = (tail + __popc(hm & lt)) & (kQ - 1);
              uint4* dst = reinterpret_cast<uint4*>(qval + slot * kQStride);
#pragma unroll
              for (int k = 0; k < 8; ++k)
                dst[k] = make_uint4(r[c][4 * k], r[c][4 * k + 1], r[c][4 * k + 2], r[c][4 * k + 3]);
              qmeta[slot] = (j0 + c * 32) | lane;
              qthr[slot] = thr;
            }
            tail += cnt;
          }
        }
      }
      if (!ok || !room(1)) break;
      // close the item: the rows' floors travel in the entry's values
      const int slot = tail & (kQ - 1);
      qval[slot * kQStride + lane] = __float_as_uint(floor_v);
      if (lane == 0) qmeta[slot] = kQEnd;
      ++tail;
      publish();
    }
    if (room(1)) {  // no more items (or an abort): release the merging warp
      if (lane == 0) qmeta[tail & (kQ - 1)] = kQDone;
      ++tail;
      publish();
    }
  } else {
    // ---------------- list merging ----------------
    // Warp iw owns the lists of half iw, fed by the queues of epilogue warps
    // 4 iw .. 4 iw + 3.  It takes up to 32 queued chunks at a time, one per
    // lane, and each lane merges its chunk's winners into its row's list
    // (lanes whose chunks share a list take turns), then publishes the list's
    // minimum for the screen.  A queue's closing entry writes its 32 lists out
    // with their thresholds and empties them for the next work item.
    const int iw = warp - 2 - kEpiWarps;
    const unsigned lt = (1u << lane) - 1u;
    int head[4] = {0, 0, 0, 0}, item_no[4] = {0, 0, 0, 0};
    unsigned done_mask = 0;
    uint64_t idle_since = 0;
    int patience = 0;
    while (done_mask != 0xFu) {
      // -- gather: entries available in the four queues, up to each queue's next closing entry
      int avail[4];
      int total = 0;
      {
        const int my_tail = lane < 4 ? ld_acquire(qpos + (iw * 4 + lane) * 2) : 0;  // lanes 0-3: one queue each
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int tl = __shfl_sync(kFull, my_tail, k);
          avail[k] = (done_mask >> k) & 1u ? 0 : tl - head[k];
        }
      }
      // lane i takes the i-th available entry (queues in order); closing entries stop their queue's run
      int my_k = -1, my_pos = 0;
      {
        int before = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int ew = iw * 4 + k;
          // first closing entry among this queue's available ones (lanes look at one each)
          const bool look = lane < avail[k];
          const int meta = look ? qmeta_all[ew * kQ + ((head[k] + lane) & (kQ - 1))] : 0;
          const unsigned closing = __ballot_sync(kFull, look && meta < 0);
          const int run = closing ? __ffs(closing) - 1 : avail[k];  // ordinary entries before it
          const int take = min(run, 32 - before);                    // those that still find a lane
          if (lane >= before && lane < before + take) my_k = k, my_pos = head[k] + (lane - before);
          avail[k] = closing && take == run ? -(take + 1) : take;  // negative: the closing entry is next
          before += take;
        }
        total = before;
      }
      // a short wait lets a batch grow (the merge costs about the same for 1 or 32 chunks)
      bool closing_any = false;
#pragma unroll
      for (int k = 0; k < 4; ++k) closing_any |= avail[k] < 0;
      if (total < 8 && !closing_any && patience < 8) {
        ++patience;
        __nanosleep(256);
        continue;
      }
      patience = 0;
      bool progress = total > 0;
      // -- merge: one chunk per lane
      if (my_k >= 0) {
        const int ew = iw * 4 + my_k;
        const int slot = my_pos & (kQ - 1);
        const int meta = qmeta_all[ew * kQ + slot];
        const float thr_e = qthr_all[ew * kQ + slot];
        const uint32_t* vals = qval_all + (ew * kQ + slot) * kQStride;
        const int h = meta & 31;
        const int jc = meta & ~31;
        const int qw = (ew + 2) & 3;
        const int Lm = iw * kTM + qw * 32 + h;
        const int ino = my_k == 0 ? item_no[0] : my_k == 1 ? item_no[1] : my_k == 2 ? item_no[2] : item_no[3];
        const int w = blockIdx.x + ino * gridDim.x;
        const int p = (w / ncs) * kTM + qw * 32 + h;
        const int self = p < m ? (rows ? rows[p] : p) : -1;
        unsigned win = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint4 v4 = reinterpret_cast<const uint4*>(vals)[k];
          win |= (fabsf(__uint_as_float(v4.x)) > thr_e ? 1u : 0u) << (4 * k);
          win |= (fabsf(__uint_as_float(v4.y)) > thr_e ? 1u : 0u) << (4 * k + 1);
          win |= (fabsf(__uint_as_float(v4.z)) > thr_e ? 1u : 0u) << (4 * k + 2);
          win |= (fabsf(__uint_as_float(v4.w)) > thr_e ? 1u : 0u) << (4 * k + 3);
        }
        if (self - jc >= 0 && self - jc < 32) win &= ~(1u << (self - jc));
        if (n - jc < 32) win &= n - jc <= 0 ? 0u : (1u << (n - jc)) - 1u;
        // lanes whose chunks share a list take turns, in lane order
        const unsigned active = __activemask();
        const unsigned peers = __match_any_sync(active, Lm);
        const int turn = __popc(peers & lt);
        const int turns = __popc(peers);
        const int rounds = __reduce_max_sync(active, unsigned(turns));
        for (int tr = 0; tr < rounds; ++tr) {
          if (tr == turn) {
            int cnt = lcnt[Lm], minp = lminp[Lm];
            float minv = lmin[Lm];
            while (win) {
              const int e = __ffs(win) - 1;
              win &= win - 1;
              list_offer(lv, li, Lm, cnt, minv, minp, fabsf(__uint_as_float(vals[e])), jc + e);
            }
            lcnt[Lm] = cnt, lmin[Lm] = minv, lminp[Lm] = minp;
            *reinterpret_cast<volatile unsigned long long*>(pubs + Lm) =
                (static_cast<unsigned long long>(unsigned(w)) << 32) | __float_as_uint(cnt < kC ? -1.f : minv);
          }
          __syncwarp(active);
        }
      }
      __syncwarp();
      // -- release the merged entries; then a closing entry at the head of a queue
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int ew = iw * 4 + k;
        const int run = avail[k] < 0 ? -avail[k] - 1 : avail[k];
        head[k] += run;
        if (avail[k] < 0) {
          const int slot = head[k] & (kQ - 1);
          const int meta = qmeta_all[ew * kQ + slot];
          if (meta == kQEnd) {
            const int qw = (ew + 2) & 3;
            const int Lx = iw * kTM + qw * 32 + lane;  // lane x: list of row x of that quarter
            const int w = blockIdx.x + item_no[k] * gridDim.x;
            const int rb = w / ncs, cs = w - rb * ncs;
            const int px = rb * kTM + qw * 32 + lane;
            const float floor_x = __uint_as_float(qval_all[(ew * kQ + slot) * kQStride + lane]);
            const int cnt = lcnt[Lx];
            if (px < m) {
              const int64_t o = (int64_t(cs) * m + px) * (2 * kC) + iw * kC;
              for (int c = 0; c < kC; ++c) {
                cand_idx[o + c] = c < cnt ? li[c * kLists + Lx] : -1;
                cand_val[o + c] = c < cnt ? lv[c * kLists + Lx] : -1.f;
              }
              // every column left out has a screened value <= this (-1: no floor, list never full)
              thr_out[(int64_t(cs) * m + px) * 2 + iw] = fmaxf(floor_x, cnt < kC ? -1.f : lmin[Lx]);
            }
            lcnt[Lx] = 0, lmin[Lx] = -1.f, lminp[Lx] = 0;
            ++item_no[k];
          } else {
            done_mask |= 1u << k;
          }
          ++head[k];
          progress = true;
        }
      }
      __syncwarp();
      if (lane < 4)  // the slots are free again (lanes 0-3: one queue each)
        st_release(qpos + (iw * 4 + lane) * 2 + 1, lane == 0 ? head[0] : lane == 1 ? head[1] : lane == 2 ? head[2] : head[3]);
      if (progress) {
        idle_since = 0;
      } else {  // nothing queued: leave the issue slots to the epilogue warps for a while
        const uint64_t now = tc::globaltimer_ns();
        if (idle_since == 0) idle_since = now;
        if (__any_sync(kFull, aborted(bs)) || now - idle_since > tc::kWaitLimitNs) break;
        __nanosleep(200);
      }
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
