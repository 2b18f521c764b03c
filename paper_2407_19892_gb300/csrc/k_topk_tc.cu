// Tensor-core screen for the per-row top-k of Psi = V diag(psi) V^T
// (Algorithm 1: threshold simultaneously with recomposition), sm_103a.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0      TMA producer: the CTA's 128 A rows (bf16(V psi)) once per row
//               block, then every B tile (bf16(V), 256 rows) into a 4-stage
//               shared-memory ring;
//   warp 1      MMA issuer (one thread): per B tile D[128 x 256] = A B^T
//               (K = 64 in four K=16 steps), FP32 in TMEM, double-buffered
//               (2 x 256 of the 512 TMEM columns);
//   warps 2-9   epilogue: two threads per row (one per 128-column half of the
//               tile), each with a kC-slot candidate list; tcgen05.ld 32
//               columns at a time, one max per element against the pair's
//               shared threshold, and only when it is beaten a per-lane insert
//               (a bitmask of the winners, values pulled out of registers by a
//               select tree).
// A list is four sub-lists of 8 slots with their minima cached, so replacing
// the list's minimum rescans 8 slots, not 32.  Inserts are rare and
// scattered over the lanes, so a lane that hits a chunk parks the chunk's 32
// values in a shared-memory stash (one slot per thread) instead of inserting
// at once; after each tile the warp drains the stashes together once 8 lanes
// have one (a lane whose slot is taken inserts at once).  The pair's threshold is the
// larger of the two lists' minima (each list publishes its minimum in shared
// memory once full); a stale read only admits more candidates.  Every column
// left out of a row's two lists has a screened value <= the larger final
// minimum.  Each row gets 2 kC candidates and two thresholds; the rescore
// keeps the kC largest screened values and folds the largest dropped one into
// the row's certification threshold.  All CTAs sweep the B tiles in the same order (L2 reuse).  Every
// wait is bounded; on timeout the kernel records GMGM_DEV_TIMEOUT and leaves
// after freeing its TMEM.
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
constexpr int kTN = 256;                     // columns per B tile (MMA N)
constexpr int kKP = 64;                      // padded K (bf16 elements, one 128-byte row)
constexpr int kStages = 3;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kATile = kTM * kKP * 2;        // 16 KB
constexpr int kBTile = kTN * kKP * 2;        // 32 KB
constexpr int kSub = 8;                      // slots per sub-list
constexpr int kNSub = kC / kSub;             // sub-lists per list
constexpr int kLists = 2 * kTM;              // (row, half) lists per CTA
constexpr int kSlot = 36;                    // stash slot stride (words): 32 values, 16-byte aligned, 4-way banks
constexpr int kBatch = 8;                    // stashed lanes that trigger a drain
constexpr unsigned kFull = 0xffffffffu;
constexpr long long kSpin = 1ll << 23;       // polls per bounded wait

struct __align__(8) Bars {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t accf[2];
  uint64_t acce[2];
  uint64_t afull;
  uint64_t aempty;
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

constexpr size_t kSmemBytes = 1024 /*align slack*/ + size_t(kATile) + size_t(kStages) * kBTile +
                              size_t(2) * kC * kLists * 4 + size_t(2) * kNSub * kLists * 4 + size_t(kLists) * 8 +
                              size_t(32) * kEpiWarps * kSlot * 4 + sizeof(Bars);

__device__ __forceinline__ void raise_abort(Bars* bs, int* status) {
  atomicExch(&bs->abort, 1);
  set_status(status, GMGM_DEV_TIMEOUT);
}

__device__ __forceinline__ bool aborted(Bars* bs) { return *reinterpret_cast<volatile int*>(&bs->abort) != 0; }

// One (row, half) candidate list, slot-major (stride kLists): fill, then
// replace the minimum.  Slots [8s, 8s+8) form sub-list s, whose minimum and
// its slot sit in smv/smp (also slot-major).  Out of line (inserts are
// rare); state by value.
struct ListState {
  int cnt;
  int minsub;  // sub-list holding the minimum
  float minv;  // minimum once full, else -1
};

// r[e] for a per-lane runtime e without leaving registers: a 5-level select
// tree over constant indices (31 selects).
__device__ __forceinline__ uint32_t pick32(const uint32_t (&r)[32], int e) {
  uint32_t a[16], b[8], c[4], d[2];
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = (e & 16) ? r[q + 16] : r[q];
#pragma unroll
  for (int q = 0; q < 8; ++q) b[q] = (e & 8) ? a[q + 8] : a[q];
#pragma unroll
  for (int q = 0; q < 4; ++q) c[q] = (e & 4) ? b[q + 4] : b[q];
#pragma unroll
  for (int q = 0; q < 2; ++q) d[q] = (e & 2) ? c[q + 2] : c[q];
  return (e & 1) ? d[1] : d[0];
}

// Minimum (value, slot) of sub-list sub.
__device__ __forceinline__ void sub_min(const float* lv, int sub, float& mv, int& mp) {
  mv = lv[(sub * kSub) * kLists];
  mp = sub * kSub;
#pragma unroll
  for (int c = 1; c < kSub; ++c) {
    const float x = lv[(sub * kSub + c) * kLists];
    if (x < mv) mv = x, mp = sub * kSub + c;
  }
}

// The published minimum carries the row block it belongs to (high word), so
// a partner still in the previous row block is never mistaken for this one.
__device__ __noinline__ ListState offer(float* lv, int* li, float* smv, int* smp, unsigned long long* pub, unsigned tag,
                                        ListState st, float v, int j) {
  if (st.cnt < kC) {
    lv[st.cnt * kLists] = v;
    li[st.cnt * kLists] = j;
    if (++st.cnt < kC) return st;
#pragma unroll
    for (int s = 0; s < kNSub; ++s) {
      float mv;
      int mp;
      sub_min(lv, s, mv, mp);
      smv[s * kLists] = mv;
      smp[s * kLists] = mp;
    }
  } else {
    const int s = st.minsub;
    const int p = smp[s * kLists];
    lv[p * kLists] = v;
    li[p * kLists] = j;
    float mv;
    int mp;
    sub_min(lv, s, mv, mp);
    smv[s * kLists] = mv;
    smp[s * kLists] = mp;
  }
  st.minv = smv[0];
  st.minsub = 0;
#pragma unroll
  for (int s = 1; s < kNSub; ++s) {
    const float x = smv[s * kLists];
    if (x < st.minv) st.minv = x, st.minsub = s;
  }
  *reinterpret_cast<volatile unsigned long long*>(pub) =
      (static_cast<unsigned long long>(tag) << 32) | __float_as_uint(st.minv);  // publish for the partner
  return st;
}

__device__ __forceinline__ float partner_min(const volatile unsigned long long* partner, unsigned tag) {
  const unsigned long long pv = *partner;
  return unsigned(pv >> 32) == tag ? __uint_as_float(unsigned(pv)) : -1.f;
}

// Insert the winners of one stashed chunk (32 values, columns sj..sj+31)
// against the current threshold.
__device__ __noinline__ ListState drain(const uint32_t* slot, int sj, int i, int n, float* lv, int* li, float* smv,
                                        int* smp, unsigned long long* pub, const volatile unsigned long long* partner,
                                        unsigned tag, ListState st) {
  uint32_t v[32];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint4 w = reinterpret_cast<const uint4*>(slot)[k];
    v[4 * k] = w.x, v[4 * k + 1] = w.y, v[4 * k + 2] = w.z, v[4 * k + 3] = w.w;
  }
  float thr = fmaxf(st.minv, partner_min(partner, tag));
  uint32_t mask = 0;
#pragma unroll
  for (int e = 0; e < 32; ++e) mask |= (fabsf(__uint_as_float(v[e])) > thr ? 1u : 0u) << e;
  while (mask) {
    const int e = __ffs(mask) - 1;
    mask &= mask - 1;
    const float x = fabsf(__uint_as_float(pick32(v, e)));
    const int j = sj + e;
    if (x > thr && j < n && j != i) {
      st = offer(lv, li, smv, smp, pub, tag, st, x, j);
      thr = fmaxf(st.minv, partner_min(partner, tag));
    }
  }
  return st;
}

__global__ void __launch_bounds__(kThreads, 1)
    screen_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int n,
                     int ksteps, int32_t* __restrict__ cand_idx, float* __restrict__ cand_val,
                     float* __restrict__ thr_out, int* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + kATile;
  float* lv = reinterpret_cast<float*>(sB + kStages * kBTile);
  int* li = reinterpret_cast<int*>(lv + kC * kLists);
  float* smv_all = reinterpret_cast<float*>(li + kC * kLists);        // [kNSub][kLists] sub-list minima
  int* smp_all = reinterpret_cast<int*>(smv_all + kNSub * kLists);     // [kNSub][kLists] their slots
  unsigned long long* pubs = reinterpret_cast<unsigned long long*>(smp_all + kNSub * kLists);  // [kLists] (tag, minimum)
  uint32_t* stash = reinterpret_cast<uint32_t*>(pubs + kLists);  // [kEpiWarps * 32][kSlot]
  Bars* bs = reinterpret_cast<Bars*>(stash + 32 * kEpiWarps * kSlot);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) tc::mbar_init(&bs->full[s], 1), tc::mbar_init(&bs->empty[s], 1);
    for (int b = 0; b < 2; ++b) tc::mbar_init(&bs->accf[b], 1), tc::mbar_init(&bs->acce[b], kEpiWarps);
    tc::mbar_init(&bs->afull, 1);
    tc::mbar_init(&bs->aempty, 1);
    tc::mbar_init(&bs->done, 1);
    bs->abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  for (int L = threadIdx.x; L < kLists; L += blockDim.x) pubs[L] = ~0ull;  // no row block yet
  if (warp == 1) tc::tmem_alloc(&bs->tmem_base, 512);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = bs->tmem_base;
  const int nrb = (n + kTM - 1) / kTM;
  const int ntiles = (n + kTN - 1) / kTN;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      long long issued = 0;
      int rbi = 0;
      for (int rb = blockIdx.x; rb < nrb && !aborted(bs); rb += gridDim.x, ++rbi) {
        if (!tc::mbar_wait(&bs->aempty, (rbi & 1) ^ 1, kSpin)) {
          raise_abort(bs, status);
          break;
        }
        tc::mbar_arrive_expect_tx(&bs->afull, kATile);
        tc::tma_load_2d(sA, &tmA, &bs->afull, 0, rb * kTM);
        for (int t = 0; t < ntiles; ++t, ++issued) {
          const int s = int(issued % kStages);
          const uint32_t k = uint32_t(issued / kStages);
          if (!tc::mbar_wait(&bs->empty[s], (k & 1) ^ 1, kSpin)) {
            raise_abort(bs, status);
            break;
          }
          tc::mbar_arrive_expect_tx(&bs->full[s], kBTile);
          tc::tma_load_2d(sB + s * kBTile, &tmB, &bs->full[s], 0, t * kTN);
        }
        if (aborted(bs)) break;
      }
      if (aborted(bs)) {
        // let the loads already in flight land before the CTA can exit
        for (long long x = issued > kStages ? issued - kStages : 0; x < issued; ++x)
          tc::mbar_wait(&bs->full[x % kStages], uint32_t(x / kStages) & 1, kSpin);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = tc::idesc_bf16_f32(kTM, kTN);
      const uint32_t abase = tc::smem_u32(sA);
      long long used = 0, accu = 0;
      int rbi = 0;
      for (int rb = blockIdx.x; rb < nrb && !aborted(bs); rb += gridDim.x, ++rbi) {
        if (!tc::mbar_wait(&bs->afull, rbi & 1, kSpin)) {
          raise_abort(bs, status);
          break;
        }
        for (int t = 0; t < ntiles; ++t, ++used, ++accu) {
          const int s = int(used % kStages);
          const int b = int(accu & 1);
          if (!tc::mbar_wait(&bs->full[s], uint32_t(used / kStages) & 1, kSpin) ||
              !tc::mbar_wait(&bs->acce[b], (uint32_t(accu >> 1) & 1) ^ 1, kSpin)) {
            raise_abort(bs, status);
            break;
          }
          tc::fence_after_sync();
          const uint32_t bbase = tc::smem_u32(sB + s * kBTile);
          const uint32_t d = tmem + uint32_t(b * kTN);
          for (int ks = 0; ks < ksteps; ++ks)
            tc::mma_bf16(d, tc::sdesc_k128(abase + ks * 32), tc::sdesc_k128(bbase + ks * 32), idesc, ks > 0);
          tc::mma_commit(&bs->empty[s]);
          tc::mma_commit(&bs->accf[b]);
        }
        tc::mma_commit(&bs->aempty);
      }
      // drain: every MMA issued so far has completed once `done` fires
      tc::mma_commit(&bs->done);
      tc::mbar_wait(&bs->done, 0, kSpin);
    }
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;
    const int half = ew >> 2;  // 128-column half of the tile
    const int q = warp & 3;    // TMEM lane quarter this warp may access
    const int row_local = q * 32 + lane;
    const int L = half * kTM + row_local;
    float* mlv = lv + L;
    int* mli = li + L;
    float* msv = smv_all + L;
    int* msp = smp_all + L;
    unsigned long long* mine = pubs + L;
    const volatile unsigned long long* partner = pubs + (1 - half) * kTM + row_local;
    uint32_t* slot = stash + (ew * 32 + lane) * kSlot;
    long long accu = 0;
    for (int rb = blockIdx.x; rb < nrb; rb += gridDim.x) {
      if (__any_sync(kFull, aborted(bs))) break;
      const int i = rb * kTM + row_local;
      const unsigned tag = unsigned(rb);
      ListState st{0, 0, -1.f};
      bool parked = false;  // this lane's stash slot holds a chunk
      int sj = 0;           // its first column
      bool ok = true;
      for (int t = 0; t < ntiles; ++t, ++accu) {
        const int b = int(accu & 1);
        ok = __all_sync(kFull, tc::mbar_wait(&bs->accf[b], uint32_t(accu >> 1) & 1, kSpin));
        if (!ok) {
          if (lane == 0) raise_abort(bs, status);
          break;
        }
        tc::fence_after_sync();
        const uint32_t taddr = tmem + (uint32_t(q * 32) << 16) + uint32_t(b * kTN + half * 128);
        const int j0 = t * kTN + half * 128;
        // the whole 128-column slice in one round trip, then hand the
        // accumulator back to the MMA warp before scanning
        uint32_t r[4][32];
        __syncwarp();
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::tmem_ld_32x32b_x32(taddr + c * 32, r[c]);
        tc::tmem_ld_wait();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bs->acce[b]);
        float thr = fmaxf(st.minv, partner_min(partner, tag));
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;  // four short max chains
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            m0 = fmaxf(m0, fabsf(__uint_as_float(r[c][e + 0])));
            m1 = fmaxf(m1, fabsf(__uint_as_float(r[c][e + 1])));
            m2 = fmaxf(m2, fabsf(__uint_as_float(r[c][e + 2])));
            m3 = fmaxf(m3, fabsf(__uint_as_float(r[c][e + 3])));
          }
          if (fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)) > thr) {
            if (!parked) {
#pragma unroll
              for (int k = 0; k < 8; ++k)
                reinterpret_cast<uint4*>(slot)[k] = make_uint4(r[c][4 * k], r[c][4 * k + 1], r[c][4 * k + 2], r[c][4 * k + 3]);
              parked = true;
              sj = j0 + c * 32;
            } else {
              uint32_t mask = 0;
#pragma unroll
              for (int e = 0; e < 32; ++e) mask |= (fabsf(__uint_as_float(r[c][e])) > thr ? 1u : 0u) << e;
              while (mask) {
                const int e = __ffs(mask) - 1;
                mask &= mask - 1;
                const float v = fabsf(__uint_as_float(pick32(r[c], e)));
                const int j = j0 + c * 32 + e;
                if (v > thr && j < n && j != i) {
                  st = offer(mlv, mli, msv, msp, mine, tag, st, v, j);
                  thr = fmaxf(st.minv, partner_min(partner, tag));
                }
              }
            }
          }
        }
        if (__popc(__ballot_sync(kFull, parked)) >= kBatch) {
          if (parked) st = drain(slot, sj, i, n, mlv, mli, msv, msp, mine, partner, tag, st);
          parked = false;
          __syncwarp();
        }
      }
      if (!ok || __any_sync(kFull, aborted(bs))) break;
      if (parked) st = drain(slot, sj, i, n, mlv, mli, msv, msp, mine, partner, tag, st);
      if (i < n) {
        for (int c = 0; c < kC; ++c) {
          cand_idx[int64_t(i) * (2 * kC) + half * kC + c] = c < st.cnt ? mli[c * kLists] : -1;
          cand_val[int64_t(i) * (2 * kC) + half * kC + c] = c < st.cnt ? mlv[c * kLists] : -1.f;
        }
        thr_out[int64_t(i) * 2 + half] = st.minv;  // -1 while the list was never full
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 512);
  }
}

// bf16 operands of the screen: A = bf16(V psi), B = bf16(V), n x 64, K zero-padded.
__global__ void prep_tc_kernel(const void* V, int v64, int64_t ldv, const double* __restrict__ psi, int64_t n, int r,
                               __nv_bfloat16* __restrict__ A, __nv_bfloat16* __restrict__ B) {
  const int64_t total = n * kKP;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / kKP;
    const int k = int(e - i * kKP);
    double v = 0.0;
    if (k < r) v = v64 ? static_cast<const double*>(V)[i * ldv + k] : double(static_cast<const float*>(V)[i * ldv + k]);
    A[e] = __float2bfloat16_rn(k < r ? float(v * psi[k]) : 0.f);
    B[e] = __float2bfloat16_rn(float(v));
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
bool make_map(CUtensorMap* m, void* base, int64_t rows, int boxrows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cuuint64_t(kKP), cuuint64_t(rows)};
  cuuint64_t strides[1] = {cuuint64_t(kKP) * 2};
  cuuint32_t box[2] = {cuuint32_t(kKP), cuuint32_t(boxrows)};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t topk_tc_scratch_bytes(int64_t d, int r, gmgm_prec prec) {
  if (prec != GMGM_BF16) return 0;
  return Carve::round(size_t(d) * kKP * 2) * 2 + 1024;
}

cudaError_t launch_screen_tc(gmgm_handle* h, int64_t d, int r, const void* V, int v64, int64_t ldv, const double* psi,
                             gmgm_prec prec, int32_t* cidx, float* cval, float* thr, void* scratch) {
  if (prec != GMGM_BF16 || r > kKP || d > (int64_t(1) << 30)) return cudaErrorNotSupported;
  Carve c(scratch);
  __nv_bfloat16* A = c.take<__nv_bfloat16>(size_t(d) * kKP);
  __nv_bfloat16* B = c.take<__nv_bfloat16>(size_t(d) * kKP);
  {
    const int64_t total = d * kKP;
    const unsigned blocks = unsigned(std::min<int64_t>((total + 255) / 256, int64_t(h->num_sms) * 16));
    prep_tc_kernel<<<blocks, 256, 0, h->stream>>>(V, v64, ldv, psi, d, r, A, B);
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, d, kTM) || !make_map(&mb, B, d, kTN)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(screen_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemBytes));
  if (e != cudaSuccess) return e;
  const int nrb = int((d + kTM - 1) / kTM);
  const int grid = std::min(nrb, h->num_sms);
  const int ksteps = (r + 15) / 16;
  screen_tc_kernel<<<grid, kThreads, kSmemBytes, h->stream>>>(ma, mb, int(d), ksteps, cidx, cval, thr, h->d_status);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace gmgm
