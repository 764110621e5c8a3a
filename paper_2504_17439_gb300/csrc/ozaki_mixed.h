// The digit-sliced tensor-core GEMM of the mixed precision, with digit tiles
// reused across products.
//
// One operand carries 2 digits on a fixed-point grid (the DF tensor, see
// MGW_MIXED), the other 7 per-row digits; the products kept are the 13 with
// s + r <= 8 (streamed digit s, resident digit r).  The kernel of ozaki.h
// loads one A tile and one B tile per digit product, so every tile feeds one
// MMA and shared memory is written as fast as it is read.  Here the K loop
// runs in chunks of kCkb K blocks, and inside a chunk level by level
// (l = 2..8): the 2-digit ("resident") operand of the chunk is loaded once
// and serves all 13 products, and each digit s of the 7-digit ("streamed")
// operand is loaded once and serves levels s + 1 and s + 2.  Per K block the
// copies shrink from 13 (A + B) tiles to 7 streamed + 2 resident.
//
// Accumulation is as in ozaki.h, re-cut for the chunk order: each exact
// level (2..7) of one chunk is a phase in one of two alternating FP32 TMEM
// accumulators, flushed into 64-bit integers (levels 2..5 in the epilogue
// warps' registers, 6..7 in TMEM); a chunk holds at most 2 products x kCkb
// x 64 terms of magnitude <= 2^14 per level, so every phase sum is an
// integer below 2^22 in its level's unit, exact in FP32 and converted with
// one FFMA against 1.5 x 2^23.  Level 8 accumulates in a third FP32
// accumulator over all of K (below 2^-56 of the top, as in ozaki.h).
//
// CTA (384 threads): warp 0 loads the resident digit sets (two chunks in
// flight), warps 1-2 the streamed ones (a ring of kRing digit sets, warp 1
// the even ones, warp 2 the odd), warp 3 allocates TMEM (512 columns) and
// issues the MMAs, warps 4-11 are the epilogue (as in ozaki.h).  TMEM:
// accumulators [0,96) and [96,192), level 8 [192,288), levels 6..7 integer
// words [288,480).  All waits are time-bounded.
#pragma once

#include "ozaki.h"

namespace mgw {
namespace oz {

constexpr int kCkb = 2;    // K blocks per chunk
constexpr int kRing = 4;   // streamed digit sets in flight
constexpr int kRSets = 2;  // resident digit sets (chunks) in flight

// kRB: B is the resident (2-digit) operand and A streams (7 digits); else A
// is resident and B streams.
template <bool kRB>
struct MixedLayout {
  static constexpr int kRRows = kRB ? BN : BM, kSRows = kRB ? BM : BN;
  static constexpr int kRTile = kRRows * BK * 2, kSTile = kSRows * BK * 2;
  static constexpr int kRSet = kGridSlices * kCkb * kRTile;  // both digits of one chunk
  static constexpr int kSSet = kCkb * kSTile;               // one digit of one chunk
  static constexpr int kSOff = kRSets * kRSet;
  static constexpr int kBarOff = kSOff + kRing * kSSet;
  static constexpr int kSmem = 1024 + kBarOff + kBarBytes + BN * 4;
  static_assert(kSmem <= 232448, "dynamic shared memory above the 227 KB opt-in limit");
  static_assert(kRTile % 1024 == 0 && kSTile % 1024 == 0, "tiles on 1024-byte swizzle atoms");
};

// integer value of an FP32 phase sum v scaled by `up` (an exact integer of
// magnitude <= 2^22): the magic 1.5 x 2^23 puts it in the low mantissa bits
__device__ __forceinline__ int exact_int(float v, float up) {
  return __float_as_int(fmaf(v, up, 12582912.0f)) - 0x4B400000;
}

template <bool kRB, class ALoad, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
ozaki_mixed_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                   const int* __restrict__ ea, const int* __restrict__ eb, int M, int N, int K, int col_band,
                   int ksplit, ALoad al, Epi epi, int* status) {
  using namespace tc;
  using Lay = MixedLayout<kRB>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* rfull = reinterpret_cast<uint64_t*>(smem + Lay::kBarOff);  // [kRSets]
  uint64_t* rempty = rfull + kRSets;                                    // [kRSets]
  uint64_t* sfull = rempty + kRSets;                                    // [kRing]
  uint64_t* sempty = sfull + kRing;                                     // [kRing]
  uint64_t* accf = sempty + kRing;                                      // [3]: buffers 0, 1 and level 8
  uint64_t* acce = accf + 3;                                            // [2]
  uint64_t* drain = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* col_exp = reinterpret_cast<int*>(smem + Lay::kBarOff + kBarBytes);  // [BN]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int MT = (M + BM - 1) / BM, NT = (N + BN - 1) / BN;
  int mt, nt;
  if (col_band) {
    const int band = (int)(blockIdx.x / (unsigned)(kBandN * MT));
    const int rem = (int)(blockIdx.x % (unsigned)(kBandN * MT));
    const int bw = min(kBandN, NT - band * kBandN);
    nt = band * kBandN + rem % bw;
    mt = rem / bw;
  } else {
    const int band = (int)(blockIdx.x / (unsigned)(kBand * NT));
    const int rem = (int)(blockIdx.x % (unsigned)(kBand * NT));
    const int bh = min(kBand, MT - band * kBand);
    mt = band * kBand + rem % bh;
    nt = rem / bh;
  }
  const int m0 = mt * BM, n0 = nt * BN;
  if (epi.skip_tile(m0, n0, M, N)) return;
  if (*reinterpret_cast<volatile int*>(status) != kOk) return;
  const int k0 = (int)blockIdx.y * ksplit;
  const int kb_total = (min(ksplit, K - k0) + BK - 1) / BK;
  const int nch = (kb_total + kCkb - 1) / kCkb;
  const int r0 = kRB ? n0 : m0, s0 = kRB ? m0 : n0;  // first row of the resident / streamed operand
  const CUtensorMap* mR = kRB ? &mB : &mA;
  const CUtensorMap* mS = kRB ? &mA : &mB;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kRSets; ++i) {
      mbar_init(&rfull[i], 1);
      mbar_init(&rempty[i], 1);
    }
    for (int i = 0; i < kRing; ++i) {
      mbar_init(&sfull[i], 1);
      mbar_init(&sempty[i], 1);
    }
    for (int b = 0; b < 3; ++b) mbar_init(&accf[b], 1);
    for (int b = 0; b < 2; ++b) mbar_init(&acce[b], 8);
    mbar_init(drain, 1);
    fence_barrier_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto chunk_kb = [&](int c) { return min(kCkb, kb_total - c * kCkb); };

  if (warp == 0) {
    // ---------------- resident digit sets: both digits of chunk c into set c % kRSets
    if (elect_one()) {
      prefetch_tmap(&mA);
      prefetch_tmap(&mB);
    }
    __syncwarp();
    int c = 0;
    for (; c < nch; ++c) {
      const int set = c % kRSets, use = c / kRSets;
      if (!mbar_wait(&rempty[set], (use & 1) ^ 1, kWaitNs)) {
        if (lane == 0) atomicCAS(status, kOk, kTimeoutEmpty);
        break;
      }
      const int kb = chunk_kb(c);
      if (elect_one()) {
        mbar_arrive_expect_tx(&rfull[set], (uint32_t)(kGridSlices * kb * Lay::kRTile));
        for (int d = 0; d < kGridSlices; ++d)
          for (int j = 0; j < kb; ++j) {
            uint8_t* dst = smem + set * Lay::kRSet + (d * kCkb + j) * Lay::kRTile;
            const int k = k0 + (c * kCkb + j) * BK;
            if (kRB) tma_load_3d(dst, mR, &rfull[set], k, r0, d);
            else al.load(mR, dst, &rfull[set], k, r0, d);
          }
      }
      __syncwarp();
    }
    // before leaving, the sets issued last have landed
    for (int g = (c > kRSets ? c - kRSets : 0); g < c; ++g)
      if (!mbar_wait(&rfull[g % kRSets], (g / kRSets) & 1, kWaitNs) && lane == 0)
        atomicCAS(status, kOk, kTimeoutDrain);
  } else if (warp == 1 || warp == 2) {
    // ---------------- streamed digit sets: digit s of chunk c is set g = 7c + s - 1,
    // ring entry g % kRing; warp 1 issues the even g, warp 2 the odd
    const int mine = warp - 1;
    int g = 0;
    bool ok = true;
    for (int c = 0; c < nch && ok; ++c) {
      const int kb = chunk_kb(c);
      for (int s = 1; s <= kSlices; ++s, ++g) {
        if ((g & 1) != mine) continue;
        const int ent = g % kRing, use = g / kRing;
        if (!mbar_wait(&sempty[ent], (use & 1) ^ 1, kWaitNs)) {
          if (lane == 0) atomicCAS(status, kOk, kTimeoutEmpty);
          ok = false;
          break;
        }
        if (elect_one()) {
          mbar_arrive_expect_tx(&sfull[ent], (uint32_t)(kb * Lay::kSTile));
          for (int j = 0; j < kb; ++j) {
            uint8_t* dst = smem + Lay::kSOff + ent * Lay::kSSet + j * Lay::kSTile;
            const int k = k0 + (c * kCkb + j) * BK;
            if (kRB) al.load(mS, dst, &sfull[ent], k, s0, s - 1);
            else tma_load_3d(dst, mS, &sfull[ent], k, s0, s - 1);
          }
        }
        __syncwarp();
      }
    }
    // this warp's sets among the last kRing issued have landed
    for (int q = (g > kRing ? g - kRing : 0); q < g; ++q)
      if ((q & 1) == mine && !mbar_wait(&sfull[q % kRing], (q / kRing) & 1, kWaitNs) && lane == 0)
        atomicCAS(status, kOk, kTimeoutDrain);
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issue: chunk by chunk, level by level
    const uint32_t idesc = idesc_bf16_f32(BM, BN);
    bool aborted = false, issued = false;
    int p = 0;  // exact phases so far
    for (int c = 0; c < nch && !aborted; ++c) {
      const int set = c % kRSets, kb = chunk_kb(c);
      if (!mbar_wait(&rfull[set], (c / kRSets) & 1, kWaitNs)) {
        if (lane == 0) atomicCAS(status, kOk, kTimeoutFull);
        aborted = true;
        break;
      }
      tc_fence_after();
      const uint32_t rbase = smem_u32(smem + set * Lay::kRSet);
      for (int l = 2; l <= kLowTop && !aborted; ++l) {
        const bool exact = l <= kExactTop;
        const int b = p & 1;
        uint32_t d;
        bool first;
        if (exact) {
          if (!mbar_wait(&acce[b], ((p >> 1) & 1) ^ 1, kWaitNs)) {
            if (lane == 0) atomicCAS(status, kOk, kTimeoutEpi);
            aborted = true;
            break;
          }
          tc_fence_after();
          d = tmem + (uint32_t)(b * BN);
          first = true;
        } else {
          d = tmem + (uint32_t)(2 * BN);
          first = c == 0;
        }
        // digit s = l - 1 of this chunk arrives here (the first level using it)
        if (l - 1 <= kSlices) {
          const int g = c * kSlices + (l - 2);
          if (!mbar_wait(&sfull[g % kRing], (g / kRing) & 1, kWaitNs)) {
            if (lane == 0) atomicCAS(status, kOk, kTimeoutFull);
            aborted = true;
            break;
          }
          tc_fence_after();
        }
        // products (s, r) = (l - 1, 1) and (l - 2, 2)
        for (int r = 1; r <= kGridSlices; ++r) {
          const int s = l - r;
          if (s < 1 || s > kSlices) continue;
          const int g = c * kSlices + (s - 1);
          const uint32_t sbase = smem_u32(smem + Lay::kSOff + (g % kRing) * Lay::kSSet);
          if (elect_one()) {
            for (int j = 0; j < kb; ++j) {
              const uint64_t ds = sdesc_k128(sbase + j * Lay::kSTile);
              const uint64_t dr = sdesc_k128(rbase + ((r - 1) * kCkb + j) * Lay::kRTile);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t da = (kRB ? ds : dr) + (uint64_t)(kk * 2), db = (kRB ? dr : ds) + (uint64_t)(kk * 2);
                mma_bf16(d, da, db, idesc, (first && j == 0 && kk == 0) ? 0u : 1u);
              }
            }
          }
          __syncwarp();
          first = false;
          issued = true;
        }
        if (elect_one()) {
          if (exact) mma_commit(&accf[b]);
          // digit l - 2 served its last product (with r = 2); at level 8 also digit 7
          if (l >= 3) mma_commit(&sempty[(c * kSlices + (l - 3)) % kRing]);
          if (l == kLowTop) {
            mma_commit(&sempty[(c * kSlices + (kSlices - 1)) % kRing]);
            mma_commit(&rempty[set]);
            if (c == nch - 1) mma_commit(&accf[2]);
          }
        }
        __syncwarp();
        if (exact) ++p;
      }
    }
    if (aborted && issued) {
      if (elect_one()) mma_commit(drain);
      __syncwarp();
      if (!mbar_wait(drain, 0, kWaitNs) && lane == 0) atomicCAS(status, kOk, kTimeoutDrain);
      tc_fence_after();
    }
  } else if (warp >= kEpiWarp0) {
    // ---------------- epilogue warps 4..11
    const int quad = warp & 3, half = (warp - kEpiWarp0) >> 2;
    const int row_local = quad * 32 + lane;
    const int col_base = half * kCols;
    long long acc[kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) acc[j] = 0;
    const int row = m0 + row_local;
    const int ei = row < M ? ea[row] : 0;
    {
      const int te = threadIdx.x - 32 * kEpiWarp0;
      if (te < BN) col_exp[te] = n0 + te < N ? eb[n0 + te] : 0;
      named_bar(1, 256);
    }
    // this thread's 48 elements of the level-6..7 integer accumulator: 96 words
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    const uint32_t tw = tmem + lanes + (uint32_t)(3 * BN) + (uint32_t)(2 * col_base);
    {
      uint32_t z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0u;
#pragma unroll
      for (int c = 0; c < kCols / 8; ++c) tmem_st16u(tw + 16 * c, z);
    }
    bool ok = true;
    int p = 0;
    for (int c = 0; c < nch && ok; ++c) {
      for (int l = 2; l <= kExactTop; ++l, ++p) {
        const int b = p & 1;
        if (!mbar_wait(&accf[b], (p >> 1) & 1, kWaitNs * 4)) {
          if (lane == 0) atomicCAS(status, kOk, kTimeoutAccum);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + lanes + (uint32_t)(b * BN + col_base);
        const float up = __int_as_float((127 + 8 * (l - 2)) << 23);  // 2^8(l-2): v up is the phase's integer
        if (l <= kRegTop) {
          const int shift = 8 * (kRegTop - l);
#pragma unroll
          for (int q = 0; q < kCols / 16; ++q) {
            float v[16];
            tmem_ld16(ta + q * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[q * 16 + j] += (long long)exact_int(v[j], up) << shift;
          }
        } else {
          // levels 6..7 in units of 2^-40: the integer scaled by 2^8(7-l)
          const int shift = 8 * (kExactTop - l);
#pragma unroll 1
          for (int q = 0; q < kCols / 16; ++q) {
            float v[16];
            tmem_ld16(ta + q * 16, v);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              uint32_t w[16];
              tmem_ld16u(tw + 32 * q + 16 * hh, w);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                long long t = (long long)(((unsigned long long)w[2 * j + 1] << 32) | w[2 * j]);
                t += (long long)exact_int(v[hh * 8 + j], up) << shift;
                w[2 * j] = (uint32_t)(unsigned long long)t;
                w[2 * j + 1] = (uint32_t)((unsigned long long)t >> 32);
              }
              tmem_st16u(tw + 32 * q + 16 * hh, w);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[b]);
      }
    }
    if (ok && !mbar_wait(&accf[2], 0, kWaitNs * 4)) {
      if (lane == 0) atomicCAS(status, kOk, kTimeoutAccum);
      ok = false;
    }
    if (ok) {
      tc_fence_after();
      // value = 2^(e_i + f_j - 16) (acc 2^-24 + acc67 2^-40 + level 8), the
      // loop rolled with acc[] rotated as in ozaki.h
      const uint32_t ta = tmem + lanes + (uint32_t)(2 * BN + col_base);
#pragma unroll 1
      for (int q = 0; q < kCols / 8; ++q) {
        float v[8];
        tmem_ld8(ta + q * 8, v);
        uint32_t w[16];
        tmem_ld16u(tw + 16 * q, w);
        long long r[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long a67 = (long long)(((unsigned long long)w[2 * j + 1] << 32) | w[2 * j]);
          r[j] = __double_as_longlong(combine_parts(acc[j], a67, v[j], ei + col_exp[col_base + q * 8 + j] - 16));
        }
#pragma unroll
        for (int j = 0; j < kCols - 8; ++j) acc[j] = acc[j + 8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[kCols - 8 + j] = r[j];
      }
      tc_fence_before();
      epi(row_local, col_base, m0, n0, M, N, acc, reinterpret_cast<double*>(smem));
    } else {
      epi.abort();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// kRB: B is the 2-digit operand (its map holds 2 digit planes), A the 7-digit
// one; otherwise the reverse.  Same launch order, K splits and checks as
// ozaki_launch.
template <bool kRB, class ALoad, class Epi>
mgw_status ozaki_mixed_launch(mgw_handle* h, const CUtensorMap& mA, const CUtensorMap& mB, const int* ea,
                              const int* eb, int M, int N, int K, const ALoad& al, const Epi& epi, int* dstatus,
                              const char* what, int nsplit = 1) {
  if (K >= (1 << 24))
    return fail(h, MGW_ERR_UNSUPPORTED, "%s: K = %d too large for the digit-sliced GEMM", what, K);
  using Lay = MixedLayout<kRB>;
  auto kern = ozaki_mixed_kernel<kRB, ALoad, Epi>;
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kSmem);
  MGW_CUDA(h, attr);
  const long MT = (M + BM - 1) / BM, NT = (N + BN - 1) / BN;
  const int ksplit = (int)(split_kblocks(K, nsplit) * BK);
  dim3 grid((unsigned)(MT * NT), (unsigned)split_count(K, nsplit), 1);
  const double rows_a = (double)MT * BM, rows_b = (double)NT * BN;
  const double by_rows = rows_a + (double)((MT + kBand - 1) / kBand) * rows_b;
  const double by_cols = (double)((NT + kBandN - 1) / kBandN) * rows_a + rows_b;
  const int col_band = by_cols < by_rows ? 1 : 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
  }
  kern<<<grid, kThreads, Lay::kSmem, h->stream>>>(mA, mB, ea, eb, M, N, K, col_band, ksplit, al, epi, dstatus);
  mgw_status st = check_launch(h, what);
  if (h->prof) {
    cudaEventRecord(e1, h->stream);
    h->spans.push_back({what, e0, e1});
  }
  return st;
}

}  // namespace oz
}  // namespace mgw
