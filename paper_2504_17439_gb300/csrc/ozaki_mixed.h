// The digit-sliced tensor-core GEMM of the mixed precision, with digit tiles
// reused across products and one TMEM accumulator per level.
//
// One operand carries 2 digits on a fixed-point grid (the DF tensor, see
// MGW_MIXED), the other 7 per-row digits; the products kept are the 13 with
// s + r <= 8 (streamed digit s, resident digit r).  The K loop runs in chunks
// of kCkb K blocks, and inside a chunk level by level (l = 2..8): the
// 2-digit ("resident") operand of the chunk is loaded once and serves all 13
// products, and each digit s of the 7-digit ("streamed") operand is loaded
// once and serves levels s + 1 and s + 2.  Per K block the copies are 7
// streamed + 2 resident tiles instead of 13 (A + B) pairs.
//
// Accumulation.  Every exact level has its own FP32 accumulator in TMEM.  A
// term of level l is an integer of magnitude <= 2^14 times
// 2^-8(l-2) (two digits of magnitude <= 2^7), so a chunk adds at most
// 2 products x 128 terms x 2^14 = 2^22 such units to a level (2^21 to level
// 2, which has one product).  The exact levels 2..6 therefore accumulate over
// a window of 4 chunks (8 for level 2) with every partial sum an integer
// multiple of the level's unit of magnitude <= 2^24 units, exact in FP32; at
// the end of a window the epilogue warps convert the sum to an integer and
// add it, in units of level 6 (2^-32), to one 64-bit integer per output
// element while the MMAs run on.  The windows of levels 3..6 are staggered
// by one chunk each, so a chunk ends 1.125 windows on average (a flush of
// every level at every chunk would put six rounds of the epilogue's integer
// adds on the MMA's critical path).
// Levels 7 and 8 (below 2^-40 of the top; the digits carry their scales, so
// the two levels add up in one accumulator) accumulate in FP32 over all of
// K: one rounding of at most 2^-24 of a partial sum below 2^-25 K of the top
// unit per MMA.  The final value is the 64-bit sum plus that FP32 sum, rounded
// once.  K per launch split stays <= kMixedMaxK so that the 64-bit sum (level
// 2 alone reaches 2^14 K 2^32) cannot overflow.
//
// Tile width.  Six accumulators of 64 columns (384 of the 512 TMEM columns,
// each starting on a multiple of 64) make the tile 128 x 64.
//
// CTA (384 threads): warp 0 loads the resident digit sets (two chunks in
// flight), warps 1-2 the streamed ones (a ring of Lay::kRing digit sets, warp
// 1 the even ones, warp 2 the odd), warp 3 allocates TMEM (512 columns) and
// issues the MMAs, warps 4-11 are the epilogue (each owns 32 columns of one
// row).  All waits are time-bounded.
#pragma once

#include "ozaki.h"

namespace mgw {
namespace oz {

constexpr int kMBN = 64;              // tile columns
constexpr int kMCols = kMBN / 2;      // output columns per epilogue thread
constexpr int kTailA = 5 * kMBN;      // TMEM columns of the two FP32 tail accumulators (levels 7-8)
constexpr int kTailB = 6 * kMBN;
constexpr int kCkb = 2;               // K blocks per chunk
constexpr int kRSets = 2;             // resident digit sets (chunks) in flight
constexpr int kWinTop = 6;            // levels 2..6 exact, in windows of chunks
constexpr int kWinLevels = kWinTop - 1;
constexpr long kMixedMaxK = 1L << 16;  // K per launch split: |sum| < 2^14 K 2^32 (1 + 2^-7) < 2^63

// window of an exact level: 8 chunks for level 2 (one product), 4 for 3..6,
// the ends of levels 3..6 staggered so that one of them ends at every chunk
__host__ __device__ __forceinline__ bool window_end(int c, int l, int nch) {
  if (c == nch - 1) return true;
  return l == 2 ? (c & 7) == 7 : ((c + l - 3) & 3) == 3;
}

// TMEM column of level l's accumulator: the exact levels 2..6 one each,
// level 7 the first tail accumulator, level 8 the second
__host__ __device__ __forceinline__ int acc_col(int l) {
  return l <= kWinTop ? (l - 2) * kMBN : (l == kWinTop + 1 ? kTailA : kTailB);
}

// kRB: B is the resident (2-digit) operand and A streams (7 digits); else A
// is resident and B streams.
template <bool kRB>
struct MixedLayout {
  static constexpr int kRRows = kRB ? kMBN : BM, kSRows = kRB ? BM : kMBN;
  static constexpr int kRTile = kRRows * BK * 2, kSTile = kSRows * BK * 2;
  static constexpr int kRSet = kGridSlices * kCkb * kRTile;  // both digits of one chunk
  static constexpr int kSSet = kCkb * kSTile;               // one digit of one chunk
  static constexpr int kSOff = kRSets * kRSet;
  static constexpr int kTail = 1024 + kBarBytes + kMBN * 4;  // alignment slack, barriers, column exponents
  static constexpr int kRingFit = (232448 - kTail - kSOff) / kSSet;
  static constexpr int kRing = kRingFit > 8 ? 8 : kRingFit;  // streamed digit sets in flight
  static constexpr int kBarOff = kSOff + kRing * kSSet;
  static constexpr int kSmem = kBarOff + kTail;
  static_assert(kRing >= 3, "the streamed ring needs three sets to overlap loads with two levels of MMAs");
  static_assert(kSmem <= 232448, "dynamic shared memory above the 227 KB opt-in limit");
  static_assert(kRTile % 1024 == 0 && kSTile % 1024 == 0, "tiles on 1024-byte swizzle atoms");
  static_assert(kBarOff >= BM * (kMBN + 1) * 8, "the epilogue's staging tile fits in the operand buffers");
  static_assert((2 * kRSets + 2 * kRing + 2 * kWinLevels + 2) * 8 + 4 <= kBarBytes, "barriers fit");
  static_assert(kMCols == 32 && kMBN % 64 == 0, "32-column TMEM loads, accumulators on 64-column boundaries");
};

// the 64-bit sum (units 2^-32 of the top) plus the two FP32 tail sums of
// levels 7 and 8 (multiples of 2^-48, so exact in units of 2^-64), times 2^E
__device__ __forceinline__ double combine_windowed(long long acc, float ta, float tb, int E) {
  return hi_lo_to_double(acc, __float2ll_rn(ta * 0x1p64f) + __float2ll_rn(tb * 0x1p64f), E - 32);
}

// a window sum of level l (v 2^8(l-2) is its integer), added in units of level 6
template <int L>
__device__ __forceinline__ void add_window(long long (&acc)[kMCols], const uint32_t (&w)[kMCols]) {
  constexpr float up = (float)(1ull << (8 * (L - 2)));
  constexpr long long scale = 1ll << (8 * (kWinTop - L));
#pragma unroll
  for (int j = 0; j < kMCols; ++j) acc[j] += (long long)__float2int_rn(__uint_as_float(w[j]) * up) * scale;
}

// The MMAs of one streamed digit over the KB K blocks of a chunk, unrolled,
// every descriptor computed before the first MMA: the tensor pipe takes the
// next MMA only when the issuing thread reaches it, so the thread runs the
// MMAs back to back.  pair: the products (s, 1) into d1 and (s, 2) into d2
// per K slice, the first of each accumulator with a1 / a2 (0: overwrite);
// otherwise (digit 7) the single product alternating between the two tail
// accumulators.
template <bool kRB, class Lay, int KB>
__device__ __forceinline__ void issue_digit(bool pair, uint32_t d1, uint32_t d2, uint32_t tmem, uint32_t slo,
                                            uint32_t rlo, uint32_t idesc, uint32_t a1, uint32_t a2) {
  using namespace tc;
  constexpr uint32_t kS = Lay::kSTile >> 4, kR = Lay::kRTile >> 4;  // tile strides in descriptor units
  constexpr int kSteps = KB * (BK / 16);
  if (pair) {
#pragma unroll
    for (int t = 0; t < kSteps; ++t) {
      const uint32_t j = (uint32_t)(t / (BK / 16)), o = (uint32_t)((t % (BK / 16)) * 2);
      const uint64_t ds = sdesc_join(slo + j * kS + o);
      const uint64_t dr1 = sdesc_join(rlo + j * kR + o), dr2 = sdesc_join(rlo + (kCkb + j) * kR + o);
      const uint32_t f1 = t == 0 ? a1 : 1u, f2 = t == 0 ? a2 : 1u;
      // (s, 2) first: the run then ends on d1 = level s + 1 and the next
      // digit starts on level s + 3, never on the accumulator just written
      if (kRB) {
        mma_bf16_fill(d2, ds, dr2, idesc, f2);
        mma_bf16_lastuse(d1, ds, dr1, idesc, f1);
      } else {
        mma_bf16(d2, dr2, ds, idesc, f2);
        mma_bf16(d1, dr1, ds, idesc, f1);
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < kSteps; ++t) {
      const uint32_t j = (uint32_t)(t / (BK / 16)), o = (uint32_t)((t % (BK / 16)) * 2);
      const uint64_t ds = sdesc_join(slo + j * kS + o), dr1 = sdesc_join(rlo + j * kR + o);
      const uint32_t dt = tmem + (uint32_t)(t & 1 ? kTailA : kTailB);  // digit 6 ended on tail A
      if (kRB) mma_bf16(dt, ds, dr1, idesc, 1u);
      else mma_bf16(dt, dr1, ds, idesc, 1u);
    }
  }
}

// One tile of the product: `tile` is the tile's index in the launch order
// (row or column bands), k0 / ksplit the K range.  The tensor maps may sit in
// the kernel's parameters or in global memory (grouped launches).
template <bool kRB, class ALoad, class Epi>
__device__ __forceinline__ void mixed_tile(const CUtensorMap* pA, const CUtensorMap* pB, const int* __restrict__ ea,
                                           const int* __restrict__ eb, int M, int N, int K, long tile, int col_band,
                                           int k0, int ksplit, const ALoad& al, const Epi& epi, int* status) {
  using namespace tc;
  using Lay = MixedLayout<kRB>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* rfull = reinterpret_cast<uint64_t*>(smem + Lay::kBarOff);  // [kRSets]
  uint64_t* rempty = rfull + kRSets;                                    // [kRSets]
  uint64_t* sfull = rempty + kRSets;                                    // [kRing]
  uint64_t* sempty = sfull + Lay::kRing;                                // [kRing]
  uint64_t* accf = sempty + Lay::kRing;    // [kWinLevels + 1]: a window sum of level 2..6; levels 7-8 done
  uint64_t* acce = accf + kWinLevels + 1;  // [kWinLevels]: a window sum has been read
  uint64_t* drain = acce + kWinLevels;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* col_exp = reinterpret_cast<int*>(smem + Lay::kBarOff + kBarBytes);  // [kMBN]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int MT = (M + BM - 1) / BM, NT = (N + kMBN - 1) / kMBN;
  int mt, nt;
  if (col_band) {
    const int band = (int)(tile / (kBandN * (long)MT));
    const int rem = (int)(tile % (kBandN * (long)MT));
    const int bw = min(kBandN, NT - band * kBandN);
    nt = band * kBandN + rem % bw;
    mt = rem / bw;
  } else {
    const int band = (int)(tile / (kBand * (long)NT));
    const int rem = (int)(tile % (kBand * (long)NT));
    const int bh = min(kBand, MT - band * kBand);
    mt = band * kBand + rem % bh;
    nt = rem / bh;
  }
  const int m0 = mt * BM, n0 = nt * kMBN;
  if (epi.skip_tile(m0, n0, M, N, kMBN)) return;
  if (*reinterpret_cast<volatile int*>(status) != kOk) return;
  const int kb_total = (min(ksplit, K - k0) + BK - 1) / BK;
  const int nch = (kb_total + kCkb - 1) / kCkb;
  const int r0 = kRB ? n0 : m0, s0 = kRB ? m0 : n0;  // first row of the resident / streamed operand
  const CUtensorMap* mR = kRB ? pB : pA;
  const CUtensorMap* mS = kRB ? pA : pB;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kRSets; ++i) {
      mbar_init(&rfull[i], 1);
      mbar_init(&rempty[i], 1);
    }
    for (int i = 0; i < Lay::kRing; ++i) {
      mbar_init(&sfull[i], 1);
      mbar_init(&sempty[i], 1);
    }
    for (int b = 0; b <= kWinLevels; ++b) mbar_init(&accf[b], 1);
    for (int b = 0; b < kWinLevels; ++b) mbar_init(&acce[b], 8);
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
      prefetch_tmap(pA);
      prefetch_tmap(pB);
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
        const int ent = g % Lay::kRing, use = g / Lay::kRing;
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
    for (int q = (g > Lay::kRing ? g - Lay::kRing : 0); q < g; ++q)
      if ((q & 1) == mine && !mbar_wait(&sfull[q % Lay::kRing], (q / Lay::kRing) & 1, kWaitNs) && lane == 0)
        atomicCAS(status, kOk, kTimeoutDrain);
  } else if (warp == kMmaWarp) {
    // ---------------- MMA issue: chunk by chunk, digit by digit of the
    // streamed operand.  Digit s takes part in (s, 1) of level s + 1 and
    // (s, 2) of level s + 2; per K slice the two MMAs go to different
    // accumulators, so neither waits for the other's result, and when A is
    // the streamed operand the second one reads A from the collector the
    // first one filled.  Digit 7 has (7, 1) only: its K slices alternate
    // between the two tail accumulators.  After digit s, level s + 1 is
    // complete for the chunk and digit s is free.  The tensor pipe takes the
    // next MMA only when this thread reaches it, so the per-digit work
    // between MMA runs is kept to a barrier test, bit tests and adds: the
    // digit loop is unrolled, window starts and ends are bit masks made once
    // per chunk, and the ring slot advances by one.
    const uint32_t idesc = idesc_bf16_f32(BM, kMBN);
    bool aborted = false, issued = false;
    unsigned rel = 0;  // bit l - 2: parity of the next completion of acce[l - 2]
    int ent = 0;       // ring slot of the next streamed digit, and its phase parity
    uint32_t eph = 0;
    bool ready = false;  // that slot was seen full ahead of time
    const uint32_t sslot0 = sdesc_lo(smem_u32(smem + Lay::kSOff));  // descriptor low word of ring slot 0
    for (int c = 0; c < nch && !aborted; ++c) {
      const int set = c % kRSets, kb = chunk_kb(c);
      if (!mbar_wait(&rfull[set], (c / kRSets) & 1, kWaitNs)) {
        if (lane == 0) atomicCAS(status, kOk, kTimeoutFull);
        aborted = true;
        break;
      }
      tc_fence_after();
      const uint32_t rlo = sdesc_lo(smem_u32(smem + set * Lay::kRSet));
      // bit l - 2: a window of level l starts / ends at this chunk
      unsigned startm = 0, endm = 0;
#pragma unroll
      for (int l = 2; l <= kWinTop; ++l) {
        if (c == 0 || window_end(c - 1, l, nch)) startm |= 1u << (l - 2);
        if (window_end(c, l, nch)) endm |= 1u << (l - 2);
      }
#pragma unroll
      for (int s = 1; s <= kSlices; ++s) {
        // exact levels whose first product of the chunk comes with this
        // digit: level 2 with (1, 1), level s + 2 with (s, 2)
        const unsigned first = (s == 1 ? 1u : 0u) | (s + 2 <= kWinTop ? 1u << s : 0u);
        if (c > 0 && (startm & first)) {
#pragma unroll
          for (int l = 2; l <= kWinTop; ++l) {
            if (!((startm & first) >> (l - 2) & 1u)) continue;
            if (!mbar_wait(&acce[l - 2], (rel >> (l - 2)) & 1u, kWaitNs)) {
              if (lane == 0) atomicCAS(status, kOk, kTimeoutEpi);
              aborted = true;
              break;
            }
            rel ^= 1u << (l - 2);
          }
          if (aborted) break;
          tc_fence_after();
        }
        const bool zero1 = s == 1 && (startm & 1u);
        const bool zero2 = s + 2 <= kWinTop ? ((startm >> s) & 1u) != 0 : (s + 2 <= kLowTop && c == 0);
        if (!ready && !mbar_wait(&sfull[ent], eph, kWaitNs)) {
          if (lane == 0) atomicCAS(status, kOk, kTimeoutFull);
          aborted = true;
          break;
        }
        tc_fence_after();
        // the next digit's slot, tested now so that the answer is back by the
        // time this digit's MMAs are issued
        const int ent_n = ent + 1 == Lay::kRing ? 0 : ent + 1;
        const uint32_t eph_n = ent + 1 == Lay::kRing ? eph ^ 1u : eph;
        const bool ready_n = mbar_test(&sfull[ent_n], eph_n);
        const uint32_t slo = sslot0 + (uint32_t)(ent * (Lay::kSSet >> 4));
        const int l1 = s + 1, l2 = s + 2;
        const uint32_t d1 = tmem + (uint32_t)acc_col(l1), d2 = tmem + (uint32_t)acc_col(l2);
        if (elect_one()) {
          const uint32_t a1 = zero1 ? 0u : 1u, a2 = zero2 ? 0u : 1u;
          if (kb == kCkb)
            issue_digit<kRB, Lay, kCkb>(s < kSlices, d1, d2, tmem, slo, rlo, idesc, a1, a2);
          else
            issue_digit<kRB, Lay, 1>(s < kSlices, d1, d2, tmem, slo, rlo, idesc, a1, a2);
          if (l1 <= kWinTop && ((endm >> (l1 - 2)) & 1u)) mma_commit(&accf[l1 - 2]);
          mma_commit(&sempty[ent]);
          if (s == kSlices) {
            mma_commit(&rempty[set]);
            if (c == nch - 1) mma_commit(&accf[kWinLevels]);
          }
        }
        __syncwarp();
        issued = true;
        ent = ent_n;
        eph = eph_n;
        ready = __all_sync(0xffffffffu, ready_n);
      }
    }
    if (aborted && issued) {
      if (elect_one()) mma_commit(drain);
      __syncwarp();
      if (!mbar_wait(drain, 0, kWaitNs) && lane == 0) atomicCAS(status, kOk, kTimeoutDrain);
      tc_fence_after();
    }
  } else if (warp >= kEpiWarp0) {
    // ---------------- epilogue warps 4..11: tile row quad * 32 + lane,
    // columns half * 32 .. half * 32 + 31
    const int quad = warp & 3, half = (warp - kEpiWarp0) >> 2;
    const int row_local = quad * 32 + lane;
    const int col_base = half * kMCols;
    long long acc[kMCols];
#pragma unroll
    for (int j = 0; j < kMCols; ++j) acc[j] = 0;
    const int row = m0 + row_local;
    const int ei = row < M ? ea[row] : 0;
    {
      const int te = threadIdx.x - 32 * kEpiWarp0;
      if (te < kMBN) col_exp[te] = n0 + te < N ? eb[n0 + te] : 0;
      named_bar(1, 256);
    }
    const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col_base;
    bool ok = true;
    unsigned full = 0;  // bit l - 2: parity of the next completion of accf[l - 2]
    for (int c = 0; c < nch && ok; ++c) {
      for (int l = 2; l <= kWinTop; ++l) {
        if (!window_end(c, l, nch)) continue;
        if (!mbar_wait(&accf[l - 2], (full >> (l - 2)) & 1u, kWaitNs * 4)) {
          if (lane == 0) atomicCAS(status, kOk, kTimeoutAccum);
          ok = false;
          break;
        }
        full ^= 1u << (l - 2);
        tc_fence_after();
        uint32_t w[kMCols];
        tmem_ld32(ta + (uint32_t)((l - 2) * kMBN), w);
        // the accumulator is free for the next window as soon as it is read
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce[l - 2]);
        switch (l) {
          case 2: add_window<2>(acc, w); break;
          case 3: add_window<3>(acc, w); break;
          case 4: add_window<4>(acc, w); break;
          case 5: add_window<5>(acc, w); break;
          default: add_window<6>(acc, w); break;
        }
      }
    }
    if (ok && !mbar_wait(&accf[kWinLevels], 0, kWaitNs * 4)) {
      if (lane == 0) atomicCAS(status, kOk, kTimeoutAccum);
      ok = false;
    }
    if (ok) {
      tc_fence_after();
      // value = 2^(e_i + f_j - 16) (acc 2^-32 + levels 7-8), the loop rolled
      // with acc[] rotated as in ozaki.h
      const uint32_t t7 = ta + (uint32_t)kTailA, t8 = ta + (uint32_t)kTailB;
#pragma unroll 1
      for (int q = 0; q < kMCols / 8; ++q) {
        float fa[8], fb[8];
        tmem_ld8(t7 + q * 8, fa);
        tmem_ld8(t8 + q * 8, fb);
        long long r[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
          r[j] = __double_as_longlong(
              combine_windowed(acc[j], fa[j], fb[j], ei + col_exp[col_base + q * 8 + j] - 16));
#pragma unroll
        for (int j = 0; j < kMCols - 8; ++j) acc[j] = acc[j + 8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[kMCols - 8 + j] = r[j];
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

template <bool kRB, class ALoad, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
ozaki_mixed_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                   const int* __restrict__ ea, const int* __restrict__ eb, int M, int N, int K, int col_band,
                   int ksplit, ALoad al, Epi epi, int* status) {
  mixed_tile<kRB>(&mA, &mB, ea, eb, M, N, K, (long)blockIdx.x, col_band, (int)blockIdx.y * ksplit, ksplit, al, epi,
                  status);
}

// One problem of a grouped launch: its operands' tensor maps (in global
// memory, written before the launch), exponents, sizes, launch order and
// epilogue.  K stays whole (<= kMixedMaxK).
template <class Epi>
struct alignas(64) MixedItem {
  CUtensorMap mA, mB;
  const int* ea;
  const int* eb;
  int M, N, K, col_band;
  Epi epi;
};

// Many independent products of one kind in one launch: CTA x finds its
// problem b by bisection of the tile prefix sums (start[b] <= x <
// start[b + 1]) and runs that problem's tile x - start[b].
template <bool kRB, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
ozaki_mixed_grouped_kernel(const MixedItem<Epi>* __restrict__ items, const long* __restrict__ start, int nitems,
                           int* status) {
  const long x = (long)blockIdx.x;
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  const MixedItem<Epi>* it = items + lo;
  if (threadIdx.x == 0) {  // the maps were written through the generic proxy
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&it->mA) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&it->mB) : "memory");
  }
  __syncthreads();
  const Epi epi = it->epi;
  mixed_tile<kRB>(&it->mA, &it->mB, it->ea, it->eb, it->M, it->N, it->K, x - start[lo], it->col_band, 0, it->K,
                  ARowsPlain{}, epi, status);
}

// splits a launch needs so that K per split stays within kMixedMaxK
inline int mixed_min_split(long K) { return (int)((K + kMixedMaxK - 1) / kMixedMaxK); }

// kRB: B is the 2-digit operand (its map holds 2 digit planes, box kMBN
// rows), A the 7-digit one (box BM rows); otherwise A holds 2 digits (box BM
// rows) and B 7 (box kMBN rows).  Same launch order, K splits and checks as
// ozaki_launch; K per split must not exceed kMixedMaxK.
template <bool kRB, class ALoad, class Epi>
mgw_status ozaki_mixed_launch(mgw_handle* h, const CUtensorMap& mA, const CUtensorMap& mB, const int* ea,
                              const int* eb, int M, int N, int K, const ALoad& al, const Epi& epi, int* dstatus,
                              const char* what, int nsplit = 1) {
  using Lay = MixedLayout<kRB>;
  const long ksplit = split_kblocks(K, nsplit) * BK;
  if (ksplit > kMixedMaxK)
    return fail(h, MGW_ERR_UNSUPPORTED, "%s: K = %d in %d split(s) leaves %ld per split, above %ld", what, K,
                nsplit, ksplit, kMixedMaxK);
  auto kern = ozaki_mixed_kernel<kRB, ALoad, Epi>;
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::kSmem);
  MGW_CUDA(h, attr);
  const long MT = (M + BM - 1) / BM, NT = (N + kMBN - 1) / kMBN;
  dim3 grid((unsigned)(MT * NT), (unsigned)split_count(K, nsplit), 1);
  const double rows_a = (double)MT * BM, rows_b = (double)NT * kMBN;
  const double by_rows = rows_a + (double)((MT + kBand - 1) / kBand) * rows_b;
  const double by_cols = (double)((NT + kBandN - 1) / kBandN) * rows_a + rows_b;
  const int col_band = by_cols < by_rows ? 1 : 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
  }
  kern<<<grid, kThreads, Lay::kSmem, h->stream>>>(mA, mB, ea, eb, M, N, K, col_band, (int)ksplit, al, epi,
                                                   dstatus);
  mgw_status st = check_launch(h, what);
  if (h->prof) {
    cudaEventRecord(e1, h->stream);
    h->spans.push_back({what, e0, e1});
  }
  return st;
}

}  // namespace oz
}  // namespace mgw
