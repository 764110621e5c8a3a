// FP64-accurate GEMM on the BF16 tensor cores (sm_103a) by exact digit
// slicing (an Ozaki-type scheme written for tcgen05).
//
// Each row r of an FP64 operand X is scaled by 2^-e_r (|X_r| / 2^e_r < 1/2)
// and split into S signed base-256 digits, X_r 2^-e_r = sum_s d_s 2^-8s with
// |d_s| <= 128; the digits are stored as BF16 pre-scaled by 2^-8(s-1), so a
// product of digit arrays s and u carries the factor 2^-8(s+u-2).  Then
//   A B^T = 2^(e_i + f_j - 16) sum_{s,u} (dA_s dB_u^T)
// and every digit product is an integer GEMM that the tensor core
// accumulates EXACTLY in FP32 as long as the running sum stays below 2^24:
// for level l = s + u (l - 1 products) that holds for K chunks of at most
// 1024 / (l - 1).  Levels 2..7 (the top 21 products) are accumulated exactly
// chunk by chunk and flushed into 64-bit integers per element: levels 2..5
// into registers of the epilogue warps, levels 6..7 into the spare half of
// TMEM.  Level S+1 = 8 (7 products, below 2^-56 of the top) accumulates in
// FP32 over the whole K: the tensor core truncates as it accumulates, and
// only this deepest level can afford that.  With S = 7 (28 products) the
// result carries about 53 bits.
//
// CTA: 128 x 96 output tile, 384 threads:
//   warps 0-1  TMA producers (digit tiles of A and B, 3D maps: k, row, digit);
//              warp p owns barrier groups p and p + 2 and fills their slots,
//              taking each group's uses in order (a parity wait is sound only
//              one phase ahead); warp 2 has no role
//   warp 3     TMEM allocation (512 columns) and the MMA issuer
//   warps 4-11 epilogue: warp w reads TMEM lanes 32 (w % 4).., columns
//              48 ((w - 4) / 4)..; each thread owns 48 elements of one row
// TMEM (512 columns): two FP32 accumulators [0,96) and [96,192) alternate
// between phases so the flush of one overlaps the MMAs of the next; columns
// [192,384) hold the level-6..7 integer accumulator (two words per element).
// The tile is 96 wide so that the levels-2..5 integers (48 x int64 per
// thread) fit the register budget of a 384-thread block: twelve warps put
// three on each SM sub-partition, whose 16K registers allow 168 per thread.
// Stage slots (one K block of one digit product: 16 KB of A, 12 KB of B)
// come in groups of two behind one full and one empty barrier, so the MMA
// thread waits once per eight MMAs.  All waits are time-bounded.
//
// Launch: one CTA per output tile in row-band or column-band order (the
// launcher takes the one fetching fewer operand rows), optionally split
// along K (blockIdx.y; the epilogue places each split's partial result), and
// an epilogue may skip tiles it does not need (the lower triangle of a
// symmetric result) before any set-up.
#pragma once

#include "tc_common.h"
#include "mgw_internal.h"

#include <algorithm>

namespace mgw {
namespace oz {

constexpr int BM = 128, BN = 96, BK = 64;
constexpr int kCols = BN / 2;          // output columns per epilogue thread
constexpr int kSlices = 7;
constexpr int kGridSlices = 2;        // digits of a tensor sliced on one fixed-point grid (mixed precision)
constexpr int kExactTop = 7;          // levels 2..7 accumulated exactly
constexpr int kRegTop = 5;            // levels 2..5 in registers, 6..7 in TMEM
constexpr int kThreads = 384;
constexpr int kProducers = 2;   // warps 0..1; warp p fills barrier groups p, p + 2
constexpr int kMmaWarp = 3;
constexpr int kEpiWarp0 = 4;    // warps 4..11 (warp 2 has no role)
static_assert(kThreads / 32 - kEpiWarp0 == 8, "eight epilogue warps, two per TMEM lane quadrant");
constexpr int kStages = 8;     // stage slots (one K block of one digit product each)
constexpr int kGroup = 2;      // slots per full/empty barrier
constexpr int kGroups = kStages / kGroup;
static_assert(kGroups % kProducers == 0, "each barrier group has one producer warp");
constexpr int kBand = 8;       // tile rows per row band of the launch order (L2 reuse)
constexpr int kBandN = 19;     // tile columns per column band: 8 x 19 = 152 CTAs, one wave
constexpr int kTileBytes = BM * BK * 2;  // one A digit tile (16 KB)
constexpr int kTileBytesB = BN * BK * 2; // one B digit tile (12 KB)
constexpr int kStageBytes = kTileBytes + kTileBytesB;
constexpr int kBarBytes = 256;         // mbarriers and the TMEM address
constexpr int kSmemBytes = 1024 + kStages * kStageBytes + kBarBytes + BN * 4;  // + the tile's column exponents
static_assert(kSmemBytes <= 232448, "dynamic shared memory above the 227 KB opt-in limit");
constexpr uint64_t kWaitNs = 2000000000ull;

// W 2^E for a nonzero 64-bit integer W, rounded to the nearest double
// (ties to even), subnormal and overflowing results included, with integer
// operations only.  The significand is taken in units of the result's last
// place 2^u, u = max(p + E - 52, -1074) for the leading bit p of |W|; adding
// it to (u + 1074) 2^52 gives the IEEE pattern of normal and subnormal
// results alike, a rounding carry moving into the exponent field.  There is
// no FP64 instruction here, not even in an untaken branch: the FP64 pipe of
// this part runs at a small fraction of the integer rate (removing an ldexp
// fallback cut the final combine from 35-116k to 35-67k cycles per tile).
__device__ __forceinline__ double i64_ldexp(long long W, int E) {
  const unsigned long long sign = (unsigned long long)(W < 0) << 63;
  const unsigned long long M = W < 0 ? 0ull - (unsigned long long)W : (unsigned long long)W;
  const int p = 63 - __clzll((long long)M);
  const int u = max(p + E - 52, -1074);
  const int r = u - E;  // right shift of M onto the last place, >= p - 52 >= -52
  unsigned long long q;
  if (r <= 0) {
    q = M << -r;
  } else if (r >= 64) {
    q = 0;  // |W| <= 2^63: at most half the last place, ties to the even 0
  } else {
    q = M >> r;
    const unsigned long long rem = M & ((1ull << r) - 1), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  // |E| < 2400 for exponents of FP64 operands, so u + 1074 < 4096 fits the shift
  unsigned long long bits = ((unsigned long long)(u + 1074) << 52) + q;
  if ((bits >> 52) >= 2047) bits = 0x7FF0000000000000ull;  // overflow to infinity
  return __longlong_as_double((long long)(bits | sign));
}

// (acc 2^-24 + a67 2^-40 + v) 2^E as a double, FP64 units untouched.
// hi = acc + floor(a67 / 2^16) carries the value in units of 2^-24
// (|hi| < K 2^39 < 2^63 for K < 2^24); the rest, lo = (a67 mod 2^16) 2^16 +
// round(v 2^56) in units of 2^-56 (|v| < 2^-1), is folded in at the finest
// scale 2^-(24+sh), sh <= 32, that keeps hi 2^sh below 2^62.  When sh < 32
// the result already holds more than 53 bits of hi, so rounding lo to that
// scale moves it by under half a unit of its last place.
// round(v 2^56) for |v| < 2^-1 from the float's fields (ties away from zero)
__device__ __forceinline__ long long f32_fixed56(float v) {
  const unsigned b = __float_as_uint(v);
  const int ex = (int)((b >> 23) & 255);
  const long long m = (long long)((b & 0x7FFFFFu) | (ex ? 0x800000u : 0u));
  const int sh = (ex ? ex : 1) - 150 + 56;  // |v| 2^56 = m 2^sh, sh <= 31
  long long r;
  if (sh >= 0) r = m << sh;
  else if (sh > -26) r = (m >> -sh) + ((m >> (-sh - 1)) & 1);
  else r = 0;
  return (b >> 31) ? -r : r;
}

// (hi + lo 2^-32) 2^Ehi as a double for |hi| < 2^63, |lo| < 2^62: lo is
// folded in at the finest scale 2^(Ehi - sh), sh <= 32, that keeps hi 2^sh
// below 2^62 (see combine_parts)
__device__ __forceinline__ double hi_lo_to_double(long long hi, long long lo, int Ehi) {
  const unsigned long long ah = hi < 0 ? 0ull - (unsigned long long)hi : (unsigned long long)hi;
  int sh = ah ? __clzll((long long)ah) - 2 : 32;
  sh = sh > 32 ? 32 : (sh < 0 ? 0 : sh);
  const long long W = (long long)((unsigned long long)hi << sh) +
                      ((lo + (sh < 32 ? (1ll << (31 - sh)) : 0)) >> (32 - sh));
  if (W == 0) return 0.0;
  return i64_ldexp(W, Ehi - sh);
}
__device__ __forceinline__ double combine_parts(long long acc, long long a67, float v, int E) {
  return hi_lo_to_double(acc + (a67 >> 16), ((a67 & 0xFFFF) << 16) + f32_fixed56(v), E - 24);
}

// The operands may carry different digit counts: SA digits for A, SB for B
// (SA, SB <= 7).  Level l = s + u then holds the products s <= SA, u <= SB;
// levels above kLowTop = 8 are dropped (below 2^-64 of the top), so with
// SA = SB = 7 there are 28 products and with one operand on two digits 13.
constexpr int kLowTop = kSlices + 1;
__host__ __device__ constexpr int level_lo(int l, int SB) { return l - SB > 1 ? l - SB : 1; }
__host__ __device__ constexpr int level_hi(int l, int SA) { return SA < l - 1 ? SA : l - 1; }
__host__ __device__ constexpr int level_products(int l, int SA, int SB) {
  return level_hi(l, SA) >= level_lo(l, SB) ? level_hi(l, SA) - level_lo(l, SB) + 1 : 0;
}
__host__ __device__ constexpr int digit_products(int SA, int SB) {
  int n = 0;
  for (int l = 2; l <= kLowTop; ++l) n += level_products(l, SA, SB);
  return n;
}
// K chunk (multiple of BK) over which an exact level's FP32 sum stays below
// 2^24: np products of two digits of magnitude <= 2^7 per k
__host__ __device__ inline int chunk_of_level(int l, int SA, int SB) {
  int c = 1024 / level_products(l, SA, SB);
  return (c / BK) * BK;
}

// Walks the (phase, product, K block) sequence every role follows.  A phase
// is one exact level over one K chunk, or (last) all low levels over all K.
template <int SA, int SB>
struct Schedule {
  static_assert(SA >= 1 && SB >= 1 && SA <= kSlices && SB <= kSlices, "1..7 digits per operand");
  static_assert(SA + SB >= kLowTop, "every level 2..8 holds at least one product");
  int K;
  int kb_total;
  __device__ Schedule(int K_) : K(K_), kb_total((K_ + BK - 1) / BK) {}
  // calls f(phase, is_last, level_for_exact_or_0, s, u, kb, first_mma_of_phase, last_item_of_phase)
  template <class F>
  __device__ void run(F&& f) const {
    int phase = 0;
    for (int l = 2; l <= kExactTop; ++l) {
      const int cb = chunk_of_level(l, SA, SB) / BK;
      for (int c0 = 0; c0 < kb_total; c0 += cb) {
        const int c1 = min(kb_total, c0 + cb);
        const int s_lo = level_lo(l, SB), s_hi = level_hi(l, SA);
        bool first = true;
        for (int s = s_lo; s <= s_hi; ++s)
          for (int kb = c0; kb < c1; ++kb) {
            const bool last = (s == s_hi) && (kb == c1 - 1);
            if (!f(phase, false, l, s, l - s, kb, first, last)) return;
            first = false;
          }
        ++phase;
      }
    }
    bool first = true;
    for (int l = kExactTop + 1; l <= kLowTop; ++l) {
      const int s_lo = level_lo(l, SB), s_hi = level_hi(l, SA);
      for (int s = s_lo; s <= s_hi; ++s)
        for (int kb = 0; kb < kb_total; ++kb) {
          const bool last = (l == kLowTop) && (s == s_hi) && (kb == kb_total - 1);
          if (!f(phase, true, 0, s, l - s, kb, first, last)) return;
          first = false;
        }
    }
  }
  __device__ int items() const { return digit_products(SA, SB) * kb_total; }
  __device__ int phases() const {
    int p = 0;
    for (int l = 2; l <= kExactTop; ++l) {
      const int cb = chunk_of_level(l, SA, SB) / BK;
      p += (kb_total + cb - 1) / cb;
    }
    return p + 1;
  }
};

// Row loader of the A digit tiles: 2D rows (row0 = tile row) or the grouped
// moment rows of the Sigma Y stage (all nmom orders of PB aux rows).
struct ARowsPlain {
  __device__ void load(const CUtensorMap* m, void* dst, uint64_t* bar, int k, int row0, int digit) const {
    tc::tma_load_3d(dst, m, bar, k, row0, digit);
  }
};

template <int SA, int SB, class ALoad, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                  const int* __restrict__ ea, const int* __restrict__ eb, int M, int N, int K, int col_band,
                  int ksplit, ALoad al, Epi epi,
                  int* status) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);  // [kGroups]
  uint64_t* empty = full + kGroups;
  uint64_t* accf = empty + kGroups;  // [2] accumulator b ready for the epilogue
  uint64_t* acce = accf + 2;         // [2] accumulator b drained by the epilogue
  uint64_t* drain = acce + 2;        // MMAs issued before an abort have completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* col_exp = reinterpret_cast<int*>(smem + kStages * kStageBytes + kBarBytes);  // [BN]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // banded tile order.  Row bands: kBand tile rows sweep the tile columns
  // together, the band's A digit tiles stay in L2 and B streams once per band.
  // Column bands: kBandN tile columns sweep the tile rows, every wave re-touches
  // the band's B tiles (they stay in L2) and A streams once per band.
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
  // tiles the epilogue does not need (the lower triangle of a symmetric
  // result) end here, before any barrier, TMEM or shared-memory set-up
  if (epi.skip_tile(m0, n0, M, N, BN)) return;
  // a wait of an earlier CTA (or launch on this status word) gave up: the
  // result is void, so do no set-up and no work (a failing launch then ends
  // within one wave instead of every CTA waiting out its own limits)
  if (*reinterpret_cast<volatile int*>(status) != kOk) return;
  // split z = blockIdx.y covers k in [k0, k0 + ksplit); its partial result
  // goes where the epilogue puts split z
  const int k0 = (int)blockIdx.y * ksplit;
  const Schedule<SA, SB> sched(min(ksplit, K - k0));

  if (threadIdx.x == 0) {
    for (int g = 0; g < kGroups; ++g) {
      mbar_init(&full[g], 1);
      mbar_init(&empty[g], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 8);
    }
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

  if (warp < kProducers) {
    // the whole warp walks the schedule; one elected lane issues
    if (warp == 0 && elect_one()) {
      prefetch_tmap(&mA);
      prefetch_tmap(&mB);
    }
    __syncwarp();
    // stage slots come in groups of kGroup behind one full and one empty
    // barrier; group g uses barrier pair g % kGroups and is issued by the
    // producer that owns that pair, which takes its pairs' uses in order
    // (a parity wait is sound only one phase ahead)
    const int total = sched.items();
    int it = 0;
    sched.run([&](int, bool, int, int s, int u, int kb, bool, bool) {
      const int g = it / kGroup, gs = g % kGroups;
      if (gs % kProducers == warp) {
        if (it % kGroup == 0) {
          if (!mbar_wait(&empty[gs], ((g / kGroups) & 1) ^ 1, kWaitNs)) {
            if (lane == 0) atomicCAS(status, kOk, kTimeoutEmpty);
            return false;
          }
        }
        if (elect_one()) {
          if (it % kGroup == 0)
            mbar_arrive_expect_tx(&full[gs], (uint32_t)(min(kGroup, total - g * kGroup) * kStageBytes));
          uint8_t* sa = smem + (it % kStages) * kStageBytes;
          al.load(&mA, sa, &full[gs], k0 + kb * BK, m0, s - 1);
          tma_load_3d(sa + kTileBytes, &mB, &full[gs], k0 + kb * BK, n0, u - 1);
        }
        __syncwarp();
      }
      ++it;
      return true;
    });
    // before leaving, this producer's groups among the last kGroups have landed
    // (no copy may still write into this CTA's shared memory once it exits)
    const int ng = (it + kGroup - 1) / kGroup;
    for (int g = (ng > kGroups ? ng - kGroups : 0); g < ng; ++g)
      if ((g % kGroups) % kProducers == warp && !mbar_wait(&full[g % kGroups], (g / kGroups) & 1, kWaitNs) &&
          lane == 0)
        atomicCAS(status, kOk, kTimeoutDrain);
  } else if (warp == kMmaWarp) {
    // the whole warp walks the schedule and waits; one elected lane issues
    const uint32_t idesc = idesc_bf16_f32(BM, BN);
    const int total = sched.items();
    int it = 0;
    bool aborted = false;
    sched.run([&](int phase, bool, int, int, int, int, bool first, bool last) {
      const int b = phase & 1, use = phase >> 1;
      if (first) {
        if (!mbar_wait(&acce[b], (use & 1) ^ 1, kWaitNs)) {
          if (lane == 0) atomicCAS(status, kOk, kTimeoutEpi);
          aborted = true;
          return false;
        }
        tc_fence_after();
      }
      // one wait per group of kGroup slots
      const int g = it / kGroup, gs = g % kGroups;
      if (it % kGroup == 0) {
        if (!mbar_wait(&full[gs], (g / kGroups) & 1, kWaitNs)) {
          if (lane == 0) atomicCAS(status, kOk, kTimeoutFull);
          aborted = true;
          return false;
        }
        tc_fence_after();
      }
      const int st = it % kStages;
      const uint32_t sa = smem_u32(smem + st * kStageBytes);
      const uint64_t da = sdesc_k128(sa), db = sdesc_k128(sa + kTileBytes);
      const uint32_t d = tmem + (uint32_t)(b * BN);
      if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          mma_bf16(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (first && kk == 0) ? 0u : 1u);
        if (it % kGroup == kGroup - 1 || it == total - 1) mma_commit(&empty[gs]);
        if (last) mma_commit(&accf[b]);
      }
      __syncwarp();
      ++it;
      return true;
    });
    // after an abort the MMAs already issued must finish before TMEM is freed
    if (aborted && it > 0) {
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
    // the tile's column exponents, read once here: a global load per element
    // in the final combine would wait on L2 while the other SMs stream digit
    // tiles through it
    {
      const int te = threadIdx.x - 32 * kEpiWarp0;
      if (te < BN) col_exp[te] = n0 + te < N ? eb[n0 + te] : 0;
      named_bar(1, 256);
    }
    // this thread's 48 elements of the level-6..7 integer accumulator: 96 words
    const uint32_t tw = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(2 * BN) + (uint32_t)(2 * col_base);
    {
      uint32_t z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0u;
#pragma unroll
      for (int c = 0; c < kCols / 8; ++c) tmem_st16u(tw + 16 * c, z);
    }
    bool ok = true;
    const int nph = sched.phases();
    int l_of_phase = 2, chunk_idx = 0;
    for (int phase = 0; phase < nph && ok; ++phase) {
      const int b = phase & 1, use = phase >> 1;
      const bool is_low = phase == nph - 1;
      if (!mbar_wait(&accf[b], use & 1, kWaitNs * 4)) {
        if (lane == 0) atomicCAS(status, kOk, kTimeoutAccum);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * BN + col_base);
      if (!is_low) {
        // level of this phase, walking the same chunking as Schedule
        const int l = l_of_phase;
        if (l <= kRegTop) {
          const float up = (float)(1 << (8 * (l - 2)));   // v * 2^8(l-2) is an integer
          const int shift = 8 * (kRegTop - l);
#pragma unroll
          for (int c = 0; c < kCols / 16; ++c) {
            float v[16];
            tmem_ld16(ta + c * 16, v);
#pragma unroll
            for (int j = 0; j < 16; ++j)
              acc[c * 16 + j] += (long long)__float2int_rn(v[j] * up) << shift;
          }
        } else {
          // levels 6..7 in units of 2^-40 (d~ units): I_l = v 2^8(l-2), scaled by 2^8(7-l)
          const float up = l == 6 ? 0x1p32f : 0x1p40f;
          const int shift = 8 * (kExactTop - l);
#pragma unroll 1
          for (int c = 0; c < kCols / 16; ++c) {  // 16 elements (32 words) at a time
            float v[16];
            tmem_ld16(ta + c * 16, v);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              uint32_t w[16];
              tmem_ld16u(tw + 32 * c + 16 * hh, w);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                long long t = (long long)(((unsigned long long)w[2 * j + 1] << 32) | w[2 * j]);
                t += (long long)__float2int_rn(v[hh * 8 + j] * up) << shift;
                w[2 * j] = (uint32_t)(unsigned long long)t;
                w[2 * j + 1] = (uint32_t)((unsigned long long)t >> 32);
              }
              tmem_st16u(tw + 32 * c + 16 * hh, w);
            }
          }
        }
        const int cbl = chunk_of_level(l, SA, SB) / BK;
        const int nchunks = (sched.kb_total + cbl - 1) / cbl;
        if (++chunk_idx == nchunks) { chunk_idx = 0; ++l_of_phase; }
      } else {
        // last phase: value = 2^(e_i + f_j - 16) (acc 2^-24 + acc67 2^-40 + low).
        // This runs once per tile, long after the code was last fetched, so the
        // loop over groups of 8 elements stays rolled: fully unrolled, 48
        // inlined combines made it wait on instruction fetches from L2.  acc[]
        // rotates by 8 per group, so every group reads acc[0..7] (register
        // indices stay static) and the results end in element order.
#pragma unroll 1
        for (int c = 0; c < kCols / 8; ++c) {
          float v[8];
          tmem_ld8(ta + c * 8, v);
          uint32_t w[16];
          tmem_ld16u(tw + 16 * c, w);
          long long r[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long long a67 = (long long)(((unsigned long long)w[2 * j + 1] << 32) | w[2 * j]);
            r[j] = __double_as_longlong(combine_parts(acc[j], a67, v[j], ei + col_exp[col_base + c * 8 + j] - 16));
          }
#pragma unroll
          for (int j = 0; j < kCols - 8; ++j) acc[j] = acc[j + 8];
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[kCols - 8 + j] = r[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
    if (ok) {
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

// ---- host side

struct Sliced {  // digits [ns][rows][ld] BF16 + exponents [rows] + row maxima scratch [rows]
  void* digits = nullptr;
  int* exps = nullptr;
  unsigned long long* rmax = nullptr;
  long rows = 0, ld = 0;
  int ns = kSlices;  // digits per element
};

// slice a row-major FP64 matrix X[rows][K] (row stride lds) -> digits, exponents
mgw_status slice_rows(mgw_handle* h, long rows, long K, const double* X, long lds, Sliced& out);
// the same on the tensor's grid (two digits, exponent *gexp for every row)
mgw_status slice_rows_grid(mgw_handle* h, long rows, long K, const double* X, long lds, const int* gexp,
                           Sliced& out);
// slice the stacked moments W[nmom][naux][naux] into grouped rows: result row
// R = g*128 + t*PB + pl holds W[t][g*PB + pl][:] (zero past nmom*PB or naux)
mgw_status slice_grouped(mgw_handle* h, int nmom, int PB, int naux, const double* W, Sliced& out);
// slice the transpose: rows r of the result are columns of X: Y[r][k] = X[k * ldx + r]
mgw_status slice_cols(mgw_handle* h, long rows, long K, const double* X, long ldx, Sliced& out);
// slice a gathered matrix: element (r, k) = X[roff(r) + koff(k)] with
// roff(r) = (r / rdiv) rhi + (r % rdiv) rlo, koff(k) = (k / kdiv) khi + (k % kdiv) klo;
// CTAs take 32 consecutive rows, so rlo = 1 keeps the reads coalesced
struct Gather { long rdiv, rhi, rlo, kdiv, khi, klo; };
mgw_status slice_gather(mgw_handle* h, long rows, long K, const double* X, const Gather& g, Sliced& out);
// workspace for rows x K elements of ns digits + exponents
size_t sliced_doubles(long rows, long K, int ns = kSlices);
void place_sliced(double* mem, long rows, long K, Sliced& s, int ns = kSlices);
// Fixed-point slicing on one grid for a whole tensor (two digits, the BF16
// hi/lo split of the mixed precision): ex = the exponent with |x| 2^-ex < 1/2
// for every element, each element rounded to a multiple of 2^(ex-16) and
// written as two balanced base-256 digits, every row exponent set to ex.
// The rounded tensor is the same whatever rows and K the slicing takes, so
// every product of the path sees one tensor.  global_exponent computes ex
// into gexp (device) from the max |x| of n elements.
mgw_status global_exponent(mgw_handle* h, long n, const double* X, unsigned long long* gmax, int* gexp);
mgw_status slice_gather_grid(mgw_handle* h, long rows, long K, const double* X, const Gather& g, const int* gexp,
                             Sliced& out);
// X' = X rounded to that grid (the FP64 values the two digits represent)
mgw_status round_to_grid(mgw_handle* h, long n, const double* X, const int* gexp, double* Xr);
// A tensor already on its grid as 16-bit integers q (value q 2^(e-16)):
// slice a gather of it (two digits, exponent e for every row), read a gather
// of its values, and quantize FP64 values into it (*overflow set when a value
// lies outside the grid's range |x| < 2^(e-1))
mgw_status slice_gather_q(mgw_handle* h, long rows, long K, const short* X, const Gather& g, int e, Sliced& out);
mgw_status dequantize_gather(mgw_handle* h, long rows, long K, const short* X, const Gather& g, int e, double* out);
mgw_status quantize(mgw_handle* h, long n, const double* L, int e, short* Lq, int* overflow);
// 3D tensor map over digits: (k, row, digit), box (64, box_rows, 1)
mgw_status digit_map(mgw_handle* h, CUtensorMap* map, const Sliced& s, int box_rows);

// K blocks per split and the number of splits a launch with nsplit requested
// makes (each split a whole number of BK blocks, none empty)
inline long split_kblocks(long K, int nsplit) {
  const long kb = (K + BK - 1) / BK;
  const long ns = std::max(1L, std::min<long>(nsplit, kb));
  return (kb + ns - 1) / ns;
}
inline int split_count(long K, int nsplit) {
  const long kb = (K + BK - 1) / BK, kbs = split_kblocks(K, nsplit);
  return (int)((kb + kbs - 1) / kbs);
}
// Splits to request for a launch of `kept` tiles: kept tiles x splits should
// fill whole waves of one CTA per SM, and every CTA also pays a fixed set-up
// and final combine of about 3 K blocks' worth of MMA time.  Minimises
// waves x (K blocks per split + 3) over 1..16 splits.
inline int best_split(long kept, long K, int sms) {
  int best = 1;
  double best_cost = 0.0;
  for (int s = 1; s <= 16; ++s) {
    const long waves = (kept * split_count(K, s) + sms - 1) / sms;
    const double cost = (double)waves * ((double)split_kblocks(K, s) + 3.0);
    if (s == 1 || cost < best_cost) {
      best = s;
      best_cost = cost;
    }
  }
  return best;
}
// C [M][N] (ldc) = A [M][K] (lda) B [K][N] (ldb), row-major, as an
// FP64-accurate digit-sliced product (28 products); synchronises to read the
// wait status.  Its digits live in slot buffers, so it may run inside a call
// that holds workspace-arena pointers.
mgw_status gemm_fp64_tc_nn(mgw_handle* h, int M, int N, int K, const double* A, long lda, const double* B, long ldb,
                           double* C, long ldc, const char* what);
// sum of the split buffers: out[i] = (accumulate ? out[i] : 0) + sum_z part[z count + i]
mgw_status reduce_splits(mgw_handle* h, long count, int nsplit, const double* part, double* out, int accumulate);

// SA, SB: digits of A and B (the tensor maps must hold that many planes)
template <int SA = kSlices, int SB = kSlices, class ALoad, class Epi>
mgw_status ozaki_launch(mgw_handle* h, const CUtensorMap& mA, const CUtensorMap& mB, const int* ea,
                        const int* eb, int M, int N, int K, const ALoad& al, const Epi& epi, int* dstatus,
                        const char* what, int nsplit = 1) {
  if (K >= (1 << 24))  // the exact 128-bit combine of the epilogue needs K < 2^24
    return fail(h, MGW_ERR_UNSUPPORTED, "%s: K = %d too large for the digit-sliced GEMM", what, K);
  auto kern = ozaki_gemm_kernel<SA, SB, ALoad, Epi>;
  // once per instantiation (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  MGW_CUDA(h, attr);
  const long MT = (M + BM - 1) / BM, NT = (N + BN - 1) / BN;
  const int ksplit = (int)(split_kblocks(K, nsplit) * BK);
  dim3 grid((unsigned)(MT * NT), (unsigned)split_count(K, nsplit), 1);
  // launch order with the smaller estimate of operand rows fetched from DRAM:
  // the resident operand once, the streamed one once per band
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
  kern<<<grid, kThreads, kSmemBytes, h->stream>>>(mA, mB, ea, eb, M, N, K, col_band, ksplit, al, epi, dstatus);
  mgw_status st = check_launch(h, what);
  if (h->prof) {
    cudaEventRecord(e1, h->stream);
    h->spans.push_back({what, e0, e1});
  }
  return st;
}

}  // namespace oz
}  // namespace mgw

namespace mgw {
namespace oz {

// Per-element epilogue adaptor: f(row, col, value) for every in-range element.
template <class F>
struct EpiElem {
  F f;
  __device__ bool skip_tile(int m0, int n0, int M, int N, int bn) const { return f.skip_tile(m0, n0, M, N, bn); }
  template <int KC>
  __device__ void operator()(int row_local, int col_base, int m0, int n0, int M, int N, const long long (&v)[KC],
                             double*) const {
    const int row = m0 + row_local;
    if (row >= M) return;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      const int col = n0 + col_base + j;
      if (col < N) f(row, col, __longlong_as_double(v[j]));
    }
  }
  __device__ void abort() const {}
};

struct FStore {  // C[row][col] = alpha v + beta C
  double* C; long ldc; double alpha, beta;
  __device__ bool skip_tile(int, int, int, int, int) const { return false; }
  __device__ void operator()(int r, int c, double v) const {
    double* q = C + (long)r * ldc + c;
    *q = beta == 0.0 ? alpha * v : alpha * v + beta * *q;
  }
};
// C = A B^T known to be symmetric (M == N): elements with row <= col write
// (row, col) and (col, row), the rest are dropped, and tiles wholly below the
// diagonal are skipped (the upper element of each pair lies in a kept tile).
// Split z of a K-split launch writes the z-th buffer, split_stride apart.
__host__ __device__ inline bool sym_tile_lower(int m0, int n0, int N, int bn = BN) {
  return (n0 + bn < N ? n0 + bn : N) - 1 < m0;
}
struct FStoreSym {
  double* C; long ldc; long split_stride;
  __device__ bool skip_tile(int m0, int n0, int, int N, int bn) const { return sym_tile_lower(m0, n0, N, bn); }
  __device__ void operator()(int r, int c, double v) const {
    if (r > c) return;
    double* base = C + (long)blockIdx.y * split_stride;
    base[(long)r * ldc + c] = v;
    if (r != c) base[(long)c * ldc + r] = v;
  }
};
struct FDiagUpdate {  // T[row][col] = T d[col] + alpha v
  double* T; long ldt; const double* d; double alpha;
  __device__ bool skip_tile(int, int, int, int, int) const { return false; }
  __device__ void operator()(int r, int c, double v) const {
    double* q = T + (long)r * ldt + c;
    *q = *q * d[c] + alpha * v;
  }
};
// Sigma(n) = A B^T with rows p and columns (n, q): a symmetric result in (p, q).
// Elements with p <= q write (p, q) and (q, p); the rest are dropped, and a
// tile whose every column has q below its first row is skipped outright (the
// upper element of each pair lies in a kept tile).  Split z of a K-split
// launch writes the z-th buffer, split_stride doubles apart.
__host__ __device__ inline bool sigma_tile_lower(int m0, int n0, int N, int nmo, int bn = BN) {
  const int c1 = (n0 + bn < N ? n0 + bn : N) - 1;
  return n0 / nmo == c1 / nmo && c1 % nmo < m0;
}
struct FSigmaN {
  double* sig; int nmo; double beta; long split_stride;
  __device__ bool skip_tile(int m0, int n0, int, int N, int bn) const {
    return sigma_tile_lower(m0, n0, N, nmo, bn);
  }
  __device__ void operator()(int r, int c, double v) const {
    const int n = c / nmo, q = c % nmo;
    if (r > q) return;
    double* base = sig + (long)blockIdx.y * split_stride + (long)n * nmo * nmo;
    double* p = base + (long)r * nmo + q;
    *p = beta == 0.0 ? v : v + *p;
    if (r != q) {
      double* t = base + (long)q * nmo + r;
      *t = beta == 0.0 ? v : v + *t;
    }
  }
};

}  // namespace oz
}  // namespace mgw
