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
// CTA: 128 x 96 output tile, 320 threads:
//   warp 0     TMA producer (digit tiles of A and B, 3D maps: k, row, digit)
//   warp 1     TMEM allocation (512 columns) and the MMA issuer
//   warps 2-9  epilogue: warp w reads TMEM lanes 32 (w % 4).., columns
//              48 ((w - 2) / 4)..; each thread owns 48 elements of one row
// TMEM (512 columns): two FP32 accumulators [0,96) and [96,192) alternate
// between phases so the flush of one overlaps the MMAs of the next; columns
// [192,384) hold the level-6..7 integer accumulator (two words per element).
// The tile is 96 wide so that the levels-2..5 integers (48 x int64 per
// thread) fit the register budget of a 320-thread block: ten warps put three
// on one SM sub-partition, whose 16K registers then allow 168 per thread.
// All waits are time-bounded.
#pragma once

#include "tc_common.h"
#include "mgw_internal.h"

namespace mgw {
namespace oz {

constexpr int BM = 128, BN = 96, BK = 64;
constexpr int kCols = BN / 2;          // output columns per epilogue thread
constexpr int kSlices = 7;
constexpr int kExactTop = 7;          // levels 2..7 accumulated exactly
constexpr int kRegTop = 5;            // levels 2..5 in registers, 6..7 in TMEM
constexpr int kThreads = 320;
constexpr int kStages = 7;
constexpr int kTileBytes = BM * BK * 2;  // one A digit tile (16 KB)
constexpr int kTileBytesB = BN * BK * 2; // one B digit tile (12 KB)
constexpr int kStageBytes = kTileBytes + kTileBytesB;
constexpr int kSmemBytes = 1024 + kStages * kStageBytes + 256;
constexpr uint64_t kWaitNs = 2000000000ull;

__host__ __device__ inline int chunk_of_level(int l) {  // K chunk (multiple of BK) of an exact level
  int c = 1024 / (l - 1);
  return (c / BK) * BK;
}

// Walks the (phase, product, K block) sequence every role follows.  A phase
// is one exact level over one K chunk, or (last) all low levels over all K.
struct Schedule {
  int K;
  int kb_total;
  __device__ Schedule(int K_) : K(K_), kb_total((K_ + BK - 1) / BK) {}
  // calls f(phase, is_last, level_for_exact_or_0, s, u, kb, first_mma_of_phase, last_item_of_phase)
  template <class F>
  __device__ void run(F&& f) const {
    int phase = 0;
    for (int l = 2; l <= kExactTop; ++l) {
      const int cb = chunk_of_level(l) / BK;
      for (int c0 = 0; c0 < kb_total; c0 += cb) {
        const int c1 = min(kb_total, c0 + cb);
        const int s_lo = max(1, l - kSlices), s_hi = min(kSlices, l - 1);
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
    for (int l = kExactTop + 1; l <= kSlices + 1; ++l) {
      const int s_lo = max(1, l - kSlices), s_hi = min(kSlices, l - 1);
      for (int s = s_lo; s <= s_hi; ++s)
        for (int kb = 0; kb < kb_total; ++kb) {
          const bool last = (l == kSlices + 1) && (s == s_hi) && (kb == kb_total - 1);
          if (!f(phase, true, 0, s, l - s, kb, first, last)) return;
          first = false;
        }
    }
  }
  __device__ int phases() const {
    int p = 0;
    for (int l = 2; l <= kExactTop; ++l) {
      const int cb = chunk_of_level(l) / BK;
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

template <class ALoad, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                  const int* __restrict__ ea, const int* __restrict__ eb, int M, int N, int K, ALoad al, Epi epi,
                  int* status) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* accf = empty + kStages;  // [2] accumulator b ready for the epilogue
  uint64_t* acce = accf + 2;         // [2] accumulator b drained by the epilogue
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const Schedule sched(K);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 8);
    }
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_tmap(&mA);
      prefetch_tmap(&mB);
      int it = 0, issued = 0;
      sched.run([&](int, bool, int, int s, int u, int kb, bool, bool) {
        const int st = it % kStages;
        if (!mbar_wait(&empty[st], ((it / kStages) & 1) ^ 1, kWaitNs)) {
          atomicCAS(status, kOk, kTimeoutEmpty);
          return false;
        }
        uint8_t* sa = smem + st * kStageBytes;
        mbar_arrive_expect_tx(&full[st], kStageBytes);
        al.load(&mA, sa, &full[st], kb * BK, m0, s - 1);
        tma_load_3d(sa + kTileBytes, &mB, &full[st], kb * BK, n0, u - 1);
        ++it;
        ++issued;
        return true;
      });
      for (int i = (issued > kStages ? issued - kStages : 0); i < issued; ++i)
        mbar_wait(&full[i % kStages], (i / kStages) & 1, kWaitNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(BM, BN);
      int it = 0;
      sched.run([&](int phase, bool, int, int, int, int, bool first, bool last) {
        const int b = phase & 1, use = phase >> 1;
        if (first) {
          if (!mbar_wait(&acce[b], (use & 1) ^ 1, kWaitNs)) {
            atomicCAS(status, kOk, kTimeoutEpi);
            return false;
          }
          tc_fence_after();
        }
        const int st = it % kStages;
        if (!mbar_wait(&full[st], (it / kStages) & 1, kWaitNs)) {
          atomicCAS(status, kOk, kTimeoutFull);
          return false;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + st * kStageBytes);
        const uint64_t da = sdesc_k128(sa), db = sdesc_k128(sa + kTileBytes);
        const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          mma_bf16(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (first && kk == 0) ? 0u : 1u);
        mma_commit(&empty[st]);
        if (last) mma_commit(&accf[b]);
        ++it;
        return true;
      });
    }
  } else {
    // ---------------- epilogue warps 2..9
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int row_local = quad * 32 + lane;
    const int col_base = half * kCols;
    long long acc[kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) acc[j] = 0;
    const int row = m0 + row_local;
    const int ei = row < M ? ea[row] : 0;
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
          for (int c = 0; c < kCols / 8; ++c) {  // 8 elements (16 words) at a time
            float v[16];
            tmem_ld16(ta + (c >> 1) * 16, v);
            uint32_t w[16];
            tmem_ld16u(tw + 16 * c, w);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              long long t = (long long)(((unsigned long long)w[2 * j + 1] << 32) | w[2 * j]);
              t += (long long)__float2int_rn(v[(c & 1) * 8 + j] * up) << shift;
              w[2 * j] = (uint32_t)(unsigned long long)t;
              w[2 * j + 1] = (uint32_t)((unsigned long long)t >> 32);
            }
            tmem_st16u(tw + 16 * c, w);
          }
        }
        const int nchunks = (sched.kb_total + chunk_of_level(l) / BK - 1) / (chunk_of_level(l) / BK);
        if (++chunk_idx == nchunks) { chunk_idx = 0; ++l_of_phase; }
      } else {
        // last phase: value = 2^(e_i + f_j - 16) (acc 2^-24 + acc67 2^-40 + low), kept in acc's registers
#pragma unroll
        for (int c = 0; c < kCols / 8; ++c) {
          float v[16];
          tmem_ld16(ta + (c >> 1) * 16, v);
          uint32_t w[16];
          tmem_ld16u(tw + 16 * c, w);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int e = c * 8 + j;
            const int col = n0 + col_base + e;
            const int fj = col < N ? eb[col] : 0;
            const long long a67 = (long long)(((unsigned long long)w[2 * j + 1] << 32) | w[2 * j]);
            acc[e] = __double_as_longlong(
                ldexp((double)acc[e] * 0x1p-24 + (double)a67 * 0x1p-40 + (double)v[(c & 1) * 8 + j], ei + fj - 16));
          }
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
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---- host side

struct Sliced {  // digits [kSlices][rows][ld] BF16 + exponents [rows]
  void* digits = nullptr;
  int* exps = nullptr;
  long rows = 0, ld = 0;
};

// slice a row-major FP64 matrix X[rows][K] (row stride lds) -> digits, exponents
mgw_status slice_rows(mgw_handle* h, long rows, long K, const double* X, long lds, Sliced& out);
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
size_t sliced_doubles(long rows, long K);           // workspace for rows x K digits + exponents
void place_sliced(double* mem, long rows, long K, Sliced& s);
// 3D tensor map over digits: (k, row, digit), box (64, box_rows, 1)
mgw_status digit_map(mgw_handle* h, CUtensorMap* map, const Sliced& s, int box_rows);

template <class ALoad, class Epi>
mgw_status ozaki_launch(mgw_handle* h, const CUtensorMap& mA, const CUtensorMap& mB, const int* ea,
                        const int* eb, int M, int N, int K, const ALoad& al, const Epi& epi, int* dstatus,
                        const char* what) {
  auto kern = ozaki_gemm_kernel<ALoad, Epi>;
  static bool attr = false;
  if (!attr) {
    MGW_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    attr = true;
  }
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
  }
  kern<<<grid, kThreads, kSmemBytes, h->stream>>>(mA, mB, ea, eb, M, N, K, al, epi, dstatus);
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
  __device__ void operator()(int row_local, int col_base, int m0, int n0, int M, int N,
                             const long long (&v)[kCols], double*) const {
    const int row = m0 + row_local;
    if (row >= M) return;
#pragma unroll 4
    for (int j = 0; j < kCols; ++j) {
      const int col = n0 + col_base + j;
      if (col < N) f(row, col, __longlong_as_double(v[j]));
    }
  }
  __device__ void abort() const {}
};

struct FStore {  // C[row][col] = alpha v + beta C
  double* C; long ldc; double alpha, beta;
  __device__ void operator()(int r, int c, double v) const {
    double* q = C + (long)r * ldc + c;
    *q = beta == 0.0 ? alpha * v : alpha * v + beta * *q;
  }
};
struct FDiagUpdate {  // T[row][col] = T d[col] + alpha v
  double* T; long ldt; const double* d; double alpha;
  __device__ void operator()(int r, int c, double v) const {
    double* q = T + (long)r * ldt + c;
    *q = *q * d[c] + alpha * v;
  }
};
struct FSigmaN {  // column (n, q): Sigma(n)[row][q] (+)= v
  double* sig; int nmo; double beta;
  __device__ void operator()(int r, int c, double v) const {
    const int n = c / nmo, q = c % nmo;
    double* p = sig + ((long)n * nmo + r) * nmo + q;
    *p = beta == 0.0 ? v : v + *p;
  }
};

}  // namespace oz
}  // namespace mgw
