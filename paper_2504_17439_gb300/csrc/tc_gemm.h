// Tensor-core GEMM for sm_103a: D(M x N) = sum over operand pairs of
// A_i(M x K) B_j(N x K)^T, BF16 operands (K-major, TMA-loaded with 128-byte
// swizzle), FP32 accumulation in TMEM, user epilogue on the accumulator.
//
// One CTA computes one 128 x BN tile.  Warp roles (192 threads):
//   warp 0  TMA producer (one lane): fills a STAGES-deep ring of (A, B) tiles
//   warp 1  TMEM allocator and MMA issuer (one lane): 4 x tcgen05.mma (K=16)
//           per 64-wide K block, commits each stage back to the producer
//   warps 2-5 epilogue: tcgen05.ld of 32 TMEM lanes x 16 columns at a time
// The K loop runs over every (pair, K block); the split-precision products
// (hi*hi + hi*lo + lo*hi) therefore accumulate into one FP32 tile.
#pragma once

#include "mgw_internal.h"
#include "tc_common.h"

namespace mgw {
namespace tc {

constexpr int BM = 128, BK = 64;
constexpr int kThreads = 192;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait, then the kernel reports a timeout

struct PairTable {
  int n;           // number of products
  int a[4], b[4];  // indices into the A / B tensor-map arrays
};

template <int BN, int STAGES>
struct SmemLayout {
  static constexpr int kA = BM * BK * 2;   // bytes of one A tile
  static constexpr int kB = BN * BK * 2;   // bytes of one B tile
  static constexpr int kStage = kA + kB;
  static constexpr int kBars = 2 * STAGES + 1;
  static constexpr int kBytes = 1024 /*align slack*/ + STAGES * kStage + kBars * 8 + 16;
};

// Coordinates of a tile: for 2D maps (c0 = k, c1 = row); 3D maps are handled by
// the loader functor, which gets (k, row0) and issues its own copies.
struct Loader2D {
  __device__ void load_a(const CUtensorMap* m, void* dst, uint64_t* bar, int k, int row0) const {
    tma_load_2d(dst, m, bar, k, row0);
  }
  __device__ void load_b(const CUtensorMap* m, void* dst, uint64_t* bar, int k, int row0) const {
    tma_load_2d(dst, m, bar, k, row0);
  }
  static constexpr bool kRowsA3D = false;
};

template <int BN, int STAGES, class Loader, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
               const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
               PairTable pairs, int M, int N, int K, Loader ld, Epi epi, int* status) {
  using L = SmemLayout<BN, STAGES>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * L::kStage);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const int kblocks = (K + BK - 1) / BK;
  const int iters = kblocks * pairs.n;
  constexpr uint32_t kCols = BN < 32 ? 32 : BN;  // TMEM columns (power of two >= 32)

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool abort = false;

  if (warp == 0 && lane == 0) {
    // ---------------- producer
    const CUtensorMap* As[2] = {&mA0, &mA1};
    const CUtensorMap* Bs[2] = {&mB0, &mB1};
    prefetch_tmap(&mA0);
    prefetch_tmap(&mB0);
    int issued = 0;
    for (int it = 0; it < iters; ++it) {
      const int s = it % STAGES;
      const uint32_t par = ((it / STAGES) & 1) ^ 1;
      if (!mbar_wait(&empty[s], par, kWaitNs)) {
        atomicCAS(status, kOk, kTimeoutEmpty);
        abort = true;
        break;
      }
      const int p = it / kblocks, kb = it % kblocks;
      uint8_t* sa = smem + s * L::kStage;
      uint8_t* sb = sa + L::kA;
      mbar_arrive_expect_tx(&full[s], L::kStage);
      ld.load_a(As[pairs.a[p]], sa, &full[s], kb * BK, m0);
      ld.load_b(Bs[pairs.b[p]], sb, &full[s], kb * BK, n0);
      ++issued;
    }
    // every issued copy has landed before the CTA may leave (normally immediate)
    for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
      mbar_wait(&full[it % STAGES], (it / STAGES) & 1, kWaitNs);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16_f32(BM, BN);
    for (int it = 0; it < iters; ++it) {
      const int s = it % STAGES;
      if (!mbar_wait(&full[s], (it / STAGES) & 1, kWaitNs)) {
        atomicCAS(status, kOk, kTimeoutFull);
        abort = true;
        break;
      }
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + s * L::kStage);
      const uint32_t sb = sa + L::kA;
      const uint64_t da = sdesc_k128(sa), db = sdesc_k128(sb);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        // advance 16 elements (32 bytes) along K inside the swizzled rows
        mma_bf16(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (it > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&empty[s]);
    }
    if (!abort) mma_commit(accum);
  } else if (warp >= 2) {
    // ---------------- epilogue
    const int quad = warp & 3;  // TMEM lane quadrant this warp may access
    const int row = m0 + quad * 32 + lane;
    bool ok = mbar_wait(accum, 0, kWaitNs * 4);
    if (!ok) {
      if (lane == 0) atomicCAS(status, kOk, kTimeoutAccum);
    } else {
      tc_fence_after();
      const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(tl + c, v);
        if (n0 + c < N) epi(row, n0 + c, v, M, N);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kCols);
  }
}

// host side -----------------------------------------------------------------

// Encode a 2D BF16 tensor map over a row-major [rows][ld] array (K contiguous),
// box = (64 elements of K) x box_rows, 128-byte swizzle, zero fill out of bounds.
mgw_status make_map_2d(mgw_handle* h, CUtensorMap* map, const void* base, long rows, long cols, long ld,
                       int box_rows);
// 3D BF16 map: dims (d0 contiguous, d1, d2) with byte strides s1, s2; box (64, b1, b2).
mgw_status make_map_3d(mgw_handle* h, CUtensorMap* map, const void* base, long d0, long d1, long d2, long s1,
                       long s2, int b1, int b2);

template <int BN, int STAGES, class Loader, class Epi>
mgw_status tc_gemm_launch(mgw_handle* h, const CUtensorMap* A, const CUtensorMap* B, PairTable pairs, int M,
                          int N, int K, const Loader& ld, const Epi& epi, int* dstatus, const char* what) {
  using L = SmemLayout<BN, STAGES>;
  auto kern = tc_gemm_kernel<BN, STAGES, Loader, Epi>;
  // once per instantiation (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kBytes);
  MGW_CUDA(h, attr);
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), 1);
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (h->prof) {
    cudaEventCreate(&ea);
    cudaEventCreate(&eb);
    cudaEventRecord(ea, h->stream);
  }
  kern<<<grid, kThreads, L::kBytes, h->stream>>>(A[0], A[1], B[0], B[1], pairs, M, N, K, ld, epi, dstatus);
  mgw_status st = check_launch(h, what);
  if (h->prof) {
    cudaEventRecord(eb, h->stream);
    h->spans.push_back({what, ea, eb});
  }
  return st;
}

// FP64 -> (hi, lo) BF16 split of a row-major [rows][cols] matrix into padded
// [rows][ld] arrays (ld >= cols, multiple of 8; padding zero): hi = bf16(x),
// lo = bf16(x - hi).
mgw_status split_bf16(mgw_handle* h, long rows, long cols, const double* src, long lds, void* hi, void* lo,
                      long ld);

// Read the device status word written by tensor-core kernels (synchronises).
mgw_status check_tc_status(mgw_handle* h, int* dstatus, const char* what);

}  // namespace tc
}  // namespace mgw
