// Host helpers of the tensor-core GEMM (tensor maps, BF16 split) and the
// public split-precision GEMM entry point.
#include "tc_gemm.h"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

namespace mgw {
namespace tc {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // looked up once; the initialisation of a function-local static is
  // thread-safe, so handles driven from several host threads may race here
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
  return fn;
}

mgw_status make_map_2d(mgw_handle* h, CUtensorMap* map, const void* base, long rows, long cols, long ld,
                       int box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(h, MGW_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15))
    return fail(h, MGW_ERR_ARG, "tensor map: base or row stride not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(h, MGW_ERR_CUDA, "cuTensorMapEncodeTiled (2D) failed: %d", (int)r);
  return MGW_OK;
}

mgw_status make_map_3d(mgw_handle* h, CUtensorMap* map, const void* base, long d0, long d1, long d2, long s1,
                       long s2, int b1, int b2) {
  auto fn = encode_fn();
  if (!fn) return fail(h, MGW_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (s1 & 15) || (s2 & 15))
    return fail(h, MGW_ERR_ARG, "tensor map: base or strides not 16-byte aligned");
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)s1, (cuuint64_t)s2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)b1, (cuuint32_t)b2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(h, MGW_ERR_CUDA, "cuTensorMapEncodeTiled (3D) failed: %d", (int)r);
  return MGW_OK;
}

__global__ void k_split_bf16(long rows, long cols, const double* src, long lds, __nv_bfloat16* hi,
                             __nv_bfloat16* lo, long ld) {
  const long total = rows * ld;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    long r = i / ld, c = i % ld;
    double x = c < cols ? src[r * lds + c] : 0.0;
    __nv_bfloat16 a = __double2bfloat16(x);
    double rest = x - (double)__bfloat162float(a);
    hi[i] = a;
    lo[i] = __double2bfloat16(rest);
  }
}

mgw_status split_bf16(mgw_handle* h, long rows, long cols, const double* src, long lds, void* hi, void* lo,
                      long ld) {
  long total = rows * ld;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_split_bf16<<<(unsigned)blocks, 256, 0, h->stream>>>(rows, cols, src, lds, (__nv_bfloat16*)hi,
                                                        (__nv_bfloat16*)lo, ld);
  return check_launch(h, "split_bf16");
}

mgw_status check_tc_status(mgw_handle* h, int* dstatus, const char* what) {
  int st = 0;
  MGW_CUDA(h, cudaMemcpyAsync(&st, dstatus, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (st != kOk) return fail(h, MGW_ERR_TIMEOUT, "%s: tensor-core pipeline wait timed out (code %d)", what, st);
  return MGW_OK;
}

// Epilogue: C[row][col] = alpha * acc (+ beta * C), FP64 output
struct EpiStoreF64 {
  double* C;
  long ldc;
  double alpha, beta;
  __device__ void operator()(int row, int col0, const float (&v)[16], int M, int N) const {
    if (row >= M) return;
    double* c = C + (long)row * ldc + col0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (col0 + j < N) c[j] = beta == 0.0 ? alpha * (double)v[j] : alpha * (double)v[j] + beta * c[j];
    }
  }
};

}  // namespace tc
}  // namespace mgw

using namespace mgw;
using namespace mgw::tc;

extern "C" mgw_status mgw_gemm_bf16x3(mgw_handle* h, int M, int N, int K, const double* A, const double* B,
                                      double* C) {
  if (!h) return MGW_ERR_ARG;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return fail(h, MGW_ERR_ARG, "mgw_gemm_bf16x3: bad arguments");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long ld = (K + 7) / 8 * 8;
  Arena ar;
  double *ah, *al, *bh, *bl, *st;
  // bf16 buffers: count in doubles (4 bf16 per double), rounded up
  ar.add(&ah, (M * ld + 3) / 4);
  ar.add(&al, (M * ld + 3) / 4);
  ar.add(&bh, (N * ld + 3) / 4);
  ar.add(&bl, (N * ld + 3) / 4);
  ar.add(&st, 1);
  MGW_TRY(ar.commit(h));
  int* dstatus = reinterpret_cast<int*>(st);
  MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
  MGW_TRY(split_bf16(h, M, K, A, K, ah, al, ld));
  MGW_TRY(split_bf16(h, N, K, B, K, bh, bl, ld));
  CUtensorMap ma[2], mb[2];
  constexpr int BN = 256;
  MGW_TRY(make_map_2d(h, &ma[0], ah, M, K, ld, BM));
  MGW_TRY(make_map_2d(h, &ma[1], al, M, K, ld, BM));
  MGW_TRY(make_map_2d(h, &mb[0], bh, N, K, ld, BN));
  MGW_TRY(make_map_2d(h, &mb[1], bl, N, K, ld, BN));
  PairTable pairs{3, {0, 0, 1, 0}, {0, 1, 0, 0}};
  EpiStoreF64 epi{C, N, 1.0, 0.0};
  MGW_TRY((tc_gemm_launch<BN, 4>(h, ma, mb, pairs, M, N, K, Loader2D{}, epi, dstatus, "tc_gemm_bf16x3")));
  return check_tc_status(h, dstatus, "mgw_gemm_bf16x3");
}
