// Digit slicing for the FP64-accurate tensor-core GEMM, tensor maps, and
// the public entry point mgw_gemm_fp64_emu.
#include "ozaki.h"
#include "tc_gemm.h"

#include <cuda_bf16.h>

namespace mgw {
namespace oz {

__device__ __forceinline__ int row_exponent(double mx) {
  // 2^e > 2 |x| for every x of the row: |x| 2^-e < 1/2
  return mx > 0.0 ? ilogb(mx) + 2 : 0;
}

// digits of x 2^-e: balanced base-256, d_s stored as bf16(d_s 2^-8(s-1))
__device__ __forceinline__ void digits_of(double x, int e, __nv_bfloat16 (&d)[kSlices]) {
  double y = ldexp(x, 8 - e);
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const double q = rint(y);
    d[s] = __double2bfloat16(ldexp(q, -8 * s));
    y = (y - q) * 256.0;
  }
}

// source row of a result row: plain (row r of X) or grouped moments
struct RowsPlain {
  const double* X; long lds;
  __device__ const double* row(long r) const { return X + r * lds; }
};
struct RowsGrouped {
  const double* W; int nmom, PB, naux;
  __device__ const double* row(long R) const {
    const long g = R / 128;
    const int rr = (int)(R % 128), t = rr / PB, P = (int)g * PB + rr % PB;
    if (rr >= nmom * PB || P >= naux) return nullptr;
    return W + ((long)t * naux + P) * naux;
  }
};

// one warp per row of a row-major source (a null row slices as zero)
template <class Rows>
__global__ void k_slice_rows(long rows, long K, Rows src, __nv_bfloat16* dig, long ld, int* exps) {
  const long r = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const double* xr = src.row(r);
  double mx = 0.0;
  if (xr)
    for (long k = lane; k < K; k += 32) mx = fmax(mx, fabs(xr[k]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = row_exponent(mx);
  if (lane == 0) exps[r] = e;
  const long plane = rows * ld;
  for (long k = lane; k < ld; k += 32) {
    __nv_bfloat16 d[kSlices];
    digits_of((xr && k < K) ? xr[k] : 0.0, e, d);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) dig[s * plane + r * ld + k] = d[s];
  }
}

// 32 result rows per CTA (256 threads); result row r, element k = X[k*ldx + r]
__global__ void k_slice_cols(long rows, long K, const double* __restrict__ X, long ldx, __nv_bfloat16* dig, long ld,
                             int* exps) {
  __shared__ double smax[8][32];
  __shared__ int sexp[32];
  __shared__ __nv_bfloat16 sd[kSlices][32][65];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long r0 = (long)blockIdx.x * 32;
  const long r = r0 + lane;
  double mx = 0.0;
  if (r < rows)
    for (long k = w; k < K; k += 8) mx = fmax(mx, fabs(X[k * ldx + r]));
  smax[w][lane] = mx;
  __syncthreads();
  if (w == 0) {
    double m = smax[0][lane];
    for (int i = 1; i < 8; ++i) m = fmax(m, smax[i][lane]);
    const int e = row_exponent(m);
    sexp[lane] = e;
    if (r < rows) exps[r] = e;
  }
  __syncthreads();
  const int e = sexp[lane];
  const long plane = rows * ld;
  for (long k0 = 0; k0 < ld; k0 += 64) {
    for (int kk = w; kk < 64; kk += 8) {
      const long k = k0 + kk;
      const double x = (r < rows && k < K) ? X[k * ldx + r] : 0.0;
      __nv_bfloat16 d[kSlices];
      digits_of(x, e, d);
#pragma unroll
      for (int s = 0; s < kSlices; ++s) sd[s][lane][kk] = d[s];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSlices * 32 * 64; i += 256) {
      const int s = i / (32 * 64), rr = (i / 64) % 32, kk = i % 64;
      const long k = k0 + kk;
      if (r0 + rr < rows && k < ld) dig[s * plane + (r0 + rr) * ld + k] = sd[s][rr][kk];
    }
    __syncthreads();
  }
}

mgw_status slice_rows(mgw_handle* h, long rows, long K, const double* X, long lds, Sliced& out) {
  k_slice_rows<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
      rows, K, RowsPlain{X, lds}, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps);
  return check_launch(h, "slice_rows");
}

mgw_status slice_grouped(mgw_handle* h, int nmom, int PB, int naux, const double* W, Sliced& out) {
  k_slice_rows<<<(unsigned)((out.rows * 32 + 255) / 256), 256, 0, h->stream>>>(
      out.rows, naux, RowsGrouped{W, nmom, PB, naux}, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps);
  return check_launch(h, "slice_grouped");
}

mgw_status slice_cols(mgw_handle* h, long rows, long K, const double* X, long ldx, Sliced& out) {
  k_slice_cols<<<(unsigned)((rows + 31) / 32), 256, 0, h->stream>>>(
      rows, K, X, ldx, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps);
  return check_launch(h, "slice_cols");
}

// 32 result rows per CTA (256 threads); element (r, k) = X[roff(r) + koff(k)]
__global__ void k_slice_gather(long rows, long K, const double* __restrict__ X, Gather g, __nv_bfloat16* dig,
                               long ld, int* exps) {
  __shared__ double smax[8][32];
  __shared__ int sexp[32];
  __shared__ __nv_bfloat16 sd[kSlices][32][65];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long r0 = (long)blockIdx.x * 32;
  const long r = r0 + lane;
  const long ro = r < rows ? (r / g.rdiv) * g.rhi + (r % g.rdiv) * g.rlo : 0;
  double mx = 0.0;
  if (r < rows)
    for (long k = w; k < K; k += 8) mx = fmax(mx, fabs(X[ro + (k / g.kdiv) * g.khi + (k % g.kdiv) * g.klo]));
  smax[w][lane] = mx;
  __syncthreads();
  if (w == 0) {
    double m = smax[0][lane];
    for (int i = 1; i < 8; ++i) m = fmax(m, smax[i][lane]);
    const int e = row_exponent(m);
    sexp[lane] = e;
    if (r < rows) exps[r] = e;
  }
  __syncthreads();
  const int e = sexp[lane];
  const long plane = rows * ld;
  for (long k0 = 0; k0 < ld; k0 += 64) {
    for (int kk = w; kk < 64; kk += 8) {
      const long k = k0 + kk;
      const double x = (r < rows && k < K) ? X[ro + (k / g.kdiv) * g.khi + (k % g.kdiv) * g.klo] : 0.0;
      __nv_bfloat16 d[kSlices];
      digits_of(x, e, d);
#pragma unroll
      for (int s = 0; s < kSlices; ++s) sd[s][lane][kk] = d[s];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSlices * 32 * 64; i += 256) {
      const int s = i / (32 * 64), rr = (i / 64) % 32, kk = i % 64;
      const long k = k0 + kk;
      if (r0 + rr < rows && k < ld) dig[s * plane + (r0 + rr) * ld + k] = sd[s][rr][kk];
    }
    __syncthreads();
  }
}

mgw_status slice_gather(mgw_handle* h, long rows, long K, const double* X, const Gather& g, Sliced& out) {
  k_slice_gather<<<(unsigned)((rows + 31) / 32), 256, 0, h->stream>>>(
      rows, K, X, g, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps);
  return check_launch(h, "slice_gather");
}

mgw_status digit_map(mgw_handle* h, CUtensorMap* map, const Sliced& s, int box_rows) {
  return tc::make_map_3d(h, map, s.digits, s.ld, s.rows, kSlices, s.ld * 2, s.rows * s.ld * 2, box_rows, 1);
}

// bytes of the digit planes + exponents of `rows` x K (in doubles, rounded)
size_t sliced_doubles(long rows, long K) {
  const long ld = (K + 63) / 64 * 64;
  return (size_t)((kSlices * rows * ld * 2 + 7) / 8) + (size_t)((rows * 4 + 7) / 8) + 64;
}

struct EpiStoreRows {
  double* C;
  long ldc;
  __device__ void operator()(int row_local, int col_base, int m0, int n0, int M, int N,
                             const long long (&v)[kCols], double*) const {
    const int row = m0 + row_local;
    if (row >= M) return;
#pragma unroll
    for (int j = 0; j < kCols; ++j) {
      const int col = n0 + col_base + j;
      if (col < N) C[(long)row * ldc + col] = __longlong_as_double(v[j]);
    }
  }
  __device__ void abort() const {}
};

}  // namespace oz
}  // namespace mgw

using namespace mgw;
using namespace mgw::oz;

namespace mgw {
namespace oz {
void place_sliced(double* mem, long rows, long K, Sliced& s) {
  const long ld = (K + 63) / 64 * 64;
  s.rows = rows;
  s.ld = ld;
  s.digits = mem;
  s.exps = reinterpret_cast<int*>(mem + (kSlices * rows * ld * 2 + 7) / 8);
}
}  // namespace oz
}  // namespace mgw

extern "C" mgw_status mgw_gemm_fp64_emu(mgw_handle* h, int M, int N, int K, const double* A, const double* B,
                                        double* C) {
  if (!h) return MGW_ERR_ARG;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return fail(h, MGW_ERR_ARG, "mgw_gemm_fp64_emu: bad arguments");
  MGW_CUDA(h, cudaSetDevice(h->device));
  Arena ar;
  double *da, *db, *st;
  ar.add(&da, sliced_doubles(M, K));
  ar.add(&db, sliced_doubles(N, K));
  ar.add(&st, 1);
  MGW_TRY(ar.commit(h));
  Sliced sa, sb;
  const long ld = (K + 63) / 64 * 64;
  sa.rows = M; sa.ld = ld; sa.digits = da; sa.exps = reinterpret_cast<int*>(da + (kSlices * (long)M * ld * 2 + 7) / 8);
  sb.rows = N; sb.ld = ld; sb.digits = db; sb.exps = reinterpret_cast<int*>(db + (kSlices * (long)N * ld * 2 + 7) / 8);
  int* dstatus = reinterpret_cast<int*>(st);
  MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
  MGW_TRY(slice_rows(h, M, K, A, K, sa));
  MGW_TRY(slice_rows(h, N, K, B, K, sb));
  CUtensorMap ma, mb;
  MGW_TRY(digit_map(h, &ma, sa, BM));
  MGW_TRY(digit_map(h, &mb, sb, BN));
  MGW_TRY((ozaki_launch(h, ma, mb, sa.exps, sb.exps, M, N, K, ARowsPlain{}, EpiStoreRows{C, N}, dstatus,
                        "gemm_fp64_emu")));
  return tc::check_tc_status(h, dstatus, "mgw_gemm_fp64_emu");
}
