// Digit slicing for the FP64-accurate tensor-core GEMM, tensor maps, and
// the public entry point mgw_gemm_fp64_emu.
#include "ozaki.h"
#include "ozaki_mixed.h"
#include "tc_gemm.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mgw {
namespace oz {

__device__ __forceinline__ int row_exponent(double mx) {
  // 2^e > 2 |x| for every x of the row: |x| 2^-e < 1/2
  return mx > 0.0 ? ilogb(mx) + 2 : 0;
}

// X = round(x 2^(bits - e)) from the IEEE fields, integer arithmetic only
// (nearest, ties away from zero); |X| < 2^(bits-1) when |x| < 2^(e-1)
__device__ __forceinline__ long long fixed_of(double x, int e, int bits) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int bexp = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & ((1ull << 52) - 1);
  int ex;  // |x| = m 2^ex
  if (bexp == 0) {
    ex = -1074;
  } else {
    m |= 1ull << 52;
    ex = bexp - 1075;
  }
  const int sh = ex + bits - e;
  long long X;
  if (sh >= 0) {
    X = (long long)(m << sh);  // sh <= 2 because |x| < 2^(e-1) and bits <= 56
  } else if (sh > -60) {
    const int r = -sh;
    X = (long long)((m >> r) + ((m >> (r - 1)) & 1ull));
  } else {
    X = 0;
  }
  return (b >> 63) ? -X : X;
}

// NS digits of x 2^-e: balanced base-256, d_s stored as bf16(d_s 2^-8(s-1)).
// X = round(x 2^(8 NS - e)) (|X| < 2^(8 NS - 1)), then d_NS, ..., d_2 in
// [-128, 127] from the low end and d_1 = what is left (|d_1| <= 128), so
// x 2^-e = sum_s d_s 2^-8s to within half a unit of 2^-8NS.
template <int NS>
__device__ __forceinline__ void digits_of(double x, int e, __nv_bfloat16 (&d)[NS]) {
  long long X = fixed_of(x, e, 8 * NS);
#pragma unroll
  for (int s = NS - 1; s >= 1; --s) {
    const int dv = (int)((X + 128) & 255) - 128;
    X = (X - dv) >> 8;
    d[s] = __float2bfloat16_rn(__int2float_rn(dv) * __int_as_float((127 - 8 * s) << 23));
  }
  d[0] = __float2bfloat16_rn(__int2float_rn((int)X));
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

// one warp per row of a row-major source (a null row slices as zero); with
// gexp the exponent is the tensor's grid exponent instead of the row's own
template <class Rows, int NS>
__global__ void k_slice_rows(long rows, long K, Rows src, __nv_bfloat16* dig, long ld, int* exps,
                             const int* gexp) {
  const long r = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const double* xr = src.row(r);
  int e;
  if (gexp) {
    e = *gexp;
  } else {
    double mx = 0.0;
    if (xr)
      for (long k = lane; k < K; k += 32) mx = fmax(mx, fabs(xr[k]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    e = row_exponent(mx);
  }
  if (lane == 0) exps[r] = e;
  const long plane = rows * ld;
  for (long k = lane; k < ld; k += 32) {
    __nv_bfloat16 d[NS];
    digits_of<NS>((xr && k < K) ? xr[k] : 0.0, e, d);
#pragma unroll
    for (int s = 0; s < NS; ++s) dig[s * plane + r * ld + k] = d[s];
  }
}

mgw_status slice_rows(mgw_handle* h, long rows, long K, const double* X, long lds, Sliced& out) {
  ProfSpan span(h, "slice_rows");
  if (out.ns != kSlices) return fail(h, MGW_ERR_ARG, "slice_rows: %d-digit planes", out.ns);
  k_slice_rows<RowsPlain, kSlices><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
      rows, K, RowsPlain{X, lds}, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps, nullptr);
  return check_launch(h, "slice_rows");
}

mgw_status slice_rows_grid(mgw_handle* h, long rows, long K, const double* X, long lds, const int* gexp,
                           Sliced& out) {
  ProfSpan span(h, "slice_rows");
  if (out.ns != kGridSlices) return fail(h, MGW_ERR_ARG, "slice_rows_grid: %d-digit planes", out.ns);
  k_slice_rows<RowsPlain, kGridSlices><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, h->stream>>>(
      rows, K, RowsPlain{X, lds}, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps, gexp);
  return check_launch(h, "slice_rows_grid");
}

mgw_status slice_grouped(mgw_handle* h, int nmom, int PB, int naux, const double* W, Sliced& out) {
  ProfSpan span(h, "slice_grouped");
  if (out.ns != kSlices) return fail(h, MGW_ERR_ARG, "slice_grouped: %d-digit planes", out.ns);
  k_slice_rows<RowsGrouped, kSlices><<<(unsigned)((out.rows * 32 + 255) / 256), 256, 0, h->stream>>>(
      out.rows, naux, RowsGrouped{W, nmom, PB, naux}, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps,
      nullptr);
  return check_launch(h, "slice_grouped");
}

// max |x| over n elements into *gmax (bit pattern; zeroed by the caller)
__global__ void k_absmax(long n, const double* __restrict__ X, unsigned long long* gmax) {
  double m = 0.0;
  const long stride = (long)gridDim.x * blockDim.x;
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
#pragma unroll 4
  for (; i < n; i += stride) m = fmax(m, fabs(X[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(gmax, (unsigned long long)__double_as_longlong(m));
  }
}
__global__ void k_grid_exponent(const unsigned long long* gmax, int* gexp) {
  *gexp = row_exponent(__longlong_as_double((long long)*gmax));
}

mgw_status global_exponent(mgw_handle* h, long n, const double* X, unsigned long long* gmax, int* gexp) {
  ProfSpan span(h, "global_exponent");
  MGW_CUDA(h, cudaMemsetAsync(gmax, 0, sizeof(unsigned long long), h->stream));
  if (n > 0) {
    const long blocks = std::min<long>((n + 255) / 256, 152L * 8);
    k_absmax<<<(unsigned)blocks, 256, 0, h->stream>>>(n, X, gmax);
    MGW_TRY(check_launch(h, "absmax"));
  }
  k_grid_exponent<<<1, 1, 0, h->stream>>>(gmax, gexp);
  return check_launch(h, "grid_exponent");
}

// Xr = X rounded to the grid 2^(ex - 8 kGridSlices): the value its digits carry
__global__ void k_round_to_grid(long n, const double* __restrict__ X, const int* __restrict__ gexp, double* Xr) {
  const int e = *gexp;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long long q = fixed_of(X[i], e, 8 * kGridSlices);
    // |q| < 2^15: exact in a double, and the power of two scales it exactly
    Xr[i] = ldexp((double)q, e - 8 * kGridSlices);
  }
}

mgw_status round_to_grid(mgw_handle* h, long n, const double* X, const int* gexp, double* Xr) {
  if (n <= 0) return MGW_OK;
  k_round_to_grid<<<(unsigned)std::min<long>((n + 255) / 256, 152L * 16), 256, 0, h->stream>>>(n, X, gexp, Xr);
  return check_launch(h, "round_to_grid");
}

// Gathered sources with rows contiguous in memory: element (r, k) sits at
// X[ro(r) + ko(k)], ro(r) = (r / rdiv) rhi + (r % rdiv) rlo and ko likewise.
// A lane owns a row, so each warp load is 32 consecutive doubles.
struct KWalk {  // k -> (k / kdiv, k % kdiv), stepped without dividing
  long q, rem;
  const Gather& g;
  __device__ KWalk(long k, const Gather& g_) : q(k / g_.kdiv), rem(k % g_.kdiv), g(g_) {}
  __device__ long off() const { return q * g.khi + rem * g.klo; }
  __device__ void step(int d) {
    rem += d;
    if (rem >= g.kdiv) {
      q += rem / g.kdiv;
      rem %= g.kdiv;
    }
  }
};

// pass 1: row maxima over a K range per CTA, merged with atomicMax on the
// bit patterns (non-negative doubles order like their bits)
__global__ void k_gather_rowmax(long rows, long K, const double* __restrict__ X, Gather g, long kper,
                                unsigned long long* rmax) {
  __shared__ double sm[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long r = blockIdx.x * 32L + lane;
  const long kbeg = blockIdx.y * kper, kend = min(K, kbeg + kper);
  double m = 0.0;
  if (r < rows && kbeg + w < kend) {
    const double* xr = X + (r / g.rdiv) * g.rhi + (r % g.rdiv) * g.rlo;
    KWalk kw(kbeg + w, g);
#pragma unroll 4
    for (long k = kbeg + w; k < kend; k += 8) {
      m = fmax(m, fabs(xr[kw.off()]));
      kw.step(8);
    }
  }
  sm[w][lane] = m;
  __syncthreads();
  if (w == 0 && r < rows) {
    for (int i = 1; i < 8; ++i) m = fmax(m, sm[i][lane]);
    atomicMax(rmax + r, (unsigned long long)__double_as_longlong(m));
  }
}

// pass 2: one 32-row x 64-k tile per CTA; digits staged in shared memory and
// written along k (128 B per row and digit plane).  With gexp every row takes
// the tensor's grid exponent (no max pass).
template <int NS>
__global__ void k_gather_digits(long rows, long K, const double* __restrict__ X, Gather g,
                                const unsigned long long* __restrict__ rmax, const int* __restrict__ gexp,
                                __nv_bfloat16* dig, long ld, int* exps) {
  __shared__ __align__(4) __nv_bfloat16 sd[NS][32][66];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long r0 = blockIdx.x * 32L, r = r0 + lane;
  const long k0 = blockIdx.y * 64L;
  int e = 0;
  if (r < rows) {
    e = gexp ? *gexp : row_exponent(__longlong_as_double((long long)rmax[r]));
    if (blockIdx.y == 0) exps[r] = e;
  }
  const double* xr = r < rows ? X + (r / g.rdiv) * g.rhi + (r % g.rdiv) * g.rlo : X;
  KWalk kw(k0 + w, g);
#pragma unroll 2
  for (int kk = w; kk < 64; kk += 8) {
    const long k = k0 + kk;
    const double x = (r < rows && k < K) ? xr[kw.off()] : 0.0;
    kw.step(8);
    __nv_bfloat16 d[NS];
    digits_of<NS>(x, e, d);
#pragma unroll
    for (int s = 0; s < NS; ++s) sd[s][lane][kk] = d[s];
  }
  __syncthreads();
  const long plane = rows * ld;
  for (int i = threadIdx.x; i < NS * 32 * 32; i += 256) {  // 32-bit words: two k per word
    const int s = i / (32 * 32), rr = (i / 32) % 32, kp = (i % 32) * 2;
    if (r0 + rr < rows && k0 + kp < ld)
      *reinterpret_cast<uint32_t*>(dig + s * plane + (r0 + rr) * ld + k0 + kp) =
          *reinterpret_cast<const uint32_t*>(&sd[s][rr][kp]);
  }
}

mgw_status slice_gather(mgw_handle* h, long rows, long K, const double* X, const Gather& g, Sliced& out) {
  ProfSpan span(h, "slice_gather");
  if (out.ns != kSlices) return fail(h, MGW_ERR_ARG, "slice_gather: %d-digit planes", out.ns);
  if (rows <= 0) return MGW_OK;
  if (out.ld == 0) {  // K = 0: no digits, zero exponents
    MGW_CUDA(h, cudaMemsetAsync(out.exps, 0, sizeof(int) * rows, h->stream));
    return MGW_OK;
  }
  MGW_CUDA(h, cudaMemsetAsync(out.rmax, 0, sizeof(unsigned long long) * rows, h->stream));
  const long gx = (rows + 31) / 32;
  // K split so that about eight CTAs per SM run the max pass
  const long want = std::max(1L, (152L * 8 + gx - 1) / gx);
  const long ksplit = std::min(want, std::max(1L, (K + 255) / 256));
  const long kper = (K + ksplit - 1) / ksplit;
  if (K > 0) {
    k_gather_rowmax<<<dim3((unsigned)gx, (unsigned)ksplit), 256, 0, h->stream>>>(rows, K, X, g, kper, out.rmax);
    MGW_TRY(check_launch(h, "gather_rowmax"));
  }
  k_gather_digits<kSlices><<<dim3((unsigned)gx, (unsigned)(out.ld / 64)), 256, 0, h->stream>>>(
      rows, K, X, g, out.rmax, nullptr, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps);
  return check_launch(h, "gather_digits");
}

mgw_status slice_gather_grid(mgw_handle* h, long rows, long K, const double* X, const Gather& g, const int* gexp,
                             Sliced& out) {
  ProfSpan span(h, "slice_gather_grid");
  if (out.ns != kGridSlices) return fail(h, MGW_ERR_ARG, "slice_gather_grid: %d-digit planes", out.ns);
  if (rows <= 0) return MGW_OK;
  if (out.ld == 0) {
    MGW_CUDA(h, cudaMemsetAsync(out.exps, 0, sizeof(int) * rows, h->stream));
    return MGW_OK;
  }
  const long gx = (rows + 31) / 32;
  k_gather_digits<kGridSlices><<<dim3((unsigned)gx, (unsigned)(out.ld / 64)), 256, 0, h->stream>>>(
      rows, K, X, g, nullptr, gexp, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps);
  return check_launch(h, "gather_digits_grid");
}

// The same gather from a tensor already on its grid, held as 16-bit
// integers q (value q 2^(e-16)): the two digits come straight from q, exactly
// as digits_of<2> gives them for the value, and every row takes exponent e.
__global__ void k_gather_digits_q(long rows, long K, const short* __restrict__ X, Gather g, int e,
                                  __nv_bfloat16* dig, long ld, int* exps) {
  __shared__ __align__(4) __nv_bfloat16 sd[kGridSlices][32][66];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long r0 = blockIdx.x * 32L, r = r0 + lane;
  const long k0 = blockIdx.y * 64L;
  if (r < rows && blockIdx.y == 0) exps[r] = e;
  const short* xr = r < rows ? X + (r / g.rdiv) * g.rhi + (r % g.rdiv) * g.rlo : X;
  KWalk kw(k0 + w, g);
#pragma unroll 2
  for (int kk = w; kk < 64; kk += 8) {
    const long k = k0 + kk;
    const int q = (r < rows && k < K) ? (int)xr[kw.off()] : 0;
    kw.step(8);
    const int d2 = ((q + 128) & 255) - 128;
    const int d1 = (q - d2) >> 8;
    sd[0][lane][kk] = __float2bfloat16_rn((float)d1);
    sd[1][lane][kk] = __float2bfloat16_rn((float)d2 * 0x1p-8f);
  }
  __syncthreads();
  const long plane = rows * ld;
  for (int i = threadIdx.x; i < kGridSlices * 32 * 32; i += 256) {
    const int s = i / (32 * 32), rr = (i / 32) % 32, kp = (i % 32) * 2;
    if (r0 + rr < rows && k0 + kp < ld)
      *reinterpret_cast<uint32_t*>(dig + s * plane + (r0 + rr) * ld + k0 + kp) =
          *reinterpret_cast<const uint32_t*>(&sd[s][rr][kp]);
  }
}

mgw_status slice_gather_q(mgw_handle* h, long rows, long K, const short* X, const Gather& g, int e, Sliced& out) {
  ProfSpan span(h, "slice_gather_grid");
  if (out.ns != kGridSlices) return fail(h, MGW_ERR_ARG, "slice_gather_q: %d-digit planes", out.ns);
  if (rows <= 0) return MGW_OK;
  if (out.ld == 0) {
    MGW_CUDA(h, cudaMemsetAsync(out.exps, 0, sizeof(int) * rows, h->stream));
    return MGW_OK;
  }
  k_gather_digits_q<<<dim3((unsigned)((rows + 31) / 32), (unsigned)(out.ld / 64)), 256, 0, h->stream>>>(
      rows, K, X, g, e, static_cast<__nv_bfloat16*>(out.digits), out.ld, out.exps);
  return check_launch(h, "gather_digits_q");
}

// out[r][k] = q 2^(e-16) for element (r, k) of a gathered 16-bit grid tensor
__global__ void k_dequantize_gather(long rows, long K, const short* __restrict__ X, Gather g, int e, double* out) {
  const double unit = ldexp(1.0, e - 8 * kGridSlices);
  const long total = rows * K;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long r = i / K, k = i % K;
    out[i] = (double)X[(r / g.rdiv) * g.rhi + (r % g.rdiv) * g.rlo + (k / g.kdiv) * g.khi + (k % g.kdiv) * g.klo] * unit;
  }
}

mgw_status dequantize_gather(mgw_handle* h, long rows, long K, const short* X, const Gather& g, int e, double* out) {
  if (rows <= 0 || K <= 0) return MGW_OK;
  k_dequantize_gather<<<(unsigned)std::min<long>((rows * K + 255) / 256, 152L * 16), 256, 0, h->stream>>>(
      rows, K, X, g, e, out);
  return check_launch(h, "dequantize_gather");
}

// Lq = round(L 2^(16 - e)) (ties away from zero) as 16-bit integers; a value
// with |L| >= 2^(e-1) (outside the grid's range) raises *overflow
__global__ void k_quantize(long n, const double* __restrict__ L, int e, short* Lq, int* overflow) {
  const double lim = ldexp(1.0, e - 1);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double x = L[i];
    if (!(fabs(x) < lim)) {
      atomicOr(overflow, 1);
      Lq[i] = 0;
      continue;
    }
    Lq[i] = (short)fixed_of(x, e, 8 * kGridSlices);
  }
}

mgw_status quantize(mgw_handle* h, long n, const double* L, int e, short* Lq, int* overflow) {
  if (n <= 0) return MGW_OK;
  k_quantize<<<(unsigned)std::min<long>((n + 255) / 256, 152L * 16), 256, 0, h->stream>>>(n, L, e, Lq, overflow);
  return check_launch(h, "quantize");
}

mgw_status slice_cols(mgw_handle* h, long rows, long K, const double* X, long ldx, Sliced& out) {
  // element (r, k) = X[k * ldx + r]: a gather with undivided row and k indices
  return slice_gather(h, rows, K, X, Gather{rows + 1, 0, 1, K + 1, 0, ldx}, out);
}

mgw_status digit_map(mgw_handle* h, CUtensorMap* map, const Sliced& s, int box_rows) {
  return tc::make_map_3d(h, map, s.digits, s.ld, s.rows, s.ns, s.ld * 2, s.rows * s.ld * 2, box_rows, 1);
}

// bytes of the digit planes + exponents of `rows` x K (in doubles, rounded)
size_t sliced_doubles(long rows, long K, int ns) {
  const long ld = (K + 63) / 64 * 64;
  return (size_t)((ns * rows * ld * 2 + 7) / 8) + (size_t)((rows * 4 + 7) / 8) + (size_t)rows + 64;
}

__global__ void k_sum_splits(long count, int nsplit, const double* __restrict__ part, double* out,
                             int accumulate) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    double acc = accumulate ? out[i] : 0.0;
    for (int z = 0; z < nsplit; ++z) acc += part[(long)z * count + i];
    out[i] = acc;
  }
}

mgw_status reduce_splits(mgw_handle* h, long count, int nsplit, const double* part, double* out, int accumulate) {
  k_sum_splits<<<(unsigned)std::min<long>((count + 255) / 256, 152L * 16), 256, 0, h->stream>>>(count, nsplit, part,
                                                                                               out, accumulate);
  return check_launch(h, "reduce_splits");
}

struct EpiStoreRows {  // split z of a K-split launch writes C + z split_stride
  double* C;
  long ldc;
  long split_stride;
  __device__ bool skip_tile(int, int, int, int, int) const { return false; }
  template <int KC>
  __device__ void operator()(int row_local, int col_base, int m0, int n0, int M, int N, const long long (&v)[KC],
                             double*) const {
    const int row = m0 + row_local;
    if (row >= M) return;
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      const int col = n0 + col_base + j;
      if (col < N) C[(long)blockIdx.y * split_stride + (long)row * ldc + col] = __longlong_as_double(v[j]);
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
void place_sliced(double* mem, long rows, long K, Sliced& s, int ns) {
  const long ld = (K + 63) / 64 * 64;
  s.rows = rows;
  s.ld = ld;
  s.ns = ns;
  s.digits = mem;
  s.exps = reinterpret_cast<int*>(mem + (ns * rows * ld * 2 + 7) / 8);
  s.rmax = reinterpret_cast<unsigned long long*>(mem + (ns * rows * ld * 2 + 7) / 8 + (rows * 4 + 7) / 8);
}
}  // namespace oz
}  // namespace mgw

namespace mgw {
namespace oz {
// One CTA waits, with the pipeline's bounded wait, on an mbarrier that
// nothing ever arrives at; the wait must give up after limit_ns and raise
// the status word (the error path every tensor-core kernel takes).
__global__ void k_bounded_wait_selftest(unsigned long long limit_ns, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  __syncthreads();
  if (!tc::mbar_wait(&bar, 0, limit_ns) && threadIdx.x == 0) atomicCAS(status, tc::kOk, tc::kTimeoutFull);
}
}  // namespace oz
}  // namespace mgw

extern "C" mgw_status mgw_selftest_bounded_wait(mgw_handle* h, double limit_s) {
  if (!h) return MGW_ERR_ARG;
  if (!(limit_s > 0.0 && limit_s <= 10.0))
    return fail(h, MGW_ERR_ARG, "mgw_selftest_bounded_wait: limit %g s outside (0, 10]", limit_s);
  MGW_CUDA(h, cudaSetDevice(h->device));
  Arena ar;
  double* st;
  ar.add(&st, 1);
  MGW_TRY(ar.commit(h));
  int* dstatus = reinterpret_cast<int*>(st);
  MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
  oz::k_bounded_wait_selftest<<<1, 32, 0, h->stream>>>((unsigned long long)(limit_s * 1e9), dstatus);
  MGW_TRY(check_launch(h, "bounded_wait_selftest"));
  return tc::check_tc_status(h, dstatus, "mgw_selftest_bounded_wait");
}

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
  place_sliced(da, M, K, sa);
  place_sliced(db, N, K, sb);
  int* dstatus = reinterpret_cast<int*>(st);
  MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
  MGW_TRY(slice_rows(h, M, K, A, K, sa));
  MGW_TRY(slice_rows(h, N, K, B, K, sb));
  CUtensorMap ma, mb;
  MGW_TRY(digit_map(h, &ma, sa, BM));
  MGW_TRY(digit_map(h, &mb, sb, BN));
  MGW_TRY((ozaki_launch(h, ma, mb, sa.exps, sb.exps, M, N, K, ARowsPlain{}, EpiStoreRows{C, N, 0}, dstatus,
                        "gemm_fp64_emu")));
  return tc::check_tc_status(h, dstatus, "mgw_gemm_fp64_emu");
}

namespace mgw {
namespace oz {
mgw_status gemm_fp64_tc_nn(mgw_handle* h, int M, int N, int K, const double* A, long lda, const double* B, long ldb,
                           double* C, long ldc, const char* what) {
  if (M < 1 || N < 1 || K < 1) return MGW_OK;
  // slot buffers, not the workspace arena: callers run this inside calls that
  // hold arena pointers, and growing the arena would move them
  double *da, *db, *st;
  MGW_TRY(slot_buffer(h, 85, sliced_doubles(M, K), &da));
  MGW_TRY(slot_buffer(h, 86, sliced_doubles(N, K), &db));
  MGW_TRY(slot_buffer(h, 87, 1, &st));
  Sliced sa, sb;
  place_sliced(da, M, K, sa);
  place_sliced(db, N, K, sb);
  int* dstatus = reinterpret_cast<int*>(st);
  MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
  MGW_TRY(slice_rows(h, M, K, A, lda, sa));
  MGW_TRY(slice_cols(h, N, K, B, ldb, sb));
  CUtensorMap ma, mb;
  MGW_TRY(digit_map(h, &ma, sa, BM));
  MGW_TRY(digit_map(h, &mb, sb, BN));
  MGW_TRY((ozaki_launch(h, ma, mb, sa.exps, sb.exps, M, N, K, ARowsPlain{}, EpiStoreRows{C, ldc, 0}, dstatus, what)));
  return tc::check_tc_status(h, dstatus, what);
}
}  // namespace oz
}  // namespace mgw

extern "C" mgw_status mgw_gemm_mixed(mgw_handle* h, int M, int N, int K, const double* A, const double* B,
                                     double* C) {
  if (!h) return MGW_ERR_ARG;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return fail(h, MGW_ERR_ARG, "mgw_gemm_mixed: bad arguments");
  MGW_CUDA(h, cudaSetDevice(h->device));
  // K beyond kMixedMaxK runs in splits, summed from partial products
  const int nsplit = mixed_min_split(K);
  const int nz = split_count(K, nsplit);
  Arena ar;
  double *da, *db, *st, *part = nullptr;
  ar.add(&da, sliced_doubles(M, K));
  ar.add(&db, sliced_doubles(N, K, kGridSlices));
  ar.add(&st, 3);
  if (nz > 1) ar.add(&part, (size_t)nz * M * N);
  MGW_TRY(ar.commit(h));
  Sliced sa, sb;
  place_sliced(da, M, K, sa);
  place_sliced(db, N, K, sb, kGridSlices);
  int* dstatus = reinterpret_cast<int*>(st);
  int* gexp = reinterpret_cast<int*>(st + 2);
  MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
  MGW_TRY(slice_rows(h, M, K, A, K, sa));
  MGW_TRY(global_exponent(h, (long)N * K, B, reinterpret_cast<unsigned long long*>(st + 1), gexp));
  MGW_TRY(slice_rows_grid(h, N, K, B, K, gexp, sb));
  CUtensorMap ma, mb;
  MGW_TRY(digit_map(h, &ma, sa, BM));
  MGW_TRY(digit_map(h, &mb, sb, kMBN));
  if (nz == 1) {
    MGW_TRY((ozaki_mixed_launch<true>(h, ma, mb, sa.exps, sb.exps, M, N, K, ARowsPlain{}, EpiStoreRows{C, N, 0},
                                      dstatus, "gemm_mixed")));
  } else {
    MGW_TRY((ozaki_mixed_launch<true>(h, ma, mb, sa.exps, sb.exps, M, N, K, ARowsPlain{},
                                      EpiStoreRows{part, N, (long)M * N}, dstatus, "gemm_mixed", nsplit)));
    MGW_TRY(reduce_splits(h, (long)M * N, nz, part, C, 0));
  }
  return tc::check_tc_status(h, dstatus, "mgw_gemm_mixed");
}

extern "C" int mgw_grid_exponent(double absmax) {
  if (!(absmax > 0.0) || !std::isfinite(absmax)) return 0;
  return std::ilogb(absmax) + 2;  // absmax < 2^(e-1)
}

extern "C" mgw_status mgw_df_absmax(mgw_handle* h, long count, const double* L, double* absmax_host) {
  if (!h) return MGW_ERR_ARG;
  if (count < 0 || (count > 0 && !L) || !absmax_host) return fail(h, MGW_ERR_ARG, "mgw_df_absmax: bad arguments");
  MGW_CUDA(h, cudaSetDevice(h->device));
  Arena ar;
  double* st;
  ar.add(&st, 2);
  MGW_TRY(ar.commit(h));
  MGW_TRY(global_exponent(h, count, L, reinterpret_cast<unsigned long long*>(st), reinterpret_cast<int*>(st + 1)));
  unsigned long long bits = 0;
  MGW_CUDA(h, cudaMemcpyAsync(&bits, st, sizeof bits, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  double v;
  std::memcpy(&v, &bits, sizeof v);
  *absmax_host = v;
  return MGW_OK;
}

extern "C" mgw_status mgw_df_quantize(mgw_handle* h, long count, const double* L, int e, short* Lq,
                                      int* overflow_host) {
  if (!h) return MGW_ERR_ARG;
  if (count < 0 || (count > 0 && (!L || !Lq)) || e < -1000 || e > 1000)
    return fail(h, MGW_ERR_ARG, "mgw_df_quantize: bad arguments");
  MGW_CUDA(h, cudaSetDevice(h->device));
  Arena ar;
  double* st;
  ar.add(&st, 1);
  MGW_TRY(ar.commit(h));
  int* flag = reinterpret_cast<int*>(st);
  MGW_CUDA(h, cudaMemsetAsync(flag, 0, sizeof(int), h->stream));
  MGW_TRY(quantize(h, count, L, e, Lq, flag));
  if (overflow_host) {
    MGW_CUDA(h, cudaMemcpyAsync(overflow_host, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    MGW_CUDA(h, cudaStreamSynchronize(h->stream));
    if (*overflow_host) return fail(h, MGW_ERR_ARG, "mgw_df_quantize: a value lies outside |L| < 2^(e-1), e = %d", e);
  }
  return MGW_OK;
}
