// The warm-start network of the fsGW loop: three dense layers with SiLU,
//   z1 = W1 x + b1, a1 = silu(z1); z2 = W2 a1 + b2, a2 = silu(z2); y = W3 a2 + b3,
// weights held in BF16 for every product (FP32 master copy for the
// optimiser), biases, activations and accumulation in FP32.  Parameters are
// one packed vector [W1 | b1 | W2 | b2 | W3 | b3]; the BF16 copy has the same
// layout.  Training: mean-squared error, Adam.  Not in the paper.
#include "mgw_internal.h"

#include <cuda_bf16.h>

namespace mgw {
namespace mlp {

struct Offsets {
  long w1, b1, w2, b2, w3, b3, n;
  Offsets(int d_in, int width, int d_out) {
    w1 = 0;
    b1 = w1 + (long)width * d_in;
    w2 = b1 + width;
    b2 = w2 + (long)width * width;
    w3 = b2 + width;
    b3 = w3 + (long)d_out * width;
    n = b3 + d_out;
  }
};

// C[M][N] (+)= sum_k A(m,k) B(k,n), FP32 accumulate; operands via accessors
struct AF32 {  // A(m,k) = p[m*ld + k]  (or transposed: p[k*ld + m])
  const float* p; long ld; int trans;
  __device__ float at(long m, long k) const { return trans ? p[k * ld + m] : p[m * ld + k]; }
};
struct BBf16 {  // B(k,n) = W[n*ld + k] (trans = 0, "x W^T")  or W[k*ld + n] (trans = 1, "dz W")
  const __nv_bfloat16* p; long ld; int trans;
  __device__ float at(long k, long n) const { return __bfloat162float(trans ? p[k * ld + n] : p[n * ld + k]); }
};
struct BF32 {  // B(k,n) = p[k*ld + n]
  const float* p; long ld;
  __device__ float at(long k, long n) const { return p[k * ld + n]; }
};

template <class AOp, class BOp>
__global__ void __launch_bounds__(256) k_sgemm(long M, long N, long K, AOp A, BOp B, float* C, long ldc,
                                               const float* bias, float beta) {
  constexpr int T = 32;
  __shared__ float As[T][T + 1], Bs[T][T + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 outputs each
  const long m0 = (long)blockIdx.y * T, n0 = (long)blockIdx.x * T;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (long k0 = 0; k0 < K; k0 += T) {
    for (int i = threadIdx.x; i < T * T; i += 256) {
      const int r = i / T, c = i % T;
      const long m = m0 + r, k = k0 + c;
      As[r][c] = (m < M && k < K) ? A.at(m, k) : 0.f;
      const long kk = k0 + r, n = n0 + c;
      Bs[r][c] = (kk < K && n < N) ? B.at(kk, n) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < T; ++k) {
      const float a0 = As[ty][k], a1 = As[ty + 16][k];
      const float b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const long m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= M || n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      float* c = C + m * ldc + n;
      *c = beta == 0.f ? v : v + beta * *c;
    }
}

template <class AOp, class BOp>
static mgw_status sgemm(mgw_handle* h, long M, long N, long K, AOp A, BOp B, float* C, long ldc,
                        const float* bias, float beta, const char* what) {
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32));
  k_sgemm<<<grid, 256, 0, h->stream>>>(M, N, K, A, B, C, ldc, bias, beta);
  return check_launch(h, what);
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

__global__ void k_silu(long n, const float* z, float* a) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) a[i] = z[i] * sigm(z[i]);
}
__global__ void k_silu_bwd(long n, const float* z, float* d) {  // d <- d * silu'(z)
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) {
    const float s = sigm(z[i]);
    d[i] *= s * (1.f + z[i] * (1.f - s));
  }
}
__global__ void k_colsum(long rows, long cols, const float* d, float* out) {  // out[c] = sum_r d[r][c]
  long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (long r = 0; r < rows; ++r) s += d[r * cols + c];
  out[c] = s;
}
__global__ void k_round_bf16(long n, const float* p, __nv_bfloat16* w) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) w[i] = __float2bfloat16_rn(p[i]);
}
__global__ void k_adam(long n, float* p, __nv_bfloat16* w, const float* g, float* m, float* v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  w[i] = __float2bfloat16_rn(pi);
}
// dY = (Y - T) / B; loss[0] = sum (Y - T)^2 / (2B)
__global__ void k_mse(long n, long B, const float* Y, const float* T, float* dY, float* loss) {
  __shared__ float s[256];
  float acc = 0.f;
  for (long i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d / (float)B;
    acc += d * d;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = s[0] / (2.f * (float)B);
}

static unsigned nb(long n) { return (unsigned)((n + 255) / 256); }

}  // namespace mlp
}  // namespace mgw

using namespace mgw;
using namespace mgw::mlp;

extern "C" {

long mgw_mlp_nparams(int d_in, int width, int d_out) { return Offsets(d_in, width, d_out).n; }

mgw_status mgw_mlp_round(mgw_handle* h, long n, const float* params, unsigned short* wbf16) {
  if (!h || n < 1 || !params || !wbf16) return MGW_ERR_ARG;
  k_round_bf16<<<nb(n), 256, 0, h->stream>>>(n, params, reinterpret_cast<__nv_bfloat16*>(wbf16));
  return check_launch(h, "mlp_round");
}

mgw_status mgw_mlp_forward(mgw_handle* h, int d_in, int width, int d_out, const float* params,
                           const unsigned short* wbf16, int batch, const float* X, float* Y, float* acts) {
  if (!h) return MGW_ERR_ARG;
  if (d_in < 1 || width < 1 || d_out < 1 || batch < 1 || !params || !wbf16 || !X || !Y)
    return fail(h, MGW_ERR_ARG, "mgw_mlp_forward: bad arguments");
  const Offsets o(d_in, width, d_out);
  const auto* w = reinterpret_cast<const __nv_bfloat16*>(wbf16);
  const long bw = (long)batch * width;
  Arena ar;
  double* tmp = nullptr;
  if (!acts) {
    ar.add(&tmp, (4 * bw + 1) / 2);
    MGW_TRY(ar.commit(h));
    acts = reinterpret_cast<float*>(tmp);
  }
  float *z1 = acts, *a1 = acts + bw, *z2 = acts + 2 * bw, *a2 = acts + 3 * bw;
  MGW_TRY(sgemm(h, batch, width, d_in, AF32{X, d_in, 0}, BBf16{w + o.w1, d_in, 0}, z1, width, params + o.b1, 0.f,
                "mlp_fwd1"));
  k_silu<<<nb(bw), 256, 0, h->stream>>>(bw, z1, a1);
  MGW_TRY(check_launch(h, "silu"));
  MGW_TRY(sgemm(h, batch, width, width, AF32{a1, width, 0}, BBf16{w + o.w2, width, 0}, z2, width, params + o.b2,
                0.f, "mlp_fwd2"));
  k_silu<<<nb(bw), 256, 0, h->stream>>>(bw, z2, a2);
  MGW_TRY(check_launch(h, "silu"));
  MGW_TRY(sgemm(h, batch, d_out, width, AF32{a2, width, 0}, BBf16{w + o.w3, width, 0}, Y, d_out, params + o.b3,
                0.f, "mlp_fwd3"));
  return MGW_OK;
}

mgw_status mgw_mlp_backward(mgw_handle* h, int d_in, int width, int d_out, const unsigned short* wbf16, int batch,
                            const float* X, const float* acts, const float* dY, float* grad) {
  if (!h) return MGW_ERR_ARG;
  if (d_in < 1 || width < 1 || d_out < 1 || batch < 1 || !wbf16 || !X || !acts || !dY || !grad)
    return fail(h, MGW_ERR_ARG, "mgw_mlp_backward: bad arguments");
  const Offsets o(d_in, width, d_out);
  const auto* w = reinterpret_cast<const __nv_bfloat16*>(wbf16);
  const long bw = (long)batch * width;
  const float *z1 = acts, *a1 = acts + bw, *z2 = acts + 2 * bw, *a2 = acts + 3 * bw;
  Arena ar;
  double* tmp = nullptr;
  ar.add(&tmp, bw + 1);  // two [batch][width] float buffers
  MGW_TRY(ar.commit(h));
  float* d2 = reinterpret_cast<float*>(tmp);
  float* d1 = d2 + bw;
  // layer 3: gW3 = dY^T a2, gb3 = sum dY; da2 = dY W3
  MGW_TRY(sgemm(h, d_out, width, batch, AF32{dY, d_out, 1}, BF32{a2, width}, grad + o.w3, width, nullptr, 0.f,
                "mlp_bwd_w3"));
  k_colsum<<<nb(d_out), 256, 0, h->stream>>>(batch, d_out, dY, grad + o.b3);
  MGW_TRY(check_launch(h, "colsum"));
  MGW_TRY(sgemm(h, batch, width, d_out, AF32{dY, d_out, 0}, BBf16{w + o.w3, width, 1}, d2, width, nullptr, 0.f,
                "mlp_bwd_in3"));
  k_silu_bwd<<<nb(bw), 256, 0, h->stream>>>(bw, z2, d2);
  MGW_TRY(check_launch(h, "silu_bwd"));
  // layer 2
  MGW_TRY(sgemm(h, width, width, batch, AF32{d2, width, 1}, BF32{a1, width}, grad + o.w2, width, nullptr, 0.f,
                "mlp_bwd_w2"));
  k_colsum<<<nb(width), 256, 0, h->stream>>>(batch, width, d2, grad + o.b2);
  MGW_TRY(check_launch(h, "colsum"));
  MGW_TRY(sgemm(h, batch, width, width, AF32{d2, width, 0}, BBf16{w + o.w2, width, 1}, d1, width, nullptr, 0.f,
                "mlp_bwd_in2"));
  k_silu_bwd<<<nb(bw), 256, 0, h->stream>>>(bw, z1, d1);
  MGW_TRY(check_launch(h, "silu_bwd"));
  // layer 1
  MGW_TRY(sgemm(h, width, d_in, batch, AF32{d1, width, 1}, BF32{X, d_in}, grad + o.w1, d_in, nullptr, 0.f,
                "mlp_bwd_w1"));
  k_colsum<<<nb(width), 256, 0, h->stream>>>(batch, width, d1, grad + o.b1);
  return check_launch(h, "colsum");
}

mgw_status mgw_mlp_mse(mgw_handle* h, int batch, int d_out, const float* Y, const float* T, float* dY,
                       float* loss) {
  if (!h || batch < 1 || d_out < 1 || !Y || !T || !dY || !loss) return MGW_ERR_ARG;
  k_mse<<<1, 256, 0, h->stream>>>((long)batch * d_out, batch, Y, T, dY, loss);
  return check_launch(h, "mse");
}

mgw_status mgw_mlp_adam(mgw_handle* h, long n, float* params, unsigned short* wbf16, const float* grad, float* m,
                        float* v, int step, float lr) {
  if (!h || n < 1 || !params || !wbf16 || !grad || !m || !v || step < 1) return MGW_ERR_ARG;
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<nb(n), 256, 0, h->stream>>>(n, params, reinterpret_cast<__nv_bfloat16*>(wbf16), grad, m, v, lr, b1, b2,
                                       1e-8f, 1.f - powf(b1, (float)step), 1.f - powf(b2, (float)step));
  return check_launch(h, "adam");
}

}  // extern "C"
