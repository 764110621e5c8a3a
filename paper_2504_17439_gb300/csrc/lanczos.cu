// Moment-driven block Lanczos for one self-energy sector (Eqs. 9-10), FP64.
//
// Given Sigma(n), n = 0..2 nblk - 1, find the coupling S0^(1/2) and the
// blocks alpha_i, beta_i of a block tridiagonal T with
//   Sigma(n) = S0^(1/2) (T^n)_{00} S0^(1/2).
// The recurrence runs on inner products that are moments: the Lanczos
// vectors are carried as coefficient lists Q_i = sum_k H^k Q_0 C_{i,k}, so
// <Q_i, H^m Q_j> = sum_{k,l} C_{i,k}^T S^(k+l+m) C_{j,l}, with
// S^(n) = S0^(-1/2) M(n) S0^(-1/2) / s^n the normalised, centred, scaled
// moments.  Every square root is the symmetric PSD one (so the blocks are
// unique); inverse square roots drop eigenvalues below rank_tol * max.
#include "mgw_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mgw {

__global__ void k_symmetrize_copy(int n, const double* src, double* dst) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)n * n) return;
  int r = (int)(i / n), c = (int)(i % n);
  dst[i] = 0.5 * (src[(long)r * n + c] + src[(long)c * n + r]);
}

__global__ void k_traces(int n, int cnt, const double* a, double* tr) {
  // one block per matrix
  int b = blockIdx.x;
  if (b >= cnt) return;
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += a[(long)b * n * n + (long)i * n + i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) tr[b] = s[0];
}

// M(n) = sum_k coef[n][k] S(k), coef row-major [cnt][cnt]
struct CenterCoef { double c[24 * 24]; };
__global__ void k_center(long nn, int cnt, const double* S, double* M, CenterCoef cf) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  double v[24];
  for (int k = 0; k < cnt; ++k) v[k] = S[(long)k * nn + i];
  for (int n = 0; n < cnt; ++n) {
    double acc = 0.0;
    for (int k = 0; k <= n; ++k) acc = fma(cf.c[n * 24 + k], v[k], acc);
    M[(long)n * nn + i] = acc;
  }
}

// rows of V (eigenvectors) scaled: out[a][i] = V[row0 + a][i] * f(lambda[row0 + a])
__global__ void k_scale_rows(int r, int n, const double* V, int row0, const double* lam, double powr,
                             double* out, long ldo) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)r * n) return;
  int a = (int)(i / n), c = (int)(i % n);
  out[(long)a * ldo + c] = V[(long)(row0 + a) * n + c] * pow(lam[row0 + a], powr);
}

__global__ void k_axpby_identity(int r, double* a, long lda, double s, double c) {  // a = s a + c I
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)r * r) return;
  int p = (int)(i / r), q = (int)(i % r);
  double v = s * a[(long)p * lda + q];
  if (p == q) v += c;
  a[(long)p * lda + q] = v;
}

__global__ void k_copy2d(int rows, int cols, const double* src, long lds, double* dst, long ldd) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)rows * cols) return;
  int p = (int)(i / cols), q = (int)(i % cols);
  dst[(long)p * ldd + q] = src[(long)p * lds + q];
}

static unsigned nb(long n) { return (unsigned)((n + 255) / 256); }

struct PsdRoot {
  // symmetric square root and pseudo-inverse square root of an r x r PSD matrix
  static mgw_status run(mgw_handle* h, int r, const double* S, double rank_tol, double floor, double* sq,
                        double* isq, double* evec, double* lam, double* tmp, int* rank_out) {
    MGW_CUDA(h, cudaMemcpyAsync(evec, S, sizeof(double) * r * r, cudaMemcpyDeviceToDevice, h->stream));
    MGW_TRY(syevd(h, r, evec, lam));
    std::vector<double> hl(r);
    MGW_CUDA(h, cudaMemcpyAsync(hl.data(), lam, sizeof(double) * r, cudaMemcpyDeviceToHost, h->stream));
    MGW_CUDA(h, cudaStreamSynchronize(h->stream));
    double lmax = std::max(std::max(hl[r - 1], 0.0), floor);
    int kept = 0;
    for (int i = 0; i < r; ++i)
      if (lmax > 0 && hl[i] > rank_tol * lmax) ++kept;
    int row0 = r - kept;
    *rank_out = kept;
    MGW_CUDA(h, cudaMemsetAsync(sq, 0, sizeof(double) * r * r, h->stream));
    MGW_CUDA(h, cudaMemsetAsync(isq, 0, sizeof(double) * r * r, h->stream));
    if (kept == 0) return MGW_OK;
    // sq = V_k^T diag(sqrt l) V_k,  isq = V_k^T diag(1/sqrt l) V_k   (rows of evec are eigenvectors)
    k_scale_rows<<<nb((long)kept * r), 256, 0, h->stream>>>(kept, r, evec, row0, lam, 0.5, tmp, r);
    MGW_TRY(check_launch(h, "scale_rows"));
    MGW_TRY(gemm_tn(h, r, r, kept, 1.0, evec + (long)row0 * r, r, tmp, r, 0.0, sq, r));
    k_scale_rows<<<nb((long)kept * r), 256, 0, h->stream>>>(kept, r, evec, row0, lam, -0.5, tmp, r);
    MGW_TRY(check_launch(h, "scale_rows"));
    MGW_TRY(gemm_tn(h, r, r, kept, 1.0, evec + (long)row0 * r, r, tmp, r, 0.0, isq, r));
    return MGW_OK;
  }
};

}  // namespace mgw

using namespace mgw;

extern "C" mgw_status mgw_block_lanczos(mgw_handle* h, const mgw_options* o, int nmo, int nmom, const double* sig,
                                        double* coup, double* alpha, double* beta, int* rank) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (nmo < 1 || nmom < 2 || nmom > 24 || (nmom % 2) || !sig || !coup || !alpha || !rank)
    return fail(h, MGW_ERR_ARG, "mgw_block_lanczos: bad sizes or null pointer");
  const int nblk = nmom / 2;
  if (nblk > 1 && !beta) return fail(h, MGW_ERR_ARG, "mgw_block_lanczos: beta is NULL");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long n2 = (long)nmo * nmo;
  const int cnt = 2 * nblk;

  // workspace: S[cnt] M[cnt] Sh[cnt] evec lam tmp tmp2 sq isq + coefficient lists
  const int ncoef = nblk * (nblk + 1) / 2 + 2 * (nblk + 1);
  Arena ar;
  double *S, *M, *Sh, *evec, *lam, *tmp, *tmp2, *sq, *isq, *Pt, *tr, *coefs, *Vr, *lam0;
  ar.add(&S, cnt * n2);
  ar.add(&M, cnt * n2);
  ar.add(&Sh, cnt * n2);
  ar.add(&evec, n2);
  ar.add(&lam, nmo);
  ar.add(&tmp, n2);
  ar.add(&tmp2, n2);
  ar.add(&sq, n2);
  ar.add(&isq, n2);
  ar.add(&Pt, n2);
  ar.add(&Vr, n2);
  ar.add(&lam0, nmo);
  ar.add(&tr, 2 * cnt);
  ar.add(&coefs, (size_t)ncoef * n2);
  MGW_TRY(ar.commit(h));

  for (int n = 0; n < cnt; ++n)
    k_symmetrize_copy<<<nb(n2), 256, 0, h->stream>>>(nmo, sig + n * n2, S + n * n2);
  MGW_TRY(check_launch(h, "symmetrize"));
  k_traces<<<cnt, 256, 0, h->stream>>>(nmo, cnt, S, tr);
  MGW_TRY(check_launch(h, "traces"));
  std::vector<double> htr(cnt);
  MGW_CUDA(h, cudaMemcpyAsync(htr.data(), tr, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  const double tr0 = htr[0];
  const double c = tr0 > 0 ? htr[1] / tr0 : 0.0;
  if (!std::isfinite(c)) return fail(h, MGW_ERR_ARG, "mgw_block_lanczos: non-finite moments");

  // centre: M(n) = sum_k C(n,k) (-c)^(n-k) S(k)
  CenterCoef cf{};
  for (int n = 0; n < cnt; ++n) {
    double bin = 1.0;
    for (int k = n; k >= 0; --k) {
      // C(n,k) with k descending: start at C(n,n) = 1
      cf.c[n * 24 + k] = bin * std::pow(-c, n - k);
      bin = bin * k / (n - k + 1);
    }
  }
  k_center<<<nb(n2), 256, 0, h->stream>>>(n2, cnt, S, M, cf);
  MGW_TRY(check_launch(h, "center"));
  k_traces<<<cnt, 256, 0, h->stream>>>(nmo, cnt, M, tr);
  MGW_TRY(check_launch(h, "traces"));
  MGW_CUDA(h, cudaMemcpyAsync(htr.data(), tr, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  const int top = cnt - 2;
  double s = 1.0;
  if (top > 0 && tr0 > 0 && htr[top] > 0) s = std::pow(htr[top] / htr[0], 1.0 / top);

  // zero the outputs (padding stays zero when the rank is deficient)
  MGW_CUDA(h, cudaMemsetAsync(coup, 0, sizeof(double) * n2, h->stream));
  MGW_CUDA(h, cudaMemsetAsync(alpha, 0, sizeof(double) * nblk * n2, h->stream));
  if (nblk > 1) MGW_CUDA(h, cudaMemsetAsync(beta, 0, sizeof(double) * (nblk - 1) * n2, h->stream));

  // eigen-decomposition of M(0) = Sigma(0)
  MGW_CUDA(h, cudaMemcpyAsync(evec, M, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
  MGW_TRY(syevd(h, nmo, evec, lam));
  std::vector<double> hl(nmo);
  MGW_CUDA(h, cudaMemcpyAsync(hl.data(), lam, sizeof(double) * nmo, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  const double lmax = std::max(hl[nmo - 1], 0.0);
  int r = 0;
  for (int i = 0; i < nmo; ++i)
    if (lmax > 0 && hl[i] > o->rank_tol * lmax) ++r;
  *rank = r;
  if (r == 0) return MGW_OK;
  const int row0 = nmo - r;
  const bool full = r == nmo;
  const long r2 = (long)r * r;
  // keep the retained eigenvectors (rows) and eigenvalues of Sigma(0)
  MGW_CUDA(h, cudaMemcpyAsync(Vr, evec + (long)row0 * nmo, sizeof(double) * r * nmo, cudaMemcpyDeviceToDevice,
                              h->stream));
  MGW_CUDA(h, cudaMemcpyAsync(lam0, lam + row0, sizeof(double) * r, cudaMemcpyDeviceToDevice, h->stream));

  // Pt = diag(lambda^-1/2) V_r  (r x nmo);  Sh(n) = Pt M(n) Pt^T / s^n
  k_scale_rows<<<nb((long)r * nmo), 256, 0, h->stream>>>(r, nmo, evec, row0, lam, -0.5, Pt, nmo);
  MGW_TRY(check_launch(h, "scale_rows"));
  for (int n = 0; n < cnt; ++n) {
    MGW_TRY(gemm_nn(h, r, nmo, nmo, 1.0, Pt, nmo, M + n * n2, nmo, 0.0, tmp, nmo));
    MGW_TRY(gemm_nt(h, r, r, nmo, 1.0 / std::pow(s, n), tmp, nmo, Pt, nmo, 0.0, Sh + n * r2, r));
  }

  // coefficient lists: C[i][k], k = 0..i, each r x r; R[k], k = 0..i+1
  std::vector<std::vector<double*>> C(nblk);
  double* next = coefs;
  auto take = [&]() { double* p = next; next += r2; return p; };
  std::vector<double*> R(nblk + 1);
  for (int k = 0; k <= nblk; ++k) R[k] = take();
  double* RR = take();
  std::vector<double*> hbeta(nblk);  // beta_{i} (r x r, scaled)
  for (int i = 0; i < nblk; ++i) {
    C[i].resize(i + 1);
    for (int k = 0; k <= i; ++k) C[i][k] = take();
  }
  for (int i = 1; i < nblk; ++i) hbeta[i] = take();
  std::vector<double*> halpha(nblk);
  // scaled alpha blocks (r x r) live in M, which is no longer needed
  for (int i = 0; i < nblk; ++i) halpha[i] = M + (long)i * r2;

  // C[0][0] = I
  MGW_CUDA(h, cudaMemsetAsync(C[0][0], 0, sizeof(double) * r2, h->stream));
  MGW_TRY(add_identity(h, r, C[0][0], 1.0));

  // inner(X, Y, m) = sum_{k,l} X_k^T Sh(k+l+m) Y_l  -> out (r x r)
  auto inner = [&](const std::vector<double*>& X, const std::vector<double*>& Y, int m, double* out) -> mgw_status {
    MGW_CUDA(h, cudaMemsetAsync(out, 0, sizeof(double) * r2, h->stream));
    for (size_t k = 0; k < X.size(); ++k) {
      for (size_t l = 0; l < Y.size(); ++l)
        MGW_TRY(gemm_nn(h, r, r, r, 1.0, Sh + (long)(k + l + m) * r2, r, Y[l], r, l == 0 ? 0.0 : 1.0, tmp, r));
      MGW_TRY(gemm_tn(h, r, r, r, 1.0, X[k], r, tmp, r, 1.0, out, r));
    }
    return MGW_OK;
  };

  for (int i = 0; i < nblk; ++i) {
    MGW_TRY(inner(C[i], C[i], 1, tmp2));
    k_symmetrize_copy<<<nb(r2), 256, 0, h->stream>>>(r, tmp2, halpha[i]);
    MGW_TRY(check_launch(h, "symmetrize"));
    if (i == nblk - 1) break;
    // R_k = C[i][k-1] - C[i][k] alpha_i - C[i-1][k] beta_i^T
    std::vector<double*> Rl(R.begin(), R.begin() + i + 2);
    for (int k = 0; k <= i + 1; ++k) {
      MGW_CUDA(h, cudaMemsetAsync(Rl[k], 0, sizeof(double) * r2, h->stream));
      if (k >= 1)
        MGW_CUDA(h, cudaMemcpyAsync(Rl[k], C[i][k - 1], sizeof(double) * r2, cudaMemcpyDeviceToDevice, h->stream));
      if (k <= i) MGW_TRY(gemm_nn(h, r, r, r, -1.0, C[i][k], r, halpha[i], r, 1.0, Rl[k], r));
      if (i >= 1 && k <= i - 1) MGW_TRY(gemm_nt(h, r, r, r, -1.0, C[i - 1][k], r, hbeta[i], r, 1.0, Rl[k], r));
    }
    MGW_TRY(inner(Rl, Rl, 0, RR));
    int rb = 0;
    // rank of the normalised residual judged against max(lambda_max, 1); a
    // vanishing residual gives beta = 0 and a decoupled remainder of the chain
    MGW_TRY(PsdRoot::run(h, r, RR, o->rank_tol, 1.0, hbeta[i + 1], sq, evec, lam, tmp2, &rb));
    for (int k = 0; k <= i + 1; ++k) MGW_TRY(gemm_nn(h, r, r, r, 1.0, Rl[k], r, sq, r, 0.0, C[i + 1][k], r));
  }

  // unscale: alpha = s alpha' + c I, beta = s beta'; then rotate to the orbital basis when full rank
  for (int i = 0; i < nblk; ++i) {
    k_axpby_identity<<<nb(r2), 256, 0, h->stream>>>(r, halpha[i], r, s, c);
    MGW_TRY(check_launch(h, "unscale"));
  }
  for (int i = 1; i < nblk; ++i) {
    k_axpby_identity<<<nb(r2), 256, 0, h->stream>>>(r, hbeta[i], r, s, 0.0);
    MGW_TRY(check_launch(h, "unscale"));
  }
  if (full) {
    for (int i = 0; i < nblk; ++i) {
      MGW_TRY(gemm_tn(h, nmo, nmo, nmo, 1.0, Vr, nmo, halpha[i], nmo, 0.0, tmp, nmo));
      MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, tmp, nmo, Vr, nmo, 0.0, alpha + i * n2, nmo));
    }
    for (int i = 1; i < nblk; ++i) {
      MGW_TRY(gemm_tn(h, nmo, nmo, nmo, 1.0, Vr, nmo, hbeta[i], nmo, 0.0, tmp, nmo));
      MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, tmp, nmo, Vr, nmo, 0.0, beta + (i - 1) * n2, nmo));
    }
    // coup = V^T diag(lambda^1/2) V
    k_scale_rows<<<nb(n2), 256, 0, h->stream>>>(nmo, nmo, Vr, 0, lam0, 0.5, tmp, nmo);
    MGW_TRY(check_launch(h, "scale_rows"));
    MGW_TRY(gemm_tn(h, nmo, nmo, nmo, 1.0, Vr, nmo, tmp, nmo, 0.0, coup, nmo));
  } else {
    for (int i = 0; i < nblk; ++i) {
      k_copy2d<<<nb(r2), 256, 0, h->stream>>>(r, r, halpha[i], r, alpha + i * n2, nmo);
      MGW_TRY(check_launch(h, "copy2d"));
    }
    for (int i = 1; i < nblk; ++i) {
      k_copy2d<<<nb(r2), 256, 0, h->stream>>>(r, r, hbeta[i], r, beta + (i - 1) * n2, nmo);
      MGW_TRY(check_launch(h, "copy2d"));
    }
    // coup[i][a] = V[a][i] * sqrt(lambda_a)  (nmo x r in the leading columns)
    k_scale_rows<<<nb((long)r * nmo), 256, 0, h->stream>>>(r, nmo, Vr, 0, lam0, 0.5, tmp, nmo);
    MGW_TRY(check_launch(h, "scale_rows"));
    // transpose tmp (r x nmo) into coup (nmo x r, ld nmo)
    MGW_TRY(gemm_tn(h, nmo, r, r, 1.0, tmp, nmo, C[0][0], r, 0.0, coup, nmo));
  }
  return MGW_OK;
}
