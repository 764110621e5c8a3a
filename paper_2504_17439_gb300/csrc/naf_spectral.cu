// Natural auxiliary functions (Sec. II D, Eq. 14) and the spectral function
// of the upfolded Hamiltonian's poles (Eqs. 11-12).
//
// NAF: M = V V^T over the orbital pairs (all, or all but virtual-virtual),
// eigendecomposed; the eigenvectors with eigenvalue above eps_naf (absolute)
// become the new auxiliary functions, L'_{A,pq} = sum_P U_{PA} L_{P,pq}.
// The pair product is the FP64 GEMM with upper-triangle tiles mirrored (M is
// symmetric), the eigensolve is cuSOLVER syevd, the projection a plain GEMM.
//
// Spectral function: A(w) = (1/pi) sum_a weight_a delta / ((w - E_a)^2 +
// delta^2), one thread per frequency with the poles staged through shared
// memory in tiles; FP64 arithmetic (bound by the FP64 pipe).
#include "mgw_internal.h"

#include <algorithm>
#include <vector>

namespace mgw {

// V[P][j] over the pairs of Eq. 14 without the virtual-virtual block:
// j < nocc nmo -> (v, w) = (j / nmo, j % nmo); then (nocc + j' / nocc, j' % nocc)
__global__ void k_gather_pairs_no_vv(int naux, int nocc, int nmo, const double* __restrict__ L, double* V) {
  const long np = (long)nocc * nmo + (long)(nmo - nocc) * nocc;
  const long total = (long)naux * np;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long P = i / np, j = i % np;
    long v, w;
    if (j < (long)nocc * nmo) {
      v = j / nmo;
      w = j % nmo;
    } else {
      const long jj = j - (long)nocc * nmo;
      v = nocc + jj / nocc;
      w = jj % nocc;
    }
    V[i] = L[((long)P * nmo + v) * nmo + w];
  }
}

// U[a][:] = evec[n - 1 - a][:] for a < k (rows of the k largest eigenvalues,
// descending); lam_desc[i] = lam_asc[n - 1 - i]
__global__ void k_top_rows(int n, int k, const double* __restrict__ evec, const double* __restrict__ lam_asc,
                           double* U, double* lam_desc) {
  const long total = (long)k * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long a = i / n, c = i % n;
    U[i] = evec[(long)(n - 1 - a) * n + c];
  }
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    lam_desc[i] = lam_asc[n - 1 - i];
}

constexpr int kPoleTile = 256;

__global__ void __launch_bounds__(kPoleTile) k_spectral(int dim, const double* __restrict__ E,
                                                        const double* __restrict__ weight, double delta, int nw,
                                                        const double* __restrict__ omega, double* A) {
  __shared__ double sE[kPoleTile], sW[kPoleTile];
  const int j = blockIdx.x * kPoleTile + threadIdx.x;
  const double w = j < nw ? omega[j] : 0.0;
  const double d2 = delta * delta;
  double acc = 0.0;
  for (int a0 = 0; a0 < dim; a0 += kPoleTile) {
    const int a = a0 + threadIdx.x;
    sE[threadIdx.x] = a < dim ? E[a] : 0.0;
    sW[threadIdx.x] = a < dim ? weight[a] : 0.0;
    __syncthreads();
    const int na = min(kPoleTile, dim - a0);
    for (int b = 0; b < na; ++b) {
      const double d = w - sE[b];
      acc += sW[b] / (d * d + d2);
    }
    __syncthreads();
  }
  if (j < nw) A[j] = acc * (delta / 3.141592653589793);
}

}  // namespace mgw

using namespace mgw;

extern "C" mgw_status mgw_naf_compress(mgw_handle* h, int nocc, int nvir, int naux, const double* L,
                                       double eps_naf, int all_pairs, double* L_naf, double* lam, int* n_naf) {
  if (!h) return MGW_ERR_ARG;
  if (nocc < 1 || nvir < 0 || naux < 1 || !L || !L_naf || !lam || !n_naf)
    return fail(h, MGW_ERR_ARG, "mgw_naf_compress: bad sizes or null pointer");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const int nmo = nocc + nvir;
  const long n2 = (long)nmo * nmo;
  const long np = all_pairs ? n2 : (long)nocc * nmo + (long)nvir * nocc;
  Arena ar;
  double *V = nullptr, *M = nullptr, *lam_asc = nullptr, *U = nullptr;
  if (!all_pairs) ar.add(&V, (size_t)naux * np);
  ar.add(&M, (size_t)naux * naux);
  ar.add(&lam_asc, naux);
  ar.add(&U, (size_t)naux * naux);
  MGW_TRY(ar.commit(h));
  const double* Vp = L;
  if (!all_pairs) {
    const long total = (long)naux * np;
    k_gather_pairs_no_vv<<<(unsigned)std::min<long>((total + 255) / 256, 152L * 32), 256, 0, h->stream>>>(
        naux, nocc, nmo, L, V);
    MGW_TRY(check_launch(h, "naf_gather_pairs"));
    Vp = V;
  }
  // M = V V^T (Eq. 14): symmetric, upper tiles mirrored
  MGW_TRY((dgemm<64, 64>(h, naux, naux, np, 1, ARowMajor{Vp, np, 0}, BNMajor{Vp, np, 0},
                         EpiStore{M, naux, 0, 1.0, 0.0}, "naf_metric", /*tri=*/1)));
  MGW_TRY(syevd(h, naux, M, lam_asc));
  std::vector<double> hl(naux);
  MGW_CUDA(h, cudaMemcpyAsync(hl.data(), lam_asc, sizeof(double) * naux, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  int k = 0;
  for (int i = 0; i < naux; ++i) k += hl[i] > eps_naf ? 1 : 0;
  const long rows = std::max(k, 1);
  k_top_rows<<<(unsigned)std::min<long>((rows * naux + 255) / 256, 152L * 32), 256, 0, h->stream>>>(
      naux, k, M, lam_asc, U, lam);
  MGW_TRY(check_launch(h, "naf_top_rows"));
  // L'[a][pq] = sum_P U[a][P] L[P][pq]
  if (k > 0) MGW_TRY(gemm_nn(h, k, n2, naux, 1.0, U, naux, L, n2, 0.0, L_naf, n2));
  *n_naf = k;
  return MGW_OK;
}

extern "C" mgw_status mgw_spectral_function(mgw_handle* h, int dim, const double* E, const double* weight,
                                            double delta, int nomega, const double* omega, double* A) {
  if (!h) return MGW_ERR_ARG;
  if (dim < 1 || nomega < 1 || !(delta > 0.0) || !E || !weight || !omega || !A)
    return fail(h, MGW_ERR_ARG, "mgw_spectral_function: bad sizes, delta or null pointer");
  MGW_CUDA(h, cudaSetDevice(h->device));
  k_spectral<<<(unsigned)((nomega + kPoleTile - 1) / kPoleTile), kPoleTile, 0, h->stream>>>(dim, E, weight, delta,
                                                                                            nomega, omega, A);
  return check_launch(h, "spectral_function");
}
