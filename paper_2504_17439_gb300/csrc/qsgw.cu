// Static potential of quasiparticle self-consistent GW (Sec. III D,
// Eqs. 36-39) from the two block-Lanczos chains.
//
// Each chain's external block T (block tridiagonal: alpha on the diagonal,
// beta below, beta^T above) is diagonalised, T = U diag(e) U^T, and its
// couplings to the orbitals become v = [coup, 0, ..] U (pole decoupling), so
// the chain contributes sum_l v_pl v_ql / (w - e_l) to Sigma(w).  Then with
// D_pl = eps_p - e_l:
//   broadened (Eqs. 36-37): V = (A + A^T) / 2, A_pq = sum_l v_pl v_ql D_pl / (D_pl^2 + delta^2)
//   SRG (Eqs. 38-39):       V_pq = sum_l (D_pl + D_ql) / (D_pl^2 + D_ql^2) v_pl v_ql (1 - exp(-(D_pl^2 + D_ql^2) s))
// The first is a scaled GEMM; the second does not factor and runs as one
// thread per (p, q) looping over the poles.
#include "mgw_internal.h"

#include <algorithm>

namespace mgw {

// T[nb r][nb r] of one chain from its padded blocks (leading dimension nmo)
__global__ void k_chain_matrix(int nb, int r, int nmo, const double* alpha, const double* beta, double* T) {
  const long dim = (long)nb * r;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < dim * dim; idx += (long)gridDim.x * blockDim.x) {
    const long i = idx / dim, j = idx % dim;
    const long bi = i / r, bj = j / r, ii = i % r, jj = j % r;
    const long n2 = (long)nmo * nmo;
    double v = 0.0;
    if (bi == bj) v = alpha[bi * n2 + ii * nmo + jj];
    else if (bi == bj + 1) v = beta[bj * n2 + ii * nmo + jj];   // beta_{bj} below the diagonal
    else if (bj == bi + 1) v = beta[bi * n2 + jj * nmo + ii];   // its transpose above
    T[idx] = v;
  }
}

// Rv[p][l] = v[p][l] D_pl / (D_pl^2 + delta^2)
__global__ void k_broadened_rows(int nmo, int npoles, const double* eps, const double* e, const double* v,
                                 double delta, double* Rv) {
  const long total = (long)nmo * npoles;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long p = idx / npoles, l = idx % npoles;
    const double d = eps[p] - e[l];
    Rv[idx] = v[idx] * d / (d * d + delta * delta);
  }
}

__global__ void k_symmetrise(int n, const double* A, double* V) {
  const long total = (long)n * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long p = idx / n, q = idx % n;
    V[idx] = 0.5 * (A[p * n + q] + A[q * n + p]);
  }
}

__global__ void k_srg_potential(int nmo, int npoles, const double* eps, const double* e, const double* v, double s,
                                double* V) {
  const long total = (long)nmo * nmo;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long p = idx / nmo, q = idx % nmo;
    const double ep = eps[p], eq = eps[q];
    double acc = 0.0;
    for (int l = 0; l < npoles; ++l) {
      const double dp = ep - e[l], dq = eq - e[l];
      const double s2 = dp * dp + dq * dq;
      if (s2 > 0.0) acc += (dp + dq) / s2 * (-expm1(-s2 * s)) * v[p * npoles + l] * v[q * npoles + l];
    }
    V[idx] = acc;
  }
}

static unsigned grid_for(long n) { return (unsigned)std::min<long>((n + 255) / 256, 152L * 32); }

}  // namespace mgw

using namespace mgw;

extern "C" mgw_status mgw_qsgw_potential(mgw_handle* h, int nmo, int nblk, int rank_h, int rank_p,
                                         const double* eps, const double* coup_h, const double* alpha_h,
                                         const double* beta_h, const double* coup_p, const double* alpha_p,
                                         const double* beta_p, int reg, double delta, double srg_s, double* V) {
  if (!h) return MGW_ERR_ARG;
  if (nmo < 1 || nblk < 1 || rank_h < 0 || rank_h > nmo || rank_p < 0 || rank_p > nmo || !eps || !V ||
      (reg != 0 && reg != 1) || (reg == 0 && !(delta > 0.0)) || (reg == 1 && !(srg_s >= 0.0)))
    return fail(h, MGW_ERR_ARG, "mgw_qsgw_potential: bad sizes, regularisation or null pointer");
  if ((rank_h > 0 && (!coup_h || !alpha_h || (nblk > 1 && !beta_h))) ||
      (rank_p > 0 && (!coup_p || !alpha_p || (nblk > 1 && !beta_p))))
    return fail(h, MGW_ERR_ARG, "mgw_qsgw_potential: missing chain blocks");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long n2 = (long)nmo * nmo;
  const int npoles = nblk * (rank_h + rank_p);
  if (npoles == 0) {
    MGW_CUDA(h, cudaMemsetAsync(V, 0, sizeof(double) * n2, h->stream));
    return MGW_OK;
  }
  const long dmax = (long)nblk * std::max(rank_h, rank_p);
  Arena ar;
  double *T, *e, *v, *Rv, *A;
  ar.add(&T, dmax * dmax);
  ar.add(&e, npoles);
  ar.add(&v, (long)nmo * npoles);
  ar.add(&Rv, (long)nmo * npoles);
  ar.add(&A, n2);
  MGW_TRY(ar.commit(h));
  int off = 0;
  for (int sec = 0; sec < 2; ++sec) {
    const int r = sec == 0 ? rank_h : rank_p;
    if (r == 0) continue;
    const long dim = (long)nblk * r;
    k_chain_matrix<<<grid_for(dim * dim), 256, 0, h->stream>>>(nblk, r, nmo, sec == 0 ? alpha_h : alpha_p,
                                                              sec == 0 ? beta_h : beta_p, T);
    MGW_TRY(check_launch(h, "qsgw_chain_matrix"));
    MGW_TRY(syevd(h, (int)dim, T, e + off));  // rows of T: eigenvectors
    // v[:, off + l] = coup[:, :r] U[:r, l], U[k][l] = T[l][k]
    MGW_TRY(gemm_nt(h, nmo, dim, r, 1.0, sec == 0 ? coup_h : coup_p, nmo, T, dim, 0.0, v + off, npoles));
    off += (int)dim;
  }
  if (reg == 0) {
    k_broadened_rows<<<grid_for((long)nmo * npoles), 256, 0, h->stream>>>(nmo, npoles, eps, e, v, delta, Rv);
    MGW_TRY(check_launch(h, "qsgw_broadened_rows"));
    MGW_TRY(gemm_nt(h, nmo, nmo, npoles, 1.0, Rv, npoles, v, npoles, 0.0, A, nmo));
    k_symmetrise<<<grid_for(n2), 256, 0, h->stream>>>(nmo, A, V);
    return check_launch(h, "qsgw_symmetrise");
  }
  k_srg_potential<<<grid_for(n2), 256, 0, h->stream>>>(nmo, npoles, eps, e, v, srg_s, V);
  return check_launch(h, "qsgw_srg_potential");
}
