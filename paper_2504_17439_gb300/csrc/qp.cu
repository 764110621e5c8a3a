// Upfolded Hamiltonian (Eq. 9), its eigenvalues and the physical rows of its
// eigenvectors (tridiag.cu: only those rows are formed), QP energies
// (Eq. 34), Aufbau chemical potential and correlated density (Eq. 40), FP64.
#include "mgw_internal.h"

#include <cmath>

namespace mgw {

static unsigned nblocks(long n) { return (unsigned)((n + 255) / 256); }

// dst[(r0 + i) * ld + c0 + j] = src[i * lds + j] (+ shift on the diagonal); and the transpose
// at (c0 + j, r0 + i) when `mirror`.
__global__ void k_place(int rows, int cols, const double* src, long lds, double* H, long ld, long r0, long c0,
                        double diag_shift, int mirror) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)rows * cols) return;
  int i = (int)(idx / cols), j = (int)(idx % cols);
  double v = src[(long)i * lds + j];
  if (i == j && diag_shift != 0.0) v += diag_shift;
  H[(r0 + i) * ld + c0 + j] = v;
  if (mirror) H[(c0 + j) * ld + r0 + i] = v;
}

// weight[a] = sum_p chi[p][a]^2 (chi: the physical rows of the eigenvectors)
__global__ void k_weights(int dim, int nmo, const double* __restrict__ chi, double* weight) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= dim) return;
  double acc = 0.0;
  for (int p = 0; p < nmo; ++p) {
    const double v = chi[(long)p * dim + a];
    acc += v * v;
  }
  weight[a] = acc;
}

// eps_qp[p] = E[argmax_a chi[p][a]^2], ties to the lowest a
__global__ void k_qp_argmax(int dim, int nmo, const double* __restrict__ chi, const double* E, double* eps_qp) {
  const int p = blockIdx.x;
  if (p >= nmo) return;
  __shared__ double sv[256];
  __shared__ int si[256];
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int a = threadIdx.x; a < dim; a += blockDim.x) {
    double v = chi[(long)p * dim + a];
    v *= v;
    if (v > best || (v == best && a < bi)) { best = v; bi = a; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double v = sv[threadIdx.x + w];
      int i = si[threadIdx.x + w];
      if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && i < si[threadIdx.x])) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = i;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) eps_qp[p] = E[si[0]];
}

// Aufbau: sequential cumulative N(m) = 2 sum_{a<m} weight[a] (same order as a
// plain running sum), m minimising |N(m) - nelec| with ties to the smaller m.
__global__ void k_aufbau(int dim, const double* E, const double* weight, double nelec, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double cum = 0.0, best = fabs(0.0 - nelec), nbest = 0.0;
  int m = 0;
  for (int a = 0; a < dim; ++a) {
    cum += weight[a];
    double Nm = 2.0 * cum;
    double err = fabs(Nm - nelec);
    if (err < best) { best = err; m = a + 1; nbest = Nm; }
  }
  double mu;
  if (m == 0) mu = E[0] - 1.0;
  else if (m == dim) mu = E[dim - 1] + 1.0;
  else mu = 0.5 * (E[m - 1] + E[m]);
  out[0] = mu;
  out[1] = nbest;
  out[2] = (double)m;
}

}  // namespace mgw

using namespace mgw;

extern "C" mgw_status mgw_qp_solve(mgw_handle* h, const mgw_options* o, int nmo, int nblk, int rank_h, int rank_p,
                                   const double* fock, const double* coup_h, const double* alpha_h,
                                   const double* beta_h, const double* coup_p, const double* alpha_p,
                                   const double* beta_p, double zeta, double nelec, double* E, double* weight,
                                   double* chi_phys, double* eps_qp, double* rho, double* mu_host,
                                   double* nelec_host, int* m_host) {
  if (!h) return MGW_ERR_ARG;
  (void)o;
  if (nmo < 1 || nblk < 1 || rank_h < 0 || rank_h > nmo || rank_p < 0 || rank_p > nmo || !fock || !E || !weight ||
      !eps_qp || !std::isfinite(zeta) || !std::isfinite(nelec))
    return fail(h, MGW_ERR_ARG, "mgw_qp_solve: bad arguments");
  if ((rank_h > 0 && (!coup_h || !alpha_h || (nblk > 1 && !beta_h))) ||
      (rank_p > 0 && (!coup_p || !alpha_p || (nblk > 1 && !beta_p))))
    return fail(h, MGW_ERR_ARG, "mgw_qp_solve: null block pointer");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long n2 = (long)nmo * nmo;
  const long dim = nmo + (long)nblk * (rank_h + rank_p);
  Arena ar;
  double *H, *scal;
  ar.add(&H, dim * dim);
  ar.add(&scal, 4);
  MGW_TRY(ar.commit(h));
  MGW_CUDA(h, cudaMemsetAsync(H, 0, sizeof(double) * dim * dim, h->stream));
  k_place<<<nblocks(n2), 256, 0, h->stream>>>(nmo, nmo, fock, nmo, H, dim, 0, 0, 0.0, 0);
  MGW_TRY(check_launch(h, "place"));
  long off = nmo;
  for (int sec = 0; sec < 2; ++sec) {
    const int r = sec == 0 ? rank_h : rank_p;
    const double* cp = sec == 0 ? coup_h : coup_p;
    const double* al = sec == 0 ? alpha_h : alpha_p;
    const double* be = sec == 0 ? beta_h : beta_p;
    if (r == 0) continue;
    // coupling: physical rows x first block of the chain (nmo x r, ld nmo), and its transpose
    k_place<<<nblocks((long)nmo * r), 256, 0, h->stream>>>(nmo, r, cp, nmo, H, dim, 0, off, 0.0, 1);
    MGW_TRY(check_launch(h, "place"));
    for (int i = 0; i < nblk; ++i) {
      long o0 = off + (long)i * r;
      k_place<<<nblocks((long)r * r), 256, 0, h->stream>>>(r, r, al + i * n2, nmo, H, dim, o0, o0, zeta, 0);
      MGW_TRY(check_launch(h, "place"));
      if (i + 1 < nblk) {  // beta_{i+1} below the diagonal, its transpose above
        k_place<<<nblocks((long)r * r), 256, 0, h->stream>>>(r, r, be + i * n2, nmo, H, dim, o0 + r, o0, 0.0, 1);
        MGW_TRY(check_launch(h, "place"));
      }
    }
    off += (long)nblk * r;
  }
  // eigenvalues (ascending) and the physical rows of the eigenvectors only
  double* chi = chi_phys;
  if (!chi) MGW_TRY(slot_buffer(h, 84, (size_t)nmo * dim, &chi));
  MGW_TRY(eig_physical_rows(h, (int)dim, nmo, H, E, chi, dim));
  k_weights<<<(unsigned)((dim + 127) / 128), 128, 0, h->stream>>>((int)dim, nmo, chi, weight);
  MGW_TRY(check_launch(h, "weights"));
  k_qp_argmax<<<nmo, 256, 0, h->stream>>>((int)dim, nmo, chi, E, eps_qp);
  MGW_TRY(check_launch(h, "qp_argmax"));
  k_aufbau<<<1, 32, 0, h->stream>>>((int)dim, E, weight, nelec, scal);
  MGW_TRY(check_launch(h, "aufbau"));
  double hs[3];
  MGW_CUDA(h, cudaMemcpyAsync(hs, scal, sizeof hs, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  const int m = (int)hs[2];
  if (mu_host) *mu_host = hs[0];
  if (nelec_host) *nelec_host = hs[1];
  if (m_host) *m_host = m;
  if (rho) {
    if (m == 0) {
      MGW_CUDA(h, cudaMemsetAsync(rho, 0, sizeof(double) * n2, h->stream));
    } else {
      // rho[p][q] = 2 sum_{a<m} chi[p][a] chi[q][a]
      MGW_TRY(gemm_nt(h, nmo, nmo, m, 2.0, chi, dim, chi, dim, 0.0, rho, nmo));
    }
  }
  return MGW_OK;
}
