// The DF tensor carried to the quasi-molecular orbitals (QMOs) of the
// upfolded Hamiltonian, the step that scGW, GW0 and G0W (Algorithm 5, Sec.
// III E) take between iterations: with chi_px the physical rows of H~'s
// eigenvectors (one column per pole x) and the first m poles occupied
// (Aufbau, Eq. 40),
//   Lt[Q][x][p]   = sum_q L[Q][p][q] chi[q][x]            (V^_{Q,px}, x-major)
//   Via[Q][i][a]  = sum_p chi[p][i] Lt[Q][m + a][p],  i < m <= m + a < nx.
// Lt is the x-major layout mgw_sigma_moments_x reads; Via is the
// particle-hole block of the next response (i a over occupied x virtual
// QMOs).  Both are batched FP64 GEMMs over Q.
#include "mgw_internal.h"

using namespace mgw;

extern "C" mgw_status mgw_qmo_tensors(mgw_handle* h, int nmo, int naux, int nx, int m, const double* L,
                                      const double* chi, double* Lt, double* Via) {
  if (!h) return MGW_ERR_ARG;
  if (nmo < 1 || naux < 1 || nx < 1 || m < 0 || m > nx || !L || !chi || !Lt || (m > 0 && m < nx && !Via))
    return fail(h, MGW_ERR_ARG, "mgw_qmo_tensors: bad sizes or null pointer");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long n2 = (long)nmo * nmo, sx = (long)nx * nmo;
  // Lt_Q = chi^T L_Q (L_Q symmetric): A(x, q) = chi[q][x], B(q, p) = L_Q[q][p]
  MGW_TRY((dgemm<64, 64>(h, nx, nmo, nmo, naux, AKMajor2{chi, nmo + 1L, 0, nx, 0}, BRowMajor{L, nmo, n2},
                         EpiStore{Lt, nmo, sx, 1.0, 0.0}, "qmo_rotate")));
  if (m == 0 || m == nx) return MGW_OK;
  // Via_Q = chi[:, :m]^T Lt_Q[m:, :]^T: A(i, p) = chi[p][i], B(p, a) = Lt_Q[m + a][p]
  const long nv = nx - m;
  MGW_TRY((dgemm<64, 64>(h, m, nv, nmo, naux, AKMajor2{chi, nmo + 1L, 0, nx, 0}, BNMajor{Lt + (long)m * nmo, nmo, sx},
                         EpiStore{Via, nv, (long)m * nv, 1.0, 0.0}, "qmo_particle_hole")));
  return MGW_OK;
}
