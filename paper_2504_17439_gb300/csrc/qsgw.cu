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

// ---------------------------------------------------------------------------
// One outer step of qsGW (Sec. III D, Eq. 35; reading of the loop: the
// static potential is built in the orbitals of the GW step, carried to the
// reference basis as C V C^T and held fixed while the field is solved).

namespace mgw {

__global__ void k_density_from_columns(int nmo, int nocc, const double* C, double* rho) {  // rho = 2 C_occ C_occ^T
  const long n2 = (long)nmo * nmo;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n2; idx += (long)gridDim.x * blockDim.x) {
    const long p = idx / nmo, q = idx % nmo;
    double acc = 0.0;
    for (int i = 0; i < nocc; ++i) acc += C[p * nmo + i] * C[q * nmo + i];
    rho[idx] = 2.0 * acc;
  }
}
__global__ void k_rows_to_columns(int n, const double* a, double* b) {  // b = a^T
  const long n2 = (long)n * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n2; idx += (long)gridDim.x * blockDim.x)
    b[(idx % n) * n + idx / n] = a[idx];
}
// out[0] = max |a - b|, out[1] = max |c| (one block)
__global__ void k_two_maxabs(long n, const double* a, const double* b, const double* c, double* out) {
  __shared__ double s0[256], s1[256];
  double m0 = 0.0, m1 = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) {
    m0 = fmax(m0, fabs(a[i] - b[i]));
    m1 = fmax(m1, fabs(c[i]));
  }
  s0[threadIdx.x] = m0;
  s1[threadIdx.x] = m1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s0[threadIdx.x] = fmax(s0[threadIdx.x], s0[threadIdx.x + w]);
      s1[threadIdx.x] = fmax(s1[threadIdx.x], s1[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s0[0];
    out[1] = s1[0];
  }
}
// dots[j] = <x, ys[j]>, one block per j
__global__ void k_gram_row(long n, int cnt, const double* x, const double* ys, long ystride, double* dots) {
  const int j = blockIdx.x;
  if (j >= cnt) return;
  __shared__ double s[256];
  double acc = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * ys[(long)j * ystride + i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) dots[j] = s[0];
}
__global__ void k_lincomb(long n, double a, const double* x, double b, double* y) {  // y = a x + b y
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

}  // namespace mgw

extern "C" mgw_status mgw_qsgw_step(mgw_handle* h, const mgw_options* o, mgw_qsgw_state* st) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (!st || st->nocc < 1 || st->nvir < 1 || st->naux < 1 || st->nmom_max < 0 || st->nmom_max > 11 || !st->h ||
      !st->L || !st->C || !st->eps || !st->F || !st->V || (st->reg != 0 && st->reg != 1) ||
      (st->reg == 0 && !(st->delta > 0.0)) || (st->reg == 1 && !(st->srg_s >= 0.0)) || !(st->scf_tol > 0.0) ||
      st->scf_max_iter < 1)
    return fail(h, MGW_ERR_ARG, "mgw_qsgw_step: bad state");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const int nocc = st->nocc, nvir = st->nvir, naux = st->naux, nmo = nocc + nvir;
  const int nmom = 2 * st->nmom_max + 2, nblk = st->nmom_max + 1;
  const long n2 = (long)nmo * nmo, ov = (long)nocc * nvir;
  const int space = std::max(1, std::min(st->diis_space, 32));
  const unsigned g2 = grid_for(n2);

  double *Lm, *tmpL, *Lov, *W, *sh, *sp, *ch, *ah, *bh, *cp, *ap, *bp, *Vmo, *rho, *rho_new, *Fx, *err, *hF, *hE;
  double *work, *evals, *dots, *v;
  MGW_TRY(slot_buffer(h, 40, (size_t)naux * n2, &Lm));
  MGW_TRY(slot_buffer(h, 41, (size_t)naux * n2, &tmpL));
  MGW_TRY(slot_buffer(h, 42, (size_t)naux * ov, &Lov));
  MGW_TRY(slot_buffer(h, 43, (size_t)nmom * naux * naux, &W));
  MGW_TRY(slot_buffer(h, 44, (size_t)nmom * n2, &sh));
  MGW_TRY(slot_buffer(h, 45, (size_t)nmom * n2, &sp));
  MGW_TRY(slot_buffer(h, 46, n2, &ch));
  MGW_TRY(slot_buffer(h, 47, (size_t)nblk * n2, &ah));
  MGW_TRY(slot_buffer(h, 48, (size_t)std::max(1, nblk - 1) * n2, &bh));
  MGW_TRY(slot_buffer(h, 49, n2, &cp));
  MGW_TRY(slot_buffer(h, 50, (size_t)nblk * n2, &ap));
  MGW_TRY(slot_buffer(h, 51, (size_t)std::max(1, nblk - 1) * n2, &bp));
  MGW_TRY(slot_buffer(h, 52, n2, &Vmo));
  MGW_TRY(slot_buffer(h, 53, n2, &rho));
  MGW_TRY(slot_buffer(h, 54, n2, &rho_new));
  MGW_TRY(slot_buffer(h, 55, n2, &Fx));
  MGW_TRY(slot_buffer(h, 56, n2, &err));
  MGW_TRY(slot_buffer(h, 57, (size_t)space * n2, &hF));
  MGW_TRY(slot_buffer(h, 58, (size_t)space * n2, &hE));
  MGW_TRY(slot_buffer(h, 59, 2 * n2, &work));
  MGW_TRY(slot_buffer(h, 60, nmo, &evals));
  MGW_TRY(slot_buffer(h, 61, 64, &dots));
  MGW_TRY(slot_buffer(h, 62, naux, &v));

  // 1. the GW moments and chains in the current orbitals: L' = C^T L C
  const double* C = st->C;
  MGW_TRY((dgemm<64, 64>(h, nmo, nmo, nmo, naux, ARowMajor{st->L, nmo, n2}, BRowMajor{C, nmo, 0},
                         EpiStore{tmpL, nmo, n2, 1.0, 0.0}, "gemm_nn")));
  MGW_TRY((dgemm<64, 64>(h, nmo, nmo, nmo, naux, AKMajor2{C, nmo, 0, nmo, 0}, BRowMajor{tmpL, nmo, n2},
                         EpiStore{Lm, nmo, n2, 1.0, 0.0}, "gemm_tn")));
  MGW_TRY(mgw_extract_ov(h, nocc, nvir, naux, Lm, Lov));
  MGW_TRY(mgw_response_moments(h, o, nocc, nvir, naux, nmom, st->eps, Lov, W));
  MGW_TRY(mgw_sigma_moments(h, o, nocc, nvir, naux, nmom, st->eps, Lm, W, sh, sp));
  int rh = 0, rp = 0;
  MGW_TRY(mgw_block_lanczos(h, o, nmo, nmom, sh, ch, ah, nblk > 1 ? bh : nullptr, &rh));
  MGW_TRY(mgw_block_lanczos(h, o, nmo, nmom, sp, cp, ap, nblk > 1 ? bp : nullptr, &rp));
  // 2. the static potential (Eqs. 36-39) in these orbitals, then V_ref = C V C^T
  MGW_TRY(mgw_qsgw_potential(h, nmo, nblk, rh, rp, st->eps, ch, ah, bh, cp, ap, bp, st->reg, st->delta, st->srg_s,
                             Vmo));
  MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, C, nmo, Vmo, nmo, 0.0, work, nmo));
  MGW_TRY(gemm_nt(h, nmo, nmo, nmo, 1.0, work, nmo, C, nmo, 0.0, st->V, nmo));

  // 3. Eq. 35 with V_ref fixed: F = f[rho] + V_ref, rho from the nocc lowest
  // orbitals, Pulay DIIS on the commutator F rho - rho F
  k_density_from_columns<<<g2, 256, 0, h->stream>>>(nmo, nocc, C, rho);
  MGW_TRY(check_launch(h, "qsgw_density"));
  std::vector<int> order;  // history slots, oldest first
  std::vector<double> B;   // Gram matrix of the errors in `order`
  int it = 0;
  bool converged = false;
  for (; it < st->scf_max_iter; ++it) {
    MGW_TRY(fock_build(h, nmo, naux, st->h, st->L, rho, st->F, v, tmpL));
    k_lincomb<<<g2, 256, 0, h->stream>>>(n2, 1.0, st->V, 1.0, st->F);
    MGW_TRY(check_launch(h, "qsgw_add_potential"));
    MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, st->F, nmo, rho, nmo, 0.0, err, nmo));     // F rho
    MGW_TRY(gemm_nn(h, nmo, nmo, nmo, -1.0, rho, nmo, st->F, nmo, 1.0, err, nmo));    // - rho F
    int slot;
    if ((int)order.size() < space) {
      slot = (int)order.size();
    } else {
      slot = order.front();
      order.erase(order.begin());
      const int n = (int)order.size() + 1;
      std::vector<double> nb((size_t)(n - 1) * (n - 1));
      for (int i = 1; i < n; ++i)
        for (int j = 1; j < n; ++j) nb[(size_t)(i - 1) * (n - 1) + (j - 1)] = B[(size_t)i * n + j];
      B.swap(nb);
    }
    order.push_back(slot);
    MGW_CUDA(h, cudaMemcpyAsync(hF + slot * n2, st->F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
    MGW_CUDA(h, cudaMemcpyAsync(hE + slot * n2, err, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
    k_gram_row<<<space, 256, 0, h->stream>>>(n2, space, err, hE, n2, dots);
    MGW_TRY(check_launch(h, "qsgw_gram"));
    std::vector<double> hd(space);
    MGW_CUDA(h, cudaMemcpyAsync(hd.data(), dots, sizeof(double) * space, cudaMemcpyDeviceToHost, h->stream));
    MGW_CUDA(h, cudaStreamSynchronize(h->stream));
    const int n = (int)order.size();
    {
      std::vector<double> nb((size_t)n * n);
      for (int i = 0; i < n - 1; ++i)
        for (int j = 0; j < n - 1; ++j) nb[(size_t)i * n + j] = B[(size_t)i * (n - 1) + j];
      for (int i = 0; i < n; ++i) nb[(size_t)i * n + (n - 1)] = nb[(size_t)(n - 1) * n + i] = hd[order[i]];
      B.swap(nb);
    }
    // the extrapolated field (plain F until three vectors are held), dropping
    // the oldest vectors while the DIIS system is singular
    const double* Fuse = st->F;
    if (n > 2) {
      std::vector<double> c;
      int use0 = 0;
      for (; use0 < n; ++use0) {
        const int k = n - use0;
        std::vector<double> sub((size_t)k * k);
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < k; ++j) sub[(size_t)i * k + j] = B[(size_t)(i + use0) * n + (j + use0)];
        if (diis_solve(sub, k, c)) break;
      }
      if (use0 < n) {
        for (int i = 0; i < (int)c.size(); ++i) {
          k_lincomb<<<g2, 256, 0, h->stream>>>(n2, c[i], hF + order[i + use0] * n2, i == 0 ? 0.0 : 1.0, Fx);
          MGW_TRY(check_launch(h, "qsgw_diis"));
        }
        Fuse = Fx;
      }
    }
    MGW_CUDA(h, cudaMemcpyAsync(work, Fuse, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
    MGW_TRY(syevd(h, nmo, work, evals));  // rows of work: eigenvectors
    k_rows_to_columns<<<g2, 256, 0, h->stream>>>(nmo, work, work + n2);
    MGW_TRY(check_launch(h, "qsgw_columns"));
    k_density_from_columns<<<g2, 256, 0, h->stream>>>(nmo, nocc, work + n2, rho_new);
    MGW_TRY(check_launch(h, "qsgw_density"));
    k_two_maxabs<<<1, 256, 0, h->stream>>>(n2, rho_new, rho, err, dots + 32);
    MGW_TRY(check_launch(h, "qsgw_change"));
    double ch2[2];
    MGW_CUDA(h, cudaMemcpyAsync(ch2, dots + 32, sizeof ch2, cudaMemcpyDeviceToHost, h->stream));
    MGW_CUDA(h, cudaStreamSynchronize(h->stream));
    std::swap(rho, rho_new);
    if (ch2[0] < st->scf_tol && ch2[1] < 1e3 * st->scf_tol) {
      converged = true;
      ++it;
      break;
    }
  }
  // 4. the field of the final density and its orbitals
  MGW_TRY(fock_build(h, nmo, naux, st->h, st->L, rho, st->F, v, tmpL));
  k_lincomb<<<g2, 256, 0, h->stream>>>(n2, 1.0, st->V, 1.0, st->F);
  MGW_TRY(check_launch(h, "qsgw_add_potential"));
  MGW_CUDA(h, cudaMemcpyAsync(work, st->F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
  MGW_TRY(syevd(h, nmo, work, evals));
  k_rows_to_columns<<<g2, 256, 0, h->stream>>>(nmo, work, st->C);
  MGW_TRY(check_launch(h, "qsgw_columns"));
  k_two_maxabs<<<1, 256, 0, h->stream>>>(nmo, evals, st->eps, evals, dots + 40);
  MGW_TRY(check_launch(h, "qsgw_de"));
  double de[2];
  MGW_CUDA(h, cudaMemcpyAsync(de, dots + 40, sizeof de, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaMemcpyAsync(st->eps, evals, sizeof(double) * nmo, cudaMemcpyDeviceToDevice, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  st->de = de[0];
  st->scf_iters = it;
  st->scf_converged = converged ? 1 : 0;
  return MGW_OK;
}
