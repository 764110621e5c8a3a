// One outer iteration of Fock self-consistent GW (Algorithm 2, Sec. III F).
//
//  1. rotate the DF tensor into the current orbitals C and build the
//     self-energy moments and both block-Lanczos chains there;
//  2. carry the chains' coupling into the fixed reference basis (W~ = C W~_mo);
//  3. alternate a search for the relative chemical potential zeta (the
//     Aufbau electron count of Eq. 40 for H~(zeta) against N) with a
//     DIIS-accelerated Fock loop F <- F[rho] at fixed zeta, until both hold;
//  4. eps, C <- eigh(F) and the QP energies (Eq. 34) in that eigenbasis.
// Numerical choices (the paper gives the loops, not their numerics):
// zeta as the root of N(zeta) - N nearest to the current zeta (outward scan
// in 0.01 Ha steps, Illinois regula falsi, golden-section fallback); Pulay DIIS on F with error F[rho] - F, space
// o->diis_space, plain steps first twice, until max |delta rho| < 1e-8
// (<= 100 steps); at most 20 zeta/Fock rounds.
#include "mgw_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mgw {

static unsigned nbk(long n) { return (unsigned)std::min<long>((n + 255) / 256, 152L * 16); }

__global__ void k_transpose(int n, const double* a, double* b) {  // b = a^T
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)n * n) return;
  int r = (int)(i / n), c = (int)(i % n);
  b[(long)c * n + r] = a[i];
}
__global__ void k_axpby(long n, double a, const double* x, double b, double* y) {  // y = a x + b y
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}
__global__ void k_sub(long n, const double* a, const double* b, double* c) {  // c = a - b
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    c[i] = a[i] - b[i];
}
// dots[j] = <x, ys[j]> for j < cnt (one block per j); maxabs of (a - b) in dots[cnt]
__global__ void k_dots(long n, int cnt, const double* x, const double* ys, long ystride, double* dots) {
  __shared__ double s[256];
  int j = blockIdx.x;
  double acc = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) acc += x[i] * ys[(long)j * ystride + i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && j < cnt) dots[j] = s[0];
}
__global__ void k_maxabs_diff(long n, const double* a, const double* b, double* out) {
  __shared__ double s[256];
  double m = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(a[i] - b[i]));
  s[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// Solve the DIIS system on the host: minimise |sum c_i e_i| s.t. sum c_i = 1.
// Gaussian elimination with partial pivoting on the bordered matrix; a
// vanishing pivot drops the oldest vector (returned as `drop`).
static bool diis_coefficients(const std::vector<double>& B, int n, std::vector<double>& c) {
  const int m = n + 1;
  std::vector<double> A((size_t)m * m), r(m, 0.0);
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(B[(size_t)i * n + i]));
  if (!(scale > 0)) scale = 1.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[(size_t)i * m + j] = B[(size_t)i * n + j] / scale;
  for (int i = 0; i < n; ++i) A[(size_t)i * m + n] = A[(size_t)n * m + i] = -1.0;
  A[(size_t)n * m + n] = 0.0;
  r[n] = -1.0;
  for (int k = 0; k < m; ++k) {
    int p = k;
    for (int i = k + 1; i < m; ++i)
      if (std::fabs(A[(size_t)i * m + k]) > std::fabs(A[(size_t)p * m + k])) p = i;
    if (std::fabs(A[(size_t)p * m + k]) < 1e-14) return false;
    if (p != k) {
      for (int j = 0; j < m; ++j) std::swap(A[(size_t)p * m + j], A[(size_t)k * m + j]);
      std::swap(r[p], r[k]);
    }
    for (int i = k + 1; i < m; ++i) {
      double f = A[(size_t)i * m + k] / A[(size_t)k * m + k];
      for (int j = k; j < m; ++j) A[(size_t)i * m + j] -= f * A[(size_t)k * m + j];
      r[i] -= f * r[k];
    }
  }
  std::vector<double> x(m);
  for (int i = m - 1; i >= 0; --i) {
    double acc = r[i];
    for (int j = i + 1; j < m; ++j) acc -= A[(size_t)i * m + j] * x[j];
    x[i] = acc / A[(size_t)i * m + i];
  }
  c.assign(x.begin(), x.begin() + n);
  return true;
}

}  // namespace mgw

mgw_status mgw::fock_build(mgw_handle* h, int nmo, int naux, const double* hcore, const double* L,
                           const double* r, double* out, double* v, double* tmp) {
  const long n2 = (long)nmo * nmo;
  // v_P = sum_rs L_Prs rho_rs ; J = sum_P v_P L_P
  MGW_TRY(gemm_nn(h, naux, 1, n2, 1.0, L, n2, r, 1, 0.0, v, 1));
  MGW_CUDA(h, cudaMemcpyAsync(out, hcore, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
  MGW_TRY(gemm_nn(h, 1, n2, naux, 1.0, v, naux, L, n2, 1.0, out, n2));
  // tmp_P = rho L_P (batched); K_pq = sum_{P,r} tmp[P][r][p] L[P][r][q]
  MGW_TRY((dgemm<64, 64>(h, nmo, nmo, nmo, naux, ARowMajor{r, nmo, 0}, BRowMajor{L, nmo, n2},
                         EpiStore{tmp, nmo, n2, 1.0, 0.0}, "gemm_nn")));
  MGW_TRY((dgemm<64, 64>(h, nmo, nmo, (long)naux * nmo, 1, AKMajor2{tmp, nmo, n2, nmo, 0}, BRowMajor{L, nmo, 0},
                         EpiStore{out, nmo, 0, -0.5, 1.0}, "gemm_tn")));
  return MGW_OK;
}

bool mgw::diis_solve(const std::vector<double>& B, int n, std::vector<double>& c) {
  return diis_coefficients(B, n, c);
}

namespace mgw {

struct FsgwCtx {
  mgw_handle* h;
  const mgw_options* o;
  int nmo, naux, nblk, rh, rp;
  long n2;
  const double* hcore;
  const double* L;
  double *coup_h, *alpha_h, *beta_h, *coup_p, *alpha_p, *beta_p;  // chains, coupling in the reference basis
  double *E, *weight, *epsqp, *rho, *rho_old, *Fn, *tmp, *v, *dots;
  double nelec;

  mgw_status qp(const double* F, double zeta, double* rho_out, double* ne, double* mu, int* m) {
    return mgw_qp_solve(h, o, nmo, nblk, rh, rp, F, coup_h, alpha_h, beta_h, coup_p, alpha_p, beta_p, zeta, nelec,
                        E, weight, nullptr, epsqp, rho_out, mu, ne, m);
  }

  // F[rho] = h + J - K/2
  mgw_status fock(const double* r, double* out) { return fock_build(h, nmo, naux, hcore, L, r, out, v, tmp); }

  mgw_status nerr(const double* F, double zeta, double* err) {
    double ne = 0, mu = 0;
    int m = 0;
    MGW_TRY(qp(F, zeta, nullptr, &ne, &mu, &m));
    *err = std::fabs(ne - nelec);
    return MGW_OK;
  }

  // Illinois regula falsi on a bracket [a, b] with ga * gb < 0
  mgw_status illinois(const double* F, double a, double ga, double b, double gb, double* zc, double* gcv,
                      int* evals) {
    double c = std::fabs(ga) < std::fabs(gb) ? a : b, gc = std::fabs(ga) < std::fabs(gb) ? ga : gb;
    for (int it = 0; it < 60; ++it) {
      if (std::fabs(gc) <= 1e-10 || std::fabs(b - a) < 1e-9) break;
      c = b - gb * (b - a) / (gb - ga);
      MGW_TRY(gval(F, c, &gc, evals));
      if (gc * gb < 0) { a = b; ga = gb; } else { ga *= 0.5; }
      b = c;
      gb = gc;
    }
    *zc = c;
    *gcv = gc;
    return MGW_OK;
  }

  mgw_status gval(const double* F, double z, double* gz, int* evals) {  // g = N(z) - N
    double ne = 0, mu = 0;
    int m = 0;
    MGW_TRY(qp(F, z, nullptr, &ne, &mu, &m));
    *gz = ne - nelec;
    ++*evals;
    return MGW_OK;
  }

  // root of g(zeta) = N(zeta) - N nearest to *zeta: outward scan in steps of
  // 0.01 Ha for a sign change, Illinois regula falsi on it (accepted when
  // |g| <= 1e-6, else it was a jump of the filling and the scan goes on),
  // golden section on |g| over [-1, 1] as the fallback
  mgw_status zeta_search(const double* F, double* zeta, double* ferr, int* evals, const double* g_at_start = nullptr) {
    const double lo = -1.0, hi = 1.0, step = 0.01, tol = 1e-10, accept = 1e-6;
    const double z0 = std::min(std::max(*zeta, lo), hi);
    double g0;
    if (g_at_start && z0 == *zeta) g0 = *g_at_start;
    else MGW_TRY(gval(F, z0, &g0, evals));
    if (std::fabs(g0) <= tol) { *zeta = z0; *ferr = std::fabs(g0); return MGW_OK; }
    double pz[2] = {z0, z0}, pg[2] = {g0, g0};
    for (int k = 1;; ++k) {
      bool moved = false;
      for (int si = 0; si < 2; ++si) {
        const double side = si == 0 ? 1.0 : -1.0;
        const double z = z0 + side * k * step;
        if (z < lo - 1e-12 || z > hi + 1e-12) continue;
        moved = true;
        double gz;
        MGW_TRY(gval(F, z, &gz, evals));
        const double zp = pz[si], gp = pg[si];
        pz[si] = z;
        pg[si] = gz;
        if (std::fabs(gz) <= tol) { *zeta = z; *ferr = std::fabs(gz); return MGW_OK; }
        if (gz * gp < 0) {
          double c, gc;
          MGW_TRY(illinois(F, zp, gp, z, gz, &c, &gc, evals));
          if (std::fabs(gc) <= accept) { *zeta = c; *ferr = std::fabs(gc); return MGW_OK; }
        }
      }
      if (!moved) break;
    }
    // fallback: golden section on |g| over [lo, hi]
    const double r = (std::sqrt(5.0) - 1.0) / 2.0;
    double a = lo, b = hi, c = b - r * (b - a), d = a + r * (b - a), fc, fd;
    MGW_TRY(gval(F, c, &fc, evals));
    MGW_TRY(gval(F, d, &fd, evals));
    fc = std::fabs(fc);
    fd = std::fabs(fd);
    while (b - a > 1e-8 && *evals < 400 && std::min(fc, fd) > tol) {
      if (fc <= fd) {
        b = d; d = c; fd = fc;
        c = b - r * (b - a);
        MGW_TRY(gval(F, c, &fc, evals));
        fc = std::fabs(fc);
      } else {
        a = c; c = d; fc = fd;
        d = a + r * (b - a);
        MGW_TRY(gval(F, d, &fd, evals));
        fd = std::fabs(fd);
      }
    }
    if (fc <= fd) { *zeta = c; *ferr = fc; } else { *zeta = d; *ferr = fd; }
    return MGW_OK;
  }

  // DIIS Fock loop at fixed zeta; F updated in place, returns iterations
  mgw_status fock_loop(double* F, double zeta, double* dF, double* dE, int space, int* iters) {
    std::vector<int> order;           // slots of the history, oldest first
    std::vector<double> B;            // Gram matrix of the errors in `order`
    bool have_old = false;
    for (int it = 0; it < 100; ++it) {
      double ne, mu;
      int m;
      MGW_TRY(qp(F, zeta, rho, &ne, &mu, &m));
      MGW_TRY(fock(rho, Fn));
      if (have_old) {
        k_maxabs_diff<<<1, 256, 0, h->stream>>>(n2, rho, rho_old, dots + 64);
        MGW_TRY(check_launch(h, "maxabs"));
        double dr = 0;
        MGW_CUDA(h, cudaMemcpyAsync(&dr, dots + 64, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        MGW_CUDA(h, cudaStreamSynchronize(h->stream));
        if (dr < 1e-8) {
          MGW_CUDA(h, cudaMemcpyAsync(F, Fn, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
          *iters = it + 1;
          return MGW_OK;
        }
      }
      MGW_CUDA(h, cudaMemcpyAsync(rho_old, rho, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
      have_old = true;
      // push (Fn, Fn - F) into the history ring
      int slot;
      if ((int)order.size() < space) {
        slot = (int)order.size();
      } else {
        slot = order.front();
        order.erase(order.begin());
        // drop the oldest row/column of B
        const int n = (int)order.size() + 1;
        std::vector<double> nb((size_t)(n - 1) * (n - 1));
        for (int i = 1; i < n; ++i)
          for (int j = 1; j < n; ++j) nb[(size_t)(i - 1) * (n - 1) + (j - 1)] = B[(size_t)i * n + j];
        B.swap(nb);
      }
      order.push_back(slot);
      MGW_CUDA(h, cudaMemcpyAsync(dF + slot * n2, Fn, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
      k_sub<<<nbk(n2), 256, 0, h->stream>>>(n2, Fn, F, dE + slot * n2);
      MGW_TRY(check_launch(h, "sub"));
      // new row of the Gram matrix
      k_dots<<<space, 256, 0, h->stream>>>(n2, space, dE + slot * n2, dE, n2, dots);
      MGW_TRY(check_launch(h, "dots"));
      std::vector<double> hd(space);
      MGW_CUDA(h, cudaMemcpyAsync(hd.data(), dots, sizeof(double) * space, cudaMemcpyDeviceToHost, h->stream));
      MGW_CUDA(h, cudaStreamSynchronize(h->stream));
      const int n = (int)order.size();
      std::vector<double> nb((size_t)n * n);
      for (int i = 0; i < n - 1; ++i)
        for (int j = 0; j < n - 1; ++j) nb[(size_t)i * n + j] = B[(size_t)i * (n - 1) + j];
      for (int i = 0; i < n; ++i) nb[(size_t)i * n + (n - 1)] = nb[(size_t)(n - 1) * n + i] = hd[order[i]];
      B.swap(nb);
      if (it < 2) {
        MGW_CUDA(h, cudaMemcpyAsync(F, Fn, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
        continue;
      }
      std::vector<double> c;
      int use0 = 0;
      // solve on the trailing block, dropping the oldest vectors while singular
      for (use0 = 0; use0 < n; ++use0) {
        const int k = n - use0;
        std::vector<double> sub((size_t)k * k);
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < k; ++j) sub[(size_t)i * k + j] = B[(size_t)(i + use0) * n + (j + use0)];
        if (diis_coefficients(sub, k, c)) break;
      }
      if (use0 == n) {
        MGW_CUDA(h, cudaMemcpyAsync(F, Fn, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
        continue;
      }
      for (int i = 0; i < (int)c.size(); ++i) {
        k_axpby<<<nbk(n2), 256, 0, h->stream>>>(n2, c[i], dF + order[i + use0] * n2, i == 0 ? 0.0 : 1.0, F);
        MGW_TRY(check_launch(h, "axpby"));
      }
    }
    *iters = 100;
    return MGW_OK;
  }
};

}  // namespace mgw

using namespace mgw;

// the closed-shell Hartree-Fock density 2 on the first nocc diagonal
// elements, and diag(eps) in `d`
__global__ void k_hf_density(int nmo, int nocc, const double* eps, double* rho, double* d) {
  const long n2 = (long)nmo * nmo;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n2; i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nmo), c = (int)(i % nmo);
    rho[i] = (r == c && r < nocc) ? 2.0 : 0.0;
    d[i] = r == c ? eps[r] : 0.0;
  }
}

extern "C" mgw_status mgw_hf_core(mgw_handle* h, int nocc, int nmo, int naux, const double* eps, const double* L,
                                  double* hcore) {
  if (!h) return MGW_ERR_ARG;
  if (nocc < 1 || nmo <= nocc || naux < 1 || !eps || !L || !hcore)
    return fail(h, MGW_ERR_ARG, "mgw_hf_core: bad sizes or null pointer");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long n2 = (long)nmo * nmo;
  Arena ar;
  double *rho = nullptr, *v = nullptr, *tmp = nullptr;
  ar.add(&rho, n2);
  ar.add(&v, naux);
  ar.add(&tmp, (long)naux * n2);
  MGW_TRY(ar.commit(h));
  k_hf_density<<<(unsigned)std::min<long>((n2 + 255) / 256, 152L * 8), 256, 0, h->stream>>>(nmo, nocc, eps, rho,
                                                                                            hcore);
  MGW_TRY(check_launch(h, "hf_density"));
  // hcore = diag(eps) - J[rho] + K[rho]/2: v_P = sum_rs L_Prs rho_rs, J = sum_P v_P L_P
  MGW_TRY(gemm_nn(h, naux, 1, n2, 1.0, L, n2, rho, 1, 0.0, v, 1));
  MGW_TRY(gemm_nn(h, 1, n2, naux, -1.0, v, naux, L, n2, 1.0, hcore, n2));
  // tmp_P = rho L_P; K_pq = sum_{P,r} tmp[P][r][p] L[P][r][q]
  MGW_TRY((dgemm<64, 64>(h, nmo, nmo, nmo, naux, ARowMajor{rho, nmo, 0}, BRowMajor{L, nmo, n2},
                         EpiStore{tmp, nmo, n2, 1.0, 0.0}, "gemm_nn")));
  return dgemm<64, 64>(h, nmo, nmo, (long)naux * nmo, 1, AKMajor2{tmp, nmo, n2, nmo, 0}, BRowMajor{L, nmo, 0},
                       EpiStore{hcore, nmo, 0, 0.5, 1.0}, "gemm_tn");
}

extern "C" mgw_status mgw_fsgw_step(mgw_handle* h, const mgw_options* o, mgw_fsgw_state* st) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (!st || st->nocc < 1 || st->nvir < 1 || st->naux < 1 || st->nmom_max < 0 || st->nmom_max > 11 || !st->h ||
      !st->L || !st->F || !st->C || !st->eps || !st->eps_qp)
    return fail(h, MGW_ERR_ARG, "mgw_fsgw_step: bad state");
  MGW_CUDA(h, cudaSetDevice(h->device));
  const int nocc = st->nocc, nvir = st->nvir, naux = st->naux, nmo = nocc + nvir;
  const int nmom = 2 * st->nmom_max + 2, nblk = st->nmom_max + 1;
  const long n2 = (long)nmo * nmo, ov = (long)nocc * nvir;
  const int space = std::max(1, std::min(o->diis_space, 32));

  double *Lm, *tmpL, *Lov, *W, *sh, *sp, *ch, *ah, *bh, *cp, *ap, *bp, *crh, *crp;
  double *E, *weight, *epsqp, *rho, *rho_old, *Fn, *dF, *dE, *misc, *dots, *v;
  const long dim = nmo + (long)nblk * 2 * nmo;
  MGW_TRY(slot_buffer(h, 0, (size_t)naux * n2, &Lm));
  MGW_TRY(slot_buffer(h, 1, (size_t)naux * n2, &tmpL));
  MGW_TRY(slot_buffer(h, 2, (size_t)naux * ov, &Lov));
  MGW_TRY(slot_buffer(h, 3, (size_t)nmom * naux * naux, &W));
  MGW_TRY(slot_buffer(h, 4, (size_t)nmom * n2, &sh));
  MGW_TRY(slot_buffer(h, 5, (size_t)nmom * n2, &sp));
  MGW_TRY(slot_buffer(h, 6, n2, &ch));
  MGW_TRY(slot_buffer(h, 7, (size_t)nblk * n2, &ah));
  MGW_TRY(slot_buffer(h, 8, (size_t)std::max(1, nblk - 1) * n2, &bh));
  MGW_TRY(slot_buffer(h, 9, n2, &cp));
  MGW_TRY(slot_buffer(h, 10, (size_t)nblk * n2, &ap));
  MGW_TRY(slot_buffer(h, 11, (size_t)std::max(1, nblk - 1) * n2, &bp));
  MGW_TRY(slot_buffer(h, 12, n2, &crh));
  MGW_TRY(slot_buffer(h, 13, n2, &crp));
  MGW_TRY(slot_buffer(h, 14, dim, &E));
  MGW_TRY(slot_buffer(h, 15, dim, &weight));
  MGW_TRY(slot_buffer(h, 16, nmo, &epsqp));
  MGW_TRY(slot_buffer(h, 17, n2, &rho));
  MGW_TRY(slot_buffer(h, 18, n2, &rho_old));
  MGW_TRY(slot_buffer(h, 19, n2, &Fn));
  MGW_TRY(slot_buffer(h, 20, (size_t)space * n2, &dF));
  MGW_TRY(slot_buffer(h, 21, (size_t)space * n2, &dE));
  MGW_TRY(slot_buffer(h, 22, 4 * n2, &misc));
  MGW_TRY(slot_buffer(h, 23, 128, &dots));
  MGW_TRY(slot_buffer(h, 24, naux, &v));
  double *Forig = nullptr, *Fstep = nullptr;  // the step's starting F, and F - F_prev
  if (st->F_prev) {
    MGW_TRY(slot_buffer(h, 25, n2, &Forig));
    MGW_TRY(slot_buffer(h, 26, n2, &Fstep));
  }
  MGW_CUDA(h, cudaMemsetAsync(dE, 0, sizeof(double) * space * n2, h->stream));

  if (st->init) {  // orbitals of the given Fock matrix
    MGW_CUDA(h, cudaMemcpyAsync(misc, st->F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
    MGW_TRY(syevd(h, nmo, misc, st->eps));
    k_transpose<<<nbk(n2), 256, 0, h->stream>>>(nmo, misc, st->C);
    MGW_TRY(check_launch(h, "transpose"));
    st->init = 0;
  }
  // 1. DF tensor in the orbitals C: L'_Q = C^T L_Q C
  const double* C = st->C;
  MGW_TRY((dgemm<64, 64>(h, nmo, nmo, nmo, naux, ARowMajor{st->L, nmo, n2}, BRowMajor{C, nmo, 0},
                         EpiStore{tmpL, nmo, n2, 1.0, 0.0}, "gemm_nn")));
  MGW_TRY((dgemm<64, 64>(h, nmo, nmo, nmo, naux, AKMajor2{C, nmo, 0, nmo, 0}, BRowMajor{tmpL, nmo, n2},
                         EpiStore{Lm, nmo, n2, 1.0, 0.0}, "gemm_tn")));
  MGW_TRY(mgw_extract_ov(h, nocc, nvir, naux, Lm, Lov));
  mgw_options oo = *o;
  MGW_TRY(mgw_response_moments(h, &oo, nocc, nvir, naux, nmom, st->eps, Lov, W));
  MGW_TRY(mgw_sigma_moments(h, &oo, nocc, nvir, naux, nmom, st->eps, Lm, W, sh, sp));
  int rh = 0, rp = 0;
  MGW_TRY(mgw_block_lanczos(h, &oo, nmo, nmom, sh, ch, ah, nblk > 1 ? bh : nullptr, &rh));
  MGW_TRY(mgw_block_lanczos(h, &oo, nmo, nmom, sp, cp, ap, nblk > 1 ? bp : nullptr, &rp));
  // 2. coupling into the reference basis
  MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, C, nmo, ch, nmo, 0.0, crh, nmo));
  MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, C, nmo, cp, nmo, 0.0, crp, nmo));
  if (st->sigma_ref) {
    for (int n = 0; n < nmom; ++n) {
      k_axpby<<<nbk(n2), 256, 0, h->stream>>>(n2, 1.0, sh + n * n2, 0.0, misc);
      k_axpby<<<nbk(n2), 256, 0, h->stream>>>(n2, 1.0, sp + n * n2, 1.0, misc);
      MGW_TRY(check_launch(h, "axpby"));
      MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, C, nmo, misc, nmo, 0.0, misc + n2, nmo));
      MGW_TRY(gemm_nt(h, nmo, nmo, nmo, 1.0, misc + n2, nmo, C, nmo, 0.0, st->sigma_ref + n * n2, nmo));
    }
  }

  FsgwCtx cx{h, o, nmo, naux, nblk, rh, rp, n2, st->h, st->L, crh, ah, bh, crp, ap, bp,
             E, weight, epsqp, rho, rho_old, Fn, tmpL, v, dots, 2.0 * nocc};
  // Fock-matrix proposal: F <- F + beta (F - F_prev), beta from the network
  // (none: beta = 0, the plain start); the DIIS loop below starts from it
  st->wf_beta = 0.0;
  const double prev_target = st->wf_target;
  st->wf_target = 0.0;
  for (int i = 0; i < MGW_WS_FEATURES; ++i) st->wf_feat[i] = 0.f;
  double dd = 0.0;  // |F - F_prev|^2
  if (st->F_prev) {
    MGW_CUDA(h, cudaMemcpyAsync(Forig, st->F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
    if (st->fock_hist) {
      k_sub<<<nbk(n2), 256, 0, h->stream>>>(n2, st->F, st->F_prev, Fstep);
      k_maxabs_diff<<<1, 256, 0, h->stream>>>(n2, st->F, st->F_prev, dots + 104);
      k_dots<<<1, 256, 0, h->stream>>>(n2, 1, Fstep, Fstep, n2, dots + 105);
      MGW_TRY(check_launch(h, "fock_step"));
      double hv[2], fe[2];
      MGW_CUDA(h, cudaMemcpyAsync(hv, dots + 104, sizeof hv, cudaMemcpyDeviceToHost, h->stream));
      MGW_CUDA(h, cudaMemcpyAsync(fe, st->eps + nocc - 1, sizeof fe, cudaMemcpyDeviceToHost, h->stream));
      MGW_CUDA(h, cudaStreamSynchronize(h->stream));
      dd = hv[1];
      const float f[MGW_WS_FEATURES] = {(float)(std::log10(hv[0] + 1e-14) / 10.0), (float)(10.0 * hv[0]),
                                        (float)prev_target, (float)(prev_target != 0.0), (float)st->zeta,
                                        (float)(fe[1] - fe[0]), (float)nocc / (float)nmo, 1.0f};
      for (int i = 0; i < MGW_WS_FEATURES; ++i) st->wf_feat[i] = f[i];
      if (st->wf_params && st->wf_wbf16 && st->wf_width > 0 && dd > 0.0) {
        float* xy = reinterpret_cast<float*>(dots + 112);  // 8 inputs + 1 output
        MGW_CUDA(h, cudaMemcpyAsync(xy, f, sizeof f, cudaMemcpyHostToDevice, h->stream));
        MGW_TRY(mgw_mlp_forward(h, MGW_WS_FEATURES, st->wf_width, 1, st->wf_params, st->wf_wbf16, 1, xy, xy + 8,
                                nullptr));
        float y = 0.f;
        MGW_CUDA(h, cudaMemcpyAsync(&y, xy + 8, sizeof y, cudaMemcpyDeviceToHost, h->stream));
        MGW_CUDA(h, cudaStreamSynchronize(h->stream));
        const double beta = std::min(2.0, std::max(-0.5, (double)y));
        if (std::isfinite(beta) && beta != 0.0) {
          k_axpby<<<nbk(n2), 256, 0, h->stream>>>(n2, beta, Fstep, 1.0, st->F);
          MGW_TRY(check_launch(h, "fock_proposal"));
          st->wf_beta = beta;
        }
      }
    }
  }

  // 3. zeta / Fock rounds
  int inner = 0, evals = 0;
  double zeta = st->zeta;
  const double zeta_prev = zeta;
  st->ws_hit = 0;
  for (int rep = 0; rep < 20; ++rep) {
    double ferr = 0;
    if (rep == 0) {
      // features of the first search: frontier energies of the current
      // orbitals, the count error at the previous zeta, the occupation ratio
      double fe[2];
      MGW_CUDA(h, cudaMemcpyAsync(fe, st->eps + nocc - 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      double g0;
      MGW_TRY(cx.gval(st->F, zeta, &g0, &evals));  // synchronises
      const float f[MGW_WS_FEATURES] = {(float)fe[0], (float)fe[1], (float)(fe[1] - fe[0]), (float)g0,
                                        (float)(10.0 * g0), (float)zeta, (float)nocc / (float)nmo, 1.0f};
      for (int i = 0; i < MGW_WS_FEATURES; ++i) st->ws_feat[i] = f[i];
      bool done = std::fabs(g0) <= 1e-10;  // the previous zeta still holds
      if (done) ferr = std::fabs(g0);
      if (!done && st->ws_params && st->ws_wbf16 && st->ws_width > 0) {
        // prediction zeta_hat = zeta_prev + y, then the root from the two
        // points (zeta_prev, g0), (zeta_hat, g_hat); when that fails the
        // plain search below runs as if there were no prediction
        float* xy = reinterpret_cast<float*>(dots + 96);  // 8 inputs + 1 output
        MGW_CUDA(h, cudaMemcpyAsync(xy, f, sizeof f, cudaMemcpyHostToDevice, h->stream));
        MGW_TRY(mgw_mlp_forward(h, MGW_WS_FEATURES, st->ws_width, 1, st->ws_params, st->ws_wbf16, 1, xy, xy + 8,
                                nullptr));
        float y = 0.f;
        MGW_CUDA(h, cudaMemcpyAsync(&y, xy + 8, sizeof y, cudaMemcpyDeviceToHost, h->stream));
        MGW_CUDA(h, cudaStreamSynchronize(h->stream));
        double zh = std::min(1.0, std::max(-1.0, zeta + (double)y));
        if (std::fabs(zh - zeta) < 1e-9) zh = zeta + (zeta < 1.0 ? 1e-6 : -1e-6);
        double gh;
        MGW_TRY(cx.gval(st->F, zh, &gh, &evals));
        // secant steps from the last two points until they bracket the root
        // (then Illinois, accepted as in the plain search) or hit it
        double za = zeta, ga = g0, zb = zh, gb = gh, zc = zh, gc = gh;
        bool bracketed = false;
        for (int it = 0; it < 4 && std::fabs(gb) > 1e-10; ++it) {
          if (ga * gb < 0) {
            MGW_TRY(cx.illinois(st->F, za, ga, zb, gb, &zc, &gc, &evals));
            bracketed = true;
            break;
          }
          if (gb == ga) break;
          const double zs = zb - gb * (zb - za) / (gb - ga);
          if (!std::isfinite(zs) || zs < -1.0 || zs > 1.0 || std::fabs(zs - zb) > 0.02) break;
          double gs;
          MGW_TRY(cx.gval(st->F, zs, &gs, &evals));
          za = zb;
          ga = gb;
          zb = zs;
          gb = gs;
        }
        if (!bracketed) {
          zc = zb;
          gc = gb;
        }
        if (std::fabs(gc) <= 1e-10 || (bracketed && std::fabs(gc) <= 1e-6)) {
          zeta = zc;
          ferr = std::fabs(gc);
          done = true;
          st->ws_hit = 1;
        }
      }
      if (!done) MGW_TRY(cx.zeta_search(st->F, &zeta, &ferr, &evals, &g0));
      st->ws_target = zeta - zeta_prev;
    } else {
      MGW_TRY(cx.zeta_search(st->F, &zeta, &ferr, &evals));
    }
    int k = 0;
    MGW_TRY(cx.fock_loop(st->F, zeta, dF, dE, space, &k));
    inner += k;
    double now = 0;
    MGW_TRY(cx.nerr(st->F, zeta, &now));
    if (now <= std::max(ferr, 1e-10) + 1e-12 && k <= 2) break;
  }
  // the beta that would have started at the converged F along F - F_prev
  // (least squares, a training target); F_prev <- this step's starting F
  if (st->F_prev) {
    if (st->fock_hist && dd > 0.0) {
      k_sub<<<nbk(n2), 256, 0, h->stream>>>(n2, st->F, Forig, Fn);
      k_dots<<<1, 256, 0, h->stream>>>(n2, 1, Fn, Fstep, n2, dots + 106);
      MGW_TRY(check_launch(h, "fock_target"));
      double ed = 0.0;
      MGW_CUDA(h, cudaMemcpyAsync(&ed, dots + 106, sizeof ed, cudaMemcpyDeviceToHost, h->stream));
      MGW_CUDA(h, cudaStreamSynchronize(h->stream));
      st->wf_target = ed / dd;
    }
    MGW_CUDA(h, cudaMemcpyAsync(st->F_prev, Forig, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
    st->fock_hist = 1;
  }
  // 4. new orbitals and the QP energies in their basis
  MGW_CUDA(h, cudaMemcpyAsync(misc, st->F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, h->stream));
  MGW_TRY(syevd(h, nmo, misc, st->eps));
  k_transpose<<<nbk(n2), 256, 0, h->stream>>>(nmo, misc, st->C);  // columns = eigenvectors
  MGW_TRY(check_launch(h, "transpose"));
  // F_mo = C^T F C, coupling_mo = C^T coupling_ref
  MGW_TRY(gemm_tn(h, nmo, nmo, nmo, 1.0, st->C, nmo, st->F, nmo, 0.0, misc + n2, nmo));
  MGW_TRY(gemm_nn(h, nmo, nmo, nmo, 1.0, misc + n2, nmo, st->C, nmo, 0.0, misc + 2 * n2, nmo));
  MGW_TRY(gemm_tn(h, nmo, nmo, nmo, 1.0, st->C, nmo, crh, nmo, 0.0, ch, nmo));
  MGW_TRY(gemm_tn(h, nmo, nmo, nmo, 1.0, st->C, nmo, crp, nmo, 0.0, cp, nmo));
  double ne = 0, mu = 0;
  int m = 0;
  MGW_TRY(mgw_qp_solve(h, o, nmo, nblk, rh, rp, misc + 2 * n2, ch, ah, bh, cp, ap, bp, zeta, 2.0 * nocc, E, weight,
                       nullptr, st->eps_qp, nullptr, &mu, &ne, &m));
  st->zeta = zeta;
  st->mu = mu;
  st->nelec = ne;
  st->inner_iters = inner;
  st->zeta_evals = evals;
  return MGW_OK;
}
