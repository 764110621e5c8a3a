// Eigenvalues of a symmetric matrix and the first `nrows` rows of its
// eigenvectors, the two things the QP step needs of the upfolded
// Hamiltonian (Eq. 9): E for the poles and the Aufbau count (Eq. 40), the
// physical rows chi_pa for the weights and the QP argmax (Eq. 34).
//
//   1. Householder tridiagonalisation H = Q T Q^T (cuSOLVER sytrd: plain
//      dense linear algebra, like a GEMM);
//   2. every eigenvalue of T by bisection on the Sturm count, one thread per
//      eigenvalue (own kernel);
//   3. the eigenvectors z_a of T by inverse iteration with the computed
//      eigenvalue, one thread per eigenvalue: LU of T - lambda I with partial
//      pivoting, three solves from a fixed pseudo-random start (own kernel);
//      eigenvalues closer than 1e-9 of the spectral radius are
//      re-orthogonalised (modified Gram-Schmidt, own kernel);
//   4. the physical rows of Q (cuSOLVER ormtr applied to nrows unit vectors:
//      4 n^2 nrows flops instead of the 2 n^3 of a full back-transformation),
//      then chi = Q[0:nrows, :] Z as an FP64-accurate digit-sliced product on
//      the tensor cores.
// A full eigen-decomposition (syevd) does 1. plus a divide-and-conquer
// tridiagonal solve with every eigenvector and the back-transformation of
// all of them; here only nrows of n rows are ever formed.
//
// The 32-bit dense solver API refuses some large matrices: ormtr answered
// status 3 (invalid value) at n = 36 499 for any number of columns, while
// n = 20 400 runs.  Where its workspace queries refuse the size, the 64-bit
// syevd (Xsyevd) runs instead, with every eigenvector, and its first nrows
// rows are copied out.
#include "mgw_internal.h"
#include "ozaki.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

namespace mgw {

static unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }

// Gershgorin interval, max e^2 and the spectral bound: out = {lo, hi, emax2}
__global__ void k_tri_bounds(int n, const double* d, const double* e, double* out) {
  __shared__ double slo[256], shi[256], se[256];
  double lo = DBL_MAX, hi = -DBL_MAX, em = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i + 1 < n) em = fmax(em, e[i] * e[i]);
  }
  slo[threadIdx.x] = lo;
  shi[threadIdx.x] = hi;
  se[threadIdx.x] = em;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + w]);
      shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + w]);
      se[threadIdx.x] = fmax(se[threadIdx.x], se[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double span = fmax(fabs(slo[0]), fabs(shi[0]));
    out[0] = slo[0] - 2.0 * DBL_EPSILON * span;
    out[1] = shi[0] + 2.0 * DBL_EPSILON * span;
    out[2] = se[0];
  }
}

__global__ void k_square(int n, const double* e, double* e2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) e2[i] = e[i] * e[i];
}

// number of eigenvalues of T below x: negative pivots of the LDL^T
// factorisation of T - x I (Sturm count), pivots of magnitude below pivmin
// taken as -pivmin
__device__ __forceinline__ int sturm_count(int n, const double* __restrict__ d, const double* __restrict__ e2,
                                           double x, double pivmin) {
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// eigenvalue k (ascending, 0-based) of T by bisection: the count below lo
// stays <= k, below hi > k, until the interval is at the rounding level
__global__ void k_bisect(int n, const double* __restrict__ d, const double* __restrict__ e2,
                         const double* __restrict__ bounds, double* lam) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double lo = bounds[0], hi = bounds[1];
  const double pivmin = DBL_MIN * fmax(1.0, bounds[2]);
  for (int it = 0; it < 128; ++it) {
    const double tol = 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + pivmin;
    if (hi - lo <= tol) break;
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(n, d, e2, mid, pivmin) > k) hi = mid;
    else lo = mid;
  }
  lam[k] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double start_entry(int i, int a) {  // fixed pseudo-random in (-1, 1)
  unsigned long long x = (unsigned long long)i * 0x9E3779B97F4A7C15ull + (unsigned long long)a * 0xBF58476D1CE4E5B9ull;
  x ^= x >> 31;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 29;
  return (double)(long long)(x >> 11) * (1.0 / 4503599627370496.0) - 1.0;
}

// Eigenvectors z_a of T for the eigenvalues lam[a0 .. a0 + nb) by inverse
// iteration: Gaussian elimination of T - lambda I with partial pivoting (U
// with two superdiagonals, multipliers, row swaps), then three solves, each
// normalised.  Thread j of the batch keeps its factors at index i * nb + j
// (consecutive threads, consecutive addresses); the vector is built in place
// in column a0 + j of Z [n][ldz].
__global__ void k_inverse_iteration(int n, const double* __restrict__ d, const double* __restrict__ e,
                                    const double* __restrict__ lam, int a0, int nb, double* U0, double* U1,
                                    double* U2, double* ML, unsigned char* PV, double* Z, long ldz, double tnorm) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int a = a0 + j;
  const double x = lam[a];
  const double tiny = DBL_EPSILON * fmax(tnorm, DBL_MIN);
  // factorisation
  double ai = d[0] - x, bi = n > 1 ? e[0] : 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    const double c = e[i], an = d[i + 1] - x, bn = i + 2 < n ? e[i + 1] : 0.0;
    const long o = (long)i * nb + j;
    if (fabs(ai) >= fabs(c)) {
      if (ai == 0.0) ai = tiny;
      const double m = c / ai;
      U0[o] = ai;
      U1[o] = bi;
      U2[o] = 0.0;
      ML[o] = m;
      PV[o] = 0;
      ai = an - m * bi;
      bi = bn;
    } else {
      const double m = ai / c;
      U0[o] = c;
      U1[o] = an;
      U2[o] = bn;
      ML[o] = m;
      PV[o] = 1;
      const double t = bi - m * an;
      bi = -m * bn;
      ai = t;
    }
  }
  if (fabs(ai) < tiny) ai = ai < 0.0 ? -tiny : tiny;
  U0[(long)(n - 1) * nb + j] = ai;
  // start vector, then three solves
  double nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double v = start_entry(i, a);
    Z[(long)i * ldz + a] = v;
    nrm += v * v;
  }
  double scale = 1.0 / sqrt(nrm);
  for (int rep = 0; rep < 3; ++rep) {
    // forward: y <- L^-1 P y (with the current scale folded in)
    double yi = Z[a] * scale;
    for (int i = 0; i + 1 < n; ++i) {
      const long o = (long)i * nb + j;
      double yn = Z[(long)(i + 1) * ldz + a] * scale;
      if (PV[o]) {
        const double t = yi;
        yi = yn;
        yn = t;
      }
      Z[(long)i * ldz + a] = yi;
      yi = yn - ML[o] * yi;
    }
    Z[(long)(n - 1) * ldz + a] = yi;
    // backward: U x = y
    double x1 = 0.0, x2 = 0.0;  // x_{i+1}, x_{i+2}
    nrm = 0.0;
    for (int i = n - 1; i >= 0; --i) {
      const long o = (long)i * nb + j;
      const double v = (Z[(long)i * ldz + a] - U1[o] * x1 - U2[o] * x2) / U0[o];
      Z[(long)i * ldz + a] = v;
      nrm += v * v;
      x2 = x1;
      x1 = v;
    }
    scale = 1.0 / sqrt(nrm);
  }
  for (int i = 0; i < n; ++i) Z[(long)i * ldz + a] *= scale;
}

// modified Gram-Schmidt over the columns [c0, c1) of Z (one block per cluster)
__global__ void k_cluster_mgs(int n, const int* __restrict__ cl, double* Z, long ldz) {
  const int c0 = cl[2 * blockIdx.x], c1 = cl[2 * blockIdx.x + 1];
  __shared__ double red[256];
  for (int k = c0; k < c1; ++k) {
    for (int q = c0; q <= k; ++q) {
      double acc = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        acc += q < k ? Z[(long)i * ldz + q] * Z[(long)i * ldz + k] : Z[(long)i * ldz + k] * Z[(long)i * ldz + k];
      red[threadIdx.x] = acc;
      __syncthreads();
      for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
      }
      const double s = red[0];
      __syncthreads();
      if (q < k) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) Z[(long)i * ldz + k] -= s * Z[(long)i * ldz + q];
      } else {
        const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) Z[(long)i * ldz + k] *= inv;
      }
      __syncthreads();
    }
  }
}

// C (column-major n x nrows) = the first nrows columns of the identity
__global__ void k_unit_columns(int n, int nrows, double* C) {
  const long total = (long)n * nrows;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long p = idx / n, i = idx % n;
    C[idx] = i == p ? 1.0 : 0.0;
  }
}

// chi[p][a] = V[a n + p] for p < nrows: the first rows of column-major
// eigenvectors, through a 32 x 32 shared-memory tile
__global__ void k_rows_of_columns(int n, int nrows, const double* __restrict__ V, double* __restrict__ chi,
                                  long ldchi) {
  __shared__ double t[32][33];
  const long a0 = (long)blockIdx.x * 32, p0 = (long)blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {  // read down a column (p fastest)
    const long a = a0 + j, p = p0 + threadIdx.x;
    t[j][threadIdx.x] = (a < n && p < nrows) ? V[a * n + p] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {  // write along a row (a fastest)
    const long p = p0 + j, a = a0 + threadIdx.x;
    if (p < nrows && a < n) chi[p * ldchi + a] = t[threadIdx.x][j];
  }
}

static mgw_status eig_dense_64(mgw_handle* h, int n, int nrows, double* H, double* E, double* chi, long ldchi) {
  ProfSpan span(h, "syevd_64");
  cusolverDnParams_t params = nullptr;
  MGW_SOLVER(h, cusolverDnCreateParams(&params));
  size_t dbytes = 0, hbytes = 0;
  cusolverStatus_t s = cusolverDnXsyevd_bufferSize(h->solver, params, CUSOLVER_EIG_MODE_VECTOR,
                                                   CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, H, n, CUDA_R_64F, E,
                                                   CUDA_R_64F, &dbytes, &hbytes);
  void* dwork = nullptr;
  std::vector<char> hwork(std::max<size_t>(hbytes, 1));
  if (s == CUSOLVER_STATUS_SUCCESS) {
    const cudaError_t ce = cudaMallocAsync(&dwork, std::max<size_t>(dbytes, 16), h->stream);
    if (ce != cudaSuccess) {
      cusolverDnDestroyParams(params);
      return fail(h, MGW_ERR_NOMEM, "syevd_64: %zu bytes of workspace: %s", dbytes, cudaGetErrorString(ce));
    }
    s = cusolverDnXsyevd(h->solver, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, H, n,
                         CUDA_R_64F, E, CUDA_R_64F, dwork, dbytes, hwork.data(), hbytes, h->dinfo);
    cudaFreeAsync(dwork, h->stream);
  }
  cusolverDnDestroyParams(params);
  if (s != CUSOLVER_STATUS_SUCCESS) return fail(h, MGW_ERR_CUDA, "syevd_64: cusolver status %d (n = %d)", (int)s, n);
  int info = 0;
  MGW_CUDA(h, cudaMemcpyAsync(&info, h->dinfo, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (info != 0) return fail(h, MGW_ERR_NO_CONV, "syevd_64: info = %d (n = %d)", info, n);
  k_rows_of_columns<<<dim3(cdiv(n, 32), cdiv(nrows, 32)), dim3(32, 8), 0, h->stream>>>(n, nrows, H, chi, ldchi);
  return check_launch(h, "rows_of_columns");
}

mgw_status eig_physical_rows(mgw_handle* h, int n, int nrows, double* H, double* E, double* chi, long ldchi) {
  if (n <= 0) return MGW_OK;
  // workspace queries first: where the 32-bit routines refuse the size, the
  // 64-bit syevd runs instead (the queries read no data; H stands in for
  // every device pointer they take)
  int lwork = 0, lw2 = 0;
  const bool fits32 =
      cusolverDnDsytrd_bufferSize(h->solver, CUBLAS_FILL_MODE_LOWER, n, H, n, H, H, H, &lwork) ==
          CUSOLVER_STATUS_SUCCESS &&
      cusolverDnDormtr_bufferSize(h->solver, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, n, nrows, H, n,
                                  H, H, n, &lw2) == CUSOLVER_STATUS_SUCCESS;
  if (!fits32) return eig_dense_64(h, n, nrows, H, E, chi, ldchi);
  const long n2 = (long)n * n;
  const int nb = std::min(n, 4096);  // eigenvectors per inverse-iteration batch
  double *d, *e, *e2, *tau, *bounds, *P, *Z, *U0, *U1, *U2, *ML;
  unsigned char* PV;
  MGW_TRY(slot_buffer(h, 70, (size_t)n, &d));
  MGW_TRY(slot_buffer(h, 71, (size_t)n, &e));
  MGW_TRY(slot_buffer(h, 72, (size_t)n, &e2));
  MGW_TRY(slot_buffer(h, 73, (size_t)n, &tau));
  MGW_TRY(slot_buffer(h, 74, 4, &bounds));
  MGW_TRY(slot_buffer(h, 75, (size_t)n * nrows, &P));
  MGW_TRY(slot_buffer(h, 76, (size_t)n2, &Z));
  MGW_TRY(slot_buffer(h, 77, (size_t)n * nb, &U0));
  MGW_TRY(slot_buffer(h, 78, (size_t)n * nb, &U1));
  MGW_TRY(slot_buffer(h, 79, (size_t)n * nb, &U2));
  MGW_TRY(slot_buffer(h, 80, (size_t)n * nb, &ML));
  double* pvd;
  MGW_TRY(slot_buffer(h, 81, ((size_t)n * nb + 7) / 8, &pvd));
  PV = reinterpret_cast<unsigned char*>(pvd);

  // 1. H = Q T Q^T (lower storage; H is symmetric, row- and column-major alike)
  lwork = std::max(std::max(lwork, lw2), 1);
  double* work;
  MGW_TRY(slot_buffer(h, 82, (size_t)lwork, &work));
  MGW_SOLVER(h, cusolverDnDsytrd(h->solver, CUBLAS_FILL_MODE_LOWER, n, H, n, d, e, tau, work, lwork, h->dinfo));
  // 4a. the first nrows rows of Q: column p of Q^T e_p, column-major n x nrows = row-major [nrows][n]
  k_unit_columns<<<cdiv((long)n * nrows, 256) > 152u * 16 ? 152u * 16 : cdiv((long)n * nrows, 256), 256, 0,
                   h->stream>>>(n, nrows, P);
  MGW_TRY(check_launch(h, "unit_columns"));
  MGW_SOLVER(h, cusolverDnDormtr(h->solver, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, n, nrows, H, n,
                                 tau, P, n, work, lwork, h->dinfo));
  // 2. eigenvalues of T
  k_tri_bounds<<<1, 256, 0, h->stream>>>(n, d, e, bounds);
  k_square<<<cdiv(n, 256), 256, 0, h->stream>>>(n - 1, e, e2);
  MGW_TRY(check_launch(h, "tri_bounds"));
  {
    ProfSpan span(h, "tri_bisect");
    k_bisect<<<cdiv(n, 128), 128, 0, h->stream>>>(n, d, e2, bounds, E);
    MGW_TRY(check_launch(h, "tri_bisect"));
  }
  // 3. eigenvectors of T, in batches, then clusters re-orthogonalised
  std::vector<double> hE(n);
  MGW_CUDA(h, cudaMemcpyAsync(hE.data(), E, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  const double tnorm = std::max(std::fabs(hE.front()), std::fabs(hE.back()));
  {
    ProfSpan span(h, "tri_inverse_iteration");
    for (int a0 = 0; a0 < n; a0 += nb) {
      const int cnt = std::min(nb, n - a0);
      k_inverse_iteration<<<cdiv(cnt, 128), 128, 0, h->stream>>>(n, d, e, E, a0, cnt, U0, U1, U2, ML, PV, Z, n,
                                                                  tnorm);
      MGW_TRY(check_launch(h, "tri_inverse_iteration"));
    }
  }
  std::vector<int> clusters;
  const double ctol = 1e-9 * std::max(tnorm, 1.0);
  for (int i = 0; i < n;) {
    int k = i + 1;
    while (k < n && hE[k] - hE[k - 1] < ctol) ++k;
    if (k - i > 1) {
      clusters.push_back(i);
      clusters.push_back(k);
    }
    i = k;
  }
  if (!clusters.empty()) {
    int* dcl;
    double* cld;
    MGW_TRY(slot_buffer(h, 83, (clusters.size() + 1) / 2, &cld));
    dcl = reinterpret_cast<int*>(cld);
    MGW_CUDA(h, cudaMemcpyAsync(dcl, clusters.data(), sizeof(int) * clusters.size(), cudaMemcpyHostToDevice,
                                h->stream));
    k_cluster_mgs<<<(unsigned)(clusters.size() / 2), 256, 0, h->stream>>>(n, dcl, Z, n);
    MGW_TRY(check_launch(h, "tri_cluster_mgs"));
    MGW_CUDA(h, cudaStreamSynchronize(h->stream));  // the host cluster list outlives no call
  }
  // 4b. chi = Q[0:nrows, :] Z on the tensor cores (FP64-accurate)
  return oz::gemm_fp64_tc_nn(h, nrows, n, n, P, n, Z, n, chi, ldchi, "qp_back_transform");
}

}  // namespace mgw
