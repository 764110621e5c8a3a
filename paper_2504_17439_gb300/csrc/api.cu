// Handle lifecycle, options, workspace, errors, and the dense FP64 helpers
// shared by the stages of the path.
#include "mgw_internal.h"

#include <cmath>
#include <cstring>

namespace mgw {

mgw_status fail(mgw_handle* h, mgw_status s, const char* fmt, ...) {
  if (h) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return s;
}

mgw_status ws_reserve(mgw_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return MGW_OK;
  // queued work may still use the old block
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->ws) MGW_CUDA(h, cudaFree(h->ws));
  h->ws = nullptr;
  h->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&h->ws, bytes);
  if (e != cudaSuccess) {
    h->ws = nullptr;
    return fail(h, MGW_ERR_NOMEM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  h->ws_bytes = bytes;
  return MGW_OK;
}

mgw_status slot_buffer(mgw_handle* h, int id, size_t count, double** out) {
  if ((int)h->slots.size() <= id) h->slots.resize(id + 1, {nullptr, 0});
  auto& sl = h->slots[id];
  const size_t bytes = count * sizeof(double);
  if (sl.second < bytes) {
    MGW_CUDA(h, cudaStreamSynchronize(h->stream));
    if (sl.first) MGW_CUDA(h, cudaFree(sl.first));
    sl.first = nullptr;
    sl.second = 0;
    cudaError_t e = cudaMalloc(&sl.first, bytes);
    if (e != cudaSuccess) {
      sl.first = nullptr;
      return fail(h, MGW_ERR_NOMEM, "slot buffer of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    sl.second = bytes;
  }
  *out = static_cast<double*>(sl.first);
  return MGW_OK;
}

mgw_status gemm_nn(mgw_handle* h, long M, long N, long K, double alpha, const double* A, long lda,
                   const double* B, long ldb, double beta, double* C, long ldc) {
  return dgemm<64, 64>(h, M, N, K, 1, ARowMajor{A, lda, 0}, BRowMajor{B, ldb, 0},
                       EpiStore{C, ldc, 0, alpha, beta}, "gemm_nn");
}
mgw_status gemm_nt(mgw_handle* h, long M, long N, long K, double alpha, const double* A, long lda,
                   const double* B, long ldb, double beta, double* C, long ldc) {
  return dgemm<64, 64>(h, M, N, K, 1, ARowMajor{A, lda, 0}, BNMajor{B, ldb, 0},
                       EpiStore{C, ldc, 0, alpha, beta}, "gemm_nt");
}
mgw_status gemm_tn(mgw_handle* h, long M, long N, long K, double alpha, const double* A, long lda,
                   const double* B, long ldb, double beta, double* C, long ldc) {
  // A stored as [K][M]: A(m,k) = A[k*lda + m]
  return dgemm<64, 64>(h, M, N, K, 1, AKMajor2{A, K > 0 ? K : 1, 0, lda, 0}, BRowMajor{B, ldb, 0},
                       EpiStore{C, ldc, 0, alpha, beta}, "gemm_tn");
}

mgw_status syevd(mgw_handle* h, int n, double* a, double* w) {
  if (n <= 0) return MGW_OK;
  int lwork = 0;
  MGW_SOLVER(h, cusolverDnDsyevd_bufferSize(h->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                            n, a, n, w, &lwork));
  double* work = nullptr;
  MGW_CUDA(h, cudaMallocAsync(&work, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1), h->stream));
  cusolverStatus_t s = cusolverDnDsyevd(h->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                        a, n, w, work, lwork, h->dinfo);
  cudaFreeAsync(work, h->stream);
  if (s != CUSOLVER_STATUS_SUCCESS) return fail(h, MGW_ERR_CUDA, "syevd: cusolver status %d", (int)s);
  int info = 0;
  MGW_CUDA(h, cudaMemcpyAsync(&info, h->dinfo, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (info != 0) return fail(h, MGW_ERR_NO_CONV, "syevd: info = %d (n = %d)", info, n);
  // column-major eigenvectors of a symmetric matrix == row-major rows
  return MGW_OK;
}

mgw_status potrf_potrs(mgw_handle* h, int n, double* a, int nrhs, double* b, bool* not_pd) {
  *not_pd = false;
  int lwork = 0;
  MGW_SOLVER(h, cusolverDnDpotrf_bufferSize(h->solver, CUBLAS_FILL_MODE_LOWER, n, a, n, &lwork));
  double* work = nullptr;
  MGW_CUDA(h, cudaMallocAsync(&work, sizeof(double) * (size_t)(lwork > 0 ? lwork : 1), h->stream));
  cusolverStatus_t s = cusolverDnDpotrf(h->solver, CUBLAS_FILL_MODE_LOWER, n, a, n, work, lwork, h->dinfo);
  cudaFreeAsync(work, h->stream);
  if (s != CUSOLVER_STATUS_SUCCESS) return fail(h, MGW_ERR_CUDA, "potrf: cusolver status %d", (int)s);
  int info = 0;
  MGW_CUDA(h, cudaMemcpyAsync(&info, h->dinfo, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  if (info != 0) {
    *not_pd = true;
    return fail(h, MGW_ERR_NOT_PD, "potrf: leading minor %d not positive definite", info);
  }
  // b is row-major [nrhs][n] == column-major n x nrhs; the solve acts on rows
  MGW_SOLVER(h, cusolverDnDpotrs(h->solver, CUBLAS_FILL_MODE_LOWER, n, nrhs, a, n, b, n, h->dinfo));
  return MGW_OK;
}

__global__ void k_energy_differences(int nocc, int nvir, const double* eps, double* D) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long ov = (long)nocc * nvir;
  if (idx >= ov) return;
  int i = (int)(idx / nvir), a = (int)(idx % nvir);
  D[idx] = eps[nocc + a] - eps[i];
}
mgw_status energy_differences(mgw_handle* h, int nocc, int nvir, const double* eps, double* D) {
  long ov = (long)nocc * nvir;
  k_energy_differences<<<(unsigned)((ov + 255) / 256), 256, 0, h->stream>>>(nocc, nvir, eps, D);
  return check_launch(h, "energy_differences");
}

__global__ void k_scale_columns(long rows, long cols, const double* src, const double* d, double* dst) {
  long total = rows * cols;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    dst[i] = src[i] * d[i % cols];
}
mgw_status scale_columns(mgw_handle* h, long rows, long cols, const double* src, const double* d,
                         double* dst) {
  long total = rows * cols;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_scale_columns<<<(unsigned)blocks, 256, 0, h->stream>>>(rows, cols, src, d, dst);
  return check_launch(h, "scale_columns");
}

__global__ void k_add_identity(int n, double* a, double s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[(long)i * n + i] += s;
}
mgw_status add_identity(mgw_handle* h, int n, double* a, double s) {
  k_add_identity<<<(n + 255) / 256, 256, 0, h->stream>>>(n, a, s);
  return check_launch(h, "add_identity");
}

__global__ void k_extract_ov(int nocc, int nvir, int naux, const double* L, double* Lov) {
  long ov = (long)nocc * nvir;
  long total = ov * naux;
  int nmo = nocc + nvir;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    long Q = idx / ov;
    long r = idx % ov;
    int i = (int)(r / nvir), a = (int)(r % nvir);
    Lov[idx] = L[(Q * nmo + i) * nmo + nocc + a];
  }
}

}  // namespace mgw

using namespace mgw;

extern "C" {

void mgw_options_default(mgw_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->screening = MGW_TDA;
  o->precision = MGW_FP64;
  o->nquad = 48;
  o->xchunk = 0;
  o->rank_tol = 1e-12;
  o->max_iter = 50;
  o->conv_e = 5.0e-3 / 27.211386245988;
  o->conv_mom = 1e-4;
  o->diis_space = 12;
  o->batch_graph = 1;
  o->batch_autotune = 1;
  o->rpa_offset = 0;
}

mgw_status mgw_create(mgw_handle** out, int device, void* stream) {
  if (!out) return MGW_ERR_ARG;
  *out = nullptr;
  mgw_handle* h = new (std::nothrow) mgw_handle();
  if (!h) return MGW_ERR_NOMEM;
  h->device = device;
  h->stream = static_cast<cudaStream_t>(stream);
  if (cudaSetDevice(device) != cudaSuccess) { delete h; return MGW_ERR_CUDA; }
  if (cusolverDnCreate(&h->solver) != CUSOLVER_STATUS_SUCCESS) { delete h; return MGW_ERR_CUDA; }
  cusolverDnSetStream(h->solver, h->stream);
  if (cudaMalloc(&h->dinfo, sizeof(int)) != cudaSuccess) {
    cusolverDnDestroy(h->solver);
    delete h;
    return MGW_ERR_NOMEM;
  }
  *out = h;
  return MGW_OK;
}

static void clear_spans(mgw_handle* h) {
  for (auto& sp : h->spans) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  h->spans.clear();
}

mgw_status mgw_profile(mgw_handle* h, int enable) {
  if (!h) return MGW_ERR_ARG;
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  clear_spans(h);
  h->prof = enable != 0;
  return MGW_OK;
}

mgw_status mgw_profile_query(mgw_handle* h, const char* name, long* count, double* total_ms) {
  if (!h || !name || !count || !total_ms) return MGW_ERR_ARG;
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  long c = 0;
  double t = 0.0;
  for (auto& sp : h->spans) {
    if (std::strcmp(sp.name, name) != 0 && std::strcmp(name, "*") != 0) continue;
    float ms = 0.f;
    MGW_CUDA(h, cudaEventElapsedTime(&ms, sp.a, sp.b));
    ++c;
    t += ms;
  }
  *count = c;
  *total_ms = t;
  return MGW_OK;
}

long mgw_launch_count(const mgw_handle* h) { return h ? h->launches : 0; }

mgw_status mgw_destroy(mgw_handle* h) {
  if (!h) return MGW_OK;
  cudaStreamSynchronize(h->stream);
  clear_spans(h);
  if (h->batched_plan_free) h->batched_plan_free(h->batched_plan);
  if (h->mixed_plan_free) h->mixed_plan_free(h->mixed_plan);
  if (h->chain_pool_free) h->chain_pool_free(h->chain_pool);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (auto& sl : h->slots)
    if (sl.first) cudaFree(sl.first);
  if (h->ws) cudaFree(h->ws);
  if (h->dinfo) cudaFree(h->dinfo);
  if (h->solver) cusolverDnDestroy(h->solver);
  delete h;
  return MGW_OK;
}

mgw_status mgw_set_stream(mgw_handle* h, void* stream) {
  if (!h) return MGW_ERR_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  cusolverDnSetStream(h->solver, h->stream);
  return MGW_OK;
}

const char* mgw_last_error(const mgw_handle* h) { return h ? h->err.c_str() : "null handle"; }

size_t mgw_workspace_bytes(const mgw_handle* h) { return h ? h->ws_bytes : 0; }

mgw_status mgw_extract_ov(mgw_handle* h, int nocc, int nvir, int naux, const double* L, double* Lov) {
  if (!h) return MGW_ERR_ARG;
  if (nocc < 1 || nvir < 1 || naux < 1 || !L || !Lov)
    return fail(h, MGW_ERR_ARG, "mgw_extract_ov: bad arguments");
  long total = (long)nocc * nvir * naux;
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_extract_ov<<<(unsigned)blocks, 256, 0, h->stream>>>(nocc, nvir, naux, L, Lov);
  return check_launch(h, "extract_ov");
}

}  // extern "C"
