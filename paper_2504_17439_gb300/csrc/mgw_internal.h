// Internal declarations of libmgw: the handle, workspace, error plumbing and
// the FP64 tiled GEMM template every FP64 contraction of the library uses.
#pragma once

#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "mgw.h"

struct mgw_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  cusolverDnHandle_t solver = nullptr;
  void* ws = nullptr;        // device workspace, grows to the high-water mark
  size_t ws_bytes = 0;
  int* dinfo = nullptr;      // device int for solver status words
  std::string err;
  // buffers that persist across inner entry-point calls (which may move ws)
  std::vector<std::pair<void*, size_t>> slots;
  // tracing: launches counted always; CUDA-event pairs per GEMM launch when enabled
  long launches = 0;
  bool prof = false;
  struct Span { const char* name; cudaEvent_t a, b; };
  std::vector<Span> spans;
  // batched Sigma build: the captured graph and tables of the last problem
  // table, replayed while it is unchanged; a stream of its own to capture on
  void* batched_plan = nullptr;
  void (*batched_plan_free)(void*) = nullptr;
  // mixed-precision batched build (batched_mixed.cu): workspace, item tables
  // and the captured graph of the last problem table
  void* mixed_plan = nullptr;
  void (*mixed_plan_free)(void*) = nullptr;
  // whole-chain batches (batched_chain.cu): sub-handles driven by host threads
  void* chain_pool = nullptr;
  void (*chain_pool_free)(void*) = nullptr;
  cudaStream_t capture_stream = nullptr;
  // when set, tensor-core pipelines record wait timeouts here and return
  // without synchronising; whoever set it reads the word once at the end
  int* defer_status = nullptr;
};

namespace mgw {

mgw_status fail(mgw_handle* h, mgw_status s, const char* fmt, ...);

#define MGW_CUDA(h, call)                                                          \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return mgw::fail((h), MGW_ERR_CUDA, "%s failed: %s (%s:%d)", #call,           \
                       cudaGetErrorString(e_), __FILE__, __LINE__);                \
  } while (0)

#define MGW_SOLVER(h, call)                                                        \
  do {                                                                             \
    cusolverStatus_t s_ = (call);                                                  \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                             \
      return mgw::fail((h), MGW_ERR_CUDA, "%s failed: cusolver status %d (%s:%d)", \
                       #call, (int)s_, __FILE__, __LINE__);                        \
  } while (0)

#define MGW_TRY(expr)                 \
  do {                                \
    mgw_status st_ = (expr);          \
    if (st_ != MGW_OK) return st_;    \
  } while (0)

// Ensure the handle's workspace holds at least `bytes`; grows (never shrinks).
mgw_status ws_reserve(mgw_handle* h, size_t bytes);

// A persistent device buffer of at least `count` doubles in slot `id` of the
// handle (grows, never moves while large enough; freed by mgw_destroy).
mgw_status slot_buffer(mgw_handle* h, int id, size_t count, double** out);

// Bump allocator over the handle's workspace for the duration of one call.
struct Arena {
  size_t need = 0;
  std::vector<std::pair<double**, size_t>> slots;
  void add(double** p, size_t count) {
    slots.push_back({p, count});
    need += ((count * sizeof(double) + 255) / 256) * 256;
  }
  mgw_status commit(mgw_handle* h) {
    mgw_status s = ws_reserve(h, need);
    if (s != MGW_OK) return s;
    char* base = static_cast<char*>(h->ws);
    size_t off = 0;
    for (auto& sl : slots) {
      *sl.first = reinterpret_cast<double*>(base + off);
      off += ((sl.second * sizeof(double) + 255) / 256) * 256;
    }
    return MGW_OK;
  }
};

inline mgw_status check_launch(mgw_handle* h, const char* what) {
  ++h->launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(h, MGW_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return MGW_OK;
}

// CUDA-event span around the launches queued during its lifetime, recorded
// under `what` when profiling is on (mgw_profile)
struct ProfSpan {
  mgw_handle* h;
  const char* what;
  cudaEvent_t ea = nullptr;
  ProfSpan(mgw_handle* h_, const char* w) : h(h_), what(w) {
    if (h->prof) {
      cudaEventCreate(&ea);
      cudaEventRecord(ea, h->stream);
    }
  }
  ~ProfSpan() {
    if (!ea) return;
    cudaEvent_t eb = nullptr;
    cudaEventCreate(&eb);
    cudaEventRecord(eb, h->stream);
    h->spans.push_back({what, ea, eb});
  }
  ProfSpan(const ProfSpan&) = delete;
  ProfSpan& operator=(const ProfSpan&) = delete;
};

// ---------------------------------------------------------------------------
// FP64 GEMM  C(m, n) (op)= sum_k A(m, k) B(k, n)
// 256 threads as a 16 x 16 grid, each owning a (BM/16) x (BN/16) block of
// C in a strided pattern (rows ty + 16 i, columns tx + 16 j), K stepped by 16
// with a double-buffered shared-memory stage fed from registers.  FP64 FMA is
// the bound on this part, so the tile only has to keep the DFMA pipe busy.
//
// Operand accessors give the address of element (m, k) of A / (k, n) of B
// for one batch entry; `kContig` says which index is contiguous in memory so
// the tile loads coalesce along it.

struct ARowMajor {  // A(m,k) = p[m*ld + k]
  const double* p; long ld; long bstride;
  static constexpr bool kContig = true;
  __device__ const double* base(int b) const { return p + (long)b * bstride; }
  __device__ long off(long m, long k) const { return m * ld + k; }
  __device__ bool ok(long, long) const { return true; }
};
struct AKMajor2 {  // A(m,k) = p[(k/kdiv)*kshi + (k%kdiv)*kslo + m]
  const double* p; long kdiv, kshi, kslo; long bstride;
  static constexpr bool kContig = false;
  __device__ const double* base(int b) const { return p + (long)b * bstride; }
  __device__ long off(long m, long k) const { return (k / kdiv) * kshi + (k % kdiv) * kslo + m; }
  __device__ bool ok(long, long) const { return true; }
};
// Rows of the stacked moments W[t][P][:] in groups of PB aux rows with all
// nmom orders of a group adjacent; a group occupies gsz >= nmom*PB rows:
// m = g*gsz + t*PB + pl, P = g*PB + pl (rows past nmom*PB are padding).
struct AGroupedMoments {
  const double* p; int nmom, PB, naux, gsz;
  static constexpr bool kContig = true;
  __device__ const double* base(int) const { return p; }
  __device__ bool split(long m, int& t, int& P) const {
    long g = m / gsz; int r = (int)(m % gsz);
    t = r / PB; P = (int)g * PB + r % PB;
    return r < nmom * PB && P < naux;
  }
  __device__ long off(long m, long k) const {
    int t, P; split(m, t, P);
    return ((long)t * naux + P) * naux + k;
  }
  __device__ bool ok(long m, long) const { int t, P; return split(m, t, P); }
};
struct BRowMajor {  // B(k,n) = p[k*ld + n]
  const double* p; long ld; long bstride;
  static constexpr bool kContig = false;
  __device__ const double* base(int b) const { return p + (long)b * bstride; }
  __device__ long off(long k, long n) const { return k * ld + n; }
};
struct BNMajor {  // B(k,n) = p[n*ld + k]
  const double* p; long ld; long bstride;
  static constexpr bool kContig = true;
  __device__ const double* base(int b) const { return p + (long)b * bstride; }
  __device__ long off(long k, long n) const { return n * ld + k; }
};

// Epilogues: called once per owned element after the K loop.
struct EpiStore {  // C = alpha*acc + beta*C
  double* c; long ldc; long bstride; double alpha, beta;
  __device__ void operator()(int b, long m, long n, double acc) const {
    double* q = c + (long)b * bstride + m * ldc + n;
    *q = beta == 0.0 ? alpha * acc : alpha * acc + beta * *q;
  }
};
struct EpiDiagUpdate {  // C = C * d[n] + alpha*acc   (the D-plus-low-rank update)
  double* c; long ldc; const double* d; double alpha;
  __device__ void operator()(int, long m, long n, double acc) const {
    double* q = c + m * ldc + n;
    *q = *q * d[n] + alpha * acc;
  }
};

template <class Epi, class = void>
struct is_tile_epi { static constexpr bool value = false; };
template <class Epi>
struct is_tile_epi<Epi, decltype(void(Epi::kTile))> { static constexpr bool value = Epi::kTile; };

// Launch shape options of dgemm_kernel:
//  tri    - M == N, symmetric result: blockIdx.x enumerates the upper-triangle
//           tiles only (BM == BN) and the epilogue writes (m,n) and (n,m)
//  kchunk - split K: blockIdx.z = batch + nbatch * split, split s covers
//           k in [s*kchunk, (s+1)*kchunk); the epilogue gets the full z
struct LaunchShape { int tri = 0; int nbatch = 1; long kchunk = 0; };

// One output tile: C(m0.., n0..) over k in [kbeg, kend), epilogue batch index bz.
template <int BM, int BN, class AOp, class BOp, class Epi>
__device__ __forceinline__ void dgemm_tile(long M, long N, long K, const AOp& A, const BOp& B, const Epi& epi,
                                           long tile_m, long tile_n, int batch, int bz, long kbeg, long kend,
                                           int tri, double* smem) {
  constexpr int BK = 16, TM = BM / 16, TN = BN / 16;
  constexpr int LA = BM * BK / 256, LB = BN * BK / 256;
  constexpr int SA = BK * (BM + 1), SB = BK * (BN + 1);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long m0 = tile_m * BM, n0 = tile_n * BN;
  const double* Ab = A.base(batch);
  const double* Bb = B.base(batch);
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  double ra[LA], rb[LB];

  auto gload = [&](long k0) {
#pragma unroll
    for (int e = 0; e < LA; ++e) {
      int idx = tid + e * 256, mm, kk;
      if (AOp::kContig) { mm = idx / BK; kk = idx % BK; } else { kk = idx / BM; mm = idx % BM; }
      long m = m0 + mm, k = k0 + kk;
      ra[e] = (m < M && k < kend && A.ok(m, k)) ? __ldg(Ab + A.off(m, k)) : 0.0;
    }
#pragma unroll
    for (int e = 0; e < LB; ++e) {
      int idx = tid + e * 256, nn, kk;
      if (BOp::kContig) { nn = idx / BK; kk = idx % BK; } else { kk = idx / BN; nn = idx % BN; }
      long n = n0 + nn, k = k0 + kk;
      rb[e] = (n < N && k < kend) ? __ldg(Bb + B.off(k, n)) : 0.0;
    }
  };
  auto sstore = [&](int buf) {
    double* As = smem + buf * SA;
    double* Bs = smem + 2 * SA + buf * SB;
#pragma unroll
    for (int e = 0; e < LA; ++e) {
      int idx = tid + e * 256, mm, kk;
      if (AOp::kContig) { mm = idx / BK; kk = idx % BK; } else { kk = idx / BM; mm = idx % BM; }
      As[kk * (BM + 1) + mm] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < LB; ++e) {
      int idx = tid + e * 256, nn, kk;
      if (BOp::kContig) { nn = idx / BK; kk = idx % BK; } else { kk = idx / BN; nn = idx % BN; }
      Bs[kk * (BN + 1) + nn] = rb[e];
    }
  };

  gload(kbeg);
  sstore(0);
  __syncthreads();
  int cur = 0;
  for (long k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) gload(k0 + BK);
    const double* As = smem + cur * SA;
    const double* Bs = smem + 2 * SA + cur * SB;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk * (BM + 1) + ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk * (BN + 1) + tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) sstore(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
  if constexpr (is_tile_epi<Epi>::value) {
    epi.template tile<BM, BN, TM, TN>(bz, m0, n0, M, N, acc, smem, 2 * SA + 2 * SB);
  } else {
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      long m = m0 + ty + 16 * i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        long n = n0 + tx + 16 * j;
        if (n >= N) continue;
        if (tri) {
          if (m > n) continue;  // the (n, m) thread of a diagonal tile is the writer
          epi(bz, m, n, acc[i][j]);
          if (m != n) epi(bz, n, m, acc[i][j]);
        } else {
          epi(bz, m, n, acc[i][j]);
        }
      }
    }
  }
}

template <int BM, int BN>
struct DgemmSmem { static constexpr int kDoubles = 2 * 16 * (BM + 1) + 2 * 16 * (BN + 1); };

__device__ __forceinline__ void tri_tile(long t, long T, long& i, long& j) {
  i = 0;
  while (t >= T - i) { t -= T - i; ++i; }
  j = i + t;
}

template <int BM, int BN, class AOp, class BOp, class Epi>
__global__ void __launch_bounds__(256)
dgemm_kernel(long M, long N, long K, AOp A, BOp B, Epi epi, LaunchShape ls) {
  __shared__ double smem[DgemmSmem<BM, BN>::kDoubles];
  long tile_m = blockIdx.y, tile_n = blockIdx.x;
  if (ls.tri) tri_tile(blockIdx.x, (N + BN - 1) / BN, tile_m, tile_n);
  const int bz = blockIdx.z;
  const int batch = bz % ls.nbatch;
  const long kbeg = ls.kchunk > 0 ? (long)(bz / ls.nbatch) * ls.kchunk : 0;
  const long kend = ls.kchunk > 0 ? (kbeg + ls.kchunk < K ? kbeg + ls.kchunk : K) : K;
  dgemm_tile<BM, BN>(M, N, K, A, B, epi, tile_m, tile_n, batch, bz, kbeg, kend, ls.tri, smem);
}

// Grouped GEMM: one launch over many independent problems of different
// shapes.  tile_start[p] is the first linear tile of problem p (prefix sum,
// tile_start[nprob] = total); a CTA finds its problem by binary search.
template <class AOp, class BOp, class Epi>
struct GroupItem {
  long M, N, K;
  AOp A;
  BOp B;
  Epi epi;
  int tri;
};

template <int BM, int BN, class AOp, class BOp, class Epi>
__global__ void __launch_bounds__(256)
dgemm_grouped_kernel(const GroupItem<AOp, BOp, Epi>* items, const long* tile_start, int nprob) {
  __shared__ double smem[DgemmSmem<BM, BN>::kDoubles];
  const long t = blockIdx.x;
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const GroupItem<AOp, BOp, Epi> it = items[lo];
  const long local = t - tile_start[lo];
  const long tn = (it.N + BN - 1) / BN;
  long tile_m, tile_n;
  if (it.tri) tri_tile(local, tn, tile_m, tile_n);
  else { tile_m = local / tn; tile_n = local % tn; }
  dgemm_tile<BM, BN>(it.M, it.N, it.K, it.A, it.B, it.epi, tile_m, tile_n, 0, 0, 0, it.K, it.tri, smem);
}

template <int BM, int BN, class AOp, class BOp, class Epi>
mgw_status dgemm(mgw_handle* h, long M, long N, long K, int batch, const AOp& A, const BOp& B,
                 const Epi& epi, const char* what, int tri = 0, int nsplit = 1) {
  if (M <= 0 || N <= 0 || batch <= 0) return MGW_OK;
  LaunchShape ls;
  ls.tri = tri;
  ls.nbatch = batch;
  if (nsplit > 1) ls.kchunk = ((K + nsplit - 1) / nsplit + 15) / 16 * 16;
  const long splits = ls.kchunk > 0 ? (K + ls.kchunk - 1) / ls.kchunk : 1;
  const long tn = (N + BN - 1) / BN, tm = (M + BM - 1) / BM;
  dim3 grid(tri ? (unsigned)(tn * (tn + 1) / 2) : (unsigned)tn, tri ? 1u : (unsigned)tm,
            (unsigned)(batch * splits));
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (h->prof) {
    cudaEventCreate(&ea);
    cudaEventCreate(&eb);
    cudaEventRecord(ea, h->stream);
  }
  dgemm_kernel<BM, BN, AOp, BOp, Epi><<<grid, 256, 0, h->stream>>>(M, N, K, A, B, epi, ls);
  mgw_status st = check_launch(h, what);
  if (h->prof) {
    cudaEventRecord(eb, h->stream);
    h->spans.push_back({what, ea, eb});
  }
  return st;
}

// Plain row-major helpers: C = alpha * op(A) op(B) + beta * C (single matrix).
mgw_status gemm_nn(mgw_handle* h, long M, long N, long K, double alpha, const double* A, long lda,
                   const double* B, long ldb, double beta, double* C, long ldc);
mgw_status gemm_nt(mgw_handle* h, long M, long N, long K, double alpha, const double* A, long lda,
                   const double* B, long ldb, double beta, double* C, long ldc);
mgw_status gemm_tn(mgw_handle* h, long M, long N, long K, double alpha, const double* A, long lda,
                   const double* B, long ldb, double beta, double* C, long ldc);

// Dense FP64 helpers built on the solver library (symmetric eigensolve,
// Cholesky factor + solve).  Row-major symmetric matrices; on return of
// syevd, row j of `a` holds eigenvector j (eigenvalues ascending in w).
mgw_status syevd(mgw_handle* h, int n, double* a, double* w);
// Eigenvalues E [n] (ascending) of the symmetric H [n][n] and the first
// nrows rows of its eigenvectors, chi[p][a] = X_pa (ld ldchi); H is
// overwritten (tridiag.cu)
mgw_status eig_physical_rows(mgw_handle* h, int n, int nrows, double* H, double* E, double* chi, long ldchi);
mgw_status potrf_potrs(mgw_handle* h, int n, double* a, int nrhs, double* b, bool* not_pd);

// Small elementwise kernels
mgw_status energy_differences(mgw_handle* h, int nocc, int nvir, const double* eps, double* D);
// mgw_sigma_moments_batched under MGW_MIXED: one grouped tensor-core launch
// per stage over all systems (batched_mixed.cu)
mgw_status sigma_moments_batched_mixed(mgw_handle* h, const mgw_options* o, int nsys, int nmom,
                                       const mgw_system* sys);
mgw_status scale_columns(mgw_handle* h, long rows, long cols, const double* src, const double* d,
                         double* dst);  // dst[r][c] = src[r][c] * d[c]
mgw_status add_identity(mgw_handle* h, int n, double* a, double s);  // a += s * I
// Fock build of a restricted closed-shell reference, F[rho] = hcore + J[rho]
// - K[rho]/2 with J_pq = sum_P L_Ppq sum_rs L_Prs rho_rs and K_pq =
// sum_P sum_rs L_Ppr rho_rs L_Psq (rho spin-summed); scratch v [naux],
// tmp [naux][nmo][nmo]
mgw_status fock_build(mgw_handle* h, int nmo, int naux, const double* hcore, const double* L, const double* rho,
                      double* out, double* v, double* tmp);
// Pulay DIIS coefficients on the host: minimise |sum c_i e_i| subject to
// sum c_i = 1 from the Gram matrix B [n][n] of the errors; false if singular
bool diis_solve(const std::vector<double>& B, int n, std::vector<double>& c);


// ---- Y-stage tile epilogue of the FP64 Sigma build (Eqs. 6-7): rows of the
// tile are (t, pl) with t = r / PB, pl = r % PB; columns (x_local, q) of the
// chunk.  The epilogue stages the tile in shared memory, half the columns at
// a time, and writes only
//   Z(n)[P][(x,q)] = sum_{t<=n} c(n,t) eps_x^(n-t) Y(t)[P][(x,q)],
// c(n,t) = 2 C(n,t) s^t from a table (s = -1 hole, +1 particle), so Y never
// reaches HBM.  Coef gives the table: held by value (one launch, one sector)
// or through a device pointer (grouped launches over many systems).
constexpr int kMaxBinomMom = 24;
struct BinomCoef {
  double c[kMaxBinomMom * (kMaxBinomMom + 1) / 2];  // c(n,t) at n(n+1)/2 + t
  __device__ const double* row(int n) const { return c + n * (n + 1) / 2; }
};
struct BinomCoefRef {
  const BinomCoef* p;
  __device__ const double* row(int n) const { return p->row(n); }
};
template <class Coef>
struct EpiBinomialT {
  static constexpr bool kTile = true;
  double* Z;           // [nmom][naux][ncol]
  const double* eps;   // eps_x of the chunk's first x at eps[0]
  int nmom, PB, naux, nmo;
  long ncol;           // xc * nmo
  Coef bc;

  template <int BM, int BN, int TM, int TN>
  __device__ void tile(int, long m0, long n0, long, long N, double (&acc)[TM][TN], double* smem, int) const {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    constexpr int HALF = BN / 2;  // stage half the columns at a time
    static_assert((TN % 2) == 0, "TN must be even");
    const long g = m0 / BM;       // tile == one group of PB aux rows
    for (int hf = 0; hf < 2; ++hf) {
      __syncthreads();
      // acc columns tx + 16 j with j in [hf*TN/2, (hf+1)*TN/2) -> smem [BM][HALF+1]
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN / 2; ++jj) {
          const int j = hf * (TN / 2) + jj;
          smem[(ty + 16 * i) * (HALF + 1) + tx + 16 * j - hf * HALF] = acc[i][j];
        }
      __syncthreads();
      for (int pi = tid; pi < PB * HALF; pi += 256) {
        const int pl = pi / HALF, col = pi % HALF;
        const long P = g * PB + pl, n = n0 + hf * HALF + col;
        if (P >= naux || n >= N) continue;
        const double e = eps[n / nmo];
        double y[kMaxBinomMom], pe[kMaxBinomMom];
        pe[0] = 1.0;
        for (int t = 0; t < nmom; ++t) {
          y[t] = smem[(t * PB + pl) * (HALF + 1) + col];
          if (t + 1 < nmom) pe[t + 1] = pe[t] * e;
        }
        for (int nn = 0; nn < nmom; ++nn) {
          const double* cr = bc.row(nn);
          double z = 0.0;
          for (int t = 0; t <= nn; ++t) z = fma(cr[t] * pe[nn - t], y[t], z);
          Z[((long)nn * naux + P) * ncol + n] = z;
        }
      }
    }
  }
};
// the table c(n,t) = 2 C(n,t) s^t for one sector
inline void binomial_table(int nmom, double s, BinomCoef& bc) {
  for (int n = 0; n < nmom; ++n) {
    double c = 1.0, sg = 1.0;
    for (int t = 0; t <= n; ++t) {
      bc.c[n * (n + 1) / 2 + t] = 2.0 * c * sg;
      c = c * (n - t) / (t + 1);
      sg *= s;
    }
  }
}

}  // namespace mgw
