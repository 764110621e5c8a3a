// The tensor-core Y stage's epilogue (binomial weighting of the moments),
// shared by the single-system Sigma build and the grouped batch.
#pragma once

#include "mgw_internal.h"
#include "ozaki.h"

namespace mgw {

// Binomial epilogue of the tensor-core Y stage.  Each of the 256 epilogue
// threads holds KC FP64 results of one tile row (t, pl) (the tile has 2 KC
// columns: 96 on the FP64_TC path, 64 on the mixed one); they are staged in
// shared memory (the freed pipeline buffers) and recombined per (pl, column).
// Z(n) = 2 sum_t C(n,t) s^t e^(n-t) Y(t) is a Taylor shift: with e' = s e,
// repeated a_t += e' a_(t-1) (t descending, nmom - 1 sweeps) turns a_t = Y(t)
// into sum_t C(n,t) e'^(n-t) Y(t), and Z(n) = 2 s^n a_n.  NMAX >= nmom bounds
// the unrolled sweeps so that a[] stays in registers.
template <int NMAX>
struct EpiBinomialTC {
  double* Z;
  const double* eps;
  int nmom, PB, naux, nmo;
  long ncol;
  double sgn;
  __device__ bool skip_tile(int, int, int, int, int) const { return false; }
  template <int KC>
  __device__ __forceinline__ void operator()(int row_local, int col_base, int m0, int n0, int, int N,
                                             const long long (&v)[KC], double* smem) const {
    constexpr int TBN = 2 * KC, LD = TBN + 1;
    const int tid = threadIdx.x - 32 * oz::kEpiWarp0;
    const int pairs = PB * TBN;
    // eps_x of this thread's next (pl, column) pair, loaded one pair ahead
    auto eps_of = [&](int pi) { const long n = n0 + pi % TBN; return n < N ? eps[n / nmo] : 0.0; };
    double e_next = tid < pairs ? eps_of(tid) : 0.0;
#pragma unroll
    for (int j = 0; j < KC; ++j) smem[row_local * LD + col_base + j] = __longlong_as_double(v[j]);
    tc::named_bar(1, 256);
    const long g = m0 / 128;
    for (int pi = tid; pi < pairs; pi += 256) {
      const double e_cur = e_next;
      if (pi + 256 < pairs) e_next = eps_of(pi + 256);
      const int pl = pi / TBN, col = pi % TBN;
      const long P = g * PB + pl;
      const long n = n0 + col;
      if (P >= naux || n >= N) continue;
      const double es = sgn * e_cur;
      double a[NMAX];
#pragma unroll
      for (int t = 0; t < NMAX; ++t) a[t] = t < nmom ? smem[(t * PB + pl) * LD + col] : 0.0;
#pragma unroll
      for (int j = 1; j < NMAX; ++j) {
        if (j < nmom) {
#pragma unroll
          for (int t = NMAX - 1; t >= j; --t) a[t] = fma(es, a[t - 1], a[t]);
        }
      }
      double f = 2.0;
#pragma unroll
      for (int t = 0; t < NMAX; ++t) {
        if (t < nmom) Z[((long)t * naux + P) * ncol + n] = f * a[t];
        f *= sgn;
      }
    }
  }
  __device__ void abort() const { tc::named_bar(1, 256); }
};

}  // namespace mgw
