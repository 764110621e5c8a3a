// Many independent systems of uneven size in one pass: the TDA response
// recursion and the Sigma-moment build of every system, each stage issued as
// ONE grouped launch over all systems (dgemm_grouped_kernel: a CTA finds its
// system and tile from a prefix sum of tile counts).  Per stage:
//   order t:   W_s(t) = T_s V_s^T  (all s, upper tiles)   -> 1 launch
//              T_s <- T_s o D_s + 2 W_s(t) V_s          -> 1 launch
//   round r:   Y stage + binomial for chunk r of every s  -> 1 launch
//              GEMM2 for chunk r of every s, every n      -> 1 launch
// Chunks of Green's-function indices are sized per system so that all
// systems finish in about the same number of rounds.
#include "mgw_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mgw {

// the binomial epilogue of sigma.cu, restated for grouped use (same arithmetic)
struct BinomCoefB {
  double c[24 * 25 / 2];
};
struct EpiBinomialB {
  static constexpr bool kTile = true;
  double* Z;
  const double* eps;
  int nmom, PB, naux, nmo;
  long ncol;
  const BinomCoefB* bc;  // device pointer (hole, particle tables)
  template <int BM, int BN, int TM, int TN>
  __device__ void tile(int, long m0, long n0, long, long N, double (&acc)[TM][TN], double* smem, int) const {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    constexpr int HALF = BN / 2;
    const long g = m0 / BM;
    for (int hf = 0; hf < 2; ++hf) {
      __syncthreads();
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN / 2; ++jj) {
          int j = hf * (TN / 2) + jj;
          smem[(ty + 16 * i) * (HALF + 1) + tx + 16 * j - hf * HALF] = acc[i][j];
        }
      __syncthreads();
      for (int pi = tid; pi < PB * HALF; pi += 256) {
        int pl = pi / HALF, col = pi % HALF;
        long P = g * PB + pl, n = n0 + hf * HALF + col;
        if (P >= naux || n >= N) continue;
        double e = eps[n / nmo];
        double y[24], pe[24];
        pe[0] = 1.0;
        for (int t = 0; t < nmom; ++t) {
          y[t] = smem[(t * PB + pl) * (HALF + 1) + col];
          if (t + 1 < nmom) pe[t + 1] = pe[t] * e;
        }
        for (int nn = 0; nn < nmom; ++nn) {
          const double* cr = bc->c + nn * (nn + 1) / 2;
          double z = 0.0;
          for (int t = 0; t <= nn; ++t) z = fma(cr[t] * pe[nn - t], y[t], z);
          Z[((long)nn * naux + P) * ncol + n] = z;
        }
      }
    }
  }
};

template <int BM, int BN, class AOp, class BOp, class Epi>
static mgw_status grouped(mgw_handle* h, const std::vector<GroupItem<AOp, BOp, Epi>>& items, const char* what) {
  if (items.empty()) return MGW_OK;
  std::vector<long> start(items.size() + 1, 0);
  for (size_t i = 0; i < items.size(); ++i) {
    const long tn = (items[i].N + BN - 1) / BN, tm = (items[i].M + BM - 1) / BM;
    start[i + 1] = start[i] + (items[i].tri ? tn * (tn + 1) / 2 : tn * tm);
  }
  const size_t ib = sizeof(GroupItem<AOp, BOp, Epi>) * items.size();
  const size_t sb = sizeof(long) * start.size();
  double* buf = nullptr;
  MGW_CUDA(h, cudaMallocAsync(reinterpret_cast<void**>(&buf), ib + sb + 256, h->stream));
  char* base = reinterpret_cast<char*>(buf);
  auto* ditems = reinterpret_cast<GroupItem<AOp, BOp, Epi>*>(base);
  auto* dstart = reinterpret_cast<long*>(base + ((ib + 255) / 256) * 256);
  MGW_CUDA(h, cudaMemcpyAsync(ditems, items.data(), ib, cudaMemcpyHostToDevice, h->stream));
  MGW_CUDA(h, cudaMemcpyAsync(dstart, start.data(), sb, cudaMemcpyHostToDevice, h->stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
  }
  dgemm_grouped_kernel<BM, BN, AOp, BOp, Epi>
      <<<(unsigned)start.back(), 256, 0, h->stream>>>(ditems, dstart, (int)items.size());
  mgw_status st = check_launch(h, what);
  if (h->prof) {
    cudaEventRecord(e1, h->stream);
    h->spans.push_back({what, e0, e1});
  }
  // host copies of pageable memory complete before cudaMemcpyAsync returns;
  // the device buffer is released in stream order
  cudaFreeAsync(buf, h->stream);
  return st;
}

}  // namespace mgw

using namespace mgw;

extern "C" mgw_status mgw_sigma_moments_batched(mgw_handle* h, const mgw_options* o, int nsys, int nmom,
                                                const mgw_system* sys) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (nsys < 1 || !sys || nmom < 1 || nmom > 24)
    return fail(h, MGW_ERR_ARG, "mgw_sigma_moments_batched: bad arguments");
  if (o->screening != MGW_TDA)
    return fail(h, MGW_ERR_UNSUPPORTED, "mgw_sigma_moments_batched: TDA screening only");
  for (int s = 0; s < nsys; ++s)
    if (sys[s].nocc < 1 || sys[s].nvir < 1 || sys[s].naux < 1 || !sys[s].eps || !sys[s].L || !sys[s].sig_hole ||
        !sys[s].sig_part)
      return fail(h, MGW_ERR_ARG, "mgw_sigma_moments_batched: bad system %d", s);
  MGW_CUDA(h, cudaSetDevice(h->device));
  constexpr int BM = 96, BN = 64;
  const int PB = std::max(1, BM / nmom);
  const int rounds_per_sector = 4;

  // workspace per system: D, Lov, T, W, Z (chunked), all in one arena
  struct Sys {
    long nmo, ov, naux, xc_h, xc_p;
    double *D, *Lov, *T, *W, *Z;
  };
  std::vector<Sys> S(nsys);
  Arena ar;
  for (int s = 0; s < nsys; ++s) {
    Sys& q = S[s];
    q.nmo = sys[s].nocc + sys[s].nvir;
    q.ov = (long)sys[s].nocc * sys[s].nvir;
    q.naux = sys[s].naux;
    q.xc_h = std::max(1L, ((long)sys[s].nocc + rounds_per_sector - 1) / rounds_per_sector);
    q.xc_p = std::max(1L, ((long)sys[s].nvir + rounds_per_sector - 1) / rounds_per_sector);
    const long xc = std::max(q.xc_h, q.xc_p);
    ar.add(&q.D, q.ov);
    ar.add(&q.Lov, q.naux * q.ov);
    ar.add(&q.T, q.naux * q.ov);
    ar.add(&q.W, (long)nmom * q.naux * q.naux);
    ar.add(&q.Z, (long)nmom * q.naux * xc * q.nmo);
  }
  double* coef = nullptr;
  ar.add(&coef, 2 * sizeof(BinomCoefB) / sizeof(double));
  MGW_TRY(ar.commit(h));

  // binomial tables 2 C(n,t) s^t for s = -1 (hole) and +1 (particle)
  BinomCoefB hc[2];
  for (int sec = 0; sec < 2; ++sec) {
    const double sgn = sec == 0 ? -1.0 : 1.0;
    for (int n = 0; n < nmom; ++n) {
      double c = 1.0, sg = 1.0;
      for (int t = 0; t <= n; ++t) {
        hc[sec].c[n * (n + 1) / 2 + t] = 2.0 * c * sg;
        c = c * (n - t) / (t + 1);
        sg *= sgn;
      }
    }
  }
  MGW_CUDA(h, cudaMemcpyAsync(coef, hc, sizeof hc, cudaMemcpyHostToDevice, h->stream));
  const BinomCoefB* dcoef = reinterpret_cast<const BinomCoefB*>(coef);

  for (int s = 0; s < nsys; ++s) {
    MGW_TRY(mgw_extract_ov(h, sys[s].nocc, sys[s].nvir, sys[s].naux, sys[s].L, S[s].Lov));
    MGW_TRY(energy_differences(h, sys[s].nocc, sys[s].nvir, sys[s].eps, S[s].D));
    MGW_CUDA(h, cudaMemcpyAsync(S[s].T, S[s].Lov, sizeof(double) * S[s].naux * S[s].ov, cudaMemcpyDeviceToDevice,
                                h->stream));
  }

  // TDA recursion, one grouped launch per GEMM kind and order
  for (int t = 0; t < nmom; ++t) {
    std::vector<GroupItem<ARowMajor, BNMajor, EpiStore>> wi;
    for (int s = 0; s < nsys; ++s) {
      const Sys& q = S[s];
      wi.push_back({q.naux, q.naux, q.ov, ARowMajor{q.T, q.ov, 0}, BNMajor{q.Lov, q.ov, 0},
                    EpiStore{q.W + (long)t * q.naux * q.naux, q.naux, 0, 1.0, 0.0}, 1});
    }
    MGW_TRY((grouped<64, 64>(h, wi, "w_gemm_grouped")));
    if (t + 1 == nmom) break;
    std::vector<GroupItem<ARowMajor, BRowMajor, EpiDiagUpdate>> ti;
    for (int s = 0; s < nsys; ++s) {
      const Sys& q = S[s];
      ti.push_back({q.naux, q.ov, q.naux, ARowMajor{q.W + (long)t * q.naux * q.naux, q.naux, 0},
                    BRowMajor{q.Lov, q.ov, 0}, EpiDiagUpdate{q.T, q.ov, q.D, 2.0}, 0});
    }
    MGW_TRY((grouped<64, 64>(h, ti, "t_update_grouped")));
  }

  // Sigma build: rounds of chunks (hole sector, then particle sector)
  for (int sec = 0; sec < 2; ++sec) {
    for (int r = 0;; ++r) {
      std::vector<GroupItem<AGroupedMoments, BRowMajor, EpiBinomialB>> yi;
      std::vector<GroupItem<AKMajor2, BRowMajor, EpiStore>> gi;
      for (int s = 0; s < nsys; ++s) {
        const Sys& q = S[s];
        const long xbeg = sec == 0 ? 0 : sys[s].nocc, xend = sec == 0 ? sys[s].nocc : q.nmo;
        const long xc = sec == 0 ? q.xc_h : q.xc_p;
        const long x0 = xbeg + r * xc;
        if (x0 >= xend) continue;
        const long nx = std::min(xc, xend - x0);
        const long ncol = nx * q.nmo;
        const long ngroups = (q.naux + PB - 1) / PB;
        yi.push_back({ngroups * BM, ncol, q.naux, AGroupedMoments{q.W, nmom, PB, (int)q.naux, BM},
                      BRowMajor{sys[s].L + x0 * q.nmo, q.nmo * q.nmo, 0},
                      EpiBinomialB{q.Z, sys[s].eps + x0, nmom, PB, (int)q.naux, (int)q.nmo, ncol, dcoef + sec}, 0});
        double* sig = sec == 0 ? sys[s].sig_hole : sys[s].sig_part;
        for (int n = 0; n < nmom; ++n)
          gi.push_back({q.nmo, q.nmo, q.naux * nx, AKMajor2{sys[s].L + x0 * q.nmo, nx, q.nmo * q.nmo, q.nmo, 0},
                        BRowMajor{q.Z + (long)n * q.naux * ncol, q.nmo, 0},
                        EpiStore{sig + (long)n * q.nmo * q.nmo, q.nmo, 0, 1.0, r == 0 ? 0.0 : 1.0}, 1});
      }
      if (yi.empty()) break;
      MGW_TRY((grouped<BM, BN>(h, yi, "sigma_y_binomial_grouped")));
      MGW_TRY((grouped<64, 64>(h, gi, "sigma_gemm2_grouped")));
    }
  }
  return MGW_OK;
}
