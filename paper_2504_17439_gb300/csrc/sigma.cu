// Hole and particle self-energy moments, FP64 path (Eqs. 6-7 with Eq. 15).
//
//   Sigma(n)_pq = 2 sum_x sum_t C(n,t) s^t eps_x^(n-t) [L_x^T W(t) L_x]_pq,
//   s = -1 for the hole sector (x occupied), +1 for the particle sector.
//
// Per chunk of Green's-function indices x (all in one sector):
//  1. Y-stage GEMM with every moment order stacked along M:
//       Y(t)[P][(x,q)] = sum_Q W(t)[P][Q] L[Q][x][q]       (L symmetric in x,q)
//     Its M tile holds all nmom orders of a few aux rows P, so the epilogue
//     applies the binomial weighting in shared memory and writes only
//       Z(n)[P][(x,q)] = 2 sum_{t<=n} C(n,t) s^t eps_x^(n-t) Y(t)[P][(x,q)];
//     Y never reaches HBM.
//  2. GEMM2, batched over n:  Sigma(n)[p][q] += sum_{P,x} L[P][x][p] Z(n)[P][(x,q)].
//
// With precision MGW_FP64_TC the Y stage runs on the tensor cores as an
// FP64-accurate digit-sliced GEMM (ozaki.h): W is sliced once in grouped-row
// order (a 128-row tile holds all nmom orders of PB = 128/nmom aux rows), each
// x-chunk of L is sliced as its transpose, and the same binomial weighting
// runs in that kernel's epilogue from shared memory.  With MGW_MIXED both
// products take L on one fixed-point grid for the whole tensor (two digits, a
// BF16 hi/lo split: L' = L rounded to a multiple of 2^(e-16), |L| < 2^(e-1))
// and W, Z on seven digits: 13 digit products instead of 28, every one exact.
// The result is then the moments of the system whose DF tensor is L' (a
// consistent moment sequence, which the block Lanczos step needs), computed
// to FP64 accuracy; L' differs from L by at most 2^-17 of max |L|.
#include "mgw_internal.h"
#include "ozaki.h"
#include "ozaki_mixed.h"
#include "sigma_epi.h"
#include "tc_gemm.h"

#include <algorithm>
#include <cmath>

namespace mgw {

constexpr int kMaxMom = kMaxBinomMom;

// K splits of the tensor-core GEMM2 (rows p, columns (n, q), K = nx naux),
// chosen for its kept (upper-triangle) tiles
static int gemm2_splits(int nmo, int nmom, long K2, int sms, int bn) {
  const int MT = (nmo + oz::BM - 1) / oz::BM;
  const int N = nmom * nmo, NT = (N + bn - 1) / bn;
  long kept = 0;
  for (int mt = 0; mt < MT; ++mt)
    for (int nt = 0; nt < NT; ++nt) kept += oz::sigma_tile_lower(mt * oz::BM, nt * bn, N, nmo, bn) ? 0 : 1;
  return oz::best_split(kept, K2, sms);
}

// sig[i] = (accumulate ? sig[i] : 0) + sum_s part[s * count + i]
__global__ void k_reduce_splits(long count, int nsplit, const double* part, double* sig, int accumulate) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    double acc = accumulate ? sig[i] : 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[(long)s * count + i];
    sig[i] = acc;
  }
}

}  // namespace mgw

using namespace mgw;

// The Sigma build over Green's-function indices x = 0..nxs-1 (the first
// nhole of them holes), with L [naux][nxs][nmo] (row x of slab P is
// L_{P,x q}; for the orbitals themselves nxs = nmo and the slabs are
// symmetric), from the FP64 tensor L, or (Lq != null, MGW_MIXED only) from
// the tensor already on its grid as 16-bit integers with exponent eq.
static mgw_status sigma_impl(mgw_handle* h, const mgw_options* o, int nmo, int nxs, int nhole, int naux, int nmom,
                             const double* eps_G, const double* L, const short* Lq, int eq, const double* Wmom,
                             double* sig_hole, double* sig_part) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (nmo < 1 || nxs < 1 || nhole < 0 || nhole > nxs || naux < 1 || nmom < 1 || nmom > kMaxMom || !eps_G ||
      (!L && !Lq) || !Wmom || !sig_hole || !sig_part)
    return fail(h, MGW_ERR_ARG, "mgw_sigma_moments: bad sizes or null pointer");
  if (Lq && o->precision != MGW_MIXED)
    return fail(h, MGW_ERR_UNSUPPORTED, "mgw_sigma_moments_q: the 16-bit grid tensor is the MGW_MIXED input");
  if (o->precision != MGW_FP64 && o->precision != MGW_FP64_TC && o->precision != MGW_MIXED)
    return fail(h, MGW_ERR_UNSUPPORTED, "mgw_sigma_moments: precision %d not built", o->precision);
  // MGW_MIXED: L enters both products as the same tensor L' (L rounded to one
  // 16-bit fixed-point grid, two digits); W, Y and Z keep seven digits
  const bool mixed = o->precision == MGW_MIXED;
  const bool tc = o->precision == MGW_FP64_TC || mixed;
  const int lns = mixed ? oz::kGridSlices : oz::kSlices;
  MGW_CUDA(h, cudaSetDevice(h->device));
  const long sx = (long)nxs * nmo;  // slab stride of L
  constexpr int BM = 96, BN = 64;
  const int PB = std::max(1, BM / nmom);
  const long ngroups = (naux + PB - 1) / PB;

  // chunk of x per pass: Z holds nmom * naux * xc * nmo doubles (~1 GiB budget)
  const double per_x = (double)nmom * naux * nmo * sizeof(double);
  int xc = o->xchunk > 0 ? o->xchunk : (int)std::max(1.0, std::floor((1024.0 * 1024 * 1024) / per_x));
  xc = std::min(xc, nxs);

  // GEMM2 (symmetric output, upper tiles) is split along K until the launch
  // has enough CTAs to fill the GPU several times over
  const long tiles2 = ((nmo + 63) / 64) * ((nmo + 63) / 64 + 1) / 2;
  int nsplit = (int)std::max(1L, std::min(16L, (152L * 8 + tiles2 * nmom - 1) / (tiles2 * nmom)));
  const long n2 = (long)nmo * nmo;
  // the tensor-core GEMM2 keeps one partial Sigma per K split (sized for the
  // largest chunk, whose K is the largest)
  int sms = 152;
  MGW_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  // (the mixed kernel's tiles are kMBN wide, and its K per split is bounded)
  const int bn = mixed ? oz::kMBN : oz::BN;
  auto splits_tc = [&](long K2) {
    const int r = gemm2_splits(nmo, nmom, K2, sms, bn);
    return mixed ? std::max(r, oz::mixed_min_split(K2)) : r;
  };
  const int nsplit_tc = tc ? oz::split_count((long)xc * naux, splits_tc((long)xc * naux)) : 1;

  // tensor-core Y stage: grouped W digits (once) and per-chunk L digits
  const int PBt = std::max(1, 128 / nmom);
  const long ngroups_t = (naux + PBt - 1) / PBt;
  Arena ar;
  double *Z = nullptr, *part = nullptr, *wdig = nullptr, *ldig = nullptr, *st = nullptr;
  double *adig = nullptr, *zdig = nullptr;
  ar.add(&Z, (size_t)nmom * naux * xc * nmo);
  ar.add(&part, (size_t)std::max(nsplit, nsplit_tc) * nmom * n2);
  if (tc) {
    ar.add(&wdig, oz::sliced_doubles(ngroups_t * 128, naux));
    ar.add(&ldig, oz::sliced_doubles((long)xc * nmo, naux, lns));
    ar.add(&adig, oz::sliced_doubles(nmo, (long)xc * naux, lns));          // GEMM2 A: rows p, K = (x, P)
    ar.add(&zdig, oz::sliced_doubles((long)nmom * nmo, (long)xc * naux));  // GEMM2 B: rows (n, q)
    ar.add(&st, 3);  // status word; the grid's max |L| and exponent
  }
  MGW_TRY(ar.commit(h));
  oz::Sliced sw, sl;
  CUtensorMap mw;
  int* dstatus = h->defer_status ? h->defer_status : reinterpret_cast<int*>(st);
  if (tc) {
    if (nmom > 128) return fail(h, MGW_ERR_UNSUPPORTED, "mgw_sigma_moments: nmom > 128 on the tensor-core path");
    if (!h->defer_status) MGW_CUDA(h, cudaMemsetAsync(dstatus, 0, sizeof(int), h->stream));
    oz::place_sliced(wdig, ngroups_t * 128, naux, sw);
    MGW_TRY(oz::slice_grouped(h, nmom, PBt, naux, Wmom, sw));
    MGW_TRY(oz::digit_map(h, &mw, sw, oz::BM));
    if (mixed && !Lq)
      MGW_TRY(oz::global_exponent(h, (long)naux * sx, L, reinterpret_cast<unsigned long long*>(st + 1),
                                  reinterpret_cast<int*>(st + 2)));
  }
  const int* gexp = tc ? reinterpret_cast<const int*>(st + 2) : nullptr;

  for (int sector = 0; sector < 2; ++sector) {
    const int xbeg = sector == 0 ? 0 : nhole, xend = sector == 0 ? nhole : nxs;
    const double sgn = sector == 0 ? -1.0 : 1.0;
    double* sig = sector == 0 ? sig_hole : sig_part;
    BinomCoef bc;
    binomial_table(nmom, sgn, bc);
    bool first = true;
    for (int x0 = xbeg; x0 < xend; x0 += xc) {
      const int nx = std::min(xc, xend - x0);
      const long ncol = (long)nx * nmo;
      if (tc) {
        oz::place_sliced(ldig, ncol, naux, sl, lns);
        const oz::Gather gy{ncol + 1, 0, 1, naux + 1L, 0, sx};  // rows (x, q), K = P
        if (Lq)
          MGW_TRY(oz::slice_gather_q(h, ncol, naux, Lq + (long)x0 * nmo, gy, eq, sl));
        else if (mixed)
          MGW_TRY(oz::slice_gather_grid(h, ncol, naux, L + (long)x0 * nmo, gy, gexp, sl));
        else
          MGW_TRY(oz::slice_cols(h, ncol, naux, L + (long)x0 * nmo, sx, sl));
        CUtensorMap ml;
        MGW_TRY(oz::digit_map(h, &ml, sl, bn));
        auto launch_y = [&](auto epi) {
          if (mixed)
            return oz::ozaki_mixed_launch<true>(h, mw, ml, sw.exps, sl.exps, (int)(ngroups_t * 128), (int)ncol,
                                                naux, oz::ARowsPlain{}, epi, dstatus, "sigma_y_binomial_tc");
          return oz::ozaki_launch(h, mw, ml, sw.exps, sl.exps, (int)(ngroups_t * 128), (int)ncol, naux,
                                  oz::ARowsPlain{}, epi, dstatus, "sigma_y_binomial_tc");
        };
        if (nmom <= 12)
          MGW_TRY(launch_y(EpiBinomialTC<12>{Z, eps_G + x0, nmom, PBt, naux, nmo, ncol, sgn}));
        else if (nmom <= 16)
          MGW_TRY(launch_y(EpiBinomialTC<16>{Z, eps_G + x0, nmom, PBt, naux, nmo, ncol, sgn}));
        else
          MGW_TRY(launch_y(EpiBinomialTC<kMaxMom>{Z, eps_G + x0, nmom, PBt, naux, nmo, ncol, sgn}));
      } else {
        EpiBinomialT<BinomCoef> epi{Z, eps_G + x0, nmom, PB, naux, nmo, ncol, bc};
        AGroupedMoments A{Wmom, nmom, PB, naux, BM};
        BRowMajor B{L + (long)x0 * nmo, sx, 0};
        MGW_TRY((dgemm<BM, BN>(h, ngroups * BM, ncol, naux, 1, A, B, epi, "sigma_y_binomial")));
      }
      // Sigma(n) (+)= sum_{P,x} L[P][x][p] Z(n)[(P,x)][q]
      if (tc) {
        // on the tensor cores: A rows p, B rows (n, q), both with K = (x_local, P)
        const long K2 = (long)nx * naux;
        oz::Sliced sa2, sz2;
        oz::place_sliced(adig, nmo, K2, sa2, lns);
        oz::place_sliced(zdig, (long)nmom * nmo, K2, sz2);
        const oz::Gather ga2{nmo + 1L, 0, 1, naux, nmo, sx};
        if (Lq)
          MGW_TRY(oz::slice_gather_q(h, nmo, K2, Lq + (long)x0 * nmo, ga2, eq, sa2));
        else if (mixed)
          MGW_TRY(oz::slice_gather_grid(h, nmo, K2, L + (long)x0 * nmo, ga2, gexp, sa2));
        else
          MGW_TRY(oz::slice_gather(h, nmo, K2, L + (long)x0 * nmo, ga2, sa2));
        MGW_TRY(oz::slice_gather(h, (long)nmom * nmo, K2, Z, oz::Gather{nmo, (long)naux * ncol, 1, naux, nmo, ncol},
                                 sz2));
        CUtensorMap ma2, mz2;
        MGW_TRY(oz::digit_map(h, &ma2, sa2, oz::BM));
        MGW_TRY(oz::digit_map(h, &mz2, sz2, bn));
        // upper-triangle tiles only, split along K into partial sums (one
        // buffer per split, summed into Sigma by k_reduce_splits)
        // at most nsplit_tc splits: the K-bounded split count of this chunk
        // is at most that of the largest chunk, which nsplit_tc covers
        const int ns2 = std::max(std::min(nsplit_tc, gemm2_splits(nmo, nmom, K2, sms, bn)),
                                 mixed ? oz::mixed_min_split(K2) : 1);
        const int nz = oz::split_count(K2, ns2);
        auto launch_g2 = [&](const oz::FSigmaN& f, int nsp) {
          const oz::EpiElem<oz::FSigmaN> epi{f};
          if (mixed)
            return oz::ozaki_mixed_launch<false>(h, ma2, mz2, sa2.exps, sz2.exps, nmo, nmom * nmo, (int)K2,
                                                 oz::ARowsPlain{}, epi, dstatus, "sigma_gemm2_tc", nsp);
          return oz::ozaki_launch(h, ma2, mz2, sa2.exps, sz2.exps, nmo, nmom * nmo, (int)K2, oz::ARowsPlain{}, epi,
                                  dstatus, "sigma_gemm2_tc", nsp);
        };
        if (nz == 1) {
          MGW_TRY(launch_g2(oz::FSigmaN{sig, nmo, first ? 0.0 : 1.0, 0}, 1));
        } else {
          MGW_TRY(launch_g2(oz::FSigmaN{part, nmo, 0.0, (long)nmom * n2}, ns2));
          const long cnt = (long)nmom * n2;
          k_reduce_splits<<<(unsigned)std::min<long>((cnt + 255) / 256, 152L * 16), 256, 0, h->stream>>>(
              cnt, nz, part, sig, first ? 0 : 1);
          MGW_TRY(check_launch(h, "reduce_splits"));
        }
        first = false;
        continue;
      }
      AKMajor2 A2{L + (long)x0 * nmo, nx, sx, nmo, 0};
      BRowMajor B2{Z, nmo, (long)naux * ncol};
      const long K2 = (long)naux * nx;
      const int ns = (int)std::min<long>(nsplit, std::max(1L, K2 / 256));
      if (ns == 1) {
        EpiStore e2{sig, nmo, n2, 1.0, first ? 0.0 : 1.0};
        MGW_TRY((dgemm<64, 64>(h, nmo, nmo, K2, nmom, A2, B2, e2, "sigma_gemm2", /*tri=*/1)));
      } else {
        // partial sums per K split, z = n + nmom * split, then one reduction pass
        EpiStore e2{part, nmo, n2, 1.0, 0.0};
        MGW_TRY((dgemm<64, 64>(h, nmo, nmo, K2, nmom, A2, B2, e2, "sigma_gemm2", /*tri=*/1, ns)));
        const long cnt = (long)nmom * n2;
        const long kchunk = ((K2 + ns - 1) / ns + 15) / 16 * 16;
        const int nsp = (int)((K2 + kchunk - 1) / kchunk);
        k_reduce_splits<<<(unsigned)std::min<long>((cnt + 255) / 256, 152L * 16), 256, 0, h->stream>>>(
            cnt, nsp, part, sig, first ? 0 : 1);
        MGW_TRY(check_launch(h, "reduce_splits"));
      }
      first = false;
    }
    if (first) MGW_CUDA(h, cudaMemsetAsync(sig, 0, sizeof(double) * nmom * nmo * nmo, h->stream));
  }
  if (tc && !h->defer_status) return tc::check_tc_status(h, dstatus, "mgw_sigma_moments");
  return MGW_OK;
}

extern "C" mgw_status mgw_sigma_moments(mgw_handle* h, const mgw_options* o, int nocc, int nvir, int naux,
                                        int nmom, const double* eps_G, const double* L, const double* Wmom,
                                        double* sig_hole, double* sig_part) {
  if (!L) return h ? fail(h, MGW_ERR_ARG, "mgw_sigma_moments: null L") : MGW_ERR_ARG;
  if (nocc < 1 || nvir < 1) return h ? fail(h, MGW_ERR_ARG, "mgw_sigma_moments: bad sizes") : MGW_ERR_ARG;
  return sigma_impl(h, o, nocc + nvir, nocc + nvir, nocc, naux, nmom, eps_G, L, nullptr, 0, Wmom, sig_hole,
                    sig_part);
}

extern "C" mgw_status mgw_sigma_moments_x(mgw_handle* h, const mgw_options* o, int nmo, int nx, int nhole, int naux,
                                          int nmom, const double* eps_x, const double* Lx, const double* Wmom,
                                          double* sig_hole, double* sig_part) {
  if (!Lx) return h ? fail(h, MGW_ERR_ARG, "mgw_sigma_moments_x: null Lx") : MGW_ERR_ARG;
  return sigma_impl(h, o, nmo, nx, nhole, naux, nmom, eps_x, Lx, nullptr, 0, Wmom, sig_hole, sig_part);
}

extern "C" mgw_status mgw_sigma_moments_q(mgw_handle* h, const mgw_options* o, int nocc, int nvir, int naux,
                                          int nmom, const double* eps_G, const short* Lq, int e,
                                          const double* Wmom, double* sig_hole, double* sig_part) {
  if (!Lq) return h ? fail(h, MGW_ERR_ARG, "mgw_sigma_moments_q: null Lq") : MGW_ERR_ARG;
  mgw_options m;
  if (o) m = *o;
  else mgw_options_default(&m);
  m.precision = MGW_MIXED;
  if (nocc < 1 || nvir < 1) return h ? fail(h, MGW_ERR_ARG, "mgw_sigma_moments_q: bad sizes") : MGW_ERR_ARG;
  return sigma_impl(h, &m, nocc + nvir, nocc + nvir, nocc, naux, nmom, eps_G, nullptr, Lq, e, Wmom, sig_hole,
                    sig_part);
}
