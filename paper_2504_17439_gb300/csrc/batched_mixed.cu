// Mixed-precision batch of Sigma-moment builds over many systems of uneven
// size: every tensor-core product of every system's TDA response and Sigma
// build runs in grouped launches of ozaki_mixed_grouped_kernel, one launch
// per stage over all systems --
//   order t:             W_s(t) = T_s V'_s^T, then T_s <- T_s o D_s + 2 W_s(t) V'_s
//   sector, round r:     the Y stage (binomial epilogue) of chunk r of every s,
//                        then GEMM2 of chunk r of every s
// -- a CTA finding its system and tile in a prefix sum of tile counts.  The
// digit slicing between stages (memory-bound, a few small kernels per system)
// is issued per system.  The whole sequence is captured once as a CUDA graph
// and replayed while the systems' sizes and pointers stay the same.
//
// Launch order per product (row or column bands) is chosen per item as in
// ozaki_mixed_launch.  The Green's-function indices of every system are split
// evenly over the fewest rounds whose buffers (all systems' chunks of Z and
// their digits are live in a round) fit in 60% of the free device memory,
// each chunk within GEMM2's K bound; a round's launches hold the systems that
// still have a chunk.
#include "mgw_internal.h"
#include "ozaki_mixed.h"
#include "sigma_epi.h"
#include "tc_gemm.h"

#include <algorithm>
#include <cstring>
#include <vector>

namespace mgw {
namespace {

constexpr int kBinomMax = 16;  // nmom <= 16 (N <= 7); the Y epilogue's sweeps are unrolled to 12 or 16
using EpiW = oz::EpiElem<oz::FStoreSym>;
using EpiT = oz::EpiElem<oz::FDiagUpdate>;
using EpiG = oz::EpiElem<oz::FSigmaN>;

enum StageKind { kGW = 0, kGT = 1, kGY = 2, kGG = 3 };
const char* const kGroupName[4] = {"w_gemm_grouped_mixed", "t_update_grouped_mixed", "sigma_y_grouped_mixed",
                                   "sigma_gemm2_grouped_mixed"};

struct SysWs {  // one system's workspace and digit planes
  long nmo = 0, ov = 0, naux = 0, xc[2] = {0, 0};
  double *D = nullptr, *Lov = nullptr, *T = nullptr, *W = nullptr, *Z = nullptr, *st = nullptr;
  double *dv = nullptr, *dvt = nullptr, *dt = nullptr, *dw = nullptr, *dwg = nullptr;
  double *dl = nullptr, *da = nullptr, *dz = nullptr;
  oz::Sliced sv, svt, stt, sww, swg;
  int* gexp_v() const { return reinterpret_cast<int*>(st + 1); }
  int* gexp_l() const { return reinterpret_cast<int*>(st + 3); }
};

struct Stage {
  int kind;
  size_t off_items, off_start;
  int nitems;
  long ntiles;
};

struct Blob {  // host image of the item tables, 256-byte aligned entries
  std::vector<char> b;
  size_t add(const void* p, size_t n) {
    const size_t off = (b.size() + 255) / 256 * 256;
    b.resize(off + n);
    std::memcpy(b.data() + off, p, n);
    return off;
  }
};

struct MixedPlan {
  std::vector<long long> key;
  void* dmem = nullptr;
  size_t dmem_bytes = 0;
  char* dtab = nullptr;
  size_t dtab_bytes = 0;
  std::vector<SysWs> S;
  std::vector<Stage> stages;
  int rounds = 1;
  long graph_launches = 0;
  int* dstatus = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~MixedPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (dtab) cudaFree(dtab);
    if (dmem) cudaFree(dmem);
  }
};
void free_mixed_plan(void* p) { delete static_cast<MixedPlan*>(p); }

int band_order(long M, long N) {  // as ozaki_mixed_launch: the order that fetches fewer operand rows
  const long MT = (M + oz::BM - 1) / oz::BM, NT = (N + oz::kMBN - 1) / oz::kMBN;
  const double rows_a = (double)MT * oz::BM, rows_b = (double)NT * oz::kMBN;
  const double by_rows = rows_a + (double)((MT + oz::kBand - 1) / oz::kBand) * rows_b;
  const double by_cols = (double)((NT + oz::kBandN - 1) / oz::kBandN) * rows_a + rows_b;
  return by_cols < by_rows ? 1 : 0;
}

// Builds the item tables (tab != nullptr) or issues the sequence
// (tab == nullptr): one walk for both, so the two always agree.  The slicing
// between stages runs only when issuing; the tensor maps are encoded only
// when building.
template <class EpiY>
struct Walker {
  mgw_handle* h;
  MixedPlan* P;
  const mgw_system* sys;
  int nsys, nmom;
  Blob* tab;
  size_t next = 0;  // next stage to issue

  template <class Epi>
  mgw_status stage(int kind, const std::vector<oz::MixedItem<Epi>>& items) {
    if (items.empty()) return MGW_OK;
    if (tab) {
      std::vector<long> start(items.size() + 1, 0);
      for (size_t i = 0; i < items.size(); ++i) {
        const long MT = (items[i].M + oz::BM - 1) / oz::BM, NT = (items[i].N + oz::kMBN - 1) / oz::kMBN;
        start[i + 1] = start[i] + MT * NT;
      }
      Stage L;
      L.kind = kind;
      L.off_items = tab->add(items.data(), sizeof(oz::MixedItem<Epi>) * items.size());
      L.off_start = tab->add(start.data(), sizeof(long) * start.size());
      L.nitems = (int)items.size();
      L.ntiles = start.back();
      P->stages.push_back(L);
      return MGW_OK;
    }
    const Stage& L = P->stages[next++];
    if (L.kind != kind) return fail(h, MGW_ERR_ARG, "grouped mixed batch: stage table out of step");
    return kind == kGG ? launch<false, Epi>(L) : launch<true, Epi>(L);
  }

  template <bool kRB, class Epi>
  mgw_status launch(const Stage& L) {
    using Lay = oz::MixedLayout<kRB>;
    auto kern = oz::ozaki_mixed_grouped_kernel<kRB, Epi>;
    const auto* items = reinterpret_cast<const oz::MixedItem<Epi>*>(P->dtab + L.off_items);
    const auto* start = reinterpret_cast<const long*>(P->dtab + L.off_start);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, h->stream);
    }
    kern<<<(unsigned)L.ntiles, oz::kThreads, Lay::kSmem, h->stream>>>(items, start, L.nitems, P->dstatus);
    const mgw_status st = check_launch(h, kGroupName[L.kind]);
    if (h->prof) {
      cudaEventRecord(e1, h->stream);
      h->spans.push_back({kGroupName[L.kind], e0, e1});
    }
    return st;
  }

  // appends one problem (when issuing, a blank one: only the count matters,
  // so that an empty stage is skipped in both walks alike)
  template <class Epi>
  mgw_status item(std::vector<oz::MixedItem<Epi>>& v, const oz::Sliced& a, const oz::Sliced& b, long M, long N,
                  long K, const Epi& epi) {
    oz::MixedItem<Epi> it;
    std::memset(static_cast<void*>(&it), 0, sizeof it);
    if (!tab) {
      v.push_back(it);
      return MGW_OK;
    }
    MGW_TRY(oz::digit_map(h, &it.mA, a, oz::BM));
    MGW_TRY(oz::digit_map(h, &it.mB, b, oz::kMBN));
    it.ea = a.exps;
    it.eb = b.exps;
    it.M = (int)M;
    it.N = (int)N;
    it.K = (int)K;
    it.col_band = band_order(M, N);
    it.epi = epi;
    v.push_back(it);
    return MGW_OK;
  }

  mgw_status run() {
    const bool issue = tab == nullptr;
    if (issue) MGW_CUDA(h, cudaMemsetAsync(P->dstatus, 0, sizeof(int), h->stream));
    // the response: V' and V'^T on V's grid, T(0) = V'
    if (issue)
      for (int s = 0; s < nsys; ++s) {
        SysWs& q = P->S[s];
        MGW_TRY(mgw_extract_ov(h, sys[s].nocc, sys[s].nvir, sys[s].naux, sys[s].L, q.Lov));
        MGW_TRY(energy_differences(h, sys[s].nocc, sys[s].nvir, sys[s].eps, q.D));
        MGW_TRY(oz::global_exponent(h, q.naux * q.ov, q.Lov, reinterpret_cast<unsigned long long*>(q.st),
                                    q.gexp_v()));
        MGW_TRY(oz::slice_rows_grid(h, q.naux, q.ov, q.Lov, q.ov, q.gexp_v(), q.sv));
        MGW_TRY(oz::slice_gather_grid(h, q.ov, q.naux, q.Lov, oz::Gather{q.ov + 1, 0, 1, q.naux + 1, 0, q.ov},
                                      q.gexp_v(), q.svt));
        MGW_TRY(oz::round_to_grid(h, q.naux * q.ov, q.Lov, q.gexp_v(), q.T));
      }
    for (int n = 0; n < nmom; ++n) {
      if (issue)
        for (int s = 0; s < nsys; ++s) {
          SysWs& q = P->S[s];
          MGW_TRY(oz::slice_rows(h, q.naux, q.ov, q.T, q.ov, q.stt));
        }
      std::vector<oz::MixedItem<EpiW>> wi;
      for (int s = 0; s < nsys; ++s) {
        SysWs& q = P->S[s];
        MGW_TRY(item(wi, q.stt, q.sv, q.naux, q.naux, q.ov,
                     EpiW{oz::FStoreSym{q.W + (long)n * q.naux * q.naux, q.naux, 0}}));
      }
      MGW_TRY(stage(kGW, wi));
      if (n + 1 == nmom) break;
      if (issue)
        for (int s = 0; s < nsys; ++s) {
          SysWs& q = P->S[s];
          MGW_TRY(oz::slice_rows(h, q.naux, q.naux, q.W + (long)n * q.naux * q.naux, q.naux, q.sww));
        }
      std::vector<oz::MixedItem<EpiT>> ti;
      for (int s = 0; s < nsys; ++s) {
        SysWs& q = P->S[s];
        MGW_TRY(item(ti, q.sww, q.svt, q.naux, q.ov, q.naux, EpiT{oz::FDiagUpdate{q.T, q.ov, q.D, 2.0}}));
      }
      MGW_TRY(stage(kGT, ti));
    }
    // the Sigma build: grouped moment rows once, then rounds of x per sector
    const int PBt = std::max(1, 128 / nmom);
    if (issue)
      for (int s = 0; s < nsys; ++s) {
        SysWs& q = P->S[s];
        MGW_TRY(oz::slice_grouped(h, nmom, PBt, (int)q.naux, q.W, q.swg));
        MGW_TRY(oz::global_exponent(h, q.naux * q.nmo * q.nmo, sys[s].L,
                                    reinterpret_cast<unsigned long long*>(q.st + 2), q.gexp_l()));
      }
    for (int sec = 0; sec < 2; ++sec) {
      const double sgn = sec == 0 ? -1.0 : 1.0;
      for (int r = 0; r < P->rounds; ++r) {
        std::vector<oz::Sliced> sl(nsys), sa(nsys), sz(nsys);
        std::vector<char> on(nsys, 0);
        std::vector<oz::MixedItem<EpiY>> yi;
        for (int s = 0; s < nsys; ++s) {
          SysWs& q = P->S[s];
          const long xbeg = sec == 0 ? 0 : sys[s].nocc, xend = sec == 0 ? sys[s].nocc : q.nmo;
          const long x0 = xbeg + r * q.xc[sec];
          if (x0 >= xend) continue;
          on[s] = 1;
          const long nx = std::min(q.xc[sec], xend - x0), ncol = nx * q.nmo, sx = q.nmo * q.nmo;
          oz::place_sliced(q.dl, ncol, q.naux, sl[s], oz::kGridSlices);
          if (issue)
            MGW_TRY(oz::slice_gather_grid(h, ncol, q.naux, sys[s].L + x0 * q.nmo,
                                          oz::Gather{ncol + 1, 0, 1, q.naux + 1, 0, sx}, q.gexp_l(), sl[s]));
          const long ngroups = (q.naux + PBt - 1) / PBt;
          MGW_TRY(item(yi, q.swg, sl[s], ngroups * 128, ncol, q.naux,
                       EpiY{q.Z, sys[s].eps + x0, nmom, PBt, (int)q.naux, (int)q.nmo, ncol, sgn}));
        }
        MGW_TRY(stage(kGY, yi));
        std::vector<oz::MixedItem<EpiG>> gi;
        for (int s = 0; s < nsys; ++s) {
          if (!on[s]) continue;
          SysWs& q = P->S[s];
          const long xbeg = sec == 0 ? 0 : sys[s].nocc, xend = sec == 0 ? sys[s].nocc : q.nmo;
          const long x0 = xbeg + r * q.xc[sec];
          const long nx = std::min(q.xc[sec], xend - x0), ncol = nx * q.nmo, sx = q.nmo * q.nmo;
          const long K2 = nx * q.naux;
          oz::place_sliced(q.da, q.nmo, K2, sa[s], oz::kGridSlices);
          oz::place_sliced(q.dz, (long)nmom * q.nmo, K2, sz[s]);
          if (issue) {
            MGW_TRY(oz::slice_gather_grid(h, q.nmo, K2, sys[s].L + x0 * q.nmo,
                                          oz::Gather{q.nmo + 1, 0, 1, q.naux, q.nmo, sx}, q.gexp_l(), sa[s]));
            MGW_TRY(oz::slice_gather(h, (long)nmom * q.nmo, K2, q.Z,
                                     oz::Gather{q.nmo, q.naux * ncol, 1, q.naux, q.nmo, ncol}, sz[s]));
          }
          double* sig = sec == 0 ? sys[s].sig_hole : sys[s].sig_part;
          MGW_TRY(item(gi, sa[s], sz[s], q.nmo, (long)nmom * q.nmo, K2,
                       EpiG{oz::FSigmaN{sig, (int)q.nmo, r == 0 ? 0.0 : 1.0, 0}}));
        }
        MGW_TRY(stage(kGG, gi));
      }
    }
    return MGW_OK;
  }
};

// bytes of one system's workspace for rounds of xc[] Green's-function indices
size_t system_doubles(const mgw_system& s, int nmom, const long xc[2]) {
  const long nmo = s.nocc + s.nvir, ov = (long)s.nocc * s.nvir, naux = s.naux;
  const long xm = std::max(xc[0], xc[1]);
  const int PBt = std::max(1, 128 / nmom);
  const long ngroups = (naux + PBt - 1) / PBt;
  size_t n = 0;
  n += (size_t)ov + 2 * (size_t)naux * ov + (size_t)nmom * naux * naux + (size_t)nmom * naux * xm * nmo + 8;
  n += oz::sliced_doubles(naux, ov, oz::kGridSlices) + oz::sliced_doubles(ov, naux, oz::kGridSlices);
  n += oz::sliced_doubles(naux, ov) + oz::sliced_doubles(naux, naux) + oz::sliced_doubles(ngroups * 128, naux);
  n += oz::sliced_doubles(xm * nmo, naux, oz::kGridSlices) + oz::sliced_doubles(nmo, xm * naux, oz::kGridSlices);
  n += oz::sliced_doubles((long)nmom * nmo, xm * naux);
  return n + 64 * 16;  // alignment of each buffer
}

// Green's-function indices per round of one system for `rounds` rounds: an
// even split of each sector, capped by GEMM2's K bound (xc naux <=
// kMixedMaxK); a system whose cap forces more rounds takes them
void rounds_xc(const mgw_system& s, int rounds, long xc[2]) {
  const long kcap = std::max(1L, oz::kMixedMaxK / std::max(1, s.naux));
  const long nx[2] = {(long)s.nocc, (long)s.nvir};
  for (int sec = 0; sec < 2; ++sec) xc[sec] = std::max(1L, std::min(kcap, (nx[sec] + rounds - 1) / rounds));
}

}  // namespace

namespace {
template <class EpiY>
mgw_status batched_mixed(mgw_handle* h, const mgw_options* o, int nsys, int nmom, const mgw_system* sys) {
  if (nmom > kBinomMax)
    return fail(h, MGW_ERR_UNSUPPORTED, "mgw_sigma_moments_batched: MGW_MIXED takes nmom <= %d", kBinomMax);
  for (int s = 0; s < nsys; ++s)
    if ((long)sys[s].nocc * sys[s].nvir > oz::kMixedMaxK || sys[s].naux > oz::kMixedMaxK)
      return fail(h, MGW_ERR_UNSUPPORTED, "mgw_sigma_moments_batched: system %d has a contraction above %ld", s,
                  oz::kMixedMaxK);
  if (!h->mixed_plan) {
    h->mixed_plan = new MixedPlan();
    h->mixed_plan_free = free_mixed_plan;
  }
  MixedPlan* P = static_cast<MixedPlan*>(h->mixed_plan);
  std::vector<long long> key = {nsys, nmom};
  for (int s = 0; s < nsys; ++s)
    for (long long v : {(long long)sys[s].nocc, (long long)sys[s].nvir, (long long)sys[s].naux,
                        (long long)(uintptr_t)sys[s].eps, (long long)(uintptr_t)sys[s].L,
                        (long long)(uintptr_t)sys[s].sig_hole, (long long)(uintptr_t)sys[s].sig_part})
      key.push_back(v);

  if (!(P->key == key && P->exec && o->batch_graph)) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
    P->key.clear();
    // rounds: the fewest whose per-round buffers of all systems fit in 60%
    // of the free memory (every system split evenly over them, within GEMM2's
    // K bound)
    size_t free_b = 0, total_b = 0;
    MGW_CUDA(h, cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = (size_t)(0.6 * (double)(free_b + P->dmem_bytes));
    long max_nx = 1;
    for (int s = 0; s < nsys; ++s) max_nx = std::max(max_nx, (long)std::max(sys[s].nocc, sys[s].nvir));
    int split = 1, rounds = 1;
    size_t need = 0;
    for (split = 1; split <= max_nx; ++split) {
      need = 0;
      rounds = 1;
      for (int s = 0; s < nsys; ++s) {
        long xc[2];
        rounds_xc(sys[s], split, xc);
        need += system_doubles(sys[s], nmom, xc) * sizeof(double);
        rounds = std::max(rounds, (int)std::max((sys[s].nocc + xc[0] - 1) / xc[0], (sys[s].nvir + xc[1] - 1) / xc[1]));
      }
      if (need <= budget) break;
    }
    if (need > budget)
      return fail(h, MGW_ERR_NOMEM, "mgw_sigma_moments_batched: %zu bytes of workspace above the budget", need);
    need += 256;
    if (P->dmem_bytes < need) {
      if (P->dmem) cudaFree(P->dmem);
      P->dmem = nullptr;
      P->dmem_bytes = 0;
      MGW_CUDA(h, cudaMalloc(&P->dmem, need));
      P->dmem_bytes = need;
    }
    // carve the workspace
    P->rounds = rounds;
    P->S.assign(nsys, SysWs());
    char* cur = static_cast<char*>(P->dmem);
    auto take = [&](size_t ndoubles) {
      double* p = reinterpret_cast<double*>(cur);
      cur += (ndoubles * sizeof(double) + 511) / 512 * 512;
      return p;
    };
    P->dstatus = reinterpret_cast<int*>(take(1));
    for (int s = 0; s < nsys; ++s) {
      SysWs& q = P->S[s];
      q.nmo = sys[s].nocc + sys[s].nvir;
      q.ov = (long)sys[s].nocc * sys[s].nvir;
      q.naux = sys[s].naux;
      rounds_xc(sys[s], split, q.xc);
      const long xm = std::max(q.xc[0], q.xc[1]);
      const int PBt = std::max(1, 128 / nmom);
      const long ngroups = (q.naux + PBt - 1) / PBt;
      q.D = take(q.ov);
      q.Lov = take(q.naux * q.ov);
      q.T = take(q.naux * q.ov);
      q.W = take((long)nmom * q.naux * q.naux);
      q.Z = take((long)nmom * q.naux * xm * q.nmo);
      q.st = take(4);
      q.dv = take(oz::sliced_doubles(q.naux, q.ov, oz::kGridSlices));
      q.dvt = take(oz::sliced_doubles(q.ov, q.naux, oz::kGridSlices));
      q.dt = take(oz::sliced_doubles(q.naux, q.ov));
      q.dw = take(oz::sliced_doubles(q.naux, q.naux));
      q.dwg = take(oz::sliced_doubles(ngroups * 128, q.naux));
      q.dl = take(oz::sliced_doubles(xm * q.nmo, q.naux, oz::kGridSlices));
      q.da = take(oz::sliced_doubles(q.nmo, xm * q.naux, oz::kGridSlices));
      q.dz = take(oz::sliced_doubles((long)nmom * q.nmo, xm * q.naux));
      oz::place_sliced(q.dv, q.naux, q.ov, q.sv, oz::kGridSlices);
      oz::place_sliced(q.dvt, q.ov, q.naux, q.svt, oz::kGridSlices);
      oz::place_sliced(q.dt, q.naux, q.ov, q.stt);
      oz::place_sliced(q.dw, q.naux, q.naux, q.sww);
      oz::place_sliced(q.dwg, ngroups * 128, q.naux, q.swg);
    }
    if ((size_t)(cur - static_cast<char*>(P->dmem)) > P->dmem_bytes)
      return fail(h, MGW_ERR_ARG, "grouped mixed batch: workspace carve overran its sizing");
    // item tables
    P->stages.clear();
    Blob blob;
    Walker<EpiY> build{h, P, sys, nsys, nmom, &blob};
    MGW_TRY(build.run());
    if (P->dtab_bytes < blob.b.size()) {
      if (P->dtab) cudaFree(P->dtab);
      P->dtab = nullptr;
      P->dtab_bytes = 0;
      MGW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&P->dtab), blob.b.size()));
      P->dtab_bytes = blob.b.size();
    }
    MGW_CUDA(h, cudaMemcpy(P->dtab, blob.b.data(), blob.b.size(), cudaMemcpyHostToDevice));
    // the kernels' shared-memory opt-in, before any capture
    MGW_CUDA(h, cudaFuncSetAttribute(oz::ozaki_mixed_grouped_kernel<true, EpiW>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, oz::MixedLayout<true>::kSmem));
    MGW_CUDA(h, cudaFuncSetAttribute(oz::ozaki_mixed_grouped_kernel<true, EpiT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, oz::MixedLayout<true>::kSmem));
    MGW_CUDA(h, cudaFuncSetAttribute(oz::ozaki_mixed_grouped_kernel<true, EpiY>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, oz::MixedLayout<true>::kSmem));
    MGW_CUDA(h, cudaFuncSetAttribute(oz::ozaki_mixed_grouped_kernel<false, EpiG>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, oz::MixedLayout<false>::kSmem));
    if (o->batch_graph) {
      if (!h->capture_stream) MGW_CUDA(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
      cudaStream_t user = h->stream;
      const bool prof = h->prof;
      h->stream = h->capture_stream;
      h->prof = false;
      const long before = h->launches;
      const cudaError_t ce = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
      Walker<EpiY> go{h, P, sys, nsys, nmom, nullptr};
      const mgw_status st = ce == cudaSuccess ? go.run() : MGW_ERR_CUDA;
      P->graph_launches = h->launches - before;  // kernels in the graph, counted when it runs
      h->launches = before;
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = ce == cudaSuccess ? cudaStreamEndCapture(h->stream, &graph) : ce;
      h->stream = user;
      h->prof = prof;
      if (st != MGW_OK || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != MGW_OK ? st : fail(h, MGW_ERR_CUDA, "grouped mixed batch capture failed: %s",
                                        cudaGetErrorString(ee));
      }
      const cudaError_t ie = cudaGraphInstantiate(&P->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        P->exec = nullptr;
        return fail(h, MGW_ERR_CUDA, "grouped mixed batch graph instantiation failed: %s", cudaGetErrorString(ie));
      }
      P->key = key;
    } else {
      Walker<EpiY> go{h, P, sys, nsys, nmom, nullptr};
      MGW_TRY(go.run());
      return tc::check_tc_status(h, P->dstatus, "mgw_sigma_moments_batched");
    }
  }
  MGW_CUDA(h, cudaGraphLaunch(P->exec, h->stream));
  h->launches += P->graph_launches;
  return tc::check_tc_status(h, P->dstatus, "mgw_sigma_moments_batched");
}

}  // namespace

mgw_status sigma_moments_batched_mixed(mgw_handle* h, const mgw_options* o, int nsys, int nmom,
                                       const mgw_system* sys) {
  return nmom <= 12 ? batched_mixed<EpiBinomialTC<12>>(h, o, nsys, nmom, sys)
                    : batched_mixed<EpiBinomialTC<kBinomMax>>(h, o, nsys, nmom, sys);
}

}  // namespace mgw
