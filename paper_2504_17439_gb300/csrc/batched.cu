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
//
// A plan per handle keeps, for the last problem table: the tile shape chosen
// for each stage kind (timed on the first call), every launch's item table
// and tile prefix sums in one device buffer, and the whole sequence captured
// as a CUDA graph, replayed while the table and workspace are unchanged.
#include "mgw_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace mgw {

// the Y stage's binomial epilogue (mgw_internal.h) with its coefficient
// table read through a device pointer (one table per sector for all systems)
using EpiBinomialB = EpiBinomialT<BinomCoefRef>;


// Candidate tile shapes of the grouped FP64 GEMM; static shared memory of
// (BM + BN + 2) * 32 doubles stays within 48 KB.  Triangular stages (W(t),
// GEMM2) enumerate square tiles and keep 64 x 64.
constexpr int kCfgs = 3;
static void cfg_shape(int c, int& bm, int& bn) {
  bm = c == 1 ? 96 : 64;
  bn = c == 2 ? 96 : 64;
}

enum StageKind { kStW = 0, kStT = 1, kStY = 2, kStG2 = 3, kStKinds = 4 };
static const char* kStageName[kStKinds] = {"w_gemm_grouped", "t_update_grouped", "sigma_y_binomial_grouped",
                                           "sigma_gemm2_grouped"};

// one grouped launch: where its items and tile prefix sums sit in the tables
struct Launch {
  int kind;
  size_t off_items, off_start;
  int nitems;
  long ntiles;
};

struct Blob {  // host image of the tables buffer, 256-byte aligned entries
  std::vector<char> b;
  size_t add(const void* p, size_t n) {
    const size_t off = (b.size() + 255) / 256 * 256;
    b.resize(off + n);
    std::memcpy(b.data() + off, p, n);
    return off;
  }
};

struct Sys {
  long nmo, ov, naux, xc_h, xc_p;
  double *D, *Lov, *T, *W, *Z;
};

template <class Item>
static void add_launch(Blob& blob, std::vector<Launch>& out, int kind, const std::vector<Item>& items, int bm, int bn) {
  if (items.empty()) return;
  std::vector<long> start(items.size() + 1, 0);
  for (size_t i = 0; i < items.size(); ++i) {
    const long tn = (items[i].N + bn - 1) / bn, tm = (items[i].M + bm - 1) / bm;
    start[i + 1] = start[i] + (items[i].tri ? tn * (tn + 1) / 2 : tn * tm);
  }
  Launch L;
  L.kind = kind;
  L.off_items = blob.add(items.data(), sizeof(Item) * items.size());
  L.off_start = blob.add(start.data(), sizeof(long) * start.size());
  L.nitems = (int)items.size();
  L.ntiles = start.back();
  out.push_back(L);
}

// the item tables of every launch, in issue order, for tile shapes cfg[kind]
static std::vector<Launch> build_launches(const std::vector<Sys>& S, const mgw_system* sys, int nsys, int nmom,
                                          const int cfg[kStKinds], const BinomCoef* dcoef, int rounds, Blob& blob) {
  std::vector<Launch> out;
  int bmT, bnT, bmY, bnY;
  cfg_shape(cfg[kStT], bmT, bnT);
  cfg_shape(cfg[kStY], bmY, bnY);
  const int PB = std::max(1, bmY / nmom);
  for (int t = 0; t < nmom; ++t) {
    std::vector<GroupItem<ARowMajor, BNMajor, EpiStore>> wi;
    for (int s = 0; s < nsys; ++s) {
      const Sys& q = S[s];
      wi.push_back({q.naux, q.naux, q.ov, ARowMajor{q.T, q.ov, 0}, BNMajor{q.Lov, q.ov, 0},
                    EpiStore{q.W + (long)t * q.naux * q.naux, q.naux, 0, 1.0, 0.0}, 1});
    }
    add_launch(blob, out, kStW, wi, 64, 64);
    if (t + 1 == nmom) break;
    std::vector<GroupItem<ARowMajor, BRowMajor, EpiDiagUpdate>> ti;
    for (int s = 0; s < nsys; ++s) {
      const Sys& q = S[s];
      ti.push_back({q.naux, q.ov, q.naux, ARowMajor{q.W + (long)t * q.naux * q.naux, q.naux, 0},
                    BRowMajor{q.Lov, q.ov, 0}, EpiDiagUpdate{q.T, q.ov, q.D, 2.0}, 0});
    }
    add_launch(blob, out, kStT, ti, bmT, bnT);
  }
  for (int sec = 0; sec < 2; ++sec) {
    for (int r = 0; r < rounds; ++r) {
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
        yi.push_back({ngroups * bmY, ncol, q.naux, AGroupedMoments{q.W, nmom, PB, (int)q.naux, bmY},
                      BRowMajor{sys[s].L + x0 * q.nmo, q.nmo * q.nmo, 0},
                      EpiBinomialB{q.Z, sys[s].eps + x0, nmom, PB, (int)q.naux, (int)q.nmo, ncol, BinomCoefRef{dcoef + sec}}, 0});
        double* sig = sec == 0 ? sys[s].sig_hole : sys[s].sig_part;
        for (int n = 0; n < nmom; ++n)
          gi.push_back({q.nmo, q.nmo, q.naux * nx, AKMajor2{sys[s].L + x0 * q.nmo, nx, q.nmo * q.nmo, q.nmo, 0},
                        BRowMajor{q.Z + (long)n * q.naux * ncol, q.nmo, 0},
                        EpiStore{sig + (long)n * q.nmo * q.nmo, q.nmo, 0, 1.0, r == 0 ? 0.0 : 1.0}, 1});
      }
      add_launch(blob, out, kStY, yi, bmY, bnY);
      add_launch(blob, out, kStG2, gi, 64, 64);
    }
  }
  return out;
}

template <int BM, int BN, class AOp, class BOp, class Epi>
static mgw_status launch_dev(mgw_handle* h, const char* dbase, const Launch& L) {
  const auto* items = reinterpret_cast<const GroupItem<AOp, BOp, Epi>*>(dbase + L.off_items);
  const auto* start = reinterpret_cast<const long*>(dbase + L.off_start);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
  }
  dgemm_grouped_kernel<BM, BN, AOp, BOp, Epi><<<(unsigned)L.ntiles, 256, 0, h->stream>>>(items, start, L.nitems);
  mgw_status st = check_launch(h, kStageName[L.kind]);
  if (h->prof) {
    cudaEventRecord(e1, h->stream);
    h->spans.push_back({kStageName[L.kind], e0, e1});
  }
  return st;
}

template <class AOp, class BOp, class Epi>
static mgw_status launch_cfg(mgw_handle* h, int cfg, const char* dbase, const Launch& L) {
  if (L.ntiles <= 0) return MGW_OK;
  switch (cfg) {
    case 1: return launch_dev<96, 64, AOp, BOp, Epi>(h, dbase, L);
    case 2: return launch_dev<64, 96, AOp, BOp, Epi>(h, dbase, L);
    default: return launch_dev<64, 64, AOp, BOp, Epi>(h, dbase, L);
  }
}

static mgw_status issue_launch(mgw_handle* h, const int cfg[kStKinds], const char* dbase, const Launch& L) {
  switch (L.kind) {
    case kStW: return launch_cfg<ARowMajor, BNMajor, EpiStore>(h, 0, dbase, L);
    case kStT: return launch_cfg<ARowMajor, BRowMajor, EpiDiagUpdate>(h, cfg[kStT], dbase, L);
    case kStY: return launch_cfg<AGroupedMoments, BRowMajor, EpiBinomialB>(h, cfg[kStY], dbase, L);
    default: return launch_cfg<AKMajor2, BRowMajor, EpiStore>(h, 0, dbase, L);
  }
}

// the whole build: per-system preparation, then every grouped launch
static mgw_status issue_all(mgw_handle* h, const std::vector<Sys>& S, const mgw_system* sys, int nsys,
                            const int cfg[kStKinds], const char* dbase, const std::vector<Launch>& launches) {
  for (int s = 0; s < nsys; ++s) {
    MGW_TRY(mgw_extract_ov(h, sys[s].nocc, sys[s].nvir, sys[s].naux, sys[s].L, S[s].Lov));
    MGW_TRY(energy_differences(h, sys[s].nocc, sys[s].nvir, sys[s].eps, S[s].D));
    MGW_CUDA(h, cudaMemcpyAsync(S[s].T, S[s].Lov, sizeof(double) * S[s].naux * S[s].ov, cudaMemcpyDeviceToDevice,
                                h->stream));
  }
  for (const Launch& L : launches) MGW_TRY(issue_launch(h, cfg, dbase, L));
  return MGW_OK;
}

// Tensor-core batched build: the single-system FP64-accurate pipeline per
// system, systems spread over kBranches sub-handles (stream, workspace and
// deferred status word each) so that small systems run concurrently.
constexpr int kBranches = 4;
struct TcBranches {
  mgw_handle* sub[kBranches] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t stream[kBranches] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[kBranches] = {nullptr, nullptr, nullptr, nullptr};
  int* dstat = nullptr;  // [kBranches]
  double* lov[kBranches] = {nullptr, nullptr, nullptr, nullptr};
  double* w[kBranches] = {nullptr, nullptr, nullptr, nullptr};
  size_t lov_n[kBranches] = {0, 0, 0, 0}, w_n[kBranches] = {0, 0, 0, 0};
  ~TcBranches() {
    for (int b = 0; b < kBranches; ++b) {
      if (sub[b]) mgw_destroy(sub[b]);
      if (stream[b]) cudaStreamDestroy(stream[b]);
      if (join[b]) cudaEventDestroy(join[b]);
      if (lov[b]) cudaFree(lov[b]);
      if (w[b]) cudaFree(w[b]);
    }
    if (fork) cudaEventDestroy(fork);
    if (dstat) cudaFree(dstat);
  }
};

struct BatchedPlan {
  TcBranches* tcb = nullptr;
  std::vector<long long> shape_key;  // sizes only: the tuned tile shapes stay valid for it
  std::vector<long long> key;        // sizes, pointers, workspace: the graph and tables stay valid
  int cfg[kStKinds] = {0, 0, 0, 0};
  bool tuned = false;
  char* dtables = nullptr;
  size_t dtables_bytes = 0;
  std::vector<Launch> launches;
  cudaGraphExec_t exec = nullptr;
  ~BatchedPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (dtables) cudaFree(dtables);
    delete tcb;
  }
};
static void free_plan(void* p) { delete static_cast<BatchedPlan*>(p); }

static mgw_status upload(mgw_handle* h, const Blob& blob, char** d, size_t* bytes) {
  if (*bytes < blob.b.size()) {
    if (*d) cudaFree(*d);
    *d = nullptr;
    *bytes = 0;
    MGW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(d), blob.b.size()));
    *bytes = blob.b.size();
  }
  if (!blob.b.empty()) MGW_CUDA(h, cudaMemcpy(*d, blob.b.data(), blob.b.size(), cudaMemcpyHostToDevice));
  return MGW_OK;
}

static mgw_status grow(mgw_handle* h, double** p, size_t* have, size_t n) {
  if (*have >= n) return MGW_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  MGW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(double)));
  *have = n;
  return MGW_OK;
}

static mgw_status batched_tc(mgw_handle* h, BatchedPlan* plan, const mgw_options* o, int nsys, int nmom,
                             const mgw_system* sys) {
  if (!plan->tcb) plan->tcb = new TcBranches();
  TcBranches& B = *plan->tcb;
  for (int b = 0; b < kBranches; ++b) {
    if (!B.stream[b]) MGW_CUDA(h, cudaStreamCreateWithFlags(&B.stream[b], cudaStreamNonBlocking));
    if (!B.sub[b]) {
      const mgw_status st = mgw_create(&B.sub[b], h->device, B.stream[b]);
      if (st != MGW_OK) return fail(h, st, "batched tensor-core build: sub-handle creation failed");
    }
    if (!B.join[b]) MGW_CUDA(h, cudaEventCreateWithFlags(&B.join[b], cudaEventDisableTiming));
  }
  if (!B.fork) MGW_CUDA(h, cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming));
  if (!B.dstat) MGW_CUDA(h, cudaMalloc(reinterpret_cast<void**>(&B.dstat), sizeof(int) * kBranches));

  // largest systems first, each to the least loaded branch (cost ~ Y stage);
  // a branch's first system is then its largest, so its workspace grows once
  std::vector<int> order(nsys);
  std::vector<double> cost(nsys);
  for (int s = 0; s < nsys; ++s) {
    const double nmo = sys[s].nocc + sys[s].nvir;
    cost[s] = (double)sys[s].naux * sys[s].naux * nmo * nmo;
    order[s] = s;
  }
  std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int> branch(nsys);
  double load[kBranches] = {0, 0, 0, 0};
  for (int s : order) {
    const int b = (int)(std::min_element(load, load + kBranches) - load);
    branch[s] = b;
    load[b] += cost[s];
  }
  for (int s = 0; s < nsys; ++s) {
    const int b = branch[s];
    const long ov = (long)sys[s].nocc * sys[s].nvir;
    MGW_TRY(grow(h, &B.lov[b], &B.lov_n[b], (size_t)sys[s].naux * ov));
    MGW_TRY(grow(h, &B.w[b], &B.w_n[b], (size_t)nmom * sys[s].naux * sys[s].naux));
  }

  long sub_launches0 = 0;
  for (int b = 0; b < kBranches; ++b) sub_launches0 += B.sub[b]->launches;
  MGW_CUDA(h, cudaEventRecord(B.fork, h->stream));
  for (int b = 0; b < kBranches; ++b) {
    MGW_CUDA(h, cudaStreamWaitEvent(B.stream[b], B.fork, 0));
    MGW_CUDA(h, cudaMemsetAsync(B.dstat + b, 0, sizeof(int), B.stream[b]));
    B.sub[b]->defer_status = B.dstat + b;
  }
  mgw_status st = MGW_OK;
  for (int s : order) {
    const int b = branch[s];
    mgw_handle* sub = B.sub[b];
    st = mgw_extract_ov(sub, sys[s].nocc, sys[s].nvir, sys[s].naux, sys[s].L, B.lov[b]);
    if (st == MGW_OK)
      st = mgw_response_moments(sub, o, sys[s].nocc, sys[s].nvir, sys[s].naux, nmom, sys[s].eps, B.lov[b], B.w[b]);
    if (st == MGW_OK)
      st = mgw_sigma_moments(sub, o, sys[s].nocc, sys[s].nvir, sys[s].naux, nmom, sys[s].eps, sys[s].L, B.w[b],
                             sys[s].sig_hole, sys[s].sig_part);
    if (st != MGW_OK) {
      h->err = std::string("batched tensor-core build, system ") + std::to_string(s) + ": " + sub->err;
      break;
    }
  }
  for (int b = 0; b < kBranches; ++b) {
    B.sub[b]->defer_status = nullptr;
    h->launches += B.sub[b]->launches;
    MGW_CUDA(h, cudaEventRecord(B.join[b], B.stream[b]));
    MGW_CUDA(h, cudaStreamWaitEvent(h->stream, B.join[b], 0));
  }
  h->launches -= sub_launches0;
  if (st != MGW_OK) return st;
  // wait timeouts of any branch, read once after the join
  int hst[kBranches];
  MGW_CUDA(h, cudaMemcpyAsync(hst, B.dstat, sizeof hst, cudaMemcpyDeviceToHost, h->stream));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int b = 0; b < kBranches; ++b)
    if (hst[b] != 0)
      return fail(h, MGW_ERR_TIMEOUT, "batched tensor-core build: pipeline wait timed out (code %d)", hst[b]);
  return MGW_OK;
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
  if (o->precision != MGW_FP64 && o->precision != MGW_FP64_TC && o->precision != MGW_MIXED)
    return fail(h, MGW_ERR_UNSUPPORTED, "mgw_sigma_moments_batched: precision %d not built", o->precision);
  MGW_CUDA(h, cudaSetDevice(h->device));
  if (!h->batched_plan) {
    h->batched_plan = new BatchedPlan();
    h->batched_plan_free = free_plan;
  }
  if (o->precision == MGW_MIXED) return sigma_moments_batched_mixed(h, o, nsys, nmom, sys);
  if (o->precision == MGW_FP64_TC)
    return batched_tc(h, static_cast<BatchedPlan*>(h->batched_plan), o, nsys, nmom, sys);
  const int rounds = 4;  // Green's-function chunks per sector and system

  // workspace per system: D, Lov, T, W, Z (chunked), all in one arena
  std::vector<Sys> S(nsys);
  Arena ar;
  for (int s = 0; s < nsys; ++s) {
    Sys& q = S[s];
    q.nmo = sys[s].nocc + sys[s].nvir;
    q.ov = (long)sys[s].nocc * sys[s].nvir;
    q.naux = sys[s].naux;
    q.xc_h = std::max(1L, ((long)sys[s].nocc + rounds - 1) / rounds);
    q.xc_p = std::max(1L, ((long)sys[s].nvir + rounds - 1) / rounds);
    const long xc = std::max(q.xc_h, q.xc_p);
    ar.add(&q.D, q.ov);
    ar.add(&q.Lov, q.naux * q.ov);
    ar.add(&q.T, q.naux * q.ov);
    ar.add(&q.W, (long)nmom * q.naux * q.naux);
    ar.add(&q.Z, (long)nmom * q.naux * xc * q.nmo);
  }
  double* coef = nullptr;
  ar.add(&coef, 2 * sizeof(BinomCoef) / sizeof(double));
  MGW_TRY(ar.commit(h));
  const BinomCoef* dcoef = reinterpret_cast<const BinomCoef*>(coef);

  // binomial tables 2 C(n,t) s^t for s = -1 (hole) and +1 (particle)
  BinomCoef hc[2];
  binomial_table(nmom, -1.0, hc[0]);
  binomial_table(nmom, 1.0, hc[1]);
  MGW_CUDA(h, cudaMemcpyAsync(coef, hc, sizeof hc, cudaMemcpyHostToDevice, h->stream));

  // plan keys: the problem's sizes, and its sizes with every pointer
  std::vector<long long> shape_key = {nsys, nmom};
  for (int s = 0; s < nsys; ++s) {
    shape_key.push_back(sys[s].nocc);
    shape_key.push_back(sys[s].nvir);
    shape_key.push_back(sys[s].naux);
  }
  std::vector<long long> key = shape_key;
  key.push_back((long long)(uintptr_t)S[0].D);
  for (int s = 0; s < nsys; ++s)
    for (const void* p : {(const void*)sys[s].eps, (const void*)sys[s].L, (const void*)sys[s].sig_hole,
                          (const void*)sys[s].sig_part})
      key.push_back((long long)(uintptr_t)p);

  BatchedPlan* plan = static_cast<BatchedPlan*>(h->batched_plan);
  if (plan->key == key && plan->exec && o->batch_graph) {  // replay
    MGW_CUDA(h, cudaGraphLaunch(plan->exec, h->stream));
    h->launches += 3L * nsys + (long)plan->launches.size();
    return MGW_OK;
  }
  if (plan->shape_key != shape_key) plan->tuned = false;

  // tile shapes: time the candidates of the non-triangular stages on this
  // table.  The stages run here on whatever the workspace holds (their inputs
  // are not recomputed first): FP64 FMA issue and memory traffic do not depend
  // on the values, NaN and subnormal operands included, so the timing of a
  // candidate is that of a real build of the same shapes.
  if (o->batch_autotune && !plan->tuned) {
    int best[kStKinds] = {0, 0, 0, 0};
    for (int kind : {kStT, kStY}) {
      float best_ms = 0.f;
      for (int c = 0; c < kCfgs; ++c) {
        int cfg[kStKinds] = {best[0], best[1], best[2], best[3]};
        cfg[kind] = c;
        Blob blob;
        std::vector<Launch> ls = build_launches(S, sys, nsys, nmom, cfg, dcoef, rounds, blob);
        MGW_TRY(upload(h, blob, &plan->dtables, &plan->dtables_bytes));
        cudaEvent_t a, b;
        MGW_CUDA(h, cudaEventCreate(&a));
        MGW_CUDA(h, cudaEventCreate(&b));
        MGW_CUDA(h, cudaEventRecord(a, h->stream));
        for (const Launch& L : ls)
          if (L.kind == kind) MGW_TRY(issue_launch(h, cfg, plan->dtables, L));
        MGW_CUDA(h, cudaEventRecord(b, h->stream));
        MGW_CUDA(h, cudaEventSynchronize(b));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (c == 0 || ms < best_ms) {
          best_ms = ms;
          best[kind] = c;
        }
      }
    }
    std::memcpy(plan->cfg, best, sizeof best);
    plan->tuned = true;
    plan->shape_key = shape_key;
  } else if (!o->batch_autotune && !plan->tuned) {
    const int fixed[kStKinds] = {0, 0, 1, 0};  // 96 x 64 Y-stage tiles
    std::memcpy(plan->cfg, fixed, sizeof fixed);
  }

  // the tables of the chosen shapes, once, in a buffer the plan owns
  if (plan->exec) {
    cudaGraphExecDestroy(plan->exec);
    plan->exec = nullptr;
  }
  Blob blob;
  plan->launches = build_launches(S, sys, nsys, nmom, plan->cfg, dcoef, rounds, blob);
  MGW_TRY(upload(h, blob, &plan->dtables, &plan->dtables_bytes));
  plan->key = key;

  if (!o->batch_graph) return issue_all(h, S, sys, nsys, plan->cfg, plan->dtables, plan->launches);

  // capture the whole build on the handle's own stream, then launch the graph
  if (!h->capture_stream) MGW_CUDA(h, cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
  cudaStream_t user = h->stream;
  const bool prof = h->prof;
  h->stream = h->capture_stream;
  h->prof = false;
  cudaError_t ce = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  mgw_status st = ce == cudaSuccess ? issue_all(h, S, sys, nsys, plan->cfg, plan->dtables, plan->launches)
                                    : MGW_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = ce == cudaSuccess ? cudaStreamEndCapture(h->stream, &graph) : ce;
  h->stream = user;
  h->prof = prof;
  if (st != MGW_OK || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    plan->key.clear();
    return st != MGW_OK ? st : fail(h, MGW_ERR_CUDA, "batched build capture failed: %s", cudaGetErrorString(ee));
  }
  const cudaError_t ie = cudaGraphInstantiate(&plan->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    plan->exec = nullptr;
    plan->key.clear();
    return fail(h, MGW_ERR_CUDA, "batched build graph instantiation failed: %s", cudaGetErrorString(ie));
  }
  MGW_CUDA(h, cudaGraphLaunch(plan->exec, h->stream));
  return MGW_OK;
}
