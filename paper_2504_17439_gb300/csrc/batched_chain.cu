// Whole-chain batches over many independent systems: the G0W0 chain
// (response moments, Sigma moments, block Lanczos of both sectors, QP solve
// with the Aufbau filling) and the response moments alone.  Systems are
// spread, largest first, over kChainBranches sub-handles, and each branch is
// driven by a host thread of its own: the Lanczos rank decisions and the QP
// solve's host scalars synchronise the host, and separate threads keep one
// system's synchronisation from stalling the others.  Every system runs the
// single-system entry points, so its results are those of a lone call.
#include "mgw_internal.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

namespace mgw {

constexpr int kChainBranches = 4;

struct ChainPool {
  mgw_handle* sub[kChainBranches] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t stream[kChainBranches] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[kChainBranches] = {nullptr, nullptr, nullptr, nullptr};
  ~ChainPool() {
    for (int b = 0; b < kChainBranches; ++b) {
      if (sub[b]) mgw_destroy(sub[b]);
      if (stream[b]) cudaStreamDestroy(stream[b]);
      if (join[b]) cudaEventDestroy(join[b]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};
static void free_pool(void* p) { delete static_cast<ChainPool*>(p); }

static mgw_status pool_of(mgw_handle* h, ChainPool** out) {
  if (!h->chain_pool) {
    h->chain_pool = new ChainPool();
    h->chain_pool_free = free_pool;
  }
  ChainPool& P = *static_cast<ChainPool*>(h->chain_pool);
  for (int b = 0; b < kChainBranches; ++b) {
    if (!P.stream[b]) MGW_CUDA(h, cudaStreamCreateWithFlags(&P.stream[b], cudaStreamNonBlocking));
    if (!P.sub[b]) {
      const mgw_status st = mgw_create(&P.sub[b], h->device, P.stream[b]);
      if (st != MGW_OK) return fail(h, st, "whole-chain batch: sub-handle creation failed");
    }
    if (!P.join[b]) MGW_CUDA(h, cudaEventCreateWithFlags(&P.join[b], cudaEventDisableTiming));
  }
  if (!P.fork) MGW_CUDA(h, cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
  *out = &P;
  return MGW_OK;
}

// systems per branch: largest cost first, each to the least loaded branch
static std::vector<std::vector<int>> assign(const std::vector<double>& cost) {
  std::vector<int> order(cost.size());
  for (size_t s = 0; s < cost.size(); ++s) order[s] = (int)s;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> groups(kChainBranches);
  double load[kChainBranches] = {0, 0, 0, 0};
  for (int s : order) {
    const int b = (int)(std::min_element(load, load + kChainBranches) - load);
    groups[b].push_back(s);
    load[b] += cost[s];
  }
  return groups;
}

// body(sub, s) for every system s of each branch, on that branch's thread;
// the branches start after the work queued on h->stream and h->stream waits
// for all of them
template <class Body>
static mgw_status run_branches(mgw_handle* h, ChainPool& P, const std::vector<std::vector<int>>& groups,
                               Body body) {
  MGW_CUDA(h, cudaEventRecord(P.fork, h->stream));
  for (int b = 0; b < kChainBranches; ++b) MGW_CUDA(h, cudaStreamWaitEvent(P.stream[b], P.fork, 0));
  std::vector<mgw_status> st(kChainBranches, MGW_OK);
  std::vector<std::string> err(kChainBranches);
  std::vector<long> launches0(kChainBranches);
  std::vector<std::thread> threads;
  for (int b = 0; b < kChainBranches; ++b) {
    launches0[b] = P.sub[b]->launches;
    if (groups[b].empty()) continue;
    threads.emplace_back([&, b]() {
      if (cudaSetDevice(h->device) != cudaSuccess) {
        st[b] = MGW_ERR_CUDA;
        err[b] = "cudaSetDevice failed on a branch thread";
        return;
      }
      for (int s : groups[b]) {
        const mgw_status r = body(P.sub[b], s);
        if (r != MGW_OK) {
          st[b] = r;
          err[b] = "system " + std::to_string(s) + ": " + P.sub[b]->err;
          return;
        }
      }
    });
  }
  for (auto& t : threads) t.join();
  for (int b = 0; b < kChainBranches; ++b) {
    h->launches += P.sub[b]->launches - launches0[b];
    MGW_CUDA(h, cudaEventRecord(P.join[b], P.stream[b]));
    MGW_CUDA(h, cudaStreamWaitEvent(h->stream, P.join[b], 0));
  }
  for (int b = 0; b < kChainBranches; ++b)
    if (st[b] != MGW_OK) return fail(h, st[b], "whole-chain batch, %s", err[b].c_str());
  return MGW_OK;
}

__global__ void k_diag_matrix(int n, const double* d, double* m) {  // m = diag(d)
  const long n2 = (long)n * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n2; i += (long)gridDim.x * blockDim.x)
    m[i] = (i / n == i % n) ? d[i / n] : 0.0;
}

// one G0W0 chain on a sub-handle, with buffers in its persistent slots
static mgw_status g0w0_one(mgw_handle* sub, const mgw_options* o, int nmom_max, mgw_g0w0_system& y) {
  const int nocc = y.nocc, nvir = y.nvir, naux = y.naux, nmo = nocc + nvir;
  const int nmom = 2 * nmom_max + 2, nblk = nmom_max + 1;
  const long ov = (long)nocc * nvir, n2 = (long)nmo * nmo, dim = nmo + 2L * nblk * nmo;
  double *Lov, *W, *sh, *sp, *ch, *ah, *bh, *cp, *ap, *bp, *fock, *E, *weight;
  MGW_TRY(slot_buffer(sub, 0, (size_t)naux * ov, &Lov));
  MGW_TRY(slot_buffer(sub, 1, (size_t)nmom * naux * naux, &W));
  MGW_TRY(slot_buffer(sub, 2, (size_t)nmom * n2, &sh));
  MGW_TRY(slot_buffer(sub, 3, (size_t)nmom * n2, &sp));
  MGW_TRY(slot_buffer(sub, 4, n2, &ch));
  MGW_TRY(slot_buffer(sub, 5, (size_t)nblk * n2, &ah));
  MGW_TRY(slot_buffer(sub, 6, (size_t)std::max(1, nblk - 1) * n2, &bh));
  MGW_TRY(slot_buffer(sub, 7, n2, &cp));
  MGW_TRY(slot_buffer(sub, 8, (size_t)nblk * n2, &ap));
  MGW_TRY(slot_buffer(sub, 9, (size_t)std::max(1, nblk - 1) * n2, &bp));
  MGW_TRY(slot_buffer(sub, 10, n2, &fock));
  MGW_TRY(slot_buffer(sub, 11, dim, &E));
  MGW_TRY(slot_buffer(sub, 12, dim, &weight));
  MGW_TRY(mgw_extract_ov(sub, nocc, nvir, naux, y.L, Lov));
  MGW_TRY(mgw_response_moments(sub, o, nocc, nvir, naux, nmom, y.eps, Lov, W));
  MGW_TRY(mgw_sigma_moments(sub, o, nocc, nvir, naux, nmom, y.eps, y.L, W, sh, sp));
  MGW_TRY(mgw_block_lanczos(sub, o, nmo, nmom, sh, ch, ah, nblk > 1 ? bh : nullptr, &y.rank_h));
  MGW_TRY(mgw_block_lanczos(sub, o, nmo, nmom, sp, cp, ap, nblk > 1 ? bp : nullptr, &y.rank_p));
  k_diag_matrix<<<(unsigned)std::min<long>((n2 + 255) / 256, 152L * 8), 256, 0, sub->stream>>>(nmo, y.eps, fock);
  MGW_TRY(check_launch(sub, "diag_matrix"));
  int m = 0;
  return mgw_qp_solve(sub, o, nmo, nblk, y.rank_h, y.rank_p, fock, ch, ah, nblk > 1 ? bh : nullptr, cp, ap,
                      nblk > 1 ? bp : nullptr, 0.0, 2.0 * nocc, E, weight, nullptr, y.eps_qp, nullptr, &y.mu,
                      &y.nelec, &m);
}

}  // namespace mgw

using namespace mgw;

extern "C" mgw_status mgw_g0w0_batched(mgw_handle* h, const mgw_options* o, int nsys, int nmom_max,
                                       mgw_g0w0_system* sys) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (nsys < 1 || !sys || nmom_max < 0 || nmom_max > 11)
    return fail(h, MGW_ERR_ARG, "mgw_g0w0_batched: bad arguments");
  std::vector<double> cost(nsys);
  for (int s = 0; s < nsys; ++s) {
    if (sys[s].nocc < 1 || sys[s].nvir < 1 || sys[s].naux < 1 || !sys[s].eps || !sys[s].L || !sys[s].eps_qp)
      return fail(h, MGW_ERR_ARG, "mgw_g0w0_batched: bad system %d", s);
    const double nmo = sys[s].nocc + sys[s].nvir;
    cost[s] = (double)sys[s].naux * sys[s].naux * nmo * nmo + 9.0 * std::pow(nmo * (1 + 2 * (nmom_max + 1)), 3);
  }
  MGW_CUDA(h, cudaSetDevice(h->device));
  ChainPool* P = nullptr;
  MGW_TRY(pool_of(h, &P));
  return run_branches(h, *P, assign(cost),
                      [&](mgw_handle* sub, int s) { return g0w0_one(sub, o, nmom_max, sys[s]); });
}

extern "C" mgw_status mgw_response_moments_batched(mgw_handle* h, const mgw_options* o, int nsys, int nmom,
                                                   const mgw_response_system* sys) {
  if (!h) return MGW_ERR_ARG;
  mgw_options def;
  mgw_options_default(&def);
  if (!o) o = &def;
  if (nsys < 1 || !sys || nmom < 1 || nmom > 64)
    return fail(h, MGW_ERR_ARG, "mgw_response_moments_batched: bad arguments");
  std::vector<double> cost(nsys);
  for (int s = 0; s < nsys; ++s) {
    if (sys[s].nocc < 1 || sys[s].nvir < 1 || sys[s].naux < 1 || !sys[s].eps_W || !sys[s].Lov || !sys[s].Wmom)
      return fail(h, MGW_ERR_ARG, "mgw_response_moments_batched: bad system %d", s);
    cost[s] = (double)sys[s].naux * sys[s].naux * sys[s].nocc * sys[s].nvir;
  }
  MGW_CUDA(h, cudaSetDevice(h->device));
  ChainPool* P = nullptr;
  MGW_TRY(pool_of(h, &P));
  return run_branches(h, *P, assign(cost), [&](mgw_handle* sub, int s) {
    const mgw_response_system& y = sys[s];
    return mgw_response_moments(sub, o, y.nocc, y.nvir, y.naux, nmom, y.eps_W, y.Lov, y.Wmom);
  });
}

extern "C" mgw_status mgw_sync_status(mgw_handle* h) {
  if (!h) return MGW_ERR_ARG;
  MGW_CUDA(h, cudaSetDevice(h->device));
  MGW_CUDA(h, cudaStreamSynchronize(h->stream));
  MGW_CUDA(h, cudaGetLastError());
  return MGW_OK;
}
