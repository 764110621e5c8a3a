"""Batched Sigma-moment build (grouped launches over systems of uneven size)
against the oracle per system, and against the single-system entry points."""
import numpy as np
import pytest
import torch

import mgw_inputs
from oracle import mgw_oracle as orc

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_batched_sigma_matches_oracle_per_system():
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    h = mgw.Handle(0)
    shapes = mgw_inputs.batch_shapes(7, seed=77, nmo_lo=8, nmo_hi=40, nmom_max=3)
    nmom = 8
    systems, refs = [], []
    for i, sh in enumerate(shapes):
        eps = mgw_inputs.orbital_energies(sh.nocc, sh.nvir, 500 + i)
        L = mgw_inputs.df_tensor(sh.naux, sh.nmo, 500 + i) * 2.0
        W = orc.tda_response_moments(orc.particle_hole_block(L, sh.nocc), orc.energy_differences(eps, sh.nocc), nmom)
        refs.append(orc.sigma_moments(eps, sh.nocc, L, W))
        systems.append(dict(nocc=sh.nocc, nvir=sh.nvir, naux=sh.naux, eps=torch.from_numpy(eps).cuda(),
                            L=torch.from_numpy(L).cuda()))
    outs = h.mgw_sigma_moments_batched(mgw.options(), nmom, systems)
    for (gh, gp), (rh, rp) in zip(outs, refs):
        gh, gp = gh.cpu().numpy(), gp.cpu().numpy()
        for n in range(nmom):
            assert rel(gh[n], rh[n]) < 1e-9, n
            assert rel(gp[n], rp[n]) < 1e-9, n
    h.close()


def test_batched_graph_replay_and_plain_issue_agree():
    """The captured graph replayed on new input values, and the same build
    issued launch by launch without tuning, both match the oracle."""
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    h = mgw.Handle(0)
    shapes = mgw_inputs.batch_shapes(5, seed=78, nmo_lo=10, nmo_hi=36, nmom_max=2)
    nmom = 6
    systems = []
    for i, sh in enumerate(shapes):
        eps = mgw_inputs.orbital_energies(sh.nocc, sh.nvir, 600 + i)
        L = mgw_inputs.df_tensor(sh.naux, sh.nmo, 600 + i) * 2.0
        systems.append(dict(nocc=sh.nocc, nvir=sh.nvir, naux=sh.naux, eps=torch.from_numpy(eps).cuda(),
                            L=torch.from_numpy(L).cuda()))
    o = mgw.options()
    outs = h.mgw_sigma_moments_batched(o, nmom, systems)  # tune + capture
    # new values in the same input tensors: the replay must read them
    for i, (sy, sh) in enumerate(zip(systems, shapes)):
        sy["eps"].copy_(torch.from_numpy(mgw_inputs.orbital_energies(sh.nocc, sh.nvir, 700 + i)))
        sy["L"].copy_(torch.from_numpy(mgw_inputs.df_tensor(sh.naux, sh.nmo, 700 + i) * 2.0))
    launches0 = h.launches
    outs = h.mgw_sigma_moments_batched(o, nmom, systems, out=outs)  # replay
    assert h.launches > launches0
    plain = h.mgw_sigma_moments_batched(mgw.options(batch_graph=0, batch_autotune=0), nmom, systems)
    for i, ((gh, gp), (ph, pp), sh) in enumerate(zip(outs, plain, shapes)):
        eps = mgw_inputs.orbital_energies(sh.nocc, sh.nvir, 700 + i)
        L = mgw_inputs.df_tensor(sh.naux, sh.nmo, 700 + i) * 2.0
        W = orc.tda_response_moments(orc.particle_hole_block(L, sh.nocc), orc.energy_differences(eps, sh.nocc), nmom)
        rh, rp = orc.sigma_moments(eps, sh.nocc, L, W)
        for n in range(nmom):
            for got in (gh, ph):
                assert rel(got[n].cpu().numpy(), rh[n]) < 1e-9, (i, n)
            for got in (gp, pp):
                assert rel(got[n].cpu().numpy(), rp[n]) < 1e-9, (i, n)
    h.close()


def test_batched_tensor_core_path_matches_oracle():
    """The tensor-core batched build (per-system FP64-accurate pipelines over
    concurrent streams) against the oracle, at the FP64 parity tolerance, on
    two calls in a row (the second reuses the sub-handles' workspaces)."""
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    h = mgw.Handle(0)
    shapes = mgw_inputs.batch_shapes(6, seed=79, nmo_lo=10, nmo_hi=48, nmom_max=2)
    nmom = 6
    systems, refs = [], []
    for i, sh in enumerate(shapes):
        eps = mgw_inputs.orbital_energies(sh.nocc, sh.nvir, 800 + i)
        L = mgw_inputs.df_tensor(sh.naux, sh.nmo, 800 + i) * 2.0
        W = orc.tda_response_moments(orc.particle_hole_block(L, sh.nocc), orc.energy_differences(eps, sh.nocc), nmom)
        refs.append(orc.sigma_moments(eps, sh.nocc, L, W))
        systems.append(dict(nocc=sh.nocc, nvir=sh.nvir, naux=sh.naux, eps=torch.from_numpy(eps).cuda(),
                            L=torch.from_numpy(L).cuda()))
    o = mgw.options(precision=mgw.MGW_FP64_TC)
    for call in range(2):
        outs = h.mgw_sigma_moments_batched(o, nmom, systems)
        for (gh, gp), (rh, rp) in zip(outs, refs):
            gh, gp = gh.cpu().numpy(), gp.cpu().numpy()
            for n in range(nmom):
                assert rel(gh[n], rh[n]) < 1e-9, (call, n)
                assert rel(gp[n], rp[n]) < 1e-9, (call, n)
    h.close()


def test_batched_mixed_grouped_launches_match_oracle():
    """The mixed-precision batch (one grouped tensor-core launch per stage over
    all systems, replayed from a CUDA graph on the second call) against the
    oracle on the tensors the mixed path contracts (V and L rounded to their
    own 16-bit grids), at the FP64 parity tolerance, per system."""
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    h = mgw.Handle(0)
    shapes = mgw_inputs.batch_shapes(7, seed=83, nmo_lo=10, nmo_hi=70, nmom_max=2)
    nmom = 6
    systems, refs = [], []
    for i, sh in enumerate(shapes):
        eps = mgw_inputs.orbital_energies(sh.nocc, sh.nvir, 850 + i)
        L = mgw_inputs.df_tensor(sh.naux, sh.nmo, 850 + i) * 2.0
        V = orc.particle_hole_block(L, sh.nocc)
        W = orc.tda_response_moments(orc.fixed_point_grid(V), orc.energy_differences(eps, sh.nocc), nmom)
        refs.append(orc.sigma_moments(eps, sh.nocc, orc.fixed_point_grid(L), W))
        systems.append(dict(nocc=sh.nocc, nvir=sh.nvir, naux=sh.naux, eps=torch.from_numpy(eps).cuda(),
                            L=torch.from_numpy(L).cuda()))
    o = mgw.options(precision=mgw.MGW_MIXED)
    outs = None
    for call in range(2):
        outs = h.mgw_sigma_moments_batched(o, nmom, systems, out=outs)
        for (gh, gp), (rh, rp) in zip(outs, refs):
            gh, gp = gh.cpu().numpy(), gp.cpu().numpy()
            for n in range(nmom):
                assert rel(gh[n], rh[n]) < 1e-9, (call, n)
                assert rel(gp[n], rp[n]) < 1e-9, (call, n)
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_g0w0_and_response_batched_match_single_system_calls(precision):
    """The whole-chain batch (sub-handles on host threads) gives each system
    the single-system chain's QP energies, Aufbau count and ranks; the batched
    response moments equal the single-system ones."""
    from paper_2504_17439_gb300 import build, driver, mgw

    build.build()
    h = mgw.Handle(0)
    o = mgw.options(precision=mgw.MGW_FP64 if precision == "fp64" else mgw.MGW_FP64_TC)
    shapes = mgw_inputs.batch_shapes(7, seed=81, nmo_lo=10, nmo_hi=60, nmom_max=3)
    systems = []
    for i, sh in enumerate(shapes):
        eps = torch.from_numpy(mgw_inputs.orbital_energies(sh.nocc, sh.nvir, 900 + i)).cuda()
        L = torch.from_numpy(mgw_inputs.df_tensor(sh.naux, sh.nmo, 900 + i) * 2.0).cuda()
        systems.append(dict(nocc=sh.nocc, nvir=sh.nvir, naux=sh.naux, eps=eps, L=L,
                            Lov=h.mgw_extract_ov(sh.nocc, sh.nvir, L)))
    res = h.mgw_g0w0_batched(o, 3, systems)
    Ws = h.mgw_response_moments_batched(o, 8, systems)
    h.mgw_sync_status()
    for sy, r, W in zip(systems, res, Ws):
        ref = driver.g0w0(h, sy["eps"], sy["L"], sy["nocc"], 3, opts=mgw.options(precision=o.precision))
        assert r["rank_h"] == ref["hole"][3] and r["rank_p"] == ref["part"][3]
        assert abs(r["nelec"] - ref["nelec"]) < 1e-9
        assert float((r["eps_qp"] - ref["eps_qp"]).abs().max()) < 1e-9
        Wr = h.mgw_response_moments(o, sy["nocc"], sy["nvir"], sy["naux"], 8, sy["eps"], sy["Lov"])
        assert float((W - Wr).abs().max()) <= 1e-12 * float(Wr.abs().max())
    h.close()
