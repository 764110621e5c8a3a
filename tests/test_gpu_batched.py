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
