"""fsGW on the GPU (mgw_fsgw_step, Algorithm 2) against the oracle's fsGW.

The loops take their decisions (golden-section steps, DIIS subspace) on
floating-point values that differ by rounding between the two sides, so the
trajectories are compared where they are well defined: the converged QP
energies, Fock matrix, zeta and electron count.
"""
import numpy as np
import pytest
import torch

import mgw_inputs
from oracle import mgw_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    return mgw.Handle(0)


@pytest.mark.parametrize("nocc,nvir,naux,N,seed", [(3, 9, 40, 2, 5), (4, 14, 70, 3, 6)])
def test_fsgw_converges_to_the_oracle_fixed_point(h, nocc, nvir, naux, N, seed):
    from paper_2504_17439_gb300 import driver

    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    L = mgw_inputs.df_tensor(naux, nocc + nvir, seed) * 2.0
    hcore = orc.hf_core_hamiltonian(eps, L, nocc)
    ref = orc.fsgw(hcore, L, eps, nocc, N, conv_e=1e-8, conv_mom=1e-8, max_outer=60)
    got = driver.fsgw(h, torch.from_numpy(hcore).cuda(), torch.from_numpy(L).cuda(), torch.from_numpy(eps).cuda(),
                      nocc, N, conv_e=1e-8, conv_mom=1e-8, max_outer=60)
    assert ref["converged"] and got["converged"]
    assert np.abs(got["eps_qp"].cpu().numpy() - ref["eps_qp"]).max() < 1e-6
    assert np.abs(got["F"].cpu().numpy() - ref["F"]).max() < 1e-6
    assert abs(got["history"][-1]["nelec"] - 2 * nocc) < 1e-8


def test_fsgw_from_a_rotated_start_matches(h):
    from paper_2504_17439_gb300 import driver

    eps = mgw_inputs.orbital_energies(3, 9, 5)
    L = mgw_inputs.df_tensor(40, 12, 5) * 2.0
    hcore = orc.hf_core_hamiltonian(eps, L, 3)
    U = mgw_inputs.random_orthogonal(12, 9)
    Lr = orc.rotate_df(L, U)
    r0 = driver.fsgw(h, torch.from_numpy(hcore).cuda(), torch.from_numpy(L).cuda(), torch.from_numpy(eps).cuda(),
                     3, 2, conv_e=1e-8, conv_mom=1e-8)
    r1 = driver.fsgw(h, torch.from_numpy(U.T @ hcore @ U).cuda(), torch.from_numpy(Lr).cuda(),
                     torch.from_numpy(eps).cuda(), 3, 2, conv_e=1e-8, conv_mom=1e-8,
                     F0=torch.from_numpy(U.T @ np.diag(eps) @ U).cuda())
    assert r0["converged"] and r1["converged"]
    assert np.abs(r1["eps_qp"].cpu().numpy() - r0["eps_qp"].cpu().numpy()).max() < 1e-6


@pytest.mark.parametrize("nocc,nvir,naux,seed", [(3, 9, 30, 41), (7, 30, 130, 42), (1, 1, 1, 43)])
def test_hf_core_matches_oracle(nocc, nvir, naux, seed):
    """mgw_hf_core against the oracle's h = diag(eps) - J[rho_HF] + K[rho_HF]/2."""
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    h = mgw.Handle(0)
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    L = mgw_inputs.df_tensor(naux, nocc + nvir, seed) * 2.0
    ref = orc.hf_core_hamiltonian(eps, L, nocc)
    got = h.mgw_hf_core(nocc, torch.from_numpy(eps).cuda(), torch.from_numpy(L).cuda()).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    h.close()
