"""Pins of the fsGW oracle (Algorithm 2): the Fock build against an explicit
four-index contraction, the fixed-point conditions the paper states
(electron number imposed exactly through zeta, density consistent with the
Fock matrix), invariance under a rotation of the reference basis, and
independence of the converged result from the starting Fock matrix."""
import numpy as np

import mgw_inputs
from oracle import mgw_oracle as orc


def system(nocc=3, nvir=9, naux=40, seed=5, scale=2.0):
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    L = mgw_inputs.df_tensor(naux, nocc + nvir, seed) * scale
    return eps, L


def test_fock_build_against_four_index_integrals():
    eps, L = system()
    g = np.random.default_rng(2)
    rho = g.standard_normal((12, 12))
    rho = rho + rho.T
    eri = np.einsum("Ppq,Prs->pqrs", L, L)  # (pq|rs), Eq. 13
    J = np.einsum("pqrs,rs->pq", eri, rho)
    K = np.einsum("prsq,rs->pq", eri, rho)
    h = g.standard_normal((12, 12))
    h = h + h.T
    assert np.allclose(orc.fock_build(h, L, rho), h + J - 0.5 * K, atol=1e-13)


def test_core_hamiltonian_reproduces_reference_fock():
    eps, L = system()
    h = orc.hf_core_hamiltonian(eps, L, 3)
    rho = np.zeros((12, 12))
    rho[:3, :3] = 2.0 * np.eye(3)
    assert np.abs(orc.fock_build(h, L, rho) - np.diag(eps)).max() < 1e-14


def test_fsgw_fixed_point_conditions():
    eps, L = system()
    h = orc.hf_core_hamiltonian(eps, L, 3)
    r = orc.fsgw(h, L, eps, 3, 2)
    assert r["converged"]
    last = r["history"][-1]
    assert abs(last["nelec"] - 6.0) < 1e-8  # Eq. 40 count imposed through zeta
    # F is the Fock matrix of the correlated density it produces
    e, C = np.linalg.eigh(r["F"])
    Lm = orc.rotate_df(L, C)
    W = orc.tda_response_moments(orc.particle_hole_block(Lm, 3), orc.energy_differences(e, 3), 6)
    sh, sp = orc.sigma_moments(e, 3, Lm, W)
    hole, part = orc.block_lanczos(sh, 3), orc.block_lanczos(sp, 3)
    qp = orc.qp_solve(r["F"], (C @ hole[0], hole[1], hole[2]), (C @ part[0], part[1], part[2]), 6.0, r["zeta"])
    assert np.abs(orc.fock_build(h, L, qp["rho"]) - r["F"]).max() < 5e-4


def test_fsgw_invariant_under_rotation_of_the_reference_basis():
    eps, L = system()
    h = orc.hf_core_hamiltonian(eps, L, 3)
    r0 = orc.fsgw(h, L, eps, 3, 2)
    U = mgw_inputs.random_orthogonal(12, 9)
    Lr = orc.rotate_df(L, U)
    hr = U.T @ h @ U
    r1 = orc.fsgw(hr, Lr, eps, 3, 2, F0=U.T @ np.diag(eps) @ U)
    assert r1["converged"] and r0["converged"]
    assert np.abs(r1["eps_qp"] - r0["eps_qp"]).max() < 1e-7


def test_fsgw_independent_of_starting_fock_matrix():
    eps, L = system()
    h = orc.hf_core_hamiltonian(eps, L, 3)
    r0 = orc.fsgw(h, L, eps, 3, 2, conv_e=1e-7, conv_mom=1e-7, max_outer=60)
    g = np.random.default_rng(4)
    P = g.standard_normal((12, 12)) * 0.02
    r1 = orc.fsgw(h, L, eps, 3, 2, conv_e=1e-7, conv_mom=1e-7, max_outer=60, F0=np.diag(eps) + P + P.T)
    assert r0["converged"] and r1["converged"]
    assert np.abs(r1["eps_qp"] - r0["eps_qp"]).max() < 1e-5
