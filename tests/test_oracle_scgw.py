"""Pins of the scGW / GW0 / G0W oracle (Sec. III E, Algorithm 5) against
routes independent of it: the QMO tensors against the MO ones and an
explicit four-index transformation, the self-energy moments over a QMO space
against the Lehmann convolution of explicitly diagonalised poles, and the
whole iteration against a driver that takes every moment from that
convolution."""
import numpy as np
import pytest

import brute
import mgw_inputs
from oracle import mgw_oracle as orc


def system(nocc=3, nvir=5, naux=12, seed=7, scale=3.0):
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    return eps, mgw_inputs.df_tensor(naux, nocc + nvir, seed) * scale


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_qmo_tensors_of_the_reference_orbitals_are_the_mo_tensors():
    eps, L = system()
    Vhat, Via = orc.qmo_tensors(L, np.eye(8), 3)
    assert np.abs(Vhat - L).max() == 0.0
    assert np.abs(Via - orc.particle_hole_block(L, 3)).max() == 0.0


def test_qmo_pair_integrals_equal_the_four_index_transformation():
    eps, L = system()
    g = orc.g0w0(eps, L, 3, 2)
    chi, m = g["chi"], g["m"]
    _, Via = orc.qmo_tensors(L, chi, m)
    eri = np.einsum("Ppq,Prs->pqrs", L, L)
    ref = np.einsum("pi,qa,pqrs,rj,sb->iajb", chi[:, :m], chi[:, m:], eri, chi[:, :m], chi[:, m:], optimize=True)
    nia = m * (chi.shape[1] - m)
    assert rel(Via.T @ Via, ref.reshape(nia, nia)) < 1e-12


def test_self_energy_moments_over_qmos_equal_the_lehmann_convolution():
    eps, L = system()
    g = orc.g0w0(eps, L, 3, 2)
    E, m = g["E"], g["m"]
    Vhat, Via = orc.qmo_tensors(L, g["chi"], m)
    D = orc.energy_differences(E, m)
    nmom = 6
    sh, sp = orc.sigma_moments(E, m, Vhat, orc.response_moments(Via, D, nmom))
    bh, bp = brute.sigma_lehmann_general(E, m, Vhat, Via, D, nmom)
    for n in range(nmom):
        assert rel(sh[n], bh[n]) < 1e-10 and rel(sp[n], bp[n]) < 1e-10


def test_first_iteration_is_g0w0():
    eps, L = system()
    r = orc.scgw(eps, L, 3, 2, max_iter=1)
    assert np.abs(r["eps_qp"] - orc.g0w0(eps, L, 3, 2)["eps_qp"]).max() < 1e-12


@pytest.mark.parametrize("g0,w0", [(False, False), (False, True), (True, False)])
def test_scgw_iterations_match_a_lehmann_driver(g0, w0):
    eps, L = system()
    ref = brute.scgw_lehmann(orc, eps, L, 3, 1, g0, w0, 3)
    for k in range(3):
        got = orc.scgw(eps, L, 3, 1, g0=g0, w0=w0, max_iter=k + 1, conv=0.0)
        assert np.abs(got["eps_qp"] - ref[k]).max() < 1e-9, k
    # the spaces really change: the third iteration differs from G0W0
    assert np.abs(ref[2] - ref[0]).max() > 1e-7
