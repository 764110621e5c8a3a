"""Pins of the qsGW oracle (Sec. III D, Eqs. 35-39) against routes independent
of it: the downfolded self-energy of Eq. 10, expansions of both static
potentials in the self-energy moments, the exact all-pole self-energy of a
tiny system, and the fixed-point conditions of Eq. 35."""
import numpy as np
import pytest

import brute
import mgw_inputs
from oracle import mgw_oracle as orc


def system(nocc=3, nvir=5, naux=12, seed=7, scale=2.0):
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    return eps, mgw_inputs.df_tensor(naux, nocc + nvir, seed) * scale


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def chains(eps, L, nocc, nmom_max=2):
    r = orc.g0w0(eps, L, nocc, nmom_max)
    return r, r["hole"][:3], r["part"][:3]


def test_decoupled_poles_reproduce_the_downfolded_self_energy():
    # sum_l v_pl v_ql / (z - e_l) over both chains = W~ (z - d~)^-1 W~^T (Eq. 10)
    eps, L = system()
    _, hole, part = chains(eps, L, 3)
    nmo = eps.size
    H = orc.upfolded_hamiltonian(np.zeros((nmo, nmo)), hole, part)
    Wt, dt = H[:nmo, nmo:], H[nmo:, nmo:]
    (vh, eh), (vp, ep) = orc.decoupled_poles(hole), orc.decoupled_poles(part)
    v, e = np.concatenate([vh, vp], axis=1), np.concatenate([eh, ep])
    for z in (0.3 + 0.05j, -1.7 + 0.2j, 2.5 + 0.01j):
        ref = Wt @ np.linalg.solve(z * np.eye(dt.shape[0]) - dt, Wt.T)
        got = (v / (z - e)) @ v.T
        assert rel(got, ref) < 1e-11


def test_srg_potential_to_first_order_in_s_is_built_from_the_first_two_moments():
    # (D_p + D_q)(1 - exp(-(D_p^2 + D_q^2) s)) / (D_p^2 + D_q^2) -> s (D_p + D_q):
    # V -> s sum_l (eps_p + eps_q - 2 e_l) v_pl v_ql = s (E M0 + M0 E - 2 M1)
    eps, L = system()
    r, hole, part = chains(eps, L, 3)
    M0 = r["sigma_hole"][0] + r["sigma_part"][0]
    M1 = r["sigma_hole"][1] + r["sigma_part"][1]
    E, s = np.diag(eps), 1e-9
    ref = s * (E @ M0 + M0 @ E - 2.0 * M1)
    assert rel(orc.qsgw_potential(eps, hole, part, "srg", srg_s=s), ref) < 1e-6


def test_broadened_potential_at_large_delta_is_built_from_the_first_two_moments():
    # D / (D^2 + delta^2) -> D / delta^2: V -> (E M0 + M0 E) / 2 - M1, over delta^2
    eps, L = system()
    r, hole, part = chains(eps, L, 3)
    M0 = r["sigma_hole"][0] + r["sigma_part"][0]
    M1 = r["sigma_hole"][1] + r["sigma_part"][1]
    E, d = np.diag(eps), 1e5
    ref = (0.5 * (E @ M0 + M0 @ E) - M1) / d**2
    assert rel(orc.qsgw_potential(eps, hole, part, "eta", delta=d), ref) < 1e-6


def test_both_regularisations_share_the_unregularised_diagonal():
    # on the diagonal both tend to Re Sigma_pp(eps_p) = sum_l v_pl^2 / D_pl
    eps, L = system()
    _, hole, part = chains(eps, L, 3)
    Vs = orc.qsgw_potential(eps, hole, part, "srg", srg_s=1e9)
    Ve = orc.qsgw_potential(eps, hole, part, "eta", delta=1e-10)
    assert np.abs(np.diag(Vs) - np.diag(Ve)).max() < 1e-12 * np.abs(np.diag(Ve)).max()
    assert np.abs(orc.qsgw_potential(eps, hole, part, "srg", srg_s=0.0)).max() == 0.0


@pytest.mark.parametrize("reg", ["eta", "srg"])
@pytest.mark.parametrize("nocc,nvir,naux,nmom_max", [(1, 2, 4, 1), (1, 3, 5, 2)])
def test_potential_from_the_moments_equals_the_exact_pole_potential(reg, nocc, nvir, naux, nmom_max):
    # chains long enough to span every pole: the static potential of the
    # moment-conserving self-energy is that of the exact all-pole one, whose
    # external block is already diagonal (one block per sector, no beta)
    eps = mgw_inputs.orbital_energies(nocc, nvir, 3)
    L = mgw_inputs.df_tensor(naux, nocc + nvir, 3) * 3.0
    _, hole, part = chains(eps, L, nocc, nmom_max)
    got = orc.qsgw_potential(eps, hole, part, reg, delta=0.05, srg_s=20.0)
    nmo, nh = eps.size, nocc * nocc * nvir
    H = brute.exact_upfolded(eps, L, nocc)
    v, e = H[:nmo, nmo:], np.diag(H[nmo:, nmo:])

    def one_block(cols):
        return (v[:, cols], np.diag(e[cols])[None], np.zeros((0, cols.size, cols.size)))

    ref = orc.qsgw_potential(eps, one_block(np.arange(nh)), one_block(np.arange(nh, e.size)), reg, 0.05, 20.0)
    assert rel(got, ref) < 1e-12


def test_scf_without_a_potential_stays_at_the_hartree_fock_state():
    eps, L = system()
    h = orc.hf_core_hamiltonian(eps, L, 3)
    e, C, F, _ = orc.qsgw_scf(h, L, np.zeros((8, 8)), np.eye(8), 3)
    assert np.abs(e - eps).max() < 1e-10


@pytest.mark.parametrize("reg", ["eta", "srg"])
def test_qsgw_fixed_point(reg):
    # at convergence F = f[rho(C)] + C V(eps, C) C^T has eigenpairs (eps, C),
    # with V rebuilt from those very energies and orbitals
    eps, L = system(scale=3.0)
    h = orc.hf_core_hamiltonian(eps, L, 3)
    r = orc.qsgw(h, L, eps, 3, 2, reg=reg, delta=1e-3, srg_s=100.0, conv=1e-10)
    assert r["converged"]
    e, C = r["eps"], r["C"]
    assert np.abs(e - eps).max() > 1e-4  # the potential moved the energies
    Lm = orc.rotate_df(L, C)
    W = orc.response_moments(orc.particle_hole_block(Lm, 3), orc.energy_differences(e, 3), 6)
    sh, sp = orc.sigma_moments(e, 3, Lm, W)
    V = orc.qsgw_potential(e, orc.block_lanczos(sh, 3), orc.block_lanczos(sp, 3), reg, 1e-3, 100.0)
    rho = 2.0 * C[:, :3] @ C[:, :3].T
    F = orc.fock_build(h, L, rho) + C @ V @ C.T
    assert np.abs(F @ C - C * e[None, :]).max() < 1e-8


def test_qsgw_invariant_under_rotation_of_the_reference_basis():
    eps, L = system(scale=3.0)
    h = orc.hf_core_hamiltonian(eps, L, 3)
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((8, 8)))
    a = orc.qsgw(h, L, eps, 3, 2, conv=1e-10)
    b = orc.qsgw(Q.T @ h @ Q, np.einsum("ap,Qab,bq->Qpq", Q, L, Q), eps, 3, 2, conv=1e-10, C0=Q.T)
    assert a["converged"] and b["converged"]
    assert np.abs(a["eps"] - b["eps"]).max() < 1e-9
