"""Edge cases of the oracle's next-row functions (NAF, spectral function,
qsGW potential, scGW): empty and full truncations, a single virtual orbital,
a single pole, a sector without poles, the one-pair system."""
import math

import numpy as np

import mgw_inputs
from oracle import mgw_oracle as orc


def test_naf_keeps_nothing_above_the_spectrum_and_everything_below_it():
    L = mgw_inputs.df_tensor(9, 6, 2)
    _, lam = orc.naf_basis(L, 2, -1.0, "full")
    assert orc.naf_compress(L, 2, lam[0] * 2.0, "full").shape == (0, 6, 6)
    assert orc.naf_compress(L, 2, -1.0, "full").shape == (9, 6, 6)


def test_naf_pair_mask_with_a_single_virtual_orbital_drops_one_pair():
    mask = orc.naf_pairs(5, 4, "no_vv")
    assert mask.sum() == 24 and not mask[4, 4]


def test_spectral_function_of_one_pole_is_its_lorentzian():
    w = np.linspace(-1.0, 1.0, 11)
    A = orc.spectral_function(np.array([0.2]), np.array([0.7]), w, 0.05)
    assert np.allclose(A, 0.7 * 0.05 / math.pi / ((w - 0.2) ** 2 + 0.0025), rtol=1e-14, atol=0.0)
    assert np.all(orc.spectral_function(np.array([0.2, 0.4]), np.zeros(2), w, 0.05) == 0.0)


def test_qsgw_potential_of_a_chain_without_poles_is_the_other_chains():
    eps = mgw_inputs.orbital_energies(3, 5, 7)
    L = mgw_inputs.df_tensor(12, 8, 7) * 2.0
    r = orc.g0w0(eps, L, 3, 2)
    empty = (np.zeros((8, 0)), np.zeros((3, 0, 0)), np.zeros((2, 0, 0)))
    for reg in ("eta", "srg"):
        only_p = orc.qsgw_potential(eps, empty, r["part"], reg)
        only_h = orc.qsgw_potential(eps, r["hole"], empty, reg)
        both = orc.qsgw_potential(eps, r["hole"], r["part"], reg)
        assert np.abs(only_p + only_h - both).max() < 1e-14 * np.abs(both).max()
        assert np.abs(orc.qsgw_potential(eps, empty, empty, reg)).max() == 0.0


def test_scgw_runs_on_the_one_pair_system():
    eps = np.array([-0.6, 0.4])
    L = np.zeros((1, 2, 2))
    L[0, 0, 1] = L[0, 1, 0] = 0.3
    first = orc.scgw(eps, L, 1, 1, max_iter=1)
    assert np.abs(first["eps_qp"] - orc.g0w0(eps, L, 1, 1)["eps_qp"]).max() < 1e-12
    r = orc.scgw(eps, L, 1, 1, conv=1e-10)
    assert r["converged"] and np.all(np.isfinite(r["eps_qp"]))
