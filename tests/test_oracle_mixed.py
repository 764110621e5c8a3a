"""Pins of the input rounding of the mixed-precision mode (oracle
fixed_point_grid) and of the claim it rests on: the moments of the rounded
system move the QP energies by far less than the 1 meV tolerance of the
mixed path.

The rounding is not in the paper; it is this library's precision mode.  It is
pinned by hand-computed values, the half-unit error bound, the integer grid,
ties away from zero, idempotence and exact covariance under powers of two.
"""
import math

import numpy as np

import mgw_inputs
from oracle import mgw_oracle as orc

HA_TO_MEV = 27211.386245988


def test_known_values():
    # max 0.3: floor(log2 0.3) = -2, e = 0, grid 2^-16
    x = np.array([0.3, -0.1, 1e-6, 0.0])
    r = orc.fixed_point_grid(x)
    assert r[0] == 19661 / 65536      # 0.3 * 65536 = 19660.8
    assert r[1] == -6554 / 65536      # -6553.6
    assert r[2] == 0.0 and r[3] == 0.0
    # 8 bits on the same tensor: grid 2^-8
    r8 = orc.fixed_point_grid(x, bits=8)
    assert r8[0] == 77 / 256 and r8[1] == -26 / 256  # 76.8, -25.6


def test_ties_go_away_from_zero():
    # max 0.25: e = 0, grid 2^-16; 2.5 and -2.5 grid units are ties
    x = np.array([0.25, 5 * 2.0**-17, -5 * 2.0**-17, 3 * 2.0**-17])
    r = orc.fixed_point_grid(x)
    assert r[1] == 3 * 2.0**-16 and r[2] == -3 * 2.0**-16 and r[3] == 2 * 2.0**-16


def test_bound_grid_and_idempotence():
    g = np.random.default_rng(3)
    for scale in (1e-3, 0.7, 5.0):
        x = g.standard_normal((40, 30)) * scale
        r = orc.fixed_point_grid(x)
        e = math.frexp(np.abs(x).max())[1] + 1
        assert np.abs(x).max() < 2.0 ** (e - 1) <= 2 * np.abs(x).max()
        unit = 2.0 ** (e - 16)
        q = r / unit
        assert np.array_equal(q, np.round(q)) and np.abs(q).max() <= 2**15
        assert np.abs(r - x).max() <= unit / 2
        assert np.array_equal(orc.fixed_point_grid(r), r)
        assert np.array_equal(orc.fixed_point_grid(x * 8.0), r * 8.0)


def test_rounded_system_keeps_qp_energies_within_a_fraction_of_a_meV():
    # the mixed path's moments are those of the rounded system; its QP
    # energies differ from the unrounded ones by much less than 1 meV
    shape, seed = mgw_inputs.workload("g0w0-nmo24-naux72")
    eps, L = mgw_inputs.system(shape, seed)
    for N in (5, 7):
        ref = orc.g0w0(eps, L, shape.nocc, N)
        D = orc.energy_differences(eps, shape.nocc)
        Lov = orc.fixed_point_grid(orc.particle_hole_block(L, shape.nocc))
        W = orc.response_moments(Lov, D, 2 * N + 2)
        sh, sp = orc.sigma_moments(eps, shape.nocc, orc.fixed_point_grid(L), W)
        qp = orc.qp_solve(np.diag(eps), orc.block_lanczos(sh, N + 1)[:3], orc.block_lanczos(sp, N + 1)[:3],
                          2.0 * shape.nocc)
        d = np.abs(qp["eps_qp"] - ref["eps_qp"]).max() * HA_TO_MEV
        assert d < 0.1, (N, d)


def test_rounding_a_part_on_the_whole_tensors_grid():
    g = np.random.default_rng(4)
    x = g.standard_normal((6, 50))
    whole = orc.fixed_point_grid(x)
    m = float(np.abs(x).max())
    parts = np.concatenate([orc.fixed_point_grid(x[:, :20], ref_max=m), orc.fixed_point_grid(x[:, 20:], ref_max=m)],
                           axis=1)
    assert np.array_equal(parts, whole)
