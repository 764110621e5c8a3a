"""Pins of the CPU oracle against definitions independent of it.

Every check reaches the expected value by another route: explicit matrix
powers, full diagonalisation and Lehmann sums, the spin-orbital formulation,
closed forms for a one-pair system, the exact all-pole upfolded Hamiltonian,
and plain integrals with known values.  A dropped term, a wrong sign or
factor, or a transposed operand in the oracle fails at least one of them
(tests/test_oracle_mutations.py plants such mistakes and checks that).
"""
import math

import numpy as np
import pytest

import brute
import mgw_inputs
from oracle import mgw_oracle as orc


def small_system(nocc=3, nvir=5, naux=12, seed=7, scale=1.0):
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    L = mgw_inputs.df_tensor(naux, nocc + nvir, seed) * scale
    return eps, L


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- quadrature


def test_clenshaw_curtis_exact_on_polynomials():
    # CC with n+1 points integrates polynomials of degree <= n exactly
    for n in (2, 8, 16, 48):
        x, w = orc.clenshaw_curtis(n)
        for deg in range(0, n + 1):
            exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
            assert abs(np.dot(w, x**deg) - exact) < 1e-13


def test_mapped_rule_known_integrals():
    # the rule drops the z = inf node, so it is exact only for integrands that
    # decay faster than 1/z^2, which both integrands of Eqs. 24-25 do
    z, w = orc.quadrature_rule(48, 0.4, 4.5)
    for b in (0.3, 1.0, 4.0):
        # int_0^inf dz / (b^2 + z^2)^2 = pi / (4 b^3)
        assert abs(np.dot(w, 1.0 / (b * b + z * z) ** 2) - math.pi / (4 * b**3)) < 1e-12
        # int_0^inf dz / ((b^2 + z^2)(c^2 + z^2)) = pi / (2 b c (b + c))
        c = math.sqrt(2.0)
        assert abs(np.dot(w, 1.0 / ((b * b + z * z) * (c * c + z * z))) - math.pi / (2 * b * c * (b + c))) < 1e-12
    # int_0^inf exp(-s z) dz = 1/s
    for s in (0.8, 2.0, 9.0):
        assert abs(np.dot(w, np.exp(-s * z)) - 1.0 / s) < 1e-10


# ---------------------------------------------------------------- response


def test_tda_recursion_equals_matrix_powers():
    eps, L = small_system()
    nocc = 3
    D = orc.energy_differences(eps, nocc)
    Lov = orc.particle_hole_block(L, nocc)
    W = orc.tda_response_moments(Lov, D, 8)
    Wb = brute.tda_W_bruteforce(eps, L, nocc, 8)
    for n in range(8):
        assert rel(W[n], Wb[n]) < 1e-12, n


def test_rpa_recursion_equals_eigenproblem():
    eps, L = small_system(scale=3.0)
    nocc = 3
    D = orc.energy_differences(eps, nocc)
    Lov = orc.particle_hole_block(L, nocc)
    W = orc.rpa_response_moments(Lov, D, 8, nq=48)
    Wb = brute.rpa_W_bruteforce(eps, L, nocc, 8)
    for n in range(8):
        assert rel(W[n], Wb[n]) < 1e-10, n


def test_rpa_eta0_quadrature_converges_to_exact():
    eps, L = small_system(nocc=4, nvir=9, naux=20, scale=3.0)
    nocc = 4
    D = orc.energy_differences(eps, nocc)
    Lov = orc.particle_hole_block(L, nocc)
    eta0, _, _, V = brute.rpa_eta_bruteforce(eps, L, nocc, 0)
    exact = V @ eta0
    errs = [rel(orc.rpa_eta0(Lov, D, nq), exact) for nq in (8, 16, 32, 48)]
    assert errs[-1] < 1e-12
    assert errs[0] > errs[1] > errs[2]  # exponential decay with the node count


def test_rpa_g_offset_exact_equals_the_integral():
    """The closed-form G_offset (Cauchy matrix) against Eq. 25's integral taken
    numerically element by element with adaptive quadrature (scipy), a route
    independent of both the closed form and the Clenshaw-Curtis rule."""
    integrate = pytest.importorskip("scipy.integrate")
    eps, L = small_system(nocc=2, nvir=3, naux=4, scale=3.0)
    D = orc.energy_differences(eps, 2)
    V = orc.particle_hole_block(L, 2)
    VD, M = V * D[None, :], V.T @ V
    got = orc.rpa_g_offset_exact(V, D)
    for P in range(V.shape[0]):
        for ia in range(D.size):
            f = lambda z: 4.0 * np.sum(VD[P] * np.exp(-z * D) * M[:, ia]) * math.exp(-z * D[ia])
            val, _ = integrate.quad(f, 0.0, np.inf, epsabs=1e-15, epsrel=1e-13, limit=200)
            assert abs(got[P, ia] - (VD[P, ia] + val)) < 1e-12 * max(1.0, abs(got[P, ia]))


def test_rpa_eta0_exact_offset_matches_bruteforce():
    """eta~(0) with the exact G_offset (only G_main by quadrature) against the
    brute-force A/B diagonalisation; and the quadrature G_offset converges to
    the exact one with the node count."""
    eps, L = small_system(nocc=4, nvir=9, naux=20, scale=3.0)
    nocc = 4
    D = orc.energy_differences(eps, nocc)
    Lov = orc.particle_hole_block(L, nocc)
    eta0, _, _, V = brute.rpa_eta_bruteforce(eps, L, nocc, 0)
    assert rel(orc.rpa_eta0(Lov, D, 48, "exact"), V @ eta0) < 1e-12
    exact = orc.rpa_g_offset_exact(Lov, D)
    errs = []
    for nq in (8, 16, 32):
        z, w = orc.quadrature_rule(nq, float(D.min()), float(D.max()))
        G = Lov * D[None, :]
        for zj, wj in zip(z, w):
            E = np.exp(-zj * D)
            G = G + 4.0 * wj * (((Lov * (D * E)[None, :]) @ Lov.T) @ (Lov * E[None, :]))
        errs.append(rel(G, exact))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9


def test_rpa_eta0_one_pair_closed_form():
    # nocc = nvir = naux = 1: eta(0) = d / Omega, Omega = sqrt(d (d + 4 v^2))
    eps = np.array([-0.7, 0.9])
    v = 0.37
    L = np.array([[[0.2, v], [v, -0.1]]])
    D = orc.energy_differences(eps, 1)
    d = D[0]
    Om = math.sqrt(d * (d + 4 * v * v))
    t0 = orc.rpa_eta0(orc.particle_hole_block(L, 1), D, 48)
    assert abs(t0[0, 0] - v * d / Om) < 1e-13
    t0 = orc.rpa_eta0(orc.particle_hole_block(L, 1), D, 48, "exact")
    assert abs(t0[0, 0] - v * d / Om) < 1e-13


# ---------------------------------------------------------------- self-energy


@pytest.mark.parametrize("screening", ["tda", "rpa"])
def test_sigma_moments_equal_lehmann_sums(screening):
    eps, L = small_system(scale=2.0)
    nocc, nmom = 3, 8
    D = orc.energy_differences(eps, nocc)
    W = orc.response_moments(orc.particle_hole_block(L, nocc), D, nmom, screening, 48)
    sh, sp = orc.sigma_moments(eps, nocc, L, W)
    bh, bp = brute.sigma_lehmann(eps, L, nocc, nmom, screening)
    for n in range(nmom):
        assert rel(sh[n], bh[n]) < 1e-10, ("hole", n)
        assert rel(sp[n], bp[n]) < 1e-10, ("particle", n)


def test_sigma_spin_factor_against_spin_orbital_formulation():
    eps, L = small_system(nocc=2, nvir=4, naux=6, scale=2.0)
    nocc, nmom = 2, 6
    W = orc.tda_response_moments(orc.particle_hole_block(L, nocc), orc.energy_differences(eps, nocc), nmom)
    sh, sp = orc.sigma_moments(eps, nocc, L, W)
    bh, bp = brute.sigma_spin_orbital(eps, L, nocc, nmom)
    for n in range(nmom):
        assert rel(sh[n], bh[n]) < 1e-10
        assert rel(sp[n], bp[n]) < 1e-10


def test_sigma_one_pair_closed_form():
    eps = np.array([-0.7, 0.9])
    v = 0.37
    L = np.array([[[0.2, v], [v, -0.1]]])
    d = eps[1] - eps[0]
    Om = d + 2 * v * v
    W = orc.tda_response_moments(orc.particle_hole_block(L, 1), orc.energy_differences(eps, 1), 6)
    sh, sp = orc.sigma_moments(eps, 1, L, W)
    for n in range(6):
        eh = 2 * v * v * np.outer(L[0, :, 0], L[0, :, 0]) * (eps[0] - Om) ** n
        ep = 2 * v * v * np.outer(L[0, :, 1], L[0, :, 1]) * (eps[1] + Om) ** n
        assert np.allclose(sh[n], eh, rtol=1e-13, atol=1e-15)
        assert np.allclose(sp[n], ep, rtol=1e-13, atol=1e-15)


def test_sigma_rows_subset_matches_full():
    eps, L = small_system()
    W = orc.tda_response_moments(orc.particle_hole_block(L, 3), orc.energy_differences(eps, 3), 6)
    sh, sp = orc.sigma_moments(eps, 3, L, W)
    rh, rp = orc.sigma_moments(eps, 3, L, W, rows=[1, 6])
    assert np.array_equal(rh, sh[:, [1, 6]]) and np.array_equal(rp, sp[:, [1, 6]])


def test_zero_interaction_gives_zero_sigma_and_bare_energies():
    eps = mgw_inputs.orbital_energies(3, 5, 3)
    L = np.zeros((6, 8, 8))
    res = orc.g0w0(eps, L, 3, 3)
    assert np.all(res["sigma_hole"] == 0) and np.all(res["sigma_part"] == 0)
    assert np.array_equal(res["eps_qp"], eps)
    assert res["hole"][3] == 0 and res["part"][3] == 0


# ---------------------------------------------------------------- block Lanczos


def moments_from_blocks(coup, alpha, beta, nmom):
    T = brute.block_tridiagonal(alpha, beta)
    r = alpha.shape[1]
    out = []
    Tn = np.eye(T.shape[0])
    for _ in range(nmom):
        out.append(coup @ Tn[:r, :r] @ coup.T)
        Tn = Tn @ T
    return np.stack(out)


@pytest.mark.parametrize("nmom_max", [1, 3, 5])
def test_block_lanczos_reproduces_moments(nmom_max):
    eps, L = small_system(nocc=3, nvir=6, naux=14, scale=2.0)
    nocc = 3
    nmom = 2 * nmom_max + 2
    W = orc.tda_response_moments(orc.particle_hole_block(L, nocc), orc.energy_differences(eps, nocc), nmom)
    sh, sp = orc.sigma_moments(eps, nocc, L, W)
    for sig in (sh, sp):
        coup, alpha, beta, r = orc.block_lanczos(sig, nmom_max + 1)
        assert r == eps.size
        rec = moments_from_blocks(coup, alpha, beta, nmom)
        for n in range(nmom):
            assert rel(rec[n], sig[n]) < 1e-9, n
        # symmetric normalisation: beta blocks symmetric PSD, coupling = S0^(1/2)
        for b in beta:
            assert np.allclose(b, b.T, atol=1e-12)
            assert np.linalg.eigvalsh(b).min() > -1e-10
        assert np.allclose(coup @ coup, sig[0], rtol=1e-10, atol=1e-14)


def test_block_lanczos_exact_when_poles_fit():
    # hole sector has nocc * ov = 1*2 = 2 poles: Sigma(0) has rank 2 < nmo = 3,
    # and two blocks of size 2 hold every pole, so every moment is reproduced
    eps, L = small_system(nocc=1, nvir=2, naux=2, seed=11, scale=3.0)
    nocc = 1
    W = orc.tda_response_moments(orc.particle_hole_block(L, nocc), orc.energy_differences(eps, nocc), 10)
    sh, _ = orc.sigma_moments(eps, nocc, L, W)
    coup, alpha, beta, r = orc.block_lanczos(sh, 1)
    assert r == 2
    rec = moments_from_blocks(coup, alpha, beta, 10)
    for n in range(10):
        assert rel(rec[n], sh[n]) < 1e-9


# ---------------------------------------------------------------- H~, QP, Aufbau


def test_upfolded_hamiltonian_downfolds_to_the_moments():
    eps, L = small_system(nocc=3, nvir=5, naux=12, scale=2.0)
    nocc, nmom_max = 3, 2
    res = orc.g0w0(eps, L, nocc, nmom_max)
    H = orc.upfolded_hamiltonian(np.diag(eps), res["hole"][:3], res["part"][:3])
    nmo = eps.size
    Wt = H[:nmo, nmo:]
    dt = H[nmo:, nmo:]
    Dn = np.eye(dt.shape[0])
    for n in range(2 * nmom_max + 2):
        assert rel(Wt @ Dn @ Wt.T, res["sigma_hole"][n] + res["sigma_part"][n]) < 1e-9
        Dn = Dn @ dt


def test_qp_energies_converge_to_exact_upfolded():
    shape, seed = mgw_inputs.workload("g0w0-nmo24-naux72")
    eps, L = mgw_inputs.system(shape, seed)
    L = L * 3.0  # stronger coupling so the moment truncation is visible
    nocc = shape.nocc
    Hx = brute.exact_upfolded(eps, L, nocc)
    Ex, Xx = np.linalg.eigh(Hx)
    exact = orc.qp_energies(Ex, Xx[: eps.size])
    front = [nocc - 1, nocc]  # HOMO, LUMO
    errs = []
    for N in (1, 3, 5, 7):
        r = orc.g0w0(eps, L, nocc, N)
        errs.append(np.abs(r["eps_qp"][front] - exact[front]).max())
    assert errs[-1] < errs[0]
    assert errs[-1] < 2e-3


def test_exact_termination_reproduces_exact_spectrum():
    # tiny system whose every pole fits in the block tridiagonal chain
    eps, L = small_system(nocc=1, nvir=2, naux=2, seed=11, scale=3.0)
    nocc = 1
    Hx = brute.exact_upfolded(eps, L, nocc)
    Ex = np.linalg.eigvalsh(Hx)
    r = orc.g0w0(eps, L, nocc, 3)
    H = orc.upfolded_hamiltonian(np.diag(eps), r["hole"][:3], r["part"][:3])
    wts = np.linalg.eigh(H)
    E = wts[0][np.sum(wts[1][:3] ** 2, axis=0) > 1e-10]
    Exw = np.linalg.eigh(Hx)
    Ex = Exw[0][np.sum(Exw[1][:3] ** 2, axis=0) > 1e-10]
    assert E.size == Ex.size and np.allclose(E, Ex, atol=1e-8)


def test_qp_argmax_and_aufbau_brute_force():
    g = np.random.default_rng(5)
    for _ in range(20):
        E = np.sort(g.normal(size=15))
        chi = g.normal(size=(4, 15))
        wts = np.sum(chi**2, axis=0) / 4.0
        eqp = orc.qp_energies(E, chi)
        for p in range(4):
            best = max(range(15), key=lambda a: (chi[p, a] ** 2, -a))
            assert eqp[p] == E[best]
        nel = g.uniform(0, 2 * wts.sum())
        m, mu, n_out = orc.aufbau(E, wts, nel)
        cands = [abs(2 * wts[:k].sum() - nel) for k in range(16)]
        assert abs(cands[m] - min(cands)) < 1e-12
        assert abs(n_out - 2 * wts[:m].sum()) < 1e-12
        if 0 < m < 15:
            assert E[m - 1] <= mu <= E[m]


def test_hole_poles_below_particle_poles():
    shape, seed = mgw_inputs.workload("g0w0-nmo24-naux72")
    eps, L = mgw_inputs.system(shape, seed)
    r = orc.g0w0(eps, L, shape.nocc, 3)
    # physical weight sums to nmo; Aufbau fills nocc orbitals for a weakly
    # correlated system and puts mu in the HOMO-LUMO gap
    assert abs(r["weight"].sum() - eps.size) < 1e-9
    assert abs(r["nelec"] - 2 * shape.nocc) < 0.05
    assert r["eps_qp"][shape.nocc - 1] < r["mu"] < r["eps_qp"][shape.nocc]


def test_evgw_reaches_a_fixed_point():
    eps, L = small_system(nocc=3, nvir=5, naux=12, scale=2.0)
    out = orc.evgw(eps, L, 3, 2, conv_e=1e-9, max_iter=60)
    assert out["converged"]
    # at the fixed point the QP energies regenerate themselves
    r = orc.g0w0(out["eps_qp"], L, 3, 2, fock=np.diag(eps))
    assert np.abs(r["eps_qp"] - out["eps_qp"]).max() < 1e-8


def test_tda_rows_subset_matches_full():
    eps, L = small_system()
    D = orc.energy_differences(eps, 3)
    Lov = orc.particle_hole_block(L, 3)
    W = orc.tda_response_moments(Lov, D, 6)
    Wr = orc.tda_response_moments(Lov, D, 6, rows=[0, 5, 11])
    assert np.allclose(Wr, W[:, [0, 5, 11]], rtol=1e-13, atol=1e-16)


# ------------------------------------------------------- spectral function


def _g0w0_poles(nmom_max=2):
    eps, L = small_system(scale=2.0)
    r = orc.g0w0(eps, L, 3, nmom_max)
    H = orc.upfolded_hamiltonian(np.diag(eps), r["hole"][:3], r["part"][:3])
    return eps.size, H, r["E"], r["weight"]


def test_spectral_function_equals_the_downfolded_green_function():
    # Eq. 12 from the poles of H~ against -Im tr G by downfolding (Eq. 10)
    nmo, H, E, weight = _g0w0_poles()
    omega = np.linspace(E.min() - 0.5, E.max() + 0.5, 41)
    for delta in (0.02, 0.1):
        got = orc.spectral_function(E, weight, omega, delta)
        ref = brute.spectral_downfolded(H, nmo, omega, delta)
        assert rel(got, ref) < 1e-10


def test_spectral_function_window_integrals_and_total_weight():
    # a window integral of A equals the Lorentzian antiderivative summed over
    # poles, and the weights of H~'s eigenvectors add up to nmo
    nmo, H, E, weight = _g0w0_poles()
    assert abs(weight.sum() - nmo) < 1e-10
    delta = 0.05
    a, b = E.min() - 0.3, E.min() + 2.0
    x = np.linspace(a, b, 200001)
    A = orc.spectral_function(E, weight, x, delta)
    h = x[1] - x[0]
    numeric = h * (A.sum() - 0.5 * (A[0] + A[-1]))
    exact = np.sum(weight * (np.arctan((b - E) / delta) - np.arctan((a - E) / delta))) / math.pi
    assert abs(numeric - exact) < 1e-6 * exact


# ------------------------------------------- natural auxiliary functions


@pytest.mark.parametrize("pairs", ["no_vv", "full"])
def test_naf_metric_matches_the_explicit_pair_sum(pairs):
    eps, L = small_system(nocc=3, nvir=5, naux=10)
    _, lam = orc.naf_basis(L, 3, 1e-5, pairs)
    ref = np.sort(np.linalg.eigvalsh(brute.naf_metric_pairs(L, 3, pairs)))[::-1]
    assert np.abs(lam - ref).max() < 1e-12 * ref.max()


@pytest.mark.parametrize("pairs", ["no_vv", "full"])
def test_naf_truncation_error_is_the_dropped_spectrum(pairs):
    # Eckart-Young: projecting the pair columns on the kept eigenvectors of M
    # leaves a squared Frobenius error equal to the dropped eigenvalues
    eps, L = small_system(nocc=3, nvir=5, naux=14)
    V = L[:, orc.naf_pairs(8, 3, pairs)]
    _, lam = orc.naf_basis(L, 3, -1.0, pairs)
    thresh = 0.5 * (lam[5] + lam[6])  # keep six
    U, _ = orc.naf_basis(L, 3, thresh, pairs)
    assert U.shape[1] == 6
    resid = V - U @ (U.T @ V)
    assert abs(np.sum(resid**2) - lam[6:].sum()) < 1e-10 * lam.sum()


def test_naf_without_truncation_leaves_the_sigma_moments_unchanged():
    # keeping every NAF rotates the auxiliary basis; Sigma(n) is invariant
    eps, L = small_system(nocc=3, nvir=5, naux=12, scale=2.0)
    Ln = orc.naf_compress(L, 3, -1.0, "full")
    assert Ln.shape == L.shape
    a = orc.g0w0(eps, L, 3, 2)
    b = orc.g0w0(eps, Ln, 3, 2)
    for n in range(6):
        assert rel(b["sigma_hole"][n], a["sigma_hole"][n]) < 1e-12
        assert rel(b["sigma_part"][n], a["sigma_part"][n]) < 1e-12


@pytest.mark.parametrize("pairs", ["no_vv", "full"])
def test_naf_of_an_exactly_low_rank_tensor_keeps_its_rank_and_moments(pairs):
    # L of rank 5 spread over 12 auxiliary functions: NAF keeps exactly 5 and
    # the G0W0 moments and QP energies are those of the uncompressed tensor
    nocc, nmo, naux, r = 3, 8, 12, 5
    g = np.random.default_rng(11)
    B = g.standard_normal((r, nmo, nmo))
    B = 0.1 * (B + B.transpose(0, 2, 1)) / 2
    L = np.tensordot(g.standard_normal((naux, r)), B, axes=1)
    eps = mgw_inputs.orbital_energies(nocc, nmo - nocc, 5)
    Ln = orc.naf_compress(L, nocc, 1e-5, pairs)
    assert Ln.shape[0] == r
    a = orc.g0w0(eps, L, nocc, 2)
    b = orc.g0w0(eps, Ln, nocc, 2)
    for n in range(6):
        assert rel(b["sigma_hole"][n], a["sigma_hole"][n]) < 1e-10
        assert rel(b["sigma_part"][n], a["sigma_part"][n]) < 1e-10
    assert np.abs(b["eps_qp"] - a["eps_qp"]).max() < 1e-9
