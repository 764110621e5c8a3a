"""Plant plausible mistakes in a copy of the oracle and check a pin catches each.

Each case rewrites one line of an oracle function's source (a dropped term,
a wrong sign or factor, the garbled W^(n) index of Eqs. 6-7, a transposed
operand), executes the mutant in a namespace of its own and runs the same
brute-force comparison the pins use.  The mutant must fail it.  The real
oracle module is never modified.
"""
import inspect
import math
import types

import numpy as np
import pytest

import brute
import mgw_inputs
from oracle import mgw_oracle as orc


def mutant(func_names, old, new):
    """A copy of the oracle module with `old` replaced by `new` inside one of
    the named functions (exactly one occurrence), executed whole in a fresh
    namespace so every function of the copy calls the mutated one."""
    full = inspect.getsource(orc)
    hit = 0
    for name in func_names:
        src = inspect.getsource(getattr(orc, name))
        if old in src:
            hit += src.count(old)
            assert full.count(src) == 1
            full = full.replace(src, src.replace(old, new))
    assert hit == 1, (old, hit)
    mod = types.ModuleType("oracle_mutant")
    exec(compile(full, "<oracle mutant>", "exec"), mod.__dict__)
    return mod


def system(nocc=3, nvir=5, naux=12, seed=7, scale=2.0):
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    return eps, mgw_inputs.df_tensor(naux, nocc + nvir, seed) * scale


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def sigma_pin_error(mod, screening="tda"):
    eps, L = system()
    nmom = 8
    D = mod.energy_differences(eps, 3)
    W = mod.response_moments(mod.particle_hole_block(L, 3), D, nmom, screening, 48)
    sh, sp = mod.sigma_moments(eps, 3, L, W)
    bh, bp = brute.sigma_lehmann(eps, L, 3, nmom, screening)
    return max(max(rel(sh[n], bh[n]), rel(sp[n], bp[n])) for n in range(nmom))


def offset_pin_error(mod):
    """eta~(0) with the exact G_offset against the brute-force A/B solution."""
    eps, L = system(nocc=3, nvir=6, naux=14, scale=3.0)
    D = mod.energy_differences(eps, 3)
    Lov = mod.particle_hole_block(L, 3)
    eta0, _, _, V = brute.rpa_eta_bruteforce(eps, L, 3, 0)
    return rel(mod.rpa_eta0(Lov, D, 48, "exact"), V @ eta0)


def lanczos_pin_error(mod):
    eps, L = system(nocc=3, nvir=6, naux=14)
    nmom = 8
    W = orc.tda_response_moments(orc.particle_hole_block(L, 3), orc.energy_differences(eps, 3), nmom)
    sh, _ = orc.sigma_moments(eps, 3, L, W)
    coup, alpha, beta, r = mod.block_lanczos(sh, 4)
    T = brute.block_tridiagonal(alpha, beta)
    err, Tn = 0.0, np.eye(T.shape[0])
    for n in range(nmom):
        err = max(err, rel(coup @ Tn[:r, :r] @ coup.T, sh[n]))
        Tn = Tn @ T
    return err


def qp_pin_error(mod):
    eps, L = system()
    r = orc.g0w0(eps, L, 3, 2)
    H = mod.upfolded_hamiltonian(np.diag(eps), r["hole"][:3], r["part"][:3])
    nmo = eps.size
    Wt, dt = H[:nmo, nmo:], H[nmo:, nmo:]
    err, Dn = 0.0, np.eye(dt.shape[0])
    for n in range(6):
        err = max(err, rel(Wt @ Dn @ Wt.T, r["sigma_hole"][n] + r["sigma_part"][n]))
        Dn = Dn @ dt
    return err


def spectral_pin_error(mod):
    eps, L = system()
    r = orc.g0w0(eps, L, 3, 2)
    H = orc.upfolded_hamiltonian(np.diag(eps), r["hole"][:3], r["part"][:3])
    omega = np.linspace(r["E"].min() - 0.5, r["E"].max() + 0.5, 31)
    got = mod.spectral_function(r["E"], r["weight"], omega, 0.05)
    return rel(got, brute.spectral_downfolded(H, eps.size, omega, 0.05))


def naf_pin_error(mod):
    # the metric against the explicit pair sum, the truncation error against
    # the dropped spectrum (Eckart-Young), Sigma(n) unchanged without truncation
    eps, L = system(naux=14)
    err = 0.0
    for pairs in ("no_vv", "full"):
        _, lam = mod.naf_basis(L, 3, -1.0, pairs)
        ref = np.sort(np.linalg.eigvalsh(brute.naf_metric_pairs(L, 3, pairs)))[::-1]
        err = max(err, np.abs(lam - ref).max() / ref.max())
        V = L[:, orc.naf_pairs(8, 3, pairs)]
        U, _ = mod.naf_basis(L, 3, 0.5 * (ref[5] + ref[6]), pairs)
        resid = V - U @ (U.T @ V)
        err = max(err, abs(np.sum(resid**2) - ref[6:].sum()) / ref.sum())
    a = orc.g0w0(eps, L, 3, 2)
    b = orc.g0w0(eps, mod.naf_compress(L, 3, -1.0, "full"), 3, 2)
    return max(err, max(rel(b["sigma_hole"][n], a["sigma_hole"][n]) for n in range(6)))


def qsgw_pin_error(mod):
    # decoupled poles against Eq. 10's downfolding, both potentials against
    # their expansions in the first two moments, the Hartree-Fock state of the
    # field without a potential, and the fixed point of Eq. 35
    eps, L = system(scale=3.0)
    r = orc.g0w0(eps, L, 3, 2)
    hole, part = r["hole"][:3], r["part"][:3]
    nmo = eps.size
    H = orc.upfolded_hamiltonian(np.zeros((nmo, nmo)), hole, part)
    Wt, dt = H[:nmo, nmo:], H[nmo:, nmo:]
    (vh, eh), (vp, ep) = mod.decoupled_poles(hole), mod.decoupled_poles(part)
    v, e = np.concatenate([vh, vp], axis=1), np.concatenate([eh, ep])
    z = 0.3 + 0.05j
    err = rel((v / (z - e)) @ v.T, Wt @ np.linalg.solve(z * np.eye(dt.shape[0]) - dt, Wt.T))
    M0 = r["sigma_hole"][0] + r["sigma_part"][0]
    M1 = r["sigma_hole"][1] + r["sigma_part"][1]
    E = np.diag(eps)
    err = max(err, rel(mod.qsgw_potential(eps, hole, part, "srg", srg_s=1e-9), 1e-9 * (E @ M0 + M0 @ E - 2.0 * M1)))
    err = max(err, rel(mod.qsgw_potential(eps, hole, part, "eta", delta=1e5), (0.5 * (E @ M0 + M0 @ E) - M1) / 1e10))
    h = orc.hf_core_hamiltonian(eps, L, 3)
    e0 = mod.qsgw_scf(h, L, np.zeros((nmo, nmo)), np.eye(nmo), 3)[0]
    err = max(err, np.abs(e0 - eps).max())
    q = mod.qsgw(h, L, eps, 3, 2, conv=1e-10)
    e, C = q["eps"], q["C"]
    Lm = orc.rotate_df(L, C)
    W = orc.response_moments(orc.particle_hole_block(Lm, 3), orc.energy_differences(e, 3), 6)
    sh, sp = orc.sigma_moments(e, 3, Lm, W)
    V = orc.qsgw_potential(e, orc.block_lanczos(sh, 3), orc.block_lanczos(sp, 3))
    F = orc.fock_build(h, L, 2.0 * C[:, :3] @ C[:, :3].T) + C @ V @ C.T
    return max(err, np.abs(F @ C - C * e[None, :]).max() * 1e2)


def scgw_pin_error(mod):
    # the self-energy moments over a QMO space against the Lehmann
    # convolution, and three scGW iterations against the Lehmann driver
    eps, L = system(scale=3.0)
    g = orc.g0w0(eps, L, 3, 2)
    E, m = g["E"], g["m"]
    Vhat, Via = mod.qmo_tensors(L, g["chi"], m)
    D = orc.energy_differences(E, m)
    sh, sp = mod.sigma_moments(E, m, Vhat, orc.response_moments(Via, D, 6))
    Vh0, Via0 = orc.qmo_tensors(L, g["chi"], m)
    bh, bp = brute.sigma_lehmann_general(E, m, Vh0, Via0, D, 6)
    err = max(max(rel(sh[n], bh[n]), rel(sp[n], bp[n])) for n in range(6))
    ref = brute.scgw_lehmann(orc, eps, L, 3, 1, False, False, 3)
    got = mod.scgw(eps, L, 3, 1, max_iter=3, conv=0.0)["eps_qp"]
    return max(err, np.abs(got - ref[2]).max() * 1e3)


CASES = [
    # (functions, old, new, pin, screening)
    (["tda_response_moments"], "T * D[None, :] + 2.0 *", "T * D[None, :] + 1.0 *", "sigma", "tda"),
    (["tda_response_moments"], "T * D[None, :] + 2.0 * (W[n] @ Lov)", "2.0 * (W[n] @ Lov)", "sigma", "tda"),
    (["tda_response_moments"], "W[n] = T @ Lov.T", "W[n] = Lov @ T.T @ np.eye(Lov.shape[0]) * 0 + T @ T.T", "sigma", "tda"),
    (["rpa_response_moments"], "(D * D)[None, :] + 4.0", "(D * D)[None, :] + 2.0", "sigma", "rpa"),
    (["rpa_response_moments"], "Lov * D[None, :]]", "Lov]", "sigma", "rpa"),
    (["rpa_eta0"], "G_off += 4.0 * wj", "G_off += 2.0 * wj", "sigma", "rpa"),
    (["rpa_eta0"], "(np.linalg.inv(eye + Q) - eye)", "(np.linalg.inv(eye + Q) + eye)", "sigma", "rpa"),
    (["rpa_eta0"], "S = eye + 4.0 *", "S = eye - 4.0 *", "sigma", "rpa"),
    (["rpa_g_offset_exact"], "C = 1.0 / (D[:, None] + D[None, :])", "C = 0.5 / np.sqrt(D[:, None] * D[None, :])",
     "offset", None),
    (["rpa_g_offset_exact"], "return VD + 4.0 * VD @", "return VD + 2.0 * VD @", "offset", None),
    (["rpa_g_offset_exact"], "((Lov.T @ Lov) * C)", "((Lov.T @ Lov) @ C)", "offset", None),
    (["sigma_moments"], "sign = -1.0 if hole else 1.0", "sign = 1.0", "sigma", "tda"),
    (["sigma_moments"], "wgt = 2.0 *", "wgt = 1.0 *", "sigma", "tda"),
    # the W^(n) index printed inside the t-sum of Eqs. 6-7
    (["sigma_moments"], "out[n] += np.tensordot(wgt, Wx[xs], axes=1)",
     "out[n] += np.tensordot(wgt, ((Lxp @ W[n]) @ Lx)[xs], axes=1)", "sigma", "tda"),
    (["sigma_moments"], "math.comb(n, t)", "1", "sigma", "tda"),
    (["sigma_moments"], "eps[xs] ** (n - t)", "eps[xs] ** t", "sigma", "tda"),
    (["sigma_moments"], "Wx = (Lxp @ W[t]) @ Lx", "Wx = (Lxp @ W[t]) @ Lx * (1 + 0.01)", "sigma", "tda"),
    (["block_lanczos"], "Rk -= C[i][k] @ a", "Rk -= a @ C[i][k] * 0.5", "lanczos", None),
    (["block_lanczos"], "Rk -= C[i - 1][k] @ beta[i - 1].T", "Rk -= C[i - 1][k] @ beta[i - 1].T * 0.0", "lanczos", None),
    (["block_lanczos"], "acc += Xk.T @ Sh[k + l + m] @ Yl", "acc += Xk.T @ Sh[k + l] @ Yl", "lanczos", None),
    (["block_lanczos"], "alpha = [s * a + c * eye for a in alpha]", "alpha = [s * a for a in alpha]", "lanczos", None),
    (["upfolded_hamiltonian"], "H[o + r : o + 2 * r, o : o + r] = beta[i]", "H[o + r : o + 2 * r, o : o + r] = 0.5 * beta[i]", "qp", None),
    (["upfolded_hamiltonian"], "H[:nmo, off : off + r] = coup", "H[:nmo, off : off + r] = coup.T @ coup", "qp", None),
    (["spectral_function"], "A += wa * delta /", "A += wa * delta * delta /", "spectral", None),
    (["spectral_function"], "return A / math.pi", "return A / (2.0 * math.pi)", "spectral", None),
    (["spectral_function"], "((w - Ea) ** 2 + delta * delta)", "((w + Ea) ** 2 + delta * delta)", "spectral", None),
    (["naf_pairs"], "mask[nocc:, nocc:] = False", "mask[:nocc, :nocc] = False", "naf", None),
    (["naf_basis"], "return U[:, lam > eps_naf], lam", "return U[:, lam >= -1.0], lam", "naf", None),
    (["naf_basis"], "lam, U = lam[::-1], U[:, ::-1]", "lam, U = lam[::-1], U", "naf", None),
    (["naf_compress"], "np.tensordot(U.T, L, axes=1)", "np.tensordot(U.T, L, axes=1) * 1.01", "naf", None),
    (["qsgw_potential"], "R = Dl / (Dl * Dl + delta * delta)", "R = Dl / (Dl * Dl + 2.0 * delta * delta)", "qsgw", None),
    (["qsgw_potential"], "return 0.5 * (A + A.T)", "return A", "qsgw", None),
    (["qsgw_potential"], "(1.0 - np.exp(-s2 * srg_s))", "(1.0 - np.exp(-s2 * srg_s * 0.5))", "qsgw", None),
    (["qsgw_potential"], "(d[:, None] + d[None, :]) / s2", "(d[:, None] - d[None, :]) / s2", "qsgw", None),
    (["decoupled_poles"], "return coup @ U[:r, :], e", "return coup @ U[:r, :], -e", "qsgw", None),
    (["qsgw_scf"], "rho_new = 2.0 * C[:, :nocc]", "rho_new = 1.0 * C[:, :nocc]", "qsgw", None),
    (["qsgw"], "Vref = C @ V @ C.T", "Vref = C.T @ V @ C", "qsgw", None),
    (["scgw"], 'epsG, mG, Vhat = qp["E"], qp["m"], Vq', 'epsG, mG, Vhat = qp["E"], nocc, Vq', "scgw", None),
    (["qmo_tensors"], 'np.einsum("Qpq,qx->Qpx", L, chi,', 'np.einsum("Qpq,qx->Qpx", L, chi / np.sqrt((chi**2).sum(0)),', "scgw", None),
    (["qmo_tensors"], 'np.einsum("pi,Qpx->Qix", chi[:, :m],', 'np.einsum("pi,Qpx->Qix", chi[:, :m][:, ::-1],', "scgw", None),
    (["sigma_moments"], "(False, slice(nocc, nx), sp)", "(False, slice(nocc, nmo), sp)", "scgw", None),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_pins_catch_planted_mistake(case):
    funcs, old, new, pin, screening = CASES[case]
    mod = mutant(funcs, old, new)
    if pin == "sigma":
        err = sigma_pin_error(mod, screening)
    elif pin == "lanczos":
        err = lanczos_pin_error(mod)
    elif pin == "spectral":
        err = spectral_pin_error(mod)
    elif pin == "naf":
        err = naf_pin_error(mod)
    elif pin == "qsgw":
        err = qsgw_pin_error(mod)
    elif pin == "scgw":
        err = scgw_pin_error(mod)
    elif pin == "offset":
        err = offset_pin_error(mod)
    else:
        err = qp_pin_error(mod)
    assert not (err < 1e-6), f"planted mistake went unnoticed: {old!r} -> {new!r} (err {err})"


def test_unmutated_copy_passes_every_pin():
    mod = mutant(["sigma_moments"], "wgt = 2.0 *", "wgt = 2.0 *")
    assert sigma_pin_error(mod, "tda") < 1e-10
    assert sigma_pin_error(mod, "rpa") < 1e-9
    assert lanczos_pin_error(mod) < 1e-9
    assert qp_pin_error(mod) < 1e-9
    assert spectral_pin_error(mod) < 1e-10
    assert naf_pin_error(mod) < 1e-10
    assert qsgw_pin_error(mod) < 1e-6
    assert scgw_pin_error(mod) < 1e-6
    assert offset_pin_error(mod) < 1e-10
    assert math.isfinite(lanczos_pin_error(orc))
