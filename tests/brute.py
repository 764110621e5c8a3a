"""Brute-force references that pin the oracle to definitions, not to itself.

Each function here reaches a quantity by a route independent of the oracle's
recursions: explicit particle-hole matrices and their powers, full
diagonalisation and Lehmann sums over explicit poles, the spin-orbital
(unrestricted-spin) formulation with no spin factors put in by hand, and the
exact (all-pole) upfolded Hamiltonian.  numpy's eigh/eig/matrix_power are
the library routines used.
"""
from __future__ import annotations

import numpy as np


def ph_eri(L, nocc):
    """(ia|jb) = sum_P V_{P,ia} V_{P,jb} (Eq. 13) over particle-hole pairs."""
    V = L[:, :nocc, nocc:].reshape(L.shape[0], -1)
    return V.T @ V, V


def tda_A(eps, L, nocc):
    """Restricted singlet TDA matrix A = D + 2 V^T V (Eqs. 20-21)."""
    K, V = ph_eri(L, nocc)
    D = (eps[None, nocc:] - eps[:nocc, None]).ravel()
    return np.diag(D) + 2.0 * K, V, D


def tda_W_bruteforce(eps, L, nocc, nmom):
    """W(n) = V A^n V^T with the explicit matrix power (eta(n) = A^n, Eq. 31)."""
    A, V, _ = tda_A(eps, L, nocc)
    return np.stack([V @ np.linalg.matrix_power(A, n) @ V.T for n in range(nmom)])


def rpa_eta_bruteforce(eps, L, nocc, n):
    """RPA eta(n) = (X+Y) Omega^n (X+Y)^T from the explicit non-Hermitian
    RPA eigenproblem [[A, B], [-B, -A]] (Eqs. 21-22), normalised so that
    X^T X - Y^T Y = 1; positive roots only."""
    K, V = ph_eri(L, nocc)
    D = (eps[None, nocc:] - eps[:nocc, None]).ravel()
    A = np.diag(D) + 2.0 * K
    B = 2.0 * K
    big = np.block([[A, B], [-B, -A]])
    w, vec = np.linalg.eig(big)
    w = w.real
    vec = vec.real
    pos = w > 0
    w, vec = w[pos], vec[:, pos]
    order = np.argsort(w)
    w, vec = w[order], vec[:, order]
    ov = D.size
    X, Y = vec[:ov], vec[ov:]
    norm = np.sum(X * X, axis=0) - np.sum(Y * Y, axis=0)
    X = X / np.sqrt(norm)[None, :]
    Y = Y / np.sqrt(norm)[None, :]
    XpY = X + Y
    return (XpY * w[None, :] ** n) @ XpY.T, w, XpY, V


def rpa_W_bruteforce(eps, L, nocc, nmom):
    out = []
    for n in range(nmom):
        eta, _, _, V = rpa_eta_bruteforce(eps, L, nocc, n)
        out.append(V @ eta @ V.T)
    return np.stack(out)


def poles_and_residues(eps, L, nocc, screening="tda"):
    """Neutral excitations Omega_nu and the restricted singlet residues
    w_{p x nu} = sqrt(2) sum_ia (px|ia) (X+Y)_{ia,nu}."""
    K, V = ph_eri(L, nocc)
    D = (eps[None, nocc:] - eps[:nocc, None]).ravel()
    if screening == "tda":
        Om, X = np.linalg.eigh(np.diag(D) + 2.0 * K)
        amp = X
    else:
        _, Om, amp, _ = rpa_eta_bruteforce(eps, L, nocc, 0)
    # (px|ia) as [p][x][ia]
    pxia = np.einsum("Ppx,Pj->pxj", L, V)
    w = np.sqrt(2.0) * np.einsum("pxj,jn->pxn", pxia, amp)
    return Om, w


def sigma_lehmann(eps, L, nocc, nmom, screening="tda"):
    """Sigma(n,<) = sum_{k,nu} w w (eps_k - Omega_nu)^n and
    Sigma(n,>) = sum_{c,nu} w w (eps_c + Omega_nu)^n (Eqs. 2-5 for the
    explicit pole representation)."""
    Om, w = poles_and_residues(eps, L, nocc, screening)
    nmo = eps.size
    sh = np.zeros((nmom, nmo, nmo))
    sp = np.zeros((nmom, nmo, nmo))
    for n in range(nmom):
        eh = (eps[:nocc, None] - Om[None, :]) ** n  # [k][nu]
        ep = (eps[nocc:, None] + Om[None, :]) ** n
        sh[n] = np.einsum("pkn,qkn,kn->pq", w[:, :nocc], w[:, :nocc], eh)
        sp[n] = np.einsum("pcn,qcn,cn->pq", w[:, nocc:], w[:, nocc:], ep)
    return sh, sp


def sigma_spin_orbital(eps, L, nocc, nmom):
    """TDA self-energy moments in a spin-orbital basis (2 nmo spin orbitals,
    every same-spin particle-hole pair kept, A_so = Delta + (ia|jb) with no
    spin factor); returns the alpha-alpha block, which a restricted
    calculation must reproduce."""
    nmo = eps.size
    nvir = nmo - nocc
    K, V = ph_eri(L, nocc)
    D = (eps[None, nocc:] - eps[:nocc, None]).ravel()
    ov = D.size
    # spin-orbital ph space: (sigma, i, a), sigma in {alpha, beta}
    A = np.zeros((2 * ov, 2 * ov))
    for s in range(2):
        for t in range(2):
            A[s * ov:(s + 1) * ov, t * ov:(t + 1) * ov] = K
    A += np.diag(np.concatenate([D, D]))
    Om, X = np.linalg.eigh(A)
    pxia = np.einsum("Ppx,Pj->pxj", L, V)  # spatial (px|jb)
    # alpha-spin p, x: couples to both spin blocks of the excitation vector
    w = np.einsum("pxj,jn->pxn", pxia, X[:ov] + X[ov:])
    sh = np.zeros((nmom, nmo, nmo))
    sp = np.zeros((nmom, nmo, nmo))
    for n in range(nmom):
        eh = (eps[:nocc, None] - Om[None, :]) ** n
        ep = (eps[nocc:, None] + Om[None, :]) ** n
        sh[n] = np.einsum("pkn,qkn,kn->pq", w[:, :nocc], w[:, :nocc], eh)
        sp[n] = np.einsum("pcn,qcn,cn->pq", w[:, nocc:], w[:, nocc:], ep)
    assert nvir > 0
    return sh, sp


def exact_upfolded(eps, L, nocc, screening="tda"):
    """Exact (all poles) upfolded GW Hamiltonian: the physical block diag(eps)
    coupled to every pole eps_k - Omega_nu (hole) and eps_c + Omega_nu
    (particle) with residues w (the infinite-moment limit of Eq. 9)."""
    Om, w = poles_and_residues(eps, L, nocc, screening)
    nmo = eps.size
    nov = Om.size
    Wh = w[:, :nocc, :].reshape(nmo, -1)
    Wp = w[:, nocc:, :].reshape(nmo, -1)
    dh = (eps[:nocc, None] - Om[None, :]).ravel()
    dp = (eps[nocc:, None] + Om[None, :]).ravel()
    dim = nmo + dh.size + dp.size
    H = np.zeros((dim, dim))
    H[:nmo, :nmo] = np.diag(eps)
    H[:nmo, nmo:nmo + dh.size] = Wh
    H[:nmo, nmo + dh.size:] = Wp
    H[nmo:, :nmo] = H[:nmo, nmo:].T
    H[nmo:nmo + dh.size, nmo:nmo + dh.size] = np.diag(dh)
    H[nmo + dh.size:, nmo + dh.size:] = np.diag(dp)
    assert nov == (nmo - nocc) * nocc
    return H


def block_tridiagonal(alpha, beta):
    nb, r = alpha.shape[0], alpha.shape[1]
    T = np.zeros((nb * r, nb * r))
    for i in range(nb):
        T[i * r:(i + 1) * r, i * r:(i + 1) * r] = alpha[i]
        if i + 1 < nb:
            T[(i + 1) * r:(i + 2) * r, i * r:(i + 1) * r] = beta[i]
            T[i * r:(i + 1) * r, (i + 1) * r:(i + 2) * r] = beta[i].T
    return T


def spectral_downfolded(H, nmo, omega, delta):
    """A(w) = -(1/pi) Im tr G(w + i delta) with G of the physical block by
    downfolding H~ (Eq. 10): G(z) = [z - f - W~ (z - d~)^-1 W~^T]^-1, solved
    with dense complex linear algebra, no eigendecomposition."""
    f, Wt, dt = H[:nmo, :nmo], H[:nmo, nmo:], H[nmo:, nmo:]
    out = []
    for w in np.atleast_1d(omega):
        z = complex(w, delta)
        sig = Wt @ np.linalg.solve(z * np.eye(dt.shape[0]) - dt, Wt.T)
        G = np.linalg.inv(z * np.eye(nmo) - f - sig)
        out.append(-np.trace(G).imag / np.pi)
    return np.array(out)


def naf_metric_pairs(L, nocc, pairs):
    """M_PQ of Eq. 14 by an explicit loop over orbital pairs (v, w), skipping
    the virtual-virtual block unless pairs == 'full'."""
    naux, nmo, _ = L.shape
    M = np.zeros((naux, naux))
    for v in range(nmo):
        for w in range(nmo):
            if pairs != "full" and v >= nocc and w >= nocc:
                continue
            col = L[:, v, w]
            M += np.outer(col, col)
    return M


def sigma_lehmann_general(Ex, mx, Vhat, Via, D, nmom):
    """TDA self-energy moments for a Green's function with poles E_x (holes
    x < mx) and couplings V^_{Q,px}, screened over an (i, a) space with
    energy differences D and V_{Q,ia}: explicit A = D + 2 V^T V, its
    eigenpairs, residues w_{p x nu} = sqrt(2) sum_ia (px|ia) X_{ia,nu}, and
    the Lehmann sums (E_x -+ Omega_nu)^n."""
    Om, X = np.linalg.eigh(np.diag(D) + 2.0 * Via.T @ Via)
    w = np.sqrt(2.0) * np.einsum("Ppx,Pj,jn->pxn", Vhat, Via, X, optimize=True)
    nmo = Vhat.shape[1]
    sh = np.zeros((nmom, nmo, nmo))
    sp = np.zeros((nmom, nmo, nmo))
    for n in range(nmom):
        eh = (Ex[:mx, None] - Om[None, :]) ** n
        ep = (Ex[mx:, None] + Om[None, :]) ** n
        sh[n] = np.einsum("pkn,qkn,kn->pq", w[:, :mx], w[:, :mx], eh)
        sp[n] = np.einsum("pcn,qcn,cn->pq", w[:, mx:], w[:, mx:], ep)
    return sh, sp


def scgw_lehmann(orc, eps, L, nocc, nmom_max, g0, w0, iterations):
    """Algorithm 5 with every self-energy moment taken from the explicit
    Lehmann convolution (sigma_lehmann_general); the chains, H~ and the
    Aufbau filling come from the oracle module passed in.  Returns the QP
    energies of each iteration."""
    nmom, nblk, f = 2 * nmom_max + 2, nmom_max + 1, np.diag(eps)
    EG, EW, mG, mW = eps, eps, nocc, nocc
    Vhat, Via = L, L[:, :nocc, nocc:].reshape(L.shape[0], -1)
    out = []
    for _ in range(iterations):
        D = (EW[None, mW:] - EW[:mW, None]).ravel()
        sh, sp = sigma_lehmann_general(EG, mG, Vhat, Via, D, nmom)
        qp = orc.qp_solve(f, orc.block_lanczos(sh, nblk)[:3], orc.block_lanczos(sp, nblk)[:3], 2.0 * nocc)
        out.append(qp["eps_qp"])
        chi, m = qp["chi"], qp["m"]
        V2 = np.einsum("Ppq,qx->Ppx", L, chi)
        if not g0:
            EG, mG, Vhat = qp["E"], m, V2
        if not w0:
            EW, mW = qp["E"], m
            Via = np.einsum("pi,Ppa->Pia", chi[:, :m], V2[:, :, m:]).reshape(L.shape[0], -1)
    return out
