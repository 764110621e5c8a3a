"""Plain FP64 CPU oracle for the moment-conserving GW hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
runs this module; only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py use it.  It shares no code with the CUDA library: both sides
receive their inputs from mgw_inputs (which holds none of the method's
arithmetic) and nothing else.

It follows the paper (Backhouse, Allen, Scott, Booth, arXiv:2504.17439) step
by step, in its order and notation, with numpy as the only helper (matrix
products, eigh, solve).  The readings taken where the paper is silent or
garbled are listed in the docstrings that use them:

  R1  Eqs. 6-7 print W^(n) inside the sum over t; the Lehmann expansion
      (eps_k - Omega)^n = sum_t C(n,t) eps_k^(n-t) (-Omega)^t needs the t-th
      screened moment, so W^(t) is used.
  R2  Spin: for restricted orbitals the singlet pole residues carry sqrt(2),
      so Sigma(n) = 2 * sum ... with W(t) = eta~(t) V^T as in Eq. 15
      (the same factor 2 that Eqs. 21-22 put into A and B).
  R3  nmom_max = N means moments 0..2N+1 are built and conserved and the
      block tridiagonal has N+1 diagonal blocks.
  R4  Quadrature for Eqs. 24-25: Clenshaw-Curtis on x in [-1, 1] with nq+1
      points, mapped to z = a (1+x)/(1-x), a = sqrt(D_min D_max); the x = 1
      node (z = inf, integrand 0) is dropped, leaving nq nodes.  Both
      integrals use the same nodes.
  R5  Block Lanczos normalisation: symmetric (PSD) square roots for Sigma(0)
      and every beta, so the blocks are unique; inverse square roots drop
      eigenvalues below rank_tol * lambda_max (for beta, of the normalised
      residual, below rank_tol * max(lambda_max, 1); beta = 0 ends the chain).  Moments are centred by
      c = tr Sigma(1) / tr Sigma(0) and scaled by
      s = (tr M(2N) / tr M(0))^(1/2N) before the recursion (exact in
      exact arithmetic; undone on the returned blocks).
  R6  QP energy (Eq. 34): lowest alpha among the maximum weights.
  R7  Aufbau (Eq. 40, Sec. III E): m minimising |N(m) - N_elec| over the
      sorted poles, ties to the smaller m, mu = (E_{m-1} + E_m) / 2.
  R8  Sigma_inf = 0 for a canonical Hartree-Fock reference (Eq. 8).
  R10 Natural auxiliary functions (Sec. II D, Eq. 14): eps_NAF is an
      absolute threshold on the eigenvalues of M (kept: lambda > eps_NAF);
      the pair sum runs over every orbital pair but the virtual-virtual
      block by default, over all pairs for self-consistent use.
  R11 Spectral function (Eqs. 11-12): delta of Eq. 11 is a Lorentzian
      broadening, so A(w) = (1/pi) sum_a weight_a delta / ((w - E_a)^2 +
      delta^2) with weight_a = sum_p chi_pa^2.
  Q1  qsGW (Sec. III D): Eq. 36 takes the real part, so the sign attached
      to i delta in Eq. 37 does not enter V; Re Sigma_pq(w) =
      sum_l v_pl v_ql (w - e_l) / ((w - e_l)^2 + delta^2).
  Q2  Eq. 38 is printed without its sum over the decoupled poles l and
      with Sigma_pq(eps_p) on the left; it is read as the static potential
      itself, V_pq = sum_l (D_pl + D_ql) / (D_pl^2 + D_ql^2) v_pl v_ql
      (1 - exp(-(D_pl^2 + D_ql^2) s)), D_pl = eps_p - e_l (Eq. 39), already
      symmetric (the pair with D_pl = D_ql = 0 contributes its limit, 0).
  S1  scGW, Algorithm 5: the physical block of H~ stays the reference
      orbitals (f + Sigma_inf = diag(eps), R8), so the map to the
      quasi-molecular orbitals (QMOs) is the physical rows chi_px of the
      current H~'s eigenvectors; the printed accumulation chi^ <- chi^ chi is
      read as chi^ = chi (one factor, not a running product).
  S2  The occupied QMOs are the Aufbau-occupied poles of Eq. 40 (reading
      R7): the m lowest; they are the holes of Eqs. 6-7 and the i of the
      (i, a) space, the rest the particles and the a.
  S3  scGW stops when the QP energies of Eq. 34 change by less than the
      tolerance between iterations.
  Q3  Eq. 35: f[C] = h + J[rho] - K[rho]/2 with rho = 2 C_occ C_occ^T over
      the nocc lowest orbitals; V is built in the orbitals C of the GW step,
      carried to the reference basis as C V C^T and held fixed while the
      field is solved (Pulay DIIS on the commutator F rho - rho F); the
      outer loop rebuilds the moments from the new (eps, C) until the
      orbital energies change by less than the tolerance.  The qsGW energies
      are the eigenvalues of Eq. 35 (the mean-field Green's function).
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# Mean-field quantities


def energy_differences(eps: np.ndarray, nocc: int) -> np.ndarray:
    """D_{ia} = eps_a - eps_i, index ia = i*nvir + a (Eq. 20)."""
    return (eps[None, nocc:] - eps[:nocc, None]).ravel()


def particle_hole_block(L: np.ndarray, nocc: int) -> np.ndarray:
    """V_{Q,ia}: the occupied-virtual slice of the DF tensor (Algorithm 1)."""
    naux = L.shape[0]
    return np.ascontiguousarray(L[:, :nocc, nocc:]).reshape(naux, -1)


# ----------------------------------------------------------------------------
# Density-response moments eta~(n) and W(n) = eta~(n) V^T


def tda_response_moments(Lov: np.ndarray, D: np.ndarray, nmom: int, rows=None) -> np.ndarray:
    """TDA screening, Sec. II C.

    eta~(0) = V (Eq. 32); eta~(n) = eta~(n-1) (D + 2 V^T V) (Eq. 33), applied
    as eta~ D + 2 (eta~ V^T) V, the O(N_aux^2 ov) association the section
    states.  Returns W(n) = eta~(n) V^T, the aux-basis factor of Eq. 15, for
    n = 0..nmom-1 (no spin factor; see R2).  Row P of eta~(n) = V A^n
    depends on row P of V alone, so `rows` restricts P to a subset and
    returns W(n)[rows, :].
    """
    T = Lov.copy() if rows is None else Lov[np.asarray(rows)].copy()
    W = np.empty((nmom, T.shape[0], Lov.shape[0]))
    for n in range(nmom):
        W[n] = T @ Lov.T
        if n + 1 < nmom:
            T = T * D[None, :] + 2.0 * (W[n] @ Lov)
    return W


def clenshaw_curtis(n: int):
    """Clenshaw-Curtis nodes x_k = cos(k pi / n), k = 0..n, and weights on
    [-1, 1] (n even), from the closed cosine-sum form of the weights."""
    assert n % 2 == 0 and n >= 2
    k = np.arange(n + 1)
    x = np.cos(k * math.pi / n)
    w = np.empty(n + 1)
    for kk in range(n + 1):
        c = 1.0 if kk in (0, n) else 2.0
        s = 0.0
        for j in range(1, n // 2 + 1):
            b = 1.0 if j == n // 2 else 2.0
            s += b / (4.0 * j * j - 1.0) * math.cos(2.0 * j * kk * math.pi / n)
        w[kk] = c / n * (1.0 - s)
    return x, w


def quadrature_rule(nq: int, dmin: float, dmax: float):
    """Nodes z_j and weights w_j with  int_0^inf f(z) dz ~ sum_j w_j f(z_j)
    (reading R4 of the quadrature the paper defers to its ref. for Eq. 24)."""
    x, wx = clenshaw_curtis(nq)
    x, wx = x[1:], wx[1:]  # drop x = 1 (z = infinity)
    a = math.sqrt(dmin * dmax)
    z = a * (1.0 + x) / (1.0 - x)
    w = wx * 2.0 * a / (1.0 - x) ** 2
    return z, w


def rpa_g_offset_exact(Lov: np.ndarray, D: np.ndarray) -> np.ndarray:
    """G_offset of Eq. 25 with its z integral done in closed form.  Element
    (P, ia) of the integrand is sum_jb (V D)_{P,jb} e^{-z D_jb} (V^T V)_{jb,ia}
    e^{-z D_ia}, and int_0^inf e^{-z (D_jb + D_ia)} dz = 1 / (D_jb + D_ia)
    (every D > 0), so
      G_offset = V D + 4 (V D) [(V^T V) o C],  C_{jb,ia} = 1 / (D_jb + D_ia)
    (a Cauchy matrix scaling V^T V elementwise)."""
    VD = Lov * D[None, :]
    C = 1.0 / (D[:, None] + D[None, :])
    return VD + 4.0 * VD @ ((Lov.T @ Lov) * C)


def rpa_eta0(Lov: np.ndarray, D: np.ndarray, nq: int, offset: str = "quadrature") -> np.ndarray:
    """RPA zeroth moment, Sec. II B, Eqs. 23-28.

    G = G_main + G_offset with
      G_main  = 1/pi int_{-inf}^{inf} z^2 Q(z) ((I + Q(z))^-1 - I) V F(z) dz
      G_offset = V D + 4 int_0^inf V D E(z) V^T V E(z) dz
      Q(z) = 4 V F(z) D V^T,  F(z) = (D^2 + z^2)^-1,  E(z) = exp(-z D),
    the G_main integrand being even in z (so 1/pi over R = 2/pi over
    [0, inf)), both by the rule of quadrature_rule (offset="exact": G_offset
    by rpa_g_offset_exact instead); then
      eta~(0) = G D^-1 (I - 4 V^T (I + 4 V D^-1 V^T)^-1 V D^-1).
    """
    if offset not in ("quadrature", "exact"):
        raise ValueError(offset)
    naux = Lov.shape[0]
    eye = np.eye(naux)
    z, w = quadrature_rule(nq, float(D.min()), float(D.max()))
    G_main = np.zeros_like(Lov)
    G_off = Lov * D[None, :]
    for zj, wj in zip(z, w):
        F = 1.0 / (D * D + zj * zj)
        Q = 4.0 * (Lov * (F * D)[None, :]) @ Lov.T
        G_main += (2.0 / math.pi) * wj * zj * zj * ((Q @ (np.linalg.inv(eye + Q) - eye)) @ (Lov * F[None, :]))
        if offset == "quadrature":
            E = np.exp(-zj * D)
            G_off += 4.0 * wj * (((Lov * (D * E)[None, :]) @ Lov.T) @ (Lov * E[None, :]))
    if offset == "exact":
        G_off = rpa_g_offset_exact(Lov, D)
    G = G_main + G_off
    GDi = G / D[None, :]
    S = eye + 4.0 * (Lov / D[None, :]) @ Lov.T
    return GDi - 4.0 * (GDi @ Lov.T) @ np.linalg.solve(S, Lov / D[None, :])


def rpa_response_moments(Lov: np.ndarray, D: np.ndarray, nmom: int, nq: int,
                         offset: str = "quadrature") -> np.ndarray:
    """RPA screening, Sec. II B: eta~(0) from Eq. 23, eta~(1) = V D (Eq. 29),
    eta~(n) = eta~(n-2) (D^2 + 4 V^T V D) (Eq. 30), applied as
    eta~ D^2 + 4 (eta~ V^T)(V D).  Returns W(n) = eta~(n) V^T."""
    naux = Lov.shape[0]
    W = np.empty((nmom, naux, naux))
    T = [rpa_eta0(Lov, D, nq, offset), Lov * D[None, :]]
    LD = Lov * D[None, :]
    for n in range(nmom):
        if n >= 2:
            T.append(T[n - 2] * (D * D)[None, :] + 4.0 * (W[n - 2] @ LD))
        W[n] = T[n] @ Lov.T
    return W


def response_moments(Lov, D, nmom, screening="tda", nq=48, offset="quadrature"):
    if screening == "tda":
        return tda_response_moments(Lov, D, nmom)
    if screening == "rpa":
        return rpa_response_moments(Lov, D, nmom, nq, offset)
    raise ValueError(screening)


# ----------------------------------------------------------------------------
# Self-energy moments (Eqs. 6-7 with Eq. 15)


def sigma_moments(eps: np.ndarray, nocc: int, L: np.ndarray, W: np.ndarray, rows=None):
    """Hole and particle self-energy moments, Eqs. 6-7 (readings R1, R2).

    For every Green's-function index x the screened moment
    W^(t)_{px,qx} = sum_PQ V_{P,px} W(t)_{PQ} V_{Q,qx} (Eq. 15) is formed
    (all x at once, one matrix product per x), then
      Sigma(n,<)_pq = 2 sum_t C(n,t) (-1)^t sum_k eps_k^(n-t) W^(t)_{pk,qk}
      Sigma(n,>)_pq = 2 sum_t C(n,t)        sum_c eps_c^(n-t) W^(t)_{pc,qc}.
    `rows` restricts p to a subset (the full q range is returned).  The
    Green's-function index x may run over a larger space than p, q (the
    quasi-molecular orbitals of scGW, Algorithm 5): L is then V^_{Q,qx}
    [naux][nmo][nx] and eps holds the nx energies eps_x, holes first.
    """
    nmom = W.shape[0]
    nmo, nx = L.shape[1], eps.size
    p_idx = np.arange(nmo) if rows is None else np.asarray(rows)
    Lx = np.ascontiguousarray(L.transpose(2, 0, 1))  # [x][Q][q] = V_{Q,qx}
    Lxp = np.ascontiguousarray(Lx[:, :, p_idx].transpose(0, 2, 1))  # [x][p][P] = V_{P,px}
    sh = np.zeros((nmom, p_idx.size, nmo))
    sp = np.zeros((nmom, p_idx.size, nmo))
    for t in range(nmom):
        Wx = (Lxp @ W[t]) @ Lx  # [x][p][q] = W^(t)_{px,qx}
        for hole, xs, out in ((True, slice(0, nocc), sh), (False, slice(nocc, nx), sp)):
            sign = -1.0 if hole else 1.0
            for n in range(t, nmom):
                wgt = 2.0 * math.comb(n, t) * sign**t * eps[xs] ** (n - t)
                out[n] += np.tensordot(wgt, Wx[xs], axes=1)
    return sh, sp


# ----------------------------------------------------------------------------
# Block Lanczos from moments (the upfolded effective Hamiltonian of Eq. 9)


def _psd_sqrt(S, rank_tol, floor=0.0):
    """Symmetric square root and pseudo-inverse square root of a symmetric
    PSD matrix, dropping eigenvalues below rank_tol * max(lambda_max, floor)."""
    lam, U = np.linalg.eigh(0.5 * (S + S.T))
    lmax = max(lam.max(), 0.0, floor) if lam.size else 0.0
    keep = lam > rank_tol * lmax if lmax > 0 else np.zeros_like(lam, dtype=bool)
    r = int(keep.sum())
    lk, Uk = lam[keep], U[:, keep]
    sq = (Uk * np.sqrt(lk)) @ Uk.T
    isq = (Uk / np.sqrt(lk)) @ Uk.T
    return sq, isq, r, Uk, lk


def block_lanczos(sig: np.ndarray, nblk: int, rank_tol: float = 1e-12):
    """Block tridiagonal representation of one sector of the self-energy.

    Given Sigma(n), n = 0..2 nblk - 1, return the coupling S0^(1/2),
    diagonal blocks alpha_0..alpha_{nblk-1} and off-diagonal blocks
    beta_1..beta_{nblk-1} of T with Sigma(n) = S0^(1/2) (T^n)_{00} S0^(1/2)
    (the moment-conserving upfolding of Eqs. 9-10; block Lanczos three-term
    recurrence run on inner products that are moments, reading R5).

    The Lanczos vectors are kept as coefficient lists Q_i = sum_k H^k Q_0
    C_{i,k}, so <Q_i, H^m Q_j> = sum_kl C_{i,k}^T S^(k+l+m) C_{j,l}.
    Returns (coup, alpha[nblk], beta[nblk-1], rank); blocks are nmo x nmo
    when Sigma(0) is full rank, rank x rank otherwise.
    """
    nmom, nmo = sig.shape[0], sig.shape[1]
    assert nmom >= 2 * nblk
    sig = 0.5 * (sig + np.transpose(sig, (0, 2, 1)))
    # centre and scale (R5)
    tr0 = np.trace(sig[0])
    c = np.trace(sig[1]) / tr0 if tr0 > 0 else 0.0
    M = np.zeros_like(sig[: 2 * nblk])
    for n in range(2 * nblk):
        for k in range(n + 1):
            M[n] += math.comb(n, k) * (-c) ** (n - k) * sig[k]
    top = 2 * nblk - 2
    s = 1.0
    if top > 0 and tr0 > 0 and np.trace(M[top]) > 0:
        s = (np.trace(M[top]) / np.trace(M[0])) ** (1.0 / top)
    sq0, _, r, Ur, lr = _psd_sqrt(M[0], rank_tol)
    if r == 0:  # no coupling at all: an empty chain
        return np.zeros((nmo, 0)), np.zeros((nblk, 0, 0)), np.zeros((nblk - 1, 0, 0)), 0
    full = r == nmo
    P = Ur / np.sqrt(lr)[None, :]  # nmo x r
    Sh = np.stack([P.T @ (M[n] / s**n) @ P for n in range(2 * nblk)])  # r x r

    def inner(X, Y, m):
        acc = np.zeros((r, r))
        for k, Xk in enumerate(X):
            for l, Yl in enumerate(Y):
                acc += Xk.T @ Sh[k + l + m] @ Yl
        return acc

    eye = np.eye(r)
    C = [[eye]]
    alpha, beta = [], []
    for i in range(nblk):
        a = inner(C[i], C[i], 1)
        a = 0.5 * (a + a.T)
        alpha.append(a)
        if i == nblk - 1:
            break
        R = []
        for k in range(i + 2):
            Rk = np.zeros((r, r))
            if k >= 1:
                Rk += C[i][k - 1]
            if k <= i:
                Rk -= C[i][k] @ a
            if i >= 1 and k <= i - 1:
                Rk -= C[i - 1][k] @ beta[i - 1].T
            R.append(Rk)
        RR = inner(R, R, 0)
        # the residual lives in the normalised, unit-scaled problem, so its rank is
        # judged against max(lambda_max, 1): a vanishing residual (every pole
        # already represented) gives beta = 0 and a decoupled remainder
        b, binv, _, _, _ = _psd_sqrt(RR, rank_tol, floor=1.0)
        beta.append(b)
        C.append([Rk @ binv for Rk in R])
    alpha = [s * a + c * eye for a in alpha]
    beta = [s * b for b in beta]
    if full:
        # rotate every block from the eigenbasis of Sigma(0) to the orbital basis
        U = Ur
        alpha = [U @ a @ U.T for a in alpha]
        beta = [U @ b @ U.T for b in beta]
        coup = sq0
    else:
        coup = Ur * np.sqrt(lr)[None, :]
    return coup, np.array(alpha), np.array(beta).reshape(-1, r, r), r


# ----------------------------------------------------------------------------
# Upfolded Hamiltonian, QP energies, Aufbau


def upfolded_hamiltonian(fock, hole, part, zeta: float = 0.0):
    """H~ of Eq. 9: [[f + Sigma_inf, W~], [W~^T, d~ + zeta]] with
    W~ = [coup_h, 0, .., coup_p, 0, ..] and d~ = blockdiag(T_h, T_p), each T
    block tridiagonal (alpha on the diagonal, beta below, beta^T above).
    Block order: physical | hole chain | particle chain."""
    nmo = fock.shape[0]
    blocks = []
    for coup, alpha, beta in (hole, part):
        r = alpha.shape[1]
        blocks.append((coup, alpha, beta, r))
    dim = nmo + sum(b[1].shape[0] * b[3] for b in blocks)
    H = np.zeros((dim, dim))
    H[:nmo, :nmo] = fock
    off = nmo
    for coup, alpha, beta, r in blocks:
        nb = alpha.shape[0]
        H[:nmo, off : off + r] = coup
        H[off : off + r, :nmo] = coup.T
        for i in range(nb):
            o = off + i * r
            H[o : o + r, o : o + r] = alpha[i] + zeta * np.eye(r)
            if i + 1 < nb:
                H[o + r : o + 2 * r, o : o + r] = beta[i]
                H[o : o + r, o + r : o + 2 * r] = beta[i].T
        off += nb * r
    return H


def qp_energies(E: np.ndarray, chi_phys: np.ndarray) -> np.ndarray:
    """Eq. 34: eps_p^QP = E_alpha, alpha = argmax_beta |chi_{p beta}|^2
    (ties to the lowest alpha, R6)."""
    return E[np.argmax(chi_phys**2, axis=1)]


def aufbau(E: np.ndarray, weight: np.ndarray, nelec: float):
    """Aufbau filling (Eq. 40, Sec. III E, reading R7).  E ascending.
    Returns (m, mu, N(m)) with N(m) = 2 sum_{alpha < m} weight_alpha."""
    Ncum = np.concatenate([[0.0], 2.0 * np.cumsum(weight)])
    err = np.abs(Ncum - nelec)
    m = int(np.argmin(err))
    if m == 0:
        mu = E[0] - 1.0
    elif m == E.size:
        mu = E[-1] + 1.0
    else:
        mu = 0.5 * (E[m - 1] + E[m])
    return m, mu, Ncum[m]


def qp_solve(fock, hole, part, nelec: float, zeta: float = 0.0):
    """Diagonalise H~ (Eq. 9), form G's poles (Eq. 11), QP energies (Eq. 34)
    and the Aufbau chemical potential and density (Eq. 40)."""
    nmo = fock.shape[0]
    H = upfolded_hamiltonian(fock, hole, part, zeta)
    E, X = np.linalg.eigh(H)
    chi = X[:nmo]
    weight = np.sum(chi**2, axis=0)
    eqp = qp_energies(E, chi)
    m, mu, n_out = aufbau(E, weight, nelec)
    rho = 2.0 * chi[:, :m] @ chi[:, :m].T
    return dict(E=E, chi=chi, weight=weight, eps_qp=eqp, mu=mu, nelec=n_out, m=m, rho=rho)


# ----------------------------------------------------------------------------
# Spectral function (Eqs. 11-12)


def spectral_function(E: np.ndarray, weight: np.ndarray, omega, delta: float) -> np.ndarray:
    """A(w) of Eq. 12 from the Lehmann form of G in Eq. 11 (reading R11):
    Im G_pp(w) = -sum_a chi_pa^2 delta / ((w - E_a)^2 + delta^2), so
    A(w) = (1/pi) sum_a weight_a delta / ((w - E_a)^2 + delta^2)."""
    w = np.asarray(omega, dtype=float)
    A = np.zeros(w.shape)
    for Ea, wa in zip(E, weight):
        A += wa * delta / ((w - Ea) ** 2 + delta * delta)
    return A / math.pi


# ----------------------------------------------------------------------------
# Natural auxiliary functions (Sec. II D, Eq. 14)


def naf_pairs(nmo: int, nocc: int, pairs: str = "no_vv") -> np.ndarray:
    """Mask of the orbital pairs (v, w) summed in Eq. 14: all of them, or
    (the paper's default outside self-consistency) all but virtual-virtual."""
    mask = np.ones((nmo, nmo), dtype=bool)
    if pairs == "no_vv":
        mask[nocc:, nocc:] = False
    elif pairs != "full":
        raise ValueError(f"unknown pair space {pairs!r}")
    return mask


def naf_basis(L: np.ndarray, nocc: int, eps_naf: float = 1e-5, pairs: str = "no_vv"):
    """Eq. 14: M_PQ = sum_vw V_{P,vw} V_{Q,vw} over the chosen pairs; its
    eigenvectors with eigenvalue above eps_naf (absolute, reading R10) span
    the natural auxiliary functions.  Returns (U [naux][n_naf], all
    eigenvalues of M in descending order)."""
    naux, nmo, _ = L.shape
    V = L[:, naf_pairs(nmo, nocc, pairs)]
    M = V @ V.T
    lam, U = np.linalg.eigh(M)
    lam, U = lam[::-1], U[:, ::-1]
    return U[:, lam > eps_naf], lam


def naf_compress(L: np.ndarray, nocc: int, eps_naf: float = 1e-5, pairs: str = "no_vv") -> np.ndarray:
    """The DF tensor in the NAF basis, L'_{A,pq} = sum_P U_{PA} L_{P,pq}
    (Sec. II D): every later step runs with N_NAF functions for N_aux."""
    U, _ = naf_basis(L, nocc, eps_naf, pairs)
    return np.tensordot(U.T, L, axes=1)


# ----------------------------------------------------------------------------
# Input rounding of the mixed-precision mode (not in the paper)


def fixed_point_grid(X, bits=16, ref_max=None):
    """X rounded to one fixed-point grid for the whole tensor: with e the
    exponent for which max |X| < 2^(e-1) (e = floor(log2 max|X|) + 2), every
    element becomes the nearest multiple of 2^(e-bits), ties away from zero.
    This is the tensor the mixed-precision mode contracts in place of X (its
    two BF16 digits hold exactly these values); the method's moments are then
    computed for it without further rounding.  ref_max (default max |X|)
    sets the grid, so a part of a tensor can be rounded on the whole tensor's
    grid.  Not in the paper: the paper's arithmetic is FP64 throughout."""
    X = np.asarray(X, dtype=np.float64)
    m = ref_max if ref_max is not None else (float(np.abs(X).max()) if X.size else 0.0)
    if m == 0.0:
        return X.copy()
    e = math.frexp(m)[1] + 1  # m = f 2^k with 1/2 <= f < 1: floor(log2 m) = k - 1
    unit = math.ldexp(1.0, e - bits)
    return np.sign(X) * np.floor(np.abs(X) / unit + 0.5) * unit


# ----------------------------------------------------------------------------
# Drivers


def g0w0(eps, L, nocc, nmom_max, screening="tda", nq=48, eps_w=None, rank_tol=1e-12, fock=None):
    """One-shot G0W0, Algorithm 1 (Sigma_inf = 0, f = diag(eps), R8).
    eps is eps^G; eps_w (default eps) defines D for the screening; fock
    (default diag(eps)) is the physical block of H~."""
    nmo = eps.size
    nmom = 2 * nmom_max + 2
    nblk = nmom_max + 1
    epsw = eps if eps_w is None else eps_w
    D = energy_differences(epsw, nocc)
    Lov = particle_hole_block(L, nocc)
    W = response_moments(Lov, D, nmom, screening, nq)
    sh, sp = sigma_moments(eps, nocc, L, W)
    hole = block_lanczos(sh, nblk, rank_tol)
    part = block_lanczos(sp, nblk, rank_tol)
    f = np.diag(eps) if fock is None else fock
    qp = qp_solve(f, hole[:3], part[:3], 2.0 * nocc)
    return dict(W=W, sigma_hole=sh, sigma_part=sp, hole=hole, part=part, **qp)


def evgw(eps, L, nocc, nmom_max, screening="tda", nq=48, g0=False, w0=False,
         conv_e=5.0 * 3.6749322e-5, max_iter=50):
    """Eigenvalue self-consistency, Algorithm 3 / Sec. III B: eps^G and/or
    eps^W are replaced by the QP energies of Eq. 34 until they change by less
    than conv_e (5 meV by default) between iterations."""
    epsG = eps.copy()
    epsW = eps.copy()
    f = np.diag(eps)
    hist = []
    for it in range(max_iter):
        nmom = 2 * nmom_max + 2
        D = energy_differences(epsW, nocc)
        W = response_moments(particle_hole_block(L, nocc), D, nmom, screening, nq)
        sh, sp = sigma_moments(epsG, nocc, L, W)
        hole = block_lanczos(sh, nmom_max + 1)
        part = block_lanczos(sp, nmom_max + 1)
        qp = qp_solve(f, hole[:3], part[:3], 2.0 * nocc)
        e_new = qp["eps_qp"]
        dG = np.abs(e_new - epsG).max() if not g0 else 0.0
        dW = np.abs(e_new - epsW).max() if not w0 else 0.0
        hist.append(max(dG, dW))
        if not g0:
            epsG = e_new.copy()
        if not w0:
            epsW = e_new.copy()
        if max(dG, dW) < conv_e:
            return dict(eps_qp=e_new, iterations=it + 1, converged=True, history=hist)
    return dict(eps_qp=e_new, iterations=max_iter, converged=False, history=hist)


# ----------------------------------------------------------------------------
# Fock self-consistency (fsGW), Algorithm 2 / Sec. III F
#
# Readings (the paper states the loops, not their numerics):
#  F1  All static quantities live in the fixed basis of the reference
#      orbitals; the self-energy built in the current orbitals C is carried
#      there by its coupling rows: W~_ref = C W~_mo (Sigma_ref = C Sigma_mo C^T).
#  F2  F[rho] = h + J[rho] - K[rho]/2 with rho the spin-summed correlated
#      density of Eq. 40 (Tr rho = N), J_pq = sum_P L_Ppq sum_rs L_Prs rho_rs,
#      K_pq = sum_P sum_rs L_Ppr rho_rs L_Psq.
#  F3  zeta: the root of g(zeta) = N(zeta) - N (the Aufbau count of Eq. 40
#      for H~(zeta)) nearest to the current zeta.  g has many roots (each
#      change of the Aufbau filling shifts it), so the search scans outward
#      from the current zeta in steps of 0.01 Ha for the nearest sign change,
#      refines it by Illinois regula falsi (count met to 1e-10 or bracket
#      below 1e-9 Ha, at most 60 evaluations), accepts it if |g| <= 1e-6
#      (else it was a jump of the filling and the scan continues), and falls
#      back to golden section on |g| over [-1, 1] Ha if no root is found.
#  F4  Fock loop at fixed zeta: Pulay DIIS on F with error F[rho(F)] - F
#      (space 12, Sec. IV B), plain iteration for the first two steps, until
#      max |delta rho| < 1e-8 (at most 100 steps).
#  F5  Outer loop: zeta search then Fock loop, repeated (at most 20 times)
#      until the electron count and the density are both consistent; then
#      eps, C <- eigh(F); the next self-energy is built in the new orbitals.
#  F6  QP energies (Eq. 34) are assigned per orbital of the current F (its
#      eigenvectors), the basis in which Eq. 34 names the orbitals p.


def fock_build(h, L, rho):
    """F[rho] = h + J[rho] - K[rho]/2 (reading F2)."""
    J = np.einsum("Ppq,P->pq", L, np.einsum("Prs,rs->P", L, rho))
    K = np.einsum("Ppr,rs,Psq->pq", L, rho, L, optimize=True)
    return h + J - 0.5 * K


def rotate_df(L, C):
    """L'_Q = C^T L_Q C: the DF tensor in the orbitals C (Algorithm 1's
    transformed copy V^_Qpx, from the reference basis instead of AOs)."""
    return np.einsum("ap,Qab,bq->Qpq", C, L, C, optimize=True)


def zeta_search(F, hole, part, nelec, start=0.0, step=0.01, lo=-1.0, hi=1.0, tol=1e-10, accept=1e-6):
    """Reading F3.  Returns (zeta, |g(zeta)|, evaluations)."""
    count = [0]

    def g(z):
        count[0] += 1
        return qp_solve(F, hole, part, nelec, z)["nelec"] - nelec

    def refine(a, ga, b, gb):
        # Illinois regula falsi on a bracket with ga * gb < 0
        c, gc = (a, ga) if abs(ga) < abs(gb) else (b, gb)
        for _ in range(60):
            if abs(gc) <= tol or abs(b - a) < 1e-9:
                break
            c = b - gb * (b - a) / (gb - ga)
            gc = g(c)
            if gc * gb < 0:
                a, ga = b, gb
            else:
                ga *= 0.5
            b, gb = c, gc
        return c, gc

    z0 = min(max(start, lo), hi)
    g0 = g(z0)
    if abs(g0) <= tol:
        return z0, abs(g0), count[0]
    prev = {+1: (z0, g0), -1: (z0, g0)}
    k = 1
    while True:
        moved = False
        for side in (+1, -1):
            z = z0 + side * k * step
            if z < lo - 1e-12 or z > hi + 1e-12:
                continue
            moved = True
            gz = g(z)
            zp, gp = prev[side]
            prev[side] = (z, gz)
            if abs(gz) <= tol:
                return z, abs(gz), count[0]
            if gz * gp < 0:
                c, gc = refine(zp, gp, z, gz)
                if abs(gc) <= accept:
                    return c, abs(gc), count[0]
        if not moved:
            break
        k += 1
    # fallback: golden section on |g| over [lo, hi]
    r = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - r * (b - a), a + r * (b - a)
    fc, fd = abs(g(c)), abs(g(d))
    while b - a > 1e-8 and count[0] < 200 and min(fc, fd) > tol:
        if fc <= fd:
            b, d, fd = d, c, fc
            c = b - r * (b - a)
            fc = abs(g(c))
        else:
            a, c, fc = c, d, fd
            d = a + r * (b - a)
            fd = abs(g(d))
    return ((c, fc) if fc <= fd else (d, fd)) + (count[0],)


def diis_extrapolate(Fs, errs):
    """Pulay DIIS: minimise |sum_i c_i e_i| with sum_i c_i = 1."""
    n = len(Fs)
    B = np.zeros((n + 1, n + 1))
    for i in range(n):
        for j in range(n):
            B[i, j] = np.vdot(errs[i], errs[j])
    B[n, :n] = B[:n, n] = -1.0
    rhs = np.zeros(n + 1)
    rhs[n] = -1.0
    c = np.linalg.lstsq(B, rhs, rcond=None)[0][:n]
    return sum(ci * Fi for ci, Fi in zip(c, Fs))


def fock_loop(h, L, F, hole, part, nelec, zeta, diis_space=12, max_iter=100, tol=1e-8):
    """Reading F4.  Returns (F, rho, iterations)."""
    Fs, errs = [], []
    rho_old = None
    rho = None
    for it in range(max_iter):
        rho = qp_solve(F, hole, part, nelec, zeta)["rho"]
        Fn = fock_build(h, L, rho)
        if rho_old is not None and np.abs(rho - rho_old).max() < tol:
            return Fn, rho, it + 1
        rho_old = rho
        Fs.append(Fn)
        errs.append(Fn - F)
        Fs, errs = Fs[-diis_space:], errs[-diis_space:]
        F = Fn if it < 2 else diis_extrapolate(Fs, errs)
    return F, rho, max_iter


def fsgw(h, L, eps, nocc, nmom_max, screening="tda", nq=48, max_outer=30, conv_e=5.0 * 3.6749322e-5,
         conv_mom=1e-4, diis_space=12, F0=None):
    """Algorithm 2.  h, L in the reference orbital basis; eps the reference
    energies (F[rho_HF] = diag(eps) by the construction of h), or a starting
    Fock matrix F0 in the same basis (its eigenpairs give the first orbitals).
    Returns the converged QP energies, F, zeta and iteration counts."""
    nelec = 2.0 * nocc
    F = np.diag(eps).astype(float) if F0 is None else np.array(F0, dtype=float)
    e, C = (eps.copy(), np.eye(eps.size)) if F0 is None else np.linalg.eigh(F)
    zeta = 0.0
    prev_sig = None
    prev_qp = None
    history = []
    for outer in range(max_outer):
        Lm = rotate_df(L, C)
        nmom = 2 * nmom_max + 2
        D = energy_differences(e, nocc)
        W = response_moments(particle_hole_block(Lm, nocc), D, nmom, screening, nq)
        sh, sp = sigma_moments(e, nocc, Lm, W)
        hole = block_lanczos(sh, nmom_max + 1)
        part = block_lanczos(sp, nmom_max + 1)
        # carry the chains' coupling into the reference basis (F1)
        hole_r = (C @ hole[0], hole[1], hole[2])
        part_r = (C @ part[0], part[1], part[2])
        sig_ref = np.stack([C @ (a + b) @ C.T for a, b in zip(sh, sp)])
        inner = 0
        for rep in range(20):
            zeta, nerr, _ = zeta_search(F, hole_r, part_r, nelec, start=zeta)
            F, rho, k = fock_loop(h, L, F, hole_r, part_r, nelec, zeta, diis_space)
            inner += k
            n_now = qp_solve(F, hole_r, part_r, nelec, zeta)["nelec"]
            if abs(n_now - nelec) <= max(nerr, 1e-10) + 1e-12 and k <= 2:
                break
        e, C = np.linalg.eigh(F)
        # QP assignment in the eigenbasis of F (F6)
        qp = qp_solve(C.T @ F @ C, (C.T @ hole_r[0], hole[1], hole[2]), (C.T @ part_r[0], part[1], part[2]),
                      nelec, zeta)
        dsig = np.abs(sig_ref - prev_sig).max() if prev_sig is not None else np.inf
        dqp = np.abs(qp["eps_qp"] - prev_qp).max() if prev_qp is not None else np.inf
        history.append(dict(outer=outer, inner=inner, zeta=zeta, dsig=dsig, dqp=dqp, nelec=qp["nelec"]))
        prev_sig, prev_qp = sig_ref, qp["eps_qp"]
        if dsig < conv_mom and dqp < conv_e:
            return dict(eps_qp=qp["eps_qp"], F=F, zeta=zeta, converged=True, history=history, mu=qp["mu"])
    return dict(eps_qp=qp["eps_qp"], F=F, zeta=zeta, converged=False, history=history, mu=qp["mu"])


# ----------------------------------------------------------------------------
# Fully self-consistent GW on quasi-molecular orbitals (Sec. III E, Algorithm 5)


def qmo_tensors(L, chi, m):
    """The DF tensor distributed over the QMOs of H~ (Algorithm 5, reading
    S1): V^_{Q,px} = sum_q L_{Q,pq} chi_qx for every pole x, and
    V_{Q,ia} = sum_pq chi_pi L_{Q,pq} chi_qa over occupied i < m <= a (S2)."""
    Vhat = np.einsum("Qpq,qx->Qpx", L, chi, optimize=True)
    Via = np.einsum("pi,Qpx->Qix", chi[:, :m], Vhat[:, :, m:], optimize=True)
    return Vhat, Via.reshape(L.shape[0], -1)


def scgw(eps, L, nocc, nmom_max, screening="tda", nq=48, g0=False, w0=False, conv=1e-6, max_iter=40):
    """scGW, GW0 (w0) or G0W (g0) of Algorithm 5 with f + Sigma_inf =
    diag(eps) (R8).  Each iteration builds the response moments over the
    current (i, a) space, the self-energy moments over the current x space,
    the chains and H~, then (unless g0) moves G's space to the QMOs of H~
    with eps^G = E and (unless w0) the (i, a) space to occupied x virtual
    QMOs with eps^W = E (readings S1-S3)."""
    nelec = 2.0 * nocc
    f = np.diag(eps)
    nmom, nblk = 2 * nmom_max + 2, nmom_max + 1
    epsG, epsW, mG, mW = eps.copy(), eps.copy(), nocc, nocc
    Vhat, Via = L, particle_hole_block(L, nocc)
    prev = None
    history = []
    for it in range(max_iter):
        W = response_moments(Via, energy_differences(epsW, mW), nmom, screening, nq)
        sh, sp = sigma_moments(epsG, mG, Vhat, W)
        qp = qp_solve(f, block_lanczos(sh, nblk)[:3], block_lanczos(sp, nblk)[:3], nelec)
        d = np.abs(qp["eps_qp"] - prev).max() if prev is not None else np.inf
        history.append(dict(iteration=it, dqp=d, poles=qp["E"].size, nelec=qp["nelec"]))
        prev = qp["eps_qp"]
        if d < conv:
            return dict(qp, converged=True, history=history)
        Vq, Vq_ia = qmo_tensors(L, qp["chi"], qp["m"])
        if not g0:
            epsG, mG, Vhat = qp["E"], qp["m"], Vq
        if not w0:
            epsW, mW, Via = qp["E"], qp["m"], Vq_ia
    return dict(qp, converged=False, history=history)


# ----------------------------------------------------------------------------
# Quasiparticle self-consistent GW (Sec. III D, Eqs. 35-39)


def decoupled_poles(chain):
    """The external block of one chain, T = blocktridiag(alpha, beta), in its
    eigenbasis (Sec. III D): T = U diag(e) U^T, couplings v = [coup, 0, ..] U,
    so that this chain's part of Eq. 10 is sum_l v_pl v_ql / (w - e_l)."""
    coup, alpha, beta = chain[:3]
    nb, r = alpha.shape[0], alpha.shape[1]
    T = np.zeros((nb * r, nb * r))
    for i in range(nb):
        T[i * r : (i + 1) * r, i * r : (i + 1) * r] = alpha[i]
        if i + 1 < nb:
            T[(i + 1) * r : (i + 2) * r, i * r : (i + 1) * r] = beta[i]
            T[i * r : (i + 1) * r, (i + 1) * r : (i + 2) * r] = beta[i].T
    e, U = np.linalg.eigh(T)
    return coup @ U[:r, :], e


def qsgw_potential(eps, hole, part, reg="srg", delta=1e-3, srg_s=100.0):
    """Static potential of qsGW in the orbitals the chains were built in.
    reg = "eta": Eq. 36 with the Lorentzian-regularised poles of Eq. 37
    (reading Q1); reg = "srg": Eqs. 38-39 (reading Q2)."""
    vh, eh = decoupled_poles(hole)
    vp, ep = decoupled_poles(part)
    v = np.concatenate([vh, vp], axis=1)
    e = np.concatenate([eh, ep])
    Dl = eps[:, None] - e[None, :]  # D_pl of Eq. 39
    n = eps.size
    V = np.zeros((n, n))
    if reg == "eta":
        R = Dl / (Dl * Dl + delta * delta)  # Re of one Eq. 37 denominator
        A = np.einsum("pl,pl,ql->pq", R, v, v)  # A_pq = Re Sigma_pq(eps_p)
        return 0.5 * (A + A.T)
    if reg != "srg":
        raise ValueError(f"unknown regularisation {reg!r}")
    for l in range(e.size):
        d = Dl[:, l]
        s2 = d[:, None] ** 2 + d[None, :] ** 2
        with np.errstate(invalid="ignore", divide="ignore"):
            f = np.where(s2 > 0.0, (d[:, None] + d[None, :]) / s2 * (1.0 - np.exp(-s2 * srg_s)), 0.0)
        V += f * np.outer(v[:, l], v[:, l])
    return V


def qsgw_scf(h, L, Vref, C, nocc, diis_space=8, max_iter=200, tol=1e-10):
    """Eq. 35 with the static potential fixed (reading Q3): F = f[rho] + V,
    rho from the nocc lowest eigenvectors, Pulay DIIS on F rho - rho F."""
    rho = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    Fs, errs = [], []
    for it in range(max_iter):
        F = fock_build(h, L, rho) + Vref
        err = F @ rho - rho @ F
        Fs.append(F)
        errs.append(err)
        Fs, errs = Fs[-diis_space:], errs[-diis_space:]
        Fx = diis_extrapolate(Fs, errs) if len(Fs) > 2 else F
        e, C = np.linalg.eigh(Fx)
        rho_new = 2.0 * C[:, :nocc] @ C[:, :nocc].T
        drho = np.abs(rho_new - rho).max()
        rho = rho_new
        if drho < tol and np.abs(err).max() < 1e3 * tol:
            break
    F = fock_build(h, L, rho) + Vref
    e, C = np.linalg.eigh(F)
    return e, C, F, it + 1


def qsgw(h, L, eps, nocc, nmom_max, reg="srg", delta=1e-3, srg_s=100.0, screening="tda", nq=48,
         max_outer=60, conv=1e-8, C0=None):
    """Quasiparticle self-consistent GW (Sec. III D).  h, L in the reference
    orbital basis; eps and C0 the reference energies and orbitals there
    (default C0 = 1: the basis is the canonical HF one, F[rho_HF] =
    diag(eps)).  Each outer step builds the GW moments in the current
    orbitals (eps^G = eps^W = eps, L rotated to C), their block-Lanczos
    chains, the static potential (Eqs. 36-39) and then solves Eq. 35 with it
    held fixed."""
    e = eps.astype(float).copy()
    C = np.eye(eps.size) if C0 is None else np.array(C0, dtype=float)
    nmom, nblk = 2 * nmom_max + 2, nmom_max + 1
    history = []
    for outer in range(max_outer):
        Lm = rotate_df(L, C)
        W = response_moments(particle_hole_block(Lm, nocc), energy_differences(e, nocc), nmom, screening, nq)
        sh, sp = sigma_moments(e, nocc, Lm, W)
        V = qsgw_potential(e, block_lanczos(sh, nblk), block_lanczos(sp, nblk), reg, delta, srg_s)
        Vref = C @ V @ C.T
        e_new, C, F, k = qsgw_scf(h, L, Vref, C, nocc)
        de = np.abs(e_new - e).max()
        e = e_new
        history.append(dict(outer=outer, de=de, scf_iter=k))
        if de < conv:
            return dict(eps=e, C=C, F=F, V=Vref, converged=True, history=history)
    return dict(eps=e, C=C, F=F, V=Vref, converged=False, history=history)


def hf_core_hamiltonian(eps, L, nocc):
    """h = diag(eps) - J[rho_HF] + K[rho_HF]/2 so that F[rho_HF] = diag(eps)
    (the synthetic reference is a canonical Hartree-Fock state)."""
    rho = np.zeros((eps.size, eps.size))
    rho[np.arange(nocc), np.arange(nocc)] = 2.0
    return np.diag(eps) - (fock_build(np.zeros_like(rho), L, rho))
