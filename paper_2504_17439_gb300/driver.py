"""Host-side composition of the library calls: one-shot G0W0 (Algorithm 1)
and eigenvalue self-consistency (evGW, Algorithm 3).

Every numerical step runs in libmgw through the binding in mgw.py; this
module only sequences the calls and moves a few scalars.
"""
from __future__ import annotations

import torch

from . import mgw


def g0w0(h: mgw.Handle, eps_G: torch.Tensor, L: torch.Tensor, nocc: int, nmom_max: int,
         screening: int = mgw.MGW_TDA, eps_W: torch.Tensor | None = None, fock: torch.Tensor | None = None,
         opts: mgw.Options | None = None, Lov: torch.Tensor | None = None, want_chi: bool = False,
         naf_eps: float | None = None, naf_all_pairs: bool = False) -> dict:
    """Response moments -> W -> Sigma(n,<), Sigma(n,>) -> block Lanczos per
    sector -> H~ eigensolve, QP energies, Aufbau.  All tensors on the GPU.
    With naf_eps, L is first compressed to its natural auxiliary functions
    (Sec. II D, Eq. 14: eigenvalues of the pair metric above naf_eps) and
    every later step runs on n_naf instead of naux auxiliary functions."""
    n_naf = None
    if naf_eps is not None:
        L, _ = h.mgw_naf_compress(nocc, L, naf_eps, naf_all_pairs)
        n_naf = L.shape[0]
        Lov = None
    naux, nmo = L.shape[0], L.shape[1]
    nvir = nmo - nocc
    nmom = 2 * nmom_max + 2
    nblk = nmom_max + 1
    o = opts if opts is not None else mgw.options()
    o.screening = screening
    if Lov is None:
        Lov = h.mgw_extract_ov(nocc, nvir, L)
    Wmom = h.mgw_response_moments(o, nocc, nvir, naux, nmom, eps_G if eps_W is None else eps_W, Lov)
    sh, sp = h.mgw_sigma_moments(o, nocc, nvir, naux, nmom, eps_G, L, Wmom)
    ch, ah, bh, rh = h.mgw_block_lanczos(o, nmo, nmom, sh)
    cp, ap, bp, rp = h.mgw_block_lanczos(o, nmo, nmom, sp)
    f = torch.diag(eps_G) if fock is None else fock
    qp = h.mgw_qp_solve(o, nmo, nblk, rh, rp, f.contiguous(), (ch, ah, bh), (cp, ap, bp), 0.0, 2.0 * nocc,
                        want_chi=want_chi)
    return dict(W=Wmom, sigma_hole=sh, sigma_part=sp, hole=(ch, ah, bh, rh), part=(cp, ap, bp, rp), n_naf=n_naf,
                **qp)


def evgw(h: mgw.Handle, eps: torch.Tensor, L: torch.Tensor, nocc: int, nmom_max: int,
         screening: int = mgw.MGW_TDA, g0: bool = False, w0: bool = False, conv_e: float | None = None,
         max_iter: int | None = None, opts: mgw.Options | None = None) -> dict:
    """Eigenvalue self-consistency (Sec. III B): eps^G and/or eps^W take the
    QP energies of Eq. 34 until they change by less than conv_e."""
    o = opts if opts is not None else mgw.options()
    conv = o.conv_e if conv_e is None else conv_e
    iters = o.max_iter if max_iter is None else max_iter
    nvir = L.shape[1] - nocc
    Lov = h.mgw_extract_ov(nocc, nvir, L)
    fock = torch.diag(eps).contiguous()
    epsG, epsW = eps.clone(), eps.clone()
    hist = []
    for it in range(iters):
        r = g0w0(h, epsG, L, nocc, nmom_max, screening, eps_W=epsW, fock=fock, opts=o, Lov=Lov)
        e_new = r["eps_qp"]
        dG = 0.0 if g0 else float((e_new - epsG).abs().max())
        dW = 0.0 if w0 else float((e_new - epsW).abs().max())
        hist.append(max(dG, dW))
        if not g0:
            epsG = e_new.clone()
        if not w0:
            epsW = e_new.clone()
        if max(dG, dW) < conv:
            return dict(eps_qp=e_new, iterations=it + 1, converged=True, history=hist)
    return dict(eps_qp=e_new, iterations=iters, converged=False, history=hist)


def fsgw(h: mgw.Handle, hcore: torch.Tensor, L: torch.Tensor, eps: torch.Tensor, nocc: int, nmom_max: int,
         screening: int = mgw.MGW_TDA, opts: mgw.Options | None = None, conv_e: float | None = None,
         conv_mom: float | None = None, max_outer: int = 30, F0: torch.Tensor | None = None,
         warm: "WarmStart | None" = None, warm_fock: "WarmStart | None" = None) -> dict:
    """Fock self-consistency (Algorithm 2): mgw_fsgw_step until the
    reference-basis moments and the QP energies stop changing.  `warm` (a
    trained WarmStart) predicts the first zeta of every step; `warm_fock`
    predicts the step beta of the Fock-matrix proposal F + beta (F - F_prev)
    that the step's DIIS loop starts from.  The history records the features
    and targets of both that every step produced."""
    o = opts if opts is not None else mgw.options()
    o.screening = screening
    ce = o.conv_e if conv_e is None else conv_e
    cm = o.conv_mom if conv_mom is None else conv_mom
    naux, nmo = L.shape[0], L.shape[1]
    nmom = 2 * nmom_max + 2
    dev = L.device
    # the step reads raw pointers: dense row-major float64 on the device
    for name, t in (("hcore", hcore), ("L", L), ("eps", eps)):
        if not t.is_cuda or t.dtype != torch.float64:
            raise ValueError(f"{name} must be a float64 CUDA tensor")
    hcore, L, eps = hcore.contiguous(), L.contiguous(), eps.contiguous()
    # canonical reference: F = diag(eps), C = I; otherwise the first step takes
    # the orbitals of F0 itself (init = 1)
    F = torch.diag(eps).contiguous() if F0 is None else F0.clone().contiguous()
    C = torch.eye(nmo, dtype=torch.float64, device=dev)
    e = eps.clone()
    eps_qp = torch.empty(nmo, dtype=torch.float64, device=dev)
    sig = torch.empty((nmom, nmo, nmo), dtype=torch.float64, device=dev)
    st = mgw.FsgwState(nocc, nmo - nocc, naux, nmom_max, hcore.data_ptr(), L.data_ptr(), F.data_ptr(),
                       C.data_ptr(), e.data_ptr(), eps_qp.data_ptr(), sig.data_ptr(), 0.0, 0.0, 0.0, 0, 0,
                       0 if F0 is None else 1)
    if warm is not None:
        st.ws_params = warm.params.data_ptr()
        st.ws_wbf16 = warm.wbf16.data_ptr()
        st.ws_width = warm.width
    F_prev = torch.empty_like(F)
    st.F_prev = F_prev.data_ptr()
    st.fock_hist = 0
    if warm_fock is not None:
        st.wf_params = warm_fock.params.data_ptr()
        st.wf_wbf16 = warm_fock.wbf16.data_ptr()
        st.wf_width = warm_fock.width
    prev_sig = prev_qp = None
    hist = []
    for outer in range(max_outer):
        h.mgw_fsgw_step(o, st)
        dsig = float((sig - prev_sig).abs().max()) if prev_sig is not None else float("inf")
        dqp = float((eps_qp - prev_qp).abs().max()) if prev_qp is not None else float("inf")
        hist.append(dict(outer=outer, inner=st.inner_iters, zeta=st.zeta, dsig=dsig, dqp=dqp, nelec=st.nelec,
                         zeta_evals=st.zeta_evals, feat=list(st.ws_feat), target=st.ws_target, hit=st.ws_hit,
                         fock_feat=list(st.wf_feat), fock_target=st.wf_target, fock_beta=st.wf_beta,
                         fock_valid=outer > 0))
        prev_sig, prev_qp = sig.clone(), eps_qp.clone()
        if dsig < cm and dqp < ce:
            return dict(eps_qp=eps_qp, F=F, zeta=st.zeta, mu=st.mu, converged=True, history=hist)
    return dict(eps_qp=eps_qp, F=F, zeta=st.zeta, mu=st.mu, converged=False, history=hist)


def scgw(h: mgw.Handle, eps: torch.Tensor, L: torch.Tensor, nocc: int, nmom_max: int,
         screening: int = mgw.MGW_TDA, g0: bool = False, w0: bool = False, conv: float = 1e-6,
         max_iter: int = 40, opts: mgw.Options | None = None) -> dict:
    """scGW, GW0 (w0) and G0W (g0), Algorithm 5 (readings S1-S3): each
    iteration builds the response moments over the current (i, a) space, the
    self-energy moments over the current Green's-function space, both chains
    and H~ (f + Sigma_inf = diag(eps)); then (unless g0) G moves to the QMOs
    of H~ with eps^G = E, and (unless w0) the (i, a) space to occupied x
    virtual QMOs with eps^W = E, until the QP energies change by less than
    conv."""
    o = opts if opts is not None else mgw.options()
    o.screening = screening
    naux, nmo = L.shape[0], L.shape[1]
    nmom, nblk = 2 * nmom_max + 2, nmom_max + 1
    fock = torch.diag(eps).contiguous()
    epsG, epsW, mG, mW = eps.clone(), eps.clone(), nocc, nocc
    Lx = L.contiguous()                        # x-major: the orbitals' slabs are symmetric
    Via = h.mgw_extract_ov(nocc, nmo - nocc, L)
    prev, hist = None, []
    for it in range(max_iter):
        nxW = epsW.shape[0]
        W = h.mgw_response_moments(o, mW, nxW - mW, naux, nmom, epsW, Via.contiguous())
        sh, sp = h.mgw_sigma_moments_x(o, nmo, epsG.shape[0], mG, naux, nmom, epsG.contiguous(), Lx, W)
        ch, ah, bh, rh = h.mgw_block_lanczos(o, nmo, nmom, sh)
        cp, ap, bp, rp = h.mgw_block_lanczos(o, nmo, nmom, sp)
        qp = h.mgw_qp_solve(o, nmo, nblk, rh, rp, fock, (ch, ah, bh), (cp, ap, bp), 0.0, 2.0 * nocc,
                            want_chi=True)
        d = float((qp["eps_qp"] - prev).abs().max()) if prev is not None else float("inf")
        hist.append(dict(iteration=it, dqp=d, poles=qp["E"].shape[0], nelec=qp["nelec"]))
        prev = qp["eps_qp"]
        if d < conv:
            return dict(qp, converged=True, history=hist)
        Lt, Vq = h.mgw_qmo_tensors(L, qp["chi"].contiguous(), qp["m"])
        if not g0:
            epsG, mG, Lx = qp["E"], qp["m"], Lt
        if not w0:
            epsW, mW, Via = qp["E"], qp["m"], Vq
    return dict(qp, converged=False, history=hist)


def qsgw(h: mgw.Handle, hcore: torch.Tensor, L: torch.Tensor, eps: torch.Tensor, nocc: int, nmom_max: int,
         reg: str = "srg", delta: float = 1e-3, srg_s: float = 100.0, screening: int = mgw.MGW_TDA,
         opts: mgw.Options | None = None, conv: float = 1e-8, max_outer: int = 60, diis_space: int = 8,
         scf_tol: float = 1e-10, scf_max_iter: int = 200) -> dict:
    """Quasiparticle self-consistent GW (Sec. III D): mgw_qsgw_step until the
    orbital energies change by less than `conv` between outer steps.  hcore
    and L in the reference basis, eps the reference energies (a canonical
    Hartree-Fock reference: C starts as the identity)."""
    o = opts if opts is not None else mgw.options()
    o.screening = screening
    naux, nmo = L.shape[0], L.shape[1]
    dev = L.device
    for name, t in (("hcore", hcore), ("L", L), ("eps", eps)):
        if not t.is_cuda or t.dtype != torch.float64:
            raise ValueError(f"{name} must be a float64 CUDA tensor")
    hcore, L = hcore.contiguous(), L.contiguous()
    C = torch.eye(nmo, dtype=torch.float64, device=dev)
    e = eps.clone().contiguous()
    F = torch.empty((nmo, nmo), dtype=torch.float64, device=dev)
    V = torch.empty_like(F)
    st = mgw.QsgwState(nocc, nmo - nocc, naux, nmom_max, hcore.data_ptr(), L.data_ptr(), C.data_ptr(), e.data_ptr(),
                       F.data_ptr(), V.data_ptr(), {"eta": 0, "srg": 1}[reg], delta, srg_s, diis_space, scf_max_iter,
                       scf_tol)
    hist = []
    for outer in range(max_outer):
        h.mgw_qsgw_step(o, st)
        hist.append(dict(outer=outer, de=st.de, scf_iter=st.scf_iters, scf_converged=bool(st.scf_converged)))
        if st.de < conv:
            return dict(eps=e, C=C, F=F, V=V, converged=True, history=hist)
    return dict(eps=e, C=C, F=F, V=V, converged=False, history=hist)


class WarmStart:
    """The learned warm start of the fsGW zeta search: a 3-layer SiLU network
    (BF16 weights, FP32 accumulation) trained on (features, zeta - zeta_prev)
    pairs that plain fsGW runs record, with the library's own kernels."""

    def __init__(self, h: mgw.Handle, width: int = 256, seed: int = 0, device="cuda"):
        self.h = h
        self.width = width
        self.dims = (mgw.WS_FEATURES, width, 1)
        n = h.mgw_mlp_nparams(*self.dims)
        g = torch.Generator(device="cpu").manual_seed(seed)
        parts = []
        for rows, cols in ((width, mgw.WS_FEATURES), (width, 0), (width, width), (width, 0), (1, width), (1, 0)):
            if cols:
                parts.append(torch.randn(rows * cols, generator=g) * (1.0 / cols) ** 0.5)
            else:
                parts.append(torch.zeros(rows))
        self.params = torch.cat(parts).float().to(device).contiguous()
        assert self.params.numel() == n
        self.wbf16 = torch.empty(n, dtype=torch.bfloat16, device=device)
        h.mgw_mlp_round(self.params, self.wbf16)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.scale = 1.0

    def train(self, feats, targets, epochs: int = 400, lr: float = 1e-3, scale: float = 100.0) -> list:
        """Full-batch Adam on mean-squared error of scale * (zeta - zeta_prev)."""
        h = self.h
        self.scale = scale
        X = torch.as_tensor(feats, dtype=torch.float32, device=self.params.device).contiguous()
        T = (torch.as_tensor(targets, dtype=torch.float32, device=self.params.device) * scale).reshape(-1, 1)
        B = X.shape[0]
        acts = torch.empty((4, B, self.width), dtype=torch.float32, device=X.device)
        dY = torch.empty((B, 1), dtype=torch.float32, device=X.device)
        grad = torch.empty_like(self.params)
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        hist = []
        for _ in range(epochs):
            Y = h.mgw_mlp_forward(self.dims, self.params, self.wbf16, X, acts=acts)
            h.mgw_mlp_mse(Y, T, dY, loss)
            h.mgw_mlp_backward(self.dims, self.wbf16, X, acts, dY, grad)
            self.step += 1
            h.mgw_mlp_adam(self.params, self.wbf16, grad, self.m, self.v, self.step, lr)
            hist.append(float(loss.item()))
        # the step reads y in zeta units: fold 1/scale into the last layer
        n3 = self.width + 1
        self.params[-n3:] /= scale
        h.mgw_mlp_round(self.params, self.wbf16)
        return hist
