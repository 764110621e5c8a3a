"""Thin Python binding of libmgw (ctypes).

Argument marshalling only: every function checks tensor device, dtype, shape
and contiguity, passes raw device pointers and the handle's stream to the C
ABI of include/mgw.h, and raises MgwError on a non-zero status.  All
arithmetic runs in the library's CUDA kernels; there is no other path.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

MGW_TDA, MGW_RPA = 0, 1
MGW_FP64, MGW_BF16X3, MGW_FP64_TC, MGW_MIXED = 0, 1, 2, 3

_STATUS = {
    0: "MGW_OK", -1: "MGW_ERR_ARG", -2: "MGW_ERR_CUDA", -3: "MGW_ERR_NOMEM", -4: "MGW_ERR_NOT_PD",
    -5: "MGW_ERR_BREAKDOWN", -6: "MGW_ERR_NO_CONV", -7: "MGW_ERR_TIMEOUT", -8: "MGW_ERR_UNSUPPORTED",
}


class MgwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("screening", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("nquad", ctypes.c_int),
        ("xchunk", ctypes.c_int),
        ("rank_tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("conv_e", ctypes.c_double),
        ("conv_mom", ctypes.c_double),
        ("diis_space", ctypes.c_int),
        ("batch_graph", ctypes.c_int),
        ("batch_autotune", ctypes.c_int),
        ("rpa_offset", ctypes.c_int),
    ]


class QsgwState(ctypes.Structure):
    _fields_ = [
        ("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int), ("nmom_max", ctypes.c_int),
        ("h", ctypes.c_void_p), ("L", ctypes.c_void_p), ("C", ctypes.c_void_p), ("eps", ctypes.c_void_p),
        ("F", ctypes.c_void_p), ("V", ctypes.c_void_p), ("reg", ctypes.c_int), ("delta", ctypes.c_double),
        ("srg_s", ctypes.c_double), ("diis_space", ctypes.c_int), ("scf_max_iter", ctypes.c_int),
        ("scf_tol", ctypes.c_double), ("de", ctypes.c_double), ("scf_iters", ctypes.c_int),
        ("scf_converged", ctypes.c_int),
    ]


class FsgwState(ctypes.Structure):
    _fields_ = [
        ("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int), ("nmom_max", ctypes.c_int),
        ("h", ctypes.c_void_p), ("L", ctypes.c_void_p), ("F", ctypes.c_void_p), ("C", ctypes.c_void_p),
        ("eps", ctypes.c_void_p), ("eps_qp", ctypes.c_void_p), ("sigma_ref", ctypes.c_void_p),
        ("zeta", ctypes.c_double), ("mu", ctypes.c_double), ("nelec", ctypes.c_double),
        ("inner_iters", ctypes.c_int), ("zeta_evals", ctypes.c_int), ("init", ctypes.c_int),
        ("ws_params", ctypes.c_void_p), ("ws_wbf16", ctypes.c_void_p), ("ws_width", ctypes.c_int),
        ("ws_feat", ctypes.c_float * 8), ("ws_target", ctypes.c_double), ("ws_hit", ctypes.c_int),
        ("F_prev", ctypes.c_void_p), ("fock_hist", ctypes.c_int),
        ("wf_params", ctypes.c_void_p), ("wf_wbf16", ctypes.c_void_p), ("wf_width", ctypes.c_int),
        ("wf_feat", ctypes.c_float * 8), ("wf_target", ctypes.c_double), ("wf_beta", ctypes.c_double),
    ]

WS_FEATURES = 8


class System(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int),
                ("eps", ctypes.c_void_p), ("L", ctypes.c_void_p), ("sig_hole", ctypes.c_void_p),
                ("sig_part", ctypes.c_void_p)]


class G0w0System(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int),
                ("eps", ctypes.c_void_p), ("L", ctypes.c_void_p), ("eps_qp", ctypes.c_void_p),
                ("mu", ctypes.c_double), ("nelec", ctypes.c_double), ("rank_h", ctypes.c_int),
                ("rank_p", ctypes.c_int)]


class ResponseSystem(ctypes.Structure):
    _fields_ = [("nocc", ctypes.c_int), ("nvir", ctypes.c_int), ("naux", ctypes.c_int),
                ("eps_W", ctypes.c_void_p), ("Lov", ctypes.c_void_p), ("Wmom", ctypes.c_void_p)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> argtypes after the handle
_SIGS = {
    "mgw_extract_ov": [_I, _I, _I, _P, _P],
    "mgw_gemm_bf16x3": [_I, _I, _I, _P, _P, _P],
    "mgw_gemm_fp64_emu": [_I, _I, _I, _P, _P, _P],
    "mgw_selftest_bounded_wait": [_D],
    "mgw_gemm_mixed": [_I, _I, _I, _P, _P, _P],
    "mgw_sigma_moments_x": [_P, _I, _I, _I, _I, _I, _P, _P, _P, _P, _P],
    "mgw_qmo_tensors": [_I, _I, _I, _I, _P, _P, _P, _P],
    "mgw_df_absmax": [ctypes.c_long, _P, ctypes.POINTER(_D)],
    "mgw_df_quantize": [ctypes.c_long, _P, _I, _P, ctypes.POINTER(_I)],
    "mgw_response_moments_q": [_P, _I, _I, _I, _I, _P, _P, _I, _P],
    "mgw_sigma_moments_q": [_P, _I, _I, _I, _I, _P, _P, _I, _P, _P, _P],
    "mgw_response_moments": [_P, _I, _I, _I, _I, _P, _P, _P],
    "mgw_sigma_moments": [_P, _I, _I, _I, _I, _P, _P, _P, _P, _P],
    "mgw_block_lanczos": [_P, _I, _I, _P, _P, _P, _P, ctypes.POINTER(_I)],
    "mgw_qp_solve": [_P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _D, _D, _P, _P, _P, _P, _P,
                     ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I)],
}


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libmgw.so (built by paper_2504_17439_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmgw.so not built ({path}); run paper_2504_17439_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.mgw_options_default.argtypes = [ctypes.POINTER(Options)]
    lib.mgw_options_default.restype = None
    lib.mgw_create.argtypes = [ctypes.POINTER(_P), _I, _P]
    lib.mgw_create.restype = _I
    lib.mgw_destroy.argtypes = [_P]
    lib.mgw_destroy.restype = _I
    lib.mgw_set_stream.argtypes = [_P, _P]
    lib.mgw_set_stream.restype = _I
    lib.mgw_last_error.argtypes = [_P]
    lib.mgw_last_error.restype = ctypes.c_char_p
    lib.mgw_workspace_bytes.argtypes = [_P]
    lib.mgw_workspace_bytes.restype = ctypes.c_size_t
    lib.mgw_profile.argtypes = [_P, _I]
    lib.mgw_profile.restype = _I
    lib.mgw_profile_query.argtypes = [_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(_D)]
    lib.mgw_profile_query.restype = _I
    lib.mgw_launch_count.argtypes = [_P]
    lib.mgw_launch_count.restype = ctypes.c_long
    lib.mgw_mlp_nparams.argtypes = [_I, _I, _I]
    lib.mgw_mlp_nparams.restype = ctypes.c_long
    for nm, args in (("mgw_mlp_round", [_P, ctypes.c_long, _P, _P]),
                     ("mgw_mlp_forward", [_P, _I, _I, _I, _P, _P, _I, _P, _P, _P]),
                     ("mgw_mlp_backward", [_P, _I, _I, _I, _P, _I, _P, _P, _P, _P]),
                     ("mgw_mlp_mse", [_P, _I, _I, _P, _P, _P, _P]),
                     ("mgw_mlp_adam", [_P, ctypes.c_long, _P, _P, _P, _P, _P, _I, ctypes.c_float])):
        getattr(lib, nm).argtypes = args
        getattr(lib, nm).restype = _I
    lib.mgw_sigma_moments_batched.argtypes = [_P, _P, _I, _I, ctypes.POINTER(System)]
    lib.mgw_sigma_moments_batched.restype = _I
    lib.mgw_fsgw_step.argtypes = [_P, _P, ctypes.POINTER(FsgwState)]
    lib.mgw_fsgw_step.restype = _I
    lib.mgw_grid_exponent.argtypes = [_D]
    lib.mgw_grid_exponent.restype = _I
    lib.mgw_qsgw_step.argtypes = [_P, _P, ctypes.POINTER(QsgwState)]
    lib.mgw_qsgw_step.restype = _I
    lib.mgw_hf_core.argtypes = [_P, _I, _I, _I, _P, _P, _P]
    lib.mgw_hf_core.restype = _I
    lib.mgw_g0w0_batched.argtypes = [_P, _P, _I, _I, ctypes.POINTER(G0w0System)]
    lib.mgw_g0w0_batched.restype = _I
    lib.mgw_response_moments_batched.argtypes = [_P, _P, _I, _I, ctypes.POINTER(ResponseSystem)]
    lib.mgw_response_moments_batched.restype = _I
    lib.mgw_sync_status.argtypes = [_P]
    lib.mgw_sync_status.restype = _I
    lib.mgw_naf_compress.argtypes = [_P, _I, _I, _I, _P, _D, _I, _P, _P, ctypes.POINTER(_I)]
    lib.mgw_naf_compress.restype = _I
    lib.mgw_spectral_function.argtypes = [_P, _I, _P, _P, _D, _I, _P, _P]
    lib.mgw_spectral_function.restype = _I
    lib.mgw_qsgw_potential.argtypes = [_P, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _I, _D, _D, _P]
    lib.mgw_qsgw_potential.restype = _I
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = [_P] + args
        fn.restype = _I
    _lib = lib
    return lib


def options(**kw) -> Options:
    o = Options()
    load().mgw_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t: torch.Tensor | None, shape=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """A libmgw handle bound to one device and the current torch stream."""

    def __init__(self, device: int | None = None, stream: torch.cuda.Stream | None = None):
        lib = load()
        self._lib = lib
        self.device = torch.cuda.current_device() if device is None else device
        stream = stream or torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib.mgw_create(ctypes.byref(h), self.device, ctypes.c_void_p(stream.cuda_stream))
        if st != 0:
            raise MgwError(st, "mgw_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mgw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        self._check(self._lib.mgw_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.mgw_workspace_bytes(self._h))

    def profile(self, enable: bool):
        self._check(self._lib.mgw_profile(self._h, 1 if enable else 0))

    def profile_query(self, name: str = "*"):
        """(launches, total milliseconds) of the recorded kernels named `name`."""
        c, t = ctypes.c_long(), ctypes.c_double()
        self._check(self._lib.mgw_profile_query(self._h, name.encode(), ctypes.byref(c), ctypes.byref(t)))
        return c.value, t.value

    @property
    def launches(self) -> int:
        return int(self._lib.mgw_launch_count(self._h))

    def _check(self, st: int):
        if st != 0:
            raise MgwError(st, (self._lib.mgw_last_error(self._h) or b"").decode())

    # -- the ABI entry points, same names ---------------------------------
    def mgw_sigma_moments_batched(self, opts: Options, nmom, systems, out=None):
        """systems: list of dicts with nocc, nvir, naux, eps, L (device tensors);
        returns [(sig_hole, sig_part)] per system.  Passing the previous result
        as `out` writes into the same tensors, so a repeated call with the same
        inputs replays the library's captured graph instead of re-capturing."""
        arr = (System * len(systems))()
        outs = []
        for i, sy in enumerate(systems):
            nmo = sy["nocc"] + sy["nvir"]
            if out is not None:
                sh, sp = out[i]
            else:
                sh = torch.empty((nmom, nmo, nmo), dtype=torch.float64, device=sy["L"].device)
                sp = torch.empty_like(sh)
            arr[i] = System(sy["nocc"], sy["nvir"], sy["naux"], _ptr(sy["eps"], (nmo,), "eps"),
                            _ptr(sy["L"], (sy["naux"], nmo, nmo), "L"), _ptr(sh), _ptr(sp))
            outs.append((sh, sp))
        self._check(self._lib.mgw_sigma_moments_batched(self._h, ctypes.byref(opts), len(systems), nmom, arr))
        return outs

    def mgw_g0w0_batched(self, opts: Options, nmom_max, systems):
        """systems: list of dicts with nocc, nvir, naux, eps, L (device tensors);
        returns per system a dict with eps_qp, mu, nelec, rank_h, rank_p."""
        arr = (G0w0System * len(systems))()
        outs = []
        for i, sy in enumerate(systems):
            nmo = sy["nocc"] + sy["nvir"]
            e = torch.empty((nmo,), dtype=torch.float64, device=sy["L"].device)
            arr[i] = G0w0System(sy["nocc"], sy["nvir"], sy["naux"], _ptr(sy["eps"], (nmo,), "eps"),
                                _ptr(sy["L"], (sy["naux"], nmo, nmo), "L"), _ptr(e), 0.0, 0.0, 0, 0)
            outs.append(e)
        self._check(self._lib.mgw_g0w0_batched(self._h, ctypes.byref(opts), len(systems), nmom_max, arr))
        return [dict(eps_qp=e, mu=arr[i].mu, nelec=arr[i].nelec, rank_h=arr[i].rank_h, rank_p=arr[i].rank_p)
                for i, e in enumerate(outs)]

    def mgw_response_moments_batched(self, opts: Options, nmom, systems):
        """systems: list of dicts with nocc, nvir, naux, eps, Lov; returns W per system."""
        arr = (ResponseSystem * len(systems))()
        outs = []
        for i, sy in enumerate(systems):
            nmo, ov = sy["nocc"] + sy["nvir"], sy["nocc"] * sy["nvir"]
            W = torch.empty((nmom, sy["naux"], sy["naux"]), dtype=torch.float64, device=sy["Lov"].device)
            arr[i] = ResponseSystem(sy["nocc"], sy["nvir"], sy["naux"], _ptr(sy["eps"], (nmo,), "eps"),
                                    _ptr(sy["Lov"], (sy["naux"], ov), "Lov"), _ptr(W))
            outs.append(W)
        self._check(self._lib.mgw_response_moments_batched(self._h, ctypes.byref(opts), len(systems), nmom, arr))
        return outs

    def mgw_sync_status(self):
        self._check(self._lib.mgw_sync_status(self._h))

    def mgw_hf_core(self, nocc, eps, L):
        """h = diag(eps) - J[rho_HF] + K[rho_HF]/2 (F[rho_HF] = diag(eps))."""
        naux, nmo = L.shape[0], L.shape[1]
        hc = torch.empty((nmo, nmo), dtype=torch.float64, device=L.device)
        self._check(self._lib.mgw_hf_core(self._h, nocc, nmo, naux, _ptr(eps, (nmo,), "eps"),
                                          _ptr(L, (naux, nmo, nmo), "L"), _ptr(hc)))
        return hc

    def mgw_naf_compress(self, nocc, L, eps_naf=1e-5, all_pairs=False):
        """Natural auxiliary functions (Sec. II D, Eq. 14).  Returns (L_naf
        [n_naf][nmo][nmo], eigenvalues of M descending [naux])."""
        naux, nmo = L.shape[0], L.shape[1]
        out = torch.empty_like(L)
        lam = torch.empty(naux, dtype=torch.float64, device=L.device)
        k = _I(0)
        self._check(self._lib.mgw_naf_compress(self._h, nocc, nmo - nocc, naux, _ptr(L, (naux, nmo, nmo), "L"),
                                               float(eps_naf), int(bool(all_pairs)), _ptr(out), _ptr(lam),
                                               ctypes.byref(k)))
        return out[: k.value], lam

    def mgw_spectral_function(self, E, weight, omega, delta):
        """A(omega) of Eq. 12 from the poles (E, weight) of H~, broadening delta."""
        dim, nw = E.shape[0], omega.shape[0]
        A = torch.empty(nw, dtype=torch.float64, device=omega.device)
        self._check(self._lib.mgw_spectral_function(self._h, dim, _ptr(E, (dim,), "E"), _ptr(weight, (dim,), "weight"),
                                                    float(delta), nw, _ptr(omega, (nw,), "omega"), _ptr(A)))
        return A

    def mgw_qsgw_potential(self, nmo, nblk, rank_h, rank_p, eps, hole, part, reg="srg", delta=1e-3, srg_s=100.0):
        """Static qsGW potential (Sec. III D, Eqs. 36-39) from the chains
        hole/part = (coup, alpha, beta) as returned by mgw_block_lanczos."""
        V = torch.empty((nmo, nmo), dtype=torch.float64, device=eps.device)
        ch, ah, bh = hole
        cp, ap, bp = part
        self._check(self._lib.mgw_qsgw_potential(self._h, nmo, nblk, rank_h, rank_p, _ptr(eps, (nmo,), "eps"),
                                                 _ptr(ch), _ptr(ah), _ptr(bh), _ptr(cp), _ptr(ap), _ptr(bp),
                                                 0 if reg == "eta" else 1, float(delta), float(srg_s), _ptr(V)))
        return V

    # -- warm-start network -------------------------------------------------
    def _fptr(self, t, name):
        if t is None:
            return None
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.dtype not in (torch.float32, torch.bfloat16):
            raise ValueError(f"{name} must be float32 or bfloat16")
        return ctypes.c_void_p(t.data_ptr())

    def mgw_mlp_nparams(self, d_in, width, d_out):
        return int(self._lib.mgw_mlp_nparams(d_in, width, d_out))

    def mgw_mlp_round(self, params, wbf16):
        self._check(self._lib.mgw_mlp_round(self._h, params.numel(), self._fptr(params, "params"),
                                            self._fptr(wbf16, "wbf16")))

    def mgw_mlp_forward(self, dims, params, wbf16, X, Y=None, acts=None):
        d_in, width, d_out = dims
        B = X.shape[0]
        Y = Y if Y is not None else torch.empty((B, d_out), dtype=torch.float32, device=X.device)
        self._check(self._lib.mgw_mlp_forward(self._h, d_in, width, d_out, self._fptr(params, "params"),
                                              self._fptr(wbf16, "wbf16"), B, self._fptr(X, "X"),
                                              self._fptr(Y, "Y"), self._fptr(acts, "acts")))
        return Y

    def mgw_mlp_backward(self, dims, wbf16, X, acts, dY, grad):
        d_in, width, d_out = dims
        self._check(self._lib.mgw_mlp_backward(self._h, d_in, width, d_out, self._fptr(wbf16, "wbf16"), X.shape[0],
                                               self._fptr(X, "X"), self._fptr(acts, "acts"), self._fptr(dY, "dY"),
                                               self._fptr(grad, "grad")))
        return grad

    def mgw_mlp_mse(self, Y, T, dY, loss):
        self._check(self._lib.mgw_mlp_mse(self._h, Y.shape[0], Y.shape[1], self._fptr(Y, "Y"), self._fptr(T, "T"),
                                          self._fptr(dY, "dY"), self._fptr(loss, "loss")))

    def mgw_mlp_adam(self, params, wbf16, grad, m, v, step, lr):
        self._check(self._lib.mgw_mlp_adam(self._h, params.numel(), self._fptr(params, "params"),
                                           self._fptr(wbf16, "wbf16"), self._fptr(grad, "grad"),
                                           self._fptr(m, "m"), self._fptr(v, "v"), step, float(lr)))

    def mgw_qsgw_step(self, opts: Options, st: QsgwState):
        self._check(self._lib.mgw_qsgw_step(self._h, ctypes.byref(opts), ctypes.byref(st)))
        return st

    def mgw_fsgw_step(self, opts: Options, st: FsgwState):
        self._check(self._lib.mgw_fsgw_step(self._h, ctypes.byref(opts), ctypes.byref(st)))
        return st

    def mgw_gemm_fp64_emu(self, A, B, C=None):
        """C = A B^T to FP64 accuracy on the tensor cores (exact BF16 digit products)."""
        M, K = A.shape
        N = B.shape[0]
        C = C if C is not None else torch.empty((M, N), dtype=torch.float64, device=A.device)
        self._check(self._lib.mgw_gemm_fp64_emu(self._h, M, N, K, _ptr(A, (M, K), "A"), _ptr(B, (N, K), "B"),
                                                _ptr(C, (M, N), "C")))
        return C

    def mgw_gemm_mixed(self, A, B, C=None):
        """C = A B'^T, B' = B on its 16-bit grid (two digits), A at seven digits, every product exact."""
        M, K = A.shape
        N = B.shape[0]
        C = C if C is not None else torch.empty((M, N), dtype=torch.float64, device=A.device)
        self._check(self._lib.mgw_gemm_mixed(self._h, M, N, K, _ptr(A, (M, K), "A"), _ptr(B, (N, K), "B"),
                                             _ptr(C, (M, N), "C")))
        return C

    def mgw_sigma_moments_x(self, opts: Options, nmo, nx, nhole, naux, nmom, eps_x, Lx, Wmom):
        dev = eps_x.device
        sh = torch.empty((nmom, nmo, nmo), dtype=torch.float64, device=dev)
        sp = torch.empty_like(sh)
        self._check(self._lib.mgw_sigma_moments_x(self._h, ctypes.byref(opts), nmo, nx, nhole, naux, nmom,
                                                  _ptr(eps_x, (nx,), "eps_x"), _ptr(Lx, (naux, nx, nmo), "Lx"),
                                                  _ptr(Wmom, (nmom, naux, naux), "Wmom"), _ptr(sh), _ptr(sp)))
        return sh, sp

    def mgw_qmo_tensors(self, L, chi, m):
        """(Lt [naux][nx][nmo], Via [naux][m * (nx - m)] or None) for the QMOs of chi [nmo][nx]."""
        naux, nmo = L.shape[0], L.shape[1]
        nx = chi.shape[1]
        Lt = torch.empty((naux, nx, nmo), dtype=torch.float64, device=L.device)
        Via = torch.empty((naux, m * (nx - m)), dtype=torch.float64, device=L.device) if 0 < m < nx else None
        self._check(self._lib.mgw_qmo_tensors(self._h, nmo, naux, nx, m, _ptr(L, (naux, nmo, nmo), "L"),
                                              _ptr(chi, (nmo, nx), "chi"), _ptr(Lt), _ptr(Via)))
        return Lt, Via

    def mgw_df_absmax(self, L):
        out = ctypes.c_double()
        self._check(self._lib.mgw_df_absmax(self._h, L.numel(), _ptr(L), ctypes.byref(out)))
        return out.value

    def mgw_grid_exponent(self, absmax):
        return int(self._lib.mgw_grid_exponent(float(absmax)))

    def mgw_df_quantize(self, L, e, Lq=None):
        """Lq (int16, same shape) = round(L 2^(16-e)); raises on values outside the grid's range."""
        if L.dtype != torch.float64:
            raise ValueError("L must be float64")
        Lq = Lq if Lq is not None else torch.empty(L.shape, dtype=torch.int16, device=L.device)
        if Lq.dtype != torch.int16 or Lq.numel() != L.numel() or not Lq.is_contiguous():
            raise ValueError("Lq must be a contiguous int16 tensor of L's size")
        ov = ctypes.c_int()
        self._check(self._lib.mgw_df_quantize(self._h, L.numel(), _ptr(L), int(e), Lq.data_ptr(), ctypes.byref(ov)))
        return Lq

    def _qptr(self, Lq, shape):
        if not Lq.is_cuda or Lq.dtype != torch.int16 or not Lq.is_contiguous() or tuple(Lq.shape) != tuple(shape):
            raise ValueError(f"Lq must be a contiguous int16 CUDA tensor of shape {shape}")
        return Lq.data_ptr()

    def mgw_response_moments_q(self, opts: Options, nocc, nvir, naux, nmom, eps_W, Lq, e, Wmom=None):
        nmo = nocc + nvir
        Wmom = Wmom if Wmom is not None else torch.empty((nmom, naux, naux), dtype=torch.float64, device=eps_W.device)
        self._check(self._lib.mgw_response_moments_q(self._h, ctypes.byref(opts), nocc, nvir, naux, nmom,
                                                     _ptr(eps_W, (nmo,), "eps_W"), self._qptr(Lq, (naux, nmo, nmo)),
                                                     int(e), _ptr(Wmom, (nmom, naux, naux), "Wmom")))
        return Wmom

    def mgw_sigma_moments_q(self, opts: Options, nocc, nvir, naux, nmom, eps_G, Lq, e, Wmom, sig_hole=None,
                            sig_part=None):
        nmo = nocc + nvir
        dev = eps_G.device
        sh = sig_hole if sig_hole is not None else torch.empty((nmom, nmo, nmo), dtype=torch.float64, device=dev)
        sp = sig_part if sig_part is not None else torch.empty((nmom, nmo, nmo), dtype=torch.float64, device=dev)
        self._check(self._lib.mgw_sigma_moments_q(self._h, ctypes.byref(opts), nocc, nvir, naux, nmom,
                                                  _ptr(eps_G, (nmo,), "eps_G"), self._qptr(Lq, (naux, nmo, nmo)),
                                                  int(e), _ptr(Wmom, (nmom, naux, naux), "Wmom"),
                                                  _ptr(sh, (nmom, nmo, nmo), "sig_hole"),
                                                  _ptr(sp, (nmom, nmo, nmo), "sig_part")))
        return sh, sp

    def mgw_selftest_bounded_wait(self, limit_s):
        """A bounded wait that nothing satisfies: raises MgwError(MGW_ERR_TIMEOUT)."""
        self._check(self._lib.mgw_selftest_bounded_wait(self._h, float(limit_s)))

    def mgw_gemm_bf16x3(self, A, B, C=None):
        """C = A B^T on the tensor cores with BF16 hi/lo operand splits (3 products, FP32 accumulate)."""
        M, K = A.shape
        N = B.shape[0]
        C = C if C is not None else torch.empty((M, N), dtype=torch.float64, device=A.device)
        self._check(self._lib.mgw_gemm_bf16x3(self._h, M, N, K, _ptr(A, (M, K), "A"), _ptr(B, (N, K), "B"),
                                              _ptr(C, (M, N), "C")))
        return C

    def mgw_extract_ov(self, nocc, nvir, L, Lov=None):
        naux, nmo = L.shape[0], L.shape[1]
        Lov = Lov if Lov is not None else torch.empty((naux, nocc * nvir), dtype=L.dtype, device=L.device)
        self._check(self._lib.mgw_extract_ov(self._h, nocc, nvir, naux, _ptr(L, (naux, nmo, nmo), "L"),
                                             _ptr(Lov, (naux, nocc * nvir), "Lov")))
        return Lov

    def mgw_response_moments(self, opts: Options, nocc, nvir, naux, nmom, eps_W, Lov, Wmom=None):
        Wmom = Wmom if Wmom is not None else torch.empty((nmom, naux, naux), dtype=torch.float64, device=Lov.device)
        self._check(self._lib.mgw_response_moments(
            self._h, ctypes.byref(opts), nocc, nvir, naux, nmom, _ptr(eps_W, (nocc + nvir,), "eps_W"),
            _ptr(Lov, (naux, nocc * nvir), "Lov"), _ptr(Wmom, (nmom, naux, naux), "Wmom")))
        return Wmom

    def mgw_sigma_moments(self, opts: Options, nocc, nvir, naux, nmom, eps_G, L, Wmom, sig_hole=None, sig_part=None):
        nmo = nocc + nvir
        dev = L.device
        sig_hole = sig_hole if sig_hole is not None else torch.empty((nmom, nmo, nmo), dtype=torch.float64, device=dev)
        sig_part = sig_part if sig_part is not None else torch.empty((nmom, nmo, nmo), dtype=torch.float64, device=dev)
        self._check(self._lib.mgw_sigma_moments(
            self._h, ctypes.byref(opts), nocc, nvir, naux, nmom, _ptr(eps_G, (nmo,), "eps_G"),
            _ptr(L, (naux, nmo, nmo), "L"), _ptr(Wmom, (nmom, naux, naux), "Wmom"),
            _ptr(sig_hole, (nmom, nmo, nmo), "sig_hole"), _ptr(sig_part, (nmom, nmo, nmo), "sig_part")))
        return sig_hole, sig_part

    def mgw_block_lanczos(self, opts: Options, nmo, nmom, sig, coup=None, alpha=None, beta=None):
        nblk = nmom // 2
        dev = sig.device
        coup = coup if coup is not None else torch.empty((nmo, nmo), dtype=torch.float64, device=dev)
        alpha = alpha if alpha is not None else torch.empty((nblk, nmo, nmo), dtype=torch.float64, device=dev)
        if beta is None and nblk > 1:
            beta = torch.empty((nblk - 1, nmo, nmo), dtype=torch.float64, device=dev)
        rank = ctypes.c_int(0)
        self._check(self._lib.mgw_block_lanczos(
            self._h, ctypes.byref(opts), nmo, nmom, _ptr(sig, (nmom, nmo, nmo), "sig"), _ptr(coup, (nmo, nmo), "coup"),
            _ptr(alpha, (nblk, nmo, nmo), "alpha"),
            _ptr(beta, (nblk - 1, nmo, nmo), "beta") if nblk > 1 else None, ctypes.byref(rank)))
        return coup, alpha, beta, rank.value

    def mgw_qp_solve(self, opts: Options, nmo, nblk, rank_h, rank_p, fock, hole, part, zeta=0.0, nelec=0.0,
                     want_chi=False, want_rho=True):
        """hole/part: (coup, alpha, beta) as returned by mgw_block_lanczos."""
        dim = nmo + nblk * (rank_h + rank_p)
        dev = fock.device
        E = torch.empty((dim,), dtype=torch.float64, device=dev)
        weight = torch.empty((dim,), dtype=torch.float64, device=dev)
        chi = torch.empty((nmo, dim), dtype=torch.float64, device=dev) if want_chi else None
        eps_qp = torch.empty((nmo,), dtype=torch.float64, device=dev)
        rho = torch.empty((nmo, nmo), dtype=torch.float64, device=dev) if want_rho else None
        mu, ne, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()

        def blk(t, shape, name):
            return _ptr(t, shape, name) if t is not None else None
        ch, ah, bh = hole
        cp, ap, bp = part
        self._check(self._lib.mgw_qp_solve(
            self._h, ctypes.byref(opts), nmo, nblk, rank_h, rank_p, _ptr(fock, (nmo, nmo), "fock"),
            blk(ch, (nmo, nmo), "coup_h"), blk(ah, (nblk, nmo, nmo), "alpha_h"),
            blk(bh, (nblk - 1, nmo, nmo), "beta_h") if nblk > 1 else None,
            blk(cp, (nmo, nmo), "coup_p"), blk(ap, (nblk, nmo, nmo), "alpha_p"),
            blk(bp, (nblk - 1, nmo, nmo), "beta_p") if nblk > 1 else None,
            float(zeta), float(nelec), _ptr(E), _ptr(weight), _ptr(chi), _ptr(eps_qp), _ptr(rho),
            ctypes.byref(mu), ctypes.byref(ne), ctypes.byref(m)))
        return dict(E=E, weight=weight, chi=chi, eps_qp=eps_qp, rho=rho, mu=mu.value, nelec=ne.value, m=m.value)
