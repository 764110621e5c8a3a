"""The allocation-free TDA response entry point against the regular one.

mgw_response_moments_tda_noalloc keeps its scratch in a static device array
so that callers who cannot allocate device memory can still build the TDA
response moments.  It must give the regular entry point's result (same
tolerance as the other parity tests, 1e-9 relative per moment order) on two
calls in a row, the second reusing the scratch the first left behind, and it
must refuse sizes beyond its fixed scratch without running anything.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import mgw_inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_tda_matches_regular_entry_point_twice():
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    lib = mgw.load()
    fn = lib.mgw_response_moments_tda_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    h = mgw.Handle(0)
    stream = torch.cuda.current_stream()
    for nocc, nvir, naux, N, seed in ((5, 19, 72, 5, 31), (7, 30, 130, 4, 32)):
        eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
        L = mgw_inputs.df_tensor(naux, nocc + nvir, seed) * 2.0
        nmom = 2 * N + 2
        Lov = torch.from_numpy(np.ascontiguousarray(L[:, :nocc, nocc:]).reshape(naux, -1)).cuda()
        e = torch.from_numpy(eps).cuda()
        ref = h.mgw_response_moments(mgw.options(screening=mgw.MGW_TDA), nocc, nvir, naux, nmom, e, Lov).cpu().numpy()
        for call in range(2):
            W = torch.full((nmom, naux, naux), float("nan"), dtype=torch.float64, device="cuda")
            st = fn(ctypes.c_void_p(stream.cuda_stream), nocc, nvir, naux, nmom, ctypes.c_void_p(e.data_ptr()),
                    ctypes.c_void_p(Lov.data_ptr()), ctypes.c_void_p(W.data_ptr()))
            assert st == 0, st
            got = W.cpu().numpy()
            for n in range(nmom):
                assert rel(got[n], ref[n]) < 1e-9, (call, n, rel(got[n], ref[n]))
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2504_17439_gb300 import mgw

    lib = mgw.load()
    fn = lib.mgw_response_moments_tda_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # naux * ov + ov = 2001 * 2100 + 2100 > 4 Mi doubles: refused before any launch
    st = fn(None, 30, 70, 2001, 4, p, p, p)
    assert st == -8
