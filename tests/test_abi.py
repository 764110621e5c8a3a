"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mgw_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2504_17439_gb300 import build

    return build.build()


def test_header_declares_the_path_calls():
    names = declared_symbols()
    for want in ("mgw_response_moments", "mgw_sigma_moments", "mgw_block_lanczos", "mgw_qp_solve",
                 "mgw_create", "mgw_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_options_default_fills_documented_values(lib_path):
    from paper_2504_17439_gb300 import mgw

    mgw._lib = None
    o = mgw.options()
    assert o.screening == mgw.MGW_TDA and o.precision == mgw.MGW_FP64
    assert o.nquad == 48 and o.diis_space == 12
    assert abs(o.conv_e - 5e-3 / 27.211386245988) < 1e-15
    assert o.conv_mom == 1e-4 and o.rank_tol == 1e-12


def test_binding_rejects_host_tensors(lib_path):
    import torch
    from paper_2504_17439_gb300 import mgw

    with pytest.raises(ValueError):
        mgw._ptr(torch.zeros(3, dtype=torch.float64), name="x")
