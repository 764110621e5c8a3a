"""scGW, GW0 and G0W on the quasi-molecular orbitals (Algorithm 5, Sec. III E)
through the C ABI (mgw_qmo_tensors, mgw_sigma_moments_x and the single-system
calls) against the oracle's scgw: the same QP energies and poles after a
fixed number of iterations, for every variant; and the QMO tensors of one H~
against the oracle's qmo_tensors."""
import numpy as np
import pytest
import torch

import mgw_inputs
from oracle import mgw_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    hh = mgw.Handle(0)
    yield hh
    hh.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def system(nocc=3, nvir=5, naux=12, seed=7, scale=3.0):
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    return eps, mgw_inputs.df_tensor(naux, nocc + nvir, seed) * scale


def test_qmo_tensors_match_the_oracle(h):
    eps, L = system()
    r = orc.g0w0(eps, L, 3, 2)
    chi, m = r["chi"], r["m"]
    Vhat, Via = orc.qmo_tensors(L, chi, m)
    Lt, Vq = h.mgw_qmo_tensors(dev(L), dev(chi), m)
    assert np.abs(Lt.cpu().numpy() - Vhat.transpose(0, 2, 1)).max() < 1e-12 * np.abs(Vhat).max()
    assert np.abs(Vq.cpu().numpy() - Via).max() < 1e-12 * np.abs(Via).max()


@pytest.mark.parametrize("variant", ["scgw", "gw0", "g0w"])
@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_scgw_iterations_match_the_oracle(h, variant, precision):
    from paper_2504_17439_gb300 import driver, mgw

    eps, L = system()
    kw = dict(g0=variant == "g0w", w0=variant == "gw0")
    ref = orc.scgw(eps, L, 3, 2, conv=0.0, max_iter=3, **kw)
    o = mgw.options(precision=mgw.MGW_FP64 if precision == "fp64" else mgw.MGW_FP64_TC)
    got = driver.scgw(h, dev(eps), dev(L), 3, 2, conv=0.0, max_iter=3, opts=o, **kw)
    assert [x["poles"] for x in got["history"]] == [x["poles"] for x in ref["history"]]
    assert np.abs(got["eps_qp"].cpu().numpy() - ref["eps_qp"]).max() < 1e-8
    assert np.abs(got["E"].cpu().numpy() - ref["E"]).max() < 1e-7
    assert abs(got["nelec"] - ref["nelec"]) < 1e-8
