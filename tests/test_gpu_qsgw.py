"""Static qsGW potential (Sec. III D, Eqs. 36-39) on the GPU against the
oracle, from the oracle's own block-Lanczos chains padded to the library's
layout."""
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


def padded(chain, nmo, nblk):
    coup, alpha, beta, r = chain
    c = np.zeros((nmo, nmo))
    a = np.zeros((nblk, nmo, nmo))
    b = np.zeros((max(nblk - 1, 1), nmo, nmo))
    c[:, :r] = coup
    a[:, :r, :r] = alpha
    if nblk > 1:
        b[:, :r, :r] = beta
    return r, tuple(torch.from_numpy(x).cuda() for x in (c, a, b))


@pytest.mark.parametrize("reg", ["eta", "srg"])
@pytest.mark.parametrize("nocc,nvir,naux,nmom_max,seed", [(3, 5, 12, 2, 7), (5, 32, 90, 3, 4), (1, 5, 3, 2, 3)])
def test_qsgw_potential_matches_oracle(h, reg, nocc, nvir, naux, nmom_max, seed):
    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    L = mgw_inputs.df_tensor(naux, nocc + nvir, seed) * 3.0
    r = orc.g0w0(eps, L, nocc, nmom_max)
    nmo, nblk = eps.size, nmom_max + 1
    ref = orc.qsgw_potential(eps, r["hole"], r["part"], reg, delta=1e-3, srg_s=100.0)
    rh, hole = padded(r["hole"], nmo, nblk)
    rp, part = padded(r["part"], nmo, nblk)
    got = h.mgw_qsgw_potential(nmo, nblk, rh, rp, torch.from_numpy(eps).cuda(), hole, part, reg, 1e-3, 100.0)
    got = got.cpu().numpy()
    assert np.linalg.norm(got - ref) < 1e-10 * np.linalg.norm(ref)
