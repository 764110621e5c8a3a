"""The DF tensor held on its grid as 16-bit integers (the input of the
MGW_MIXED path for tensors too large for FP64 storage): quantization against
the oracle's rounding, and the response and Sigma moments computed from the
integers against the oracle on the rounded tensors (1e-9 relative per moment
order, the FP64 tolerance)."""
import numpy as np
import pytest
import torch

import mgw_inputs
from oracle import mgw_oracle as orc

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def h():
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    hh = mgw.Handle(0)
    yield hh
    hh.close()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("nocc,nvir,naux,N,seed", [(5, 19, 72, 5, 41), (7, 30, 130, 4, 42), (3, 7, 65, 3, 43)])
def test_moments_from_the_integer_tensor(h, nocc, nvir, naux, N, seed):
    from paper_2504_17439_gb300 import mgw

    eps = mgw_inputs.orbital_energies(nocc, nvir, seed)
    L = mgw_inputs.df_tensor(naux, nocc + nvir, seed) * 2.0
    nmom = 2 * N + 2
    Ld = torch.from_numpy(L).cuda()
    m = h.mgw_df_absmax(Ld)
    assert m == np.abs(L).max()
    e = h.mgw_grid_exponent(m)
    Lq = h.mgw_df_quantize(Ld, e)
    # the integers are the oracle's rounding of L on the whole tensor's grid
    Lr = orc.fixed_point_grid(L)
    assert np.array_equal(Lq.cpu().numpy().astype(np.float64) * 2.0 ** (e - 16), Lr)
    o = mgw.options()
    e_d = torch.from_numpy(eps).cuda()
    W = h.mgw_response_moments_q(o, nocc, nvir, naux, nmom, e_d, Lq, e)
    D = orc.energy_differences(eps, nocc)
    Wr = orc.tda_response_moments(orc.particle_hole_block(Lr, nocc), D, nmom)  # V' = the block of L'
    Wg = W.cpu().numpy()
    for n in range(nmom):
        assert rel(Wg[n], Wr[n]) < TOL, ("W", n, rel(Wg[n], Wr[n]))
    sh, sp = h.mgw_sigma_moments_q(o, nocc, nvir, naux, nmom, e_d, Lq, e, torch.from_numpy(Wr).cuda())
    rh, rp = orc.sigma_moments(eps, nocc, Lr, Wr)
    sh, sp = sh.cpu().numpy(), sp.cpu().numpy()
    for n in range(nmom):
        assert rel(sh[n], rh[n]) < TOL, ("hole", n)
        assert rel(sp[n], rp[n]) < TOL, ("particle", n)


def test_quantize_reports_values_outside_the_grid(h):
    from paper_2504_17439_gb300 import mgw

    L = torch.full((4, 3, 3), 0.3, dtype=torch.float64, device="cuda")
    e = h.mgw_grid_exponent(0.3)
    h.mgw_df_quantize(L, e)
    with pytest.raises(mgw.MgwError) as err:
        h.mgw_df_quantize(L, e - 1)  # 0.3 >= 2^(e-2): outside the finer grid's range
    assert err.value.status == -1
