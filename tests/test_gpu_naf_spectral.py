"""Natural auxiliary functions (Sec. II D, Eq. 14) and the spectral function
(Eqs. 11-12) on the GPU against the oracle.

NAF rows are eigenvectors, fixed up to sign: each GPU row is compared with
the oracle's after aligning its sign.  The truncation threshold sits midway
between two of the oracle's eigenvalues so both sides keep the same count.
"""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("all_pairs", [False, True])
@pytest.mark.parametrize("nocc,nvir,naux", [(3, 7, 29), (5, 40, 130)])
def test_naf_compress_matches_oracle(h, nocc, nvir, naux, all_pairs):
    nmo = nocc + nvir
    L = mgw_inputs.df_tensor(naux, nmo, 3) * 2.0
    pairs = "full" if all_pairs else "no_vv"
    _, lam_ref = orc.naf_basis(L, nocc, -1.0, pairs)
    keep = (2 * naux) // 3
    thresh = 0.5 * (lam_ref[keep - 1] + lam_ref[keep])
    ref = orc.naf_compress(L, nocc, thresh, pairs)
    got, lam = h.mgw_naf_compress(nocc, torch.from_numpy(L).cuda(), thresh, all_pairs)
    lam = lam.cpu().numpy()
    assert np.abs(lam - lam_ref).max() < 1e-10 * lam_ref[0]
    got = got.cpu().numpy()
    assert got.shape == ref.shape == (keep, nmo, nmo)
    for a in range(keep):
        s = np.sign(np.sum(got[a] * ref[a]))
        assert rel(s * got[a], ref[a]) < 1e-8, a


def test_naf_compress_of_a_low_rank_tensor_keeps_its_rank(h):
    nocc, nmo, naux, r = 4, 30, 90, 17
    g = np.random.default_rng(5)
    B = g.standard_normal((r, nmo, nmo))
    B = 0.1 * (B + B.transpose(0, 2, 1)) / 2
    L = np.tensordot(g.standard_normal((naux, r)), B, axes=1)
    got, lam = h.mgw_naf_compress(nocc, torch.from_numpy(L).cuda(), 1e-6, False)
    assert got.shape[0] == r
    # the kept rows reproduce every pair product of the original tensor
    Lf, Gf = L.reshape(naux, -1), got.cpu().numpy().reshape(r, -1)
    assert rel(Gf.T @ Gf, Lf.T @ Lf) < 1e-10


def test_spectral_function_matches_oracle(h):
    eps = mgw_inputs.orbital_energies(5, 19, 2)
    L = mgw_inputs.df_tensor(72, 24, 2)
    res = orc.g0w0(eps, L, 5, 5)
    E, weight = res["E"], res["weight"]
    assert E.size > 256 and E.size % 256  # more than one pole tile, ragged
    omega = np.linspace(E.min() - 1.0, E.max() + 1.0, 1001)
    for delta in (0.01, 0.1):
        ref = orc.spectral_function(E, weight, omega, delta)
        got = h.mgw_spectral_function(torch.from_numpy(E).cuda(), torch.from_numpy(weight).cuda(),
                                      torch.from_numpy(omega).cuda(), delta)
        assert rel(got.cpu().numpy(), ref) < 1e-12


def test_spectral_function_rejects_a_non_positive_broadening(h):
    from paper_2504_17439_gb300 import mgw

    E = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(mgw.MgwError):
        h.mgw_spectral_function(E, E, E, 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc", "mixed"])
def test_g0w0_on_natural_auxiliary_functions(h, precision):
    """The driver compresses L to its natural auxiliary functions (Eq. 14)
    and runs the whole chain on n_naf of them: QP energies as the oracle's
    chain on the oracle's compressed tensor (the rows' signs and the basis
    inside the NAF space do not enter the moments, which are bilinear in L).
    The mixed precision is held to 1 meV of that FP64 oracle."""
    from paper_2504_17439_gb300 import driver, mgw

    shape, seed = mgw_inputs.workload("g0w0-nmo24-naux72")
    eps, L = mgw_inputs.system(shape, seed)
    _, lam = orc.naf_basis(L, shape.nocc, -1.0, "no_vv")
    keep = (2 * L.shape[0]) // 3
    thresh = 0.5 * (lam[keep - 1] + lam[keep])
    ref = orc.g0w0(eps, orc.naf_compress(L, shape.nocc, thresh, "no_vv"), shape.nocc, shape.nmom_max)
    prec = {"fp64": mgw.MGW_FP64, "fp64_tc": mgw.MGW_FP64_TC, "mixed": mgw.MGW_MIXED}[precision]
    r = driver.g0w0(h, torch.from_numpy(eps).cuda(), torch.from_numpy(L).cuda(), shape.nocc, shape.nmom_max,
                    opts=mgw.options(precision=prec), naf_eps=thresh)
    assert r["n_naf"] == keep
    err = np.abs(r["eps_qp"].cpu().numpy() - ref["eps_qp"]).max()
    assert err < (3.6749e-5 if precision == "mixed" else 1e-8), err
