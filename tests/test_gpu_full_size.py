"""Parity at the 400-orbital size (nocc 60, nvir 340, naux 1600, nmom_max 7,
TDA) on every precision, in the launch configuration bench.py uses.

The oracle cannot afford every output here, so it computes samples it can
reach directly: rows of W(t) (row P of eta~(n) = V A^n depends on row P of V
alone) and rows p of Sigma(n) (from the oracle's own full W).  Whole-output
properties that hold at any size are checked too: symmetry and positivity
of Sigma(0), moment conservation of the GPU's own block Lanczos, the sum
rule of the physical weights and the Aufbau electron count.
"""
import numpy as np
import pytest
import torch

import mgw_inputs
from oracle import mgw_oracle as orc

pytestmark = pytest.mark.gpu
TOL = 1e-9


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module", params=["fp64", "fp64_tc", "mixed"])
def run(request):
    from paper_2504_17439_gb300 import build, driver, mgw

    build.build()
    shape, seed = mgw_inputs.workload("g0w0-nmo400-naux1600")
    eps, L = mgw_inputs.system(shape, seed)
    h = mgw.Handle(0)
    o = mgw.options(precision={"fp64": mgw.MGW_FP64, "fp64_tc": mgw.MGW_FP64_TC,
                               "mixed": mgw.MGW_MIXED}[request.param])
    r = driver.g0w0(h, torch.from_numpy(eps).cuda(), torch.from_numpy(L).cuda(), shape.nocc, shape.nmom_max, opts=o)
    out = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in r.items()
           if k not in ("hole", "part")}
    out["hole"] = tuple(x.cpu().numpy() if isinstance(x, torch.Tensor) else x for x in r["hole"])
    out["part"] = tuple(x.cpu().numpy() if isinstance(x, torch.Tensor) else x for x in r["part"])
    out["precision"] = request.param
    h.close()
    return shape, eps, L, out


def contracted(out, L, nocc):
    """(V, L) as the run's precision contracts them: on their 16-bit grids
    under MGW_MIXED, as given otherwise."""
    V = orc.particle_hole_block(L, nocc)
    if out["precision"] == "mixed":
        return orc.fixed_point_grid(V), orc.fixed_point_grid(L)
    return V, L


@pytest.fixture(scope="module")
def oracle_W(run):
    shape, eps, L, out = run
    D = orc.energy_differences(eps, shape.nocc)
    return orc.tda_response_moments(contracted(out, L, shape.nocc)[0], D, shape.nmom)


def test_response_rows_sampled(run):
    shape, eps, L, out = run
    rows = [0, 1, 777, 1598, 1599]
    D = orc.energy_differences(eps, shape.nocc)
    Wr = orc.tda_response_moments(contracted(out, L, shape.nocc)[0], D, shape.nmom, rows=rows)
    for n in range(shape.nmom):
        assert rel(out["W"][n][rows], Wr[n]) < TOL, (n, rel(out["W"][n][rows], Wr[n]))


def test_sigma_rows_sampled(run, oracle_W):
    shape, eps, L, out = run
    rows = [0, 59, 60, 217, 399]  # first/last occupied, first virtual, middle, last
    rh, rp = orc.sigma_moments(eps, shape.nocc, contracted(out, L, shape.nocc)[1], oracle_W, rows=rows)
    for n in range(shape.nmom):
        assert rel(out["sigma_hole"][n][rows], rh[n]) < TOL, ("hole", n)
        assert rel(out["sigma_part"][n][rows], rp[n]) < TOL, ("particle", n)


def test_sigma_whole_output_properties(run):
    shape, eps, L, out = run
    for sig in (out["sigma_hole"], out["sigma_part"]):
        for n in range(shape.nmom):
            assert np.abs(sig[n] - sig[n].T).max() <= 1e-12 * np.abs(sig[n]).max()
        assert np.linalg.eigvalsh(sig[0]).min() > -1e-12 * np.abs(sig[0]).max()


def test_gpu_blocks_conserve_gpu_moments(run):
    shape, eps, L, out = run
    nb = shape.nmom_max + 1
    for (coup, alpha, beta, r), sig in ((out["hole"], out["sigma_hole"]), (out["part"], out["sigma_part"])):
        assert r == shape.nmo
        T = np.zeros((nb * r, nb * r))
        for i in range(nb):
            T[i * r:(i + 1) * r, i * r:(i + 1) * r] = alpha[i]
            if i + 1 < nb:
                T[(i + 1) * r:(i + 2) * r, i * r:(i + 1) * r] = beta[i]
                T[i * r:(i + 1) * r, (i + 1) * r:(i + 2) * r] = beta[i].T
        V0 = np.zeros((nb * r, r))
        V0[:r] = coup.T
        V = V0.copy()
        for n in range(shape.nmom):  # Sigma(n) = coup (T^n)_00 coup^T
            assert rel(V0.T @ V, sig[n]) < 1e-8, n
            V = T @ V


def test_qp_sum_rules(run):
    shape, eps, L, out = run
    assert abs(out["weight"].sum() - shape.nmo) < 1e-8
    assert abs(out["nelec"] - 2 * shape.nocc) < 0.1
    assert out["eps_qp"][shape.nocc - 1] < out["mu"] < out["eps_qp"][shape.nocc]
    assert np.all(np.diff(out["E"]) >= 0)


@pytest.fixture(scope="module")
def oracle_full():
    shape, seed = mgw_inputs.workload("g0w0-nmo400-naux1600")
    eps, L = mgw_inputs.system(shape, seed)
    return orc.g0w0(eps, L, shape.nocc, shape.nmom_max)


def test_qp_energies_against_the_full_oracle(run, oracle_full):
    """The whole oracle chain at this size (about a minute on the host, run
    once per module).  At N = 7 the moment-to-block step amplifies rounding
    by about 1e2 per block, so two FP64 computations of the same QP energies
    already differ by a few 0.1 meV here; every tensor-core path is held to
    the mixed path's bar, 1 meV, against the unrounded FP64 oracle."""
    shape, eps, L, out = run
    if out["precision"] == "fp64":
        pytest.skip("the FP64-unit path is held to the oracle on sampled rows and at the 24-orbital size")
    d = np.abs(out["eps_qp"] - oracle_full["eps_qp"]).max()
    assert d < 3.6749e-5, d
