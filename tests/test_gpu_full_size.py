"""Parity at the benchmark's full size (nocc 60, nvir 340, naux 1600,
nmom_max 7, TDA, FP64), in the launch configuration bench.py times.

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


@pytest.fixture(scope="module", params=["fp64", "fp64_tc"])
def run(request):
    from paper_2504_17439_gb300 import build, driver, mgw

    build.build()
    shape, seed = mgw_inputs.workload("g0w0-nmo400-naux1600")
    eps, L = mgw_inputs.system(shape, seed)
    h = mgw.Handle(0)
    o = mgw.options(precision=mgw.MGW_FP64 if request.param == "fp64" else mgw.MGW_FP64_TC)
    r = driver.g0w0(h, torch.from_numpy(eps).cuda(), torch.from_numpy(L).cuda(), shape.nocc, shape.nmom_max, opts=o)
    out = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in r.items()
           if k not in ("hole", "part")}
    out["hole"] = tuple(x.cpu().numpy() if isinstance(x, torch.Tensor) else x for x in r["hole"])
    out["part"] = tuple(x.cpu().numpy() if isinstance(x, torch.Tensor) else x for x in r["part"])
    h.close()
    return shape, eps, L, out


@pytest.fixture(scope="module")
def oracle_W(run):
    shape, eps, L, _ = run
    D = orc.energy_differences(eps, shape.nocc)
    return orc.tda_response_moments(orc.particle_hole_block(L, shape.nocc), D, shape.nmom)


def test_response_rows_sampled(run):
    shape, eps, L, out = run
    rows = [0, 1, 777, 1598, 1599]
    D = orc.energy_differences(eps, shape.nocc)
    Wr = orc.tda_response_moments(orc.particle_hole_block(L, shape.nocc), D, shape.nmom, rows=rows)
    for n in range(shape.nmom):
        assert rel(out["W"][n][rows], Wr[n]) < TOL, (n, rel(out["W"][n][rows], Wr[n]))


def test_sigma_rows_sampled(run, oracle_W):
    shape, eps, L, out = run
    rows = [0, 59, 60, 217, 399]  # first/last occupied, first virtual, middle, last
    rh, rp = orc.sigma_moments(eps, shape.nocc, L, oracle_W, rows=rows)
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
