"""Parity at the pigment-molecule size: nocc 240, nvir 960 (nmo 1200), naux
4800, nmom_max 7, TDA -- the workload bench.py times -- on both tensor-core
precisions, in the launch configuration bench.py uses (automatic x chunks).

The oracle cannot build every output at this size, so it computes what it can
reach directly:
  - rows of W(t): row P of eta~(n) = V A^n depends on row P of V alone;
  - rows p of Sigma(n) from a generic symmetric moment stack drawn by the input
    module (the Sigma build is linear in W and takes any stack), the oracle's
    sum over Green's-function indices x taken chunk by chunk.
Under MGW_MIXED the oracle takes V and L rounded to their fixed-point grids
(oracle fixed_point_grid), the tensors that mode contracts; every result is
held to the FP64 tolerance (1e-9 relative per moment order).  The real chain
(response, then Sigma from it) is checked by properties that hold at any
size: symmetry and positivity of Sigma(0), and moment conservation of the
library's own block Lanczos.
"""
import numpy as np
import pytest
import torch

import mgw_inputs
from oracle import mgw_oracle as orc

pytestmark = pytest.mark.gpu
TOL = 1e-9
WORKLOAD = "g0w0-nmo1200-naux4800"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def inputs():
    shape, seed = mgw_inputs.workload(WORKLOAD)
    eps, L = mgw_inputs.system(shape, seed)
    Ws = mgw_inputs.sym_matrices(shape.nmom, shape.naux, seed)
    return shape, seed, eps, L, Ws


@pytest.fixture(scope="module", params=["fp64_tc", "mixed"])
def run(request, inputs):
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    shape, seed, eps, L, Ws = inputs
    nocc, nvir, naux, nmo, nmom = shape.nocc, shape.nvir, shape.naux, shape.nmo, shape.nmom
    h = mgw.Handle(0)
    o = mgw.options(precision=mgw.MGW_FP64_TC if request.param == "fp64_tc" else mgw.MGW_MIXED)
    e = torch.from_numpy(eps).cuda()
    Ld = torch.from_numpy(L).cuda()
    Lov = h.mgw_extract_ov(nocc, nvir, Ld)
    W = h.mgw_response_moments(o, nocc, nvir, naux, nmom, e, Lov)
    del Lov
    sh, sp = h.mgw_sigma_moments(o, nocc, nvir, naux, nmom, e, Ld, W)
    out = {"precision": request.param, "W_rows": None}
    rows = [0, 1, 2399, 4798, 4799]
    out["W_rows"] = W[:, rows, :].cpu().numpy()
    del W
    # the real chain: whole-output properties and the library's own Lanczos
    props = {}
    for name, sig in (("hole", sh), ("part", sp)):
        asym = float(max((sig[n] - sig[n].T).abs().max() / sig[n].abs().max() for n in range(nmom)))
        lam0 = torch.linalg.eigvalsh(sig[0])
        coup, alpha, beta, r = h.mgw_block_lanczos(o, nmo, nmom, sig)
        nb = shape.nmom_max + 1
        T = torch.zeros((nb * r, nb * r), dtype=torch.float64, device="cuda")
        for i in range(nb):
            T[i * r:(i + 1) * r, i * r:(i + 1) * r] = alpha[i][:r, :r]
            if i + 1 < nb:
                T[(i + 1) * r:(i + 2) * r, i * r:(i + 1) * r] = beta[i][:r, :r]
                T[i * r:(i + 1) * r, (i + 1) * r:(i + 2) * r] = beta[i][:r, :r].T
        V0 = torch.zeros((nb * r, nmo), dtype=torch.float64, device="cuda")
        V0[:r] = coup[:, :r].T
        V = V0.clone()
        cons = []
        for n in range(nmom):
            rec = V0.T @ V
            cons.append(float(torch.linalg.norm(rec - sig[n]) / torch.linalg.norm(sig[n])))
            V = T @ V
        props[name] = dict(asym=asym, lam0_min=float(lam0.min()), lam0_max=float(lam0.max()), rank=r,
                           conservation=cons)
    out["props"] = props
    del sh, sp
    # the Sigma build alone on the generic stack, for row parity
    gh, gp = h.mgw_sigma_moments(o, nocc, nvir, naux, nmom, e, Ld, torch.from_numpy(Ws).cuda())
    prow = [0, 239, 240, 777, 1199]  # first/last occupied, first virtual, middle, last
    out["sig_rows"] = (prow, gh[:, prow, :].cpu().numpy(), gp[:, prow, :].cpu().numpy())
    del gh, gp, Ld
    torch.cuda.synchronize()
    h.close()
    return out


def test_response_rows_sampled(run, inputs):
    shape, seed, eps, L, Ws = inputs
    rows = [0, 1, 2399, 4798, 4799]
    D = orc.energy_differences(eps, shape.nocc)
    Lov = orc.particle_hole_block(L, shape.nocc)
    if run["precision"] == "mixed":
        Lov = orc.fixed_point_grid(Lov)
    ref = orc.tda_response_moments(Lov, D, shape.nmom, rows=rows)
    for n in range(shape.nmom):
        assert rel(run["W_rows"][n], ref[n]) < TOL, (n, rel(run["W_rows"][n], ref[n]))


def test_sigma_rows_sampled(run, inputs):
    shape, seed, eps, L, Ws = inputs
    prow, gh, gp = run["sig_rows"]
    m = float(np.abs(L).max())
    rh = np.zeros((shape.nmom, len(prow), shape.nmo))
    rp = np.zeros_like(rh)
    chunk = 40
    for x0 in range(0, shape.nmo, chunk):
        x1 = min(shape.nmo, x0 + chunk)
        Lc = L[:, :, x0:x1]
        if run["precision"] == "mixed":
            Lc = orc.fixed_point_grid(Lc, ref_max=m)
        nh = max(0, min(shape.nocc, x1) - x0)  # the chunk's holes come first
        a, b = orc.sigma_moments(eps[x0:x1], nh, Lc, Ws, rows=prow)
        rh += a
        rp += b
    for n in range(shape.nmom):
        assert rel(gh[n], rh[n]) < TOL, ("hole", n, rel(gh[n], rh[n]))
        assert rel(gp[n], rp[n]) < TOL, ("particle", n, rel(gp[n], rp[n]))


def test_whole_output_properties(run, inputs):
    shape = inputs[0]
    for name, p in run["props"].items():
        assert p["asym"] <= 1e-12, (name, p["asym"])
        assert p["lam0_min"] > -1e-12 * p["lam0_max"], (name, p["lam0_min"])
        assert p["rank"] == shape.nmo
        assert max(p["conservation"]) < 1e-8, (name, p["conservation"])
