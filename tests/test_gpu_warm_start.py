"""Learned warm start of the fsGW zeta search.

The plain loop (driver.fsgw without a network) generates the training data:
every outer step records its search features and zeta - zeta_prev.  A
3-layer SiLU network (width 256, BF16 weights, FP32 accumulation) is trained
on them with the library's own forward/backward/Adam kernels.  On held-out
systems the warm loop must converge to the plain loop's QP energies and
spend fewer H~ diagonalisations on zeta.  A second network, trained on the
steps' least-squares Fock-step targets, proposes the starting F of each step
(F + beta (F - F_prev)); with it the loop must still reach the same QP
energies.
"""
import numpy as np
import pytest
import torch

import mgw_inputs
from oracle import mgw_oracle as orc

pytestmark = pytest.mark.gpu


def systems(n, seed0):
    out = []
    g = np.random.default_rng(seed0)
    for i in range(n):
        nmo = int(g.integers(10, 18))
        nocc = int(round(nmo / 5))
        eps = mgw_inputs.orbital_energies(nocc, nmo - nocc, seed0 + i)
        L = mgw_inputs.df_tensor(3 * nmo, nmo, seed0 + i) * 2.0
        out.append((nocc, eps, L, orc.hf_core_hamiltonian(eps, L, nocc)))
    return out


def run(h, sy, warm=None, warm_fock=None):
    from paper_2504_17439_gb300 import driver

    nocc, eps, L, hc = sy
    return driver.fsgw(h, torch.from_numpy(hc).cuda(), torch.from_numpy(L).cuda(), torch.from_numpy(eps).cuda(),
                       nocc, 2, conv_e=1e-8, conv_mom=1e-7, max_outer=40, warm=warm, warm_fock=warm_fock)


def test_warm_start_trains_and_saves_zeta_evaluations():
    from paper_2504_17439_gb300 import build, driver, mgw

    build.build()
    h = mgw.Handle(0)
    feats, targets, ffeats, ftargets = [], [], [], []
    for sy in systems(24, 1000):
        r = run(h, sy)
        assert r["converged"]
        for step in r["history"]:
            feats.append(step["feat"])
            targets.append(step["target"])
            assert step["fock_beta"] == 0.0  # no network, no proposal
            if step["fock_valid"]:
                assert np.isfinite(step["fock_target"])
                ffeats.append(step["fock_feat"])
                ftargets.append(step["fock_target"])
    net = driver.WarmStart(h, width=256, seed=1)
    losses = net.train(np.array(feats), np.array(targets), epochs=600, lr=1e-3)
    assert losses[-1] < 0.2 * losses[0]
    plain_evals = warm_evals = 0
    for sy in systems(6, 5000):
        rp = run(h, sy)
        rw = run(h, sy, warm=net)
        assert rp["converged"] and rw["converged"]
        assert np.abs(rw["eps_qp"].cpu().numpy() - rp["eps_qp"].cpu().numpy()).max() < 1e-6
        plain_evals += sum(s["zeta_evals"] for s in rp["history"])
        warm_evals += sum(s["zeta_evals"] for s in rw["history"])
    print(f"zeta evaluations: plain {plain_evals}, warm {warm_evals}")
    assert warm_evals < plain_evals
    # the Fock-matrix proposal on top: the plain DIIS loop it starts keeps the
    # fixed point (the proposal may only move the starting F)
    net_f = driver.WarmStart(h, width=256, seed=2)
    net_f.train(np.array(ffeats), np.array(ftargets), epochs=300, lr=1e-3, scale=1.0)
    inner = [0, 0]
    for sy in systems(3, 5000):
        rp = run(h, sy)
        rf = run(h, sy, warm=net, warm_fock=net_f)
        assert rf["converged"]
        assert np.abs(rf["eps_qp"].cpu().numpy() - rp["eps_qp"].cpu().numpy()).max() < 1e-6
        assert any(s["fock_beta"] != 0.0 for s in rf["history"][1:])
        inner[0] += sum(s["inner"] for s in rp["history"])
        inner[1] += sum(s["inner"] for s in rf["history"])
    print(f"Fock-loop iterations: plain {inner[0]}, with both proposals {inner[1]}")
    h.close()
