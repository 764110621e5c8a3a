"""Seeded synthetic inputs for moment-conserving GW workloads.

This module is shared by the CPU oracle, the tests and the benchmark.  It
holds no arithmetic of the GW method itself: it only draws orbital energies
and a density-fitted (DF) three-index tensor with the shapes and value
distributions of molecular workloads, from a counter-based generator.

Generator: numpy's Philox4x32-10 bit generator (a counter-based generator),
keyed per (seed, stream).  Stream 0 draws the orbital energies; stream 1+Q
draws the Q-th auxiliary slab of the DF tensor, so any slab can be
regenerated on its own without drawing the others.

Distributions (restricted closed-shell, Hartree units):
  eps_occ ~ U[-1.5, -0.3] sorted ascending, eps_vir ~ U[0.1, 3.0] sorted;
  L[Q,p,q] = 0.1/sqrt(naux) * (G[Q,p,q] + G[Q,q,p]) / 2, G ~ N(0, 1),
so every slab L[Q] is a symmetric nmo x nmo matrix, as a DF factor of the
Coulomb integrals (pq|rs) = sum_Q L[Q,p,q] L[Q,r,s] is (Eq. 13).
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import math
import os

import numpy as np

SEED_BASE = 20250417 * 1000


@dataclasses.dataclass(frozen=True)
class Shape:
    """One molecular-like system: orbital counts, aux size, moment order."""

    nocc: int
    nvir: int
    naux: int
    nmom_max: int

    @property
    def nmo(self) -> int:
        return self.nocc + self.nvir

    @property
    def ov(self) -> int:
        return self.nocc * self.nvir

    @property
    def nmom(self) -> int:
        # moments 0 .. 2*nmom_max+1 are built and conserved
        return 2 * self.nmom_max + 2


# Named workloads.  Seeds follow seed = SEED_BASE + 100*k + system.
WORKLOADS = {
    # small G0W0: brute force over the 95 x 95 particle-hole space is cheap
    "g0w0-nmo24-naux72": dict(shape=Shape(5, 19, 72, 5), seed=SEED_BASE + 0),
    # molecule-sized FP64 workload (TDA and RPA with a 48-node quadrature)
    "g0w0-nmo400-naux1600": dict(shape=Shape(60, 340, 1600, 7), seed=SEED_BASE + 100),
    # mid-size system for profiler captures: inputs above L2, a few GB on device
    "g0w0-nmo200-naux800": dict(shape=Shape(30, 170, 800, 7), seed=SEED_BASE + 300),
    # profiler captures of the headline's contraction length (K = naux = 4800)
    # on a few GB of device memory
    "g0w0-nmo200-naux4800": dict(shape=Shape(30, 170, 4800, 7), seed=SEED_BASE + 310),
    # pigment-molecule scale, mixed-precision workload
    "g0w0-nmo1200-naux4800": dict(shape=Shape(240, 960, 4800, 7), seed=SEED_BASE + 200),
    # chlorophyll-A scale (2147 orbitals, 482 electrons, naux = 4 nmo): 317 GB
    # in FP64, produced slab by slab (df_slab) and never held whole
    "g0w0-nmo2147-naux8588": dict(shape=Shape(241, 1906, 8588, 7), seed=SEED_BASE + 600),
}


def _rng(seed: int, stream: int) -> np.random.Generator:
    # Philox key: 128 bits; the low word carries the stream, the high the seed.
    key = (int(seed) << 64) | int(stream)
    return np.random.Generator(np.random.Philox(key=key))


def orbital_energies(nocc: int, nvir: int, seed: int) -> np.ndarray:
    """eps[nmo], occupied block ascending then virtual block ascending."""
    g = _rng(seed, 0)
    eo = np.sort(g.uniform(-1.5, -0.3, nocc))
    ev = np.sort(g.uniform(0.1, 3.0, nvir))
    return np.concatenate([eo, ev]).astype(np.float64)


def df_slab(q: int, naux: int, nmo: int, seed: int) -> np.ndarray:
    """The Q-th auxiliary slab L[Q] (nmo x nmo, symmetric)."""
    g = _rng(seed, 1 + q).standard_normal((nmo, nmo))
    return (0.1 / math.sqrt(naux)) * 0.5 * (g + g.T)


def df_tensor(naux: int, nmo: int, seed: int, out: np.ndarray | None = None, workers: int = 0) -> np.ndarray:
    """L[naux][nmo][nmo] in float64 (row-major).  Slabs have streams of their
    own, so they are drawn on `workers` threads (0: one per core for tensors
    above 2^26 elements) with the same values as one thread."""
    if out is None:
        out = np.empty((naux, nmo, nmo), dtype=np.float64)

    def fill(q):
        out[q] = df_slab(q, naux, nmo, seed)
    if workers == 0:
        workers = (os.cpu_count() or 1) if naux * nmo * nmo > (1 << 26) else 1
    if workers <= 1:
        for q in range(naux):
            fill(q)
    else:
        with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(fill, range(naux)))
    return out


def sym_matrices(count: int, n: int, seed: int, stream: int = 0x5E3) -> np.ndarray:
    """count symmetric n x n matrices (G + G^T) / (2 sqrt(n)), G ~ N(0, 1):
    generic stand-ins for an aux-basis moment stack when a stage is tested
    on its own."""
    out = np.empty((count, n, n))
    for t in range(count):
        g = _rng(seed, stream + t).standard_normal((n, n))
        out[t] = (g + g.T) / (2.0 * math.sqrt(n))
    return out


def system(shape: Shape, seed: int):
    """(eps, L) for one system."""
    eps = orbital_energies(shape.nocc, shape.nvir, seed)
    L = df_tensor(shape.naux, shape.nmo, seed)
    return eps, L


def workload(name: str):
    w = WORKLOADS[name]
    return w["shape"], w["seed"]


def batch_shapes(nsys: int, seed: int, nmo_lo: int = 40, nmo_hi: int = 300, nmom_max: int = 5):
    """Uneven batch: nmo ~ U{lo..hi}, nocc = round(nmo/6), naux = 4 nmo."""
    g = _rng(seed, 0xBA7C4)
    nmos = g.integers(nmo_lo, nmo_hi + 1, nsys)
    shapes = []
    for n in nmos:
        n = int(n)
        no = int(round(n / 6))
        shapes.append(Shape(no, n - no, 4 * n, nmom_max))
    return shapes


def random_orthogonal(n: int, seed: int, stream: int = 0x0A7) -> np.ndarray:
    """A Haar-random orthogonal n x n matrix (QR of a Gaussian, sign-fixed)."""
    g = _rng(seed, stream).standard_normal((n, n))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]
