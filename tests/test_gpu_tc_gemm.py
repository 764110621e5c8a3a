"""Tensor-core (tcgen05/TMA/TMEM) split-precision GEMM against an FP64 product.

The error bound follows from the arithmetic: with x = hi + lo, |lo| <= 2^-9 |x|
and |x - hi - lo| <= 2^-9 |lo|, the dropped lo*lo term and the split residues
are ~2^-16 |A||B| per product, plus FP32 accumulation (2^-24 sqrt(K)); the
test allows 2e-5 of sum_k |A_ik||B_jk|.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2504_17439_gb300 import build, mgw

    build.build()
    return mgw.Handle(0)


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 520, 200), (1, 1, 1), (257, 17, 1000), (1024, 1024, 4800)])
def test_bf16x3_gemm_matches_fp64(h, M, N, K):
    g = np.random.default_rng(M * 7 + N * 3 + K)
    A = g.standard_normal((M, K))
    B = g.standard_normal((N, K))
    C = h.mgw_gemm_bf16x3(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    err = np.abs(C - ref) / scale
    assert err.max() < 2e-5, err.max()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 520, 200), (1, 1, 1), (257, 17, 1000), (512, 384, 4800),
                                   (130, 140, 2500)])
def test_fp64_emulated_gemm_matches_fp64(h, M, N, K):
    """Digit-sliced tensor-core GEMM: error within a few 2^-53 of sum_k |A||B|
    (an FP64 GEMM's own bound), with a wide exponent spread across rows."""
    g = np.random.default_rng(M * 5 + N * 11 + K)
    A = g.standard_normal((M, K)) * np.exp2(g.integers(-20, 20, (M, 1)))
    B = g.standard_normal((N, K)) * np.exp2(g.integers(-20, 20, (N, 1)))
    A[:, :: max(1, K // 7)] *= 1e-9  # small entries inside a row
    C = h.mgw_gemm_fp64_emu(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    err = np.abs(C - ref) / scale
    assert err.max() < 8 * 2.0**-52, err.max()


@pytest.mark.parametrize("K", [4800, 1024 * 9])
def test_mixed_gemm_exact_at_the_window_bound(h, K):
    """Same-sign operands near the top of their digit ranges make every
    level's window sum approach the 2^24 units that FP32 holds exactly (K = 9216
    gives full windows of 8 chunks at level 2): the product must still come out
    within a few units in the last place of the exact K a b'."""
    from fractions import Fraction
    from oracle import mgw_oracle as orc

    M, N = 130, 70
    a, b = 0.9990234375 - 2.0**-40, 0.99609375 - 2.0**-20
    A = np.full((M, K), a)
    B = np.full((N, K), b)
    C = h.mgw_gemm_mixed(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    bq = float(orc.fixed_point_grid(B)[0, 0])
    exact = float(Fraction(a) * Fraction(bq) * K)
    ulp = np.spacing(exact)
    assert np.abs(C - exact).max() <= 4 * ulp, (np.abs(C - exact).max() / ulp)


def test_fp64_emulated_gemm_zero_rows(h):
    A = np.zeros((130, 70))
    B = np.random.default_rng(1).standard_normal((129, 70))
    A[5] = 1.5
    C = h.mgw_gemm_fp64_emu(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    ref = A @ B.T
    assert np.abs(C - ref).max() <= 1e-15 * np.abs(ref).max()
    assert np.all(C[np.arange(130) != 5] == 0)


def test_bounded_wait_gives_up_and_the_handle_stays_usable(h):
    """A wait that nothing satisfies ends after its limit with MGW_ERR_TIMEOUT
    (not a hang, not a fault), and the next tensor-core call on the same
    handle and stream is correct."""
    import time

    from paper_2504_17439_gb300 import mgw

    t0 = time.perf_counter()
    with pytest.raises(mgw.MgwError) as e:
        h.mgw_selftest_bounded_wait(0.05)
    dt = time.perf_counter() - t0
    assert e.value.status == -7 and "timed out" in str(e.value)
    assert 0.04 < dt < 5.0, dt
    g = np.random.default_rng(9)
    A, B = g.standard_normal((200, 300)), g.standard_normal((150, 300))
    C = h.mgw_gemm_fp64_emu(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    assert (np.abs(C - A @ B.T) / (np.abs(A) @ np.abs(B).T)).max() < 1e-15


@pytest.mark.parametrize("M,N,K", [(128, 96, 64), (300, 520, 200), (1, 1, 1), (257, 17, 1000), (512, 384, 4800),
                                   (130, 140, 2500), (200, 300, 100), (129, 65, 1088), (130, 70, 65536 + 700)])
def test_mixed_gemm_is_exact_for_the_rounded_operand(h, M, N, K):
    """The mixed-precision product (chunked, tile-reusing kernel): A at seven
    digits against B rounded to its 16-bit grid (the oracle's
    fixed_point_grid), within a few 2^-53 of sum_k |A||B'| -- an FP64 GEMM's
    own bound on the product with the rounded operand; K spans odd chunk
    counts and a partial last chunk."""
    from oracle import mgw_oracle as orc

    g = np.random.default_rng(M * 3 + N * 7 + K)
    A = g.standard_normal((M, K)) * np.exp2(g.integers(-20, 20, (M, 1)))
    B = g.standard_normal((N, K))
    A[:, :: max(1, K // 7)] *= 1e-9
    C = h.mgw_gemm_mixed(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    Bq = orc.fixed_point_grid(B)
    ref = A @ Bq.T
    scale = np.abs(A) @ np.abs(Bq).T
    err = np.abs(C - ref) / np.where(scale > 0, scale, 1.0)
    assert err.max() < 8 * 2.0**-52, err.max()
