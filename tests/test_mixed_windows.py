"""The accumulation windows of the mixed-precision kernel (window_end in
paper_2504_17439_gb300/csrc/ozaki_mixed.h), compiled from the kernel's own
header as host code and checked for every chunk count a launch split can
have (K <= 65536: up to 512 chunks of 128).

Each exact level l = 2..6 accumulates a window of chunks in one FP32 TMEM
accumulator; a term is a product of two digits of magnitude <= 2^7, so the
window's partial sums stay integers below 2^24 units (exact in FP32) when
window length x products(l) x 128 terms x 2^14 <= 2^24.  Also checked: the
last chunk ends every window (nothing is left unread), at most two windows
end at any other chunk (the epilogue's flush work stays spread), and the
64-bit sum of the largest split cannot overflow.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_17439_gb300", "csrc")

PROGRAM = r"""
#include "ozaki_mixed.h"
#include <cmath>
#include <cstdio>
using namespace mgw::oz;
int main() {
  const int max_nch = (int)(kMixedMaxK / (kCkb * BK));
  for (int nch = 1; nch <= max_nch; ++nch) {
    for (int l = 2; l <= kWinTop; ++l) {
      const int products = l == 2 ? 1 : 2;
      int start = 0;
      for (int c = 0; c < nch; ++c) {
        if (!window_end(c, l, nch)) continue;
        const double terms = (double)(c - start + 1) * products * kCkb * BK;
        if (terms * 16384.0 > 16777216.0) { printf("window %d..%d of level %d, nch %d\n", start, c, l, nch); return 1; }
        start = c + 1;
      }
      if (start != nch) { printf("level %d leaves chunks after %d of %d\n", l, start, nch); return 2; }
    }
    for (int c = 0; c + 1 < nch; ++c) {
      int ends = 0;
      for (int l = 2; l <= kWinTop; ++l) ends += window_end(c, l, nch) ? 1 : 0;
      if (ends > 2) { printf("%d windows end at chunk %d of %d\n", ends, c, nch); return 3; }
    }
  }
  // |sum| < 2^14 K 2^32 (1 + 2^-7) in units of 2^-32 for the largest split
  if (!(std::ldexp(1.0, 14) * (double)kMixedMaxK * std::ldexp(1.0, 32) * (1.0 + std::ldexp(1.0, -7)) <
        std::ldexp(1.0, 63))) return 4;
  printf("ok %d\n", max_nch);
  return 0;
}
"""


def test_mixed_kernel_windows_stay_exact(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "windows.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "windows"
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include")]
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", *inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, run.stdout
    assert run.stdout.startswith("ok 512")
