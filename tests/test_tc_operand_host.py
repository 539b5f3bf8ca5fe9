"""The set-up's check of the tensor-core operands (tc_operand_spectral_max in
paper_2205_05840_gb300/csrc/tc_patch.cu), built by a host program and checked
on the CPU.

The mixed-precision smoother applies the vertex-patch operator as W W^t with
W the Gram factor rounded to bf16 or fp16 (scaled by a power of two).  For the
exact W, A_p W W^t is a projection (largest eigenvalue 1); rounded operands
raise that eigenvalue as the patch matrix A_p grows ill-conditioned
(~ alpha / (beta h^2)) and as the rounding errors of W's entries happen to
fall, and the library refuses a handle whose value passes 16.  The test rebuilds the rounded factor in NumPy (IEEE round-to-nearest-even
to fp16, and to bf16 from the exact binary expansion, after the same power-of-
two scaling), computes the largest eigenvalue of W~^t A_p W~ with LAPACK, and
compares it with the library's power iteration; it also checks the projection
property of the exact factor.  No kernel is launched, so no GPU is needed."""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_05840_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "tc_patch.cuh"
using namespace ndmg;
static void wr(const std::string& p, const std::vector<double>& v) {
  FILE* f = fopen(p.c_str(), "wb"); fwrite(v.data(), sizeof(double), v.size(), f); fclose(f);
}
int main(int argc, char** argv) {
  const std::string dir = argv[1];
  const int n = atoi(argv[2]);
  const double L = atof(argv[3]), alpha = atof(argv[4]), beta = atof(argv[5]);
  LocalOps ops;
  build_local_ops(n, L, alpha, beta, &ops, 2);
  const std::vector<double> Ap = box_matrix(Box{{4, 4, 4}}, L / n, alpha, beta);
  wr(dir + "/W.bin", ops.Wv);
  wr(dir + "/Ap.bin", Ap);
  printf("%.17g %.17g\n", tc_operand_spectral_max(ops.Wv.data(), Ap, true),
         tc_operand_spectral_max(ops.Wv.data(), Ap, false));
  return 0;
}
"""

SOURCES = ["setup.cpp", "kernels.cu", "tc_patch.cu"]


@pytest.fixture(scope="module")
def driver(host_build, tmp_path_factory):
    return host_build(DRIVER, SOURCES), str(tmp_path_factory.mktemp("tc_operand_host"))


def _round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bf16 (8 significant bits), ties to even, from the
    exact double (no intermediate float rounding); normal range only."""
    m, e = np.frexp(x)                 # x = m 2^e, |m| in [1/2, 1)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _lam_max(W: np.ndarray, Ap: np.ndarray) -> float:
    return float(np.linalg.eigvalsh(W.T @ Ap @ W).max())


def _power60(W: np.ndarray, Ap: np.ndarray) -> float:
    """The Rayleigh quotient after 60 power steps from x_l = 1 + 0.01 l, as
    the library's check iterates (a lower bound of the largest eigenvalue,
    slow to converge when the top of the spectrum is clustered near 1)."""
    x = 1.0 + 0.01 * np.arange(108)
    lam = 0.0
    for _ in range(60):
        ax = Ap @ x
        t = W.T @ ax
        lam = (t @ t) / (x @ ax)
        y = W @ t
        x = y / np.linalg.norm(y)
    return float(lam)


# (n, alpha): alpha / (beta h^2) = 4.1e5 on 64^3 (the GPU test's refused bf16
# case) and on 32^3 and 128^3, 2.3e5 on 64^3, and well-conditioned patches
@pytest.mark.parametrize("n,alpha", [(16, 1.0), (64, 1.0), (128, 1.0), (64, 56.0), (64, 100.0), (32, 400.0),
                                     (128, 25.0)])
def test_operand_spectral_check_matches_lapack(driver, n, alpha):
    exe, d = driver
    out = os.path.join(d, f"run_{n}_{alpha}")
    os.makedirs(out, exist_ok=True)
    res = subprocess.run([exe, out, str(n), "1.0", repr(alpha), "1.0"], check=True, capture_output=True, text=True)
    lam_lib = dict(zip(("fp16", "bf16"), map(float, res.stdout.split())))
    W = np.fromfile(os.path.join(out, "W.bin")).reshape(108, 60)
    Ap = np.fromfile(os.path.join(out, "Ap.bin")).reshape(108, 108)
    # the exact Gram factor: A_p W W^t is a projection
    assert abs(_lam_max(W, Ap) - 1.0) < 1e-8
    sw = 2.0 ** -np.ceil(np.log2(np.abs(W).max()))
    sw2 = 4096.0 * sw
    rounded = {"fp16": (W * sw2).astype(np.float16).astype(np.float64) / sw2,
               "bf16": _round_bf16(W * sw2) / sw2}
    for prec, Wr in rounded.items():
        lam, ref, pw = lam_lib[prec], _lam_max(Wr, Ap), _power60(Wr, Ap)
        # the library rounds exactly as modelled here: its value is the same
        # power iteration on the same rounded factor
        assert abs(lam - pw) <= 1e-9 * pw, (prec, lam, pw)
        # a lower bound of the largest eigenvalue, and close to it once that
        # eigenvalue stands apart from the rest (every case near the limit 16)
        assert 1.0 - 1e-9 <= lam <= ref * (1 + 1e-9), (prec, lam, ref)
        if ref >= 2.0:
            assert abs(lam - ref) <= 1e-4 * ref, (prec, lam, ref)
    # the refusal at set-up (largest eigenvalue above 16) follows the operand
    # bit patterns, not alpha / (beta h^2) alone: at 4.1e5 bf16 gives 23 on
    # 64^3 (refused) and 7.3 on 32^3 and 128^3 (accepted); fp16 stays below 2
    assert lam_lib["fp16"] < 2.0
    refused = lam_lib["bf16"] > 16.0
    assert refused == ((n, alpha) == (64, 100.0)), lam_lib
