"""The operand image of the tensor-core smoother (tc_image in
paper_2205_05840_gb300/csrc/tc_patch.cu), built by a host program and checked
on the CPU.

The brick kernel multiplies the gathered patch residuals by W (108 x 60, the
Gram factor of the vertex-patch operator, eq. vertex space) and the result by
W^t on the tensor cores, with operands in the K-major layout of 8 x 8-element
core matrices (16-byte rows).  The set-up writes, per level, one image: B1 =
W^t scaled by sw (N = 64, K = 112), B2 = W scaled by sw2 = 4096 sw (N = 112,
K = 64), each rounded to fp16 or bf16 and zero-padded, the float 1 / (sw sw2)
after them, and B2's low-order part (W sw2 minus its rounding, rounded again)
for the second product.  The test compiles the kernel's translation unit into
a host program (nothing is launched), reads every element back through the
kernel's own layout function, and compares with W rounded by NumPy (IEEE
round-to-nearest-even).  It also checks the kernel's compile-time index maps
against the set-up's box numbering (the row order of W): the region element
the kernel gathers for patch-local edge l is that box edge, the staged region's
octant layout is a bijection, and a whole-vertex shift moves an octant index by
a fixed stride, as the gather and scatter assume."""
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
#include "tc_patch.cu"   // this translation unit: its file-local image builder and layout function
using namespace ndmg;
static void wr(const std::string& p, const void* v, size_t bytes) {
  FILE* f = fopen(p.c_str(), "wb"); fwrite(v, 1, bytes, f); fclose(f);
}
// the kernel's compile-time maps against the set-up's box numbering: per
// patch-local edge l its direction and region coordinates (local_*), the
// set-up's box coordinates of l (Box::index), the octant-layout index of the
// region element and of the same element shifted by a whole vertex (2 cells)
static int maps(const std::string& dir) {
  std::vector<int> out;
  const Box vb{{4, 4, 4}};
  for (int l = 0; l < 108; ++l) {
    int bd = -1, bi = -1, bj = -1, bk = -1;
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k <= 4; ++k)
        for (int j = 0; j <= 4; ++j)
          for (int i = 0; i <= 4; ++i)
            if (vb.index(d, i, j, k) == l) { bd = d; bi = i; bj = j; bk = k; }
    out.insert(out.end(), {local_dir(l), local_ri(l), local_rj(l), local_rk(l), bd, bi, bj, bk});
  }
  wr(dir + "/local.bin", out.data(), out.size() * sizeof(int));
  // region: every (d, i, j, k) with its octant index, and the brick extents
  std::vector<int> reg;
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < dir_len(d, 2); ++k)
      for (int j = 0; j < dir_len(d, 1); ++j)
        for (int i = 0; i < dir_len(d, 0); ++i) reg.insert(reg.end(), {d, i, j, k, region_at_c(d, i, j, k)});
  wr(dir + "/region.bin", reg.data(), reg.size() * sizeof(int));
  constexpr RegionTable tab = make_region_table();
  wr(dir + "/table.bin", tab.v, sizeof(tab.v));
  printf("%d %d %d %d %d %d %d\n", kBX, kBY, kBZ, kCX, kCY, kCZ, kRegionAll);
  return 0;
}
int main(int argc, char** argv) {
  const std::string dir = argv[1];
  if (std::string(argv[2]) == "maps") return maps(dir);
  const int n = atoi(argv[2]);
  const double alpha = atof(argv[3]);
  const bool fp16 = atoi(argv[4]) != 0;
  LocalOps ops;
  build_local_ops(n, 1.0, alpha, 1.0, &ops, 2);
  std::vector<uint8_t> img(kImgStride + kLoBytes, 0xAB);
  tc_image(ops.Wv.data(), fp16, img.data(), img.data() + kImgStride);
  // every element read back through the layout function: B1 [64][112],
  // B2 [112][64], lo [112][64] (16-bit words), then the scale
  std::vector<uint16_t> b1(kN1 * kK1), b2(kN2 * kK2), lo(kN2 * kK2);
  for (int r = 0; r < kN1; ++r)
    for (int k = 0; k < kK1; ++k) std::memcpy(&b1[r * kK1 + k], img.data() + core_off(r, k, kK1), 2);
  for (int r = 0; r < kN2; ++r)
    for (int k = 0; k < kK2; ++k) {
      std::memcpy(&b2[r * kK2 + k], img.data() + kN1 * kK1 * 2 + core_off(r, k, kK2), 2);
      std::memcpy(&lo[r * kK2 + k], img.data() + kImgStride + core_off(r, k, kK2), 2);
    }
  float inv;
  std::memcpy(&inv, img.data() + kImgBytes, sizeof(float));
  wr(dir + "/W.bin", ops.Wv.data(), ops.Wv.size() * sizeof(double));
  wr(dir + "/b1.bin", b1.data(), b1.size() * 2);
  wr(dir + "/b2.bin", b2.data(), b2.size() * 2);
  wr(dir + "/lo.bin", lo.data(), lo.size() * 2);
  printf("%d %d %d %.9g\n", kImgBytes, kImgStride, kLoBytes, (double)inv);
  return 0;
}
"""

SOURCES = ["setup.cpp", "kernels.cu"]


@pytest.fixture(scope="module")
def driver(host_build, tmp_path_factory):
    return host_build(DRIVER, SOURCES), str(tmp_path_factory.mktemp("tc_image_host"))


def _round_bf16(x: np.ndarray) -> np.ndarray:
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def _decode(bits: np.ndarray, fp16: bool) -> np.ndarray:
    if fp16:
        return bits.view(np.float16).astype(np.float64)
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n,alpha", [(16, 1.0), (128, 1.0), (64, 100.0)])
def test_operand_image_holds_the_rounded_gram_factor(driver, prec, n, alpha):
    exe, d = driver
    fp16 = prec == "fp16"
    out = os.path.join(d, f"run_{n}_{alpha}_{prec}")
    os.makedirs(out, exist_ok=True)
    res = subprocess.run([exe, out, str(n), repr(alpha), "1" if fp16 else "0"], check=True, capture_output=True,
                         text=True)
    img_bytes, stride, lo_bytes, inv = res.stdout.split()
    assert (int(img_bytes), int(stride), int(lo_bytes)) == ((64 * 112 + 112 * 64) * 2, (64 * 112 + 112 * 64) * 2 + 16,
                                                            112 * 64 * 2)
    W = np.fromfile(os.path.join(out, "W.bin")).reshape(108, 60)
    b1 = _decode(np.fromfile(os.path.join(out, "b1.bin"), dtype=np.uint16), fp16).reshape(64, 112)
    b2 = _decode(np.fromfile(os.path.join(out, "b2.bin"), dtype=np.uint16), fp16).reshape(112, 64)
    lo = _decode(np.fromfile(os.path.join(out, "lo.bin"), dtype=np.uint16), fp16).reshape(112, 64)
    rnd = (lambda x: x.astype(np.float16).astype(np.float64)) if fp16 else _round_bf16
    sw = 2.0 ** -np.ceil(np.log2(np.abs(W).max()))
    sw2 = 4096.0 * sw
    # B1 = W^t sw and B2 = W sw2, rounded; the padding rows and columns are 0
    assert np.array_equal(b1[:60, :108], rnd(W.T * sw)) and not b1[60:].any() and not b1[:, 108:].any()
    assert np.array_equal(b2[:108, :60], rnd(W * sw2)) and not b2[108:].any() and not b2[:, 60:].any()
    # the low-order part of B2, and what the two parts carry together
    assert np.array_equal(lo[:108, :60], rnd(W * sw2 - rnd(W * sw2))) and not lo[108:].any() and not lo[:, 60:].any()
    bits = 11 if fp16 else 8
    two = b2[:108, :60] + lo[:108, :60]
    assert np.abs(two - W * sw2).max() <= 2.0 ** (-2 * bits + 1) * np.abs(W * sw2).max()
    # the scale after both images undoes sw sw2
    assert float(inv) == float(np.float32(1.0 / (sw * sw2)))
    # max |W sw| in (1/2, 1]
    assert 0.5 < np.abs(W * sw).max() <= 1.0


def test_kernel_index_maps_agree_with_the_setup_numbering(driver):
    # the brick kernel gathers patch-local edge l of the patch at brick vertex
    # (a, b, c) from region element (local_r*(l) + 2 (a, b, c)) of direction
    # local_dir(l); W's row l belongs to the set-up's box edge l.  The two
    # must be the same edge: region = box coordinates - (0 along, 1 across),
    # and the octant layout must take a whole-vertex shift to a fixed stride
    exe, d = driver
    out = os.path.join(d, "maps")
    os.makedirs(out, exist_ok=True)
    res = subprocess.run([exe, out, "maps"], check=True, capture_output=True, text=True)
    BX, BY, BZ, CX, CY, CZ, nreg = map(int, res.stdout.split())
    assert (BX * BY * BZ, CX, CY, CZ) == (128, 2 * BX + 2, 2 * BY + 2, 2 * BZ + 2)
    loc = np.fromfile(os.path.join(out, "local.bin"), dtype=np.int32).reshape(108, 8)
    for l, (ld, ri, rj, rk, bd, bi, bj, bk) in enumerate(loc):
        assert ld == bd, l
        across = [1, 1, 1]
        across[bd] = 0
        assert (ri, rj, rk) == (bi - across[0], bj - across[1], bk - across[2]), l
    reg = np.fromfile(os.path.join(out, "region.bin"), dtype=np.int32).reshape(-1, 5)
    assert reg.shape[0] == nreg and sorted(reg[:, 4]) == list(range(nreg))     # octant layout: a bijection
    at = {tuple(r[:4]): r[4] for r in reg}
    ext = {0: (CX, CY - 1, CZ - 1), 1: (CX - 1, CY, CZ - 1), 2: (CX - 1, CY - 1, CZ)}
    for dd in range(3):
        assert sum(1 for r in reg if r[0] == dd) == int(np.prod(ext[dd]))
    # every patch edge of every brick vertex lies in the region, and a shift by
    # one vertex (2 cells) along an axis moves its octant index by a constant
    for ld, ri, rj, rk, *_ in loc:
        base = at[(ld, ri, rj, rk)]
        step = [at[(ld, ri + 2, rj, rk)] - base, at[(ld, ri, rj + 2, rk)] - base, at[(ld, ri, rj, rk + 2)] - base]
        for a in range(BX):
            for b in range(BY):
                for c in range(BZ):
                    assert at[(ld, ri + 2 * a, rj + 2 * b, rk + 2 * c)] == base + a * step[0] + b * step[1] + c * step[2]
    # the walking table lists the region in canonical order with its octant index
    tab = np.fromfile(os.path.join(out, "table.bin"), dtype=np.uint32)
    assert tab.size == nreg
    for q, r in enumerate(reg):
        e = int(tab[q])
        assert (e & 0x1FFF, (e >> 13) & 31, (e >> 18) & 15, e >> 22) == (r[4], r[1], r[2], r[3])
