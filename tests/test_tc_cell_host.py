"""The cell-owned tensor-core smoother's geometry and operand image
(paper_2205_05840_gb300/csrc/tc_cell.cu), built by a host program and checked
on the CPU.

In the cell-owned form every fine edge belongs to the coarse cell of its lowest
node, at one of 24 slots; the 108 edges of the vertex patch of V are the slots
of the 8 cells V + o, o in {-1, 0}^3, that the patch holds, and the kernel
applies W^t and W (the Gram factor of the vertex-space operator, eq. vertex
space) as sums over those 8 neighbours with per-neighbour blocks W'_o of W.
The test compiles the kernel's translation unit into a host program (nothing is
launched) and checks, with the kernel's own slot tables and image builder and
the set-up's box numbering: the 8 neighbours' unmasked slots name every patch
edge exactly once; the first six positions are the interior-space edges in the
order of the 6 x 6 interior operator; every GEMM1 and GEMM2 block of the image
holds W'_o, i.e. the rounded, scaled rows of W at those edges, and zero where a
neighbour holds no patch edge."""
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
#include "tc_cell.cu"   // this translation unit: its slot tables, layout and image builder
using namespace ndmg;
static void wr(const std::string& p, const void* v, size_t bytes) {
  FILE* f = fopen(p.c_str(), "wb"); fwrite(v, 1, bytes, f); fclose(f);
}
int main(int argc, char** argv) {
  const std::string dir = argv[1];
  const int n = atoi(argv[2]);
  const bool fp16 = atoi(argv[3]) != 0;
  // slot geometry: per neighbour J (bit e: offset -1 along axis e) and
  // position p: slot, masked?, patch-local edge
  std::vector<int> geo;
  for (int J = 0; J < 8; ++J)
    for (int p = 0; p < 24; ++p) {
      const int s = pos_slot(p);
      const int o[3] = {(J & 1) ? -1 : 0, (J & 2) ? -1 : 0, (J & 4) ? -1 : 0};
      const bool masked = (slot_zero_mask(s) & J) != 0;
      geo.insert(geo.end(), {J, p, s, masked ? 1 : 0, patch_local(s, o)});
    }
  wr(dir + "/geo.bin", geo.data(), geo.size() * sizeof(int));
  // the interior-space positions in the set-up's 2 x 2 x 2 box numbering
  std::vector<int> bub;
  for (int p = 0; p < 6; ++p) {
    const int s = pos_slot(p);
    bub.push_back((int)Box{{2, 2, 2}}.index(slot_d(s), slot_par(s, 0), slot_par(s, 1), slot_par(s, 2)));
  }
  wr(dir + "/bub.bin", bub.data(), bub.size() * sizeof(int));
  // the image: GEMM1 blocks [J][i] of 64 x 16 (value, position), GEMM2
  // blocks [J] of g2_n(J) x 64
  LocalOps ops;
  build_local_ops(n, 1.0, 1.0, 1.0, &ops, 2);
  const std::vector<uint8_t> img = tc_cell_image(ops.Wv, fp16);
  std::vector<int> g1;   // J, i, c, k, position, bits
  for (int J = 0; J < 8; ++J)
    for (int i = 0; i < g1_count(J); ++i) {
      const uint8_t* blk = img.data() + (size_t)(g1_block(J) + i) * 2048;
      const int sl[2] = {g1_first(J, i), g1_second(J, i)};
      for (int c = 0; c < 64; ++c)
        for (int k = 0; k < 16; ++k) {
          uint16_t b;
          std::memcpy(&b, blk + core_off(c, k, 16), 2);
          g1.insert(g1.end(), {J, i, c, k, 8 * sl[k >> 3] + (k & 7), (int)b});
        }
    }
  wr(dir + "/g1.bin", g1.data(), g1.size() * sizeof(int));
  std::vector<int> g2;   // J, p, c, bits
  for (int J = 0; J < 8; ++J) {
    const uint8_t* blk = img.data() + kG1Bytes + g2_off(J);
    for (int p = 0; p < g2_n(J); ++p)
      for (int c = 0; c < 64; ++c) {
        uint16_t b;
        std::memcpy(&b, blk + core_off(p, c, 64), 2);
        g2.insert(g2.end(), {J, p, c, (int)b});
      }
  }
  wr(dir + "/g2.bin", g2.data(), g2.size() * sizeof(int));
  wr(dir + "/W.bin", ops.Wv.data(), ops.Wv.size() * sizeof(double));
  float inv;
  std::memcpy(&inv, img.data() + kImgBytes, sizeof(float));
  printf("%zu %d %.9g\n", img.size(), kImgBytes, (double)inv);
  return 0;
}
"""

SOURCES = ["setup.cpp", "kernels.cu"]


@pytest.fixture(scope="module")
def driver(host_build, tmp_path_factory):
    return host_build(DRIVER, SOURCES), str(tmp_path_factory.mktemp("tc_cell_host"))


def _decode(bits: np.ndarray, fp16: bool) -> np.ndarray:
    bits = bits.astype(np.uint16)
    if fp16:
        return bits.view(np.float16).astype(np.float64)
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _round(x: np.ndarray, fp16: bool) -> np.ndarray:
    if fp16:
        return x.astype(np.float16).astype(np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0), e - 8)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_cell_owned_geometry_and_image(driver, prec):
    exe, d = driver
    fp16 = prec == "fp16"
    out = os.path.join(d, prec)
    os.makedirs(out, exist_ok=True)
    res = subprocess.run([exe, out, "32", "1" if fp16 else "0"], check=True, capture_output=True, text=True)
    size, img_bytes, inv = res.stdout.split()
    assert int(size) == int(img_bytes) + 16
    rd = lambda name: np.fromfile(os.path.join(out, name + ".bin"), dtype=np.int32)  # noqa: E731
    geo = rd("geo").reshape(-1, 5)
    # the 24 positions of a cell are the 24 slots, each once
    slots = geo[geo[:, 0] == 0][:, 2]
    assert sorted(slots) == sorted({int(dd | a << 2 | b << 3 | c << 4) for dd in range(3) for a in (0, 1)
                                    for b in (0, 1) for c in (0, 1)})
    # the unmasked slots of the 8 neighbours are the 108 patch edges, each once
    held = geo[geo[:, 3] == 0]
    assert (held[:, 4] >= 0).all()
    assert sorted(held[:, 4]) == list(range(108))
    # the first six positions: the interior-space edges in the 6 x 6 operator's order
    assert list(rd("bub")) == list(range(6))
    # W'_J from the image against W rounded
    W = np.fromfile(os.path.join(out, "W.bin")).reshape(108, 60)
    sw = 2.0 ** -np.ceil(np.log2(np.abs(W).max()))
    assert float(inv) == float(np.float32(1.0 / (sw * sw)))
    want = np.zeros((8, 32, 64))                     # GEMM2 blocks pad positions 24..31 with 0
    for J, p, s, masked, l in geo:
        if not masked:
            want[J, p, :60] = _round(W[l] * sw, fp16)
    g1 = rd("g1").reshape(-1, 6)
    got = _decode(g1[:, 5], fp16)
    for (J, i, c, k, p, _), v in zip(g1, got):
        if i == 1 and p // 8 == 1:          # the second MMA repeats slice 1 as zeros
            assert v == 0.0
        else:
            assert v == want[J, p, c], (J, i, c, k, p)
    # every held position reaches GEMM1 through exactly one MMA slice
    seen = {(J, p) for (J, i, c, k, p, _) in g1 if not (i == 1 and p // 8 == 1)}
    assert {(J, p) for J, p, s, masked, l in geo if not masked} <= seen
    g2 = rd("g2").reshape(-1, 4)
    got2 = _decode(g2[:, 3], fp16)
    for (J, p, c, _), v in zip(g2, got2):
        assert v == want[J, p, c], (J, p, c)
    # positions beyond a neighbour's GEMM2 block hold no patch edge for it
    n2 = {J: g2[g2[:, 0] == J][:, 1].max() + 1 for J in range(8)}
    for J, p, s, masked, l in geo:
        if p >= n2[J]:
            assert masked, (J, p)
