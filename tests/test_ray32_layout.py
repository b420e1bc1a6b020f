"""Shared-memory layout of a warp of the FP32-scoring ray kernel
(csrc/ray32_layout.h), compiled with the host C++ compiler and checked on the
CPU for every shape the kernel is built for: each region starts 16-byte
aligned, the regions are disjoint and inside the warp's bytes, and the
coefficient region is large enough for each of its three uses in turn (the
rays' exponent coefficients c_k and b_k, the k-d tree walk's node stack and box
distances, and the factor update's two binary64 vectors of n entries)."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1409_0074_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "ray32_layout.h"
int main() {
  const int rps[] = {2, 4, 8, 16}, pps[] = {4, 8, 12, 16}, ncs[] = {1, 31, 32, 33, 1000, 2000, 4096};
  for (int n = 1; n <= 128; ++n)
    for (int RP : rps)
      for (int PP : pps)
        for (int nc : ncs) {
          const lagp::WarpLayout w = lagp::warp_layout(n, PP, RP, nc);
          std::printf("%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %d\n", n, PP, RP,
                      nc, w.lf, w.kz, w.cb, w.zf, w.tau, w.x, w.gsel, w.stk, w.bnd, w.starts, w.mask,
                      w.smask, w.vm, w.bytes, lagp::roff(n), lagp::kz_ld(n), KD_STACK);
        }
  return 0;
}
"""

FIELDS = ("n PP RP nc lf kz cb zf tau x gsel stk bnd starts mask smask vm bytes "
          "roff_n kzld kd").split()


@pytest.fixture(scope="module")
def layouts(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    kd = re.search(r"#define KD_STACK (\d+)", open(os.path.join(CSRC, "kdtree.cuh")).read())
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout.cpp", d / "layout"
    src.write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O1", "-DKD_STACK=" + kd.group(1), "-I", CSRC, str(src),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [dict(zip(FIELDS, map(int, l.split()))) for l in out.splitlines()]


def test_regions_are_aligned_disjoint_and_inside(layouts):
    for w in layouts:
        n, RP, PP, nc = w["n"], w["RP"], w["PP"], w["nc"]
        cb_words = max(2 * RP * w["kzld"], 2 * w["kd"])
        # (start, words) of every region the kernel addresses, in 4-byte words
        regions = {
            "lf": (w["lf"], w["roff_n"]),              # rows 0..n-1, each padded to a quad
            "kz": (w["kz"], RP * w["kzld"]),
            "cb": (w["cb"], cb_words),
            "zf": (w["zf"], n),
            "tau": (w["tau"], RP),
            "x": (w["x"], 4 * PP),                     # xf, lof, hif, xs
            "gsel": (w["gsel"], n),
            "starts": (w["starts"], RP),
            "mask": (w["mask"], (nc + 31) // 32),
            "smask": (w["smask"], (nc + 31) // 32),
            "vm": (w["vm"], 2),                        # one double
        }
        spans = sorted(regions.values())
        for (s0, n0), (s1, _) in zip(spans, spans[1:]):
            assert s0 + n0 <= s1, w
        for name, (s, words) in regions.items():
            assert s % 4 == 0, (name, w)               # 16-byte aligned
            assert s + words <= w["bytes"] // 4, (name, w)
        assert w["bytes"] % 16 == 0


def test_coefficient_region_holds_each_of_its_uses(layouts):
    for w in layouts:
        n, RP = w["n"], w["RP"]
        cb_words = max(2 * RP * w["kzld"], 2 * w["kd"])
        # c_k and b_k rows of every ray
        assert 2 * RP * w["kzld"] <= cb_words
        # the k-d walk: KD_STACK nodes, then KD_STACK box distances
        assert w["stk"] == w["cb"] and w["bnd"] == w["cb"] + w["kd"]
        assert 2 * w["kd"] <= cb_words
        # k_j(x_new) and L^{-1} k_j(x_new): 2 n doubles, 8-byte aligned
        assert 4 * n <= cb_words and w["cb"] % 2 == 0


def test_row_storage_arithmetic(layouts):
    """roff(i) is the start of row i when rows 0..i-1 are padded to quads, and
    the kz row stride is a quad multiple of at least n with an odd quad count."""
    seen = set()
    for w in layouts:
        n = w["n"]
        if n in seen:
            continue
        seen.add(n)
        assert w["roff_n"] == sum((i + 4) & ~3 for i in range(n))
        k = w["kzld"]
        assert k >= n and k % 4 == 0 and (k // 4) % 2 == 1 and k - n < 8
