"""Host-side launch arithmetic of the kNN filter and the ray kernel
(csrc/launch_plan.h), compiled with the host C++ compiler and checked on the
CPU: which location tiles of the tensor-core kNN filter run unsplit and how
the rest are split over the design, and how many warps per CTA the ray kernel
takes by default."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1409_0074_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <initializer_list>
#include "launch_plan.h"
int main() {
  long long sms[] = {152, 148, 132, 8};
  for (long long s : sms)
    for (long long dt : {7813LL, 4000LL, 100LL, 63LL})
      for (long long t = 0; t <= 2000; ++t) {
        int64_t body = -1, nseg = -1;
        lagp::knn_tc_plan(t, s, dt, &body, &nseg);
        std::printf("K %lld %lld %lld %lld %lld\n", s, dt, t, (long long)body, (long long)nseg);
      }
  for (long long wb : {3536LL, 7440LL, 10752LL, 11216LL, 11280LL, 11968LL, 16144LL, 31600LL})
    std::printf("W %lld %d\n", wb, lagp::warps_per_cta_for_residency((size_t)wb, 233472, 1024, 20));
  return 0;
}
"""


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("plan")
    src, exe = d / "plan.cpp", d / "plan"
    src.write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    knn = [tuple(int(v) for v in l.split()[1:]) for l in out.splitlines() if l.startswith("K ")]
    warps = {int(l.split()[1]): int(l.split()[2]) for l in out.splitlines() if l.startswith("W ")}
    return knn, warps


def test_knn_tiles_are_covered_and_split_within_bounds(plan):
    knn, _ = plan
    for sms, dt, tiles, body, nseg in knn:
        assert 0 <= body <= tiles and nseg >= 1
        rest = tiles - body
        if rest == 0:
            assert nseg == 1
            continue
        # a split keeps at least 64 design tiles per segment and two segments
        assert 2 <= nseg <= dt // 64 and nseg <= 65535
        if tiles >= sms:
            # whole waves unsplit; the split tiles fill at most one wave
            assert body % sms == 0 and rest == tiles % sms and rest * nseg <= sms
        else:
            assert body == 0


def test_knn_plan_never_takes_more_waves_than_unsplit(plan):
    knn, _ = plan
    for sms, dt, tiles, body, nseg in knn:
        if tiles == 0:
            continue
        rest = tiles - body
        waves = body / sms + (-(-rest * nseg // sms)) / nseg
        assert waves <= -(-tiles // sms) + 1e-12, (sms, dt, tiles, body, nseg)


def test_knn_plan_known_sizes(plan):
    """The 100,000- and 40,000-location batches on 152 SMs with N = 1e6
    (7,813 design tiles): 760 tiles unsplit and 22 split six ways; 304 and 9
    split sixteen ways.  A one-tile batch splits 122 ways (the 64-tile floor)."""
    knn, _ = plan
    got = {(s, dt, t): (b, n) for s, dt, t, b, n in knn}
    assert got[(152, 7813, 782)] == (760, 6)
    assert got[(152, 7813, 313)] == (304, 16)
    assert got[(152, 7813, 1)] == (0, 122)
    assert got[(152, 7813, 760)] == (760, 1)
    assert got[(152, 100, 782)] == (782, 1)      # too few design tiles to split


def test_ray_warps_follow_residency(plan):
    _, warps = plan
    # 233,472 bytes per SM, 1,024 reserved per CTA, at most 20 warps
    assert warps[11280] == 4      # 5 x (4 x 11280 + 1024) fits: 20 warps; 2 per CTA gives 18
    assert warps[10752] == 2      # 20 warps either way: the tie goes to 2
    assert warps[3536] == 2
    assert warps[31600] == 1      # 7 warps alone, 6 in pairs, 4 in fours
    for wb, rw in warps.items():
        res = {c: min(233472 // (c * wb + 1024), 20 // c) * c for c in (1, 2, 4)}
        assert res[rw] == max(res.values())
