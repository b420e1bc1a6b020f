"""Host-side pieces of bench.py that decide what the bench line reports: the
algorithmic bytes of the exhaustive scorer and the source hash that keeps a
committed DRAM capture valid (CPU only)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_exhaustive_bytes_by_brute_force():
    """Per location: step m = 1..n reads rows 0..m-1 of the N' - m unselected
    candidates' cache columns and writes one row of N'; the candidate rows
    (PP floats each) are read once.  Counted here element by element."""
    n, nc, PP = 7, 40, 4
    reads = 0
    for m in range(1, n + 1):
        for _cand in range(nc - m):
            reads += m
    want = 4 * (reads + n * nc + PP * nc)
    got = bench.kernel_bytes("design32_exhaustive", dict(n=n, nc=nc, PP=PP, M_launch=3))
    assert got == 3 * want
    assert bench.kernel_bytes("ray32", dict(n=n, nc=nc, PP=PP, M_launch=3)) is None


def test_exhaustive_bytes_at_the_bench_workload():
    per_loc = bench.kernel_bytes("design32_exhaustive", dict(n=50, nc=1000, PP=8, M_launch=1))
    assert per_loc == pytest.approx(5.16e6, rel=1e-3)


def test_source_hash_ignores_comments_only():
    a = "int f(int x) {  // add one\n  return x + 1;\n}\n"
    b = "// header comment\n\nint f(int x) {  // plus one\n  return x + 1;   \n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.source_hash([a]) == bench.source_hash([b])
    assert bench.source_hash([a]) != bench.source_hash([c])
    assert bench.source_hash([a, c]) != bench.source_hash([c, a])


def test_committed_captures_are_read():
    """Each committed capture yields its own figure while the code matches,
    and nothing otherwise (never another figure)."""
    for path, key, fn in [("design32_sinusoid8d_M20000.md", "traffic_bytes_per_location",
                           bench.design32_traffic_per_location),
                          ("ray32_sinusoid8d_N1e6_M1e5_dram.md", "traffic_bytes_per_launch",
                           bench.ray32_traffic)]:
        text = open(os.path.join(ROOT, "profiles", path)).read()
        stored = float(next(l.split(": ", 1)[1] for l in text.splitlines()
                            if l.startswith(key + ": ")))
        assert stored > 0
        assert fn() in (None, stored)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and
    prints one JSON line with the arm's metric, unit and config, marked
    impl = reference, with its own cpu_baseline and a zero-copy e2e."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"].startswith("locations/sec") and d["unit"] == "locations/s"
    assert d["config"]["workload"] == "sinusoid_8d_N1000000_n50"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_ray_flops_follow_the_algorithmic_count():
    """A ray launch counts 2 j^2 + (3p + 4) j per ALC evaluation at design size
    j and N' x 3p per greedy step (the snap), summed here evaluation by
    evaluation; the executed triangular form j^2 + j + 4 j + (3p + 2) j is the
    second figure."""
    import numpy as np
    nev = np.array([[3, 5, 0], [4, 1, 2]], dtype=np.float64)   # 2 locations, j = 2, 3, 4
    n0, p, nc = 2, 3, 20
    ev = bench.eval_sums(nev, n0)
    want_algo = want_tri = 0
    for row in nev:
        for j, e in zip((2, 3, 4), row):
            want_algo += e * (2 * j * j + (3 * p + 4) * j) + nc * 3 * p
            want_tri += e * (j * j + j + 4 * j + (3 * p + 2) * j) + nc * 3 * p
    shape = dict(N=100, p=p, n0=n0, n=5, nc=nc, PP=4, M_launch=2)
    algo, tri = bench.kernel_flops("ray32", shape, ev)
    assert algo == want_algo and tri == want_tri
    algo64, tri64 = bench.kernel_flops("design64_ray", shape, ev)
    assert algo64 == want_algo and tri64 is None


def test_exhaustive_fp64_flops_by_brute_force():
    n0, n, nc, p = 2, 5, 9, 2
    want = 0
    for j in range(n0, n):
        for _cand in range(nc - j):
            want += 2 * j * j + (3 * p + 4) * j
    got, _ = bench.kernel_flops("design64_exhaustive",
                                dict(N=50, p=p, n0=n0, n=n, nc=nc, PP=4, M_launch=3), None)
    assert got == 3 * want
