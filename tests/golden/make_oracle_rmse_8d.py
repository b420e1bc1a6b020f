"""Writes tests/golden/oracle_rmse_sinusoid8d.txt: the FP64 oracle's
out-of-sample RMSE over all 100,000 predictive locations of the 8-d workload
(N = 1e6, p = 8, n0 = 6, n = 50, N' = 1000, theta = 1, g = 1e-6), for ray
search with 8 rays and for exhaustive search.  The GPU tests compare the
FP32-scoring form's RMSE over the same locations with these values, so that
the 1% bar is checked without sampling noise.

Calls only the oracle (and the seeded input generator).  The oracle is plain
binary64 C without contraction, so the values do not depend on the host.
Takes hours on a few cores:
    python tests/golden/make_oracle_rmse_8d.py [--threads T] [--search ray|exhaustive]
                                               [--out PATH]
With --search, only that search's line of the output file is (re)written.
"""
import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1409_0074_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_rmse_sinusoid8d.txt")


HEADER = ["# FP64 oracle over all 100,000 locations of the 8-d workload",
          "# (python tests/golden/make_oracle_rmse_8d.py); search rmse locations status_bad"]


def oracle_rmse(w, search, threads):
    err2, bad = 0.0, 0
    for c0 in range(0, w.M, 2000):
        r = oracle.predict(w.X, w.Y, w.Xref[c0:c0 + 2000], w.n0, w.n, w.nc, w.theta, w.g,
                           search, nrays=8, nthreads=threads)
        err2 += float(np.sum((r["mean"] - w.Ytrue[c0:c0 + 2000]) ** 2))
        bad += int(np.sum(r["status"] != 0))
        print(search, c0 + 2000, flush=True)
    return "%s %.17g %d %d" % (search, np.sqrt(err2 / w.M), w.M, bad)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--search", choices=["ray", "exhaustive"], default=None)
    ap.add_argument("--out", default=OUT)
    a = ap.parse_args()
    w = W.large_8d(M=100_000)
    rows = {}
    if os.path.exists(a.out):
        for line in open(a.out):
            if line.strip() and not line.startswith("#"):
                rows[line.split()[0]] = line.strip()
    for search in ([a.search] if a.search else ["ray", "exhaustive"]):
        rows[search] = oracle_rmse(w, search, a.threads)
        with open(a.out, "w") as fh:
            fh.write("\n".join(HEADER + [rows[k] for k in ("ray", "exhaustive") if k in rows])
                     + "\n")


if __name__ == "__main__":
    main()
