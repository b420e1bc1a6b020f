"""Rounding noise floor of the FP64 oracle (test infrastructure; calls only the
oracle).

Runs the oracle on a workload once exactly and then `seeds` times with the
ulp-jitter probe on (every correlation value multiplied by 1 +- 2^-52, a
counter-based choice per location and call), and reports how far rounding
alone moves the results:
  - the fraction of locations whose selected-index sequence changes under at
    least one seed, and the oracle's own decision gap at the first step where
    it changes (a change at a wide gap would show the gap bookkeeping wrong);
  - over the locations whose sequences never change, the largest and median
    relative change of the predictive mean and of s2.
This is the spread that any second implementation of the same method can
differ by, unless it reproduces the oracle's arithmetic operation for
operation, as the FP64 GPU form does.

    python -m oracle.noise_floor [--seeds 4] [--m4 200] [--m8 64]
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1409_0074_gb300 import workloads as W  # noqa: E402


def spread(w, search, nrays, seeds, nthreads=0):
    base = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search,
                          nrays=nrays, nthreads=nthreads)
    changed = np.zeros(w.M, bool)
    gap_at_change = []
    dmean = np.zeros(w.M)
    ds2 = np.zeros(w.M)
    try:
        for sd in range(1, seeds + 1):
            oracle.set_jitter(0x5eed0000 + sd)
            r = oracle.predict(w.X, w.Y, w.Xref, w.n0, w.n, w.nc, w.theta, w.g, search,
                               nrays=nrays, nthreads=nthreads)
            for m in range(w.M):
                diff = np.nonzero(r["selected"][m] != base["selected"][m])[0]
                if diff.size:
                    if not changed[m]:
                        gap_at_change.append(float(base["gap"][m, diff[0] - w.n0]))
                    changed[m] = True
            dmean = np.maximum(dmean, np.abs(r["mean"] - base["mean"]) / np.abs(base["mean"]))
            ds2 = np.maximum(ds2, np.abs(r["s2"] - base["s2"]) / base["s2"])
    finally:
        oracle.set_jitter(0)
    keep = ~changed
    return {"workload": w.name, "search": search, "locations": int(w.M), "seeds": seeds,
            "changed_selection_frac": float(changed.mean()),
            "gap_at_first_change_max": max(gap_at_change) if gap_at_change else None,
            "gap_at_first_change_median": (float(np.median(gap_at_change))
                                           if gap_at_change else None),
            "mean_rel_change_max": float(dmean[keep].max()) if keep.any() else None,
            "mean_rel_change_median": float(np.median(dmean[keep])) if keep.any() else None,
            "s2_rel_change_max": float(ds2[keep].max()) if keep.any() else None,
            "s2_rel_change_median": float(np.median(ds2[keep])) if keep.any() else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--m4", type=int, default=200, help="locations of the 4-d workload")
    ap.add_argument("--m8", type=int, default=64, help="locations of the 8-d workload")
    a = ap.parse_args()
    out = []
    w2 = W.dense_2d(M=100)
    out.append(spread(w2, "exhaustive", 2, a.seeds))
    out.append(spread(w2, "ray", 2, a.seeds))
    w4 = W.paper_scale_4d(M=a.m4)
    out.append(spread(w4, "exhaustive", 4, a.seeds))
    out.append(spread(w4, "ray", 4, a.seeds))
    w8 = W.large_8d(M=a.m8)
    out.append(spread(w8, "exhaustive", 8, a.seeds))
    out.append(spread(w8, "ray", 8, a.seeds))
    for o in out:
        print(json.dumps(o))


if __name__ == "__main__":
    main()
