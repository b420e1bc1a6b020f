"""Benchmark of local approximate GP prediction (Gramacy & Haaland,
arXiv:1409.0074) on one or more GB300 GPUs.

A step is one pass of the whole path -- bounding box and FP32 design copy,
kNN candidates, greedy ALC local design, predictive equations -- over one
batch of M predictive locations on the 8-d workload: N = 1e6 design points,
n0 = 6, n = 50, N' = 1000, theta = 1, g = 1e-6, ray search with p = 8 rays,
FP32 scoring and FP64 factor update.  Inputs are resident in HBM before the
timed region; a 256 MB buffer is written before every step to flush L2.

Prints one JSON line.  `value` is locations/sec over all ranks (weak scaling:
every rank predicts its own M locations; there is no collective on the data
path).  `--impl reference` times the FP64 CPU oracle instead, on a bounded
sample per step.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # SMs x FP32 lanes x FMA x max clock
FP64_PEAK_TFLOPS = 1.25                               # GB300 FP64 rate


def hbm_peak():
    """Measured copy bandwidth (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--M", type=int, default=100_000)
    ap.add_argument("--N", type=int, default=1_000_000)
    ap.add_argument("--search", default="ray", choices=["ray", "exhaustive", "ray_full"])
    ap.add_argument("--precision", default="fp32",
                    choices=["fp32", "fp32_tc", "fp64", "fp32_promote", "fp32_tc_promote"])
    ap.add_argument("--no-extras", action="store_true", help="skip the other search/precision forms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle locations (0: 32 per core)")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the uneven-size batching form (persistent kernels, CUDA graph)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving form (request stream over a serving context)")
    ap.add_argument("--serve-seconds", type=float, default=4.0,
                    help="arrival window per rate of the serving form")
    ap.add_argument("--workload", default="sinusoid_8d", choices=["sinusoid_8d", "paper_2d"],
                    help="the timed workload: the 8-d headline or the 2-d grid of Sec 5.1")
    ap.add_argument("--mle-stages", type=int, default=0, choices=[0, 1, 2],
                    help="time designs coupled with local inference for theta (one or two "
                         "stages) instead of designs at a fixed theta")
    return ap.parse_args()


def dist_init(args, backend="nccl"):
    """One process per GPU (torchrun's environment).  Locations are
    independent, so ranks share no data: each predicts its own batch (weak
    scaling); the process group carries only a barrier and the max-reduce of
    the timed region."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(M_total, rank, world):
    """Contiguous block [lo, hi) of the job's M_total locations that `rank`
    predicts; the blocks of ranks 0..world-1 are disjoint, cover the job and
    follow rank order."""
    per, extra = divmod(M_total, world)
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def rank_workload(M, N, rank, world, name="sinusoid_8d"):
    """The workload of one rank (weak scaling, M locations per rank): every
    rank draws the same design, responses and job-wide location set (seed 0,
    M * world locations) and keeps its own block of them."""
    from paper_1409_0074_gb300 import workloads as W
    if name == "paper_2d":
        w = W.paper_2d(M=min(M * world, 9801))
    else:
        w = W.large_8d(M=M * world, N=N)
    lo, hi = shard(w.M, rank, world)
    w.Xref, w.Ytrue, w.M = w.Xref[lo:hi], w.Ytrue[lo:hi], hi - lo
    return w


def whole_job_rate(units_per_rank, steps, ms, world):
    """Units per second of the whole job: all ranks' units over the slowest
    rank's time.  Returns (rate, slowest ms)."""
    ms_max = max_over_ranks(ms, world)
    return world * units_per_rank * steps / (ms_max / 1e3), ms_max


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def profile_traffic(profile, sources, key):
    """DRAM bytes from a committed ncu summary (the value of `key`), or None
    when the kernel's sources changed since that capture."""
    root = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(root, "profiles", profile)
    try:
        fields = dict(l.split(": ", 1) for l in open(path).read().splitlines() if ": " in l and
                      l.split(": ", 1)[0] in (key, "source_sha256_16"))
        csrc = os.path.join(root, "paper_1409_0074_gb300", "csrc")
        if source_hash([open(os.path.join(csrc, f)).read() for f in sources]) != \
                fields["source_sha256_16"].strip():
            return None
        return float(fields[key])
    except (OSError, KeyError, ValueError):
        return None


def source_hash(texts):
    """First 16 hex digits of the sha256 of the sources' code: `//` comments,
    trailing blanks and empty lines removed, so that a comment edit keeps a
    capture valid and any code change voids it."""
    import hashlib
    h = hashlib.sha256()
    for t in texts:
        for line in t.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def ray32_traffic():
    """DRAM bytes of one full-size ray32 launch (100,000 locations)."""
    return profile_traffic("ray32_sinusoid8d_N1e6_M1e5_dram.md",
                           ("ray32.cu", "ray32_layout.h", "common.cuh", "kdtree.cuh"),
                           "traffic_bytes_per_launch")


def design32_traffic_per_location():
    """DRAM bytes per location of the CUDA-core exhaustive scorer (n = 50, N' = 1000)."""
    return profile_traffic("design32_sinusoid8d_M20000.md", ("design_fp32.cu", "common.cuh"),
                           "traffic_bytes_per_location")


def kernel_flops(name, w, ev):
    """Algorithmic FLOPs of one launch's worth of work, and the FLOPs the
    kernel's own arithmetic form executes (None where they are the same).
      kNN: 3 N p per location (subtract, multiply, add per coordinate).
      Ray search: an ALC evaluation at design size j counts 2 j^2 (the matvec
      with K_j^{-1}) + (3p + 4) j (correlation distances, the two dots), and
      each greedy step adds the snap's N' x 3p.  The FP32 kernel forms the
      quadratic through the triangular L_j^{-1}: j^2 + j + 4 j + (3p + 2) j per
      evaluation.
    ev: sum over the launch's evaluations of j (s1) and of j^2 (s2), and its
    greedy steps."""
    if name == "knn_stream":
        return 3.0 * w["N"] * w["p"] * w["M_launch"], None
    if name in ("design32_ray", "ray32", "design64_ray"):
        p, nc = w["p"], w["nc"]
        snap = ev["steps"] * nc * 3 * p
        algo = 2 * ev["s2"] + (3 * p + 4) * ev["s1"] + snap
        tri = ev["s2"] + (5 + 3 * p + 2) * ev["s1"] + snap
        return algo, (tri if name != "design64_ray" else None)
    if name == "design64_exhaustive":
        # per step and unselected candidate: the full ALC in the explicit form
        p, nc, n0, n = w["p"], w["nc"], w["n0"], w["n"]
        per_loc = sum((nc - j) * (2 * j * j + (3 * p + 4) * j) for j in range(n0, n))
        return per_loc * w["M_launch"], None
    if name == "exh_tc":
        nc, n0, n = w["nc"], w["n0"], w["n"]
        per_loc = sum(nc * (2 * j * j + 4 * j) for j in range(n0, n))
        return per_loc * w["M_launch"], None
    return None, None


def kernel_bytes(name, w):
    """Algorithmic DRAM bytes of one launch of the CUDA-core exhaustive scorer
    (see the design notes): per location, step m = 1..n reads the cache rows
    0..m-1 of the N' - m unselected candidates and writes one row of N', and
    the candidates' FP32 rows are read once: 4 (sum_m m (N' - m) + n N' + PP N')."""
    if name != "design32_exhaustive":
        return None
    n, nc, PP = w["n"], w["nc"], w["PP"]
    per_loc = 4.0 * (sum(m * (nc - m) for m in range(1, n + 1)) + n * nc + PP * nc)
    return per_loc * w["M_launch"]


def eval_sums(nev, n0):
    """Sums over a launch's ray evaluations of j and j^2 (nev: [M][n - n0]
    evaluations per greedy step) and its greedy steps."""
    js = np.arange(n0, n0 + nev.shape[1], dtype=np.float64)
    return {"s1": float((nev * js[None, :]).sum()), "s2": float((nev * js[None, :] ** 2).sum()),
            "steps": float(nev.shape[0] * nev.shape[1])}


def roofline(name, tot_ms, launches, w, M_launch, ev=None, traffic_ok=False):
    """Roofline entry of one kernel from its profiled time: achieved work per
    launch over the average launch time, against the bound's peak.  ev: the
    evaluation sums of one launch (eval_sums), for the ray kernels."""
    per_launch_ms = tot_ms / launches
    shape = dict(N=w.N, p=w.p, n0=w.n0, n=w.n, nc=w.nc, PP=(w.p + 3) // 4 * 4,
                 M_launch=M_launch)
    nbytes = kernel_bytes(name, shape)
    if nbytes is not None:
        achieved = nbytes / (per_launch_ms / 1e3) / 1e9
        peak, src = hbm_peak()
        tpl = design32_traffic_per_location() if (w.n == 50 and w.nc == 1000 and w.p == 8
                                                   and w.N == 1_000_000) else None
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if tpl is None else tpl * M_launch,
                "peak_source": src, "launch_ms": per_launch_ms}
    algo, executed = kernel_flops(name, shape, ev)
    if algo is None:
        return None
    fp64 = name.startswith("design64")
    peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
    achieved = algo / (per_launch_ms / 1e3) / 1e12
    out = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
           "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": ray32_traffic() if (name == "ray32" and traffic_ok) else None,
           "peak_source": ("GB300 FP64 rate, nominal" if fp64 else
                           "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (nominal)"),
           "flop_count": ("2j^2 + (3p+4)j per ALC evaluation + N' x 3p per greedy step"
                          if "ray" in name else "per-step algorithmic count, see the design notes"),
           "launch_ms": per_launch_ms}
    if executed is not None:
        out["achieved_executed_form"] = executed / (per_launch_ms / 1e3) / 1e12
        out["frac_executed_form"] = out["achieved_executed_form"] / peak
    return out


def run_ours(args, rank, world):
    import torch
    from paper_1409_0074_gb300 import lagp

    dev = torch.device("cuda", torch.cuda.current_device())
    w = rank_workload(args.M, args.N, rank, world, args.workload)
    N, p, M = w.N, w.p, w.M
    s, pr = lagp.SEARCH[args.search], lagp.PRECISION[args.precision]
    R = w.nrays
    X, Y, Xr = (torch.from_numpy(a).to(dev) for a in (w.X, w.Y, w.Xref))
    wsb = lagp.laGP_workspace_bytes(N, p, M, w.n, w.nc, R, s, pr)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    mean = torch.empty(M, dtype=torch.float64, device=dev)
    s2 = torch.empty(M, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    if args.mle_stages:
        wsb = lagp.laGP_mle_workspace_bytes(N, p, M, w.n, w.nc, R, s, pr)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        theta_hat = torch.empty(M, dtype=torch.float64, device=dev)

    def step():
        flush.zero_()
        if args.mle_stages:
            lagp.laGP_build_and_predict_mle(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, 1e-3, 10.0,
                                            args.mle_stages, s, R, pr, theta_hat, mean, s2, ws,
                                            stream=stream)
        else:
            lagp.laGP_build_and_predict(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, s, R, pr, mean,
                                        s2, ws, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    rc, st = lagp.laGP_status(ws)
    if rc != 0:
        raise RuntimeError("device status %d after warm-up" % st)
    torch.cuda.synchronize()
    barrier(world)
    lagp.laGP_profile(True)
    with Clocks(torch.cuda.current_device()) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    lagp.laGP_profile(False)
    barrier(world)
    ms = e0.elapsed_time(e1)
    value, ms_max = whole_job_rate(M, args.steps, ms, world)
    prof = lagp.laGP_profile_read()
    rc, st = lagp.laGP_status(ws)
    if rc != 0:
        raise RuntimeError("device status %d in the timed region" % st)
    promoted = lagp.laGP_promoted(ws)    # of the last timed step

    # dominant kernel and its roofline
    top = max(prof.items(), key=lambda kv: kv[1][0])
    name, (tot_ms, launches) = top
    trace = lagp.predict(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, search=args.search,
                         nrays=R, precision=args.precision, want_trace=True)
    nev = trace["nevals"].cpu().numpy()[:, : w.n - w.n0].astype(np.float64)
    chunks = max(launches // args.steps, 1)
    ev = {k: v / chunks for k, v in eval_sums(nev, w.n0).items()}
    roof = roofline(name, tot_ms, launches, w, M / chunks, ev,
                    traffic_ok=(w.M == 100_000 and w.N == 1_000_000 and chunks == 1))
    if args.mle_stages:
        roof = None       # several kernel kinds share the step; see the kernel times
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches": v[1],
                   "share": v[0] / sum(x[0] for x in prof.values())} for k, v in prof.items()}
    mean_evals = float(nev.sum(axis=1).mean() / (w.n - w.n0))
    return dict(value=value, ms=ms_max, clocks=clk.summary(), roofline=roof, kernels=kernels,
                gpu_launches=int(sum(v[1] for v in prof.values())), w=w, tensors=(X, Y, Xr),
                evals_per_step=mean_evals, max_evals_per_step=float(nev.max()),
                promoted=promoted,
                rmse=float(np.sqrt(np.mean((mean.cpu().numpy() - w.Ytrue) ** 2))))


def run_e2e(args, w):
    """Same metric through the host-buffer C entry point, copies included."""
    import torch
    from paper_1409_0074_gb300 import lagp
    s, pr = lagp.SEARCH[args.search], lagp.PRECISION[args.precision]
    R = w.nrays

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()

    Xh, Yh, Rh = pinned(w.X), pinned(w.Y), pinned(w.Xref)
    mean = torch.empty(w.M, dtype=torch.float64).pin_memory().numpy()
    s2 = torch.empty(w.M, dtype=torch.float64).pin_memory().numpy()
    wsb = lagp.laGP_host_workspace_bytes(w.N, w.p, w.M, w.n, w.nc, R, s, pr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    call = lambda: lagp.laGP_build_and_predict_host(Xh, Yh, Rh, w.n0, w.n, w.nc, w.theta, w.g, s,
                                                    R, pr, mean, s2, ws)
    call()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        call()
    dt = time.perf_counter() - t0
    h2d = Xh.nbytes + Yh.nbytes + Rh.nbytes
    return {"value": w.M * args.steps / dt, "unit": "locations/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": mean.nbytes + s2.nbytes}


def run_extra(args, w, tensors, search, precision, M, steps=2):
    """Locations/sec of another search/precision form on the first M
    locations, with the roofline of its dominant kernel."""
    import torch
    from paper_1409_0074_gb300 import lagp
    X, Y, Xr = tensors
    Xr = Xr[:M].contiguous()
    s, pr = lagp.SEARCH[search], lagp.PRECISION[precision]
    wsb = lagp.laGP_workspace_bytes(w.N, w.p, M, w.n, w.nc, w.nrays, s, pr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    mean = torch.empty(M, dtype=torch.float64, device="cuda")
    s2 = torch.empty(M, dtype=torch.float64, device="cuda")
    nev = (torch.zeros((M, w.n), dtype=torch.int32, device="cuda") if search.startswith("ray")
           else None)
    go = lambda: lagp.laGP_build_and_predict(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, s,
                                             w.nrays, pr, mean, s2, ws, nevals=nev)
    go()
    torch.cuda.synchronize()
    lagp.laGP_profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        go()
    e1.record()
    torch.cuda.synchronize()
    lagp.laGP_profile(False)
    prof = lagp.laGP_profile_read()
    rc, st = lagp.laGP_status(ws)
    if rc != 0:
        raise RuntimeError("device status %d in the %s %s form" % (st, search, precision))
    name, (tot_ms, launches) = max(prof.items(), key=lambda kv: kv[1][0])
    chunks = max(launches // steps, 1)
    ev = None
    if nev is not None:
        nv = nev.cpu().numpy()[:, : w.n - w.n0].astype(np.float64)
        ev = {k: v / chunks for k, v in eval_sums(nv, w.n0).items()}
    rmse = float(np.sqrt(np.mean((mean.cpu().numpy() - w.Ytrue[:M]) ** 2)))
    return {"locations_per_s": M * steps / (e0.elapsed_time(e1) / 1e3), "locations": M,
            "rmse": rmse, "promoted_locations": lagp.laGP_promoted(ws),
            "roofline": roofline(name, tot_ms, launches, w, M / chunks, ev),
            "kernels": {k: {"ms_per_step": v[0] / steps, "launches": v[1]}
                        for k, v in prof.items()}}


def run_prescaled(args, w, tensors, n_sub=1000, steps=2):
    """Rays with pre-scaled inputs (Sec 5.3): the separable global lengthscales
    on a random 1,000-row subset (laGP_sep_mle), the design and locations
    divided by their square roots (laGP_prescale), then the FP32 ray path at
    theta = 1 on the scaled inputs over all locations.  Reports the fit's time
    and iterations, the estimate, and locations/s and RMSE of the local path."""
    import time
    import torch
    from paper_1409_0074_gb300 import lagp
    from paper_1409_0074_gb300 import workloads as W
    X, Y, Xr = tensors
    sub = torch.from_numpy(W.subset(w.N, n_sub, seed=1)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th, (it, ev, st) = lagp.sep_mle(X, Y, sub, w.g, 1.0, 1e-3, 100.0)
    fit_s = time.perf_counter() - t0
    Xs, Xrs = lagp.prescale(X, th), lagp.prescale(Xr, th)
    M = Xr.shape[0]
    s, pr = lagp.SEARCH["ray"], lagp.PRECISION["fp32"]
    wsb = lagp.laGP_workspace_bytes(w.N, w.p, M, w.n, w.nc, w.nrays, s, pr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    mean = torch.empty(M, dtype=torch.float64, device="cuda")
    s2 = torch.empty(M, dtype=torch.float64, device="cuda")
    go = lambda: lagp.laGP_build_and_predict(Xs, Y, Xrs, w.n0, w.n, w.nc, 1.0, w.g, s, w.nrays,
                                             pr, mean, s2, ws)
    go()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        go()
    e1.record()
    torch.cuda.synchronize()
    rc, stt = lagp.laGP_status(ws)
    if rc != 0:
        raise RuntimeError("device status %d in the pre-scaled form" % stt)
    return {"subset": n_sub, "fit_seconds": fit_s, "fit_iterations": it,
            "fit_evaluations": ev, "theta_global": [float(v) for v in th.cpu()],
            "search": "ray", "precision": "fp32 scoring", "theta_local": 1.0,
            "locations": M, "locations_per_s": M * steps / (e0.elapsed_time(e1) / 1e3),
            "rmse": float(np.sqrt(np.mean((mean.cpu().numpy() - w.Ytrue[:M]) ** 2)))}


def run_nrays_sweep(args, w, tensors, M=20_000, steps=2):
    """Rays per step from 1 to p on the 8-d workload (the paper's fidelity knob,
    Sec 5.4): locations/s and RMSE of the FP32-scoring ray search per count,
    on the first M locations."""
    import torch
    from paper_1409_0074_gb300 import lagp
    X, Y, Xr = tensors
    M = min(M, w.M)
    Xr = Xr[:M].contiguous()
    out = {"workload": w.name, "locations": M, "precision": "fp32 scoring", "rays": []}
    mean = torch.empty(M, dtype=torch.float64, device="cuda")
    s2 = torch.empty(M, dtype=torch.float64, device="cuda")
    for R in range(1, w.p + 1):
        wsb = lagp.laGP_workspace_bytes(w.N, w.p, M, w.n, w.nc, R, lagp.LAGP_RAY,
                                        lagp.LAGP_FP32_SCORE)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        go = lambda: lagp.laGP_build_and_predict(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g,
                                                 lagp.LAGP_RAY, R, lagp.LAGP_FP32_SCORE, mean,
                                                 s2, ws)
        go()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            go()
        e1.record()
        torch.cuda.synchronize()
        rc, st = lagp.laGP_status(ws)
        if rc != 0:
            raise RuntimeError("device status %d in the nrays sweep" % st)
        rmse = float(np.sqrt(np.mean((mean.cpu().numpy() - w.Ytrue[:M]) ** 2)))
        out["rays"].append({"nrays": R, "locations_per_s": M * steps / (e0.elapsed_time(e1) / 1e3),
                            "rmse": rmse})
        del ws
    return out


def run_paper_2d(args, steps=2):
    """The 2-d experiment of Sec 5.1 (201 x 201 grid design on [-2, 2]^2, the
    99 x 99 predictive grid, n = 50, N' = 1000, one ray): locations/s and RMSE
    of each search and arithmetic form at theta0 = 0.5; local inference for
    theta on the FP64 designs in one and two stages (laGP_build_and_predict_mle)
    with its RMSE; the estimate's kernel alone with its roofline.
    The paper's Table 1 RMSE (0.0009 ray, 0.0010 exhaustive, one stage) is
    context: its nugget and theta start are not stated."""
    import torch
    from paper_1409_0074_gb300 import lagp
    from paper_1409_0074_gb300 import workloads as W
    w = W.paper_2d()
    dev = torch.device("cuda", torch.cuda.current_device())
    X, Y, Xr = (torch.from_numpy(a).to(dev) for a in (w.X, w.Y, w.Xref))
    out = {"workload": w.name, "N": w.N, "M": w.M, "n": w.n, "N_close": w.nc, "nrays": 1,
           "theta0": w.theta, "g": w.g, "forms": {}}
    rmse = lambda t: float(np.sqrt(np.mean((t.cpu().numpy() - w.Ytrue) ** 2)))
    for search in ("ray", "exhaustive"):
        for prec in ("fp32", "fp32_promote", "fp64"):
            s, pr = lagp.SEARCH[search], lagp.PRECISION[prec]
            wsb = lagp.laGP_workspace_bytes(w.N, w.p, w.M, w.n, w.nc, 1, s, pr)
            ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
            mean = torch.empty(w.M, dtype=torch.float64, device=dev)
            s2 = torch.empty(w.M, dtype=torch.float64, device=dev)
            sel = torch.empty((w.M, w.n), dtype=torch.int32, device=dev)
            go = lambda: lagp.laGP_build_and_predict(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, s,
                                                     1, pr, mean, s2, ws, selected=sel)
            go()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                go()
            e1.record()
            torch.cuda.synchronize()
            rc, st = lagp.laGP_status(ws)
            if rc != 0:
                raise RuntimeError("device status %d in the 2-d form" % st)
            f = {"locations_per_s": w.M * steps / (e0.elapsed_time(e1) / 1e3),
                 "rmse_theta0": rmse(mean), "promoted_locations": lagp.laGP_promoted(ws)}
            if prec == "fp64" and search == "ray":
                # the local estimate alone, on these designs: its roofline
                th = torch.empty(w.M, dtype=torch.float64, device=dev)
                m2 = torch.empty(w.M, dtype=torch.float64, device=dev)
                v2 = torch.empty(w.M, dtype=torch.float64, device=dev)
                it = torch.empty(w.M, dtype=torch.int32, device=dev)
                stt = torch.zeros(1, dtype=torch.int32, device=dev)
                e0.record()
                lagp.laGP_mle_predict(X, Y, Xr, sel, w.theta, w.g, 1e-3, 10.0, th, m2, v2, stt,
                                      iters=it)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                # a Newton iteration evaluates the likelihood and its derivatives:
                # Cholesky n^3/3, K^{-1} from the factor 2n^3/3, K^{-1} K' 2n^3;
                # one more evaluation predicts at the estimate
                flops = float((it.double() + 1).sum().item()) * 3.0 * w.n ** 3
                out["mle_kernel"] = {
                    "ms": ms, "locations_per_s": w.M / (ms / 1e3),
                    "iterations_mean": float(it.double().mean().item()),
                    "roofline": {"kernel": "mle_theta", "bound": "alu",
                                 "achieved": flops / (ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                                 "unit": "TFLOP/s",
                                 "frac": flops / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                                 "flop_count": "3 n^3 per likelihood evaluation (FP64)"}}
            out["forms"]["%s_%s" % (search, prec)] = f
            del ws
    # local inference for theta, one call: one stage (design at theta0, estimate)
    # and two stages (redesign at each location's estimate), FP64 designs
    for search in ("ray", "exhaustive"):
        for stages in (1, 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = lagp.predict_mle(X, Y, Xr, w.n0, w.n, w.nc, w.theta, w.g, 1e-3, 10.0,
                                 stages=stages, search=search, nrays=1, precision="fp64")
            e1.record()
            torch.cuda.synchronize()
            out["forms"]["%s_fp64_mle_stage%d" % (search, stages)] = {
                "locations_per_s": w.M / (e0.elapsed_time(e1) / 1e3), "rmse": rmse(r["mean"]),
                "theta_median": float(r["theta"].median().item())}
    out["paper_table1_rmse_context"] = {"ray_n50_stage2": 0.0008, "ext_n50_stage2": 0.0008,
                                        "ray_n50_stage1": 0.0009, "ext_n50_stage1": 0.0010,
                                        "nn_n50": 0.0023}
    return out


def run_batching(args, steps=3):
    """Batching form: N = 1e6, p = 8, 50,000 locations with n ~ U{20..100} and
    N' ~ U{300..2000}; the launch choices autotuned on the first 10,000
    locations, the whole call captured as one CUDA graph and replayed.  Returns
    locations/s per search (FP32 scoring, FP64 update)."""
    import torch
    from paper_1409_0074_gb300 import lagp
    from paper_1409_0074_gb300 import workloads as W
    w = W.uneven_8d(M=50_000)
    dev = torch.device("cuda", torch.cuda.current_device())
    X, Y, Xr = (torch.from_numpy(a).to(dev) for a in (w.X, w.Y, w.Xref))
    nl = torch.from_numpy(w.n_arr.astype(np.int32)).to(dev)
    ncl = torch.from_numpy(w.nc_arr.astype(np.int32)).to(dev)
    n, nc = int(w.n_arr.max()), int(w.nc_arr.max())
    out = {"workload": "sinusoid_8d_N1000000_M50000_uneven", "n": "U{20..100}",
           "N_close": "U{300..2000}", "nrays": 8}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for search in ("ray", "exhaustive"):
        s = lagp.SEARCH[search]
        wsb = lagp.laGP_workspace_bytes(w.N, w.p, w.M, n, nc, 8, s, lagp.LAGP_FP32_SCORE)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        mean = torch.empty(w.M, dtype=torch.float64, device=dev)
        s2 = torch.empty(w.M, dtype=torch.float64, device=dev)
        Mt = 10_000
        code = lagp.laGP_autotune(X, Y, Xr[:Mt].contiguous(), w.n0, n, nc, w.theta, w.g, s, 8,
                                  lagp.LAGP_FP32_SCORE, mean[:Mt], s2[:Mt], ws,
                                  n_loc=nl[:Mt].contiguous(), nclose_loc=ncl[:Mt].contiguous())
        plan = lagp.Plan(X, Y, Xr, w.n0, n, nc, w.theta, w.g, s, 8, lagp.LAGP_FP32_SCORE, mean,
                         s2, ws, n_loc=nl, nclose_loc=ncl)
        plan.launch(stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(steps):
            flush.zero_()
            e0.record(stream)
            plan.launch(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        rc, st = lagp.laGP_status(ws)
        if rc != 0:
            raise RuntimeError("device status %d in the batching form" % st)
        rmse = float(np.sqrt(np.mean((mean.cpu().numpy() - w.Ytrue) ** 2)))
        out[search] = {"locations_per_s": w.M * steps / (ms / 1e3), "ms_per_call": ms / steps,
                       "tune_code": code, "graph": True, "rmse": rmse}
        plan.close()
        del ws
    return out


def serve_curve(ctx, w, rates, seconds, rng, max_batch=4096, slots=8, max_requests=None):
    """Poisson request streams at each rate through one continuous-batching
    server over the context: p50 / p99 latency (arrival to results in host
    memory), the locations/s the stream achieved and the RMSE of the served
    predictions against the true response."""
    from paper_1409_0074_gb300.serve import (CtxBackend, Server, latency_summary,
                                             poisson_requests, run_stream)
    out = []
    for rate in rates:
        count = int(rate * seconds)
        if max_requests:
            count = min(count, max_requests)
        reqs = poisson_requests(rng, rate, max(count, 4), w.p)
        srv = Server(CtxBackend(ctx, max_batch, slots), max_batch)
        wall = run_stream(srv, reqs)
        summ = latency_summary(reqs, wall)
        offered = sum(r.xref.shape[0] for r in reqs) / max(reqs[-1].arrival - reqs[0].arrival,
                                                          1e-9)
        err = np.concatenate([r.mean - w.true_response(r.xref) for r in reqs])
        summ.update({"rate_per_s": rate, "offered_locations_per_s": offered,
                     "batches": srv.batches, "mean_batch": float(np.mean(srv.batch_sizes)),
                     "rmse": float(np.sqrt(np.mean(err ** 2)))})
        out.append(summ)
    return out


def request_breakdown(ctx, w, M, rng, repeats=5):
    """Per-kernel device time of one request of M locations (n = 50) served
    alone, and its latency from submit to results in host memory."""
    import torch
    from paper_1409_0074_gb300 import lagp
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
    xr = pin((M, w.p), torch.float64)
    mean, s2 = pin((M,), torch.float64), pin((M,), torch.float64)
    lat = []
    for k in range(repeats + 1):
        xr[...] = rng.random((M, w.p))
        if k == repeats:
            lagp.laGP_profile(True)
        t0 = time.perf_counter()
        t = ctx.submit(xr, 50, mean, s2)
        ctx.wait(t)
        if k < repeats:
            lat.append((time.perf_counter() - t0) * 1e3)
    lagp.laGP_profile(False)
    prof = lagp.laGP_profile_read()
    return {"locations": M, "latency_ms_median": float(np.median(lat)),
            "kernels_ms": {k: v[0] for k, v in prof.items()},
            "device_ms": float(sum(v[0] for v in prof.values()))}


def mix_capacity(X, Y, w, precision, M=30_000, steps=2):
    """Locations/s of one direct call on the served mix (n uniform over
    {30, 50, 100}, N' = 1000, ray search with 8 rays): the device's capacity
    for that mix, against which the served rates are read."""
    import torch
    from paper_1409_0074_gb300 import lagp
    rng = np.random.default_rng(12)
    xr = torch.from_numpy(rng.random((M, w.p))).cuda()
    nl = torch.from_numpy(rng.choice(np.array([30, 50, 100], np.int32), M)).cuda()
    pr = lagp.PRECISION[precision]
    wsb = lagp.laGP_workspace_bytes(w.N, w.p, M, 100, 1000, 8, lagp.LAGP_RAY, pr)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    mean = torch.empty(M, dtype=torch.float64, device="cuda")
    s2 = torch.empty(M, dtype=torch.float64, device="cuda")
    go = lambda: lagp.laGP_build_and_predict(X, Y, xr, w.n0, 100, 1000, w.theta, w.g,
                                             lagp.LAGP_RAY, 8, pr, mean, s2, ws, n_loc=nl)
    go()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        go()
    torch.cuda.synchronize()
    return M * steps / (time.perf_counter() - t0)


def run_serving(args, rates32=(50.0, 100.0, 150.0, 200.0, 250.0, 300.0, 400.0),
                rates64=(0.5, 1.0, 2.0, 4.0)):
    """Serving form: the N = 1e6, p = 8 design resident in a serving context;
    Poisson request streams of 1..4096 locations (log-uniform), n in
    {30, 50, 100}, N' = 1000, ray search with 8 rays, through the
    continuous-batching server.  The FP32-scoring form is swept from light
    load past the device's capacity; the plain FP64 form runs through the same
    server and request distribution at the rates it can carry.  Both report
    p50 / p99 latency, locations/s and RMSE; a per-kernel breakdown of a
    1-location and a 64-location request explains the latency floor."""
    import torch
    from paper_1409_0074_gb300 import lagp
    from paper_1409_0074_gb300 import workloads as W
    from paper_1409_0074_gb300.serve import CtxBackend, Server, poisson_requests, run_stream
    w = W.large_8d(M=1)
    dev = torch.device("cuda", torch.cuda.current_device())
    X, Y = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.Y).to(dev)
    slots, max_batch, arena_gb = 8, 32768, 24
    rng = np.random.default_rng(11)
    out = {"design": "sinusoid_8d_N1000000", "request_sizes": "log-uniform 1..4096",
           "n": [30, 50, 100], "N_close": 1000, "search": "ray", "nrays": 8, "slots": slots,
           "max_batch": max_batch, "arena_gb": arena_gb}
    for prec, rates, secs in (("fp32", rates32, args.serve_seconds),
                              ("fp64", rates64, 2 * args.serve_seconds)):
        ctx = lagp.Context(X, Y, w.theta, w.g, w.n0, 1000, lagp.LAGP_RAY, 8,
                           lagp.PRECISION[prec], arena_gb << 30, max_inflight=slots)
        # warm-up (kernel load, tune table)
        srv = Server(CtxBackend(ctx, max_batch, slots), max_batch)
        run_stream(srv, poisson_requests(rng, 50.0, 6, w.p, sizes=(1, 256)))
        form = {"precision": "fp32 scoring, fp64 update" if prec == "fp32" else "fp64",
                "rates": serve_curve(ctx, w, rates, secs, rng, max_batch, slots,
                                     max_requests=3000)}
        if prec == "fp32":
            form["breakdown"] = [request_breakdown(ctx, w, M, rng) for M in (1, 64)]
        for slo in (100.0, 250.0, 500.0):
            ok = [r for r in form["rates"] if r["p99_ms"] <= slo]
            form["max_locations_per_s_at_p99_le_%dms" % slo] = (
                max(r["locations_per_s"] for r in ok) if ok else None)
        ctx.close()
        form["direct_call_capacity_same_mix"] = mix_capacity(
            X, Y, w, prec, M=30_000 if prec == "fp32" else 2000, steps=2 if prec == "fp32" else 1)
        out[prec] = form
    return out


def run_cpu_baseline(args, w, search, sample=None, one_core=False):
    """The FP64 oracle as it stands, OpenMP over locations on the host cores."""
    import oracle
    cores = os.cpu_count() or 1
    S = sample or args.cpu_sample or 32 * cores
    S = min(S, w.M)
    t0 = time.perf_counter()
    r = oracle.predict(w.X, w.Y, w.Xref[:S], w.n0, w.n, w.nc, w.theta, w.g, search,
                       nrays=w.nrays, nthreads=0)
    dt = time.perf_counter() - t0
    out = {"value": S / dt, "unit": "locations/s", "cores": int(r["threads"]), "kind": "oracle",
           "sample": "first %d of the %d locations, %s search, FP64" % (S, w.M, search),
           "seconds": dt}
    if one_core:
        S1 = min(max(4, S // (4 * cores)), w.M)
        t0 = time.perf_counter()
        oracle.predict(w.X, w.Y, w.Xref[:S1], w.n0, w.n, w.nc, w.theta, w.g, search,
                       nrays=w.nrays, nthreads=1)
        dt1 = time.perf_counter() - t0
        out["one_core"] = {"value": S1 / dt1, "unit": "locations/s", "cores": 1,
                           "sample": "first %d locations" % S1, "seconds": dt1}
    return out


def base_line(args, world, value, ms, w):
    metric = ("locations/sec at N=1e6,d=8,n=50 (%s search)" % args.search
              if args.workload == "sinusoid_8d" else
              "locations/sec, 2-d grid of Sec 5.1, n=50 (%s search)" % args.search)
    if args.mle_stages:
        metric += ", local theta in %d stage(s)" % args.mle_stages
    return {"metric": metric, "value": value,
            "unit": "locations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps if ms is not None else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic (seeded uniform design, sinusoid-plus-product response)",
            "config": {"workload": w.name, "N": w.N, "p": w.p, "M": w.M, "n0": w.n0, "n": w.n,
                       "N_close": w.nc, "theta": w.theta, "g": w.g, "search": args.search,
                       "nrays": w.nrays,
                       "precision": "fp32 scoring, fp64 update" if args.precision != "fp64"
                       else "fp64", "l2": "flushed: 256 MB written before every step",
                       "parallelism": "locations sharded over %d rank(s)" % world}}


def main():
    args = parse()
    rank, world = dist_init(args)
    if args.impl == "reference":
        if rank != 0:
            return
        w = rank_workload(args.M, args.N, 0, 1)
        cores = os.cpu_count() or 1
        S = args.cpu_sample or 8 * cores
        if args.warmup > 0:   # one short untimed pass (page-in, thread start-up)
            run_cpu_baseline(args, w, args.search, sample=min(S, cores))
        t0 = time.perf_counter()
        rates = [run_cpu_baseline(args, w, args.search, sample=S) for _ in range(args.steps)]
        dt = time.perf_counter() - t0
        value = S * args.steps / dt
        line = base_line(args, 1, value, dt * 1e3, w)
        line.update({"impl": "reference", "dtype": "f64",
                     "cpu_baseline": {"value": value, "unit": "locations/s",
                                      "cores": rates[0]["cores"], "kind": "oracle",
                                      "sample": "%d locations per step" % S},
                     "e2e": {"value": value, "unit": "locations/s", "h2d_bytes_per_step": 0,
                             "d2h_bytes_per_step": 0}})
        print(json.dumps(line))
        return

    r = run_ours(args, rank, world)
    w = r["w"]
    line = base_line(args, world, r["value"], r["ms"], w)
    line.update({"dtype": "f32/f64" if args.precision != "fp64" else "f64",
                 "roofline": r["roofline"], "clocks": r["clocks"],
                 "gpu_launches": r["gpu_launches"], "kernels": r["kernels"],
                 "rmse": r["rmse"], "ray_evals_per_step": r["evals_per_step"],
                 "ray_evals_per_step_max": r["max_evals_per_step"],
                 "promoted_locations_per_step": r["promoted"]})
    if world == 1:
        line["e2e"] = run_e2e(args, w)
        if not args.no_extras:
            ex = {}
            ex["exhaustive_fp32"] = run_extra(args, w, r["tensors"], "exhaustive", "fp32", w.M)
            ex["exhaustive_fp32_tc"] = run_extra(args, w, r["tensors"], "exhaustive", "fp32_tc",
                                                 w.M)
            ex["ray_fp32_promote"] = run_extra(args, w, r["tensors"], "ray", "fp32_promote",
                                               w.M)
            ex["ray_fp64"] = run_extra(args, w, r["tensors"], "ray", "fp64", min(w.M, 4000))
            ex["ray_full_scope_fp32"] = run_extra(args, w, r["tensors"], "ray_full", "fp32", w.M)
            ex["ray_full_scope_fp64"] = run_extra(args, w, r["tensors"], "ray_full", "fp64",
                                                  min(w.M, 4000))
            ex["exhaustive_fp64"] = run_extra(args, w, r["tensors"], "exhaustive", "fp64",
                                              min(w.M, 1000), steps=1)
            line["other_forms"] = ex
            line["nrays_sweep"] = run_nrays_sweep(args, w, r["tensors"])
            line["prescaled_form"] = run_prescaled(args, w, r["tensors"])
            line["paper_2d_form"] = run_paper_2d(args)
        if not args.no_batching:
            line["batching_form"] = run_batching(args)
        if not args.no_serving:
            line["serving_form"] = run_serving(args)
        if not args.no_cpu:
            line["cpu_baseline"] = run_cpu_baseline(args, w, args.search, one_core=True)
    else:
        line["e2e"] = None
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
