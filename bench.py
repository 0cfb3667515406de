"""ChASE time-to-solution on one GB300 (and N independent replicas).

One step = the whole hot path on one synthetic BSE Hamiltonian: generate
H on the device (Eq. (1) stand-in), then solve for the lowest nev
eigenpairs (Lanczos, filter, QR, Rayleigh-Ritz, residuals/locking, output).
Workload: N = 20000 (Nk = 1250, Nv = Nc = 4), nev = 100, nex = 40,
deg_max = 36, tol = 1e-10, complex FP64.  The filter degrees of Eq. (S1) are
raised in groups of 48 columns, the tile width of the tensor-core product
(--degree-group; 0 keeps them unchanged).  H is 6.4 GB, far larger than L2,
so no L2 flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch under torch.distributed.run: every rank solves its own
replica (weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="chase_N20000_nev100_nex40", Nk=1250, Nv=4, Nc=4, N=20000,
                nev=100, nex=40, deg_max=36, tol=1e-10, seed=0, precision="fp64",
                l2="inputs larger than L2 (H = 6.4 GB)", matvecs_per_solve=22540)
METRIC = "chase_time_to_solution"
UNIT = "s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 issue rate of the part: the measured DFMA peak when one is recorded
# next to the bench (profiles/fp64_peak.txt, written from the DFMA-loop
# probe), else the GB300 datasheet figure of 1.25 TFLOP/s.
def _fp64_peak():
    p = os.path.join(ROOT, "profiles", "fp64_peak.txt")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["fp64_tflops"]), "measured DFMA loop (profiles/fp64_peak.txt)"
    except (OSError, KeyError, ValueError):
        return 1.25, "datasheet (no measured FP64 peak recorded)"


def _traffic(precision, workload_name):
    """DRAM bytes per launch of the filter kernel from an ncu capture, when
    profiles/filter_traffic_<precision>.txt records one for the current
    kernel on this workload (JSON: {"bytes_per_launch": ..., "workload": ...})."""
    p = os.path.join(ROOT, "profiles", "filter_traffic_%s.txt" % precision)
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if not str(d.get("workload", "")).startswith(workload_name):
        return None
    return d


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device, path=None):
        self.device = device
        self.proc = None
        self.keep = path is not None
        self.path = path

    def start(self):
        try:
            if self.path is None:
                fd, self.path = tempfile.mkstemp(prefix="clocks_rank%d_" % self.device, suffix=".csv")
                os.close(fd)
            else:
                os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            summary = parse_clock_samples(f)
        if not self.keep:
            try:
                os.remove(self.path)
            except OSError:
                pass
        return summary


def parse_clock_samples(lines):
    """Summary of nvidia-smi samples (the Clocks.FIELDS columns, CSV without
    header or units): median SM clock under load, the maximum clock, and the
    throttle reasons seen active in any sample; None without samples."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def replica_seed(base_seed, rank):
    """Seed of rank `rank`'s replica: every rank solves its own Hamiltonian."""
    return base_seed + rank


def slowest(value, dist=None, device="cpu"):
    """The largest `value` over the ranks (the bench reports the slowest)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, ms_max):
    """Solves per second of the whole job: every rank finished `steps`
    replicas within the slowest rank's time."""
    return world * steps / (ms_max / 1e3)


def workload(args):
    """The benchmark workload, with optional overrides for profiling runs."""
    W = dict(WORKLOAD)
    if args.nk != W["Nk"] or args.nev != W["nev"] or args.nex != W["nex"]:
        W.update(Nk=args.nk, nev=args.nev, nex=args.nex)
        W["N"] = args.nk * W["Nv"] * W["Nc"]
        W["workload"] = "chase_N%d_nev%d_nex%d" % (W["N"], args.nev, args.nex)
        W["l2"] = "H = %.2f GB" % (16e-9 * W["N"] ** 2)
        W["matvecs_per_solve"] = 160 * (args.nev + args.nex)   # rough, for profiling runs
    return W


PRECISIONS = {"fp64": 0, "mixed": 1, "fp64_dfma": 2}
DTYPES = {"fp64": "f64 (H products: bf16 slices on tensor cores, exact int + f32 accumulation)",
          "mixed": "f64 with f32-level filter sweeps (4 bf16 slices, exact accumulation)",
          "fp64_dfma": "f64"}
def roofline(precision, st, N, workload_name):
    """Roofline of the dominant kernel, the filter's matrix product.

    Tensor-core precisions: the product kernel k_ozaki_zgemm is timed by the
    library with CUDA events around every launch on its stream, inside this
    timed region.  Its algorithmic work per launch is 8 N^2 n real flops per
    slice pair (21 pairs at FP64 accuracy, 10 at FP32 level) for n columns:
    achieved = summed work / summed launch time, against the measured BF16
    peak.  DFMA precision: the FP64-equivalent filter rate (8 N^2 per column
    product over the filter phase) against the measured DFMA peak."""
    peaks = _peaks()
    fp64_eq = st["filter_tflops"]
    tr = _traffic(precision, workload_name)
    if precision == "fp64_dfma":
        peak, src = _fp64_peak()
        return {"kernel": "zgemm_nn_kernel (filter H*Y, Chebyshev epilogue, DFMA)",
                "bound": "alu", "achieved": fp64_eq, "peak": peak, "unit": "TFLOP/s",
                "frac": fp64_eq / peak, "peak_source": src,
                "traffic": (tr or {}).get("bytes_per_launch"),
                "algorithmic_flops_per_launch_avg":
                    8.0 * N * N * st["filter_matvecs"] / max(1, st["filter_launches"])}
    achieved = st["tc_kernel_tflops"]
    peak = peaks.get("bf16_tflops_sustained") or 1700.0
    launches = max(1, st["tc_kernel_launches"])
    return {"kernel": "k_ozaki_zgemm (H*Y: BF16 slice products on tcgen05, Chebyshev epilogue)",
            "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside "
                            "a seconds-long solve)" if peaks else "fallback 1.7 PFLOP/s sustained"),
            "traffic": (tr or {}).get("bytes_per_launch"),
            "launches": st["tc_kernel_launches"],
            "avg_launch_ms": st["tc_kernel_ms"] / launches,
            "algorithmic_flops_per_launch_avg": achieved * 1e12 * st["tc_kernel_ms"] / 1e3 / launches,
            "fp64_equivalent_filter_tflops": fp64_eq}


def cpu_baseline_sample(W, seconds_budget=25.0):
    """The oracle, as it stands, on the host cores: builds the workload's H
    and times single filter matrix products over the full search space
    (m = 140 columns), then projects one solve from the per-matvec time and
    the matvec count of the device solve.  Returns (seconds per solve,
    sample description, cores)."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    H = oracle.build_h(W["seed"], W["Nk"], W["Nv"], W["Nc"])
    t_build = time.perf_counter() - t0
    m = W["nev"] + W["nex"]
    V = oracle.random_block(0, oracle.STREAM_START, W["N"], m)
    c, e, lower = 8.0, 5.0, 0.8
    reps, t_mv = 0, 0.0
    while reps < 1 or (t_mv + t_build < seconds_budget and reps < 8):
        t0 = time.perf_counter()
        oracle.chebyshev_filter(H, V, np.full(m, 1), lower, c, e)
        t_mv += time.perf_counter() - t0
        reps += 1
    per_matvec = t_mv / (reps * m)
    return per_matvec, t_build, reps, os.cpu_count()


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the host cores, on a bounded sample
    of the same workload, projected to one solve."""
    if rank != 0:
        return
    W = workload(args)
    per_mv, t_build, reps, cores = cpu_baseline_sample(W)
    # H*vector products of one solve of this workload: the oracle and the
    # device path take the same iterations and degrees (checked by the parity
    # tests), so the count of the device's FP64 solve stands for the oracle's.
    mv_total = float(W["matvecs_per_solve"])
    t_solve = t_build + per_mv * mv_total
    sample = ("oracle build_h at N=%d (%.1f s) + %d filter product(s) over %d columns; "
              "solve projected as build + %d matvecs x %.3e s"
              % (W["N"], t_build, reps, W["nev"] + W["nex"], mv_total, per_mv))
    line = {"impl": "reference", "metric": METRIC, "value": t_solve, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_solve * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": W,
            "cpu_baseline": {"value": t_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": t_solve, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2006_08498_gb300 as pkg
    from paper_2006_08498_gb300 import build as pkg_build

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        pkg_build.build()
    if dist:
        dist.barrier()
    W = workload(args)
    N, nev, nex = W["N"], W["nev"], W["nex"]
    ctx = pkg.Context(local_rank)
    H = pkg.colmajor_empty(N, N, device="cuda:%d" % local_rank)
    evecs = pkg.colmajor_empty(N, nev, device="cuda:%d" % local_rank)
    stream = torch.cuda.current_stream()

    prec = PRECISIONS[args.precision]

    def step():
        ctx.build_hamiltonian(replica_seed(W["seed"], rank), W["Nk"], W["Nv"], W["Nc"], out=H)
        return ctx.solve(H, nev, nex, tol=W["tol"], deg_max=W["deg_max"], evecs=evecs,
                         precision=prec, degree_group=args.degree_group)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local_rank, args.clock_log.replace("{rank}", str(local_rank)) if args.clock_log else None)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step()[3])
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms_max = slowest(ms, dist, device="cuda")

    # end to end through the host-buffer entry point: pinned H in, eigenvectors
    # and eigenvalues out, one call per step (the device path is already warm)
    e2e_s = None
    if not args.no_e2e:
        Hh = torch.empty((N, N), dtype=torch.complex128, pin_memory=True)
        Hh.copy_(H.T)                      # row-major storage of H^T = column-major H
        Hcol = Hh.T
        Zh = torch.empty((nev, N), dtype=torch.complex128, pin_memory=True).T
        e2e_steps = 1
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.solve_host(Hcol, nev, nex, tol=W["tol"], deg_max=W["deg_max"], evecs=Zh,
                           precision=prec, degree_group=args.degree_group)
        e2e_s = slowest((time.perf_counter() - t0) / e2e_steps, dist, device="cuda")

    if rank == 0:
        st = stats[-1]
        sec = ms_max / 1e3 / args.steps
        roof = roofline(args.precision, st, N, W["workload"])
        line = {
            "metric": METRIC, "value": sec, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": dict(W, precision=args.precision, degree_group=args.degree_group,
                           parallelism="replicas" if world > 1 else "single"),
            "throughput_solves_per_s": replica_throughput(world, args.steps, ms_max),
            "solve": {k: st[k] for k in ("iters", "matvecs", "filter_matvecs",
                                         "filter_matvecs_low", "filter_launches", "ms_lanczos",
                                         "ms_filter", "ms_qr", "ms_rr", "ms_resid",
                                         "ms_total", "filter_tflops", "tc_kernel_ms",
                                         "tc_kernel_launches", "tc_kernel_tflops")},
            "roofline": roof,
            "e2e": None if e2e_s is None else {
                "value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * N * N,
                "d2h_bytes_per_step": 16 * N * nev + 16 * nev},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats) + 2 * args.steps),
            "clocks": ck,
        }
        if world == 1 and not args.no_cpu_baseline:
            per_mv, t_build, reps, cores = cpu_baseline_sample(W)
            t_cpu = t_build + per_mv * st["matvecs"]
            line["cpu_baseline"] = {
                "value": t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": ("oracle build_h at N=%d (%.1f s) + %d filter product(s) over %d "
                           "columns (%.3e s/matvec), projected to this solve's %d matvecs"
                           % (N, t_build, reps, nev + nex, per_mv, st["matvecs"]))}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def run_serving(args):
    """Serving mix: 256 requests, Poisson arrivals, N = 16 Nk with Nk ~
    U{63..1000}, nev ~ U{10..100}, nex = max(10, ceil(nev/2)), 30% warm-start
    neighbours (same seed and Nk as an earlier request, w0 scaled by 1 + d,
    d ~ U[-0.02, 0.02]), admission by an HBM budget.  The arrival rate is set
    to 80% of the throughput measured on a calibration batch."""
    import math
    import numpy as np
    import torch
    import paper_2006_08498_gb300 as pkg
    from paper_2006_08498_gb300 import build as pkg_build
    pkg_build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(0)
    n_req = args.requests
    reqs = []
    for r in range(n_req):
        if r > 0 and rng.random() < 0.3:
            base = reqs[int(rng.integers(0, r))]
            d = float(rng.uniform(-0.02, 0.02))
            reqs.append(dict(seed=base["seed"], Nk=base["Nk"], nev=base["nev"], nex=base["nex"],
                             w0=0.3 * (1 + d), warm=base["idx"], idx=r))
        else:
            nev = int(rng.integers(10, 101))
            reqs.append(dict(seed=int(rng.integers(1, 2 ** 31)), Nk=int(rng.integers(63, 1001)),
                             nev=nev, nex=max(10, math.ceil(nev / 2)), w0=0.3, warm=None, idx=r))
    free, total = torch.cuda.mem_get_info()
    budget = int(0.85 * free)
    ctx = pkg.Context(0)
    ctx.server_create(budget, args.slots)
    prec = PRECISIONS[args.precision]

    def submit(q, tickets):
        warm = tickets.get(q["warm"], 0) if q["warm"] is not None else 0
        return ctx.submit(q["seed"], q["Nk"], 4, 4, q["nev"], q["nex"], tol=1e-10, deg_max=36,
                          precision=prec, model=dict(w0=q["w0"]), warm_ticket=warm,
                          degree_group=args.degree_group)

    # calibration: a back-to-back batch of the first 16 (cold) requests
    t0 = time.perf_counter()
    cal = [submit(dict(q, warm=None), {}) for q in reqs[:16]]
    for t in cal:
        ctx.wait(t, 3600)
        ctx.release(t)
    cap = 16 / (time.perf_counter() - t0)
    rate = 0.8 * cap
    # the timed mix
    tickets, order = {}, []
    start = time.perf_counter()
    t_next = start
    for q in reqs:
        t_next += float(rng.exponential(1.0 / rate))
        while time.perf_counter() < t_next:
            time.sleep(min(0.002, max(0.0, t_next - time.perf_counter())))
        tk = submit(q, tickets)
        tickets[q["idx"]] = tk
        order.append(tk)
    res = [ctx.wait(t, 3600) for t in order]
    end = time.perf_counter()
    lat = np.array([r["latency"] for r in res])
    ok = sum(r["status"] == pkg.BSE_OK for r in res)
    statuses = {}
    for r in res:
        statuses[str(r["status"])] = statuses.get(str(r["status"]), 0) + 1
    warm_used = sum(1 for q in reqs if q["warm"] is not None)
    ctx.server_destroy()
    ctx.close()
    line = {"metric": "chase_serving_latency_p99", "value": float(np.percentile(lat, 99)),
            "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "solves_per_s": n_req / (end - start), "requests": n_req, "ok": ok, "statuses": statuses,
            "warm_requests": warm_used, "arrival_rate_per_s": rate,
            "calibrated_capacity_per_s": cap, "slots": args.slots, "budget_bytes": budget,
            "precision": args.precision, "degree_group": args.degree_group, "data": "synthetic",
            "config": {"workload": "serving_mix_256", "N": "16*U{63..1000}", "nev": "U{10..100}",
                       "nex": "max(10, ceil(nev/2))", "warm_fraction": 0.3, "tol": 1e-10}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clock-log", default=None,
                    help="keep the nvidia-smi samples of the timed region in this CSV ({rank} = rank)")
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--serving", action="store_true", help="run the serving mix instead")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--nk", type=int, default=WORKLOAD["Nk"], help="k-points (N = 16 Nk)")
    ap.add_argument("--nev", type=int, default=WORKLOAD["nev"])
    ap.add_argument("--nex", type=int, default=WORKLOAD["nex"])
    ap.add_argument("--degree-group", type=int, default=48,
                    help="48 (default): filter degrees raised in groups of one tensor-core "
                         "tile; 0: the per-vector degrees of Eq. (S1) unchanged")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.serving:
        if rank == 0:
            run_serving(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
