"""ChASE time-to-solution on one GB300 (and N independent replicas).

One step = the whole hot path on one synthetic BSE Hamiltonian: generate
H on the device (Eq. (1) stand-in), then solve for the lowest nev
eigenpairs (Lanczos, filter, QR, Rayleigh-Ritz, residuals/locking, output).
Workload: N = 50000 (Nk = 3125, Nv = Nc = 4; H is 40 GB), nev = 200,
nex = 80, deg_max = 36, tol = 1e-10, complex FP64.  The filter degrees of
Eq. (S1) are raised in groups of 48 columns, the tile width of the
tensor-core product (--degree-group; 0 keeps them unchanged, and the line
also reports one solve that way).  H is far larger than L2, so no L2 flush
is needed between steps.

After the timed steps the line adds: one end-to-end solve through the
host-buffer entry point (H copied in, eigenvectors copied out); one solve
in the mixed precision mode with its per-eigenpair differences from the
FP64 solve; one solve with the degrees of Eq. (S1) unchanged; one solve
with H generated straight into its tensor-core slices (never stored); the
CPU oracle timed on the host's cores on a bounded sample of the same
workload; and the serving mix.

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

WORKLOAD = dict(workload="chase_N50000_nev200_nex80", Nk=3125, Nv=4, Nc=4, N=50000,
                nev=200, nex=80, deg_max=36, tol=1e-10, seed=0, precision="fp64",
                l2="inputs larger than L2 (H = 40 GB)")
METRIC = "chase_time_to_solution"
UNIT = "s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 issue rate of the part, measured on a GB300 with a loop of independent
# DFMA chains over all SMs (1.005 TFLOP/s; DMMA tensor instructions 1.047):
# the peak of the native-FP64 (DFMA) precision's roofline.
FP64_PEAK_TFLOPS = 1.005
FP64_PEAK_SOURCE = "measured DFMA-loop peak on a GB300 (1.005 TFLOP/s)"


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
    return W


PRECISIONS = {"fp64": 0, "mixed": 1, "fp64_dfma": 3}
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
        peak, src = FP64_PEAK_TFLOPS, FP64_PEAK_SOURCE
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


def cpu_oracle_sample(W, n_cols=48):
    """The CPU oracle, as it stands, on every host core, on the workload's own
    matrix: builds H (oracle.build_h), then times one filter product over
    n_cols columns (oracle.chebyshev_filter with degree 1), the QR phase on
    the full N x m search space (oracle.qr) and the Rayleigh-Ritz steps other
    than its product with H (projection, oracle.eigh of the m x m matrix,
    back-transforms, residual norms).  Returns the timings in seconds."""
    import numpy as np
    import oracle
    N, m = W["N"], W["nev"] + W["nex"]
    t0 = time.perf_counter()
    H = oracle.build_h(W["seed"], W["Nk"], W["Nv"], W["Nc"])
    t_build = time.perf_counter() - t0
    V = oracle.random_block(W["seed"], oracle.STREAM_START, N, m)
    nc = min(n_cols, m)
    t0 = time.perf_counter()
    oracle.chebyshev_filter(H, V[:, :nc], np.ones(nc, dtype=np.int64), 0.8, 8.0, 5.0)
    t_mv = (time.perf_counter() - t0) / nc
    del H
    t_qr, t_rr = _oracle_qr_rr(V)
    return dict(t_build=t_build, t_mv=t_mv, t_qr=t_qr, t_rr=t_rr, n_cols=nc)


def _oracle_qr_rr(V):
    """Seconds of one oracle QR phase on V and of one Rayleigh-Ritz without
    its H product (W = H Q stood in by a block of the same shape)."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    Q = oracle.qr(None, V)
    t_qr = time.perf_counter() - t0
    W_ = V
    t0 = time.perf_counter()
    G = Q.conj().T @ W_
    G = (G + G.conj().T) / 2.0
    theta, Y = oracle.eigh(G)
    Vr, HVr = Q @ Y, W_ @ Y
    oracle.residuals(HVr, Vr, theta, 1.0)
    t_rr = time.perf_counter() - t0
    return t_qr, t_rr


def cpu_oracle_single_thread(W, Nk_small=313, n_cols=48):
    """The same sample with one thread (a child process with the BLAS and
    OpenMP thread counts at 1), on the generator's matrix at Nk_small
    k-points (N_s = 16 Nk_small), scaled to the workload's N: products by
    (N/N_s)^2, QR and Rayleigh-Ritz by N/N_s.  None if the child fails."""
    code = (
        "import sys, json; sys.path.insert(0, %r)\n"
        "import bench\n"
        "W = dict(bench.WORKLOAD, Nk=%d); W['N'] = 16 * W['Nk']\n"
        "print(json.dumps(bench.cpu_oracle_sample(W, %d)))\n" % (ROOT, Nk_small, n_cols))
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                           text=True, timeout=300)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        return None
    f = W["N"] / (16.0 * Nk_small)
    return dict(t_build=d["t_build"] * f * f, t_mv=d["t_mv"] * f * f,
                t_qr=d["t_qr"] * f, t_rr=d["t_rr"] * f, n_small=16 * Nk_small)


def project_solve(sample, counts):
    """Seconds of one oracle solve: build, every H*vector product at the
    sampled per-column time, and per iteration one QR and one Rayleigh-Ritz."""
    return (sample["t_build"] + sample["t_mv"] * counts["matvecs"] +
            counts["iters"] * (sample["t_qr"] + sample["t_rr"]))


def oracle_counts(W, degree_group):
    """Iterations and H*vector products of the oracle's own ChASE on this
    workload: the plain oracle ChASE run to convergence with its products
    through the structured operator of the synthetic Hamiltonian (exact
    H V in O(N log N) per column), timed."""
    import oracle
    t0 = time.perf_counter()
    op = oracle.structured.BseOperator(W["seed"], W["Nk"], W["Nv"], W["Nc"])
    r = oracle.chase(op, W["nev"], W["nex"], tol=W["tol"], deg_max=W["deg_max"],
                     degree_group=degree_group)
    return dict(iters=r["iters"], matvecs=r["matvecs"], status=r["status"],
                seconds=time.perf_counter() - t0)


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the host cores.  Once (before the
    steps): the oracle's own ChASE on this workload through the structured
    operator, for its iteration and product counts.  Each step: the oracle
    timed on a bounded sample of the workload's dense matrix (one filter
    product over 16 columns, one QR phase, one Rayleigh-Ritz without its H
    product), projected to one dense-matrix solve with those counts."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    W = workload(args)
    counts = oracle_counts(W, args.degree_group)
    N, m = W["N"], W["nev"] + W["nex"]
    t0 = time.perf_counter()
    H = oracle.build_h(W["seed"], W["Nk"], W["Nv"], W["Nc"])
    t_build = time.perf_counter() - t0
    V = oracle.random_block(W["seed"], oracle.STREAM_START, N, m)
    nc = 16
    vals = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.chebyshev_filter(H, V[:, step % (m - nc):step % (m - nc) + nc],
                                np.ones(nc, dtype=np.int64), 0.8, 8.0, 5.0)
        t_mv = (time.perf_counter() - t0) / nc
        t_qr, t_rr = _oracle_qr_rr(V)
        if step >= args.warmup:
            vals.append(project_solve(dict(t_build=t_build, t_mv=t_mv, t_qr=t_qr, t_rr=t_rr),
                                      counts))
    t_solve = float(np.mean(vals))
    sample = ("per step: oracle filter product over %d of %d columns of the dense N=%d matrix, "
              "one QR phase and one Rayleigh-Ritz (without its H product), projected to one "
              "solve with the oracle's own counts (%d iterations, %d H*v products; its ChASE "
              "through the structured operator took %.1f s) plus build_h (%.1f s)"
              % (nc, m, N, counts["iters"], counts["matvecs"], counts["seconds"], t_build))
    line = {"impl": "reference", "metric": METRIC, "value": t_solve, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_solve * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(W, precision=args.precision, degree_group=args.degree_group,
                           parallelism="single"),
            "projected": True,
            "oracle_counts": counts,
            "cpu_baseline": {"value": t_solve, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
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
    half = args.storage == "half"
    if args.h_free:
        args.no_e2e = args.no_extras = args.no_cpu_baseline = True
    H = None if args.h_free else pkg.colmajor_empty(N, N, device="cuda:%d" % local_rank)
    evecs = pkg.colmajor_empty(N, nev, device="cuda:%d" % local_rank)
    stream = torch.cuda.current_stream()

    prec = PRECISIONS[args.precision]

    def step():
        if args.h_free:
            return ctx.solve_bse(replica_seed(W["seed"], rank), W["Nk"], W["Nv"], W["Nc"], nev,
                                 nex, tol=W["tol"], deg_max=W["deg_max"], evecs=evecs,
                                 precision=prec, degree_group=args.degree_group,
                                 half_storage=half)
        ctx.build_hamiltonian(replica_seed(W["seed"], rank), W["Nk"], W["Nv"], W["Nc"], out=H)
        return ctx.solve(H, nev, nex, tol=W["tol"], deg_max=W["deg_max"], evecs=evecs,
                         precision=prec, degree_group=args.degree_group, half_storage=half)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local_rank, args.clock_log.replace("{rank}", str(local_rank)) if args.clock_log else None)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    ev0.record(stream)
    stats, stats_evals = [], []
    for k in range(args.steps):
        evs[k].record(stream)
        out = step()
        stats.append(out[3])
        stats_evals.append(out[0])
    evs[args.steps].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms_max = slowest(ms, dist, device="cuda")

    # end to end through the host-buffer entry point: one call with H in
    # page-locked host memory (the library copies its lower triangle),
    # eigenvectors and eigenvalues out.  The call also allocates the
    # context's device copy of H (40 GB at N = 50000).  The buffer is filled
    # just before the call: on the GB300 host, repeated copies from the same
    # 40 GB page-locked buffer slowed down over tens of seconds (to 60-150
    # GB/s from 206), while the first copy after filling ran at full rate.
    e2e_s = None
    if not args.no_e2e:
        # page-locked host buffers from the library (bsechase_host_alloc)
        Hcol = pkg.host_empty((N, N))      # column-major H
        torch.from_numpy(Hcol).copy_(H)
        Zh = pkg.host_empty((N, nev))
        t0 = time.perf_counter()
        st_e2e = ctx.solve_host(Hcol, nev, nex, tol=W["tol"], deg_max=W["deg_max"], evecs=Zh,
                                precision=prec, degree_group=args.degree_group,
                                half_storage=half)[3]
        e2e_s = slowest(time.perf_counter() - t0, dist, device="cuda")
        del Hcol, Zh

    # one solve each of the other modes on the same matrix, after the timed
    # region: the mixed precision mode (per-eigenpair differences from the
    # FP64 solve of the last timed step) and the degrees of Eq. (S1) as they
    # are (no degree groups)
    extras = {}
    if not args.no_extras and world == 1 and args.precision == "fp64" and not half:
        ev_ref = stats_evals[-1]
        V_ref = evecs.clone()

        def timed(**kw):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = ctx.solve(H, nev, nex, tol=W["tol"], deg_max=W["deg_max"], **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            return out, e0.elapsed_time(e1) / 1e3

        (ev_m, V_m, r_m, st_m), t_m = timed(precision=PRECISIONS["mixed"],
                                             degree_group=args.degree_group)
        rel = np.abs(ev_m - ev_ref) / np.abs(ev_ref)
        # per pair: 1 - |<v_mixed, v_fp64>| (phase-free overlap of the unit vectors)
        ov = torch.abs(torch.sum(V_m.conj() * V_ref, dim=0)).cpu().numpy()
        extras["mixed"] = {
            "value": t_m, "unit": UNIT, "iters": st_m["iters"],
            "filter_matvecs": st_m["filter_matvecs"],
            "filter_matvecs_low": st_m["filter_matvecs_low"],
            "filter_matvecs_mid": st_m["filter_matvecs_mid"],
            "max_resid": float(np.max(r_m)),
            "eval_rel_diff_vs_fp64": {"max": float(np.max(rel)), "median": float(np.median(rel)),
                                      "per_pair": [float("%.3g" % x) for x in rel]},
            "evec_one_minus_overlap_vs_fp64": {"max": float(np.max(1.0 - ov)),
                                               "median": float(np.median(1.0 - ov))}}
        del V_m
        (ev_0, V_0, r_0, st_0), t_0 = timed(precision=prec, degree_group=0)
        extras["degree_group_0"] = {"value": t_0, "unit": UNIT, "iters": st_0["iters"],
                                    "matvecs": st_0["matvecs"], "max_resid": float(np.max(r_0))}
        del V_0
        # the same solve with H generated straight into its tensor-core slices
        # (chase_solve_bse: the 16 N^2 bytes of H are never stored); generator
        # included, like the timed step
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev_h, V_h, r_h, st_h = ctx.solve_bse(replica_seed(W["seed"], rank), W["Nk"], W["Nv"],
                                             W["Nc"], nev, nex, tol=W["tol"],
                                             deg_max=W["deg_max"], precision=prec,
                                             degree_group=args.degree_group)
        e1.record(stream)
        torch.cuda.synchronize()
        extras["h_not_stored"] = {
            "value": e0.elapsed_time(e1) / 1e3, "unit": UNIT, "iters": st_h["iters"],
            "device_bytes_not_stored": 16 * N * N,
            "same_bits_as_stored_h": bool(np.array_equal(ev_h, ev_ref) and
                                          torch.equal(V_h, V_ref))}
        del V_h
        # the same solve on the slices of H's lower triangle (half storage)
        (ev_t, V_t, r_t, st_t), t_t = timed(precision=prec, degree_group=args.degree_group,
                                             half_storage=True)
        T = (N + 127) // 128
        rel_t = np.abs(ev_t - ev_ref) / np.abs(ev_ref)
        extras["half_storage"] = {
            "value": t_t, "unit": UNIT, "iters": st_t["iters"], "matvecs": st_t["matvecs"],
            "max_resid": float(np.max(r_t)),
            "eval_rel_diff_vs_full": {"max": float(np.max(rel_t)),
                                      "median": float(np.median(rel_t))},
            "slice_bytes": 12 * T * (T + 1) * 128 * 64 * 2,
            "slice_bytes_full": 12 * (128 * T) ** 2 * 2,
            "tc_kernel_tflops": st_t["tc_kernel_tflops"]}
        # and without storing H: the lower triangle's slices generated (H's
        # whole footprint is the half-storage slices)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ev_g, V_g, _, st_g = ctx.solve_bse(replica_seed(W["seed"], rank), W["Nk"], W["Nv"],
                                           W["Nc"], nev, nex, tol=W["tol"], deg_max=W["deg_max"],
                                           precision=prec, degree_group=args.degree_group,
                                           half_storage=True)
        e1.record(stream)
        torch.cuda.synchronize()
        extras["h_not_stored_half_storage"] = {
            "value": e0.elapsed_time(e1) / 1e3, "unit": UNIT, "iters": st_g["iters"],
            "h_bytes_on_device": extras["half_storage"]["slice_bytes"],
            "same_bits_as_half_storage": bool(np.array_equal(ev_g, ev_t) and torch.equal(V_g, V_t))}
        del V_t, V_g, V_ref

    if rank == 0:
        st = stats[-1]
        sec = ms_max / 1e3 / args.steps
        roof = roofline(args.precision, st, N, W["workload"])
        if half or args.h_free:
            roof["traffic"] = None          # the DRAM record is the full-storage kernel's
        line = {
            "metric": METRIC, "value": sec, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": dict(W, precision=args.precision, degree_group=args.degree_group,
                           parallelism="replicas" if world > 1 else "single",
                           storage=args.storage, h_stored=not args.h_free),
            "throughput_solves_per_s": replica_throughput(world, args.steps, ms_max),
            "step_ms": {"mean": statistics.mean(step_ms), "min": min(step_ms),
                        "std": statistics.pstdev(step_ms), "n": len(step_ms)},
            "solve": {k: st[k] for k in ("iters", "matvecs", "filter_matvecs",
                                         "filter_matvecs_low", "filter_launches", "ms_lanczos",
                                         "ms_filter", "ms_qr", "ms_rr", "ms_resid",
                                         "ms_total", "filter_tflops", "tc_kernel_ms",
                                         "tc_kernel_launches", "tc_kernel_tflops")},
            "roofline": roof,
            "e2e": None if e2e_s is None else {
                "value": e2e_s, "unit": UNIT, "h2d_bytes_per_step": st_e2e["h2d_bytes"],
                "d2h_bytes_per_step": st_e2e["d2h_bytes"] + 16 * nev,
                "ms_h2d": st_e2e["ms_h2d"]},
            "gpu_launches": int(sum(s["kernel_launches"] for s in stats) + 2 * args.steps),
            "clocks": ck,
        }
        line.update(extras)
        if world == 1 and not args.no_cpu_baseline:
            counts = dict(iters=st["iters"], matvecs=st["matvecs"])
            smp = cpu_oracle_sample(W)
            t_cpu = project_solve(smp, counts)
            one = cpu_oracle_single_thread(W)
            line["cpu_baseline"] = {
                "value": t_cpu, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                "projected": True,
                "sample": ("oracle on the dense N=%d matrix, all cores: build_h %.1f s, filter "
                           "product over %d columns %.3e s per column, QR phase %.2f s, "
                           "Rayleigh-Ritz without its H product %.2f s; projected with this "
                           "solve's %d iterations and %d H*v products"
                           % (N, smp["t_build"], smp["n_cols"], smp["t_mv"], smp["t_qr"],
                              smp["t_rr"], counts["iters"], counts["matvecs"])),
                "single_thread": None if one is None else {
                    "value": project_solve(one, counts), "unit": UNIT, "cores": 1,
                    "projected": True,
                    "sample": ("the same oracle steps with one thread at N=%d, products "
                               "scaled by N^2, QR and Rayleigh-Ritz by N" % one["n_small"])}}
    ctx.close()
    if rank == 0 and world == 1 and not args.no_serving:
        # the serving mix on the freed device (its own server and contexts)
        del H, evecs
        torch.cuda.empty_cache()
        sv = serving_mix(args)
        line["serving"] = {k: sv[k] for k in ("metric", "value", "unit", "p50_s", "p99_s",
                                              "solves_per_s", "requests", "ok",
                                              "warm_requests", "arrival_rate_per_s",
                                              "calibrated_capacity_per_s", "slots",
                                              "product_batching")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_serving(args):
    """The serving mix alone: one JSON line."""
    from paper_2006_08498_gb300 import build as pkg_build
    pkg_build.build()
    print(json.dumps(serving_mix(args)), flush=True)


def serving_mix(args):
    """Serving mix: 256 requests, Poisson arrivals, N = 16 Nk with Nk ~
    U{63..1000}, nev ~ U{10..100}, nex = max(10, ceil(nev/2)), 30% warm-start
    neighbours (same seed and Nk as an earlier request, w0 scaled by 1 + d,
    d ~ U[-0.02, 0.02]), admission by an HBM budget.  The arrival rate is set
    to 80% of the throughput measured on a calibration batch.  Returns the
    result as a dict (p50/p99 latency, solves/s, statuses)."""
    import math
    import numpy as np
    import torch
    import paper_2006_08498_gb300 as pkg
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
    if args.batch_window is not None:
        ctx.server_batching(True, args.batch_window)
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
    batch = ctx.server_batch_stats()
    ctx.server_destroy()
    ctx.close()
    line = {"metric": "chase_serving_latency_p99", "value": float(np.percentile(lat, 99)),
            "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "solves_per_s": n_req / (end - start), "requests": n_req, "ok": ok, "statuses": statuses,
            "warm_requests": warm_used, "arrival_rate_per_s": rate,
            "calibrated_capacity_per_s": cap, "slots": args.slots, "budget_bytes": budget,
            "precision": args.precision, "degree_group": args.degree_group, "data": "synthetic",
            "product_batching": None if args.batch_window is None else dict(
                batch, window_s=args.batch_window),
            "config": {"workload": "serving_mix_256", "N": "16*U{63..1000}", "nev": "U{10..100}",
                       "nex": "max(10, ceil(nev/2))", "warm_fraction": 0.3, "tol": 1e-10}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving mix after the timed steps")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision and Eq. (S1)-degree solves after the timed steps")
    ap.add_argument("--clock-log", default=None,
                    help="keep the nvidia-smi samples of the timed region in this CSV ({rank} = rank)")
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--serving", action="store_true", help="run the serving mix instead")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--slots", type=int, default=3,
                    help="serving: concurrent solves (3: the p99 minimum at full throughput)")
    ap.add_argument("--batch-window", type=float, default=None,
                    help="serving: run concurrent solves' products in shared launches, "
                         "waiting up to this many seconds for company (default: off)")
    ap.add_argument("--nk", type=int, default=WORKLOAD["Nk"], help="k-points (N = 16 Nk)")
    ap.add_argument("--nev", type=int, default=WORKLOAD["nev"])
    ap.add_argument("--nex", type=int, default=WORKLOAD["nex"])
    ap.add_argument("--storage", default="full", choices=["full", "half"],
                    help="tensor-core slices of all of H (default) or of its lower triangle")
    ap.add_argument("--h-free", action="store_true",
                    help="each step solves without storing H (chase_solve_bse: the generator "
                         "writes the slices); implies --no-e2e, --no-extras and "
                         "--no-cpu-baseline")
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
