"""Benchmark: distance+gradient pairs/s on the general LCDM+radiation+curvature
batch (4096 cosmologies x 1024 redshifts, z ~ U(0, 10)).

One step = one fused forward+adjoint pass of the whole path over the batch:
FP64 root preparation per cosmology, then per pair the Carlson-integral
distances d_C, t, X and mu (FP32 arithmetic), their tangents with respect to (H0, Om, OL, Or), and the
per-cosmology FP64 reduction of the vector-Jacobian product with fixed random
cotangents (lcdm_distances_vjp).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(adaptive quadrature forward + Leibniz-rule gradient) on a bounded sample.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "distance+gradient pairs/sec (FP32 batched) vs plain FP64 forward, same GB300, ≤2e-6 rel"
UNIT = "pairs/s"
OUTPUTS = ("d_C", "t", "X", "mu")
# Outputs that carry a cotangent in the timed step.  X is computed (a forward
# output of the step) but not differentiated: its FP32 gradient is not within
# the gradient bound for nearly empty open universes (eq. 3.9 with i = B, whose
# terms are O(rho_B^2) and cancel; about 5 % of this batch's pairs), and the
# FP64 path is the one to use where dX/dtheta is needed.
COT_OUTPUTS = ("d_C", "t", "mu")
# Algorithmic work per pair of the timed step (forward d_C, t, X, mu and the
# adjoint of the cotangents on d_C, t, mu), counted by the oracle's operation
# counter (oracle/opcount.py, `python -m oracle.opcount 1000`, 1000 sampled
# pairs of this batch; its output is summarised under profiles/): real FP32
# add/sub + mul, and div + sqrt + transcendental (the special-function unit).
ALG_FLOP_PER_PAIR = 7033.1
ALG_MUFU_PER_PAIR = 390.3
# FP32 floating-point operations the step's two pair launches execute per pair
# (FFMA counted as 2, FADD and FMUL as 1: 638 in the value launch + 1703 in the
# tangent launch) and their DRAM bytes (read + write) per step, from one ncu
# capture of both launches on this workload (profiles/pairs_kernel_fp32_vjp_
# 4096x1024.md; to be set to None whenever the kernels change until re-taken).
EXEC_FLOP_PER_PAIR = 2340.6
TRAFFIC_BYTES = 110.1e6
# Derived peaks (unit counts x maximum SM clock): FP32 FMA, 152 SMs x 128 lanes
# x 2 flops; special-function unit, 152 SMs x 16 per clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
MUFU_PEAK_GOPS = 152 * 16 * 2.07e9 / 1e9


def base_config(b):
    """The workload description both arms report."""
    return {"workload": b.name + " (general LCDM+radiation+curvature batch: 4096 cosmologies x 1024 z)",
            "B": b.B, "n_per_row": 1024, "pairs_per_gpu": int(b.nnz), "outputs": list(OUTPUTS),
            "gradient": "fused VJP w.r.t. (H0, Om, OL, Or), random cotangents on d_C, t, mu (X is computed, "
                        "not differentiated: its FP32 gradient misses the bound on ~5 % of the pairs)"}


def workload(seed_offset=0):
    from paper_2212_01937_gb300 import workloads
    b = workloads.general_batch(seed=2 + seed_offset)
    return b


def sample_clocks(stop, rows):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return
    def reader():
        for line in p.stdout:
            rows.append([x.strip() for x in line.split(",")])
    t = threading.Thread(target=reader, daemon=True)
    t.start()
    stop.wait()
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    t.join(timeout=2)


def clock_summary(rows, gpu_index):
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        if len(r) < 9 or r[0] != str(gpu_index):
            continue
        try:
            sm.append(float(r[1]))
            mx = max(mx, float(r[2]))
        except ValueError:
            continue
        for n, v in zip(names, r[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
            "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(b, budget_s, seed=0):
    """Oracle (O1 quadrature + O4 Leibniz gradient) pairs/s on a random sample."""
    import oracle
    rng = np.random.default_rng(seed)
    def run(n):
        idx = np.sort(rng.choice(b.nnz, n, replace=False))
        rows = np.searchsorted(b.offsets, idx, side="right") - 1
        z = b.z[idx].astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.quad_distances(b.params[rows], z, np.arange(n + 1), grad=True)
        return time.perf_counter() - t0
    n0 = min(2000, b.nnz)
    t = run(n0)
    n = int(min(max(n0, budget_s / max(t, 1e-9) * n0), 2_000_000, b.nnz))
    t = run(n)
    return n / t, n


def cpu_model():
    """Host CPU model (lscpu's model name, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_carlson_rate(b, budget_s, seed=0):
    """The Carlson oracle (O2, eqs. 3.7-3.9 / B.1-B.3; forward values only)
    pairs/s on one thread, on a random sample.  The roots (per cosmology,
    companion matrix and exact-residual polish) are computed before the timed
    region: they are amortised over a row's pairs."""
    import oracle
    from oracle import roots as oroots
    rng = np.random.default_rng(seed)
    def run(n):
        idx = np.sort(rng.choice(b.nnz, n, replace=False))
        rows = np.searchsorted(b.offsets, idx, side="right") - 1
        z = b.z[idx].astype(np.float32).astype(np.float64)
        # the sample's rows as CSR (idx is sorted, so z is in row order): one
        # root solve per cosmology, as the method amortises it
        urows, counts = np.unique(rows, return_counts=True)
        P = b.params[urows]
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        rr = oroots.roots_x(P)
        perm = oroots.permutations(*rr)
        t0 = time.perf_counter()
        oracle.carlson_distances(P, z, offs, roots=rr, perm=perm)
        return time.perf_counter() - t0
    n0 = min(2000, b.nnz)
    t = run(n0)
    n = int(min(max(n0, budget_s / max(t, 1e-9) * n0), 2_000_000, b.nnz))
    t = run(n)
    return n / t, n


def fig3_comparator(nz=2000, budget_s=1.0):
    """The speed study of Sec. 3.2.2 (Fig. 3) on one host thread: d_C (and t
    where the method gives it) from z1 = 0 to each of nz redshifts
    z ~ logU(1e-3, 1e3) for the flat (0.3, 0.7) setup without and with
    Omega_r0 = 1e-5, by the Carlson oracle (eqs. 3.7-3.9 / B.1-B.3, complex
    FP64), the Legendre form (eqs. B.4-B.7), the hypergeometric solution
    (flat radiationless only) and adaptive quadrature (forward only).
    Pairs/s of each, best of repeated calls within budget_s; the root
    solve and the Legendre root assignment are per cosmology and excluded."""
    import oracle
    rng = np.random.default_rng(9)
    z = np.sort(10.0 ** rng.uniform(-3, 3, nz))
    off = np.array([0, nz], dtype=np.int64)
    out = {"z": "logU(1e-3, 1e3), %d values, 1 thread" % nz}

    def rate(f):
        best, t_end = None, time.perf_counter() + budget_s
        while True:
            t0 = time.perf_counter()
            f()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
            if time.perf_counter() > t_end:
                return nz / best

    from oracle import roots as oroots
    for name, p in (("flat_radiationless", [70.0, 0.3, 0.7, 0.0]), ("flat_radiation_1e-5", [70.0, 0.3, 0.7, 1e-5])):
        P = np.array([p])
        rr = oroots.roots_x(P)
        perm = oroots.permutations(*rr)
        asg = oracle.legendre_assignment(P)
        row = {"carlson": rate(lambda: oracle.carlson_distances(P, z, off, roots=rr, perm=perm)),
               "legendre": rate(lambda: oracle.legendre_distances(P, z, off, assignment=asg)),
               "quad": rate(lambda: oracle.quad_distances(P, z, off))}
        if p[3] == 0.0:
            row["hyp2f1"] = rate(lambda: oracle.hyp2f1_flat_distance(70.0, 0.3, z))
        out[name] = {k: {"value": v, "unit": UNIT} for k, v in row.items()}
    out["note"] = ("context for the paper's Fig. 3 (plotted, not tabulated); carlson and legendre give d_C, t "
                   "(carlson also X), hyp2f1 d_C only, quad all three")
    return out


def _oracle_chunk(task):
    """Worker of cpu_oracle_rate_all: the oracle on one slice of pairs
    (params rows, redshifts); returns the seconds it took."""
    import oracle
    params, z = task
    t0 = time.perf_counter()
    oracle.quad_distances(params, z, np.arange(z.size + 1), grad=True)
    return time.perf_counter() - t0


def cpu_oracle_rate_all(b, budget_s, seed=0, procs=None):
    """The same oracle run on all host cores: a spawn-started process pool
    (safe after CUDA initialisation), each process on its own slice of a random
    sample sized for about budget_s of wall time.  Returns (pairs/s, pairs,
    processes)."""
    import multiprocessing as mp
    if not procs:
        procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    rng = np.random.default_rng(seed)
    r1, _ = cpu_oracle_rate(b, budget_s=1.0, seed=seed)          # single-process rate, for sizing
    n = int(min(max(procs * 500, r1 * procs * budget_s), b.nnz))
    idx = np.sort(rng.choice(b.nnz, n, replace=False))
    rows = np.searchsorted(b.offsets, idx, side="right") - 1
    z = b.z[idx].astype(np.float32).astype(np.float64)
    cuts = np.linspace(0, n, procs + 1).astype(np.int64)
    tasks = [(b.params[rows[cuts[i]:cuts[i + 1]]], z[cuts[i]:cuts[i + 1]]) for i in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_chunk, [(b.params[:1], b.z[:1])] * procs)   # start-up and oracle load, untimed
        t0 = time.perf_counter()
        pool.map(_oracle_chunk, tasks)
        wall = time.perf_counter() - t0
    return n / wall, n, procs


def reference_arm(args):
    """--impl reference: the FP64 CPU oracle timed on the host, same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    b = workload()
    rates, walls = [], []
    nsample, procs = 0, 1
    for step in range(args.warmup + args.steps):
        r, nsample, procs = cpu_oracle_rate_all(b, budget_s=min(20.0, 60.0 / max(1, args.steps + args.warmup)),
                                                seed=step)
        if step >= args.warmup:
            rates.append(r)
            walls.append(nsample / r)
    v = float(np.mean(rates))
    # each step is a bounded random sample of the workload's pairs: the step
    # time reported is the sample's measured wall time, not an extrapolation
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(walls)),
            "pairs_per_step": int(nsample),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": base_config(b),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": "%d random pairs of the workload per step over %d processes (adaptive "
                                       "quadrature forward + Leibniz gradient)" % (nsample, procs),
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="use the default launch shape")
    ap.add_argument("--no-vi", action="store_true", help="skip the variational-inference step timing")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged log-likelihood step timing")
    ap.add_argument("--no-limits", action="store_true",
                    help="skip the general-limits and age/horizon timings")
    ap.add_argument("--no-bhm", action="store_true", help="skip the latent-redshift VI step timing")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the single-cosmology latency and full-size precision-stress lines")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    from paper_2212_01937_gb300 import lcdm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lcdm.load()

    b = workload(seed_offset=rank)   # weak scaling: each rank owns a full batch of its own
    B, npairs = b.B, b.nnz
    params = torch.tensor(b.params, device=dev)
    offsets = torch.tensor(b.offsets, device=dev)
    z = torch.tensor(b.z, dtype=torch.float32, device=dev)
    g = torch.Generator(device="cpu").manual_seed(7 + rank)
    cot = {n: torch.randn(npairs, generator=g).to(dev) for n in COT_OUTPUTS}
    call = lcdm.Call(params, z, offsets, precision="fp32")
    tune = None if args.no_autotune else lcdm.autotune(params, z, offsets, outputs=OUTPUTS, cot=cot,
                                                         precision="fp32")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step():
        return lcdm.distances_vjp(params, z, cot, offsets, outputs=OUTPUTS, call=call)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = lcdm.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stop, rows = threading.Event(), []
    th = threading.Thread(target=sample_clocks, args=(stop, rows), daemon=True)
    th.start()
    time.sleep(0.5)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record()
        res = step()
        ev[i][1].record()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    stop.set()
    th.join(timeout=10)
    launches = lcdm.launch_count() - launches0
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / args.steps
    ms, value = aggregate(ms, npairs, world, dist, dev)

    # device time of the pair kernel alone: CUDA-graph replays of (L2 flush + step)
    # minus replays of (L2 flush + root preparation), so host overheads drop out
    rcall = lcdm.Call(params, torch.zeros(B, device=dev), layout="dense", precision="fp64")
    step_g = graph_ms(lambda: (flush.zero_(), step()), dev)
    prep_g = graph_ms(lambda: (flush.zero_(), lcdm.roots(params, call=rcall)), dev)
    pair_ms = max(step_g - prep_g, 1e-6)
    prep_ms = prep_g - graph_ms(lambda: flush.zero_(), dev)

    # end to end through the C-ABI host-buffer entry point (lcdm_distances_vjp_host):
    # page-locked host arrays in, results back in host arrays, with the chunked
    # host<->device copies inside the timed region (overlapping the kernels)
    p_h = params.cpu().contiguous()
    off_h = offsets.cpu().contiguous()
    z_h = z.cpu().pin_memory()
    cot_h = {n: v.cpu().pin_memory() for n, v in cot.items()}
    host = lcdm.HostVJP(B, npairs, outputs=OUTPUTS, precision="fp32", nchunks=5, device=dev,
                        block=(tune or {}).get("block", 0), blocks_per_sm=(tune or {}).get("blocks_per_sm", 0),
                        lane_map=(tune or {}).get("lane_map", "tuned"))
    h2d = p_h.numel() * 8 + off_h.numel() * 8 + z_h.numel() * 4 + sum(v.numel() * 4 for v in cot_h.values())
    d2h = sum(host.out[n].numel() * 4 for n in OUTPUTS) + host.grad.numel() * 8 + host.status.numel() * 4

    def e2e_step():
        return host(p_h, z_h, cot_h, off_h)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms, e2e_value = aggregate(e2e_ms, npairs, world, dist, dev)

    line = None
    if rank == 0:
        clocks = clock_summary(rows, local)
        achieved = ALG_FLOP_PER_PAIR * npairs / (pair_ms / 1e3) / 1e12
        mufu = ALG_MUFU_PER_PAIR * npairs / (pair_ms / 1e3) / 1e9
        meas = {"ffma_tflops": 2 * lcdm.probe_rate("ffma", dev) / 1e12,
                "mufu_gops": lcdm.probe_rate("mufu", dev) / 1e9,
                "dfma_tflops": 2 * lcdm.probe_rate("dfma", dev) / 1e12,
                "how": "lcdm_probe: 8 independent chains per thread, 8 x 256-thread blocks per SM, best of 5"}
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES,
                "algorithmic_ops_per_pair": {"flops": ALG_FLOP_PER_PAIR, "mufu": ALG_MUFU_PER_PAIR,
                                             "source": "oracle/opcount.py, 1000 sampled pairs of this batch"},
                "frac_algorithmic": achieved / FP32_PEAK_TFLOPS,
                "frac_algorithmic_of_measured_ffma": achieved / meas["ffma_tflops"],
                "executed_flops_per_pair": EXEC_FLOP_PER_PAIR,
                "frac_executed": (None if EXEC_FLOP_PER_PAIR is None else
                                  EXEC_FLOP_PER_PAIR * npairs / (pair_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS),
                "mufu": {"achieved_gops": mufu, "peak_gops": MUFU_PEAK_GOPS, "frac": mufu / MUFU_PEAK_GOPS,
                         "frac_of_measured": mufu / meas["mufu_gops"]},
                "measured_peaks": meas,
                "kernel": "pairs_kernel<FP32,K=0,X> + pairs_kernel<FP32,K=3,t> (the step's two pair launches)",
                "kernel_ms": pair_ms, "prep_ms": prep_ms,
                "peak_note": "FP32 FMA issue: 152 SMs x 128 lanes x 2 x 2.07 GHz (derived from unit counts and "
                             "the maximum clock; MEASURED_PEAKS has HBM and bf16 only)"}
        extra = {}
        if not args.no_fp64_baseline:
            extra = fp64_baselines(lcdm, params, offsets, b, dev, value)
        extra["accuracy"] = step_accuracy(lcdm, b, params, z, offsets, cot, res, dev)
        cpu = None
        if not args.no_cpu_baseline:
            r1, n1 = cpu_oracle_rate(b, budget_s=6.0)
            r, n, procs = cpu_oracle_rate_all(b, budget_s=10.0)
            cpu = {"value": r, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": "%d random pairs of the workload split over %d processes (spawned), adaptive "
                             "quadrature forward + Leibniz gradient" % (n, procs),
                   "single_thread": {"value": r1, "cores": 1, "sample": "%d random pairs, 1 thread" % n1},
                   "cpu_model": cpu_model()}
            rc, nc = cpu_carlson_rate(b, budget_s=3.0)
            cpu["carlson_forward_single_thread"] = {
                "value": rc, "unit": UNIT, "cores": 1,
                "sample": "%d random pairs, Carlson oracle forward only (no gradient; roots outside the timed "
                          "region), 1 thread" % nc}
            cpu["fig3_comparator"] = fig3_comparator()
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(base_config(b), **{
                    "precision": "FP32 per-pair arithmetic, FP64 root preparation and reductions",
                    "l2": "flushed (256 MiB write) before every timed step",
                    "launch": tune, "wall_s_timed": t_wall}),
                "gpu_launches": launches, "clocks": clocks, "roofline": roof,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": e2e_ms, "api": "lcdm_distances_vjp_host, 5 chunks (ramped 1 2 3 2 1), page-locked host arrays"},
                "cpu_baseline": cpu}
        line.update(extra)
        if not args.no_vi:
            line["vi_step"] = vi_step_rate(dev)
        if not args.no_ragged:
            line["ragged_step"] = ragged_step_rate(dev)
        if not args.no_limits:
            line["between_step"] = between_step_rate(dev)
            line["limits_step"] = limits_rate(dev)
        if not args.no_bhm:
            line["bhm_step"] = bhm_step_rate(dev)
        if not args.no_configs:
            line["config1_fp64_latency"] = config1_rate(lcdm, dev)
            line["config5_precision_stress"] = config5_rate(lcdm, dev)
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def aggregate(ms, npairs, world, dist=None, device=None):
    """Whole-job figures under weak scaling: every rank times its own batch of
    npairs; the job's step time is the slowest rank's (max over ranks, after a
    barrier) and its rate is all ranks' pairs over that time."""
    import torch
    if dist is not None and dist.is_initialized():
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    return ms, npairs * world / (ms / 1e3)


def graph_ms(fn, dev, reps=10):
    """Device milliseconds per call of fn, from replays of one CUDA graph that
    holds `reps` calls (no host work between the kernels)."""
    import torch
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream(dev).wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            fn()
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (3 * reps)


def vi_step_rate(dev, steps=10):
    """One variational-inference step of the 10^6-supernova model (256 guide
    samples x 10^6 shared redshifts: fused log-likelihood and gradient, ELBO
    gradient, Adam), replayed from its CUDA graph."""
    import torch
    from paper_2212_01937_gb300 import vi, workloads
    d = workloads.supernovae()
    centre, scale = vi.default_guide(d.extra["truth"])
    opt = vi.GaussianVI(torch.tensor(d.z, dtype=torch.float32, device=dev), torch.tensor(d.m_obs, device=dev),
                        centre, scale, M=d.M, sigma=d.sigma, samples=256)
    for _ in range(3):
        opt.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        opt.step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"workload": d.name + " x 256 guide samples (10^6 mock SNe Ia, shared z), FP32, CUDA-graph replay",
            "ms_per_step": ms, "pairs_per_step": opt.pairs_per_step,
            "value": opt.pairs_per_step / (ms / 1e3), "unit": UNIT}


def ragged_step_rate(dev, steps=10):
    """One log-likelihood + gradient step over the ragged batch (16384
    cosmologies, floor(10^U(0, 5)) redshifts each, about 1.46e8 pairs in CSR
    layout, per-row mock magnitudes), replayed from a CUDA graph."""
    import torch
    from paper_2212_01937_gb300 import lcdm, workloads
    d = workloads.ragged_batch()
    params = torch.tensor(d.params, device=dev)
    off = torch.tensor(d.offsets, device=dev)
    z = torch.tensor(d.z, dtype=torch.float32).to(dev)
    m = torch.tensor(d.m_obs, dtype=torch.float32).to(dev)
    call = lcdm.Call(params, z, off, precision="fp32")
    ms = graph_ms(lambda: lcdm.gauss_loglike(params, z, m, off, M=d.M, sigma=d.sigma, call=call), dev, reps=steps)
    return {"workload": d.name + " (16384 cosmologies x floor(10^U(0,5)) z, CSR), FP32, CUDA-graph replay",
            "pairs_per_step": int(d.nnz), "ms_per_step": ms, "value": d.nnz / (ms / 1e3), "unit": UNIT}


def bhm_step_rate(dev, steps=10):
    """One VI step of the Sec. 4 model with latent redshifts: 10^6 mock SNe,
    4 guide samples (partial-MVN guide over (Om, OL) and every log-redshift),
    fused magnitude log-likelihood with its gradients w.r.t. (Om, OL) and each
    latent redshift, redshift likelihood and gamma prior, ELBO gradient, Adam;
    replayed from its CUDA graph."""
    import torch
    from paper_2212_01937_gb300 import bhm, workloads
    d = workloads.bhm_supernovae()
    vi = bhm.PMVNGuideVI(torch.tensor(d.extra["z_hat"], device=dev), torch.tensor(d.m_obs, device=dev), samples=4)
    for _ in range(3):
        vi.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        vi.step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"workload": d.name + " x 4 guide samples (latent redshifts, Gamma(2, rate 3) prior, sigma_mu 0.14, "
                                 "sigma_z 0.04), FP32, CUDA-graph replay",
            "ms_per_step": ms, "pairs_per_step": vi.pairs_per_step, "value": vi.pairs_per_step / (ms / 1e3),
            "unit": UNIT}


def between_step_rate(dev):
    """Fused forward + adjoint with general lower limits: 4096 rows, each with
    its own z1 ~ U(0, 3) and 1024 upper limits z2 = z1 + U(0, 10), FP32,
    cotangents on d_C, t, X, mu (the per-row shift, root preparation, pair
    maps, pair kernel and gradient chain rule), replayed from a CUDA graph."""
    import torch
    from paper_2212_01937_gb300 import lcdm, workloads
    d = workloads.between_batch()
    params = torch.tensor(d.params, device=dev)
    off = torch.tensor(d.offsets, device=dev)
    z1 = torch.tensor(d.extra["z1"], device=dev)
    z = torch.tensor(d.z, dtype=torch.float32).to(dev)
    g = torch.Generator(device="cpu").manual_seed(11)
    cot = {n: torch.randn(d.nnz, generator=g).to(dev) for n in COT_OUTPUTS}
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    f = lambda: lcdm.distances_between(params, z1, z, off, outputs=OUTPUTS, cot=cot, precision="fp32")
    ms = graph_ms(lambda: (flush.zero_(), f()), dev) - graph_ms(lambda: flush.zero_(), dev)
    return {"workload": d.name + " (z1 ~ U(0,3) per row, z2 = z1 + U(0,10)), FP32 fused VJP, "
                                 "CUDA-graph replay, L2 flushed (cotangents on d_C, t, mu)",
            "pairs_per_step": int(d.nnz), "ms_per_step": ms, "value": d.nnz / (ms / 1e3), "unit": UNIT}


def limits_rate(dev):
    """Age t(z1, inf) and comoving horizon chi(z1, inf) with their gradient,
    65536 rows (z1 half U(0, 10), half logU(10, 1100)), FP64, CUDA-graph replay."""
    import torch
    from paper_2212_01937_gb300 import lcdm, workloads
    d = workloads.limits_batch()
    params = torch.tensor(d.params, device=dev)
    z1 = torch.tensor(d.extra["z1"], device=dev)
    cc = torch.ones(d.B, dtype=torch.float64, device=dev)
    ms = graph_ms(lambda: lcdm.limits(params, z1, cot_chi=cc, cot_t=cc, grad=True), dev)
    return {"workload": d.name + " rows, age + horizon + gradient, FP64, CUDA-graph replay",
            "rows_per_step": d.B, "ms_per_step": ms, "value": d.B / (ms / 1e3), "unit": "rows/s"}


def fp64_baselines(lcdm, params, offsets, b, dev, headline):
    """The denominators named by the metric, on the same GPU and batch: the
    plain FP64 forward (d_C, t, X, mu) launched once per cosmology (4096
    launches of lcdm_distances, every call's arguments and buffers prepared
    beforehand, the launches replayed from one CUDA graph so that no host work
    is timed), and the same forward batched in one launch.  The headline's
    ratio to each is reported; the batched one is the honest denominator."""
    import ctypes
    import torch
    z64 = torch.tensor(b.z, dtype=torch.float64, device=dev)
    n = int(b.offsets[1] - b.offsets[0])
    outs = ("d_C", "t", "X", "mu")
    lib = lcdm.load()
    calls = []
    for r in range(b.B):
        c = lcdm.Call(params[r:r + 1], z64[r * n:(r + 1) * n], layout="dense", precision="fp64", block=128,
                      blocks_per_sm=1)
        out, vp = c.out_buffers(outs)
        calls.append((c, out, vp))

    def plain():
        for c, out, vp in calls:
            lib.lcdm_distances(*c.common(), vp, lcdm._ptr(c.status), *c.tail())

    bc = lcdm.Call(params, z64, offsets, precision="fp64")
    bout, bvp = bc.out_buffers(outs)

    def batched():
        lib.lcdm_distances(*bc.common(), bvp, lcdm._ptr(bc.status), *bc.tail())

    res = {}
    for name, f, reps in (("plain_per_cosmology", plain, 1), ("batched", batched, 5)):
        ms = graph_ms(f, dev, reps=reps)
        res[name] = {"value": b.nnz / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "headline_ratio": headline / (b.nnz / (ms / 1e3))}
    res["plain_per_cosmology"]["how"] = ("4096 launches (root preparation + pair kernel each, 1024 pairs), "
                                         "replayed from one CUDA graph")
    res["batched"]["how"] = "one call over the whole batch, replayed from a CUDA graph"
    res["headline_denominator"] = "batched"
    return {"fp64_forward_baseline": res}


def step_accuracy(lcdm, b, params, z, offsets, cot, res, dev, nsample=3000):
    """Accuracy of the timed step: its FP32 outputs on a random sample of
    pairs and its per-cosmology gradient, against the FP64 GPU path on the
    same inputs (the FP64 path is held to 1e-12 of the oracle by the tests).
    Per-pair Jacobians of the sample (FP32 vs FP64) give the per-output
    gradient errors, relative to the largest entry of each pair's row, and
    the count of pairs above the stated bound (3e-5 + 2e-6/z; t 1e-4 + 2e-6/z;
    X, which the step does not differentiate, 1e-3 + 2e-6/z)."""
    import torch
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(b.nnz, nsample, replace=False))
    rows = np.searchsorted(b.offsets, idx, side="right") - 1
    it = torch.tensor(idx, device=dev)
    p_s = params[torch.tensor(rows, device=dev)]
    z_s = z[it]
    off_s = torch.arange(nsample + 1, device=dev)
    names = ("d_C", "t", "X", "mu")
    j64 = lcdm.distances_jac(p_s, z_s.double(), off_s, outputs=names, precision="fp64")
    j32 = lcdm.distances_jac(p_s, z_s, off_s, outputs=names, precision="fp32")
    zz = z_s.double().cpu().numpy()
    acc = {"sample_pairs": nsample}
    for n in names:
        got = res[n][it].double().cpu().numpy()
        want = j64[n].cpu().numpy()
        if n == "mu":
            fin = np.isfinite(want)
            e = np.abs(got[fin] - want[fin])
            acc["mu_abs"] = {"max": float(e.max()), "q99": float(np.quantile(e, 0.99))}
        else:
            e = np.abs(got / want - 1)
            acc[n + "_rel"] = {"max": float(e.max()), "q99": float(np.quantile(e, 0.99))}
        J32 = j32["jac"][n].double().cpu().numpy()
        J64 = j64["jac"][n].cpu().numpy()
        ej = np.abs(J32 - J64).max(axis=1) / np.abs(J64).max(axis=1)
        c0 = {"t": 1e-4, "X": 1e-3}.get(n, 3e-5)
        acc["d" + n + "_jac_rel"] = {"max": float(ej.max()), "q99": float(np.quantile(ej, 0.99)),
                                     "bound": "%g + 2e-6/z" % c0,
                                     "pairs_above_bound": int(np.count_nonzero(ej > c0 + 2e-6 / zz))}
    g64 = lcdm.distances_vjp(params, z.double(), {k: v.double() for k, v in cot.items()}, offsets,
                             precision="fp64")["grad"]
    g32 = res["grad"]
    eg = ((g32 - g64).abs().max(dim=1).values / g64.abs().max(dim=1).values).cpu().numpy()
    acc["grad_vjp_rel_per_cosmology"] = {"max": float(eg.max()), "q99": float(np.quantile(eg, 0.99))}
    acc["reference"] = "FP64 GPU path on the same inputs (z rounded to FP32)"
    return acc


def config1_rate(lcdm, dev):
    """One flat radiationless cosmology (70, 0.3, 0.7), 10^4 redshifts
    z ~ U(0.01, 2), FP64 d_C and mu, forward only (the cubic reduction):
    microseconds per call, from a CUDA-graph replay (device time) and from
    eager calls (with the binding's host work)."""
    import torch
    from paper_2212_01937_gb300 import workloads
    d = workloads.flat_radiationless()
    params = torch.tensor(d.params, device=dev)
    z = torch.tensor(d.z, device=dev)
    off = torch.tensor(d.offsets, device=dev)
    call = lcdm.Call(params, z, off, precision="fp64")
    lib = lcdm.load()
    out, vp = call.out_buffers(("d_C", "mu"))
    f = lambda: lib.lcdm_distances(*call.common(), vp, lcdm._ptr(call.status), *call.tail())
    ms_graph = graph_ms(f, dev, reps=20)
    for _ in range(3):
        f()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(50):
        f()
    torch.cuda.synchronize()
    ms_eager = (time.perf_counter() - t0) * 1e3 / 50
    return {"workload": d.name + " (flat radiationless, z ~ U(0.01, 2)), FP64 d_C + mu, forward",
            "us_per_call_device": ms_graph * 1e3, "us_per_call_eager": ms_eager * 1e3,
            "pairs_per_call": int(d.nnz), "value": d.nnz / (ms_graph / 1e3), "unit": UNIT}


def config5_rate(lcdm, dev, steps=5):
    """Precision stress at full size: 10^4 cosmologies x 10^4 redshifts
    (half within 1e-6 of flatness, half within 1e-6 of the no-Big-Bang
    boundary), z ~ logU(1e-4, 1100), explicit Omega_k0; FP32 forward d_C, t,
    X, mu in one launch (inputs 400 MB, larger than L2).  The error per
    output on 2000 sampled pairs against the FP64 GPU path on the same z."""
    import torch
    from paper_2212_01937_gb300 import workloads
    s = workloads.precision_stress()
    params = torch.tensor(s.params, device=dev)
    off = torch.tensor(s.offsets, device=dev)
    z = torch.tensor(s.z.astype(np.float32), device=dev)
    names = ("d_C", "t", "X", "mu")
    call = lcdm.Call(params, z, off, precision="fp32")
    lib = lcdm.load()
    out, vp = call.out_buffers(names)
    f = lambda: lib.lcdm_distances(*call.common(), vp, lcdm._ptr(call.status), *call.tail())
    for _ in range(2):
        f()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        f()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rng = np.random.default_rng(3)
    idx = torch.tensor(np.sort(rng.choice(s.nnz, 2000, replace=False)), device=dev)
    rows = torch.searchsorted(off, idx, right=True) - 1
    r64 = lcdm.distances(params[rows], z[idx].double(), torch.arange(2001, device=dev), outputs=names,
                         precision="fp64")
    err = {}
    for n in names:
        a, w = out[n][idx].double(), r64[n]
        if n == "mu":
            fin = torch.isfinite(w)
            err["mu_abs_max"] = float((a[fin] - w[fin]).abs().max())
        else:
            err[n + "_rel_max"] = float((a / w - 1).abs().max())
    return {"workload": s.name + " (precision stress, near-flat and near the no-Big-Bang boundary), FP32 forward "
                                 "d_C, t, X, mu", "pairs_per_step": int(s.nnz), "ms_per_step": ms,
            "value": s.nnz / (ms / 1e3), "unit": UNIT, "status_nonzero": int((call.status != 0).sum()),
            "error_vs_fp64_gpu_2000_sampled": err}


if __name__ == "__main__":
    main()
