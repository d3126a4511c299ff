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
# Work of the dominant kernel per pair for this workload: FP32 floating-point
# operations (FFMA counted as 2, FADD and FMUL as 1) executed per pair, from
# an ncu capture of this kernel on this workload (its summary is under profiles/).
FLOP_PER_PAIR = 5501.0
# DRAM bytes (read + write) per launch of that kernel from the same capture
# (None once the kernel has changed since the counters were taken).
TRAFFIC_BYTES = 131349248
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def base_config(b):
    """The workload description both arms report."""
    return {"workload": b.name + " (general LCDM+radiation+curvature batch: 4096 cosmologies x 1024 z)",
            "B": b.B, "n_per_row": 1024, "pairs_per_gpu": int(b.nnz), "outputs": list(OUTPUTS),
            "gradient": "fused VJP w.r.t. (H0, Om, OL, Or), random cotangents on all outputs"}


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
    """The Carlson oracle (O2, eqs. 3.7-3.9 / B.1-B.3 from the companion-matrix
    roots; forward values only) pairs/s on one thread, on a random sample."""
    import oracle
    rng = np.random.default_rng(seed)
    def run(n):
        idx = np.sort(rng.choice(b.nnz, n, replace=False))
        rows = np.searchsorted(b.offsets, idx, side="right") - 1
        z = b.z[idx].astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        oracle.carlson_distances(b.params[rows], z, np.arange(n + 1))
        return time.perf_counter() - t0
    n0 = min(2000, b.nnz)
    t = run(n0)
    n = int(min(max(n0, budget_s / max(t, 1e-9) * n0), 2_000_000, b.nnz))
    t = run(n)
    return n / t, n


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
    rates = []
    nsample, procs = 0, 1
    for step in range(args.warmup + args.steps):
        r, nsample, procs = cpu_oracle_rate_all(b, budget_s=min(20.0, 60.0 / max(1, args.steps + args.warmup)),
                                                seed=step)
        if step >= args.warmup:
            rates.append(r)
    v = float(np.mean(rates))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * b.nnz / v,
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
    cot = {n: torch.randn(npairs, generator=g).to(dev) for n in OUTPUTS}
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
    host = lcdm.HostVJP(B, npairs, outputs=OUTPUTS, precision="fp32", nchunks=12, device=dev,
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
        achieved = None if FLOP_PER_PAIR is None else FLOP_PER_PAIR * npairs / (pair_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None if achieved is None else achieved / FP32_PEAK_TFLOPS, "traffic": TRAFFIC_BYTES,
                "kernel": "pairs_kernel<FP32,K=3,t,X>", "kernel_ms": pair_ms, "prep_ms": prep_ms,
                "peak_note": "FP32 FMA issue: 152 SMs x 128 lanes x 2 x 2.07 GHz (derived, nominal clock)"}
        extra = {}
        if not args.no_fp64_baseline:
            extra = fp64_baselines(lcdm, params, offsets, b, dev)
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
                "sample": "%d random pairs, Carlson oracle forward only (no gradient), 1 thread" % nc}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(base_config(b), **{
                    "precision": "FP32 per-pair arithmetic, FP64 root preparation and reductions",
                    "l2": "flushed (256 MiB write) before every timed step",
                    "launch": tune, "wall_s_timed": t_wall}),
                "gpu_launches": launches, "clocks": clocks, "roofline": roof,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": e2e_ms, "api": "lcdm_distances_vjp_host, 12 chunks, page-locked host arrays"},
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
    cot = {n: torch.randn(d.nnz, generator=g).to(dev) for n in OUTPUTS}
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    f = lambda: lcdm.distances_between(params, z1, z, off, outputs=OUTPUTS, cot=cot, precision="fp32")
    ms = graph_ms(lambda: (flush.zero_(), f()), dev) - graph_ms(lambda: flush.zero_(), dev)
    return {"workload": d.name + " (z1 ~ U(0,3) per row, z2 = z1 + U(0,10)), FP32 fused VJP, "
                                 "CUDA-graph replay, L2 flushed",
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


def fp64_baselines(lcdm, params, offsets, b, dev):
    """The denominators named by the metric: the plain FP64 forward kernel
    launched once per cosmology, and the same kernel batched."""
    import torch
    z64 = torch.tensor(b.z, dtype=torch.float64, device=dev)
    n = b.offsets[1] - b.offsets[0]
    ws = lcdm.Call(params[:1], z64[:n], layout="dense", precision="fp64", block=128, blocks_per_sm=1).ws
    outs = ("d_C", "t", "X", "mu")

    def plain():
        for r in range(b.B):
            lcdm.distances(params[r:r + 1], z64[r * n:(r + 1) * n], None, outputs=outs, layout="dense",
                           precision="fp64", block=128, blocks_per_sm=1, workspace=ws)

    def batched():
        lcdm.distances(params, z64, offsets, outputs=outs, precision="fp64")

    res = {}
    for name, f, reps in (("plain_per_cosmology", plain, 1), ("batched", batched, 3)):
        f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"value": b.nnz / (ms / 1e3), "unit": UNIT, "ms_per_step": ms}
    return {"fp64_forward_baseline": res}


if __name__ == "__main__":
    main()
