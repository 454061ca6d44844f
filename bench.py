"""Benchmark of the MHM hot path: local solves + skeleton assembly, coarse
elements per second, on the heterogeneous workload (32x32 squares = 2048 coarse
triangles, P1 locals refined 5 times = 561 DOFs, m = 2 subfaces with P2
multipliers = 18 lambda right-hand sides + 1 source, log-uniform kappa with
log10 kappa ~ U[-2, 2] per fine triangle, f = 1).

One step = mhm_local_solve_batch + mhm_assemble_skeleton over all coarse
triangles.  Prints one JSON line (see the design doc for every key).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_hetero_fp64"


def algorithmic_fmas(P, N, R):
    """Multiply-adds of the block-tridiagonal forward elimination of one K: per
    level, Cholesky of the b x b block, W = L^-1 C^T, the Schur update W^T W,
    the forward solve of R right-hand sides, their update W^T Y and the Gram
    matrix Y^T Y (symmetric halves counted once)."""
    def size(lev):
        if P == 1:
            return N + 1 - lev - (lev == 0)
        if lev == N:
            return 1
        return (2 * N - 2 * lev + 1) + (2 * N - 2 * lev) - (lev == 0)
    tot = 0.0
    for lev in range(N + 1):
        b = size(lev)
        bn = size(lev + 1) if lev < N else 0
        tot += b * (b - 1) * (b + 1) / 6.0           # Cholesky
        tot += bn * b * (b + 1) / 2.0                 # W = L^-1 C^T
        tot += b * bn * (bn + 1) / 2.0                # S' -= W^T W
        tot += R * b * (b + 1) / 2.0                  # Y = L^-1 G
        tot += bn * R * b                             # G' -= W^T Y
        tot += b * R * (R + 1) / 2.0                  # Gram += Y^T Y
    return tot


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench.csv") if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else "/tmp/clocks_bench.csv"

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            tok = [t.strip() for t in line.split(",")]
            if len(tok) < 9:
                continue
            try:
                sm.append(float(tok[1]))
                mx = max(mx, float(tok[2]))
            except ValueError:
                continue
            for nme, v in zip(names, tok[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(w, Ks, kap):
    """FP64 oracle local solves for coarse triangles Ks (run in a worker)."""
    from oracle.local import solve_local
    from oracle.mesh import build_mesh
    from oracle.run import source_fn
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    f = float(w.source_value) if w.source == "const" else source_fn("sinsin", w.source_value, w.source_freq)
    for i, K in enumerate(Ks):
        solve_local(mesh, int(K), w.r, w.degree, kap[i], f)
    return len(Ks)


def _worker_init():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def time_oracle(w, n_sample, cores, pool=None):
    """Seconds for the oracle's local solves of n_sample coarse triangles on `cores` processes."""
    from paper_1703_10435_gb300 import workloads as W
    Ks = np.arange(n_sample) % w.n_K
    kap = W.kappa_for(w, Ks)
    chunks = np.array_split(np.arange(n_sample), cores)
    t0 = time.perf_counter()
    if pool is None:
        oracle_sample(w, Ks, kap)
    else:
        futs = [pool.submit(oracle_sample, w, Ks[c], kap[c]) for c in chunks if len(c)]
        for fu in futs:
            fu.result()
    return time.perf_counter() - t0


def make_pool(cores):
    import concurrent.futures
    import multiprocessing as mp
    return concurrent.futures.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn"),
                                                  initializer=_worker_init)


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = make_pool(cores)
    n_sample = max(cores, args.ref_sample)
    time_oracle(w, cores, cores, pool)            # warm the workers
    for _ in range(args.warmup):
        time_oracle(w, cores, cores, pool)
    ts = [time_oracle(w, n_sample, cores, pool) for _ in range(args.steps)]
    pool.shutdown()
    t = float(np.sum(ts))
    value = args.steps * n_sample / t
    line = {
        "impl": "reference", "metric": "coarse elements/s (local solves + skeleton assembly)",
        "value": value, "unit": "coarse elements/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_K": w.n_K, "r": w.r, "degree": w.degree, "m": w.m, "l": w.l,
                   "sample_K_per_step": n_sample, "field": w.field},
        "cpu_baseline": {"value": value, "unit": "coarse elements/s", "cores": cores, "kind": "oracle",
                         "sample": "%d coarse triangles of the workload per step (K = 0..%d)" % (n_sample, n_sample - 1)},
        "e2e": {"value": value, "unit": "coarse elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, w, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1703_10435_gb300 import build, mhm
    from paper_1703_10435_gb300 import workloads as W
    from paper_1703_10435_gb300.pipeline import Pipeline, dirichlet_of, source_of

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    precision = mhm.MHM_MIXED if args.precision == "mixed" else mhm.MHM_FP64
    p = Pipeline.for_workload(w, local_rank, precision)
    kap_host = W.kappa_for(w)
    kap = torch.as_tensor(kap_host, device=dev).contiguous()
    src, gd = source_of(w), dirichlet_of(w)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2 (129 MB)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        p.step(kap, src, gd)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0, "local solve status nonzero"

    sampler = ClockSampler(local_rank)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.zero_()                                  # evict the inputs from L2 between steps
        ev[s][0].record(stream)
        p.local(kap, src)
        ev[s][1].record(stream)
        p.skeleton(gd)
        ev[s][2].record(stream)
    torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    local_ms = [a.elapsed_time(b) for a, b, c in ev]
    t_step = float(np.sum(step_ms))
    clocks = sampler.stop()

    # end to end through the C ABI with host buffers: kappa H2D in, skeleton (A, E, B, F) D2H out
    kap_pin = torch.as_tensor(kap_host).pin_memory()
    outs = [p.A_vals, p.E, p.BK, p.FK]
    outs_pin = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
    kap_dev2 = torch.empty_like(kap)
    h2d = kap_pin.numel() * 8
    d2h = sum(o.numel() * o.element_size() for o in outs)
    for _ in range(2):
        kap_dev2.copy_(kap_pin, non_blocking=True)
        p.step(kap_dev2, src, gd)
        for o, h in zip(outs, outs_pin):
            h.copy_(o, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        kap_dev2.copy_(kap_pin, non_blocking=True)
        p.step(kap_dev2, src, gd)
        for o, h in zip(outs, outs_pin):
            h.copy_(o, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1)

    if world > 1:
        tt = torch.tensor([t_step, t_e2e], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step, t_e2e = float(tt[0]), float(tt[1])
    if rank != 0:
        return

    value = world * w.n_K * args.steps / (t_step * 1e-3)
    e2e = world * w.n_K * args.steps / (t_e2e * 1e-3)
    # roofline of the dominant kernel (the fused local solve): FP64 pipe
    fl = 2.0 * algorithmic_fmas(w.degree, w.N, w.n_I + 1) * w.n_K
    local_s = float(np.mean(local_ms)) * 1e-3
    pipes = mhm.mhm_measure_pipes(local_rank)
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    peak_clock = clocks["sm_max_mhz"] if clocks else 2070.0
    if precision == mhm.MHM_FP64:
        # 2 FP64 FMA per clock per SM on GB300 (1.25 TFLOP/s nominal at 2.07 GHz over 152 SMs)
        peak = 2 * 2 * sms * peak_clock * 1e6 / 1e12
        roof = {"bound": "alu", "pipe": "fp64", "achieved": fl / local_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": fl / local_s / 1e12 / peak, "traffic": None,
                "peak_measured_microbench": pipes["fp64_gflops"] / 1e3,
                "kernel": "k_local_fp64", "flops_per_launch": fl}
    else:
        peak = 2 * 128 * sms * peak_clock * 1e6 / 1e12
        roof = {"bound": "alu", "pipe": "fp32", "achieved": fl / local_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": fl / local_s / 1e12 / peak, "traffic": None,
                "peak_measured_microbench": pipes["fp32_gflops"] / 1e3,
                "kernel": "k_local_mixed", "flops_per_launch": fl}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        pool = make_pool(cores)
        time_oracle(w, cores, cores, pool)
        n_sample = max(cores, args.ref_sample)
        t_cpu = time_oracle(w, n_sample, cores, pool)
        pool.shutdown()
        cpu = {"value": n_sample / t_cpu, "unit": "coarse elements/s", "cores": cores, "kind": "oracle",
               "sample": "%d coarse triangles of the workload (K = 0..%d), local solves" % (n_sample, n_sample - 1)}

    line = {
        "metric": "coarse elements/s (local solves + skeleton assembly)",
        "value": value, "unit": "coarse elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if precision == mhm.MHM_FP64 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": w.name, "n_K": w.n_K, "r": w.r, "degree": w.degree, "n_local": w.n_local,
                   "m": w.m, "l": w.l, "rhs": w.n_I + 1, "field": w.field, "seed": w.seed,
                   "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replica per GPU" if world > 1 else "single GPU"},
        "local_solve_ms": float(np.mean(local_ms)),
        "skeleton_ms": float(np.mean(np.array(step_ms) - np.array(local_ms))),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "coarse elements/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "pipes_gflops": pipes,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--ref-sample", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    from paper_1703_10435_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, w, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
