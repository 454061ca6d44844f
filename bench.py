"""Benchmark of the MHM hot path: local solves + skeleton assembly, coarse
elements per second, on the mixed-precision workload (128x128 squares = 32768
coarse triangles, P1 locals refined 5 times = 561 DOFs, m = 2 subfaces with P2
multipliers = 18 lambda right-hand sides + 1 source, kappa a Gaussian random
field of correlation length 0.02 exponentiated to contrast 1e4, f = 1).

One step = mhm_local_solve_batch + mhm_assemble_skeleton over all coarse
triangles.  Both arithmetic paths are timed: the headline `value` is the
mixed-precision path (FP32 factorisation and solves, FP64 residuals), the
all-FP64 path is reported beside it, with the L2 difference of the
multipliers and of the reconstructed u between the two, and a sample of
coarse triangles checked against the FP64 oracle.  The 2048-element
log-uniform workload is timed as a secondary line, and the P2 (131072 elements) and
uneven-level (8192 elements, levels 3..7) workloads in `more_configs` (3 warm-up and 3
timed steps each, both paths).  The three-dimensional form of the paper's experiment
(Sec. 5: 12288 and 1536 coarse tetrahedra of the unit cube, P2 locals, l = 0 multipliers
on 4 or 16 subfaces) is timed last, FP64, in `three_d`.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W]
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

WORKLOAD = "c3_grf_mixed"
SECONDARY = "c2_hetero_fp64"
MORE = "c5_p2_large,c4_channels"


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

    def __init__(self, index: int, path: str | None = None):
        import tempfile
        self.index = index
        self.proc = None
        # the raw samples (the JSON line carries their summary)
        self.path = path or os.path.join(tempfile.gettempdir(), "clocks_bench_%d.csv" % index)

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
    lf = w.l_per_face(build_mesh(w.nx, w.ny, 1, 0).tri_edges) if w.face_degree else None
    mesh = build_mesh(w.nx, w.ny, w.m, w.l if lf is None else lf)
    f = float(w.source_value) if w.source == "const" else source_fn("sinsin", w.source_value, w.source_freq)
    rk = w.r_per_K
    for i, K in enumerate(Ks):
        solve_local(mesh, int(K), w.r if rk is None else int(rk[K]), w.degree, kap[i], f)
    return len(Ks)


def _worker_init():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def time_oracle(w, n_sample, cores, pool=None):
    """Seconds for the oracle's local solves of n_sample coarse triangles on `cores` processes."""
    from paper_1703_10435_gb300 import workloads as W
    Ks = np.arange(n_sample) % w.n_K
    kap = W.kappa_for(w, Ks) if w.r_per_K is None else W.kappa_levels(w, Ks)
    chunks = np.array_split(np.arange(n_sample), cores)
    t0 = time.perf_counter()
    if pool is None:
        oracle_sample(w, Ks, kap)
    else:
        futs = [pool.submit(oracle_sample, w, Ks[c], [kap[i] for i in c]) for c in chunks if len(c)]
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
        "config": dict(workload_config(w), sample_K_per_step=n_sample, field=w.field),
        "cpu_baseline": {"value": value, "unit": "coarse elements/s", "cores": cores, "kind": "oracle",
                         "sample": "%d coarse triangles of the workload per step (K = 0..%d)" % (n_sample, n_sample - 1)},
        "e2e": {"value": value, "unit": "coarse elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measured_peaks():
    """The measured peaks of this GPU pool (HBM copy GB/s, bf16 TFLOP/s), if present."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# Kernel sources whose hash a recorded ncu traffic figure belongs to; the summary of
# kernel k on workload w is profiles/<k>_<short name of w>.md.
TRAFFIC_SOURCES = {
    "k_local_mixed": ["local_mixed.cu", "local_common.cuh", "mhm_internal.h"],
    "k_local_fp64": ["local_fp64.cu", "local_common.cuh", "mhm_internal.h"],
}
PROFILE_TAG = {"c2_hetero_fp64": "c2", "c3_grf_mixed": "c3", "c5_p2_large": "c5", "c4_channels": "c4"}


def sources_sha256(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1703_10435_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kernel` on
    `workload`, from its ncu summary under profiles/ ("traffic_bytes_per_launch", per launch
    of the bench's launch shape), or None when there is none or the kernel's sources changed
    since that capture (hash mismatch)."""
    if kernel not in TRAFFIC_SOURCES or workload not in PROFILE_TAG:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, PROFILE_TAG[workload]))).read()
        sha = sources_sha256(kernel)
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines() if line.startswith(("traffic_bytes", "sources_sha")))
    if fields.get("sources_sha256", "").strip() != sha or "traffic_bytes_per_launch" not in fields:
        return None
    return float(fields["traffic_bytes_per_launch"])


def level_counts(w):
    """{refinement level: number of K} of workload w."""
    rk = w.r_per_K
    if rk is None:
        return {w.r: w.n_K}
    return {int(r): int((rk == r).sum()) for r in np.unique(rk)}


def workload_config(w):
    """The workload's shape for the config object: uniform r, or the elements per level and
    the face degrees of a workload with a level per K."""
    cfg = {"workload": w.name, "n_K": w.n_K, "degree": w.degree, "m": w.m}
    if w.r_per_K is None:
        cfg.update({"r": w.r, "n_local": w.n_local})
    else:
        cfg["elements_per_level"] = {str(r): c for r, c in level_counts(w).items()}
    if w.face_degree is None:
        cfg["l"] = w.l
    else:
        cfg["l_per_face"] = "1 + [max adjacent r >= 5] + [max adjacent r >= 7] (1..%d)" % w.l
    cfg["rhs"] = w.n_I + 1
    return cfg


def mixed_level(w, r):
    """True where the mixed path runs level r by level-Schur refinement (P1 levels of at
    most 32 points, P2 levels of r <= 4).  Wider P1 levels run FP64 conjugate gradients
    preconditioned by the FP32 factor, P2 levels of r >= 5 the FP64 path."""
    return (1 << r) <= 32 if w.degree == 1 else r <= 4


def residual_fmas_per_pass(w, N=None):
    """FP64 multiply-adds of one refinement pass of the mixed path for one K of N
    segments per face (default: the workload's): the assembled 7-point (P1) rows of
    A_p applied to the R right-hand sides."""
    N = w.N if N is None else N
    if w.degree != 1:
        return None
    # On the right-isosceles coarse triangles of this mesh the lattice edge opposite
    # each fine triangle's right angle carries a zero weight: the lower triangles
    # couple E, W, SE, NW, the upper ones N, S, SE, NW (a 5-point row, the kernel
    # skips the zero weights).
    tot = 0
    for dirs in (((1, 0), (-1, 0), (1, -1), (-1, 1)), ((0, 1), (0, -1), (1, -1), (-1, 1))):
        nnz = 0
        for y in range(N + 1):
            for x in range(N + 1 - y):
                if x == 0 and y == 0:
                    continue
                cnt = 1
                for dx, dy in dirs:
                    X, Y = x + dx, y + dy
                    if X >= 0 and Y >= 0 and X + Y <= N and not (X == 0 and Y == 0):
                        cnt += 1
                nnz += cnt
        tot += nnz
    return tot / 2 * (w.n_I + 1)


def time_path(p, kap, src, gd, steps, warmup, flush, stream, barrier):
    """Times `steps` steps (local solves + skeleton), with the library's CUDA events
    around each of its local-solve kernel launches on the same stream; returns the
    step and local-solve times (ms) and {kernel: (launches, total ms)}."""
    import torch
    from paper_1703_10435_gb300 import mhm
    for _ in range(warmup):
        p.step(kap, src, gd)
    torch.cuda.synchronize()
    mhm.mhm_set_timing(p.mesh, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    torch.cuda.synchronize()
    for s in range(steps):
        flush.zero_()                                  # evict the inputs from L2 between steps
        ev[s][0].record(stream)
        p.local(kap, src)
        ev[s][1].record(stream)
        p.skeleton(gd)
        ev[s][2].record(stream)
    torch.cuda.synchronize()
    barrier()
    kern = mhm.mhm_kernel_times(p.mesh)
    mhm.mhm_set_timing(p.mesh, False)
    step_ms = np.array([a.elapsed_time(c) for a, b, c in ev])
    local_ms = np.array([a.elapsed_time(b) for a, b, c in ev])
    return step_ms, local_ms, kern


def oracle_locals(w, Ks, kaps):
    """The oracle's local contributions and local solutions of the coarse triangles Ks
    (a worker): per K (A_K, E_K, B_K, F_K, eta)."""
    from oracle.local import solve_local
    from oracle.mesh import build_mesh
    from oracle.run import source_fn
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    f = float(w.source_value) if w.source == "const" else source_fn("sinsin", w.source_value, w.source_freq)
    out = []
    for i, K in enumerate(Ks):
        o = solve_local(mesh, int(K), w.r, w.degree, kaps[i], f)
        out.append((o.AK, o.EK, o.BK, o.FK, o.eta))
    return out


def block_error(AK, EK, BK, FK, o):
    """Largest entry error of one K's blocks against the oracle's: A_K entries against
    sqrt(|A_ii| |A_jj|) (A_K is a Gram matrix), E_K and B_K against the block's largest
    entry (E_K against |A_K| |F_K| / |B_K| when it vanishes, as for a constant f), F_K
    relative."""
    oA, oE, oB, oF = o[0], o[1], o[2], o[3]
    d = np.sqrt(np.abs(np.diag(oA)))
    eA = float((np.abs(AK - oA) / np.maximum(np.outer(d, d), 1e-300)).max())
    bmax = max(float(np.abs(oB).max()), 1e-300)
    sE = max(float(np.abs(oE).max()), float(np.abs(oA).max()) * abs(oF) / bmax, 1e-300)
    return max(eA, float(np.abs(EK - oE).max()) / sE, float(np.abs(BK - oB).max()) / bmax,
               abs(FK - oF) / max(abs(oF), 1e-300))


def run_workload(args, w, rank, world, local_rank, dev, barrier, steps, warmup, flush, full):
    """Times both paths on workload w; with `full`, also the end-to-end run, the solution
    errors and the oracle sample.  Returns a dict of results (rank 0) or None."""
    import torch
    import torch.distributed as dist
    from paper_1703_10435_gb300 import mhm
    from paper_1703_10435_gb300 import workloads as W
    from paper_1703_10435_gb300.pipeline import Pipeline, dirichlet_of, source_of

    kap = W.kappa_for_torch(w, dev).reshape(-1).contiguous()
    src, gd = source_of(w), dirichlet_of(w)
    stream = torch.cuda.current_stream()
    p64 = Pipeline.for_workload(w, local_rank, mhm.MHM_FP64)
    pmx = Pipeline.for_workload(w, local_rank, mhm.MHM_MIXED)
    sampler = ClockSampler(local_rank, args.clocks_csv) if full else None
    if sampler:
        sampler.start()
    step64, local64, kern64 = time_path(p64, kap, src, gd, steps, warmup, flush, stream, barrier)
    stepmx, localmx, kernmx = time_path(pmx, kap, src, gd, steps, warmup, flush, stream, barrier)
    clocks = sampler.stop() if sampler else None
    for p in (p64, pmx):
        assert int(p.status.abs().sum()) == 0, "local solve status nonzero"
    t_mx, t_64 = float(stepmx.sum()), float(step64.sum())
    res = {"w": w, "p64": p64, "pmx": pmx, "kap": kap, "stepmx": stepmx, "localmx": localmx, "kern64": kern64,
           "kernmx": kernmx, "clocks": clocks, "t_mx": t_mx, "t_64": t_64}
    if full:
        # end to end through the C ABI with host buffers (mixed path): kappa H2D in,
        # skeleton system (A, E, B, F) D2H out
        kap_pin = kap.cpu().pin_memory()
        outs = [pmx.A_vals, pmx.E, pmx.BK, pmx.FK]
        outs_pin = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
        kap_dev2 = torch.empty_like(kap)
        res["h2d"] = kap_pin.numel() * 8
        res["d2h"] = sum(o.numel() * o.element_size() for o in outs)
        for _ in range(2):
            kap_dev2.copy_(kap_pin, non_blocking=True)
            pmx.step(kap_dev2, src, gd)
            for o, h in zip(outs, outs_pin):
                h.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(steps):
            kap_dev2.copy_(kap_pin, non_blocking=True)
            pmx.step(kap_dev2, src, gd)
            for o, h in zip(outs, outs_pin):
                h.copy_(o, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        res["t_e2e"] = e0.elapsed_time(e1)
        del kap_dev2
    if full and mhm.mhm_factor_store_size(pmx.mesh) > 0:
        # kept factors (Sec. 3: factored once while kappa is unchanged): one call fills the
        # store, then steps with a new source reuse it (no factor launches)
        store = torch.empty(mhm.mhm_factor_store_size(pmx.mesh), dtype=torch.uint8, device=dev)
        src2 = mhm.Source(mhm.MHM_SRC_CONST, 2.0, 1.0)   # a new source of the same kind (its quadrature cost alike)
        pmx.local(kap, src, mhm.solve_opts(factor_store=store, factor_reuse=0))
        o_re = mhm.solve_opts(factor_store=store, factor_reuse=1)
        for _ in range(warmup):
            pmx.local(kap, src2, o_re)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(steps):
            flush.zero_()
            pmx.local(kap, src2, o_re)
            pmx.skeleton(gd)
        ev1.record(stream)
        torch.cuda.synchronize()
        res["t_reuse"] = ev0.elapsed_time(ev1)
        res["store_bytes"] = store.numel()
        del store
        pmx.step(kap, src, gd)   # the timed path's outputs again (the solution check reads them)
        torch.cuda.synchronize()
    res["tuning"] = {str(r): mhm.mhm_get_tuning(pmx.mesh, r).as_dict() for r in level_counts(w)
                     if mixed_level(w, r) and w.degree == 1}
    if world > 1:
        tt = torch.tensor([res["t_mx"], res["t_64"], res.get("t_e2e", 0.0)], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        res["t_mx"], res["t_64"], res["t_e2e"] = [float(v) for v in tt]
    if full and not args.no_solution_check:
        res["error"] = solution_errors(args, w, p64, pmx, kap, src)
    return res if rank == 0 else None


class MemSampler:
    """Samples the device's used memory (cudaMemGetInfo) from a thread during a call."""

    def __init__(self, dev):
        import threading
        self.dev, self.peak, self.stop_ev = dev, 0, threading.Event()
        self.t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        import torch
        torch.cuda.set_device(self.dev)
        while not self.stop_ev.is_set():
            free, total = torch.cuda.mem_get_info(self.dev)
            self.peak = max(self.peak, total - free)
            time.sleep(0.005)

    def __enter__(self):
        import torch
        free, total = torch.cuda.mem_get_info(self.dev)
        self.base = total - free
        self.t.start()
        return self

    def __exit__(self, *exc):
        self.stop_ev.set()
        self.t.join()


def solution_errors(args, w, p64, pmx, kap, src):
    """Multipliers, u0 and reconstructed u of the mixed path against the FP64 path (whole
    batch), and a sample of coarse triangles against the FP64 oracle: the per-K blocks of
    both paths entry by entry, and u on those K from the oracle's local solutions combined
    with the path's own multipliers (Eq. "u_Hh")."""
    import torch
    from oracle.mesh import build_mesh
    from paper_1703_10435_gb300 import workloads as W
    dev = kap.device
    out = {}
    sols = {}
    from paper_1703_10435_gb300 import mhm
    for name, p in (("fp64", p64), ("mixed", pmx)):
        torch.cuda.synchronize()
        g0 = time.perf_counter()
        try:
            with MemSampler(dev) as ms:
                lam, u0 = p.solve_global()
                torch.cuda.synchronize()
        except mhm.MHMError as e:
            out["global_solve_error_" + name] = str(e)
            return out
        g1 = time.perf_counter()
        u, _ = p.reconstruct(kap, src)
        torch.cuda.synchronize()
        g2 = time.perf_counter()
        sols[name] = (lam.clone(), u0.clone(), u)
        out["global_solve_s_" + name] = g1 - g0
        out["reconstruct_s_" + name] = g2 - g1
        out["global_solve_device_bytes_above_base_" + name] = int(ms.peak - ms.base)
    (l64, z64, u64), (lmx, zmx, umx) = sols["fp64"], sols["mixed"]
    rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    out.update({"u_rel_l2_mixed_vs_fp64": rel(umx, u64), "lambda_rel_l2_mixed_vs_fp64": rel(lmx, l64),
                "u0_rel_l2_mixed_vs_fp64": rel(zmx, z64), "n_lambda": int(l64.numel()), "n_K": int(z64.numel())})
    if w.r_per_K is not None or args.oracle_sample <= 0:
        return out
    # the oracle on a sample of coarse triangles (first, last and seeded picks)
    rng = np.random.default_rng(7)
    Ks = sorted(set([0, w.n_K - 1] + [int(k) for k in rng.integers(0, w.n_K, args.oracle_sample - 2)]))
    kap_np = W.kappa_for(w, np.asarray(Ks))
    cores = min(os.cpu_count() or 1, len(Ks))
    pool = make_pool(cores)
    chunks = np.array_split(np.arange(len(Ks)), cores)
    futs = [pool.submit(oracle_locals, w, [Ks[i] for i in c], kap_np[c]) for c in chunks if len(c)]
    orc = [o for fu in futs for o in fu.result()]
    pool.shutdown()
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    nI = w.n_I
    samp = {"K": Ks, "kappa_max_abs_diff": float(np.abs(kap.view(w.n_K, -1)[Ks].cpu().numpy() - kap_np).max())}
    for name, p in (("fp64", p64), ("mixed", pmx)):
        AK, EK, BK, FK = p.blocks()
        lam, u0, u = sols[name]
        lam, u0 = lam.cpu().numpy(), u0.cpu().numpy()
        uK = u.view(w.n_K, -1)[Ks].cpu().numpy()
        be, ue = 0.0, []
        for i, (K, o) in enumerate(zip(Ks, orc)):
            be = max(be, block_error(AK[K], EK[K], BK[K], FK[K], o))
            eta = o[4]
            uo = u0[K] + eta[:, :nI] @ lam[mesh.local_lambda(K)] + eta[:, nI]
            ue.append((np.sum((uK[i] - uo) ** 2), np.sum(uo ** 2)))
        ue = np.asarray(ue)
        samp["blocks_max_entry_err_" + name] = be
        samp["u_rel_l2_vs_oracle_" + name] = float(math.sqrt(ue[:, 0].sum() / ue[:, 1].sum()))
    samp["what"] = ("per-K blocks A_K, E_K, B_K, F_K entry by entry against the oracle's (A_K per entry against "
                    "sqrt(|A_ii||A_jj|)); u on these K: the oracle's local solutions combined with the path's own "
                    "multipliers and u0, against the path's reconstructed u")
    out["oracle_sample"] = samp
    return out


THREE_D = [(8, 2, 2, 4), (4, 2, 2, 16)]   # (nc, r, k, m): 12288 and 1536 coarse tetrahedra


def local3d_flops(n, NI):
    """FP64 flops of one 3-D local solve: Cholesky of the pinned n - 1 unknowns
    ((n-1)^3 / 3), the forward substitution of N_I + 1 right-hand sides ((n-1)^2 (N_I + 1))
    and the Gram products of the face integrals (2 (n-1) (N_I (N_I + 1) / 2 + N_I))."""
    n1 = n - 1
    return n1 ** 3 / 3.0 + n1 * n1 * (NI + 1.0) + 2.0 * n1 * (NI * (NI + 1) / 2.0 + NI)


def local3d_mixed_fp64_flops(n, NI, n_sub, nb, passes):
    """FP64 flops of one mixed 3-D local solve: per refinement pass the matrix-free
    residual (n_sub nb^2 R multiply-adds), and the corrected face integrals (four dot
    products of length n - 1 per pair (j <= i) and per E_K entry)."""
    R = NI + 1
    return 2.0 * passes * n_sub * nb * nb * R + 8.0 * (n - 1) * (NI * (NI + 1) / 2.0 + NI)


def run_three_d(dev, flush, peak64, steps=5, warmup=3, n_check=2):
    """The paper's three-dimensional experiment (Sec. 5: kappa = 1, f = 12 pi^2 sin sin sin
    on the unit cube; 24 nc^3 coarse tetrahedra with 8^r sub-tetrahedra, k = 2, l = 0
    multipliers on m subfaces): local solves + skeleton gather per step in FP64 and (m <= 4)
    mixed precision, CUDA events on the launching stream, L2 flushed between steps, and a
    few elements of each path against the oracle."""
    import torch
    from paper_1703_10435_gb300 import mhm
    from oracle import tet3d as T
    stream = torch.cuda.current_stream()
    out = []
    for nc, r, P, m in THREE_D:
        M = mhm.Mesh3D(nc, r, P, m, device=dev.index)
        kap = torch.ones(M.n_K * M.n_sub, dtype=torch.float64, device=dev)
        src = mhm.Source3D(mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0)
        AK = torch.empty(M.n_K, M.n_I, M.n_I, dtype=torch.float64, device=dev)
        EK = torch.empty(M.n_K, M.n_I, dtype=torch.float64, device=dev)
        BK = torch.empty_like(EK)
        FK = torch.empty(M.n_K, dtype=torch.float64, device=dev)
        st = torch.empty(M.n_K, dtype=torch.int32, device=dev)
        it = torch.empty(M.n_K, dtype=torch.int32, device=dev)
        vals = torch.empty(M.nnz, dtype=torch.float64, device=dev)
        E = torch.empty(M.n_lambda, dtype=torch.float64, device=dev)
        o = T.build_mesh3d(nc, m)
        f = T.source3d_fn("sinsinsin", 1.0, 2.0)
        nb = 4 if P == 1 else 10

        def timed(precision):
            def local():
                mhm.mhm3d_local_solve_batch(M, kap, src, AK, EK, BK, FK, st, precision=precision, iters=it)
            for _ in range(warmup):
                local()
                mhm.mhm3d_assemble_skeleton(M, AK, EK, vals, E)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                   torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for s_ in range(steps):
                flush.zero_()
                ev[s_][0].record(stream)
                local()
                ev[s_][1].record(stream)
                mhm.mhm3d_assemble_skeleton(M, AK, EK, vals, E)
                ev[s_][2].record(stream)
            torch.cuda.synchronize()
            assert int(st.abs().sum()) == 0, "3-D local solve status nonzero"
            t_step = sum(a.elapsed_time(c) for a, b, c in ev) / steps
            t_local = sum(a.elapsed_time(b) for a, b, c in ev) / steps
            err = 0.0
            t0 = time.perf_counter()
            for K in (0, M.n_K - 1)[:n_check]:
                loc = T.solve_local3d(o, K, r, P, np.ones(M.n_sub), f)
                d = np.sqrt(np.abs(np.diag(loc.AK)))
                err = max(err, float((np.abs(AK[K].cpu().numpy() - loc.AK) / np.outer(d, d)).max()))
            t_or = (time.perf_counter() - t0) / n_check
            itv = it.cpu().numpy()
            return t_step, t_local, err, t_or, itv

        t64, l64, e64, t_or, _ = timed(mhm.MHM_FP64)
        fl64 = local3d_flops(M.n_local, M.n_I) * M.n_K
        entry = {"workload": "cube_%dx%dx%d_tets%d_sub%d_k%d_m%d" % (nc, nc, nc, M.n_K, M.n_sub, P, m),
                 "n_K": M.n_K, "local_dofs": M.n_local, "n_I": M.n_I, "lambda_unknowns": M.n_lambda,
                 "unit": "coarse elements/s",
                 "fp64": {"value": M.n_K / (t64 * 1e-3), "ms_per_step": t64, "local_ms": l64,
                          "skeleton_ms": t64 - l64,
                          "roofline": {"kernel": "k_local3d", "bound": "alu", "pipe": "fp64",
                                       "flops_per_step": fl64, "achieved": fl64 / (l64 * 1e-3) / 1e12,
                                       "peak": peak64, "unit": "TFLOP/s",
                                       "frac": fl64 / (l64 * 1e-3) / 1e12 / peak64},
                          "AK_gram_err_vs_oracle_%d_elements" % n_check: e64},
                 "cpu_oracle": {"value": 1.0 / t_or, "unit": "coarse elements/s", "cores": 1, "kind": "oracle",
                                "sample": "the %d checked elements, local solves" % n_check},
                 "inputs": "kappa = 1, f = 12 pi^2 sin(2 pi x) sin(2 pi y) sin(2 pi z) (the paper's model problem)"}
        entry["value"], entry["ms_per_step"], entry["dtype"] = entry["fp64"]["value"], t64, "f64"
        if M.n_I <= 16:
            tmx, lmx, emx, _, itv = timed(mhm.MHM_MIXED)
            passes = float(itv[itv > 0].mean()) if np.any(itv > 0) else 0.0
            flmx = local3d_mixed_fp64_flops(M.n_local, M.n_I, M.n_sub, nb, passes) * M.n_K
            entry["mixed"] = {"value": M.n_K / (tmx * 1e-3), "ms_per_step": tmx, "local_ms": lmx,
                              "skeleton_ms": tmx - lmx, "refinement_passes_mean": passes,
                              "fp64_resolved_elements": int(np.sum(itv < 0)),
                              "roofline": {"kernel": "k_local3d_mixed", "bound": "alu",
                                           "pipe": "fp64 (residuals and corrected face integrals)",
                                           "flops_per_step": flmx, "achieved": flmx / (lmx * 1e-3) / 1e12,
                                           "peak": peak64, "unit": "TFLOP/s",
                                           "frac": flmx / (lmx * 1e-3) / 1e12 / peak64},
                              "AK_gram_err_vs_oracle_%d_elements" % n_check: emx}
            entry["mixed_over_fp64"] = t64 / tmx
            entry["value"], entry["ms_per_step"], entry["dtype"] = entry["mixed"]["value"], tmx, "f32+f64"
        out.append(entry)
        del M
    return out


def run_ours(args, w, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1703_10435_gb300 import build, mhm
    from paper_1703_10435_gb300 import workloads as W

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2 (129 MB)

    def barrier():
        if world > 1:
            dist.barrier()

    r = run_workload(args, w, rank, world, local_rank, dev, barrier, args.steps, args.warmup, flush, True)
    sec = None
    if args.secondary and args.secondary != "none" and args.secondary != w.name:
        w2 = W.WORKLOADS[args.secondary]
        try:
            r2 = run_workload(args, w2, rank, world, local_rank, dev, barrier, args.steps, args.warmup, flush, False)
            if rank == 0:
                u2 = world * w2.n_K * args.steps
                sec = {"workload": w2.name, "config": workload_config(w2), "value": u2 / (r2["t_mx"] * 1e-3),
                       "fp64_value": u2 / (r2["t_64"] * 1e-3), "mixed_over_fp64": r2["t_64"] / r2["t_mx"],
                       "ms_per_step": r2["t_mx"] / args.steps, "unit": "coarse elements/s"}
            del r2
        except (AssertionError, RuntimeError, mhm.MHMError) as e:
            # a failure of a side workload is reported in the line, not fatal to the headline
            sec = {"workload": w2.name, "error": "%s: %s" % (type(e).__name__, e)}
    more = []
    for name in ([] if not args.more or args.more == "none" else args.more.split(",")):
        if name in (w.name, args.secondary):
            continue
        w3 = W.WORKLOADS[name]
        s3, ww3 = min(args.steps, 3), 3
        try:
            r3 = run_workload(args, w3, rank, world, local_rank, dev, barrier, s3, ww3, flush, False)
        except (AssertionError, RuntimeError, mhm.MHMError) as e:
            more.append({"workload": w3.name, "error": "%s: %s" % (type(e).__name__, e)})
            continue
        if rank == 0:
            u3 = world * w3.n_K * s3
            it3 = r3["pmx"].iters.cpu().numpy()
            a64, amx = r3["p64"].AK, r3["pmx"].AK
            more.append({"workload": w3.name, "config": workload_config(w3), "steps": s3, "warmup": ww3,
                         "value": u3 / (r3["t_mx"] * 1e-3), "fp64_value": u3 / (r3["t_64"] * 1e-3),
                         "mixed_over_fp64": r3["t_64"] / r3["t_mx"], "ms_per_step": r3["t_mx"] / s3,
                         "fp64_ms_per_step": r3["t_64"] / s3, "unit": "coarse elements/s",
                         "refinement_passes_mean": float(it3[it3 > 0].mean()) if np.any(it3 > 0) else 0.0,
                         "AK_rel_l2_mixed_vs_fp64": float(torch.linalg.norm(amx - a64) / torch.linalg.norm(a64))})
        del r3
    if rank != 0:
        return
    p64, pmx, kern64, kernmx = r["p64"], r["pmx"], r["kern64"], r["kernmx"]
    t_mx, t_64, t_e2e = r["t_mx"], r["t_64"], r["t_e2e"]
    clocks, localmx = r["clocks"], r["localmx"]
    itv = pmx.iters.cpu().numpy()
    passes = float(itv[itv > 0].mean()) if np.any(itv > 0) else 0.0   # elements refined in mixed precision

    units = world * w.n_K * args.steps
    value, v64, e2e = units / (t_mx * 1e-3), units / (t_64 * 1e-3), units / (t_e2e * 1e-3)
    pipes = mhm.mhm_measure_pipes(local_rank)
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    clk = clocks["sm_max_mhz"] if clocks else 2070.0
    # GB300: 2 FP64 FMA per clock per SM (1.25 TFLOP/s nominal over 152 SMs at 2.07 GHz)
    peak64 = 2 * 2 * sms * clk * 1e6 / 1e12
    # Kernel durations over the timed region: the library's CUDA events around each
    # local-solve launch, on the launching stream.
    # Algorithmic work per step, summed over the refinement levels; achieved = work per
    # step / kernel time per step.
    lv = level_counts(w)
    R = w.n_I + 1
    rk = w.r_per_K if w.r_per_K is not None else np.full(w.n_K, w.r)
    fl64 = 2.0 * sum(c * algorithmic_fmas(w.degree, 1 << rr, R) for rr, c in lv.items())
    t_k64 = kern64["k_local_fp64"][1] * 1e-3 / args.steps if "k_local_fp64" in kern64 else None
    t_kmx = kernmx["k_local_mixed"][1] * 1e-3 / args.steps if "k_local_mixed" in kernmx else None
    t_kfac = kernmx["k_schur_factor"][1] * 1e-3 / args.steps if "k_schur_factor" in kernmx else None
    n64, nmx, nfac = [kern.get(k, (0, 0.0))[0] for kern, k in ((kern64, "k_local_fp64"), (kernmx, "k_local_mixed"),
                                                                (kernmx, "k_schur_factor"))]
    fl_res, fl_tc = 0.0, 0.0
    for rr, c in lv.items():
        if not mixed_level(w, rr):
            continue
        it = itv[rk == rr]
        p_r = float(it[it > 0].mean()) if np.any(it > 0) else 0.0
        res = residual_fmas_per_pass(w, 1 << rr)
        if res is not None:
            fl_res += 2.0 * res * p_r * c
        if w.degree == 1:
            N = 1 << rr
            sizes = [N + 1 - l_ - (l_ == 0) for l_ in range(N + 1)]
            fl_tc += 2.0 * R * (2 * sum(b * b for b in sizes) - sizes[-1] ** 2) * p_r * c
    fl_res = fl_res or None
    tc = None
    if fl_tc and t_kmx:
        # dense TF32 tensor peak: the measured bf16 burst figure times the nominal tf32/bf16 ratio
        peak_bf16 = measured_peaks().get("bf16_tflops")
        peak_tf32 = peak_bf16 * (1.1 / 2.25) if peak_bf16 else None
        tc = {"pipe": "tensor (TF32, three-term split: 3 MMA per product)", "algorithmic_flops_per_step": fl_tc,
              "achieved": fl_tc / t_kmx / 1e12, "peak": peak_tf32, "unit": "TFLOP/s",
              "frac": (fl_tc / t_kmx / 1e12 / peak_tf32) if peak_tf32 else None,
              "peak_source": "MEASURED_PEAKS.json bf16 burst x 1.1/2.25 (nominal tf32/bf16)"}
    launch_kmx = t_kmx * args.steps / nmx if (t_kmx and nmx) else None
    roof_mx = {"kernel": "k_local_mixed", "bound": "alu", "pipe": "fp64 (refinement residuals)",
               "achieved": (fl_res / t_kmx / 1e12) if (fl_res and t_kmx) else None, "peak": peak64, "unit": "TFLOP/s",
               "frac": (fl_res / t_kmx / 1e12 / peak64) if (fl_res and t_kmx) else None,
               "traffic": recorded_traffic("k_local_mixed", w.name),
               "traffic_unit": "bytes per launch (%d K per launch)" % (w.n_K * args.steps // max(nmx, 1)),
               "flops_per_step": fl_res, "kernel_ms_per_step": t_kmx * 1e3 if t_kmx else None, "launches": nmx,
               "kernel_ms_per_launch": launch_kmx * 1e3 if launch_kmx else None,
               "refinement_passes_mean": passes,
               "peak_source": "2 FP64 FMA/clk/SM x SMs x max SM clock", "peak_measured_microbench": pipes["fp64_gflops"] / 1e3,
               "tensor": tc,
               "factor_kernel": {"kernel": "k_schur_factor", "kernel_ms_per_step": t_kfac * 1e3 if t_kfac else None,
                                 "launches": nfac},
               "levels": {str(k): c for k, c in lv.items()},
               "fp64_equivalent_local_solve_tflops": fl64 / (float(localmx.mean()) * 1e-3) / 1e12}
    roof_64 = {"kernel": "k_local_fp64", "bound": "alu", "pipe": "fp64",
               "achieved": fl64 / t_k64 / 1e12 if t_k64 else None, "peak": peak64, "unit": "TFLOP/s",
               "frac": fl64 / t_k64 / 1e12 / peak64 if t_k64 else None,
               "traffic": recorded_traffic("k_local_fp64", w.name),
               "flops_per_step": fl64, "kernel_ms_per_step": t_k64 * 1e3 if t_k64 else None, "launches": n64,
               "peak_measured_microbench": pipes["fp64_gflops"] / 1e3}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        pool = make_pool(cores)
        time_oracle(w, cores, cores, pool)
        n_sample = max(cores, args.ref_sample)
        t_cpu = min(time_oracle(w, n_sample, cores, pool) for _ in range(3))
        pool.shutdown()
        cpu = {"value": n_sample / t_cpu, "unit": "coarse elements/s", "cores": cores, "kind": "oracle",
               "sample": "%d coarse triangles of the workload (K = 0..%d), local solves, best of 3 runs"
                         % (n_sample, n_sample - 1)}

    three_d = None
    if world == 1 and not args.no_three_d:
        try:
            three_d = run_three_d(dev, flush, peak64)
        except (AssertionError, RuntimeError, ValueError, mhm.MHMError) as e:
            three_d = {"error": "%s: %s" % (type(e).__name__, e)}

    line = {
        "metric": "coarse elements/s (local solves + skeleton assembly)",
        "value": value, "unit": "coarse elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mx / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(workload_config(w), **{
                   "field": w.field, "seed": w.seed,
                   "precision": "mixed (FP32 factor and solves, FP64 residuals)",
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "K-range shard per GPU" if world > 1 else "single GPU"}),
        "fp64_path": {"value": v64, "ms_per_step": t_64 / args.steps, "dtype": "f64", "roofline": roof_64},
        "mixed_over_fp64": value / v64,
        "error": r.get("error"),
        "local_solve_ms": float(localmx.mean()),
        "skeleton_ms": float((r["stepmx"] - localmx).mean()),
        "roofline": roof_mx,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "coarse elements/s", "h2d_bytes_per_step": r["h2d"],
                "d2h_bytes_per_step": r["d2h"]},
        # our kernels in the timed region of the headline (mixed) path: the local-solve
        # launches recorded by the library plus the two skeleton kernels per step
        "gpu_launches": sum(n for n, _ in kernmx.values()) + 2 * args.steps,
        "clocks": clocks,
        "pipes_gflops": pipes,
        "secondary": sec,
        "more_configs": more,
        "factor_reuse": None if "t_reuse" not in r else {
            "value": units / (r["t_reuse"] * 1e-3), "unit": "coarse elements/s",
            "ms_per_step": r["t_reuse"] / args.steps, "store_bytes": r["store_bytes"],
            "what": "mixed local solves + skeleton with the level-Schur factors kept from an earlier call "
                    "(mhm_solve_opts.factor_store, factor_reuse = 1) and a new source f; L2 flushed between steps"},
        "tuning": r.get("tuning"),
        "three_d": three_d,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--ref-sample", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-csv", default=None, help="file for the raw nvidia-smi samples (default: temp dir)")
    ap.add_argument("--no-solution-check", action="store_true")
    ap.add_argument("--secondary", default=SECONDARY, help="second workload timed beside the headline ('none': no second line)")
    ap.add_argument("--more", default=MORE, help="further workloads timed briefly beside it, comma-separated ('none': none)")
    ap.add_argument("--oracle-sample", type=int, default=12, help="coarse triangles checked against the oracle")
    ap.add_argument("--no-three-d", action="store_true", help="skip the three-dimensional workloads")
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
