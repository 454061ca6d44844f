"""Small local-solve case for profiler captures.

Runs the local solves of the first `n_K` coarse triangles of a named workload
twice (the second launch is the one to capture, the first warms caches and
code), on cuda:0, and checks the status words.  Example:

    python -m paper_1703_10435_gb300.profile_case --precision mixed --n-k 152

The first 8192 coarse triangles of the 32768-element random-field workload are one
factor + solve launch pair of the bench's mixed path:

    python -m paper_1703_10435_gb300.profile_case --workload c3_grf_mixed --n-k 8192

--level r puts every coarse triangle of the workload at refinement level r (its
kappa field sampled at that level), e.g. the 256-row level windows of r = 7:

    python -m paper_1703_10435_gb300.profile_case --workload c4_channels --level 7 \
        --precision fp64 --n-k 152
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c2_hetero_fp64")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--n-k", type=int, default=152, help="coarse triangles K = 0 .. n_k - 1")
    ap.add_argument("--level", type=int, default=None, help="uniform refinement level r for every K")
    args = ap.parse_args(argv)

    import torch
    from . import build, mhm
    from . import workloads as W
    from .pipeline import Pipeline, source_of

    build.build()
    w = W.WORKLOADS[args.workload]
    if args.level is not None:
        import dataclasses
        w = dataclasses.replace(w, r=args.level, levels=None)
    n = min(args.n_k, w.n_K)
    import numpy as np
    if w.field in ("grf4", "grf6") and w.r_per_K is None:
        # random Fourier field: evaluated on the device (the blocks of K >= n are not read)
        kap = W.kappa_for_torch(w, torch.device("cuda")).reshape(-1)
    else:
        # kappa of K = 0 .. n - 1 only (the blocks sit at the same offsets as in the full field)
        kap = torch.as_tensor(W.kappa_for(w, np.arange(n)), device="cuda").reshape(-1)
    prec = mhm.MHM_MIXED if args.precision == "mixed" else mhm.MHM_FP64
    p = Pipeline.for_workload(w, 0, prec)
    opts = mhm.SolveOpts(8, 1e-12, 0, n)
    for _ in range(2):
        p.local(kap, source_of(w), opts)
    torch.cuda.synchronize()
    bad = int(p.status[:n].abs().sum())
    print("profile case: %s %s, %d coarse triangles, status sum %d" % (w.name, args.precision, n, bad))
    if bad:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
