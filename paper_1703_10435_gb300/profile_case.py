"""Small local-solve case for profiler captures.

Runs the local solves of the first `n_K` coarse triangles of a named workload
twice (the second launch is the one to capture, the first warms caches and
code), on cuda:0, and checks the status words.  Example:

    python -m paper_1703_10435_gb300.profile_case --precision mixed --n-k 152
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c2_hetero_fp64")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--n-k", type=int, default=152, help="coarse triangles K = 0 .. n_k - 1")
    args = ap.parse_args(argv)

    import torch
    from . import build, mhm
    from . import workloads as W
    from .pipeline import Pipeline, source_of

    build.build()
    w = W.WORKLOADS[args.workload]
    n = min(args.n_k, w.n_K)
    kap = torch.as_tensor(W.kappa_for(w), device="cuda")
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
