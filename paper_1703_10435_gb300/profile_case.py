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

--cube nc runs the three-dimensional local solves instead (the unit cube of the paper's
experiment, Sec. 5: 24 nc^3 tetrahedra, P2 on 64 sub-tetrahedra, m subfaces per face,
kappa = 1, f = 12 pi^2 sin sin sin), e.g. the 1536 elements of nc = 4 in mixed precision:

    python -m paper_1703_10435_gb300.profile_case --cube 4 --m 4 --precision mixed
"""
from __future__ import annotations

import argparse


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="c2_hetero_fp64")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--n-k", type=int, default=152, help="coarse triangles K = 0 .. n_k - 1")
    ap.add_argument("--level", type=int, default=None, help="uniform refinement level r for every K")
    ap.add_argument("--cube", type=int, default=None, help="3-D: cubes per side of the unit cube")
    ap.add_argument("--m", type=int, default=4, help="3-D: subfaces per face (4 or 16)")
    args = ap.parse_args(argv)

    import torch
    from . import build, mhm
    from . import workloads as W
    from .pipeline import Pipeline, source_of

    build.build()
    if args.cube is not None:
        M = mhm.Mesh3D(args.cube, 2, 2, args.m, device=0)
        dev = torch.device("cuda", 0)
        kap = torch.ones(M.n_K * M.n_sub, dtype=torch.float64, device=dev)
        AK = torch.empty(M.n_K, M.n_I, M.n_I, dtype=torch.float64, device=dev)
        EK = torch.empty(M.n_K, M.n_I, dtype=torch.float64, device=dev)
        BK, FK = torch.empty_like(EK), torch.empty(M.n_K, dtype=torch.float64, device=dev)
        st = torch.empty(M.n_K, dtype=torch.int32, device=dev)
        prec = mhm.MHM_MIXED if args.precision == "mixed" else mhm.MHM_FP64
        src = mhm.Source3D(mhm.MHM3D_SRC_SINSINSIN, 1.0, 2.0)
        for _ in range(2):
            mhm.mhm3d_local_solve_batch(M, kap, src, AK, EK, BK, FK, st, precision=prec)
        torch.cuda.synchronize()
        bad = int(st.abs().sum())
        print("profile case: cube %d, m %d, %s, %d tetrahedra, status sum %d"
              % (args.cube, args.m, args.precision, M.n_K, bad))
        if bad:
            raise SystemExit(1)
        return
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
