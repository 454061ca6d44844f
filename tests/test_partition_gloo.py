"""Multi-rank path on the CPU: two gloo ranks each solve the local problems of
their contiguous K range (the static partition of the MPI version), gather the
per-element blocks, and the assembled skeleton equals the one-shot result."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1703_10435_gb300.partition import k_range


def test_k_range_covers_disjointly():
    for n in (1, 7, 32, 2048):
        for world in (1, 2, 3, 8):
            ranges = [k_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import globalsys
    from oracle.local import solve_local
    from oracle.mesh import build_mesh
    from paper_1703_10435_gb300 import workloads as W
    from paper_1703_10435_gb300.partition import gather_blocks
    w = W.Workload("t", 2, 2, 2, 1, 2, 1, "log_uniform", "const", 1.0, seed=9)
    kap = W.kappa_for(w)
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    K0, K1 = k_range(w.n_K, rank, world)
    locs = [solve_local(mesh, K, w.r, w.degree, kap[K], 1.0) for K in range(K0, K1)]
    blocks = {"AK": torch.tensor(np.stack([l.AK for l in locs])), "EK": torch.tensor(np.stack([l.EK for l in locs])),
              "BK": torch.tensor(np.stack([l.BK for l in locs])), "FK": torch.tensor([l.FK for l in locs])}
    full = gather_blocks(blocks, K0, K1, w.n_K)
    if rank == 0:
        class L:  # per-K view with the fields the oracle's assembly reads
            pass
        views = []
        for K in range(w.n_K):
            v = L()
            v.AK, v.EK, v.BK, v.FK = (full["AK"][K].numpy(), full["EK"][K].numpy(), full["BK"][K].numpy(),
                                      float(full["FK"][K]))
            views.append(v)
        A, B, E, F = globalsys.assemble(mesh, views)
        one = [solve_local(mesh, K, w.r, w.degree, kap[K], 1.0) for K in range(w.n_K)]
        A1, B1, E1, F1 = globalsys.assemble(mesh, one)
        np.savez(out_path, dA=abs(A - A1).max(), dB=abs(B - B1).max(), dE=np.abs(E - E1).max(),
                 dF=np.abs(F - F1).max())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_partition_equals_one_shot(tmp_path):
    out = str(tmp_path / "res.npz")
    port = 29500 + (os.getpid() % 2000)
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    r = np.load(out)
    assert float(r["dA"]) == 0.0 and float(r["dB"]) == 0.0 and float(r["dE"]) == 0.0 and float(r["dF"]) == 0.0
