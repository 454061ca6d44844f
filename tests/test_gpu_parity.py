"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  FP64 path: per-K blocks A_K, E_K, B_K, F_K within 1e-10
relative (Frobenius norm per K), skeleton matrix and right-hand side within
1e-10 relative."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import globalsys
from oracle.local import solve_local
from oracle.mesh import build_mesh
from oracle.run import run, source_fn
from paper_1703_10435_gb300 import mhm, workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


def _pipeline(w, precision=mhm.MHM_FP64):
    from paper_1703_10435_gb300.pipeline import Pipeline
    return Pipeline.for_workload(w, 0, precision)


def _oracle_f(w):
    return float(w.source_value) if w.source == "const" else source_fn("sinsin", w.source_value, w.source_freq)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _compare_blocks(p, w, kap, Ks, tol=TOL64):
    AK, EK, BK, FK = p.blocks()
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    f = _oracle_f(w)
    worst = 0.0
    for K in Ks:
        o = solve_local(mesh, int(K), w.r, w.degree, kap[K], f)
        eA = _rel(AK[K], o.AK)
        # E_K vanishes exactly for constant f (its compatible part f~ is zero); then
        # both sides hold rounding noise, measured against the size E_K has for a
        # source of the same magnitude: |A_K| |F_K| / |B_K|
        scale_E = max(np.linalg.norm(o.EK), np.linalg.norm(o.AK) * abs(o.FK) / np.linalg.norm(o.BK), 1e-300)
        eE = np.linalg.norm(EK[K] - o.EK) / scale_E
        eB = _rel(BK[K], o.BK)
        eF = abs(FK[K] - o.FK) / max(abs(o.FK), 1e-300) if o.FK != 0 else abs(FK[K])
        worst = max(worst, eA, eE, eB, eF)
        assert eA < tol and eE < tol and eB < tol and eF < tol, (K, eA, eE, eB, eF)
    return worst


def _run(w, precision=mhm.MHM_FP64, opts=None):
    p = _pipeline(w, precision)
    kap = W.kappa_for(w)
    kd = torch.as_tensor(kap, device="cuda").contiguous()
    from paper_1703_10435_gb300.pipeline import dirichlet_of, source_of
    p.step(kd, source_of(w), dirichlet_of(w), opts)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    return p, kap


@pytest.mark.parametrize("name", ["c1_sin", "c1_linear"])
def test_config1_blocks_and_skeleton(name):
    w = W.WORKLOADS[name]
    p, kap = _run(w)
    _compare_blocks(p, w, kap, range(w.n_K))
    g = None if w.dirichlet is None else (lambda x, y, c=w.dirichlet: c[0] + c[1] * x + c[2] * y)
    o = run(w.nx, w.ny, w.r, w.degree, w.m, w.l, kap, _oracle_f(w), g=g)
    A = p.skeleton_scipy().toarray()
    Ao = o.A.toarray()
    assert _rel(A, Ao) < TOL64
    assert _rel(p.E.cpu().numpy(), o.E + o.G) < TOL64


@pytest.mark.parametrize("P,r,m,l,nx", [(1, 0, 1, 0, 1), (1, 1, 1, 1, 2), (1, 2, 2, 1, 2), (1, 4, 2, 2, 2),
                                        (1, 5, 2, 2, 1), (2, 0, 1, 0, 1), (2, 1, 1, 1, 2), (2, 2, 3, 1, 2),
                                        (2, 4, 3, 1, 1)])
def test_blocks_heterogeneous(P, r, m, l, nx):
    w = W.Workload("t", nx, nx, r, P, m, l, "log_uniform", "sinsin", 1.0, 1.0, seed=11)
    p, kap = _run(w)
    _compare_blocks(p, w, kap, range(w.n_K))


def test_layered_exact_recovery_through_gpu_blocks():
    """Strip-layered kappa (contrast 1e4), f = 0, g = 0 -> the oracle's global
    solve on the GPU's skeleton reproduces the oracle's multipliers."""
    w = W.Workload("t", 2, 2, 3, 1, 1, 1, "log_uniform", "const", 0.0, seed=3)
    N = w.N
    cen = W.fine_centroids(W.coarse_vertices(w.nx, w.ny), N)
    hs = 1.0 / (w.ny * N)
    ks = 10.0 ** (-2 + 4 * W.uniform01(5, np.arange(w.ny * N, dtype=np.uint64), 0, 0))
    kap = ks[np.floor(cen[..., 1] / hs).astype(int)]
    p = _pipeline(w)
    from paper_1703_10435_gb300.pipeline import source_of
    p.step(torch.as_tensor(kap, device="cuda"), source_of(w), mhm.Dirichlet((mhm.ctypes.c_double * 6)(0, 0, 1, 0, 0, 0)))
    torch.cuda.synchronize()
    o = run(w.nx, w.ny, w.r, 1, 1, 1, kap, 0.0, g=lambda x, y: y)
    assert _rel(p.skeleton_scipy().toarray(), o.A.toarray()) < TOL64
    assert _rel(p.E.cpu().numpy(), o.E + o.G) < TOL64


def test_k_range_partition_equals_one_shot():
    """Two disjoint K ranges (the multi-rank partition) write the same blocks as one call."""
    w = W.Workload("t", 4, 3, 3, 1, 2, 1, "log_uniform", "const", 1.0, seed=2)
    p1, kap = _run(w)
    A1, E1, B1, F1 = p1.blocks()
    p2 = _pipeline(w)
    kd = torch.as_tensor(kap, device="cuda")
    from paper_1703_10435_gb300.pipeline import source_of
    half = w.n_K // 2 + 1
    p2.local(kd, source_of(w), mhm.SolveOpts(8, 1e-14, 0, half))
    p2.local(kd, source_of(w), mhm.SolveOpts(8, 1e-14, half, w.n_K))
    torch.cuda.synchronize()
    A2, E2, B2, F2 = p2.blocks()
    assert np.array_equal(A1, A2) and np.array_equal(E1, E2) and np.array_equal(F1, F2)


def test_config2_full_size_sampled():
    """The bench workload (2048 K, P1 r5, m=2 l=2, log-uniform kappa) in the bench's
    launch configuration; a sample of K checked one by one against the oracle."""
    w = W.WORKLOADS["c2_hetero_fp64"]
    p, kap = _run(w)
    rng = np.random.default_rng(0)
    Ks = sorted(set([0, 1, w.n_K - 1] + list(rng.integers(0, w.n_K, 5))))
    _compare_blocks(p, w, kap, Ks)
    # skeleton properties at full size: symmetric, negative definite diagonal
    A = p.skeleton_scipy()
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    assert float(A.diagonal().max()) < 0.0


def test_repeat_calls_identical():
    w = W.WORKLOADS["c1_sin"]
    p, kap = _run(w)
    a = p.A_vals.clone()
    p.step(torch.as_tensor(kap, device="cuda"), mhm.Source(1, 1.0, 1.0))
    torch.cuda.synchronize()
    assert torch.equal(a, p.A_vals)


# ------------------------------------------------------------------ mixed precision
TOL_MIXED = 1e-9   # per-K blocks after FP64 refinement of the FP32 solves


@pytest.mark.parametrize("P,r,m,l,nx,field", [(1, 3, 1, 1, 2, "one"), (1, 0, 1, 0, 1, "log_uniform"),
                                              (1, 2, 2, 1, 2, "log_uniform"), (1, 5, 2, 2, 1, "log_uniform"),
                                              (1, 5, 2, 2, 1, "grf4"), (2, 2, 3, 1, 2, "log_uniform"),
                                              (2, 4, 3, 1, 1, "grf6")])
def test_mixed_blocks(P, r, m, l, nx, field):
    w = W.Workload("t", nx, nx, r, P, m, l, field, "sinsin", 1.0, 1.0, seed=5)
    p, kap = _run(w, mhm.MHM_MIXED, mhm.SolveOpts(10, 1e-13, 0, 0))
    assert int(p.iters.max()) <= 10
    _compare_blocks(p, w, kap, range(w.n_K), tol=TOL_MIXED)


def test_mixed_config2_full_size_and_vs_fp64():
    w = W.WORKLOADS["c2_hetero_fp64"]
    p, kap = _run(w, mhm.MHM_MIXED, mhm.SolveOpts(10, 1e-13, 0, 0))
    rng = np.random.default_rng(1)
    Ks = sorted(set([0, w.n_K - 1] + list(rng.integers(0, w.n_K, 4))))
    _compare_blocks(p, w, kap, Ks, tol=TOL_MIXED)
    A_mixed = p.skeleton_scipy()
    p64, _ = _run(w)
    A64 = p64.skeleton_scipy()
    assert abs(A_mixed - A64).max() <= TOL_MIXED * abs(A64).max()


def test_mixed_reports_nonconvergence_with_one_pass():
    """One refinement pass cannot reach 1e-13 on heterogeneous kappa: the per-K
    status says so instead of returning silently inaccurate blocks."""
    w = W.Workload("t", 1, 1, 4, 1, 1, 1, "log_uniform", "const", 1.0, seed=1)
    p = _pipeline(w, mhm.MHM_MIXED)
    from paper_1703_10435_gb300.pipeline import source_of
    p.local(torch.as_tensor(W.kappa_for(w), device="cuda"), source_of(w), mhm.SolveOpts(1, 1e-13, 0, 0, 1))
    torch.cuda.synchronize()
    assert set(p.status.cpu().tolist()) == {mhm.MHM_ERR_NOT_CONVERGED}


def test_mixed_failures_fall_back_to_fp64():
    """By default the elements whose refinement fails are solved again in FP64: status
    OK, iters -1, and blocks identical to the FP64 path's."""
    w = W.Workload("t", 2, 2, 4, 1, 1, 1, "log_uniform", "const", 1.0, seed=1)
    from paper_1703_10435_gb300.pipeline import source_of
    kap = torch.as_tensor(W.kappa_for(w), device="cuda")
    p = _pipeline(w, mhm.MHM_MIXED)
    p.local(kap, source_of(w), mhm.SolveOpts(1, 1e-13, 0, 0))
    p64 = _pipeline(w, mhm.MHM_FP64)
    p64.local(kap, source_of(w))
    torch.cuda.synchronize()
    assert set(p.status.cpu().tolist()) == {0} and set(p.iters.cpu().tolist()) == {-1}
    assert torch.equal(p.AK, p64.AK) and torch.equal(p.EK, p64.EK)
