"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  FP64 path: every entry of the per-K blocks A_K, E_K, B_K, F_K
within 1e-10 of its scale (tests/_blocks.py), skeleton matrix and right-hand
side within 1e-10 relative; mixed path: the same at 1e-9."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import globalsys
from oracle.local import solve_local
from oracle.mesh import build_mesh
from oracle.run import run, source_fn
from paper_1703_10435_gb300 import mhm, workloads as W
from _blocks import assert_blocks, gram_entry_error

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
    """Every entry of A_K, E_K, B_K, F_K of the K in Ks against the oracle (tests/_blocks.py)."""
    AK, EK, BK, FK = p.blocks()
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    f = _oracle_f(w)
    worst = 0.0
    for K in Ks:
        o = solve_local(mesh, int(K), w.r, w.degree, kap[K], f)
        worst = max(worst, assert_blocks(AK[K], EK[K], BK[K], FK[K], o, tol, K))
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
    assert _rel(A, Ao) < TOL64 and gram_entry_error(A, Ao) < TOL64
    Eo = o.E + o.G
    assert np.abs(p.E.cpu().numpy() - Eo).max() < TOL64 * np.abs(Eo).max()


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
    assert gram_entry_error(p.skeleton_scipy().toarray(), o.A.toarray()) < TOL64
    Eo = o.E + o.G
    assert np.abs(p.E.cpu().numpy() - Eo).max() < TOL64 * np.abs(Eo).max()


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


# (P1 with 25 right-hand sides runs the level-Schur solve with all column tiles in step, up
# to 24 in decoupled column groups; P1 with 37 and P2 with 49, the most a face's 16
# multipliers give, run the generic level-Schur path)
@pytest.mark.parametrize("P,r,m,l,nx,field", [(1, 3, 1, 1, 2, "one"), (1, 0, 1, 0, 1, "log_uniform"),
                                              (1, 2, 2, 1, 2, "log_uniform"), (1, 5, 2, 2, 1, "log_uniform"),
                                              (1, 5, 2, 2, 1, "grf4"), (2, 2, 3, 1, 2, "log_uniform"),
                                              (2, 4, 3, 1, 1, "grf6"), (1, 4, 2, 3, 1, "grf4"),
                                              (1, 4, 3, 3, 1, "grf4"), (2, 3, 4, 3, 1, "log_uniform")])
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


def test_status_word_reports_outcomes():
    """The mesh's outcome word (mhm_sync_status): a forced one-pass non-convergence without
    the FP64 re-solve surfaces as MHM_ERR_NOT_CONVERGED, the read clears it, the default
    re-solve reports OK with the re-solve bit, and a converged run leaves the word at 0;
    the allocation-free entry reports its failures too."""
    w = W.Workload("t", 1, 1, 4, 1, 1, 1, "log_uniform", "const", 1.0, seed=1)
    p = _pipeline(w, mhm.MHM_MIXED)
    from paper_1703_10435_gb300.pipeline import source_of
    kap = torch.as_tensor(W.kappa_for(w), device="cuda")
    assert mhm.mhm_sync_status(p.mesh) == (mhm.MHM_OK, 0)
    p.local(kap, source_of(w), mhm.SolveOpts(1, 1e-13, 0, 0, 1))
    assert mhm.mhm_sync_status(p.mesh) == (mhm.MHM_ERR_NOT_CONVERGED, 1 << mhm.MHM_ERR_NOT_CONVERGED)
    assert mhm.mhm_sync_status(p.mesh) == (mhm.MHM_OK, 0)
    p.local(kap, source_of(w), mhm.SolveOpts(1, 1e-13, 0, 0))
    assert mhm.mhm_sync_status(p.mesh) == (mhm.MHM_OK, mhm.MHM_STATUS_REFINED_IN_FP64)
    p.local(kap, source_of(w), mhm.SolveOpts(10, 1e-13, 0, 0))
    assert mhm.mhm_sync_status(p.mesh) == (mhm.MHM_OK, 0)
    mhm.mhm_local_solve_batch_noalloc(p.mesh, kap, source_of(w), mhm.SolveOpts(1, 1e-13, 0, 0), p.AK, p.EK, p.BK,
                                      p.FK, p.status, p.iters)
    assert mhm.mhm_sync_status(p.mesh)[0] == mhm.MHM_ERR_NOT_CONVERGED


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


@pytest.mark.parametrize("m,l", [(1, 0), (2, 2), (3, 3)])
def test_library_multiplier_basis_by_face_moments(m, l):
    """The library's basis of Lambda_H^{m,l} (Sec. 2, definition (i)) against closed forms:
    with zero local blocks the skeleton right-hand side is the boundary term (g, psi_j)_F,
    which for g = x^2 + y^2 is a sum of Legendre moments (tests/golden/legendre.txt); it
    pins the normalisation of P_0..P_2 (P_3 has zero moments against a quadratic), the
    direction of xi and the subface coordinates, independently of the oracle."""
    from _golden import dirichlet_moment, legendre_golden
    gold = legendre_golden()
    nx, ny = 2, 3
    mesh = build_mesh(nx, ny, m, l)
    M = mhm.Mesh(nx, ny, 2, 1, m, l, 0)
    assert np.array_equal(M.query(mhm.Q_LAMBDA_OFFSET, np.int64, M.n_faces + 1), mesh.lam_offset)
    AK = torch.zeros(M.n_K * M.n_I * M.n_I, dtype=torch.float64, device="cuda")
    EK = torch.zeros(M.n_K * M.n_I, dtype=torch.float64, device="cuda")
    A = torch.empty(M.nnz, dtype=torch.float64, device="cuda")
    E = torch.empty(M.n_lambda, dtype=torch.float64, device="cuda")
    g = mhm.Dirichlet((mhm.ctypes.c_double * 6)(0, 0, 0, 1, 0, 1))
    mhm.mhm_assemble_skeleton(M, AK, EK, g, A, E)
    torch.cuda.synchronize()
    E = E.cpu().numpy()
    assert float(A.abs().max()) == 0.0
    for e in range(mesh.n_e):
        for q in range(m):
            for p in range(l + 1):
                j = mesh.lam_offset[e] + q * (l + 1) + p
                want = dirichlet_moment(mesh, e, q, p, m, gold) if mesh.boundary[e] else 0.0
                assert E[j] == pytest.approx(want, abs=1e-14), (e, q, p)


def _f_nonpoly(x, y):
    return np.exp(x) * np.cos(3.0 * y) + 1.0 / (1.0 + x + y)


@pytest.mark.parametrize("P,r,precision", [(1, 3, mhm.MHM_FP64), (1, 4, mhm.MHM_MIXED), (2, 2, mhm.MHM_FP64),
                                           (2, 3, mhm.MHM_MIXED)])
def test_quad_source_blocks_vs_oracle(P, r, precision):
    """A non-polynomial f given by its values at the 16 collapsed-Gauss points of every fine
    triangle (MHM_SRC_QUAD, Eq. "etaf" with a general f): every block against the oracle
    evaluating the same f at its own quadrature points."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    w = W.Workload("t", 2, 2, r, P, 2, 1, "log_uniform", "const", 1.0, seed=9)
    kap = W.kappa_for(w)
    pts = W.source_points(W.coarse_vertices(w.nx, w.ny), w.N)
    vals = torch.as_tensor(_f_nonpoly(pts[..., 0], pts[..., 1]).reshape(-1), device="cuda").contiguous()
    p = Pipeline.for_workload(w, 0, precision)
    p.local(torch.as_tensor(kap, device="cuda"), mhm.quad_source(vals), mhm.SolveOpts(10, 1e-13, 0, 0))
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    AK, EK, BK, FK = p.blocks()
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    tol = TOL64 if precision == mhm.MHM_FP64 else TOL_MIXED
    for K in range(w.n_K):
        o = solve_local(mesh, K, w.r, P, kap[K], _f_nonpoly)
        assert abs(o.EK).max() > 1e-3 * abs(o.AK).max() * abs(o.FK) / abs(o.BK).max()   # a non-trivial load
        assert_blocks(AK[K], EK[K], BK[K], FK[K], o, tol, K)


def test_quad_source_refusals():
    """MHM_SRC_QUAD without values, and an unknown kind, are refused (INVALID_ARG)."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    w = W.Workload("t", 1, 1, 2, 1, 1, 0, "one", "const", 1.0)
    p = Pipeline.for_workload(w, 0)
    kd = torch.ones(w.n_K * w.n_fine, dtype=torch.float64, device="cuda")
    for src in (mhm.Source(mhm.MHM_SRC_QUAD, 0.0, 0.0, None), mhm.Source(7, 0.0, 0.0, None)):
        with pytest.raises(mhm.MHMError) as ei:
            p.local(kd, src)
        assert ei.value.code == mhm.MHM_ERR_INVALID_ARG
