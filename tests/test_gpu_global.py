"""The whole Algorithm 1 on the GPU through the C ABI: local solves, skeleton
assembly, the global saddle-point solve (Eq. "mat_global") and computeSolution
(Eq. "u_Hh"), checked against the FP64 oracle and against exact solutions the
discrete spaces contain."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reconstruct as orec
from oracle.run import run, source_fn
from paper_1703_10435_gb300 import mhm, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


def _gpu_all(w, kap, precision=mhm.MHM_FP64, dirichlet=None, exact=None, src=None):
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    p = Pipeline.for_workload(w, 0, precision)
    kd = torch.as_tensor(kap, device="cuda").contiguous()
    src = src or source_of(w)
    p.step(kd, src, dirichlet, mhm.SolveOpts(10, 1e-13, 0, 0))
    p.solve_global()
    u, err = p.reconstruct(kd, src, exact)
    torch.cuda.synchronize()
    assert int(p.status.abs().sum()) == 0
    return p, u.cpu().numpy(), None if err is None else err.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _dirichlet(c):
    c = list(c) + [0.0] * (6 - len(c))
    return mhm.Dirichlet((mhm.ctypes.c_double * 6)(*c))


def _exact(kind, c):
    c = list(c) + [0.0] * (6 - len(c))
    return mhm.Exact(kind, (mhm.ctypes.c_double * 6)(*c))


def test_linear_exact_recovery_full_pipeline():
    """kappa = 1, u = 1 + 2x - 3y (f = 0, g = u): the GPU pipeline reproduces u at
    every node of every submesh."""
    w = W.WORKLOADS["c1_linear"]
    kap = W.kappa_for(w)
    p, u, err = _gpu_all(w, kap, dirichlet=_dirichlet((1, 2, -3)), exact=_exact(mhm.MHM_EXACT_POLY, (1, 2, -3)))
    o = run(w.nx, w.ny, w.r, 1, w.m, w.l, kap, 0.0, g=lambda x, y: 1 + 2 * x - 3 * y)
    for K, loc in enumerate(o.locals):
        xy = loc.sub.node_xy
        assert np.abs(u[K] - (1 + 2 * xy[:, 0] - 3 * xy[:, 1])).max() < 1e-11
    assert math.sqrt(err[:, 0].sum()) < 1e-11 and math.sqrt(err[:, 1].sum()) < 1e-10


def test_quadratic_exact_recovery_p2_full_pipeline():
    uex = lambda x, y: x ** 2 - 2 * x * y + 3 * y ** 2 + x
    w = W.Workload("t", 2, 2, 2, 2, 1, 1, "one", "const", -8.0)
    kap = W.kappa_for(w)
    p, u, err = _gpu_all(w, kap, dirichlet=_dirichlet((0, 1, 0, 1, -2, 3)),
                         exact=_exact(mhm.MHM_EXACT_POLY, (0, 1, 0, 1, -2, 3)))
    o = run(2, 2, 2, 2, 1, 1, kap, -8.0, g=uex)
    for K, loc in enumerate(o.locals):
        xy = loc.sub.node_xy
        assert np.abs(u[K] - uex(xy[:, 0], xy[:, 1])).max() < 1e-11


@pytest.mark.parametrize("name,P,r,m,l,nx,field", [("c1_sin", 1, 3, 1, 1, 4, "one"),
                                                  ("h1", 1, 3, 2, 2, 3, "log_uniform"),
                                                  ("h2", 2, 2, 3, 1, 2, "log_uniform")])
def test_multipliers_and_solution_vs_oracle(name, P, r, m, l, nx, field):
    w = W.Workload(name, nx, nx, r, P, m, l, field, "sinsin", 1.0, 1.0, seed=4)
    kap = W.kappa_for(w)
    ex = _exact(mhm.MHM_EXACT_SINSIN, (1.0, 1.0))
    p, u, err = _gpu_all(w, kap, exact=ex)
    o = run(nx, nx, r, P, m, l, kap, source_fn("sinsin"))
    assert _rel(p.lam.cpu().numpy(), o.lam) < 1e-10
    assert _rel(p.u0.cpu().numpy(), o.u0) < 1e-10
    uo = np.stack([orec.local_u(o.mesh, K, loc, o.lam, o.u0) for K, loc in enumerate(o.locals)])
    assert _rel(u, uo) < 1e-10
    e_l2, e_h1 = orec.errors(o.mesh, o.locals, o.lam, o.u0,
                             lambda x, y: np.sin(math.pi * x) * np.sin(math.pi * y),
                             lambda x, y: (math.pi * np.cos(math.pi * x) * np.sin(math.pi * y),
                                           math.pi * np.sin(math.pi * x) * np.cos(math.pi * y)))
    assert math.sqrt(err[:, 0].sum()) == pytest.approx(e_l2, rel=1e-8)
    assert math.sqrt(err[:, 1].sum()) == pytest.approx(e_h1, rel=1e-8)


@pytest.mark.parametrize("field", ["log_uniform", "grf4"])
def test_mixed_vs_fp64_and_oracle_solution(field):
    """Mixed-precision local solves on a heterogeneous 8 x 8 mesh (128 K, P1 r = 5, 561
    unknowns per K): multipliers, u0 and the reconstructed nodal u within 1e-8 relative
    (L2) of the FP64 oracle, and of the GPU's all-FP64 path."""
    w = W.Workload("t", 8, 8, 5, 1, 2, 2, field, "const", 1.0, seed=6)
    kap = W.kappa_for(w)
    p64, u64, _ = _gpu_all(w, kap, mhm.MHM_FP64)
    pm, um, _ = _gpu_all(w, kap, mhm.MHM_MIXED)
    assert int(pm.iters.max()) >= 2               # the mixed path did refine
    assert _rel(pm.lam.cpu().numpy(), p64.lam.cpu().numpy()) < 1e-8
    assert _rel(um, u64) < 1e-8
    o = run(w.nx, w.ny, w.r, 1, w.m, w.l, kap, 1.0)
    uo = np.stack([orec.local_u(o.mesh, K, loc, o.lam, o.u0) for K, loc in enumerate(o.locals)])
    for u_, p_ in ((um, pm), (u64, p64)):
        assert _rel(p_.lam.cpu().numpy(), o.lam) < 1e-8
        assert _rel(p_.u0.cpu().numpy(), o.u0) < 1e-8
        assert _rel(u_, uo) < 1e-8


def test_quad_source_solution_vs_oracle():
    """f = exp(x) cos(3y) + 1/(1+x+y), given by its point values (MHM_SRC_QUAD), through the
    whole pipeline (local solves, skeleton, global solve, computeSolution) against the oracle
    evaluating the same f: multipliers, u0 and nodal u within 1e-10."""
    f = lambda x, y: np.exp(x) * np.cos(3.0 * y) + 1.0 / (1.0 + x + y)
    w = W.Workload("t", 3, 3, 3, 1, 2, 1, "log_uniform", "const", 1.0, seed=5)
    kap = W.kappa_for(w)
    pts = W.source_points(W.coarse_vertices(w.nx, w.ny), w.N)
    vals = torch.as_tensor(f(pts[..., 0], pts[..., 1]).reshape(-1), device="cuda").contiguous()
    p, u, _ = _gpu_all(w, kap, src=mhm.quad_source(vals))
    o = run(w.nx, w.ny, w.r, 1, w.m, w.l, kap, f)
    assert _rel(p.lam.cpu().numpy(), o.lam) < 1e-10
    assert _rel(p.u0.cpu().numpy(), o.u0) < 1e-10
    uo = np.stack([orec.local_u(o.mesh, K, loc, o.lam, o.u0) for K, loc in enumerate(o.locals)])
    assert _rel(u, uo) < 1e-10


@pytest.mark.parametrize("nx,ny,m,l,per_face", [(16, 12, 2, 1, False), (7, 5, 1, 2, False), (9, 6, 2, 2, True),
                                                (1, 1, 2, 1, False), (2, 1, 1, 0, False), (12, 10, 1, 2, False)])
def test_nested_dissection_solve_vs_oracle(nx, ny, m, l, per_face):
    """The global saddle-point solve (Eq. "mat_global") by the nested-dissection multifrontal
    factorisation, on meshes whose bisection has uneven halves, blocks inside the domain
    (whose constant u0 mode is passed up), a single leaf, and a degree per face: multipliers
    and u0 against the oracle's direct sparse solve within 1e-10.  Level 3 submeshes (nine
    trace nodes per face) keep every multiplier space here inf-sup stable, so the system is
    nonsingular."""
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    from oracle.mesh import build_mesh
    w = W.Workload("t", nx, ny, 3, 1, m, l, "log_uniform", "sinsin", 1.0, 1.0, seed=13)
    kap = W.kappa_for(w)
    lf = None
    if per_face:
        lf = np.random.default_rng(5).integers(0, l + 1, build_mesh(nx, ny, 1, 0).n_e)
    p = Pipeline(nx, ny, w.r, 1, m, l, 0, mhm.MHM_FP64, l_per_face=lf)
    kd = torch.as_tensor(kap, device="cuda").contiguous()
    p.step(kd, source_of(w))
    lam, u0 = p.solve_global()
    torch.cuda.synchronize()
    o = run(nx, ny, w.r, 1, m, l if lf is None else lf, kap, source_fn("sinsin"))
    assert _rel(lam.cpu().numpy(), o.lam) < 1e-10
    assert _rel(u0.cpu().numpy(), o.u0) < 1e-10
    # a second call with the same mesh reuses the plan and gives the same result
    lam2, u02 = p.solve_global()
    torch.cuda.synchronize()
    assert torch.equal(lam, lam2) and torch.equal(u0, u02)


def test_nested_dissection_large_fronts_vs_oracle():
    """64 x 64 squares with six multipliers per face: the separators near the root have fronts
    large enough for the library path (cuSOLVER potrf / cuBLAS trsm, syrk on the multiplier
    block, then the u0 pivots passed up by the blocks inside the domain).  Against the
    oracle's direct solve, and the residual of the GPU's own assembled system."""
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    import scipy.sparse as sp
    w = W.Workload("t", 64, 64, 3, 1, 2, 2, "log_uniform", "const", 1.0, seed=17)
    kap = W.kappa_for(w)
    p = Pipeline.for_workload(w, 0, mhm.MHM_FP64)
    p.step(torch.as_tensor(kap, device="cuda").contiguous(), source_of(w))
    lam, u0 = p.solve_global()
    torch.cuda.synchronize()
    M = p.mesh
    BK = p.BK.view(M.n_K, M.n_I).cpu().numpy()
    kl = M.query(mhm.Q_K_LAMBDA, np.int32, M.n_K * M.n_I).reshape(M.n_K, M.n_I)
    rows = np.repeat(np.arange(M.n_K), M.n_I)
    B = sp.csr_matrix((BK.ravel(), (rows, kl.ravel())), shape=(M.n_K, M.n_lambda))
    l, z = lam.cpu().numpy(), u0.cpu().numpy()
    E, F = p.E.cpu().numpy(), p.FK.cpu().numpy()
    A = p.skeleton_scipy()
    assert np.linalg.norm(A @ l + B.T @ z - E) <= 1e-12 * np.linalg.norm(A @ l)
    assert np.linalg.norm(B @ l - F) <= 1e-12 * np.linalg.norm(F)
    o = run(w.nx, w.ny, w.r, 1, w.m, w.l, kap, 1.0)
    assert _rel(l, o.lam) < 1e-10
    assert _rel(z, o.u0) < 1e-10
