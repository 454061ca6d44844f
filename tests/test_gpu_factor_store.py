"""Factorisations kept across calls (the paper factors each local matrix once and reuses
it while kappa is unchanged, Sec. 3): a call that fills the factor store and a later call
that reuses it with a new source give the blocks of fresh calls bit for bit, over one and
over several factor chunks and over a K sub-range; the reused call's blocks agree with the
oracle for the new source."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.local import solve_local
from oracle.mesh import build_mesh
from oracle.run import source_fn
from paper_1703_10435_gb300 import mhm, workloads as W
from _blocks import assert_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


FIELDS = ("AK", "EK", "BK", "FK", "status", "iters")


def _fresh(w, kd, src, K0=0, K1=0):
    from paper_1703_10435_gb300.pipeline import Pipeline
    p = Pipeline.for_workload(w, 0, mhm.MHM_MIXED)
    p.local(kd, src, mhm.solve_opts(10, 1e-13, K0, K1))
    return p


# one chunk; two chunks (P1: 9216 elements of 8192 per chunk, P2: 4608 of 4096)
@pytest.mark.parametrize("nx,ny,P,r", [(8, 8, 1, 5), (64, 72, 1, 5), (8, 8, 2, 3), (48, 48, 2, 4)])
def test_factor_store_reuse_with_new_source(nx, ny, P, r):
    from paper_1703_10435_gb300.pipeline import Pipeline
    w = W.Workload("t", nx, ny, r, P, 2, 2, "log_uniform", "const", 1.0, seed=12)
    kd = W.kappa_for_torch(w, torch.device("cuda")).reshape(-1).contiguous()
    f1 = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    f2 = mhm.Source(mhm.MHM_SRC_SINSIN, 1.0, 2.0)
    p = Pipeline.for_workload(w, 0, mhm.MHM_MIXED)
    nbytes = mhm.mhm_factor_store_size(p.mesh)
    assert nbytes > 0
    store = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    p.local(kd, f1, mhm.solve_opts(10, 1e-13, factor_store=store, factor_reuse=0))
    q = _fresh(w, kd, f1)
    torch.cuda.synchronize()
    for name in FIELDS:
        assert torch.equal(getattr(p, name), getattr(q, name)), ("keep", name)
    mhm.mhm_set_timing(p.mesh, True)
    p.local(kd, f2, mhm.solve_opts(10, 1e-13, factor_store=store, factor_reuse=1))
    times = mhm.mhm_kernel_times(p.mesh)
    assert "k_schur_factor" not in times and times["k_local_mixed"][0] >= 1
    q = _fresh(w, kd, f2)
    torch.cuda.synchronize()
    for name in FIELDS:
        assert torch.equal(getattr(p, name), getattr(q, name)), ("reuse", name)
    if nx == 8:   # the reused factors against the oracle for the new source
        AK, EK, BK, FK = p.blocks()
        kap = W.kappa_for(w)
        mesh = build_mesh(w.nx, w.ny, w.m, w.l)
        f = source_fn("sinsin", 1.0, 2.0)
        for K in (0, 37, w.n_K - 1):
            o = solve_local(mesh, K, w.r, w.degree, kap[K], f)
            assert_blocks(AK[K], EK[K], BK[K], FK[K], o, 1e-9, K)


def test_factor_store_sub_range_and_refusals():
    from paper_1703_10435_gb300.pipeline import Pipeline
    w = W.Workload("t", 6, 5, 4, 1, 1, 2, "grf4", "const", 1.0, seed=2)
    kd = W.kappa_for_torch(w, torch.device("cuda")).reshape(-1).contiguous()
    f1 = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    f2 = mhm.Source(mhm.MHM_SRC_SINSIN, -2.0, 1.0)
    p = Pipeline.for_workload(w, 0, mhm.MHM_MIXED)
    store = torch.empty(mhm.mhm_factor_store_size(p.mesh), dtype=torch.uint8, device="cuda")
    K0, K1 = 7, 41
    p.local(kd, f1, mhm.solve_opts(10, 1e-13, K0, K1, factor_store=store))
    p.local(kd, f2, mhm.solve_opts(10, 1e-13, K0, K1, factor_store=store, factor_reuse=1))
    q = _fresh(w, kd, f2, K0, K1)
    torch.cuda.synchronize()
    NI = p.mesh.n_I
    assert torch.equal(p.AK[K0 * NI * NI:K1 * NI * NI], q.AK[K0 * NI * NI:K1 * NI * NI])
    assert torch.equal(p.EK[K0 * NI:K1 * NI], q.EK[K0 * NI:K1 * NI])
    with pytest.raises(mhm.MHMError) as ei:   # reuse without a store
        o = mhm.solve_opts(10, 1e-13)
        o.factor_reuse = 1
        p.local(kd, f2, o)
    assert ei.value.code == mhm.MHM_ERR_INVALID_ARG
    with pytest.raises(mhm.MHMError) as ei:   # a store that is too small
        p.local(kd, f2, mhm.solve_opts(10, 1e-13, factor_store=store[:-256]))
    assert ei.value.code == mhm.MHM_ERR_INVALID_ARG
