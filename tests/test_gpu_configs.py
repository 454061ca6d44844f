"""The larger workloads at full size, in the launch configuration the bench
uses: 32768 coarse triangles with a random Fourier field (contrast 1e4), and
131072 coarse triangles with P2 locals (contrast 1e6); a sample of elements
checked one by one against the oracle, the whole batch against the FP64 path;
memory-admitted waves give the one-shot result; a CUDA graph of the step
replays it exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.local import solve_local
from oracle.mesh import build_mesh
from paper_1703_10435_gb300 import mhm, workloads as W
from _blocks import assert_blocks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,tol", [("c3_grf_mixed", 1e-9), ("c5_p2_large", 1e-9)])
def test_full_size_sampled_parity(name, tol):
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    w = W.WORKLOADS[name]
    kap = W.kappa_for_torch(w, torch.device("cuda"))
    pm = Pipeline.for_workload(w, 0, mhm.MHM_MIXED)
    pm.local(kap, source_of(w), mhm.SolveOpts(10, 1e-13, 0, 0))
    torch.cuda.synchronize()
    assert int(pm.status.abs().sum()) == 0
    rng = np.random.default_rng(2)
    Ks = sorted(set([0, w.n_K - 1] + list(rng.integers(0, w.n_K, 4))))
    kap_np = W.kappa_for(w, Ks)
    assert np.abs(kap_np - kap[Ks].cpu().numpy()).max() <= 1e-12 * kap_np.max()
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    AK = pm.AK.view(w.n_K, w.n_I, w.n_I)
    EK, BK, FK = pm.EK.view(w.n_K, w.n_I), pm.BK.view(w.n_K, w.n_I), pm.FK
    for i, K in enumerate(Ks):
        o = solve_local(mesh, int(K), w.r, w.degree, kap_np[i], float(w.source_value))
        assert_blocks(AK[K].cpu().numpy(), EK[K].cpu().numpy(), BK[K].cpu().numpy(), float(FK[K]), o, tol, K)
    # the whole batch against the FP64 path
    p64 = Pipeline.for_workload(w, 0, mhm.MHM_FP64)
    p64.local(kap, source_of(w))
    torch.cuda.synchronize()
    A64 = p64.AK.view(w.n_K, -1)
    err = (torch.linalg.norm(AK.view(w.n_K, -1) - A64, dim=1) / torch.linalg.norm(A64, dim=1)).max().item()
    assert err < tol


def test_waves_equal_one_shot():
    """Memory-admitted waves (kappa on the host, two alternating device buffers of half the
    budget): the one-shot result bit for bit, uniform and per-level meshes."""
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    w = W.Workload("t", 8, 8, 5, 1, 2, 2, "log_uniform", "const", 1.0, seed=3)
    kap = W.kappa_for(w)
    p1 = Pipeline.for_workload(w, 0, mhm.MHM_MIXED)
    p1.local(torch.as_tensor(kap, device="cuda"), source_of(w))
    p2 = Pipeline.for_workload(w, 0, mhm.MHM_MIXED)
    nw = p2.local_waves(kap, source_of(w), budget_bytes=40 * w.n_fine * 8)
    assert nw == (w.n_K + 19) // 20
    assert torch.equal(p1.AK, p2.AK) and torch.equal(p1.EK, p2.EK) and torch.equal(p1.status, p2.status)
    # levels 3..6 per element (the waves follow the per-K kappa offsets), both precisions
    rng = np.random.default_rng(4)
    rs = rng.integers(3, 7, 2 * 4 * 4).astype(np.int8)
    kl = np.concatenate([10.0 ** rng.uniform(-2, 2, 4 ** int(r)) for r in rs])
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    for prec in (mhm.MHM_FP64, mhm.MHM_MIXED):
        q1 = Pipeline(4, 4, 0, 1, 1, 2, 0, prec, r_per_K=rs)
        q1.local(torch.as_tensor(kl, device="cuda"), src)
        q2 = Pipeline(4, 4, 0, 1, 1, 2, 0, prec, r_per_K=rs)
        n = q2.local_waves(kl, src, budget_bytes=2 * 3 * 4096 * 8)
        assert n > 3
        for name in ("AK", "EK", "BK", "FK", "status", "iters"):
            assert torch.equal(getattr(q1, name), getattr(q2, name)), (prec, name)


@pytest.mark.parametrize("precision", [mhm.MHM_FP64, mhm.MHM_MIXED])
def test_cuda_graph_replay(precision):
    """The step (local solves + skeleton gather) captured once in a CUDA graph and
    replayed gives the eager result bit for bit."""
    from paper_1703_10435_gb300.pipeline import Pipeline, source_of
    w = W.WORKLOADS["c1_sin"]
    kap = torch.as_tensor(W.kappa_for(w), device="cuda")
    p = Pipeline.for_workload(w, 0, precision)
    src = source_of(w)
    p.step(kap, src)                      # first call: kernel attributes set outside capture
    torch.cuda.synchronize()
    ref = p.A_vals.clone()
    p.A_vals.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            p.step(kap, src, stream=s)
    torch.cuda.synchronize()
    for _ in range(3):
        p.A_vals.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(p.A_vals, ref)


def test_waves_sub_range_and_refusals():
    """Memory-admitted waves over a K range strictly inside a per-level mesh (the kappa base
    is offset by the first element's kappa offset) equal mhm_local_solve_batch over the same
    range bit for bit, and leave the elements outside it untouched; a budget below two
    elements' kappa and a NULL kappa_host are refused with INVALID_ARG."""
    from paper_1703_10435_gb300.pipeline import Pipeline
    rng = np.random.default_rng(8)
    rs = rng.integers(3, 6, 2 * 4 * 4).astype(np.int8)
    kl = np.concatenate([10.0 ** rng.uniform(-2, 2, 4 ** int(r)) for r in rs])
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    K0, K1 = 5, 27
    opts = mhm.SolveOpts(8, 1e-12, K0, K1)
    for prec in (mhm.MHM_FP64, mhm.MHM_MIXED):
        q1 = Pipeline(4, 4, 0, 1, 1, 2, 0, prec, r_per_K=rs)
        q1.local(torch.as_tensor(kl, device="cuda"), src, opts)
        q2 = Pipeline(4, 4, 0, 1, 1, 2, 0, prec, r_per_K=rs)
        q2.AK.fill_(7.0)
        n = q2.local_waves(kl, src, budget_bytes=2 * 3 * 1024 * 8, opts=opts)
        assert n > 2
        NI = q1.mesh.n_I
        for name, stride in (("AK", NI * NI), ("EK", NI), ("BK", NI), ("FK", 1), ("status", 1), ("iters", 1)):
            a, b = getattr(q1, name), getattr(q2, name)
            assert torch.equal(a[K0 * stride:K1 * stride], b[K0 * stride:K1 * stride]), (prec, name)
        assert float(q2.AK[:K0 * NI * NI].sub(7.0).abs().max()) == 0.0
        assert float(q2.AK[K1 * NI * NI:].sub(7.0).abs().max()) == 0.0
    q = Pipeline(4, 4, 0, 1, 1, 2, 0, mhm.MHM_MIXED, r_per_K=rs)
    big = 4 ** int(rs.max()) * 8
    with pytest.raises(mhm.MHMError) as ei:
        q.local_waves(kl, src, budget_bytes=2 * big - 8)
    assert ei.value.code == mhm.MHM_ERR_INVALID_ARG
    L = mhm.lib()
    n = mhm.ctypes.c_int32(0)
    ws = q.workspace
    code = L.mhm_local_solve_waves(q.mesh.handle, None, 1 << 30, mhm.ctypes.byref(src), mhm.MHM_MIXED, None,
                                   mhm._ptr(q.AK), mhm._ptr(q.EK), mhm._ptr(q.BK), mhm._ptr(q.FK),
                                   mhm._ptr(q.status), mhm._ptr(q.iters), mhm._ptr(ws),
                                   0 if ws is None else ws.numel(), mhm._stream(None), mhm.ctypes.byref(n))
    assert code == mhm.MHM_ERR_INVALID_ARG
