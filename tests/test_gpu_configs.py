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
    for i, K in enumerate(Ks):
        o = solve_local(mesh, int(K), w.r, w.degree, kap_np[i], float(w.source_value))
        assert _rel(AK[K].cpu().numpy(), o.AK) < tol, K
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
