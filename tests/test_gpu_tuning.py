"""The autotuner of the mixed path's launch shapes: every shape gives the same blocks bit
for bit (the shapes change speed only), the search sets a shape on the mesh and writes its
cache line, a second mesh with the same key reads the shape from the cache through
mhm_solve_opts.tuner_cache without searching again, and invalid shapes are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1703_10435_gb300 import mhm, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_10435_gb300 import build
    build.build()


FIELDS = ("AK", "EK", "BK", "FK", "status", "iters")


def _case():
    from paper_1703_10435_gb300.pipeline import Pipeline
    w = W.Workload("t", 24, 24, 5, 1, 2, 2, "grf4", "const", 1.0, seed=4)     # 1152 elements
    kd = W.kappa_for_torch(w, torch.device("cuda")).reshape(-1).contiguous()
    return w, kd, Pipeline.for_workload(w, 0, mhm.MHM_MIXED)


@pytest.mark.parametrize("shape", [(256, 1, 2, 0, 0, 0), (1024, 2, 3, 4, 0, 1), (8192, 3, 4, 0, 1, 2), (4096, 4, 2, 0, 0, 1),
                                   (512, 3, 4, 8, 0, 2)])
def test_every_shape_same_result(shape):
    w, kd, p = _case()
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    p.local(kd, src)
    ref = {k: getattr(p, k).clone() for k in FIELDS}
    mhm.mhm_set_tuning(p.mesh, 5, mhm.Tuning(*shape, 0.0))
    assert mhm.mhm_get_tuning(p.mesh, 5).as_dict()["chunk"] == shape[0]
    for k in FIELDS:
        getattr(p, k).zero_()
    p.local(kd, src)
    torch.cuda.synchronize()
    for k in FIELDS:
        assert torch.equal(getattr(p, k), ref[k]), (shape, k)


def test_autotune_and_cache(tmp_path):
    w, kd, p = _case()
    src = mhm.Source(mhm.MHM_SRC_CONST, 1.0, 1.0)
    cache = tmp_path / "tune.txt"
    mhm.mhm_autotune(p.mesh, kd, src, None, p.AK, p.EK, p.BK, p.FK, p.status, p.iters, p.workspace, cache)
    t = mhm.mhm_get_tuning(p.mesh, 5)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "P=1 r=5 R=19" in lines[0] and "chunk=%d " % t.chunk in lines[0]
    ms = float(lines[0].split("ms_per_K=")[1])
    assert 0.0 < ms < 1.0
    # a new mesh with the same key: the shape comes from the cache, no new line
    from paper_1703_10435_gb300.pipeline import Pipeline
    q = Pipeline.for_workload(w, 0, mhm.MHM_MIXED)
    q.local(kd, src, mhm.solve_opts(tuner_cache=cache))
    torch.cuda.synchronize()
    assert cache.read_text().splitlines() == lines
    assert mhm.mhm_get_tuning(q.mesh, 5).as_dict() == t.as_dict()
    assert int(q.status.abs().sum()) == 0
    p.local(kd, src)
    torch.cuda.synchronize()
    for k in FIELDS:
        assert torch.equal(getattr(p, k), getattr(q, k)), k
    # a key that is not in the cache yet (another level) is searched and appended
    w2 = W.Workload("t", 12, 12, 4, 1, 2, 2, "grf4", "const", 1.0, seed=4)
    q2 = Pipeline.for_workload(w2, 0, mhm.MHM_MIXED)
    kd2 = W.kappa_for_torch(w2, torch.device("cuda")).reshape(-1).contiguous()
    q2.local(kd2, src, mhm.solve_opts(tuner_cache=cache))
    torch.cuda.synchronize()
    assert len(cache.read_text().splitlines()) == 2


def test_invalid_shapes_refused():
    w, kd, p = _case()
    for bad in [(100, 3, 2, 0, 0, 0), (1024, 5, 2, 0, 0, 0), (1024, 3, 5, 0, 0, 0), (1024, 3, 2, -1, 0, 0),
                (1024, 3, 2, 0, 2, 0), (1024, 3, 2, 0, 0, 3)]:
        with pytest.raises(mhm.MHMError) as ei:
            mhm.mhm_set_tuning(p.mesh, 5, mhm.Tuning(*bad, 0.0))
        assert ei.value.code == mhm.MHM_ERR_INVALID_ARG
    with pytest.raises(mhm.MHMError):
        mhm.mhm_set_tuning(p.mesh, 3, mhm.Tuning(1024, 3, 2, 0, 0, 0, 0.0))   # no level 3 in this mesh
