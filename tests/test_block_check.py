"""The entry-by-entry block check used by the GPU parity tests (tests/_blocks.py),
exercised on the CPU: the oracle's trace-quadrature blocks and a second FP64 route
(the Gram form -Y^T Y of a pinned Cholesky) agree under it, and a sign error in a
small entry, which a Frobenius-norm comparison lets through, is caught."""
import numpy as np
import scipy.linalg

from _blocks import block_errors, gram_entry_error
from oracle.local import assemble_stiffness, solve_local
from oracle.mesh import build_mesh
from paper_1703_10435_gb300 import workloads as W


def _case():
    w = W.Workload("t", 2, 2, 3, 1, 2, 2, "log_uniform", "sinsin", 1.0, 1.0, seed=7)
    mesh = build_mesh(w.nx, w.ny, w.m, w.l)
    kap = W.kappa_for(w)[3]
    from oracle.run import source_fn
    o = solve_local(mesh, 3, w.r, 1, kap, source_fn("sinsin"))
    A = assemble_stiffness(o.sub, kap).toarray()
    m = o.mass
    gt = o.rhs - np.outer(m, o.rhs.sum(axis=0) / m.sum())
    Lc = np.linalg.cholesky(A[1:, 1:])
    Y = scipy.linalg.solve_triangular(Lc, gt[1:], lower=True)
    n_I = o.AK.shape[0]
    return o, -Y[:, :n_I].T @ Y[:, :n_I], Y[:, :n_I].T @ Y[:, n_I]


def test_second_route_passes():
    o, AK2, EK2 = _case()
    e = block_errors(AK2, EK2, o.BK, o.FK, o)
    assert max(e.values()) < 1e-10, e
    assert gram_entry_error(AK2, o.AK) < 1e-10


def test_small_entry_sign_error_caught():
    o, AK2, EK2 = _case()
    # the smallest entry of A_K in magnitude among the p = 2 rows (local slots 2, 5, ...)
    n = AK2.shape[0]
    rows = [j for j in range(n) if j % 3 == 2]
    i, j = min(((a, b) for a in rows for b in range(n) if b != a), key=lambda t: abs(o.AK[t]))
    bad = AK2.copy()
    bad[i, j] = -bad[i, j]
    bad[j, i] = -bad[j, i]
    frob = np.linalg.norm(bad - o.AK) / np.linalg.norm(o.AK)
    assert frob < 1e-4                       # a norm test at a loose tolerance misses it
    assert block_errors(bad, EK2, o.BK, o.FK, o)["A"] > 1e-8
