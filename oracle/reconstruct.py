"""computeSolution (Alg. 1; Sec. 2, Eq. "u_Hh"; Sec. 3): on every K,
u_{H,h} = u0_K + sum_i k_i eta_i + eta_f, with k_i the multiplier
coefficients of K's local basis (the sum over local DOFs starts at j = 0,
as in Eq. "etaf_comb"; the lower limit j = 1 printed in the expanded form is
read as a typo), and the L2 and broken H1 errors against an exact solution.
"""
from __future__ import annotations

import numpy as np

from .fem import basis, basis_grad_ref
from .quadrature import duffy_triangle


def local_u(mesh, K, loc, lam, u0):
    """Nodal values of u_{H,h} on K's submesh."""
    ids = mesh.local_lambda(K)
    n_I = len(ids)
    return u0[K] + loc.eta[:, :n_I] @ lam[ids] + loc.eta[:, n_I]


def errors(mesh, locals_, lam, u0, exact, exact_grad=None):
    """(L2 error, broken H1 seminorm error) by Duffy 4x4 quadrature per fine triangle."""
    ref, w = duffy_triangle(4)
    bary = np.stack([1.0 - ref[:, 0] - ref[:, 1], ref[:, 0], ref[:, 1]], axis=1)
    e2, h2 = 0.0, 0.0
    for K, loc in enumerate(locals_):
        sub = loc.sub
        u = local_u(mesh, K, loc, lam, u0)
        phi = basis(sub.P, bary)
        G = basis_grad_ref(sub.P, bary)
        nT = sub.tri_xy.shape[0]
        X = sub.physical(np.arange(nT), ref)
        uh = np.einsum("qb,tb->tq", phi, u[sub.dofs])
        jac = np.abs(sub.detJ)[:, None]
        e2 += float(np.sum(w[None, :] * jac * (uh - exact(X[..., 0], X[..., 1])) ** 2))
        if exact_grad is not None:
            Jinv = np.linalg.inv(sub.J)
            grad = np.einsum("qbk,tkc->tqbc", G, Jinv)
            guh = np.einsum("tqbc,tb->tqc", grad, u[sub.dofs])
            gx, gy = exact_grad(X[..., 0], X[..., 1])
            h2 += float(np.sum(w[None, :] * jac * ((guh[..., 0] - gx) ** 2 + (guh[..., 1] - gy) ** 2)))
    return np.sqrt(e2), np.sqrt(h2)
