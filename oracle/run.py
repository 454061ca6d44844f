"""Algorithm 1 end to end on the oracle: splitProblem, solveLocalProblem for
every K, reduceLocalProblems, computeSolution."""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import globalsys
from .local import solve_local
from .mesh import build_mesh


def source_fn(kind: str, value: float = 1.0, freq: float = 1.0):
    """f for the workloads: constant, or 2 (freq pi)^2 sin(freq pi x) sin(freq pi y)
    (whose solution with kappa = 1 and u = 0 on the boundary is sin sin)."""
    if kind == "const":
        return float(value)
    if kind == "sinsin":
        c = 2.0 * (freq * math.pi) ** 2 * value
        return lambda x, y: c * np.sin(freq * math.pi * x) * np.sin(freq * math.pi * y)
    raise ValueError(kind)


@dataclass
class OracleRun:
    mesh: object
    locals: list
    A: object
    B: object
    E: np.ndarray
    F: np.ndarray
    G: np.ndarray
    lam: np.ndarray
    u0: np.ndarray


def run(nx, ny, r, P, m, l, kappa, f, g=None, K_subset=None, do_global=True) -> OracleRun:
    """r: refinement level of every K, or one level per K (the local problems are
    independent: each K's submesh is its own, the multipliers live on the coarse
    faces).  kappa: per K (or per K of K_subset) the 4^r_K values in the
    fine-triangle order; f: constant or callable; g: callable boundary data or
    None.  K_subset limits the local solves (then no global solve is done)."""
    mesh = build_mesh(nx, ny, m, l)
    r_of = (lambda K: int(r)) if np.ndim(r) == 0 else (lambda K: int(r[K]))
    Ks = range(mesh.n_K) if K_subset is None else K_subset
    locals_ = [solve_local(mesh, K, r_of(K), P, kappa[i if K_subset is not None else K], f)
               for i, K in enumerate(Ks)]
    if K_subset is not None or not do_global:
        return OracleRun(mesh, locals_, None, None, None, None, None, None, None)
    A, B, E, F = globalsys.assemble(mesh, locals_)
    G = globalsys.dirichlet_term(mesh, g, [1 << r_of(K) for K in range(mesh.n_K)])
    lam, u0 = globalsys.solve(mesh, A, B, E, F, G)
    return OracleRun(mesh, locals_, A, B, E, F, G, lam, u0)
