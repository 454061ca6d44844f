"""Readers of the closed-form tables under tests/golden/ and the closed forms built from
them (shared by the oracle pins and the GPU tests; no method arithmetic of either side)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(t):
    from fractions import Fraction
    return float(Fraction(t))


def legendre_golden():
    """The closed-form Legendre table of tests/golden/legendre.txt as dicts."""
    sec, out = None, {"values": [], "norms": {}, "moments": {}}
    for line in open(os.path.join(GOLDEN, "legendre.txt")):
        if line.startswith("#") or not line.strip():
            continue
        if line.startswith("["):
            sec = line[1:line.index("]")]
            continue
        tok = line.split()
        if sec == "values":
            out["values"].append([_frac(t) for t in tok])
        elif sec == "norms":
            out["norms"][int(tok[0])] = _frac(tok[1])
        elif sec == "moments":
            out["moments"][(int(tok[0]), int(tok[1]))] = _frac(tok[2])
    return out


def dirichlet_moment(mesh, e, q, p, m, gold):
    """(g, psi_{q,p})_F on boundary face e for g = x^2 + y^2 from the golden moments:
    along the face x(tau) = x_lo + tau d (tau from the lower-id vertex), g = a0 + a1 tau
    + a2 tau^2; on subface q, tau = c + h xi with c = (q + 1/2)/m, h = 1/(2m), so
    (g, P_p)_F = |F| h sum_k g_k M(k, p) with M(k, p) = int x^k P_p (zero for k < p)."""
    xlo = mesh.verts[mesh.edges[e, 0]]
    d = mesh.verts[mesh.edges[e, 1]] - xlo
    a0, a1, a2 = float(xlo @ xlo), 2.0 * float(xlo @ d), float(d @ d)
    c, h = (q + 0.5) / m, 0.5 / m
    gk = (a0 + a1 * c + a2 * c * c, (a1 + 2.0 * a2 * c) * h, a2 * h * h)
    mom = lambda k: gold["moments"].get((k, p), 0.0)
    return float(np.linalg.norm(d)) * h * sum(gk[k] * mom(k) for k in range(3))


def reference_tet_golden():
    """The closed forms of tests/golden/reference_elements_3d.txt: the P1 stiffness of the
    reference tetrahedron (times 6), the P2 basis integrals over |T| and the monomial
    moments {(a, b, c): int x^a y^b z^c}."""
    sec, out = None, {"p1_stiffness": [], "p2_mass": {}, "moments": {}}
    for line in open(os.path.join(GOLDEN, "reference_elements_3d.txt")):
        if line.startswith("#") or not line.strip():
            continue
        if line.startswith("["):
            sec = line[1:line.index("]")]
            continue
        tok = line.split()
        if sec == "p1_stiffness":
            out["p1_stiffness"].append([float(t) for t in tok])
        elif sec == "p2_mass":
            out["p2_mass"][tok[0]] = _frac(tok[1])
        elif sec == "moments":
            out["moments"][(int(tok[0]), int(tok[1]), int(tok[2]))] = _frac(tok[3])
    out["p1_stiffness"] = np.asarray(out["p1_stiffness"]) / 6.0
    return out
