"""Entry-by-entry comparison of one coarse element's local contributions to Eq.
"mat_global" (A_K, E_K, B_K, F_K) with the oracle's.

A_K is a Gram matrix (A_K = -Y^T Y), so |A_ij| <= sqrt(A_ii A_jj) and a solver
error of relative size e in the columns of Y moves A_ij by about
e sqrt(A_ii A_jj): every entry is held to tol * sqrt(|A_ii| |A_jj|) (oracle
diagonal).  That scale follows the small rows of the high-order multipliers
down, so a wrong sign or value in a small entry cannot hide under the large
ones.  E_K, B_K are held entry by entry to tol times the largest entry of the
oracle's block (for a constant source E_K vanishes exactly and both sides hold
rounding noise, so its scale is then the size E_K has for a source of the same
magnitude, |A_K| |F_K| / |B_K|); F_K relative.
"""
import numpy as np


def block_errors(AK, EK, BK, FK, o):
    """Worst ratio of |error| to its allowed scale, per block (divide by tol to test)."""
    oA = np.asarray(o.AK)
    d = np.sqrt(np.abs(np.diag(oA)))
    scaleA = np.maximum(np.outer(d, d), 1e-300)
    eA = float((np.abs(np.asarray(AK) - oA) / scaleA).max())
    amax = float(np.abs(oA).max())
    bmax = max(float(np.abs(o.BK).max()), 1e-300)
    scaleE = max(float(np.abs(o.EK).max()), amax * abs(float(o.FK)) / bmax, 1e-300)
    eE = float(np.abs(np.asarray(EK) - o.EK).max()) / scaleE
    eB = float(np.abs(np.asarray(BK) - o.BK).max()) / bmax
    eF = abs(float(FK) - float(o.FK)) / max(abs(float(o.FK)), 1e-300) if o.FK != 0 else abs(float(FK))
    return {"A": eA, "E": eE, "B": eB, "F": eF}


def assert_blocks(AK, EK, BK, FK, o, tol, what=""):
    e = block_errors(AK, EK, BK, FK, o)
    assert max(e.values()) < tol, (what, e)
    return max(e.values())


def gram_entry_error(A, O):
    """max_ij |A_ij - O_ij| / sqrt(|O_ii| |O_jj|) for a (dense) symmetric semidefinite O:
    the skeleton matrix of Eq. "mat_global" is a sum of the A_K, so the same scale holds."""
    A, O = np.asarray(A), np.asarray(O)
    d = np.sqrt(np.abs(np.diag(O)))
    return float((np.abs(A - O) / np.maximum(np.outer(d, d), 1e-300)).max())
