"""Plain FP64 CPU oracle of the MHM method (test infrastructure only).

This package is the independent reference against which the CUDA path is
checked.  It is used only by the tests, by ``__graft_entry__.smoke()`` and by
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; the library
never imports, links or runs anything in it, and it shares no code with the
library (only the seeded input arrays of ``workloads`` reach both).

It follows the paper's statement of the method literally, in FP64:

* ``mesh``        coarse triangulation T_H, faces, normals and the multiplier
                  space Lambda_H^{m,l}, with a subface count and degree per
                  face (Sec. 2, definitions (i) and the global problem,
                  Eq. "global");
* ``quadrature``  Gauss-Legendre rules on segments and a collapsed (Duffy)
                  Gauss rule on triangles;
* ``fem``         the second-level space V_h(K): continuous Lagrange P1/P2 on
                  an r-times uniformly refined submesh (Sec. 2);
* ``local``       solveLocalProblem (Sec. 3, Eqs. "etaf", "etai",
                  "source_term") on a submesh of any level: assembly of
                  a(.,.)_K, the zero-mean Neumann solves by the bordered system
                  (dense LU with partial pivoting; sparse LU above 2200
                  unknowns), and the face integrals (psi_j, eta_i) and
                  (psi_j, eta_f) by quadrature of traces;
* ``globalsys``   reduceLocalProblems: assembly and direct solve of the
                  saddle-point system (Eq. "mat_global");
* ``reconstruct`` computeSolution (Eq. "u_Hh") and error norms;
* ``tet3d``       the same four steps in three dimensions, on the paper's
                  experiment (Sec. 5): tetrahedral coarse mesh of the unit
                  cube, structured tetrahedral submeshes, Lagrange P1/P2
                  locals and l = 0 multipliers on m = 4^s subfaces per face.

Every function cites the passage it follows.  The readings of points where
the paper is silent (numbering, orientation, basis of Lambda_H^{m,l},
quadrature) are the conventions documented with each function; the CUDA
path implements the same conventions in its own code.
"""
