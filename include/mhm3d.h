/*
 * mhm3d.h -- C ABI of the three-dimensional MHM local problems (the paper's
 * experiment, Sec. 5: the Darcy problem -div(kappa grad u) = f on the unit
 * cube, tetrahedral coarse elements each with its own tetrahedral submesh,
 * multipliers of degree l = 0 on m subfaces of every face, local Lagrange
 * degree k).  Same method as mhm.h (Sec. 2, Eqs. "etaf", "etai", "global",
 * "mat_global"), one GPU, FP64:
 *
 *   mhm3d_create_mesh        splitProblem (Alg. 1): T_H of the cube, faces,
 *                            normals, Lambda_H^{m,0}, per-K records and tables
 *   mhm3d_local_solve_batch  solveLocalProblem (Alg. 1, Sec. 3) for every K:
 *                            assembly on the refined submesh, the zero-mean
 *                            Neumann factorisation, the N_I + 1 solves and the
 *                            face integrals (psi_j, eta_i), (psi_j, eta_f)
 *   mhm3d_assemble_skeleton  reduceLocalProblems' gather (Eq. "mat_global"):
 *                            the global matrix A (CSR) and right-hand side E
 *
 * Conventions (the paper gives only the element counts 24, 192, 1536, 12288
 * and generates its submeshes with TetGen; these structured meshes have the
 * same counts):
 *  - nc^3 cubes; corner (i,j,k) is vertex i + (nc+1)(j + (nc+1)k), then the
 *    cube centres, then the centres of the grid faces normal to x, y, z.  Each
 *    cube is cut into 24 tetrahedra (centre, face centre, both ends of one
 *    edge of that face): faces -x,+x,-y,+y,-z,+z, on each the corners
 *    (0,0),(1,0),(1,1),(0,1) of the two other axes in increasing order and
 *    the edge from corner q to q+1 (mod 4): K = 24 cube + 4 face + edge.
 *  - Local face a of K is opposite local vertex a; global faces are numbered
 *    in order of first encounter (K ascending, a = 0..3).  Face normal:
 *    outward on the boundary, else along (x_g1 - x_g0) x (x_g2 - x_g0) for the
 *    sorted vertex ids g0 < g1 < g2; s = n . n_F^K = +-1.
 *  - Lambda_H^{m,0}, m = 4^s: the uniform refinement of each face triangle in
 *    the frame of its sorted vertices, row j: "up" then "down" triangles;
 *    psi_{F,q} is the indicator of subface q; global id F m + q, local id
 *    inside K a m + q (N_I = 4m).
 *  - Submesh: the Freudenthal refinement of K = (v0..v3) seen as the simplex
 *    {N >= A >= B >= C >= 0}, N = 2^r, barycentrics ((N-A), (A-B), (B-C), C)/N;
 *    its 8^r tetrahedra in the order: base point z (z3, then z2, then z1
 *    ascending), then the permutation of the three unit steps in
 *    lexicographic order.  kappa is given per sub-tetrahedron in that order,
 *    8^r values per K.  Local DOFs: lattice points of spacing 1/(kN),
 *    C ascending, then B = C..kN, then A = B..kN.
 *
 * Memory and execution as in mhm.h: *_dev pointers are caller-owned device
 * memory; calls taking a stream are asynchronous and stream-ordered; there is
 * no CPU fallback (a host-only mesh, device -1, answers queries only).
 */
#ifndef MHM3D_H
#define MHM3D_H

#include <stddef.h>
#include <stdint.h>

#include "mhm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhm_mesh3d mhm3d_mesh;   /* opaque, library-owned */

typedef struct {
    int32_t nc;      /* cubes per side of the unit cube (n_K = 24 nc^3) */
    int32_t r;       /* refinement level of every submesh: 8^r tetrahedra */
    int32_t degree;  /* local Lagrange degree k: 1 or 2 */
    int32_t m;       /* subfaces per face: 4^s with s <= r (Lambda_H^{m,0}) */
} mhm3d_mesh_desc;

/* splitProblem in 3-D (Alg. 1, Sec. 5's cube).  device: CUDA device for the
 * tables, or -1 for a host-only mesh (queries only).  Refused with
 * MHM_ERR_INVALID_ARG: nc < 1, r < 0, degree not 1 or 2, m not a power of 4
 * above r's refinement, a local trace space not richer than the multipliers
 * (degree 1 needs 2^r >= 2 sqrt(m): otherwise A_K has a kernel), or sizes past
 * the int32 indexing of the skeleton.  With a device, local spaces whose
 * factor and right-hand sides exceed shared memory (k = 2: r <= 2; k = 1:
 * r <= 3; and m <= 16) are refused with MHM_ERR_UNSUPPORTED. */
mhm_status mhm3d_create_mesh(const mhm3d_mesh_desc* desc, int32_t device, mhm3d_mesh** out);
void mhm3d_destroy_mesh(mhm3d_mesh* mesh);

/* Host copies of the mesh tables (bytes: the size of host_out). */
#define MHM3D_Q_SIZES 0       /* int64[8]: n_K, n_faces, n_vertices, n_lambda, n_local (DOFs per K),
                                 N_I, n_sub (tetrahedra per K), skeleton nnz */
#define MHM3D_Q_TETS 1        /* int32[n_K*4] vertex ids */
#define MHM3D_Q_TET_FACES 2   /* int32[n_K*4] face of local face a */
#define MHM3D_Q_TET_SIGNS 3   /* int8[n_K*4] s = n . n_F^K */
#define MHM3D_Q_FACES 4       /* int32[n_faces*3] sorted vertex ids */
#define MHM3D_Q_VERTICES 5    /* double[n_vertices*3] */
#define MHM3D_Q_NORMALS 6     /* double[n_faces*3] */
#define MHM3D_Q_CSR_ROWPTR 7  /* int32[n_lambda+1] skeleton CSR row pointers */
#define MHM3D_Q_CSR_COLS 8    /* int32[nnz] skeleton CSR column ids (ascending per row) */
#define MHM3D_Q_SUB_DOFS 9    /* int32[n_sub * (4 or 10)] local DOFs of each sub-tetrahedron */
#define MHM3D_Q_NODES 10      /* int32[n_local*3] lattice coordinates (A, B, C) of the local DOFs */
#define MHM3D_Q_FACE_PERM 11  /* int8[n_K*4] order of local face a's vertices (increasing local index)
                                 against its sorted global ids: the index p of the permutation, in
                                 lexicographic order, that lists them sorted */
#define MHM3D_Q_FTAB_OFF 12   /* int32[24*(m+1)] face-load table: entries [off[b+q], off[b+q+1]) of
                                 subface q, b = (6a + p)(m+1), for local face a seen with permutation p */
#define MHM3D_Q_FTAB_NODE 13  /* int16[entries] local DOF of each entry (entries = off[24(m+1)-1]) */
#define MHM3D_Q_FTAB_COUNT 14 /* int8[entries] fine face triangles of the subface that load the DOF; each
                                 puts |fine face| / 3 on it (P1: its vertices, P2: its edge midpoints) */
#define MHM3D_Q_QUAD 15       /* double[64*(4+nb)] collapsed 4x4x4 Gauss rule on the reference
                                 tetrahedron (x, y, z, w per point), then the nb basis values per point */
mhm_status mhm3d_mesh_query(const mhm3d_mesh* mesh, int32_t what, void* host_out, size_t bytes);

#define MHM3D_SRC_CONST 0     /* f = value */
#define MHM3D_SRC_SINSINSIN 1 /* f = value 3 (freq pi)^2 sin(freq pi x) sin(freq pi y) sin(freq pi z)
                                 (freq = 2: the paper's model problem, exact u = sin sin sin) */
typedef struct {
    int32_t kind;
    double value;
    double freq;
} mhm3d_source;

/* Options of mhm3d_local_solve_batch (NULL: the defaults in brackets). */
typedef struct {
    int32_t it_max;       /* MIXED: refinement passes, >= 1 [8] */
    double tol;           /* MIXED: a column is done when |S r| <= tol |S g~| (S = diag^-1/2 of
                             the pinned matrix, r = g~ - A z its FP64 residual) [1e-9] */
    int32_t no_fallback;  /* MIXED: 0 [default]: elements whose FP32 factor breaks down or whose
                             refinement does not converge are solved again in FP64 (iters -1);
                             1: they keep MHM_ERR_NOT_CONVERGED */
} mhm3d_opts;

/* solveLocalProblem for the elements K0 <= K < K1 (K1 <= 0: n_K) (Sec. 3, Eqs.
 * "etaf", "etai"): the stiffness a(u,w)_K = (kappa grad u, grad w)_K assembled on
 * the submesh from one element matrix per class of congruent sub-tetrahedra, the
 * loads N_i = -(s psi_i, phi_w)_{dK} and (f, phi_w)_K (a collapsed 4x4x4 Gauss
 * rule per sub-tetrahedron for the non-constant f), the compatibility
 * projection, and the face integrals of the zero-mean solutions.
 *   MHM_FP64: a Cholesky factorisation with local DOF 0 pinned and the forward
 *     substitution of the N_I + 1 right-hand sides, the face integrals in Gram
 *     form (s psi_j, eta_i)_{dK} = -Y_j . Y_i with Y = L^{-1} times the
 *     projected loads.
 *   MHM_MIXED (N_I <= 16, i.e. m <= 4; larger m runs MHM_FP64): the pinned
 *     matrix scaled by its diagonal is factored once in FP32 (Sec. 3: factor once,
 *     then only products with the factor), the solutions are refined in FP64
 *     against the matrix-free FP64 residual, and the face integrals use the
 *     corrected bilinear form -(g~_j . z_i + z_j . r_i), second order in the
 *     solution error.
 * Outputs (device, caller-owned, indexed by K):
 *   AK_dev[K][j][i] = (s psi_j, eta_i)_{dK}  (N_I x N_I, symmetric)
 *   EK_dev[K][j]    = -(s psi_j, eta_f)_{dK}
 *   BK_dev[K][j]    = (s psi_j, 1)_{dK}
 *   FK_dev[K]       = (f, 1)_K
 *   status_dev[K]   = 0, MHM_ERR_INVALID_ARG (FP64: non-positive pivot), or
 *                     MHM_ERR_NOT_CONVERGED (MIXED with no_fallback: FP32 breakdown or
 *                     it_max passes without convergence)
 *   iters_dev[K]    = refinement passes (1 for FP64; -1: solved again in FP64 after
 *                     the mixed refinement failed); may be NULL.
 * kappa_dev: 8^r values per K (sub-tetrahedron order above), > 0.
 * Errors: INVALID_ARG (NULL pointers, range, source kind, precision, options),
 * UNSUPPORTED (host-only mesh), CUDA (launch). */
mhm_status mhm3d_local_solve_batch(const mhm3d_mesh* mesh, const double* kappa_dev, const mhm3d_source* f,
                                   int32_t precision, const mhm3d_opts* opts, int64_t K0, int64_t K1,
                                   double* AK_dev, double* EK_dev, double* BK_dev, double* FK_dev,
                                   int32_t* status_dev, int32_t* iters_dev, void* stream);

/* reduceLocalProblems' gather (Eq. "mat_global"): A_vals_dev[nnz] of the
 * skeleton matrix A_ij = sum_K (s psi_j, eta_i)_{dK} on the CSR pattern of
 * MHM3D_Q_CSR_ROWPTR/COLS (the diagonal blocks of interior faces sum their two
 * elements in ascending K; every other block has one), and E_dev[n_lambda] =
 * sum_K E_K (homogeneous Dirichlet data, as in the paper's model problem).
 * B and F of Eq. "mat_global" are BK_dev and FK_dev as they are. */
mhm_status mhm3d_assemble_skeleton(const mhm3d_mesh* mesh, const double* AK_dev, const double* EK_dev,
                                   double* A_vals_dev, double* E_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MHM3D_H */
