/*
 * mhm.h -- C ABI of the GB300 MHM local-problem pipeline.
 *
 * The Multiscale Hybrid-Mixed method (paper Sec. 2) splits -div(kappa grad u) = f
 * on (0,1)^2 into one independent local problem per coarse triangle K of T_H
 * and a global saddle-point problem on the skeleton (Eq. "global").  This
 * library runs the local problems and the skeleton assembly on one GPU:
 *
 *   mhm_create_mesh        splitProblem (Alg. 1): T_H, faces, normals, the
 *                          multiplier space Lambda_H^{m,l}, per-K records
 *   mhm_local_solve_batch  solveLocalProblem (Alg. 1, Sec. 3, Eqs. "etaf",
 *                          "etai", "etaf_comb", "source_term") for every K:
 *                          assembly of a(.,.)_K on the refined submesh, the
 *                          zero-mean Neumann factorisation, the N_I + 1 solves
 *                          and the face integrals (psi_j, eta_i), (psi_j, eta_f)
 *   mhm_assemble_skeleton  reduceLocalProblems' gather (Eq. "mat_global"):
 *                          the global matrix A (CSR) and right-hand side E
 *   mhm_solve_global       reduceLocalProblems' solve of Eq. "mat_global"
 *   mhm_reconstruct        computeSolution (Eq. "u_Hh") and error norms
 *
 * Conventions (the paper fixes only "globally indexed" elements and faces):
 *  - Vertex (i,j) of the grid has id j(nx+1)+i; square (i,j) is split along its
 *    (i,j)-(i+1,j+1) diagonal into K = 2(j nx + i) = [(i,j),(i+1,j),(i+1,j+1)]
 *    and K+1 = [(i,j),(i+1,j+1),(i,j+1)], counter-clockwise.
 *  - Local face a of K is opposite local vertex a.  Global faces are numbered
 *    in order of first encounter (K ascending, a = 0,1,2).
 *  - Face normal n: outward on the boundary; on an interior face with vertex
 *    ids g0 < g1, n = (t_y, -t_x) for the unit tangent t from g0 to g1.  The
 *    sign seen from K is s = n . n_F^K = +-1.
 *  - Lambda_H^{m,l}: m subfaces per face counted from the lower-id vertex,
 *    Legendre P_p (p = 0..l) of the subface coordinate in [-1,1]; global index
 *    offset(face) + q(l+1) + p; local index inside K runs over a = 0,1,2.
 *    With a degree per face (mhm_mesh_desc.l_per_face) face e carries
 *    m(l_e+1) multipliers, numbered the same way with its own l_e; inside K,
 *    local face a keeps the slots a d .. a d + m(l_a+1) - 1 of a fixed stride
 *    d = m(l_max+1) (N_I = 3d per K).  The slots past m(l_a+1) are unused:
 *    their rows and columns of A_K, and their E_K and B_K entries, are zero.
 *  - Submesh: N = 2^r segments per face, local degree P (1 or 2); lattice
 *    point (i,j), i+j <= PN, is local DOF sum_{j'<j}(PN+1-j') + i.  kappa is
 *    given per fine triangle, per K in ascending order, and inside K row by
 *    row: the N-j "up" triangles then the N-1-j "down" triangles of row j.
 *    With a level per K (mhm_mesh_desc.r_per_K) K has its own N = 2^r_K and
 *    its kappa starts at MHM_Q_KAPPA_OFFSET[K].
 *
 * Memory: every pointer named *_dev is device memory owned by the caller; the
 * library keeps no reference to it after the call returns.  Host pointers
 * (*_host, descriptors) are read during the call only.  The mesh object owns
 * its own device tables until mhm_destroy_mesh.
 *
 * Execution: calls taking a stream are asynchronous and stream-ordered; their
 * status covers argument checks and launch errors.  Per-element outcomes of
 * the local solves (convergence) are written to status_dev.
 *
 * There is no CPU fallback: without an sm_103 device every compute call
 * returns MHM_ERR_UNSUPPORTED.
 */
#ifndef MHM_H
#define MHM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mhm_status;
#define MHM_OK 0
#define MHM_ERR_INVALID_ARG 1
#define MHM_ERR_OOM 2
#define MHM_ERR_CUDA 3
#define MHM_ERR_NOT_CONVERGED 4
#define MHM_ERR_TIMEOUT 5
#define MHM_ERR_UNSUPPORTED 6

/* Arithmetic of the local solves. */
#define MHM_FP64 0   /* factorisation, solves and face integrals in FP64 */
#define MHM_MIXED 1  /* FP32 factorisation and solves, FP64 residuals and refinement */

/* Source term f of -div(kappa grad u) = f (Eq. "etaf": the load (f, phi_w)_K of the
 * source subproblem, and F_K = (f, 1)_K of Eq. "mat_global").  The integrals over every
 * fine triangle use the collapsed (Duffy) 4 x 4 Gauss rule: with a_i, w_i (i = 0..3) the
 * 4-point Gauss-Legendre nodes and weights on [0, 1], point k = 4 i + j of a fine triangle
 * with vertices (X0, X1, X2) (the kappa order below lists them: "up" (i,j),(i+1,j),(i,j+1),
 * "down" (i+1,j),(i+1,j+1),(i,j+1)) is X0 + xi (X1 - X0) + eta (X2 - X0) with xi = a_i,
 * eta = a_j (1 - a_i), weight w_i w_j (1 - a_i) times twice the triangle's area. */
#define MHM_SRC_CONST 0   /* f = value */
#define MHM_SRC_SINSIN 1  /* f = value * 2 (freq pi)^2 sin(freq pi x) sin(freq pi y) */
#define MHM_SRC_QUAD 2    /* f given by its values at those 16 points of every fine triangle:
                           * values_dev (device, caller-owned, read during the call's work
                           * on the stream) holds 16 doubles per fine triangle in the layout
                           * of kappa, i.e. the 16 values of fine triangle t of K start at
                           * 16 (kappa offset of K + t); value and freq are ignored.  Any f
                           * whose point values the caller can evaluate (paper Sec. 4.2,
                           * Eq. "source_term": (f, w)_K for a general f). */

typedef struct mhm_mesh mhm_mesh;

/* Description of T_H and of the local spaces (paper Sec. 2 and Sec. 5's
 * parameters H, m, l, k and the submesh size). */
typedef struct {
    int32_t nx, ny;   /* coarse squares on (0,1)^2, each split into two triangles */
    int32_t r;        /* refinement level of every K (2^r segments per face), 0..7 */
    int32_t degree;   /* local Lagrange degree P: 1 or 2 */
    int32_t m, l;     /* subfaces per face (>= 1) and multiplier degree (>= 0) */
    const int8_t* r_per_K;  /* optional, host, n_K entries in 0..7: the refinement level
                             * of each K (each local problem is on its own submesh; the
                             * multipliers live on the coarse faces); NULL: every K at r.
                             * Read during mhm_create_mesh only. */
    const int8_t* l_per_face;  /* optional, host, n_faces = nx(ny+1) + ny(nx+1) + nx ny
                                * entries >= 0 in the global face numbering: the multiplier
                                * degree of each face (l is then ignored); NULL: every face
                                * at l.  m(l_e+1) <= 16.  Read during mhm_create_mesh only. */
} mhm_mesh_desc;

typedef struct {
    int32_t kind;     /* MHM_SRC_* */
    double value;
    double freq;
    const double* values_dev;  /* MHM_SRC_QUAD only (else ignored, may be NULL) */
} mhm_source;

/* Dirichlet data g = c[0] + c[1] x + c[2] y + c[3] x^2 + c[4] x y + c[5] y^2 on
 * the boundary (the paper treats g = 0; a polynomial g adds (g, psi_j)_F on the
 * boundary faces to the right-hand side). */
typedef struct {
    double c[6];
} mhm_dirichlet;

/* Exact solution for error norms (optional). */
#define MHM_EXACT_SINSIN 1  /* u = c[1] sin(c[0] pi x) sin(c[0] pi y) */
#define MHM_EXACT_POLY 2    /* u = c[0] + c[1] x + c[2] y + c[3] x^2 + c[4] x y + c[5] y^2 */
typedef struct {
    int32_t kind;
    double c[6];
} mhm_exact;

/* Options of the local solves. */
typedef struct {
    int32_t it_max;   /* MIXED: maximum refinement passes (>= 1) */
    double tol;       /* MIXED: a column stops when its energy-norm error estimate
                       * r^T M r <= tol * g^T M g (M the FP32 preconditioner) */
    int64_t K_begin;  /* process K in [K_begin, K_end); K_end <= 0 means n_K */
    int64_t K_end;
    int32_t no_fallback;  /* MIXED: 0 (default): elements whose refinement fails (not
                           * converged in it_max passes, FP32 pivot breakdown) are solved
                           * again by the FP64 path, their iters entry set to -1;
                           * 1: they keep their failure status.  MIXED runs P2
                           * levels of r >= 5 on the FP64 path, and P1 levels of
                           * r = 6, 7 on the wide mixed path (FP32-preconditioned
                           * FP64 conjugate gradients, see mhm_local_solve_batch). */
    /* MIXED, P1 levels of at most 32 points and P2 levels of r <= 4: keep the local
     * factorisations across calls
     * (the paper factors each local matrix once and reuses it while kappa does not change,
     * Sec. 3).  factor_store: device memory of mhm_factor_store_size bytes (caller-owned);
     * NULL: no store.  factor_reuse 0: the call factors every element of the range and
     * keeps the factors in the store; 1: the call skips the factorisation and solves with
     * the factors the store holds, which must come from an earlier call on the same mesh
     * with the same kappa over these elements (any source f).  Other levels are factored
     * on every call. */
    void* factor_store;
    size_t factor_store_bytes;
    int32_t factor_reuse;
    /* MIXED: path of a tuning cache file (NULL: none).  For every level of the mesh without
     * a launch shape yet, the call looks the shape up in the file under the key (degree,
     * level r, right-hand sides, device name, SM count); on a miss it runs mhm_autotune's
     * search on this call's inputs (synchronously: not for stream capture) and appends the
     * result to the file. */
    const char* tuner_cache;
} mhm_solve_opts;

/* ------------------------------------------------------------------ mesh --- */

/* splitProblem (Alg. 1, first step; Sec. 3): builds T_H, the skeleton, normals,
 * signs, multiplier offsets and the per-K records on the host and uploads them
 * to `device`.  *out receives a mesh handle; free it with mhm_destroy_mesh.
 * Errors: INVALID_ARG (sizes out of range), OOM, CUDA, UNSUPPORTED (device is
 * not sm_103). */
mhm_status mhm_create_mesh(const mhm_mesh_desc* desc, int32_t device, mhm_mesh** out);
void mhm_destroy_mesh(mhm_mesh* mesh);

/* Queries for sizes and for the integer structure (bit-exact parity). */
#define MHM_Q_SIZES 0          /* int64[8]: n_K, n_faces, n_vertices, n_lambda, n_fine per K,
                                  n_local per K (with per-K levels: of the finest K),
                                  N_I per K (the slot stride, 3 m (l_max+1)), skeleton nnz */
#define MHM_Q_TRI_VERTS 1      /* int32[n_K*3] vertex ids, CCW */
#define MHM_Q_TRI_FACES 2      /* int32[n_K*3] face id of local face a */
#define MHM_Q_TRI_SIGNS 3      /* int8[n_K*3]  s = n . n_F^K */
#define MHM_Q_FACE_VERTS 4     /* int32[n_faces*2] vertex ids, lower first */
#define MHM_Q_LAMBDA_OFFSET 5  /* int64[n_faces+1] first global multiplier of each face */
#define MHM_Q_K_LAMBDA 6       /* int32[n_K*N_I] global multiplier id of each local slot
                                  (-1: unused slot of a face below the largest degree) */
#define MHM_Q_CSR_ROWPTR 7     /* int32[n_lambda+1] skeleton CSR row pointers */
#define MHM_Q_CSR_COLS 8       /* int32[nnz] skeleton CSR column ids */
#define MHM_Q_VERTEX_XY 9      /* double[n_vertices*2] */
#define MHM_Q_FACE_NORMALS 10  /* double[n_faces*2] */
#define MHM_Q_R_OF_K 11        /* int8[n_K] refinement level of each K */
#define MHM_Q_KAPPA_OFFSET 12  /* int64[n_K+1] first kappa value of each K (4^r_K values per K) */
#define MHM_Q_NODAL_OFFSET 13  /* int64[n_K+1] first value of each K in mhm_reconstruct's u_nodal */
#define MHM_Q_FACE_DEGREE 14   /* int8[n_faces] multiplier degree l_e of each face */
#define MHM_Q_SYSTEM_NNZ 15    /* int64[2]: entries of the saddle-point system [A B^T; B 0] as counted
                                  before the tables are built (mhm_create_mesh refuses meshes whose
                                  count exceeds 2^31 - 1: the CSR tables index in int32), and as built */
/* Copies the queried table into host_out (bytes must be >= its size).
 * Errors: INVALID_ARG (unknown query, short buffer). */
mhm_status mhm_mesh_query(const mhm_mesh* mesh, int32_t what, void* host_out, size_t bytes);

/* ---------------------------------------------------------- local solves --- */

/* Bytes of device scratch memory mhm_local_solve_batch needs for `precision`: a
 * region per refinement level of the mesh, one after the other.  MHM_FP64 levels
 * whose level window fits in shared memory need none (0 for a mesh of those
 * only); wider windows (P1 r = 7, P2 r = 5) live in one slot per SM of
 * rows x (rows + N_I + 1) doubles.  MHM_MIXED adds its per-level buffers. */
mhm_status mhm_local_workspace_size(const mhm_mesh* mesh, int32_t precision, size_t* bytes);

/* Bytes of the factor store that mhm_solve_opts.factor_store points to: 0 when no level
 * of the mesh keeps its factors (FP64-only meshes: P1 levels wider than 32 points, P2
 * levels of r >= 5). */
mhm_status mhm_factor_store_size(const mhm_mesh* mesh, size_t* bytes);

/* solveLocalProblem for K in [opts->K_begin, opts->K_end) (all K by default):
 * for each K, assembles A = [a(phi_j, phi_i)] with a(u,w) = (kappa grad u,
 * grad w)_K on the submesh (Eq. "source_term"), the loads (f, phi_w)_K and
 * N_i = -(s psi_i, phi_w)_{dK} (Eqs. "etaf", "etai"), solves the Neumann
 * problems in the zero-mean space V_h(K) inside V_0^perp(K) (Sec. 2, item 2),
 * and writes the local contributions to Eq. "mat_global":
 *   AK_dev[K*N_I*N_I + j*N_I + i] = (s psi_j, eta_i)_{dK}   (row-major, symmetric)
 *   EK_dev[K*N_I + j]             = -(s psi_j, eta_f)_{dK}
 *   BK_dev[K*N_I + j]             = (s psi_j, 1)_{dK}
 *   FK_dev[K]                     = (f, 1)_K
 *   status_dev[K]                 = 0, or MHM_ERR_NOT_CONVERGED (MIXED refinement
 *                                   hit it_max), or MHM_ERR_INVALID_ARG (non-positive pivot),
 *                                   or MHM_ERR_UNSUPPORTED (MIXED, wide level, pinned DOF
 *                                   on lattice row 1: left to the FP64 re-solve; zero blocks)
 *   iters_dev[K]                  = refinement passes taken (1 for FP64; conjugate-gradient
 *                                   iterations on the wide MIXED levels; -1: MIXED
 *                                   refinement failed and K was solved again in FP64); may be NULL
 * Arrays are indexed by absolute K; entries outside the range are untouched.
 * kappa_dev: n_K * 4^r doubles (with a level per K: 4^r_K from
 * MHM_Q_KAPPA_OFFSET[K]), > 0.  workspace_dev: at least mhm_local_workspace_size
 * bytes (may be NULL when that size is 0).
 * stream: a cudaStream_t (NULL = legacy default stream).  On a mesh with several
 * refinement levels, MIXED puts its level-Schur levels (P1 levels of at most 32 points,
 * each within one factor chunk, up to five of them) into one factor launch and one
 * persistent solve launch that takes the levels as work buckets, largest first; that pair
 * and the other levels run concurrently: the first on `stream`, the others on
 * library-owned side streams that wait for the work `stream` held when the call was
 * made, and `stream` waits for them before its later work (stream-ordered as a whole;
 * calls on the same mesh from several host threads must not interleave).
 * MIXED on the wide P1 levels (r = 6, 7: lattice rows of 64 and 128 points, at most 16
 * right-hand sides): the FP32 level-Schur factor of the diagonally scaled pinned matrix
 * preconditions conjugate gradients in FP64 (it_max and tol then bound its iterations;
 * the error estimate r^T M r is the refinement's), one persistent launch per level with
 * a workspace slot per resident block (Sec. 3: per-element factorisations, then only
 * products with them).  Elements whose CG fails, and those whose pinned DOF lies on
 * lattice row 1 (a level 0 one point wider than the kernel's rows), are solved again by
 * the FP64 path unless opts->no_fallback.
 * Errors: INVALID_ARG (NULL pointers, bad options, workspace too small),
 * UNSUPPORTED, CUDA (launch failure). */
mhm_status mhm_local_solve_batch(const mhm_mesh* mesh, const double* kappa_dev, const mhm_source* f,
                                 int32_t precision, const mhm_solve_opts* opts, double* AK_dev,
                                 double* EK_dev, double* BK_dev, double* FK_dev, int32_t* status_dev,
                                 int32_t* iters_dev, void* workspace_dev, size_t workspace_bytes,
                                 void* stream);

/* mhm_local_solve_batch with kappa in HOST memory, in memory-admitted waves (the
 * batch's kappa need not fit on the device): the elements of [opts->K_begin,
 * opts->K_end) are cut into contiguous waves, each as long as its kappa fits in half
 * of kappa_budget_bytes, and two device buffers of at most that size (from the
 * stream-ordered allocator, freed on `stream` at the end) alternate: the copy of wave
 * w + 1 runs on a library-owned copy stream while the solves of wave w run on
 * `stream`.  kappa_host: the whole batch's kappa in the layout of kappa_dev (with a
 * level per K, element K at MHM_Q_KAPPA_OFFSET[K]); pin it (cudaHostAlloc /
 * cudaHostRegister) for the copies to overlap the solves; it must stay valid until
 * the work on `stream` completes.  Outputs, workspace and precision as in
 * mhm_local_solve_batch; *n_waves (may be NULL) gets the number of waves.  Not for
 * stream capture.  Errors: INVALID_ARG (NULL pointers, bad range, one element's kappa
 * above half the budget), OOM, and those of mhm_local_solve_batch. */
mhm_status mhm_local_solve_waves(const mhm_mesh* mesh, const double* kappa_host, size_t kappa_budget_bytes,
                                 const mhm_source* f, int32_t precision, const mhm_solve_opts* opts,
                                 double* AK_dev, double* EK_dev, double* BK_dev, double* FK_dev,
                                 int32_t* status_dev, int32_t* iters_dev, void* workspace_dev,
                                 size_t workspace_bytes, void* stream, int32_t* n_waves);

/* Allocation-free variant of mhm_local_solve_batch with precision MHM_MIXED (the
 * paper has no counterpart: it is an interface for callers that cannot allocate
 * device memory while they run, e.g. a framework whose pool owns all device
 * memory, or a latency-critical loop that must not call cudaMalloc).  Same
 * arguments and outputs as mhm_local_solve_batch with MHM_MIXED, but the scratch
 * memory comes from a fixed 32 MiB array inside the library's device image,
 * which every GPU that loads the library holds until the process exits; the call
 * allocates nothing.  Coarse elements whose per-element scratch exceeds 32 MiB
 * are rejected with MHM_ERR_INVALID_ARG; a large batch runs with as many
 * concurrent blocks as fit in the array (the FP64 levels of the MIXED precision
 * with windows wider than shared memory too).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture.  All calls share the array,
 * and each call overwrites what the previous one left there: calls that can
 * overlap on the GPU (different streams without ordering) race and must not be
 * issued.  Elements whose refinement fails keep their failure status (there is
 * no FP64 re-solve here: opts->no_fallback is treated as 1). */
mhm_status mhm_local_solve_batch_noalloc(const mhm_mesh* mesh, const double* kappa_dev, const mhm_source* f,
                                         const mhm_solve_opts* opts, double* AK_dev, double* EK_dev,
                                         double* BK_dev, double* FK_dev, int32_t* status_dev,
                                         int32_t* iters_dev, void* stream);

/* ------------------------------------------------------------ autotuner --- */

/* Launch shape of the mixed-precision local solves of one refinement level (P1 levels of
 * at most 32 points, the level-Schur path).  Every field changes speed only: the results
 * are the same bit for bit under every shape. */
typedef struct {
    int32_t chunk;          /* elements per factor + solve launch pair: 256..8192 */
    int32_t blocks_per_sm;  /* resident solve blocks per SM: 1..4 (4: a 64-register build of the kernel) */
    int32_t op_buffers;     /* level operators staged ahead in shared memory: 2..4 (the copy
                             * of level step s + op_buffers - 1 is issued at step s) */
    int32_t l2_prefetch;    /* L2 prefetch distance in level steps beyond the staged ones (0: none) */
    int32_t prefetch_all;   /* 1: prefetch an element's whole operator set into L2 at each solve */
    int32_t op_policy;      /* L2 policy of the operator copies: 0 default, 1 evict first, 2 evict last */
    double ms_per_K;        /* mhm_autotune: measured milliseconds per element of this shape
                             * (0 for a shape set by hand or the default) */
} mhm_tuning;

/* Sets / reads the launch shape of level r (0..7) of the mesh.  Errors: INVALID_ARG (NULL,
 * r out of range, a field out of range). */
mhm_status mhm_set_tuning(mhm_mesh* mesh, int32_t r, const mhm_tuning* t);
mhm_status mhm_get_tuning(const mhm_mesh* mesh, int32_t r, mhm_tuning* t);

/* Autotuner of the launch shapes: for every level of the mesh that runs the level-Schur
 * mixed path, a coordinate search over the fields of mhm_tuning: each field in turn over
 * its candidate values, the others fixed at the best so far, two sweeps;, every candidate
 * timed with CUDA events on `stream` over the level's first elements (up to 16384) with
 * this call's inputs; the fastest shape is set on the mesh and, with cache_path, appended
 * to that file under its key (degree, level r, right-hand sides, device name, SM count).
 * Arguments as in mhm_local_solve_batch (precision MIXED); the outputs hold the last
 * candidate's results (identical under every shape).  Synchronous.  Errors: those of
 * mhm_local_solve_batch, INVALID_ARG (cache file not writable). */
mhm_status mhm_autotune(mhm_mesh* mesh, const double* kappa_dev, const mhm_source* f, const mhm_solve_opts* opts,
                        double* AK_dev, double* EK_dev, double* BK_dev, double* FK_dev, int32_t* status_dev,
                        int32_t* iters_dev, void* workspace_dev, size_t workspace_bytes, const char* cache_path,
                        void* stream);

/* -------------------------------------------------------------- skeleton --- */

/* reduceLocalProblems' gather (Eq. "mat_global"): sums the per-K blocks into
 * the global skeleton matrix A (CSR pattern from MHM_Q_CSR_ROWPTR/COLS; the two
 * contributions to a face's diagonal block are added in ascending K order, no
 * atomics) and the right-hand side E_j = sum_K EK[K, local j] + (g, psi_j)_F.
 * A_vals_dev: nnz doubles; E_dev: n_lambda doubles; g may be NULL (g = 0).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
mhm_status mhm_assemble_skeleton(const mhm_mesh* mesh, const double* AK_dev, const double* EK_dev,
                                 const mhm_dirichlet* g, double* A_vals_dev, double* E_dev,
                                 void* stream);

/* ---------------------------------------------------------- global solve --- */

/* reduceLocalProblems' solve (Alg. 1; Sec. 3, Eq. "mat_global"): solves the
 * saddle-point system [A B^T; B 0] [lambda; u0] = [E; F] in FP64 on the device,
 * with A_vals_dev / E_dev from mhm_assemble_skeleton, B from BK_dev
 * (B[K, K's local multiplier j] = BK_dev[K*N_I + j]) and F = FK_dev (n_K).
 * Writes lambda_dev (n_lambda) and u0_dev (n_K).  The matrix is assembled in CSR
 * and factored by cuSOLVER's sparse QR (a library direct solver; this stage is
 * outside the local-problem hot path).  Allocates temporary device memory.
 * Errors: INVALID_ARG (NULL, singular matrix), UNSUPPORTED, CUDA. */
mhm_status mhm_solve_global(const mhm_mesh* mesh, const double* A_vals_dev, const double* E_dev,
                            const double* BK_dev, const double* FK_dev, double* lambda_dev, double* u0_dev,
                            void* stream);

/* ------------------------------------------------------------ reconstruct --- */

/* computeSolution (Alg. 1; Sec. 2, Eq. "u_Hh"; Sec. 3): u_{H,h} = u0_K +
 * sum_i k_i eta_i + eta_f on every K, computed in FP64 as one zero-mean Neumann
 * solve per K with the combined load sum_i k_i N~_i + f~ (the k_i are the global
 * multipliers of K's local basis).  Writes u_nodal_dev[K*n_local + w] for every
 * local DOF w of K (lattice order); with a level per K,
 * u_nodal_dev[MHM_Q_NODAL_OFFSET[K] + w].  If err_sq_dev is not NULL (it needs
 * `exact`), also writes err_sq_dev[2K] = ||u_{H,h} - u||^2_{L2(K)} and
 * err_sq_dev[2K+1] = |u_{H,h} - u|^2_{H1(K)}, by the collapsed 4 x 4 Gauss rule
 * on every fine triangle.  Allocates temporary device memory, stream-ordered: per
 * resident block the level factors of one element (2/3 (PN+1)^3 doubles for P1, about
 * 11 MB at r = 7, with its level window behind them when that exceeds shared memory),
 * i.e. a few GB for a level-7 launch.
 * Errors: INVALID_ARG, UNSUPPORTED (window panel beyond shared memory), OOM, CUDA. */
mhm_status mhm_reconstruct(const mhm_mesh* mesh, const double* kappa_dev, const mhm_source* f,
                           const double* lambda_dev, const double* u0_dev, const mhm_exact* exact,
                           double* u_nodal_dev, double* err_sq_dev, void* stream);

/* ---------------------------------------------------------------- status --- */

/* Outcome word of the local solves on a mesh: a device word owned by the mesh that the
 * kernels of mhm_local_solve_batch, mhm_local_solve_waves and
 * mhm_local_solve_batch_noalloc update in stream order (atomic OR), so that a caller learns
 * of failures without reading the per-K status array:
 *   bit (1u << c)  some element finished with the final per-K status c: MHM_ERR_NOT_CONVERGED
 *                  (refinement hit it_max), MHM_ERR_INVALID_ARG (non-positive pivot),
 *                  MHM_ERR_TIMEOUT (a bounded wait for the staged operators ran out),
 *                  MHM_ERR_UNSUPPORTED (a wide-level element left to an FP64 re-solve
 *                  that was turned off);
 *                  with the default FP64 re-solve of failed mixed elements, only the
 *                  outcome of the re-solve counts;
 *   MHM_STATUS_REFINED_IN_FP64  some elements whose mixed refinement failed were solved
 *                  again by the FP64 path (their status is then OK; informational). */
#define MHM_STATUS_REFINED_IN_FP64 (1u << 16)

/* Waits for the work queued on `stream` (a cudaStream_t, NULL = legacy default stream),
 * reads the mesh's outcome word into *word_out (may be NULL) and clears it.  Returns the
 * most severe final code recorded since the last read (MHM_ERR_TIMEOUT, then
 * MHM_ERR_INVALID_ARG, then MHM_ERR_UNSUPPORTED, then MHM_ERR_NOT_CONVERGED), MHM_OK if
 * none; the calls of the
 * recorded solves must have been issued on `stream` or ordered before its current work.
 * Errors: INVALID_ARG (NULL or host-only mesh), CUDA. */
mhm_status mhm_sync_status(const mhm_mesh* mesh, void* stream, uint32_t* word_out);

/* ------------------------------------------------------------------ misc --- */

/* Text of the last error raised on the calling thread ("" if none). */
const char* mhm_last_error(void);

/* Micro-benchmark of the arithmetic pipes on `device` (used for roofline
 * denominators): out[0] = FP64 FMA GFLOP/s, out[1] = FP32 FMA GFLOP/s, each
 * over the whole GPU, 2 flops per FMA.  Synchronous. */
mhm_status mhm_measure_pipes(int32_t device, double* out_host);

/* Per-kernel timing of the local solves, a measurement aid with no counterpart in
 * the paper.  After mhm_set_timing(mesh, 1), every mhm_local_solve_batch call on
 * `mesh` records a CUDA event on its stream before and after each of its kernel
 * launches (library-owned events, created on first need and reused).
 * mhm_kernel_times waits for the events recorded since timing was enabled or last
 * read and writes, for each kernel id below (MHM_N_KERNELS entries each, host
 * arrays), the number of launches and their total duration in milliseconds; it then
 * starts a new reading.  Not thread-safe for calls on the same mesh.
 * Errors: INVALID_ARG (NULL argument, host-only mesh), CUDA. */
#define MHM_KERNEL_LOCAL_FP64 0   /* FP64 local solve */
#define MHM_KERNEL_LOCAL_MIXED 1  /* mixed-precision local solve and refinement */
#define MHM_KERNEL_SCHUR_FACTOR 2 /* mixed path, P1: level Schur complement inverses */
#define MHM_N_KERNELS 3
mhm_status mhm_set_timing(mhm_mesh* mesh, int32_t enable);
mhm_status mhm_kernel_times(const mhm_mesh* mesh, int32_t* launches_host, double* ms_host);

#ifdef __cplusplus
}
#endif
#endif /* MHM_H */
