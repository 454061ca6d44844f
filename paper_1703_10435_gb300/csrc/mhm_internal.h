// Internal declarations shared by the translation units of libmhm.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "mhm.h"

namespace mhm {

// Thread-local error text behind mhm_last_error().
void set_error(const std::string& msg);
mhm_status fail(mhm_status code, const std::string& msg);
// Local-solve timing marks (no-ops unless timing is enabled on the mesh): begin starts a
// new reading; start/stop go around each kernel launch on stream s.
void timing_begin(const mhm_mesh* m);
void timing_mark(const mhm_mesh* m, int kernel, cudaStream_t s, bool start);
mhm_status cuda_fail(cudaError_t e, const char* what);
// Checks a source descriptor (known kind; MHM_SRC_QUAD carries its values).
mhm_status check_source(const mhm_source* f, const char* who);

#define MHM_CUDA_TRY(expr)                                              \
    do {                                                                \
        cudaError_t _e = (expr);                                        \
        if (_e != cudaSuccess) return ::mhm::cuda_fail(_e, #expr);      \
    } while (0)

// Maximum number of Gauss points in the device tables.
constexpr int kMaxGauss = 8;
// Largest local degree and multiplier layout handled by the device kernels.
constexpr int kMaxFaceDofs = 16;   // m (l + 1) per face
constexpr int kMaxNI = 3 * kMaxFaceDofs;

// One neighbour block (e, f) of face e's skeleton row: the K shared by e and f
// (two K when f == e on an interior face) and the local faces of e and f in them.
struct FaceNbr {
    int32_t f;
    int32_t col_off;   // offset of face f's columns inside the rows of face e
    int32_t K0, a0, b0;
    int32_t K1, a1, b1;  // K1 = -1 if only one contribution
};

// Per-K geometry and orientation record, device side (structure of arrays).
struct DeviceMesh {
    const double* geom;      // n_K * 6: v0, v1, v2
    const int8_t* sign;      // n_K * 3
    const int8_t* rev;       // n_K * 3: 1 if local face a runs from the higher-id vertex
    const double* btab;      // face-load table: dofs_per_face * (PN+1): int psi_{q,p} phi_k over [0,1]
    const double* btab_sum;  // dofs_per_face: int psi_{q,p} over [0,1]
    const double* gauss_x;   // kMaxGauss * kMaxGauss: n-point Gauss-Legendre nodes on [0,1], row n-1
    const double* gauss_w;
    const int32_t* klist;    // coarse element of each launch index (NULL: the index itself)
    const int64_t* kap_off;  // first kappa value of each K (NULL: K * 4^r)
    const int8_t* lface;     // n_K * 3: degree of local face a (NULL: every face at the largest degree)
    int fm, lmax1;           // subfaces per face; largest degree + 1 (the table's row stride per subface)
};

// Launch shape of the mixed-precision local solves of one refinement level (the
// autotuner's choices; defaults below): see mhm_tuning in mhm.h.
struct Tuning {
    int chunk = 8192;        // elements per factor + solve launch pair (<= kChunkMax)
    int blocks_per_sm = 3;   // resident solve blocks per SM (<= the kernel's occupancy)
    int nbuf = 2;            // staged level operators in the shared-memory ring (2..4)
    int l2pf = 0;            // L2 prefetch distance in level steps (0: none)
    int pf_all = 0;          // 1: prefetch the element's whole operator set into L2 per solve
    int op_policy = 1;       // L2 policy of the operator copies: 0 default, 1 evict first, 2 evict last
    int tuned = 0;           // 1: set by the autotuner or a tuning cache
};

// Multifrontal factorisation plan of the global saddle-point system (mhm_solve_global):
// built on the first call, kept by the mesh.
struct NDPlan;
void free_nd_plan(NDPlan* p);

// The coarse elements of one refinement level: the local-solve and reconstruction
// kernels run one launch per level (uniform meshes have a single level).
struct Level {
    int r = 0, N = 1, PN = 1;
    int64_t nK = 0, nfine = 0, nloc = 0;
    std::vector<int32_t> K;        // ascending; empty on a uniform mesh (K = launch index)
    std::vector<double> btab;      // face-load table of this level (dofs_per_face x (PN + 1))
    int32_t* d_K = nullptr;
    double* d_btab = nullptr;      // NULL: the mesh's table (uniform mesh)
    // mixed path, several chunks: the factor launches run on their own stream, one chunk
    // ahead of the solve launches (created on first use)
    mutable Tuning tune;
    mutable cudaStream_t fstream = nullptr;
    mutable cudaEvent_t fstart = nullptr, fdone[2] = {nullptr, nullptr}, mdone[2] = {nullptr, nullptr};
};

}  // namespace mhm

struct mhm_mesh {
    int device = 0;
    // per-kernel timing of the local solves (mhm_set_timing): events recorded on the
    // caller's stream around each launch since the last reading, pairs (start, stop)
    mutable bool timing = false;
    mutable std::vector<cudaEvent_t> tev;      // event pool, reused
    mutable std::vector<int32_t> tev_kernel;   // kernel id per recorded pair
    mutable size_t tev_used = 0;
    mhm_mesh_desc desc{};
    int64_t nK = 0, ne = 0, nv = 0, nlam = 0, nfine = 0, nloc = 0, NI = 0, nnz = 0;
    int32_t N = 1, PN = 1, dpf = 1;  // 2^r, P*N, slots per face m(l_max+1) (the per-K stride)

    // host tables
    std::vector<double> vxy;          // nv*2
    std::vector<int32_t> tri_v;       // nK*3
    std::vector<int32_t> tri_f;       // nK*3
    std::vector<int8_t> tri_s;        // nK*3
    std::vector<int8_t> tri_rev;      // nK*3
    std::vector<int32_t> face_v;      // ne*2
    std::vector<int32_t> face_K;      // ne*2 (second = -1 on the boundary)
    std::vector<double> normals;      // ne*2
    std::vector<int64_t> lam_off;     // ne+1
    std::vector<int32_t> lam_face;    // nlam: face of each global multiplier
    std::vector<int8_t> face_l;       // ne: multiplier degree of each face
    std::vector<int8_t> tri_l;        // nK*3: degree of local face a (non-uniform degrees only)
    std::vector<int32_t> k_lambda;    // nK*NI (-1: unused slot)
    std::vector<int32_t> csr_rowptr;  // nlam+1
    std::vector<int32_t> csr_cols;    // nnz
    std::vector<int32_t> nbr_ptr;     // ne+1
    std::vector<mhm::FaceNbr> nbrs;   // per face neighbour blocks
    std::vector<double> btab, btab_sum, gauss_x, gauss_w;
    // saddle-point system [A B^T; B 0] in CSR: pattern and, per entry, the source of its
    // value (>= 0: index into the skeleton CSR values; < 0: -(index into BK) - 1)
    int64_t aug_nnz = 0;
    int64_t sys_count = 0;   // the saddle-point entries as counted by the int32 guard of mhm_create_mesh
    std::vector<int32_t> aug_rowptr, aug_cols;
    std::vector<int64_t> aug_src;

    // device copies (owned)
    double* d_geom = nullptr;
    int8_t* d_sign = nullptr;
    int8_t* d_rev = nullptr;
    double* d_btab = nullptr;
    double* d_btab_sum = nullptr;
    double* d_gauss_x = nullptr;
    double* d_gauss_w = nullptr;
    int32_t* d_face_v = nullptr;
    int32_t* d_face_K = nullptr;
    int32_t* d_tri_f = nullptr;
    double* d_vxy = nullptr;
    int64_t* d_lam_off = nullptr;
    int32_t* d_csr_rowptr = nullptr;
    int32_t* d_nbr_ptr = nullptr;
    mhm::FaceNbr* d_nbrs = nullptr;
    int32_t* d_aug_rowptr = nullptr;
    int32_t* d_aug_cols = nullptr;
    int64_t* d_aug_src = nullptr;
    int32_t* d_k_lambda = nullptr;
    int32_t* d_lam_face = nullptr;
    int8_t* d_lface = nullptr;            // tri_l on the device (NULL: uniform degree)
    // outcome word of the local solves (mhm_sync_status): bit c for a final per-K status c,
    // MHM_STATUS_REFINED_IN_FP64 for FP64 re-solves; written by the kernels with atomicOr
    uint32_t* d_sword = nullptr;
    // nested-dissection factorisation of the saddle-point system (mhm_solve_global)
    mutable mhm::NDPlan* nd = nullptr;

    // refinement level per K (meshes built with r_per_K; uniform meshes leave these empty)
    bool per_k_levels = false;
    std::vector<int8_t> r_of_K;           // n_K
    std::vector<int64_t> kap_off;         // n_K + 1: first kappa value of K (4^r_K values each)
    std::vector<int64_t> nod_off;         // n_K + 1: first nodal value of K in mhm_reconstruct's output
    int64_t* d_kap_off = nullptr;
    int64_t* d_nod_off = nullptr;
    std::vector<mhm::Level> levels;       // one per level present, ascending r
    // streams and events of the concurrent per-level launches (created on first use)
    mutable std::vector<cudaStream_t> side;
    mutable std::vector<cudaEvent_t> side_done;
    mutable cudaEvent_t fork_ev = nullptr;
    // memory-admitted waves: the copy stream and its events (created on first use)
    mutable cudaStream_t wave_copy = nullptr;
    mutable cudaEvent_t wave_start = nullptr, wave_copied[2] = {nullptr, nullptr}, wave_solved[2] = {nullptr, nullptr};

    mhm::DeviceMesh dev() const {
        return mhm::DeviceMesh{d_geom,  d_sign,  d_rev,   d_btab, d_btab_sum,  d_gauss_x,
                               d_gauss_w, nullptr, nullptr, d_lface, desc.m, desc.l + 1};
    }
    mhm::DeviceMesh dev(const mhm::Level& lv) const {
        return mhm::DeviceMesh{d_geom,    d_sign, d_rev,     lv.d_btab ? lv.d_btab : d_btab, d_btab_sum, d_gauss_x,
                               d_gauss_w, lv.d_K, d_kap_off, d_lface,                        desc.m,     desc.l + 1};
    }
};

namespace mhm {
// Launchers (defined in the .cu files).
// FP64 local solves of launch indices [K0, K1) of level lv; a level whose window exceeds
// shared memory keeps it in ws (fp64_level_workspace bytes; with less, fewer blocks)
mhm_status launch_local_fp64(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                             int64_t K0, int64_t K1, double* AK, double* EK, double* BK, double* FK,
                             int32_t* status, int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t stream);
size_t fp64_level_workspace(const mhm_mesh* mesh, const Level& lv);   // 0: window in shared memory
size_t fp64_slot_bytes(const mhm_mesh* mesh, const Level& lv);        // one block's window slot (0: shared memory)
bool fp64_level_launchable(const mhm_mesh* mesh, const Level& lv);    // panel fits shared memory, R <= 64
int fp64_window_rows(const mhm_mesh* mesh, const Level& lv);
// workspace region of one level at the given precision, and of all levels (one after the other)
size_t level_workspace_bytes(const mhm_mesh* mesh, const Level& lv, int32_t precision);
size_t local_workspace_bytes(const mhm_mesh* mesh, int32_t precision);
mhm_status launch_local_mixed(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                              const mhm_solve_opts& opts, int64_t K0, int64_t K1, double* AK,
                              double* EK, double* BK, double* FK, int32_t* status, int32_t* iters,
                              void* workspace, size_t ws_bytes, cudaStream_t stream);
// Several level-Schur levels (launch index ranges [r0[i], r1[i]), workspace regions) in one
// factor launch and one persistent solve launch; levels_launchable says whether they qualify.
bool levels_launchable(const mhm_mesh* mesh, const std::vector<const Level*>& lvs, const std::vector<int64_t>& r0,
                       const std::vector<int64_t>& r1, const mhm_solve_opts& opts);
mhm_status launch_local_mixed_levels(const mhm_mesh* mesh, const std::vector<const Level*>& lvs,
                                     const std::vector<int64_t>& r0, const std::vector<int64_t>& r1,
                                     const std::vector<char*>& regions, const double* kappa, const mhm_source& f,
                                     const mhm_solve_opts& opts, double* AK, double* EK, double* BK, double* FK,
                                     int32_t* status, int32_t* iters, cudaStream_t stream);
// FP64 local solves of the K in list[0 .. *count) (device count, at most max_n) of level lv:
// the re-solve of elements whose mixed refinement failed (their iters entry becomes -1).
mhm_status launch_local_fp64_list(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                                  const int32_t* list, const int32_t* count, int64_t max_n, double* AK, double* EK,
                                  double* BK, double* FK, int32_t* status, int32_t* iters, cudaStream_t stream);
size_t mixed_level_workspace(const mhm_mesh* mesh, const Level& lv);   // one level's region (0: FP64 level)
// bytes of the factor store of the whole mesh; *offset: level lv's region (SIZE_MAX: none)
size_t factor_store_layout(const mhm_mesh* mesh, const Level* lv, size_t* offset);
// A level on the level-Schur mixed path with the separate factor kernel (the tuned path).
bool schur_split_level(const mhm_mesh* mesh, const Level& lv);
// Offset of level lv's region in the local-solve workspace of `precision`.
size_t level_region_offset(const mhm_mesh* mesh, const Level& lv, int32_t precision);
// Launch shapes from a tuning cache, or from a search on this call's inputs (tuner_cache).
mhm_status tune_from_cache_or_search(const mhm_mesh* mesh, const double* kappa, const mhm_source& f,
                                     const mhm_solve_opts& o, double* AK, double* EK, double* BK, double* FK,
                                     int32_t* status, int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t s);
// A level the MIXED precision runs on the FP64 path: P1 levels wider than 32 points, and
// levels whose window exceeds the mixed kernel's shared memory (P2 r >= 5).  The FP32 factor
// of the wide P1 levels (levels of 64 points, jumps of 1e4 in kappa) is too inaccurate to
// drive the FP64 refinement to the tolerance in a few passes, and its error estimate is not
// reliable.
bool fp64_level(const mhm_mesh* mesh, const Level& lv);
// [i0, i1): the launch indices of level lv whose K lies in [K0, K1)
void level_range(const Level& lv, int64_t K0, int64_t K1, int64_t* i0, int64_t* i1);
mhm_status launch_skeleton(const mhm_mesh* mesh, const double* AK, const double* EK,
                           const mhm_dirichlet* g, double* A_vals, double* E, cudaStream_t stream);
bool device_supported(int device);
}  // namespace mhm
