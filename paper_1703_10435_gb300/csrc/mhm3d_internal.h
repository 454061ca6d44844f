// Internal declarations of the three-dimensional local problems (mhm3d.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "mhm3d.h"
#include "mhm_internal.h"

namespace mhm3 {

// Largest local space whose pinned factor (packed lower triangle) and right-hand
// sides are held in one block's shared memory: 165 DOFs (k = 2, r = 2; k = 1, r = 3).
constexpr int kMaxLocal = 165;
constexpr int kMaxM = 16;                  // subfaces per face
constexpr int kMaxNI = 4 * kMaxM;          // multipliers per element
constexpr int kQuad = 64;                  // collapsed 4x4x4 Gauss rule per sub-tetrahedron
constexpr int kThreads = 512;

// One block (f, g) of the skeleton rows of face f: the columns of face g start at
// col_off inside each of f's rows; element K0 (and K1 on the diagonal block of an
// interior face, K0 < K1) contributes A_K[a m + q][b m + q'], a and b the local
// faces of f and g in that element.
struct Nbr3 {
    int32_t f, g, col_off;
    int32_t K0, a0, b0;
    int32_t K1, a1, b1;   // K1 = -1: one contribution
};

// shared memory bytes of one local-solve block (FP64 and mixed kernels)
int local3d_qsplit(int nsub);
size_t local3d_smem(int n, int NI, int nb, int nsub);
size_t local3d_smem_mixed(int n, int NI, int nb, int nsub);

// rule on [0,1] (Newton on the Legendre polynomial)
void gauss01(int n, double* x, double* w);

}  // namespace mhm3

struct mhm_mesh3d {
    int device = -1;
    mhm3d_mesh_desc desc{};
    int s = 0, M = 1, N = 1, PN = 1, nb = 4;
    int64_t nK = 0, nf = 0, nv = 0, nlam = 0, n = 0, NI = 0, nsub = 0, nnz = 0;

    // host tables
    std::vector<double> verts;        // nv*3
    std::vector<int32_t> tets;        // nK*4
    std::vector<int32_t> tet_faces;   // nK*4
    std::vector<int8_t> signs;        // nK*4
    std::vector<int8_t> perm;         // nK*4: order of face a's vertices against its sorted ids
    std::vector<int32_t> faces;       // nf*3 sorted
    std::vector<double> normals;      // nf*3
    std::vector<int32_t> face_ka;     // nf*4: K0, a0, K1, a1 (K1 = -1 on the boundary)
    std::vector<double> geom;         // nK*12: v0..v3
    std::vector<int32_t> nodes;       // n*3 lattice coordinates
    std::vector<int32_t> sub_dofs;    // nsub*nb
    std::vector<int8_t> sub_cls;      // nsub: permutation class
    std::vector<int8_t> sub_base;     // nsub*3: base point z
    std::vector<int32_t> inc_off;     // n+1: sub-tetrahedron slots t nb + a holding each local DOF
    std::vector<int32_t> inc_ent;     // nsub*nb, ascending per DOF
    std::vector<int32_t> ftab_off;    // 24*(m+1): entries of subface q of local face a under perm p
    std::vector<int16_t> ftab_node;   // local DOF
    std::vector<int8_t> ftab_cnt;     // fine face triangles of the subface that hold the DOF as a load node
    std::vector<double> quad;         // kQuad*4: x, y, z, w of the reference rule, then kQuad*nb basis values
    std::vector<int32_t> rowptr, cols;
    std::vector<mhm3::Nbr3> nbrs;

    // device copies (owned)
    double* d_geom = nullptr;
    int8_t* d_signs = nullptr;
    int8_t* d_perm = nullptr;
    int32_t* d_sub_dofs = nullptr;
    int8_t* d_sub_cls = nullptr;
    int8_t* d_sub_base = nullptr;
    int32_t* d_inc_off = nullptr;
    int32_t* d_inc_ent = nullptr;
    int32_t* d_ftab_off = nullptr;
    int16_t* d_ftab_node = nullptr;
    int8_t* d_ftab_cnt = nullptr;
    double* d_quad = nullptr;
    int32_t* d_rowptr = nullptr;
    mhm3::Nbr3* d_nbrs = nullptr;
    int32_t* d_face_ka = nullptr;
};

namespace mhm3 {
// builds every host table of the mesh (no device work); returns an error text or ""
std::string build_mesh3d_host(mhm_mesh3d* m);
}  // namespace mhm3
