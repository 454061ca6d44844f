// reduceLocalProblems' solve (Alg. 1; Sec. 3, Eq. "mat_global"):
//     [ A  B^T ] [lambda]   [E]
//     [ B  0   ] [u0    ] = [F]
// in FP64 on the GPU, by a multifrontal LDL^T factorisation in a nested-dissection order
// of the structured coarse mesh (the paper solves this system with a direct sparse solver,
// Pardiso or PaStiX, Sec. 4.1).
//
// Ordering.  The coarse squares [i0, i1) x [j0, j1) are bisected along their longer side
// down to blocks of at most 2 x 2 squares.  A cut along a grid line owns the faces on that
// line (its separator); a leaf owns the faces inside its block (and those on the domain
// boundary) and the u0 of its elements.  The elements of a leaf touch only its own faces
// and the faces on its block's boundary, which belong to ancestors' separators, so the
// factorisation of a node touches only its front: its own unknowns and the boundary
// faces of its block (the update unknowns).
//
// Pivoting.  A is negative definite, so eliminating a node's multipliers before its u0
// gives negative pivots and then positive ones (the Schur complement B (-A)^-1 B^T is
// positive definite on the u0 a block can fix: see "constant modes" at dissect).  So an
// LDL^T without pivoting is stable in this order and the fronts keep a fixed structure.
//
// Storage.  Every node has an F x F front (column-major, lower triangle) in one buffer:
// after its factorisation its first k columns hold L (unit lower triangle, diagonal entries
// replaced by D) and its trailing (F - k) x (F - k) block the update matrix its parent adds
// in.  Small fronts are factored one per thread block with the panel in shared memory;
// large separators holding multipliers only by the dense library routines (cuSOLVER potrf
// of the negated pivot block, cuBLAS trsm and syrk), converted to the same LDL^T form.  One step of iterative
// refinement against the assembled system follows the solve.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "mhm_internal.h"

namespace mhm {

struct NDNode {
    int depth = 0, parent = -1, child[2] = {-1, -1};
    int64_t k = 0, F = 0;               // own unknowns, front size
    int64_t front_off = 0, vec_off = 0;  // offsets (doubles) in the front and vector buffers
    int64_t map_off[2] = {0, 0};         // children's update positions in this front
    std::vector<int32_t> idx;            // the front's unknowns: own (elimination order), then update
    int32_t deferred = -1;               // a u0 passed up to the parent (see dissect)
    int64_t k_lam = 0;                   // own multipliers (the first k_lam own unknowns)
    bool big = false;                    // factored by the library routines
};

struct NDPlan {
    std::vector<NDNode> nodes;              // post-order (children before parents)
    std::vector<std::vector<int>> by_depth;
    int64_t n = 0, front_doubles = 0, vec_doubles = 0, map_ints = 0, idx_ints = 0;
    int64_t max_big_k = 0;
    // device
    double* fronts = nullptr;
    double* vecs = nullptr;
    double* x = nullptr;       // solution
    double* b = nullptr;       // right-hand side / residual
    double* vals = nullptr;    // values of the assembled saddle-point CSR (refinement)
    int64_t* dst = nullptr;    // per saddle-point entry: its place in a front (lower triangle), or -1
    int32_t* maps = nullptr;   // children's update -> parent front positions
    int32_t* idx = nullptr;    // all fronts' unknowns
    int64_t* idx_off = nullptr;
    int64_t* node_info = nullptr;   // per node: k, F, front_off, vec_off, map_off[0..1], child[0..1], idx offset
    int* dinfo = nullptr;           // potrf status per large node
    double* work = nullptr;         // potrf workspace
    int lwork = 0;
    cusolverDnHandle_t dn = nullptr;
    cublasHandle_t bl = nullptr;
};

void free_nd_plan(NDPlan* p) {
    if (!p) return;
    for (void* q : {(void*)p->fronts, (void*)p->vecs, (void*)p->x, (void*)p->b, (void*)p->vals, (void*)p->dst,
                    (void*)p->maps, (void*)p->idx, (void*)p->idx_off, (void*)p->node_info, (void*)p->dinfo,
                    (void*)p->work})
        if (q) cudaFree(q);
    if (p->dn) cusolverDnDestroy(p->dn);
    if (p->bl) cublasDestroy(p->bl);
    delete p;
}

namespace {

constexpr int kNodeInfo = 10;   // int64 fields per node on the device
constexpr int kNdThreads = 256;
constexpr size_t kSmallPanelBytes = 160 * 1024;   // panel (F x k doubles) of the one-block kernel

// ---------------------------------------------------------------- symbolic ---

struct Grid {
    int nx, ny;
    std::map<std::pair<int32_t, int32_t>, int32_t> face_of;   // (vertex, vertex) -> face
    int32_t face(int i0, int j0, int i1, int j1) const {     // face between grid vertices
        const int32_t a = j0 * (nx + 1) + i0, b = j1 * (nx + 1) + i1;
        auto it = face_of.find({std::min(a, b), std::max(a, b)});
        return it == face_of.end() ? -1 : it->second;
    }
};

// Builds the dissection tree of the rectangle [i0, i1) x [j0, j1); returns the node id.
//
// Constant modes.  Inside a block that does not touch the domain boundary, the flux
// balance of the block as a whole involves only the faces on its boundary: the rows of B
// restricted to the faces the block eliminates are a signed incidence matrix of the
// connected graph of its elements, of rank (elements - 1), so the last u0 pivot would be
// zero.  Such a block therefore passes one u0 up as an update unknown; a parent eliminates
// the u0 its children pass up after its separator, passes one of them on unless its own
// block touches the domain boundary, and the root eliminates what is left.
int dissect(const mhm_mesh* m, const Grid& g, NDPlan& P, int i0, int i1, int j0, int j1, int depth) {
    const int w = i1 - i0, h = j1 - j0;
    const bool touches = i0 == 0 || j0 == 0 || i1 == g.nx || j1 == g.ny;
    NDNode node;
    node.depth = depth;
    std::vector<int32_t> own;
    auto add_face = [&](std::vector<int32_t>& v, int32_t f) {
        if (f < 0) return;   // (every grid line segment is a face of the structured mesh)
        for (int64_t j = m->lam_off[f]; j < m->lam_off[f + 1]; ++j) v.push_back((int32_t)j);
    };
    int c0 = -1, c1 = -1;
    if (w <= 2 && h <= 2) {
        // leaf: faces inside the block and on the domain boundary, then the u0 of its elements
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i < i1; ++i)
                if ((j > j0 && j < j1) || j == 0 || j == g.ny) add_face(own, g.face(i, j, i + 1, j));
        for (int i = i0; i <= i1; ++i)
            for (int j = j0; j < j1; ++j)
                if ((i > i0 && i < i1) || i == 0 || i == g.nx) add_face(own, g.face(i, j, i, j + 1));
        for (int j = j0; j < j1; ++j)
            for (int i = i0; i < i1; ++i) add_face(own, g.face(i, j, i + 1, j + 1));
        for (int j = j0; j < j1; ++j)
            for (int i = i0; i < i1; ++i) {
                const int64_t K = 2 * ((int64_t)j * g.nx + i);
                own.push_back((int32_t)(m->nlam + K));
                own.push_back((int32_t)(m->nlam + K + 1));
            }
        if (!touches) {
            node.deferred = own.back();
            own.pop_back();
        }
    } else if (w >= h) {
        const int im = i0 + w / 2;
        c0 = dissect(m, g, P, i0, im, j0, j1, depth + 1);
        c1 = dissect(m, g, P, im, i1, j0, j1, depth + 1);
        for (int j = j0; j < j1; ++j) add_face(own, g.face(im, j, im, j + 1));
    } else {
        const int jm = j0 + h / 2;
        c0 = dissect(m, g, P, i0, i1, j0, jm, depth + 1);
        c1 = dissect(m, g, P, i0, i1, jm, j1, depth + 1);
        for (int i = i0; i < i1; ++i) add_face(own, g.face(i, jm, i + 1, jm));
    }
    if (c0 >= 0) {
        bool any = false;
        for (int c : {c0, c1})
            if (P.nodes[c].deferred >= 0) {
                own.push_back(P.nodes[c].deferred);
                any = true;
            }
        if (!touches && any) {
            node.deferred = own.back();
            own.pop_back();
        }
    }
    // update unknowns: the faces on the block's boundary that are not on the domain boundary
    std::vector<int32_t> upd;
    if (j0 > 0)
        for (int i = i0; i < i1; ++i) add_face(upd, g.face(i, j0, i + 1, j0));
    if (j1 < g.ny)
        for (int i = i0; i < i1; ++i) add_face(upd, g.face(i, j1, i + 1, j1));
    if (i0 > 0)
        for (int j = j0; j < j1; ++j) add_face(upd, g.face(i0, j, i0, j + 1));
    if (i1 < g.nx)
        for (int j = j0; j < j1; ++j) add_face(upd, g.face(i1, j, i1, j + 1));
    if (node.deferred >= 0) upd.push_back(node.deferred);
    node.k = (int64_t)own.size();
    node.idx = own;
    node.idx.insert(node.idx.end(), upd.begin(), upd.end());
    node.F = (int64_t)node.idx.size();
    node.child[0] = c0;
    node.child[1] = c1;
    P.nodes.push_back(std::move(node));
    const int id = (int)P.nodes.size() - 1;
    if (c0 >= 0) P.nodes[c0].parent = id;
    if (c1 >= 0) P.nodes[c1].parent = id;
    return id;
}

}  // namespace

mhm_status build_nd_plan(const mhm_mesh* m, NDPlan** out) {
    NDPlan* P = new NDPlan();
    Grid g;
    g.nx = m->desc.nx;
    g.ny = m->desc.ny;
    for (int64_t e = 0; e < m->ne; ++e) g.face_of[{m->face_v[2 * e], m->face_v[2 * e + 1]}] = (int32_t)e;
    dissect(m, g, *P, 0, g.nx, 0, g.ny, 0);
    P->n = m->nlam + m->nK;
    // every unknown owned by exactly one node
    std::vector<int32_t> node_of(P->n, -1), pos_of(P->n, -1);
    for (size_t id = 0; id < P->nodes.size(); ++id) {
        const NDNode& nd = P->nodes[id];
        for (int64_t t = 0; t < nd.k; ++t) {
            if (node_of[nd.idx[t]] >= 0) {
                free_nd_plan(P);
                return fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: an unknown owned twice by the dissection");
            }
            node_of[nd.idx[t]] = (int32_t)id;
            pos_of[nd.idx[t]] = (int32_t)t;
        }
    }
    for (int64_t u = 0; u < P->n; ++u)
        if (node_of[u] < 0) {
            free_nd_plan(P);
            return fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: an unknown owned by no node of the dissection");
        }
    int maxd = 0;
    for (NDNode& nd : P->nodes) maxd = std::max(maxd, nd.depth);
    P->by_depth.assign(maxd + 1, {});
    for (size_t id = 0; id < P->nodes.size(); ++id) {
        NDNode& nd = P->nodes[id];
        nd.front_off = P->front_doubles;
        P->front_doubles += nd.F * nd.F;
        nd.vec_off = P->vec_doubles;
        P->vec_doubles += nd.F;
        nd.k_lam = 0;   // own multipliers come first, then the own u0
        while (nd.k_lam < nd.k && nd.idx[nd.k_lam] < m->nlam) ++nd.k_lam;
        nd.big = (size_t)nd.F * nd.k * sizeof(double) > kSmallPanelBytes && nd.k_lam > 0;
        if (nd.big) P->max_big_k = std::max(P->max_big_k, nd.k_lam);
        P->by_depth[nd.depth].push_back((int)id);
    }
    // children's update positions in the parent's front
    std::vector<int32_t> maps;
    for (NDNode& nd : P->nodes) {
        std::map<int32_t, int32_t> pos;
        for (int64_t t = 0; t < nd.F; ++t) pos[nd.idx[t]] = (int32_t)t;
        for (int s = 0; s < 2; ++s) {
            nd.map_off[s] = (int64_t)maps.size();
            if (nd.child[s] < 0) continue;
            const NDNode& c = P->nodes[nd.child[s]];
            for (int64_t t = c.k; t < c.F; ++t) {
                auto it = pos.find(c.idx[t]);
                if (it == pos.end()) {
                    free_nd_plan(P);
                    return fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: a child's update unknown outside its parent");
                }
                maps.push_back(it->second);
            }
        }
    }
    P->map_ints = (int64_t)maps.size();
    // each saddle-point entry (r, c) goes to the front of whichever of r, c is eliminated
    // first (post-order of the nodes, then the order inside the node), lower triangle only
    std::vector<int64_t> dst(m->aug_nnz, -1);
    auto rank = [&](int32_t u) { return ((int64_t)node_of[u] << 32) | pos_of[u]; };
    for (int64_t r = 0; r < P->n; ++r) {
        for (int32_t t = m->aug_rowptr[r]; t < m->aug_rowptr[r + 1]; ++t) {
            const int32_t c = m->aug_cols[t];
            const int32_t first = rank((int32_t)r) <= rank(c) ? (int32_t)r : c;
            const NDNode& nd = P->nodes[node_of[first]];
            // positions of r and c in that front
            auto find = [&](int32_t u) -> int64_t {
                if (node_of[u] == node_of[first]) return pos_of[u];
                for (int64_t q = nd.k; q < nd.F; ++q)
                    if (nd.idx[q] == u) return q;
                return -1;
            };
            const int64_t pr = find((int32_t)r), pc = find(c);
            if (pr < 0 || pc < 0) {
                free_nd_plan(P);
                return fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: a matrix entry outside the fronts");
            }
            if (pr >= pc) dst[t] = nd.front_off + pr + pc * nd.F;
        }
    }
    std::vector<int64_t> info(P->nodes.size() * kNodeInfo), idx_off(P->nodes.size() + 1, 0);
    std::vector<int32_t> idx_all;
    for (size_t id = 0; id < P->nodes.size(); ++id) {
        const NDNode& nd = P->nodes[id];
        idx_off[id] = (int64_t)idx_all.size();
        idx_all.insert(idx_all.end(), nd.idx.begin(), nd.idx.end());
        int64_t* q = &info[id * kNodeInfo];
        q[0] = nd.k;
        q[1] = nd.F;
        q[2] = nd.front_off;
        q[3] = nd.vec_off;
        q[4] = nd.map_off[0];
        q[5] = nd.map_off[1];
        q[6] = nd.child[0];
        q[7] = nd.child[1];
        q[8] = (int64_t)idx_all.size() - nd.F;
        q[9] = nd.child[0] >= 0 ? P->nodes[nd.child[0]].F - P->nodes[nd.child[0]].k : 0;
    }
    idx_off.back() = (int64_t)idx_all.size();
    P->idx_ints = (int64_t)idx_all.size();
    // device
    auto up = [](const auto& v, auto** d) -> cudaError_t {
        using T = typename std::decay<decltype(v[0])>::type;
        cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(1, v.size()) * sizeof(T));
        if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        return e;
    };
    cudaError_t e = cudaMalloc((void**)&P->fronts, P->front_doubles * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->vecs, P->vec_doubles * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->x, P->n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->b, P->n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->vals, std::max<int64_t>(1, m->aug_nnz) * sizeof(double));
    if (e == cudaSuccess) e = up(dst, &P->dst);
    if (e == cudaSuccess) e = up(maps, &P->maps);
    if (e == cudaSuccess) e = up(idx_all, &P->idx);
    if (e == cudaSuccess) e = up(idx_off, &P->idx_off);
    if (e == cudaSuccess) e = up(info, &P->node_info);
    if (e == cudaSuccess) e = cudaMalloc((void**)&P->dinfo, std::max<size_t>(1, P->nodes.size()) * sizeof(int));
    if (e != cudaSuccess) {
        free_nd_plan(P);
        return cuda_fail(e, "mhm_solve_global: device memory of the factorisation");
    }
    if (cusolverDnCreate(&P->dn) != CUSOLVER_STATUS_SUCCESS || cublasCreate(&P->bl) != CUBLAS_STATUS_SUCCESS) {
        free_nd_plan(P);
        return fail(MHM_ERR_CUDA, "mhm_solve_global: cuSOLVER / cuBLAS handles");
    }
    if (P->max_big_k > 0) {
        int lw = 0;
        if (cusolverDnDpotrf_bufferSize(P->dn, CUBLAS_FILL_MODE_LOWER, (int)P->max_big_k, P->fronts,
                                        (int)P->max_big_k, &lw) != CUSOLVER_STATUS_SUCCESS) {
            free_nd_plan(P);
            return fail(MHM_ERR_CUDA, "mhm_solve_global: potrf workspace query");
        }
        P->lwork = lw;
        if (cudaMalloc((void**)&P->work, std::max(1, lw) * sizeof(double)) != cudaSuccess) {
            free_nd_plan(P);
            return fail(MHM_ERR_OOM, "mhm_solve_global: potrf workspace");
        }
    }
    *out = P;
    return MHM_OK;
}

namespace {

// ----------------------------------------------------------------- kernels ---

__global__ void k_fill_saddle(int64_t nnz, const int64_t* src, const double* A_vals, const double* BK, double* out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    const int64_t s = src[t];
    out[t] = s >= 0 ? A_vals[s] : BK[-s - 1];
}

__global__ void k_nd_assemble(int64_t nnz, const int64_t* dst, const double* vals, double* fronts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz && dst[t] >= 0) fronts[dst[t]] = vals[t];
}

// The update block of child slot s of every node in `list` added into the node's front
// (lower triangles on both sides).
__global__ void k_nd_extend_add(const int* list, int slot, const int64_t* info, const int32_t* maps, double* fronts) {
    const int id = list[blockIdx.x];
    const int64_t* q = info + (int64_t)id * kNodeInfo;
    const int64_t c = q[6 + slot];
    if (c < 0) return;
    const int64_t* qc = info + c * kNodeInfo;
    const int64_t kc = qc[0], Fc = qc[1], nu = Fc - kc, Fp = q[1];
    const int32_t* map = maps + q[4 + slot];
    const double* C = fronts + qc[2];
    double* Pf = fronts + q[2];
    for (int64_t t = threadIdx.x; t < nu * nu; t += blockDim.x) {
        const int64_t j = t / nu, i = t - j * nu;
        if (i < j) continue;
        const int64_t pi = map[i], pj = map[j];
        const int64_t hi = pi > pj ? pi : pj, lo = pi > pj ? pj : pi;
        Pf[hi + lo * Fp] += C[(kc + i) + (kc + j) * Fc];
    }
}

// LDL^T without pivoting of the first k columns of a front (one block per front): the
// F x k panel is factored in shared memory (column-major, right-looking, one pivot at a
// time), written back (L below the diagonal, D on it), and the trailing block takes
// U -= L21 D L21^T (lower triangle).
__global__ void __launch_bounds__(kNdThreads) k_nd_factor_small(const int* list, const int64_t* info, double* fronts,
                                                                int* bad) {
    extern __shared__ double pan[];
    const int id = list[blockIdx.x];
    const int64_t* q = info + (int64_t)id * kNodeInfo;
    const int k = (int)q[0], F = (int)q[1];
    double* Fr = fronts + q[2];
    for (int t = threadIdx.x; t < F * k; t += blockDim.x) {
        const int j = t / F, i = t - j * F;
        pan[t] = i >= j ? Fr[i + (int64_t)j * F] : 0.0;
    }
    __syncthreads();
    for (int p = 0; p < k; ++p) {
        const double d = pan[p + p * F];
        if (!(fabs(d) > 0.0) && threadIdx.x == 0) bad[id] = 1;   // zero or not finite
        const double inv = 1.0 / d;
        // rows below p of the remaining panel columns: P[i][j] -= P[i][p] P[j][p] / d
        const int nr = F - p - 1, nc = k - p - 1;
        for (int t = threadIdx.x; t < nr * nc; t += blockDim.x) {
            const int jj = t / nr, ii = t - jj * nr;
            const int i = p + 1 + ii, j = p + 1 + jj;
            if (i >= j) pan[i + j * F] -= pan[i + p * F] * pan[j + p * F] * inv;
        }
        __syncthreads();
        for (int i = p + 1 + threadIdx.x; i < F; i += blockDim.x) pan[i + p * F] *= inv;
        __syncthreads();
    }
    for (int t = threadIdx.x; t < F * k; t += blockDim.x) {
        const int j = t / F, i = t - j * F;
        if (i >= j) Fr[i + (int64_t)j * F] = pan[t];
    }
    // trailing update with the scaled columns: U[i][j] -= sum_p L[i][p] d_p L[j][p]
    const int nu = F - k;
    for (int64_t t = threadIdx.x; t < (int64_t)nu * nu; t += blockDim.x) {
        const int jj = (int)(t / nu), ii = (int)(t - (int64_t)jj * nu);
        if (ii < jj) continue;
        const int i = k + ii, j = k + jj;
        double s = 0.0;
        for (int p = 0; p < k; ++p) s = fma(pan[i + p * F] * pan[p + p * F], pan[j + p * F], s);
        Fr[i + (int64_t)j * F] -= s;
    }
}

// Negates the lower triangle of the k x k pivot block of a large front (potrf then
// factors -F11 = C C^T).
__global__ void k_nd_negate_pivots(double* Fr, int64_t F, int64_t k) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / k, i = t - j * k;
        if (i >= j) Fr[i + j * F] = -Fr[i + j * F];
    }
}

// From -F11 = C C^T and W = F21 C^-T to the LDL^T form: L11 = C diag(c)^-1, d = -c^2,
// L21 = -W diag(c)^-1 (c the diagonal of C).
__global__ void k_nd_to_ldlt(double* Fr, int64_t F, int64_t k) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < F * k; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / F, i = t - j * F;
        if (i < j) continue;
        const double cj = Fr[j + j * F];
        if (i == j) continue;
        Fr[i + j * F] = i < k ? Fr[i + j * F] / cj : -Fr[i + j * F] / cj;
    }
}
__global__ void k_nd_to_ldlt_diag(double* Fr, int64_t F, int64_t k) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (int64_t)gridDim.x * blockDim.x) {
        const double c = Fr[j + j * F];
        Fr[j + j * F] = -c * c;
    }
}

// One pivot p of a front (leading dimension F) eliminated right-looking over the trailing
// block: Fr[i][j] -= Fr[i][p] Fr[j][p] / d for F > i >= j > p; then the column is scaled.
__global__ void k_nd_pivot_update(double* Fr, int64_t F, int64_t p) {
    const double inv = 1.0 / Fr[p + p * F];
    const int64_t n = F - p - 1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t jj = t / n, ii = t - jj * n;
        if (ii < jj) continue;
        const int64_t i = p + 1 + ii, j = p + 1 + jj;
        Fr[i + j * F] -= Fr[i + p * F] * Fr[j + p * F] * inv;
    }
}
__global__ void k_nd_pivot_scale(double* Fr, int64_t F, int64_t p, int* bad) {
    const double d = Fr[p + p * F];
    if (!(fabs(d) > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *bad = 1;
        return;
    }
    for (int64_t i = p + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < F; i += (int64_t)gridDim.x * blockDim.x)
        Fr[i + p * F] /= d;
}

// Forward elimination and diagonal scaling of one level (one block per node): the front
// vector takes the own right-hand sides and the children's update vectors; own pivots in
// order, v[i] -= L[i][p] y_p for the rows below; then z = y / d on the own part.  The
// update part stays for the parent.
__global__ void __launch_bounds__(kNdThreads) k_nd_forward(const int* list, const int64_t* info, const int32_t* maps,
                                                           const int32_t* idx, const double* fronts, double* vecs,
                                                           const double* b) {
    const int id = list[blockIdx.x];
    const int64_t* q = info + (int64_t)id * kNodeInfo;
    const int64_t k = q[0], F = q[1];
    const double* Fr = fronts + q[2];
    double* v = vecs + q[3];
    const int32_t* ix = idx + q[8];
    for (int64_t i = threadIdx.x; i < F; i += blockDim.x) v[i] = i < k ? b[ix[i]] : 0.0;
    __syncthreads();
    for (int s = 0; s < 2; ++s) {   // children in a fixed order
        const int64_t c = q[6 + s];
        if (c < 0) continue;
        const int64_t* qc = info + c * kNodeInfo;
        const int64_t kc = qc[0], nu = qc[1] - kc;
        const double* vc = vecs + qc[3];
        const int32_t* map = maps + q[4 + s];
        for (int64_t i = threadIdx.x; i < nu; i += blockDim.x) v[map[i]] += vc[kc + i];
        __syncthreads();
    }
    for (int64_t p = 0; p < k; ++p) {
        const double yp = v[p];
        for (int64_t i = p + 1 + threadIdx.x; i < F; i += blockDim.x) v[i] = fma(-Fr[i + p * F], yp, v[i]);
        __syncthreads();
    }
    for (int64_t p = threadIdx.x; p < k; p += blockDim.x) v[p] /= Fr[p + p * F];
}

// Back substitution of one level (one block per node, parents before children): x at the
// update unknowns comes from the solution vector (ancestors); x_p = z_p - sum_{i > p}
// L[i][p] x_i for the own pivots from last to first; the own x go to the solution vector.
__global__ void __launch_bounds__(kNdThreads) k_nd_backward(const int* list, const int64_t* info, const int32_t* idx,
                                                            const double* fronts, double* vecs, double* x) {
    __shared__ double red[kNdThreads / 32];
    const int id = list[blockIdx.x];
    const int64_t* q = info + (int64_t)id * kNodeInfo;
    const int64_t k = q[0], F = q[1];
    const double* Fr = fronts + q[2];
    double* v = vecs + q[3];
    const int32_t* ix = idx + q[8];
    for (int64_t i = k + threadIdx.x; i < F; i += blockDim.x) v[i] = x[ix[i]];
    __syncthreads();
    for (int64_t p = k - 1; p >= 0; --p) {
        double s = 0.0;
        for (int64_t i = p + 1 + threadIdx.x; i < F; i += blockDim.x) s = fma(Fr[i + p * F], v[i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kNdThreads / 32; ++w) t += red[w];   // fixed order
            v[p] -= t;
        }
        __syncthreads();
    }
    for (int64_t p = threadIdx.x; p < k; p += blockDim.x) x[ix[p]] = v[p];
}

// r = b - M x for the assembled saddle-point CSR (one warp per row, fixed summation order).
__global__ void k_nd_residual(int64_t n, const int32_t* rowptr, const int32_t* cols, const double* vals,
                              const double* x, const double* b, double* r) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int32_t t = rowptr[row] + lane; t < rowptr[row + 1]; t += 32) s = fma(vals[t], x[cols[t]], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) r[row] = b[row] - s;
}

__global__ void k_rhs_saddle(int64_t L, int64_t nK, const double* E, const double* FK, double* rhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < L) rhs[t] = E[t];
    else if (t < L + nK) rhs[t] = FK[t - L];
}

__global__ void k_add_split(int64_t L, int64_t nK, const double* x, const double* dx, double* lam, double* u0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < L) lam[t] = x[t] + dx[t];
    else if (t < L + nK) u0[t - L] = x[t] + dx[t];
}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)std::max<int64_t>(1, (n + threads - 1) / threads); }

// Solves M x = rhs (in P->b) into x with the factors in the fronts, level by level.
mhm_status nd_solve(NDPlan* P, const int* d_lists, const std::vector<int64_t>& list_off, double* x, cudaStream_t s) {
    const int D = (int)P->by_depth.size();
    for (int d = D - 1; d >= 0; --d) {
        const int n = (int)P->by_depth[d].size();
        k_nd_forward<<<n, kNdThreads, 0, s>>>(d_lists + list_off[d], P->node_info, P->maps, P->idx, P->fronts, P->vecs,
                                              P->b);
    }
    for (int d = 0; d < D; ++d) {
        const int n = (int)P->by_depth[d].size();
        k_nd_backward<<<n, kNdThreads, 0, s>>>(d_lists + list_off[d], P->node_info, P->idx, P->fronts, P->vecs, x);
    }
    MHM_CUDA_TRY(cudaGetLastError());
    return MHM_OK;
}

}  // namespace

}  // namespace mhm

using namespace mhm;

extern "C" mhm_status mhm_solve_global(const mhm_mesh* mesh, const double* A_vals, const double* E,
                                       const double* BK, const double* FK, double* lambda, double* u0,
                                       void* stream) {
    if (!mesh) return fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: NULL mesh");
    if (mesh->device < 0) return fail(MHM_ERR_UNSUPPORTED, "mhm_solve_global: mesh was created without a device");
    if (!A_vals || !E || !BK || !FK || !lambda || !u0)
        return fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: NULL pointer argument");
    MHM_CUDA_TRY(cudaSetDevice(mesh->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!mesh->nd) {
        NDPlan* P = nullptr;
        mhm_status st = build_nd_plan(mesh, &P);
        if (st) return st;
        mesh->nd = P;
    }
    NDPlan* P = mesh->nd;
    if (cusolverDnSetStream(P->dn, s) != CUSOLVER_STATUS_SUCCESS || cublasSetStream(P->bl, s) != CUBLAS_STATUS_SUCCESS)
        return fail(MHM_ERR_CUDA, "mhm_solve_global: library stream");
    const int D = (int)P->by_depth.size();
    // node lists per depth (small and large fronts apart) in one device array
    std::vector<int32_t> lists;
    std::vector<int64_t> list_off(D), small_off(D), small_n(D);
    for (int d = 0; d < D; ++d) {
        list_off[d] = (int64_t)lists.size();
        for (int id : P->by_depth[d]) lists.push_back(id);
    }
    for (int d = 0; d < D; ++d) {
        small_off[d] = (int64_t)lists.size();
        for (int id : P->by_depth[d])
            if (!P->nodes[id].big) lists.push_back(id);
        small_n[d] = (int64_t)lists.size() - small_off[d];
    }
    int* d_lists = nullptr;
    MHM_CUDA_TRY(cudaMallocAsync((void**)&d_lists, lists.size() * sizeof(int), s));
    MHM_CUDA_TRY(cudaMemcpyAsync(d_lists, lists.data(), lists.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    const int thr = 256;
    mhm_status st = MHM_OK;
    // assembled saddle-point values, fronts zeroed and filled with the original entries
    k_fill_saddle<<<blocks_for(mesh->aug_nnz, thr), thr, 0, s>>>(mesh->aug_nnz, mesh->d_aug_src, A_vals, BK, P->vals);
    cudaMemsetAsync(P->fronts, 0, P->front_doubles * sizeof(double), s);
    cudaMemsetAsync(P->dinfo, 0, P->nodes.size() * sizeof(int), s);
    k_nd_assemble<<<blocks_for(mesh->aug_nnz, thr), thr, 0, s>>>(mesh->aug_nnz, P->dst, P->vals, P->fronts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "mhm_solve_global: assembly");
    size_t smem_max = 0;
    for (const NDNode& nd : P->nodes)
        if (!nd.big) smem_max = std::max(smem_max, (size_t)(nd.F * nd.k) * sizeof(double));
    if (!st && smem_max > 48 * 1024)
        e = cudaFuncSetAttribute(k_nd_factor_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (!st && e != cudaSuccess) st = cuda_fail(e, "mhm_solve_global: shared memory of the front kernel");
    // numeric factorisation, deepest level first
    for (int d = D - 1; d >= 0 && !st; --d) {
        const int n = (int)P->by_depth[d].size();
        for (int slot = 0; slot < 2; ++slot)
            k_nd_extend_add<<<n, thr, 0, s>>>(d_lists + list_off[d], slot, P->node_info, P->maps, P->fronts);
        if (small_n[d] > 0) {
            size_t sm = 0;
            for (int id : P->by_depth[d])
                if (!P->nodes[id].big) sm = std::max(sm, (size_t)(P->nodes[id].F * P->nodes[id].k) * sizeof(double));
            k_nd_factor_small<<<(unsigned)small_n[d], kNdThreads, sm, s>>>(d_lists + small_off[d], P->node_info,
                                                                          P->fronts, P->dinfo);
        }
        for (int id : P->by_depth[d]) {
            const NDNode& nd = P->nodes[id];
            if (!nd.big) continue;
            double* Fr = P->fronts + nd.front_off;
            // the own multipliers by the library routines, then the own u0 (the trailing
            // pivots, at most two) one at a time
            const int64_t F = nd.F, k = nd.k_lam, nu = F - k;
            k_nd_negate_pivots<<<blocks_for(k * k, thr), thr, 0, s>>>(Fr, F, k);
            if (cusolverDnDpotrf(P->dn, CUBLAS_FILL_MODE_LOWER, (int)k, Fr, (int)F, P->work, P->lwork, P->dinfo + id) !=
                CUSOLVER_STATUS_SUCCESS) {
                st = fail(MHM_ERR_CUDA, "mhm_solve_global: potrf");
                break;
            }
            if (nu > 0) {
                const double one = 1.0;
                if (cublasDtrsm(P->bl, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT,
                                (int)nu, (int)k, &one, Fr, (int)F, Fr + k, (int)F) != CUBLAS_STATUS_SUCCESS ||
                    cublasDsyrk(P->bl, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, (int)nu, (int)k, &one, Fr + k, (int)F, &one,
                                Fr + k + k * F, (int)F) != CUBLAS_STATUS_SUCCESS) {
                    st = fail(MHM_ERR_CUDA, "mhm_solve_global: trsm / syrk");
                    break;
                }
            }
            k_nd_to_ldlt<<<blocks_for(F * k, thr), thr, 0, s>>>(Fr, F, k);
            k_nd_to_ldlt_diag<<<blocks_for(k, thr), thr, 0, s>>>(Fr, F, k);
            for (int64_t piv = k; piv < nd.k; ++piv) {
                const int64_t rest = F - piv - 1;
                k_nd_pivot_update<<<(unsigned)std::min<int64_t>(4096, blocks_for(rest * rest, thr)), thr, 0, s>>>(Fr, F, piv);
                k_nd_pivot_scale<<<(unsigned)std::min<int64_t>(64, blocks_for(rest, thr)), thr, 0, s>>>(Fr, F, piv,
                                                                                                   P->dinfo + id);
            }
        }
        e = cudaGetLastError();
        if (!st && e != cudaSuccess) st = cuda_fail(e, "mhm_solve_global: factorisation");
    }
    // solve, then one step of refinement against the assembled system
    if (!st) {
        k_rhs_saddle<<<blocks_for(P->n, thr), thr, 0, s>>>(mesh->nlam, mesh->nK, E, FK, P->b);
        st = nd_solve(P, d_lists, list_off, P->x, s);
    }
    double* dx = nullptr;
    if (!st) {
        e = cudaMallocAsync((void**)&dx, P->n * sizeof(double), s);
        if (e != cudaSuccess) st = cuda_fail(e, "mhm_solve_global: cudaMallocAsync");
    }
    if (!st) {
        double* rhs = nullptr;
        e = cudaMallocAsync((void**)&rhs, P->n * sizeof(double), s);
        if (e == cudaSuccess) {
            k_rhs_saddle<<<blocks_for(P->n, thr), thr, 0, s>>>(mesh->nlam, mesh->nK, E, FK, rhs);
            k_nd_residual<<<blocks_for(P->n * 32, thr), thr, 0, s>>>(P->n, mesh->d_aug_rowptr, mesh->d_aug_cols, P->vals,
                                                                     P->x, rhs, P->b);
            st = nd_solve(P, d_lists, list_off, dx, s);
            if (!st) k_add_split<<<blocks_for(P->n, thr), thr, 0, s>>>(mesh->nlam, mesh->nK, P->x, dx, lambda, u0);
            cudaFreeAsync(rhs, s);
        } else {
            st = cuda_fail(e, "mhm_solve_global: cudaMallocAsync");
        }
    }
    if (dx) cudaFreeAsync(dx, s);
    cudaFreeAsync(d_lists, s);
    e = cudaGetLastError();
    if (!st && e != cudaSuccess) st = cuda_fail(e, "mhm_solve_global: solve");
    if (!st) {
        // a zero or non-finite pivot means a singular system: report it (synchronises)
        std::vector<int> bad(P->nodes.size());
        e = cudaMemcpyAsync(bad.data(), P->dinfo, bad.size() * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "mhm_solve_global: status");
        for (int v : bad)
            if (v != 0) return fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: singular saddle-point system (zero pivot)");
    }
    return st;
}
