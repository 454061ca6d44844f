// reduceLocalProblems' gather (Alg. 1; Sec. 3, Eq. "mat_global"): the global
// skeleton matrix A_ij = sum_K (s psi_j, eta_i)_{dK} in CSR form and the
// right-hand side E_j = -sum_K (s psi_j, eta_f)_{dK} + (g, psi_j)_F.
//
// Every CSR entry is a gather of at most two per-K values: a block (e, f) with
// f != e belongs to the single K containing both faces; the diagonal block of an
// interior face sums its two K in ascending order.  The sum order is fixed, so
// the result is deterministic without atomics.  The kernel is bound by HBM
// traffic: it reads each per-K entry once and writes each CSR value once.
#include <cuda_runtime.h>

#include "mhm_internal.h"

namespace mhm {

namespace {

struct SkelArgs {
    const double* AK;
    const double* EK;
    const int32_t* rowptr;
    const int64_t* lam_off;   // first multiplier of each face
    const int32_t* lam_face;  // face of each multiplier
    const int32_t* nbr_ptr;
    const FaceNbr* nbrs;
    const int32_t* face_K;
    const int32_t* face_v;
    const int32_t* tri_f;
    const double* vxy;
    const double* gauss_x;
    const double* gauss_w;
    int64_t nlam;
    int dpf, NI, M, L;
    int has_g;
    double gc[6];
    double* A;
    double* E;
};

// One warp per skeleton row j = (face e, local dof u); lanes over the row's entries, which
// run over the neighbour faces f of e (m(l_f+1) columns each, from FaceNbr::col_off).  Local
// slot u of a face sits at a dpf + u in the per-K blocks (stride dpf = m(l_max+1)).
__global__ void k_skeleton_A(const SkelArgs g) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= g.nlam) return;
    const int e = g.lam_face[j], u = (int)(j - g.lam_off[e]);
    const int nb0 = g.nbr_ptr[e], nb1 = g.nbr_ptr[e + 1];
    const int len = g.rowptr[j + 1] - g.rowptr[j];
    const int64_t out = g.rowptr[j];
    const int64_t nn = (int64_t)g.NI * g.NI;
    for (int c = lane; c < len; c += 32) {
        int blk = nb0;
        while (blk + 1 < nb1 && g.nbrs[blk + 1].col_off <= c) ++blk;   // at most 5 blocks
        const FaceNbr nb = g.nbrs[blk];
        const int v = c - nb.col_off;
        double val = g.AK[nb.K0 * nn + (int64_t)(nb.a0 * g.dpf + u) * g.NI + nb.b0 * g.dpf + v];
        if (nb.K1 >= 0) val += g.AK[nb.K1 * nn + (int64_t)(nb.a1 * g.dpf + u) * g.NI + nb.b1 * g.dpf + v];
        g.A[out + c] = val;
    }
}

__device__ __forceinline__ double legendre_dev(int p, double xi) {
    double a = 1.0, b = xi;
    if (p == 0) return 1.0;
    for (int k = 1; k < p; ++k) {
        const double c = ((2 * k + 1) * xi * b - k * a) / (k + 1);
        a = b;
        b = c;
    }
    return b;
}

// E_j: sum of the (one or two) per-K values in ascending K, plus the Dirichlet term.
__global__ void k_skeleton_E(const SkelArgs g) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.nlam) return;
    const int e = g.lam_face[j], u = (int)(j - g.lam_off[e]);
    double val = 0.0;
    for (int side = 0; side < 2; ++side) {
        const int K = g.face_K[2 * e + side];
        if (K < 0) continue;
        int a = 0;
        while (g.tri_f[3 * K + a] != e) ++a;
        val += g.EK[(int64_t)K * g.NI + a * g.dpf + u];
    }
    if (g.has_g && g.face_K[2 * e + 1] < 0) {
        // (g, psi_{q,p})_F on subface q, Gauss-Legendre exact for degree l + 2 (l_e + 1 =
        // the face's multipliers / m)
        const int le1 = (int)(g.lam_off[e + 1] - g.lam_off[e]) / g.M;
        const int q = u / le1, p = u - q * le1;
        const int n = min(kMaxGauss, g.L / 2 + 3);
        const double* gx = g.gauss_x + (n - 1) * kMaxGauss;
        const double* gw = g.gauss_w + (n - 1) * kMaxGauss;
        const double x0 = g.vxy[2 * g.face_v[2 * e]], y0 = g.vxy[2 * g.face_v[2 * e] + 1];
        const double x1 = g.vxy[2 * g.face_v[2 * e + 1]], y1 = g.vxy[2 * g.face_v[2 * e + 1] + 1];
        const double len = sqrt((x1 - x0) * (x1 - x0) + (y1 - y0) * (y1 - y0));
        double s = 0.0;
        for (int k = 0; k < n; ++k) {
            const double tau = (q + gx[k]) / g.M;
            const double x = x0 + tau * (x1 - x0), y = y0 + tau * (y1 - y0);
            const double gv = g.gc[0] + g.gc[1] * x + g.gc[2] * y + g.gc[3] * x * x + g.gc[4] * x * y + g.gc[5] * y * y;
            s += gw[k] * gv * legendre_dev(p, 2.0 * gx[k] - 1.0);
        }
        val += s * len / g.M;
    }
    g.E[j] = val;
}

}  // namespace

mhm_status launch_skeleton(const mhm_mesh* mesh, const double* AK, const double* EK, const mhm_dirichlet* gd,
                           double* A_vals, double* E, cudaStream_t stream) {
    SkelArgs g;
    g.AK = AK;
    g.EK = EK;
    g.rowptr = mesh->d_csr_rowptr;
    g.lam_off = mesh->d_lam_off;
    g.lam_face = mesh->d_lam_face;
    g.nbr_ptr = mesh->d_nbr_ptr;
    g.nbrs = mesh->d_nbrs;
    g.face_K = mesh->d_face_K;
    g.face_v = mesh->d_face_v;
    g.tri_f = mesh->d_tri_f;
    g.vxy = mesh->d_vxy;
    g.gauss_x = mesh->d_gauss_x;
    g.gauss_w = mesh->d_gauss_w;
    g.nlam = mesh->nlam;
    g.dpf = mesh->dpf;
    g.NI = (int)mesh->NI;
    g.M = mesh->desc.m;
    g.L = mesh->desc.l;
    g.has_g = gd != nullptr;
    for (int i = 0; i < 6; ++i) g.gc[i] = gd ? gd->c[i] : 0.0;
    g.A = A_vals;
    g.E = E;
    const int threads = 256;
    const int64_t warps = mesh->nlam;
    k_skeleton_A<<<(unsigned)((warps * 32 + threads - 1) / threads), threads, 0, stream>>>(g);
    MHM_CUDA_TRY(cudaGetLastError());
    k_skeleton_E<<<(unsigned)((mesh->nlam + threads - 1) / threads), threads, 0, stream>>>(g);
    MHM_CUDA_TRY(cudaGetLastError());
    return MHM_OK;
}

}  // namespace mhm
