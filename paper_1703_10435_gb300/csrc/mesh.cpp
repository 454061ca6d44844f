// splitProblem (Alg. 1, first step): the coarse mesh T_H, its skeleton, face
// normals and signs, the multiplier space Lambda_H^{m,l} and the tables the
// kernels read, built on the host and uploaded once.
#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <utility>

#include "mhm_internal.h"

namespace {

// Legendre P_n and its derivative at x by the three-term recurrence.
void legendre_pd(int n, double x, double* p, double* dp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// n-point Gauss-Legendre rule on [0,1]: roots of P_n by Newton from the
// Chebyshev-like initial guesses cos(pi (i + 3/4) / (n + 1/2)).
void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double p = 0, dp = 1;
        for (int it = 0; it < 100; ++it) {
            legendre_pd(n, z, &p, &dp);
            double dz = p / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre_pd(n, z, &p, &dp);
        x[n - 1 - i] = 0.5 * (z + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2) P'^2) on [-1,1], halved
    }
}

double legendre_p(int p, double xi) {
    if (p == 0) return 1.0;
    double a = 1.0, b = xi;
    for (int k = 1; k < p; ++k) {
        double c = ((2 * k + 1) * xi * b - k * a) / (k + 1);
        a = b;
        b = c;
    }
    return b;
}

// 1-D Lagrange basis of degree P on one fine segment, local coordinate t in [0,1].
void lagrange1d(int P, double t, double* v) {
    if (P == 1) {
        v[0] = 1.0 - t;
        v[1] = t;
    } else {
        v[0] = 2.0 * (t - 0.5) * (t - 1.0);
        v[1] = -4.0 * t * (t - 1.0);
        v[2] = 2.0 * t * (t - 0.5);
    }
}

template <typename T>
mhm_status upload(const std::vector<T>& h, T** d) {
    if (h.empty()) { *d = nullptr; return MHM_OK; }
    cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
    if (e == cudaErrorMemoryAllocation) return mhm::fail(MHM_ERR_OOM, "cudaMalloc failed for mesh tables");
    if (e != cudaSuccess) return mhm::cuda_fail(e, "cudaMalloc");
    e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mhm::cuda_fail(e, "cudaMemcpy");
    return MHM_OK;
}

}  // namespace

void free_mesh_device(mhm_mesh* m) {
    void* ptrs[] = {m->d_geom, m->d_sign, m->d_rev, m->d_btab, m->d_btab_sum, m->d_gauss_x,
                    m->d_gauss_w, m->d_face_v, m->d_face_K, m->d_tri_f, m->d_vxy, m->d_lam_off,
                    m->d_csr_rowptr, m->d_nbr_ptr, m->d_nbrs, m->d_aug_rowptr, m->d_aug_cols, m->d_aug_src, m->d_k_lambda,
                    m->d_lam_face, m->d_lface};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (m->d_kap_off) cudaFree(m->d_kap_off);
    if (m->d_nod_off) cudaFree(m->d_nod_off);
    if (m->d_sword) cudaFree(m->d_sword);
    m->d_sword = nullptr;
    for (mhm::Level& lv : m->levels) {
        if (lv.d_K) cudaFree(lv.d_K);
        if (lv.d_btab) cudaFree(lv.d_btab);
        lv.d_K = nullptr;
        lv.d_btab = nullptr;
        if (lv.fstream) cudaStreamDestroy(lv.fstream);
        for (cudaEvent_t e : {lv.fstart, lv.fdone[0], lv.fdone[1], lv.mdone[0], lv.mdone[1]})
            if (e) cudaEventDestroy(e);
    }
}

// Face-load table of one level: btab[jf][k] = int_0^1 psi_jf(tau) phi_k(tau) dtau, phi_k
// the 1-D Lagrange basis of degree P on N segments; Gauss pieces split at fine nodes and
// subfaces; btab_sum[jf] = int_0^1 psi_jf.
static void face_load_table(int P, int N, int M, int L, const std::vector<double>& gauss_x,
                            const std::vector<double>& gauss_w, std::vector<double>& btab,
                            std::vector<double>& btab_sum) {
    const int PN = P * N, dpf = M * (L + 1);
    btab.assign((size_t)dpf * (PN + 1), 0.0);
    btab_sum.assign(dpf, 0.0);
    std::vector<double> cuts;
    for (int k = 0; k <= N; ++k) cuts.push_back((double)k / N);
    for (int q = 1; q < M; ++q) cuts.push_back((double)q / M);
    std::sort(cuts.begin(), cuts.end());
    const int ng = (P + L + 2) / 2 + 1;
    const double* gx = &gauss_x[(ng - 1) * mhm::kMaxGauss];
    const double* gw = &gauss_w[(ng - 1) * mhm::kMaxGauss];
    for (size_t c = 0; c + 1 < cuts.size(); ++c) {
        double al = cuts[c], be = cuts[c + 1];
        if (be - al < 1e-15) continue;
        double mid = 0.5 * (al + be);
        int seg = std::min(N - 1, (int)std::floor(mid * N));
        int q = std::min(M - 1, (int)std::floor(mid * M));
        for (int g = 0; g < ng; ++g) {
            double tau = al + (be - al) * gx[g], w = (be - al) * gw[g];
            double v[3];
            lagrange1d(P, tau * N - seg, v);
            double xi = 2.0 * (tau * M - q) - 1.0;
            for (int p = 0; p <= L; ++p) {
                double psi = legendre_p(p, xi);
                int jf = q * (L + 1) + p;
                for (int b = 0; b <= P; ++b) btab[(size_t)jf * (PN + 1) + P * seg + b] += w * psi * v[b];
                btab_sum[jf] += w * psi;
            }
        }
    }
}

extern "C" mhm_status mhm_create_mesh(const mhm_mesh_desc* desc, int32_t device, mhm_mesh** out) {
    if (!desc || !out) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: NULL argument");
    *out = nullptr;
    const mhm_mesh_desc d = *desc;
    if (d.nx < 1 || d.ny < 1 || (int64_t)d.nx * d.ny > (1 << 26))
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: nx, ny out of range");
    if (d.r < 0 || d.r > 7) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: r must be in 0..7");
    int r_top = d.r;   // the finest level (sizes reported per K are of this level)
    if (d.r_per_K) {
        r_top = 0;
        for (int64_t K = 0; K < 2LL * d.nx * d.ny; ++K) {
            if (d.r_per_K[K] < 0 || d.r_per_K[K] > 7)
                return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: every r_per_K must be in 0..7");
            r_top = std::max(r_top, (int)d.r_per_K[K]);
        }
    }
    if (d.degree != 1 && d.degree != 2) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: degree must be 1 or 2");
    const int64_t n_faces = (int64_t)d.nx * (d.ny + 1) + (int64_t)d.ny * (d.nx + 1) + (int64_t)d.nx * d.ny;
    int l_max = d.l;
    if (d.l_per_face) {
        l_max = 0;
        for (int64_t e = 0; e < n_faces; ++e) {
            if (d.l_per_face[e] < 0)
                return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: every l_per_face must be >= 0");
            l_max = std::max(l_max, (int)d.l_per_face[e]);
        }
    }
    if (d.m < 1 || l_max < 0 || d.m * (l_max + 1) > mhm::kMaxFaceDofs)
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: m >= 1, l >= 0 and m(l+1) <= 16 required");
    // device < 0 builds the host tables only (queries work, compute calls return UNSUPPORTED).
    if (device >= 0) {
        if (!mhm::device_supported(device))
            return mhm::fail(MHM_ERR_UNSUPPORTED, "mhm_create_mesh: device is not an sm_103 GPU");
        cudaError_t ce = cudaSetDevice(device);
        if (ce != cudaSuccess) return mhm::cuda_fail(ce, "cudaSetDevice");
    }

    mhm_mesh* m = new mhm_mesh();
    m->device = device;
    m->desc = d;
    m->desc.r_per_K = nullptr;   // the caller's arrays are read here only
    m->desc.l_per_face = nullptr;
    m->desc.l = l_max;           // from here on: the largest face degree
    const int nx = d.nx, ny = d.ny;
    m->N = 1 << r_top;
    m->PN = d.degree * m->N;
    m->dpf = d.m * (l_max + 1);
    m->nv = (int64_t)(nx + 1) * (ny + 1);
    m->nK = 2LL * nx * ny;
    m->nfine = (int64_t)m->N * m->N;
    m->nloc = (int64_t)(m->PN + 1) * (m->PN + 2) / 2;
    m->NI = 3LL * m->dpf;

    // vertices and triangles
    m->vxy.resize(m->nv * 2);
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            m->vxy[2 * (j * (nx + 1) + i)] = (double)i / nx;
            m->vxy[2 * (j * (nx + 1) + i) + 1] = (double)j / ny;
        }
    auto vid = [nx](int i, int j) { return j * (nx + 1) + i; };
    m->tri_v.resize(m->nK * 3);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int64_t K = 2LL * (j * nx + i);
            int32_t* t = &m->tri_v[3 * K];
            t[0] = vid(i, j); t[1] = vid(i + 1, j); t[2] = vid(i + 1, j + 1);
            t[3] = vid(i, j); t[4] = vid(i + 1, j + 1); t[5] = vid(i, j + 1);
        }

    // faces in order of first encounter
    std::map<std::pair<int32_t, int32_t>, int32_t> key;
    m->tri_f.resize(m->nK * 3);
    for (int64_t K = 0; K < m->nK; ++K)
        for (int a = 0; a < 3; ++a) {
            int32_t p = m->tri_v[3 * K + (a + 1) % 3], q = m->tri_v[3 * K + (a + 2) % 3];
            auto k = std::make_pair(std::min(p, q), std::max(p, q));
            auto it = key.find(k);
            int32_t e;
            if (it == key.end()) {
                e = (int32_t)m->face_v.size() / 2;
                key.emplace(k, e);
                m->face_v.push_back(k.first);
                m->face_v.push_back(k.second);
                m->face_K.push_back((int32_t)K);
                m->face_K.push_back(-1);
            } else {
                e = it->second;
                m->face_K[2 * e + 1] = (int32_t)K;
            }
            m->tri_f[3 * K + a] = e;
        }
    m->ne = (int64_t)m->face_v.size() / 2;

    // normals, signs, orientation flags
    m->normals.resize(m->ne * 2);
    auto outward = [&](int64_t K, int a, double* n) {
        const double* P = &m->vxy[2 * m->tri_v[3 * K + (a + 1) % 3]];
        const double* Q = &m->vxy[2 * m->tri_v[3 * K + (a + 2) % 3]];
        double dx = Q[0] - P[0], dy = Q[1] - P[1], L = std::sqrt(dx * dx + dy * dy);
        n[0] = dy / L;
        n[1] = -dx / L;
    };
    for (int64_t e = 0; e < m->ne; ++e) {
        if (m->face_K[2 * e + 1] < 0) {
            int64_t K = m->face_K[2 * e];
            int a = 0;
            while (m->tri_f[3 * K + a] != e) ++a;
            outward(K, a, &m->normals[2 * e]);
        } else {
            const double* A = &m->vxy[2 * m->face_v[2 * e]];
            const double* B = &m->vxy[2 * m->face_v[2 * e + 1]];
            double tx = B[0] - A[0], ty = B[1] - A[1], L = std::sqrt(tx * tx + ty * ty);
            m->normals[2 * e] = ty / L;
            m->normals[2 * e + 1] = -tx / L;
        }
    }
    m->tri_s.resize(m->nK * 3);
    m->tri_rev.resize(m->nK * 3);
    for (int64_t K = 0; K < m->nK; ++K)
        for (int a = 0; a < 3; ++a) {
            double n[2];
            outward(K, a, n);
            int32_t e = m->tri_f[3 * K + a];
            double s = n[0] * m->normals[2 * e] + n[1] * m->normals[2 * e + 1];
            m->tri_s[3 * K + a] = s > 0 ? 1 : -1;
            m->tri_rev[3 * K + a] = m->tri_v[3 * K + (a + 1) % 3] > m->tri_v[3 * K + (a + 2) % 3] ? 1 : 0;
        }

    // multiplier numbering: face e carries m(l_e+1) multipliers; local face a of K keeps the
    // slots [a dpf, a dpf + m(l_a+1)) of the stride dpf = m(l_max+1), the rest unused (-1)
    if (m->ne != n_faces) {
        delete m;
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: internal face count mismatch");
    }
    m->face_l.assign(m->ne, (int8_t)l_max);
    if (d.l_per_face) m->face_l.assign(d.l_per_face, d.l_per_face + m->ne);
    auto dofs = [&](int64_t e) { return (int64_t)d.m * (m->face_l[e] + 1); };
    m->lam_off.resize(m->ne + 1);
    m->lam_off[0] = 0;
    for (int64_t e = 0; e < m->ne; ++e) m->lam_off[e + 1] = m->lam_off[e] + dofs(e);
    m->nlam = m->lam_off[m->ne];
    m->lam_face.resize(m->nlam);
    for (int64_t e = 0; e < m->ne; ++e)
        for (int64_t j = m->lam_off[e]; j < m->lam_off[e + 1]; ++j) m->lam_face[j] = (int32_t)e;
    bool uniform_l = true;
    for (int64_t e = 0; e < m->ne; ++e) uniform_l = uniform_l && m->face_l[e] == l_max;
    if (!uniform_l) {
        m->tri_l.resize(m->nK * 3);
        for (int64_t K = 0; K < 3 * m->nK; ++K) m->tri_l[K] = m->face_l[m->tri_f[K]];
    }
    m->k_lambda.resize(m->nK * m->NI);
    for (int64_t K = 0; K < m->nK; ++K)
        for (int a = 0; a < 3; ++a) {
            const int64_t e = m->tri_f[3 * K + a];
            for (int u = 0; u < m->dpf; ++u)
                m->k_lambda[K * m->NI + a * m->dpf + u] = u < dofs(e) ? (int32_t)(m->lam_off[e] + u) : -1;
        }

    // skeleton pattern: face e's rows couple with every face of its (one or two) K
    m->nbr_ptr.assign(m->ne + 1, 0);
    for (int64_t e = 0; e < m->ne; ++e) {
        std::map<int32_t, mhm::FaceNbr> blocks;
        for (int side = 0; side < 2; ++side) {
            int32_t K = m->face_K[2 * e + side];
            if (K < 0) continue;
            int ae = 0;
            while (m->tri_f[3 * K + ae] != e) ++ae;
            for (int b = 0; b < 3; ++b) {
                int32_t f = m->tri_f[3 * K + b];
                auto it = blocks.find(f);
                if (it == blocks.end()) {
                    mhm::FaceNbr nb{f, 0, K, ae, b, -1, 0, 0};
                    blocks.emplace(f, nb);
                } else {  // f == e on an interior face: second K, larger id
                    it->second.K1 = K;
                    it->second.a1 = ae;
                    it->second.b1 = b;
                }
            }
        }
        int32_t off = 0;
        for (auto& kv : blocks) {
            kv.second.col_off = off;
            off += (int32_t)dofs(kv.second.f);
            m->nbrs.push_back(kv.second);
        }
        m->nbr_ptr[e + 1] = (int32_t)m->nbrs.size();
    }
    // the skeleton CSR and the saddle-point CSR index their entries in int32 (as do the
    // sparse library calls of the global solve): refuse meshes beyond that
    {
        int64_t nnz = 0, bt = 0;
        for (int64_t e = 0; e < m->ne; ++e) {
            int64_t len = 0;
            for (int b = m->nbr_ptr[e]; b < m->nbr_ptr[e + 1]; ++b) len += dofs(m->nbrs[b].f);
            nnz += dofs(e) * len;
            bt += dofs(e) * (m->face_K[2 * e + 1] >= 0 ? 2 : 1);
        }
        m->sys_count = nnz + 2 * bt;
        if (nnz + 2 * bt > (int64_t)INT32_MAX) {
            delete m;
            return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_create_mesh: skeleton system beyond 2^31 entries (mesh too large)");
        }
    }
    m->csr_rowptr.assign(m->nlam + 1, 0);
    for (int64_t e = 0; e < m->ne; ++e) {
        int32_t len = 0;
        for (int b = m->nbr_ptr[e]; b < m->nbr_ptr[e + 1]; ++b) len += (int32_t)dofs(m->nbrs[b].f);
        for (int u = 0; u < dofs(e); ++u) {
            int64_t j = m->lam_off[e] + u;
            m->csr_rowptr[j + 1] = m->csr_rowptr[j] + len;
            for (int b = m->nbr_ptr[e]; b < m->nbr_ptr[e + 1]; ++b)
                for (int v = 0; v < dofs(m->nbrs[b].f); ++v)
                    m->csr_cols.push_back((int32_t)(m->lam_off[m->nbrs[b].f] + v));
        }
    }
    m->nnz = (int64_t)m->csr_cols.size();

    // saddle-point pattern: rows of A followed by the columns L + K of the (one or two)
    // K holding the row's face (B^T); then one row per K with its multipliers (B),
    // columns sorted ascending
    {
        const int64_t L = m->nlam;
        m->aug_rowptr.assign(L + m->nK + 1, 0);
        for (int64_t j = 0; j < L; ++j) {
            const int64_t e = m->lam_face[j], u = j - m->lam_off[e];
            for (int32_t t = m->csr_rowptr[j]; t < m->csr_rowptr[j + 1]; ++t) {
                m->aug_cols.push_back(m->csr_cols[t]);
                m->aug_src.push_back(t);
            }
            for (int side = 0; side < 2; ++side) {
                const int32_t K = m->face_K[2 * e + side];
                if (K < 0) continue;
                int a = 0;
                while (m->tri_f[3 * K + a] != e) ++a;
                m->aug_cols.push_back((int32_t)(L + K));
                m->aug_src.push_back(-((int64_t)K * m->NI + a * m->dpf + u) - 1);
            }
            m->aug_rowptr[j + 1] = (int32_t)m->aug_cols.size();
        }
        for (int64_t K = 0; K < m->nK; ++K) {
            std::vector<std::pair<int32_t, int64_t>> row;
            for (int64_t i = 0; i < m->NI; ++i)
                if (m->k_lambda[K * m->NI + i] >= 0) row.emplace_back(m->k_lambda[K * m->NI + i], -(K * m->NI + i) - 1);
            std::sort(row.begin(), row.end());
            for (auto& pr : row) {
                m->aug_cols.push_back(pr.first);
                m->aug_src.push_back(pr.second);
            }
            m->aug_rowptr[L + K + 1] = (int32_t)m->aug_cols.size();
        }
        m->aug_nnz = (int64_t)m->aug_cols.size();
    }

    // Gauss-Legendre tables, n = 1..kMaxGauss
    m->gauss_x.assign(mhm::kMaxGauss * mhm::kMaxGauss, 0.0);
    m->gauss_w.assign(mhm::kMaxGauss * mhm::kMaxGauss, 0.0);
    for (int n = 1; n <= mhm::kMaxGauss; ++n)
        gauss_legendre01(n, &m->gauss_x[(n - 1) * mhm::kMaxGauss], &m->gauss_w[(n - 1) * mhm::kMaxGauss]);

    // face-load table of the mesh's (finest) level, and the levels
    // (rows q (l_max+1) + p: a face of lower degree uses the rows p <= l_e of each subface)
    face_load_table(d.degree, m->N, d.m, l_max, m->gauss_x, m->gauss_w, m->btab, m->btab_sum);
    if (!d.r_per_K) {
        mhm::Level lv;
        lv.r = d.r;
        lv.N = m->N;
        lv.PN = m->PN;
        lv.nK = m->nK;
        lv.nfine = m->nfine;
        lv.nloc = m->nloc;
        m->levels.push_back(lv);
    } else {
        m->per_k_levels = true;
        m->r_of_K.assign(d.r_per_K, d.r_per_K + m->nK);
        m->kap_off.assign(m->nK + 1, 0);
        m->nod_off.assign(m->nK + 1, 0);
        for (int64_t K = 0; K < m->nK; ++K) {
            const int64_t N = 1LL << m->r_of_K[K], PN = d.degree * N;
            m->kap_off[K + 1] = m->kap_off[K] + N * N;
            m->nod_off[K + 1] = m->nod_off[K] + (PN + 1) * (PN + 2) / 2;
        }
        for (int r = 0; r <= 7; ++r) {
            mhm::Level lv;
            lv.r = r;
            lv.N = 1 << r;
            lv.PN = d.degree * lv.N;
            lv.nfine = (int64_t)lv.N * lv.N;
            lv.nloc = (int64_t)(lv.PN + 1) * (lv.PN + 2) / 2;
            for (int64_t K = 0; K < m->nK; ++K)
                if (m->r_of_K[K] == r) lv.K.push_back((int32_t)K);
            lv.nK = (int64_t)lv.K.size();
            if (lv.nK == 0) continue;
            std::vector<double> bsum;
            face_load_table(d.degree, lv.N, d.m, l_max, m->gauss_x, m->gauss_w, lv.btab, bsum);
            m->levels.push_back(std::move(lv));
        }
    }

    // per-K geometry
    std::vector<double> geom(m->nK * 6);
    for (int64_t K = 0; K < m->nK; ++K)
        for (int a = 0; a < 3; ++a) {
            geom[6 * K + 2 * a] = m->vxy[2 * m->tri_v[3 * K + a]];
            geom[6 * K + 2 * a + 1] = m->vxy[2 * m->tri_v[3 * K + a] + 1];
        }

    if (device < 0) {
        *out = m;
        return MHM_OK;
    }
    mhm_status st = MHM_OK;
    if (!st) st = upload(geom, &m->d_geom);
    if (!st) st = upload(m->tri_s, &m->d_sign);
    if (!st) st = upload(m->tri_rev, &m->d_rev);
    if (!st) st = upload(m->btab, &m->d_btab);
    if (!st) st = upload(m->btab_sum, &m->d_btab_sum);
    if (!st) st = upload(m->gauss_x, &m->d_gauss_x);
    if (!st) st = upload(m->gauss_w, &m->d_gauss_w);
    if (!st) st = upload(m->face_v, &m->d_face_v);
    if (!st) st = upload(m->face_K, &m->d_face_K);
    if (!st) st = upload(m->tri_f, &m->d_tri_f);
    if (!st) st = upload(m->vxy, &m->d_vxy);
    if (!st) st = upload(m->lam_off, &m->d_lam_off);
    if (!st) st = upload(m->csr_rowptr, &m->d_csr_rowptr);
    if (!st) st = upload(m->nbr_ptr, &m->d_nbr_ptr);
    if (!st) st = upload(m->nbrs, &m->d_nbrs);
    if (!st) st = upload(m->aug_rowptr, &m->d_aug_rowptr);
    if (!st) st = upload(m->aug_cols, &m->d_aug_cols);
    if (!st) st = upload(m->aug_src, &m->d_aug_src);
    if (!st) st = upload(m->k_lambda, &m->d_k_lambda);
    if (!st) st = upload(m->lam_face, &m->d_lam_face);
    if (!st) st = upload(m->tri_l, &m->d_lface);
    if (!st) st = upload(std::vector<uint32_t>{0u}, &m->d_sword);
    if (m->per_k_levels) {
        if (!st) st = upload(m->kap_off, &m->d_kap_off);
        if (!st) st = upload(m->nod_off, &m->d_nod_off);
        for (mhm::Level& lv : m->levels) {
            if (!st) st = upload(lv.K, &lv.d_K);
            if (!st) st = upload(lv.btab, &lv.d_btab);
        }
    }
    if (st) {
        free_mesh_device(m);
        delete m;
        return st;
    }
    *out = m;
    return MHM_OK;
}

extern "C" void mhm_destroy_mesh(mhm_mesh* m) {
    if (!m) return;
    if (m->device < 0) {
        delete m;
        return;
    }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m->device);
    free_mesh_device(m);
    mhm::free_nd_plan(m->nd);
    m->nd = nullptr;
    for (cudaEvent_t e : m->tev) cudaEventDestroy(e);
    for (cudaStream_t ss : m->side) cudaStreamDestroy(ss);
    for (cudaEvent_t e : m->side_done) cudaEventDestroy(e);
    if (m->fork_ev) cudaEventDestroy(m->fork_ev);
    if (m->wave_copy) cudaStreamDestroy(m->wave_copy);
    for (cudaEvent_t e : {m->wave_start, m->wave_copied[0], m->wave_copied[1], m->wave_solved[0], m->wave_solved[1]})
        if (e) cudaEventDestroy(e);
    cudaSetDevice(cur);
    delete m;
}

template <typename T>
static mhm_status copy_out(const std::vector<T>& v, void* out, size_t bytes) {
    if (bytes < v.size() * sizeof(T)) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_mesh_query: buffer too small");
    std::copy(v.begin(), v.end(), (T*)out);
    return MHM_OK;
}

extern "C" mhm_status mhm_mesh_query(const mhm_mesh* m, int32_t what, void* out, size_t bytes) {
    if (!m || !out) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_mesh_query: NULL argument");
    switch (what) {
        case MHM_Q_SIZES: {
            std::vector<int64_t> s = {m->nK, m->ne, m->nv, m->nlam, m->nfine, m->nloc, m->NI, m->nnz};
            return copy_out(s, out, bytes);
        }
        case MHM_Q_TRI_VERTS: return copy_out(m->tri_v, out, bytes);
        case MHM_Q_TRI_FACES: return copy_out(m->tri_f, out, bytes);
        case MHM_Q_TRI_SIGNS: return copy_out(m->tri_s, out, bytes);
        case MHM_Q_FACE_VERTS: return copy_out(m->face_v, out, bytes);
        case MHM_Q_LAMBDA_OFFSET: return copy_out(m->lam_off, out, bytes);
        case MHM_Q_K_LAMBDA: return copy_out(m->k_lambda, out, bytes);
        case MHM_Q_CSR_ROWPTR: return copy_out(m->csr_rowptr, out, bytes);
        case MHM_Q_CSR_COLS: return copy_out(m->csr_cols, out, bytes);
        case MHM_Q_VERTEX_XY: return copy_out(m->vxy, out, bytes);
        case MHM_Q_FACE_NORMALS: return copy_out(m->normals, out, bytes);
        case MHM_Q_FACE_DEGREE: return copy_out(m->face_l, out, bytes);
        case MHM_Q_SYSTEM_NNZ: {
            const std::vector<int64_t> v{m->sys_count, m->aug_nnz};
            return copy_out(v, out, bytes);
        }
        case MHM_Q_R_OF_K: {
            if (m->per_k_levels) return copy_out(m->r_of_K, out, bytes);
            return copy_out(std::vector<int8_t>(m->nK, (int8_t)m->desc.r), out, bytes);
        }
        case MHM_Q_KAPPA_OFFSET:
        case MHM_Q_NODAL_OFFSET: {
            if (m->per_k_levels) return copy_out(what == MHM_Q_KAPPA_OFFSET ? m->kap_off : m->nod_off, out, bytes);
            std::vector<int64_t> o(m->nK + 1);
            const int64_t per = what == MHM_Q_KAPPA_OFFSET ? m->nfine : m->nloc;
            for (int64_t K = 0; K <= m->nK; ++K) o[K] = K * per;
            return copy_out(o, out, bytes);
        }
        default: return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_mesh_query: unknown query");
    }
}
