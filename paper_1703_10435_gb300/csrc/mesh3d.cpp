// Host side of the three-dimensional mesh (splitProblem on the unit cube, Alg. 1;
// Sec. 5): coarse tetrahedra, faces, normals and signs, the multiplier numbering of
// Lambda_H^{m,0}, the lattice tables of the Freudenthal submesh, the face-load table
// and the skeleton CSR.  Conventions in mhm3d.h.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <map>
#include <string>

#include "mhm3d_internal.h"

namespace mhm3 {

namespace {

constexpr int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
constexpr int kEdges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

void legendre_and_derivative(int n, double x, double* p, double* dp) {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// lattice point (A, B, C) on local face a of the simplex {N >= A >= B >= C >= 0}
bool on_face(int a, const int* p, int N) {
    switch (a) {
        case 0: return p[0] == N;
        case 1: return p[0] == p[1];
        case 2: return p[1] == p[2];
        default: return p[2] == 0;
    }
}

}  // namespace

void gauss01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double p = 0, dp = 1;
        for (int it = 0; it < 100; ++it) {
            legendre_and_derivative(n, z, &p, &dp);
            const double dz = p / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre_and_derivative(n, z, &p, &dp);
        x[n - 1 - i] = 0.5 * (z + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

std::string build_mesh3d_host(mhm_mesh3d* m) {
    const int nc = m->desc.nc, P = m->desc.degree;
    const int n1 = nc + 1;
    m->N = 1 << m->desc.r;
    m->PN = P * m->N;
    m->nb = P == 1 ? 4 : 10;
    m->M = 1 << m->s;
    const int N = m->N, PN = m->PN, nb = m->nb, M = m->M, mm = m->desc.m;

    // ---- vertices
    auto corner = [&](int i, int j, int k) { return i + n1 * (j + n1 * k); };
    const int n_corner = n1 * n1 * n1;
    auto centre = [&](int i, int j, int k) { return n_corner + i + nc * (j + nc * k); };
    const int base0 = n_corner + nc * nc * nc, base1 = base0 + n1 * nc * nc, base2 = base1 + n1 * nc * nc;
    auto face_centre = [&](int d, const int* p) {
        if (d == 0) return base0 + p[0] + n1 * (p[1] + nc * p[2]);
        if (d == 1) return base1 + p[0] + nc * (p[1] + n1 * p[2]);
        return base2 + p[0] + nc * (p[1] + nc * p[2]);
    };
    m->nv = base2 + (int64_t)n1 * nc * nc;
    m->verts.assign(m->nv * 3, 0.0);
    for (int k = 0; k < n1; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i) {
                double* x = &m->verts[3 * corner(i, j, k)];
                x[0] = (double)i / nc, x[1] = (double)j / nc, x[2] = (double)k / nc;
            }
    for (int k = 0; k < nc; ++k)
        for (int j = 0; j < nc; ++j)
            for (int i = 0; i < nc; ++i) {
                double* x = &m->verts[3 * centre(i, j, k)];
                x[0] = (i + 0.5) / nc, x[1] = (j + 0.5) / nc, x[2] = (k + 0.5) / nc;
            }
    for (int d = 0; d < 3; ++d) {
        int hi[3] = {nc, nc, nc};
        hi[d] = n1;
        for (int k = 0; k < hi[2]; ++k)
            for (int j = 0; j < hi[1]; ++j)
                for (int i = 0; i < hi[0]; ++i) {
                    const int p[3] = {i, j, k};
                    double* x = &m->verts[3 * face_centre(d, p)];
                    for (int c = 0; c < 3; ++c) x[c] = (double)p[c] / nc + (c == d ? 0.0 : 0.5 / nc);
                }
    }

    // ---- tetrahedra: 24 per cube
    m->nK = 24LL * nc * nc * nc;
    m->tets.resize(m->nK * 4);
    int64_t K = 0;
    for (int ck = 0; ck < nc; ++ck)
        for (int cj = 0; cj < nc; ++cj)
            for (int ci = 0; ci < nc; ++ci) {
                const int c[3] = {ci, cj, ck};
                for (int d = 0; d < 3; ++d) {
                    int u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
                    for (int side = 0; side < 2; ++side) {
                        int p[3] = {c[0], c[1], c[2]};
                        p[d] += side;
                        const int fc = face_centre(d, p);
                        int corners[4];
                        const int duv[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
                        for (int q = 0; q < 4; ++q) {
                            int x[3] = {p[0], p[1], p[2]};
                            x[u] += duv[q][0];
                            x[v] += duv[q][1];
                            corners[q] = corner(x[0], x[1], x[2]);
                        }
                        for (int e = 0; e < 4; ++e, ++K) {
                            int32_t* t = &m->tets[4 * K];
                            t[0] = centre(ci, cj, ck), t[1] = fc, t[2] = corners[e], t[3] = corners[(e + 1) % 4];
                        }
                    }
                }
            }

    // ---- faces in order of first encounter, normals, signs, permutation codes
    std::map<std::array<int32_t, 3>, int32_t> key_to_face;
    m->tet_faces.resize(m->nK * 4);
    std::vector<int32_t> ka;   // per face: K0, a0, K1, a1
    for (K = 0; K < m->nK; ++K)
        for (int a = 0; a < 4; ++a) {
            std::array<int32_t, 3> key;
            for (int b = 0, i = 0; b < 4; ++b)
                if (b != a) key[i++] = m->tets[4 * K + b];
            std::sort(key.begin(), key.end());
            auto it = key_to_face.find(key);
            int32_t f;
            if (it == key_to_face.end()) {
                f = (int32_t)(m->faces.size() / 3);
                key_to_face.emplace(key, f);
                m->faces.insert(m->faces.end(), key.begin(), key.end());
                ka.insert(ka.end(), {(int32_t)K, a, -1, -1});
            } else {
                f = it->second;
                ka[4 * f + 2] = (int32_t)K;
                ka[4 * f + 3] = a;
            }
            m->tet_faces[4 * K + a] = f;
        }
    m->nf = (int64_t)m->faces.size() / 3;
    m->face_ka = ka;
    m->normals.resize(m->nf * 3);
    auto X = [&](int32_t v) { return &m->verts[3 * (int64_t)v]; };
    for (int64_t f = 0; f < m->nf; ++f) {
        const double *x0 = X(m->faces[3 * f]), *x1 = X(m->faces[3 * f + 1]), *x2 = X(m->faces[3 * f + 2]);
        double e1[3], e2[3], nn[3];
        for (int c = 0; c < 3; ++c) e1[c] = x1[c] - x0[c], e2[c] = x2[c] - x0[c];
        nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double len = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int c = 0; c < 3; ++c) nn[c] /= len;
        if (ka[4 * f + 2] < 0) {   // boundary: outward, away from the opposite vertex of its element
            const double* xo = X(m->tets[4 * ka[4 * f] + ka[4 * f + 1]]);
            double dot = 0;
            for (int c = 0; c < 3; ++c) dot += nn[c] * (x0[c] - xo[c]);
            if (dot < 0)
                for (int c = 0; c < 3; ++c) nn[c] = -nn[c];
        }
        for (int c = 0; c < 3; ++c) m->normals[3 * f + c] = nn[c];
    }
    m->signs.resize(m->nK * 4);
    m->perm.resize(m->nK * 4);
    m->geom.resize(m->nK * 12);
    for (K = 0; K < m->nK; ++K) {
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 3; ++c) m->geom[12 * K + 3 * b + c] = X(m->tets[4 * K + b])[c];
        for (int a = 0; a < 4; ++a) {
            const int32_t f = m->tet_faces[4 * K + a];
            const double *x0 = X(m->faces[3 * f]), *xo = X(m->tets[4 * K + a]);
            double dot = 0;
            for (int c = 0; c < 3; ++c) dot += m->normals[3 * f + c] * (x0[c] - xo[c]);
            m->signs[4 * K + a] = dot > 0 ? 1 : -1;
            // local face vertices in increasing local order; find the permutation that
            // lists them in the order of their sorted global ids
            int lf[3];
            for (int b = 0, i = 0; b < 4; ++b)
                if (b != a) lf[i++] = b;
            int code = -1;
            for (int p = 0; p < 6; ++p) {
                bool ok = true;
                for (int k = 0; k < 3; ++k) ok = ok && m->tets[4 * K + lf[kPerm[p][k]]] == m->faces[3 * f + k];
                if (ok) code = p;
            }
            if (code < 0) return "internal: face permutation not found";
            m->perm[4 * K + a] = (int8_t)code;
        }
    }
    m->nlam = m->nf * mm;
    m->NI = 4LL * mm;

    // ---- local lattice: DOFs, sub-tetrahedra (Freudenthal), classes
    std::vector<int32_t> index((size_t)(PN + 1) * (PN + 1) * (PN + 1), -1);
    auto lidx = [&](int A, int B, int C) -> int32_t& { return index[((size_t)C * (PN + 1) + B) * (PN + 1) + A]; };
    for (int C = 0; C <= PN; ++C)
        for (int B = C; B <= PN; ++B)
            for (int A = B; A <= PN; ++A) {
                lidx(A, B, C) = (int32_t)(m->nodes.size() / 3);
                m->nodes.insert(m->nodes.end(), {A, B, C});
            }
    m->n = (int64_t)m->nodes.size() / 3;
    auto inside = [&](const int* p) { return N >= p[0] && p[0] >= p[1] && p[1] >= p[2] && p[2] >= 0; };
    std::vector<std::array<int, 12>> sub_lat;
    for (int z3 = 0; z3 < N; ++z3)
        for (int z2 = 0; z2 < N; ++z2)
            for (int z1 = 0; z1 < N; ++z1)
                for (int pi = 0; pi < 6; ++pi) {
                    std::array<int, 12> T{};
                    T[0] = z1, T[1] = z2, T[2] = z3;
                    for (int s = 0; s < 3; ++s) {
                        for (int c = 0; c < 3; ++c) T[3 * (s + 1) + c] = T[3 * s + c];
                        T[3 * (s + 1) + kPerm[pi][s]] += 1;
                    }
                    bool in = true;
                    for (int v = 0; v < 4; ++v) in = in && inside(&T[3 * v]);
                    if (!in) continue;
                    sub_lat.push_back(T);
                    m->sub_cls.push_back((int8_t)pi);
                    m->sub_base.insert(m->sub_base.end(), {(int8_t)z1, (int8_t)z2, (int8_t)z3});
                    for (int v = 0; v < 4; ++v) m->sub_dofs.push_back(lidx(P * T[3 * v], P * T[3 * v + 1], P * T[3 * v + 2]));
                    if (P == 2)
                        for (const auto& e : kEdges)
                            m->sub_dofs.push_back(lidx(T[3 * e[0]] + T[3 * e[1]], T[3 * e[0] + 1] + T[3 * e[1] + 1],
                                                       T[3 * e[0] + 2] + T[3 * e[1] + 2]));
                }
    m->nsub = (int64_t)sub_lat.size();
    if (m->nsub != (int64_t)N * N * N) return "internal: Freudenthal refinement count";
    // incidence of the local DOFs: the slots t nb + a of the sub-tetrahedra that hold each
    // DOF, ascending (the kernels gather per DOF in this fixed order: no atomics)
    m->inc_off.assign(m->n + 1, 0);
    for (int32_t d : m->sub_dofs) ++m->inc_off[d + 1];
    for (int64_t w = 0; w < m->n; ++w) m->inc_off[w + 1] += m->inc_off[w];
    m->inc_ent.assign(m->sub_dofs.size(), 0);
    {
        std::vector<int32_t> fill(m->inc_off.begin(), m->inc_off.end() - 1);
        for (size_t slot = 0; slot < m->sub_dofs.size(); ++slot) m->inc_ent[fill[m->sub_dofs[slot]]++] = (int32_t)slot;
    }

    // ---- face-load table: for local face a and permutation code p, per subface q the
    // local DOFs that carry the face load of its fine triangles (P1: vertices, P2: edge
    // midpoints; each holds 1/3 of a fine triangle's area) with their multiplicity
    m->ftab_off.assign(24 * (mm + 1), 0);
    for (int a = 0; a < 4; ++a)
        for (int p = 0; p < 6; ++p) {
            int lf[3];
            for (int b = 0, i = 0; b < 4; ++b)
                if (b != a) lf[i++] = b;
            const int L1 = lf[kPerm[p][1]], L2 = lf[kPerm[p][2]];
            std::map<std::pair<int, int>, int> cnt;   // (q, node) -> count
            for (const auto& T : sub_lat)
                for (int omit = 0; omit < 4; ++omit) {
                    int tri[3], k = 0;
                    for (int v = 0; v < 4; ++v)
                        if (v != omit) tri[k++] = v;
                    bool on = true;
                    for (int v : tri) on = on && on_face(a, &T[3 * v], N);
                    if (!on) continue;
                    // barycentrics of the centroid times 3N, exact integers
                    int lam[4] = {0, 0, 0, 0};
                    for (int v : tri) {
                        const int* q = &T[3 * v];
                        lam[0] += N - q[0], lam[1] += q[0] - q[1], lam[2] += q[1] - q[2], lam[3] += q[2];
                    }
                    const int den = 3 * N;
                    const int Xs = M * lam[L1], Ys = M * lam[L2];
                    const int i = Xs / den, j = Ys / den;
                    const bool up = (Xs - i * den) + (Ys - j * den) < den;
                    const int row = j * (2 * M - j);
                    const int q = up ? row + i : row + (M - j) + i;
                    for (int u = 0; u < 3; ++u) {
                        int node;
                        if (P == 1) {
                            const int* x = &T[3 * tri[u]];
                            node = lidx(x[0], x[1], x[2]);
                        } else {
                            const int *x = &T[3 * tri[u]], *y = &T[3 * tri[(u + 1) % 3]];
                            node = lidx(x[0] + y[0], x[1] + y[1], x[2] + y[2]);
                        }
                        cnt[{q, node}] += 1;
                    }
                }
            const int base = (a * 6 + p) * (mm + 1);
            m->ftab_off[base] = (int32_t)m->ftab_node.size();
            for (int q = 0; q < mm; ++q) {
                for (const auto& kv : cnt)
                    if (kv.first.first == q) {
                        m->ftab_node.push_back((int16_t)kv.first.second);
                        m->ftab_cnt.push_back((int8_t)kv.second);
                    }
                m->ftab_off[base + q + 1] = (int32_t)m->ftab_node.size();
            }
        }

    // ---- reference quadrature (collapsed 4x4x4 Gauss rule) and basis values at its points
    double gx[4], gw[4];
    gauss01(4, gx, gw);
    m->quad.assign((size_t)kQuad * (4 + nb), 0.0);
    for (int i = 0, q = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 4; ++k, ++q) {
                const double a = gx[i], b = gx[j], c = gx[k];
                const double x = a, y = b * (1.0 - a), z = c * (1.0 - a) * (1.0 - b);
                m->quad[4 * q] = x, m->quad[4 * q + 1] = y, m->quad[4 * q + 2] = z;
                m->quad[4 * q + 3] = gw[i] * gw[j] * gw[k] * (1.0 - a) * (1.0 - a) * (1.0 - b);
                const double l[4] = {1.0 - x - y - z, x, y, z};
                double* phi = &m->quad[4 * kQuad + (size_t)q * nb];
                if (P == 1) {
                    for (int v = 0; v < 4; ++v) phi[v] = l[v];
                } else {
                    for (int v = 0; v < 4; ++v) phi[v] = l[v] * (2.0 * l[v] - 1.0);
                    for (int e = 0; e < 6; ++e) phi[4 + e] = 4.0 * l[kEdges[e][0]] * l[kEdges[e][1]];
                }
            }

    // ---- skeleton CSR: the rows of face f hold the columns of every face of the elements
    // at f (ascending); one neighbour block per (f, g)
    m->rowptr.assign(m->nlam + 1, 0);
    int64_t nnz = 0;
    for (int64_t f = 0; f < m->nf; ++f) {
        std::vector<int32_t> g;
        for (int side = 0; side < 2; ++side) {
            const int32_t Kx = ka[4 * f + 2 * side];
            if (Kx < 0) continue;
            for (int b = 0; b < 4; ++b) g.push_back(m->tet_faces[4 * (int64_t)Kx + b]);
        }
        std::sort(g.begin(), g.end());
        g.erase(std::unique(g.begin(), g.end()), g.end());
        for (size_t t = 0; t < g.size(); ++t) {
            Nbr3 nb3{};
            nb3.f = (int32_t)f, nb3.g = g[t], nb3.col_off = (int32_t)(t * mm);
            nb3.K0 = nb3.K1 = -1;
            for (int side = 0; side < 2; ++side) {
                const int32_t Kx = ka[4 * f + 2 * side];
                if (Kx < 0) continue;
                int bx = -1;
                for (int b = 0; b < 4; ++b)
                    if (m->tet_faces[4 * (int64_t)Kx + b] == g[t]) bx = b;
                if (bx < 0) continue;
                if (nb3.K0 < 0) nb3.K0 = Kx, nb3.a0 = ka[4 * f + 2 * side + 1], nb3.b0 = bx;
                else nb3.K1 = Kx, nb3.a1 = ka[4 * f + 2 * side + 1], nb3.b1 = bx;
            }
            if (nb3.K1 >= 0 && nb3.K1 < nb3.K0) {
                std::swap(nb3.K0, nb3.K1), std::swap(nb3.a0, nb3.a1), std::swap(nb3.b0, nb3.b1);
            }
            m->nbrs.push_back(nb3);
        }
        const int64_t rowlen = (int64_t)g.size() * mm;
        for (int q = 0; q < mm; ++q) {
            m->rowptr[f * mm + q] = (int32_t)nnz;
            nnz += rowlen;
            if (nnz > INT32_MAX) return "skeleton has more than 2^31 - 1 entries";
        }
    }
    m->rowptr[m->nlam] = (int32_t)nnz;
    m->nnz = nnz;
    m->cols.resize(nnz);
    for (const Nbr3& b : m->nbrs)
        for (int q = 0; q < mm; ++q)
            for (int q2 = 0; q2 < mm; ++q2) m->cols[m->rowptr[(int64_t)b.f * mm + q] + b.col_off + q2] = b.g * mm + q2;
    return "";
}

}  // namespace mhm3
