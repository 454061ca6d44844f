// Autotuner of the launch shapes of the mixed-precision local solves (no counterpart in the
// paper, whose local solves run one per CPU core).  A shape (mhm_tuning) picks, per
// refinement level on the level-Schur path, the chunk of elements per factor + solve launch
// pair, the resident solve blocks per SM, the depth of the shared-memory ring of staged
// level operators, the L2 prefetch of the operators ahead of use and the L2 policy of their
// copies.  The shapes change speed only; every shape computes the same results.
//
// The search is a coordinate descent: each field in turn over its candidate values, the
// other fields fixed at the best values so far, two sweeps; every candidate runs the
// level's first elements (up to kTuneSample) once to warm up and twice timed with CUDA
// events on the caller's stream, the faster run counting.  Results go to a text cache, one
// line per key (degree, level, right-hand sides, device name, SM count); the last line of a
// key wins.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "mhm_internal.h"

namespace mhm {

namespace {

constexpr int64_t kTuneSample = 16384;

Tuning from_public(const mhm_tuning& t) {
    Tuning u;
    u.chunk = t.chunk;
    u.blocks_per_sm = t.blocks_per_sm;
    u.nbuf = t.op_buffers;
    u.l2pf = t.l2_prefetch;
    u.pf_all = t.prefetch_all;
    u.op_policy = t.op_policy;
    return u;
}

mhm_tuning to_public(const Tuning& u, double ms) {
    mhm_tuning t;
    t.chunk = u.chunk;
    t.blocks_per_sm = u.blocks_per_sm;
    t.op_buffers = u.nbuf;
    t.l2_prefetch = u.l2pf;
    t.prefetch_all = u.pf_all;
    t.op_policy = u.op_policy;
    t.ms_per_K = ms;
    return t;
}

bool valid(const mhm_tuning& t) {
    return t.chunk >= 256 && t.chunk <= 8192 && t.blocks_per_sm >= 1 && t.blocks_per_sm <= 4 && t.op_buffers >= 2 &&
           t.op_buffers <= 4 && t.l2_prefetch >= 0 && t.l2_prefetch <= 64 && (t.prefetch_all == 0 || t.prefetch_all == 1) &&
           t.op_policy >= 0 && t.op_policy <= 2;
}

const Level* level_of(const mhm_mesh* mesh, int r) {
    for (const Level& lv : mesh->levels)
        if (lv.r == r) return &lv;
    return nullptr;
}

std::string tune_key(const mhm_mesh* mesh, const Level& lv) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, mesh->device);
    std::string name = prop.name;
    std::replace(name.begin(), name.end(), ' ', '_');
    std::ostringstream k;
    k << "P=" << mesh->desc.degree << " r=" << lv.r << " R=" << (mesh->NI + 1) << " dev=" << name
      << " sms=" << prop.multiProcessorCount;
    return k.str();
}

bool cache_lookup(const char* path, const std::string& key, Tuning* out, double* ms) {
    std::ifstream in(path);
    if (!in) return false;
    std::string line;
    bool hit = false;
    while (std::getline(in, line)) {
        const size_t bar = line.find('|');
        if (bar == std::string::npos || line.substr(0, bar) != key) continue;
        Tuning u;
        double m = 0.0;
        if (std::sscanf(line.c_str() + bar + 1, "chunk=%d bps=%d nbuf=%d l2pf=%d pfall=%d pol=%d ms_per_K=%lf", &u.chunk,
                        &u.blocks_per_sm, &u.nbuf, &u.l2pf, &u.pf_all, &u.op_policy, &m) == 7 &&
            valid(to_public(u, m))) {
            *out = u;
            *ms = m;
            hit = true;
        }
    }
    return hit;
}

bool cache_append(const char* path, const std::string& key, const Tuning& u, double ms) {
    FILE* f = std::fopen(path, "a");
    if (!f) return false;
    std::fprintf(f, "%s|chunk=%d bps=%d nbuf=%d l2pf=%d pfall=%d pol=%d ms_per_K=%.9g\n", key.c_str(), u.chunk,
                 u.blocks_per_sm, u.nbuf, u.l2pf, u.pf_all, u.op_policy, ms);
    return std::fclose(f) == 0;
}

// Milliseconds per element of level lv under its current shape (best of two timed runs).
mhm_status time_level(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                      const mhm_solve_opts& o, double* AK, double* EK, double* BK, double* FK, int32_t* status,
                      int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                      double* ms_per_K) {
    const int64_t n = std::min<int64_t>(lv.nK, kTuneSample);
    const size_t off = level_region_offset(mesh, lv, MHM_MIXED);
    const size_t need = level_workspace_bytes(mesh, lv, MHM_MIXED);
    void* region = (char*)ws + off;
    double best = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
        MHM_CUDA_TRY(cudaEventRecord(e0, s));
        mhm_status st = launch_local_mixed(mesh, lv, kappa, f, o, 0, n, AK, EK, BK, FK, status, iters, region, need, s);
        if (st) return st;
        MHM_CUDA_TRY(cudaEventRecord(e1, s));
        MHM_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        MHM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, (double)ms);   // the first run warms caches and code
    }
    *ms_per_K = best / (double)n;
    return MHM_OK;
}

// Coordinate search over the shape of one level; sets lv.tune to the best shape found.
mhm_status search_level(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                        const mhm_solve_opts& o, double* AK, double* EK, double* BK, double* FK, int32_t* status,
                        int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t s, double* best_ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MHM_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(MHM_ERR_CUDA, "mhm_autotune: cudaEventCreate");
    }
    mhm_solve_opts to = o;
    to.factor_store = nullptr;   // timing runs factor every element
    to.factor_reuse = 0;
    Tuning best = Tuning();
    best.chunk = (int)std::min<int64_t>(8192, std::max<int64_t>(256, lv.nK));
    lv.tune = best;
    double best_t = 0.0;
    mhm_status st = time_level(mesh, lv, kappa, f, to, AK, EK, BK, FK, status, iters, ws, ws_bytes, s, e0, e1, &best_t);
    struct Field {
        int Tuning::*m;
        std::vector<int> values;
    };
    const std::vector<Field> fields = {{&Tuning::nbuf, {2, 3, 4}},          {&Tuning::pf_all, {0, 1}},
                                       {&Tuning::l2pf, {0, 2, 4, 8}},       {&Tuning::op_policy, {0, 1, 2}},
                                       {&Tuning::blocks_per_sm, {2, 3, 4}},    {&Tuning::chunk, {2048, 4096, 8192}}};
    for (int sweep = 0; sweep < 2 && !st; ++sweep) {
        for (const Field& fd : fields) {
            for (int v : fd.values) {
                if (st) break;
                if (best.*(fd.m) == v) continue;
                Tuning cand = best;
                cand.*(fd.m) = v;
                lv.tune = cand;
                double t = 0.0;
                st = time_level(mesh, lv, kappa, f, to, AK, EK, BK, FK, status, iters, ws, ws_bytes, s, e0, e1, &t);
                if (!st && t < best_t) {
                    best_t = t;
                    best = cand;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    best.tuned = 1;
    lv.tune = best;
    *best_ms = best_t;
    return st;
}

}  // namespace

mhm_status tune_from_cache_or_search(const mhm_mesh* mesh, const double* kappa, const mhm_source& f,
                                     const mhm_solve_opts& o, double* AK, double* EK, double* BK, double* FK,
                                     int32_t* status, int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t s) {
    for (const Level& lv : mesh->levels) {
        if (lv.tune.tuned || !schur_split_level(mesh, lv)) continue;
        const std::string key = tune_key(mesh, lv);
        Tuning u;
        double ms = 0.0;
        if (cache_lookup(o.tuner_cache, key, &u, &ms)) {
            u.tuned = 1;
            lv.tune = u;
            continue;
        }
        mhm_status st = search_level(mesh, lv, kappa, f, o, AK, EK, BK, FK, status, iters, ws, ws_bytes, s, &ms);
        if (st) return st;
        if (!cache_append(o.tuner_cache, key, lv.tune, ms))
            return fail(MHM_ERR_INVALID_ARG, std::string("tuning cache not writable: ") + o.tuner_cache);
    }
    return MHM_OK;
}

}  // namespace mhm

using namespace mhm;

extern "C" mhm_status mhm_set_tuning(mhm_mesh* mesh, int32_t r, const mhm_tuning* t) {
    if (!mesh || !t) return fail(MHM_ERR_INVALID_ARG, "mhm_set_tuning: NULL argument");
    if (!valid(*t)) return fail(MHM_ERR_INVALID_ARG, "mhm_set_tuning: a field is out of range");
    const Level* lv = level_of(mesh, r);
    if (!lv) return fail(MHM_ERR_INVALID_ARG, "mhm_set_tuning: the mesh has no level r");
    lv->tune = from_public(*t);
    lv->tune.tuned = 1;
    return MHM_OK;
}

extern "C" mhm_status mhm_get_tuning(const mhm_mesh* mesh, int32_t r, mhm_tuning* t) {
    if (!mesh || !t) return fail(MHM_ERR_INVALID_ARG, "mhm_get_tuning: NULL argument");
    const Level* lv = level_of(mesh, r);
    if (!lv) return fail(MHM_ERR_INVALID_ARG, "mhm_get_tuning: the mesh has no level r");
    *t = to_public(lv->tune, 0.0);
    return MHM_OK;
}

extern "C" mhm_status mhm_autotune(mhm_mesh* mesh, const double* kappa, const mhm_source* f,
                                   const mhm_solve_opts* opts, double* AK, double* EK, double* BK, double* FK,
                                   int32_t* status, int32_t* iters, void* workspace, size_t ws_bytes,
                                   const char* cache_path, void* stream) {
    if (!mesh) return fail(MHM_ERR_INVALID_ARG, "mhm_autotune: NULL mesh");
    if (mesh->device < 0) return fail(MHM_ERR_UNSUPPORTED, "mhm_autotune: mesh was created without a device");
    if (!kappa || !f || !AK || !EK || !BK || !FK || !status)
        return fail(MHM_ERR_INVALID_ARG, "mhm_autotune: NULL pointer argument");
    mhm_status st = check_source(f, "mhm_autotune");
    if (st) return st;
    MHM_CUDA_TRY(cudaSetDevice(mesh->device));
    mhm_solve_opts o{};
    o.it_max = 8;
    o.tol = 1e-12;
    if (opts) o = *opts;
    if (o.it_max < 1 || !(o.tol > 0.0)) return fail(MHM_ERR_INVALID_ARG, "mhm_autotune: it_max >= 1 and tol > 0 required");
    if (ws_bytes < local_workspace_bytes(mesh, MHM_MIXED) || (local_workspace_bytes(mesh, MHM_MIXED) > 0 && !workspace))
        return fail(MHM_ERR_INVALID_ARG, "mhm_autotune: workspace smaller than mhm_local_workspace_size(MIXED)");
    cudaStream_t s = (cudaStream_t)stream;
    for (const Level& lv : mesh->levels) {
        if (!schur_split_level(mesh, lv)) continue;
        double ms = 0.0;
        st = search_level(mesh, lv, kappa, *f, o, AK, EK, BK, FK, status, iters, workspace, ws_bytes, s, &ms);
        if (st) return st;
        if (cache_path && !cache_append(cache_path, tune_key(mesh, lv), lv.tune, ms))
            return fail(MHM_ERR_INVALID_ARG, std::string("mhm_autotune: cache not writable: ") + cache_path);
    }
    return MHM_OK;
}
