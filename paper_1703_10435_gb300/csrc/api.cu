// C ABI entry points: argument checks, error reporting and dispatch to the
// kernels.  No entry point falls back to the CPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <string>

#include "mhm_internal.h"
#include "mixed_wide.h"

namespace mhm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

mhm_status fail(mhm_status code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

mhm_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MHM_ERR_OOM : MHM_ERR_CUDA;
}

void timing_begin(const mhm_mesh* m) {
    m->tev_used = 0;
    m->tev_kernel.clear();
}

void timing_mark(const mhm_mesh* m, int kernel, cudaStream_t s, bool start) {
    if (!m->timing) return;
    if (m->tev_used == m->tev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            m->timing = false;   // no timing rather than a failed solve
            return;
        }
        m->tev.push_back(e);
    }
    cudaEventRecord(m->tev[m->tev_used++], s);
    if (start) m->tev_kernel.push_back(kernel);
}

bool device_supported(int device) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return false;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    return major == 10 && minor == 3;
}

void level_range(const Level& lv, int64_t K0, int64_t K1, int64_t* i0, int64_t* i1) {
    if (lv.K.empty()) {   // uniform mesh: the launch index is K
        *i0 = K0;
        *i1 = K1;
        return;
    }
    *i0 = std::lower_bound(lv.K.begin(), lv.K.end(), (int32_t)K0) - lv.K.begin();
    *i1 = std::lower_bound(lv.K.begin(), lv.K.end(), (int32_t)std::min<int64_t>(K1, INT32_MAX)) - lv.K.begin();
}

bool fp64_level(const mhm_mesh* mesh, const Level& lv) {
    if (mesh->desc.degree == 1) return lv.N > 32;
    return fp64_window_rows(mesh, lv) > 128;
}

// MIXED: wide P1 levels (r = 6, 7) run the level-Schur factor with CG (local_mixed_wide.cu)
bool wide_level(const mhm_mesh* mesh, const Level& lv, int32_t precision) {
    return precision == MHM_MIXED && wide_mixed_level(mesh, lv);
}

size_t level_workspace_bytes(const mhm_mesh* mesh, const Level& lv, int32_t precision) {
    const size_t b = wide_level(mesh, lv, precision) ? wide_mixed_workspace(mesh, lv)
                     : (precision == MHM_FP64 || fp64_level(mesh, lv)) ? fp64_level_workspace(mesh, lv)
                                                                         : mixed_level_workspace(mesh, lv);
    return (b + 255) & ~(size_t)255;
}

size_t level_region_offset(const mhm_mesh* mesh, const Level& lv, int32_t precision) {
    size_t off = 0;
    for (const Level& l2 : mesh->levels) {
        if (&l2 == &lv) break;
        off += level_workspace_bytes(mesh, l2, precision);
    }
    return off;
}

size_t local_workspace_bytes(const mhm_mesh* mesh, int32_t precision) {
    if (mesh->device < 0) return 0;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(mesh->device);
    size_t bytes = 0;   // the levels may run at the same time: a region each
    for (const Level& lv : mesh->levels) bytes += level_workspace_bytes(mesh, lv, precision);
    cudaSetDevice(cur);
    return bytes;
}

mhm_status check_source(const mhm_source* f, const char* who) {
    if (!f) return fail(MHM_ERR_INVALID_ARG, std::string(who) + ": NULL source");
    if (f->kind != MHM_SRC_CONST && f->kind != MHM_SRC_SINSIN && f->kind != MHM_SRC_QUAD)
        return fail(MHM_ERR_INVALID_ARG, std::string(who) + ": unknown source kind");
    if (f->kind == MHM_SRC_QUAD && !f->values_dev)
        return fail(MHM_ERR_INVALID_ARG, std::string(who) + ": MHM_SRC_QUAD needs values_dev");
    return MHM_OK;
}

// Makes the mesh's device current; fails for host-only meshes.
static mhm_status enter(const mhm_mesh* mesh, const char* who) {
    if (!mesh) return fail(MHM_ERR_INVALID_ARG, std::string(who) + ": NULL mesh");
    if (mesh->device < 0)
        return fail(MHM_ERR_UNSUPPORTED, std::string(who) + ": mesh was created without a device");
    cudaError_t e = cudaSetDevice(mesh->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return MHM_OK;
}

}  // namespace mhm

using namespace mhm;

extern "C" const char* mhm_last_error(void) { return g_last_error.c_str(); }

extern "C" mhm_status mhm_local_workspace_size(const mhm_mesh* mesh, int32_t precision, size_t* bytes) {
    if (!mesh || !bytes) return fail(MHM_ERR_INVALID_ARG, "mhm_local_workspace_size: NULL argument");
    if (precision == MHM_FP64 || precision == MHM_MIXED) {
        *bytes = local_workspace_bytes(mesh, precision);
        return MHM_OK;
    }
    return fail(MHM_ERR_INVALID_ARG, "mhm_local_workspace_size: unknown precision");
}

extern "C" mhm_status mhm_factor_store_size(const mhm_mesh* mesh, size_t* bytes) {
    if (!mesh || !bytes) return fail(MHM_ERR_INVALID_ARG, "mhm_factor_store_size: NULL argument");
    int cur = 0;
    cudaGetDevice(&cur);
    if (mesh->device >= 0) cudaSetDevice(mesh->device);
    *bytes = factor_store_layout(mesh, nullptr, nullptr);
    cudaSetDevice(cur);
    return MHM_OK;
}

extern "C" mhm_status mhm_local_solve_batch(const mhm_mesh* mesh, const double* kappa, const mhm_source* f,
                                            int32_t precision, const mhm_solve_opts* opts, double* AK,
                                            double* EK, double* BK, double* FK, int32_t* status,
                                            int32_t* iters, void* workspace, size_t ws_bytes, void* stream) {
    mhm_status st = enter(mesh, "mhm_local_solve_batch");
    if (st) return st;
    if (!kappa || !f || !AK || !EK || !BK || !FK || !status)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: NULL pointer argument");
    st = check_source(f, "mhm_local_solve_batch");
    if (st) return st;
    mhm_solve_opts o{};
    o.it_max = 8;
    o.tol = 1e-12;
    o.K_begin = 0;
    o.K_end = 0;
    if (opts) o = *opts;
    const int64_t K0 = o.K_begin, K1 = o.K_end > 0 ? o.K_end : mesh->nK;
    if (K0 < 0 || K1 > mesh->nK || K0 > K1)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: K range out of bounds");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision != MHM_FP64 && precision != MHM_MIXED)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: unknown precision");
    if (precision == MHM_MIXED && (o.it_max < 1 || !(o.tol > 0.0)))
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: it_max >= 1 and tol > 0 required");
    if (precision != MHM_MIXED) {
        o.factor_store = nullptr;   // the FP64 path keeps no factors
        o.factor_reuse = 0;
    } else if (o.factor_reuse && !o.factor_store) {
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: factor_reuse needs a factor_store");
    } else if (o.factor_store && o.factor_store_bytes < factor_store_layout(mesh, nullptr, nullptr)) {
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: factor_store smaller than mhm_factor_store_size");
    } else if (o.factor_store && factor_store_layout(mesh, nullptr, nullptr) == 0) {
        o.factor_store = nullptr;   // no level keeps factors
        o.factor_reuse = 0;
    }
    {
        const size_t need = local_workspace_bytes(mesh, precision);
        if (ws_bytes < need || (need > 0 && !workspace))
            return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_batch: workspace smaller than mhm_local_workspace_size");
    }
    if (precision == MHM_MIXED && o.tuner_cache) {
        st = tune_from_cache_or_search(mesh, kappa, *f, o, AK, EK, BK, FK, status, iters, workspace, ws_bytes, s);
        if (st) return st;
    }
    // One launch sequence per refinement level.  The levels are independent (disjoint
    // elements and outputs), so with several of them the first runs on the caller's stream
    // and the others on side streams forked from it (an event after the caller's earlier
    // work) and joined back (the caller's stream waits for each); a mixed level uses its
    // own region of the workspace (levels without one get an empty region).
    std::vector<const Level*> run;
    std::vector<int64_t> r0, r1;
    for (const Level& lv : mesh->levels) {
        int64_t i0 = 0, i1 = 0;
        level_range(lv, K0, K1, &i0, &i1);
        if (i1 <= i0) continue;
        run.push_back(&lv);
        r0.push_back(i0);
        r1.push_back(i1);
    }
    // MIXED: the level-Schur levels go together into one persistent launch pair on the
    // caller's stream (coarse elements of uneven refinement level, bucketed by size),
    // beside the other levels' launch sequences
    std::vector<const Level*> group;
    std::vector<int64_t> g0, g1;
    std::vector<char*> gregion;
    if (precision == MHM_MIXED) {
        for (size_t i = 0; i < run.size(); ++i)
            if (!fp64_level(mesh, *run[i]) && schur_split_level(mesh, *run[i])) {
                group.push_back(run[i]);
                g0.push_back(r0[i]);
                g1.push_back(r1[i]);
                gregion.push_back((char*)workspace + level_region_offset(mesh, *run[i], precision));
            }
        if (levels_launchable(mesh, group, g0, g1, o)) {
            std::vector<const Level*> rest;
            std::vector<int64_t> q0, q1;
            for (size_t i = 0; i < run.size(); ++i)
                if (std::find(group.begin(), group.end(), run[i]) == group.end()) {
                    rest.push_back(run[i]);
                    q0.push_back(r0[i]);
                    q1.push_back(r1[i]);
                }
            run.swap(rest);
            r0.swap(q0);
            r1.swap(q1);
            run.insert(run.begin(), nullptr);   // the group, on the caller's stream
            r0.insert(r0.begin(), 0);
            r1.insert(r1.begin(), 0);
        } else {
            group.clear();
        }
    }
    const size_t nside = run.empty() ? 0 : run.size() - 1;
    if (nside > 0) {
        while (mesh->side.size() < nside) {
            cudaStream_t ss;
            cudaEvent_t ev;
            MHM_CUDA_TRY(cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking));
            MHM_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            mesh->side.push_back(ss);
            mesh->side_done.push_back(ev);
        }
        if (!mesh->fork_ev) MHM_CUDA_TRY(cudaEventCreateWithFlags(&mesh->fork_ev, cudaEventDisableTiming));
        MHM_CUDA_TRY(cudaEventRecord(mesh->fork_ev, s));
    }
    for (size_t i = 0; i < run.size(); ++i) {
        cudaStream_t si = i == 0 ? s : mesh->side[i - 1];
        if (i > 0) MHM_CUDA_TRY(cudaStreamWaitEvent(si, mesh->fork_ev, 0));
        if (!run[i]) {
            st = launch_local_mixed_levels(mesh, group, g0, g1, gregion, kappa, *f, o, AK, EK, BK, FK, status, iters,
                                           si);
        } else {
            const Level& lv = *run[i];
            const size_t need = level_workspace_bytes(mesh, lv, precision);
            void* region = need ? (char*)workspace + level_region_offset(mesh, lv, precision) : nullptr;
            if (wide_level(mesh, lv, precision)) {
                st = launch_local_mixed_wide(mesh, lv, kappa, *f, o, r0[i], r1[i], AK, EK, BK, FK, status, iters,
                                             region, need, si);
            } else if (precision == MHM_FP64 || fp64_level(mesh, lv)) {
                st = launch_local_fp64(mesh, lv, kappa, *f, r0[i], r1[i], AK, EK, BK, FK, status, iters, region, need,
                                       si);
            } else {
                st = launch_local_mixed(mesh, lv, kappa, *f, o, r0[i], r1[i], AK, EK, BK, FK, status, iters, region,
                                        need, si);
            }
        }
        if (st) return st;
        if (i > 0) MHM_CUDA_TRY(cudaEventRecord(mesh->side_done[i - 1], si));
    }
    for (size_t i = 0; i < nside; ++i) MHM_CUDA_TRY(cudaStreamWaitEvent(s, mesh->side_done[i], 0));
    return MHM_OK;
}

extern "C" mhm_status mhm_local_solve_waves(const mhm_mesh* mesh, const double* kappa_host, size_t kappa_budget_bytes,
                                            const mhm_source* f, int32_t precision, const mhm_solve_opts* opts,
                                            double* AK, double* EK, double* BK, double* FK, int32_t* status,
                                            int32_t* iters, void* workspace, size_t ws_bytes, void* stream,
                                            int32_t* n_waves) {
    mhm_status st = enter(mesh, "mhm_local_solve_waves");
    if (st) return st;
    if (!kappa_host || !f) return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_waves: NULL pointer argument");
    st = check_source(f, "mhm_local_solve_waves");
    if (st) return st;
    mhm_solve_opts o{};
    o.it_max = 8;
    o.tol = 1e-12;
    if (opts) o = *opts;
    const int64_t K0 = o.K_begin, K1 = o.K_end > 0 ? o.K_end : mesh->nK;
    if (K0 < 0 || K1 > mesh->nK || K0 > K1)
        return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_waves: K range out of bounds");
    // first kappa value of K (per-K levels: the mesh's offsets; uniform: K 4^r)
    auto koff = [&](int64_t K) { return mesh->per_k_levels ? mesh->kap_off[K] : K * mesh->nfine; };
    // waves: contiguous K ranges, each as long as its kappa fits in one of the two buffers
    const size_t half = kappa_budget_bytes / 2;
    std::vector<int64_t> cut{K0};
    while (cut.back() < K1) {
        const int64_t a = cut.back();
        int64_t b = a;
        while (b < K1 && (size_t)(koff(b + 1) - koff(a)) * sizeof(double) <= half) ++b;
        if (b == a)
            return fail(MHM_ERR_INVALID_ARG, "mhm_local_solve_waves: the kappa of one element exceeds half the budget");
        cut.push_back(b);
    }
    const int nw = (int)cut.size() - 1;
    if (n_waves) *n_waves = nw;
    if (nw == 0) return MHM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!mesh->wave_copy) {
        MHM_CUDA_TRY(cudaStreamCreateWithFlags(&mesh->wave_copy, cudaStreamNonBlocking));
        MHM_CUDA_TRY(cudaEventCreateWithFlags(&mesh->wave_start, cudaEventDisableTiming));
        for (int b = 0; b < 2; ++b) {
            MHM_CUDA_TRY(cudaEventCreateWithFlags(&mesh->wave_copied[b], cudaEventDisableTiming));
            MHM_CUDA_TRY(cudaEventCreateWithFlags(&mesh->wave_solved[b], cudaEventDisableTiming));
        }
    }
    // the buffers come from the stream-ordered allocator on the caller's stream; the copy
    // stream starts after them (and after the caller's earlier work)
    double* buf[2] = {nullptr, nullptr};
    const int nbuf = nw > 1 ? 2 : 1;
    for (int b = 0; b < nbuf; ++b) {
        int64_t most = 0;   // the largest wave this buffer holds
        for (int w = b; w < nw; w += 2) most = std::max<int64_t>(most, koff(cut[w + 1]) - koff(cut[w]));
        cudaError_t e = cudaMallocAsync((void**)&buf[b], (size_t)most * sizeof(double), s);
        if (e != cudaSuccess) {
            for (int i = 0; i < b; ++i) cudaFreeAsync(buf[i], s);
            return cuda_fail(e, "mhm_local_solve_waves: cudaMallocAsync");
        }
    }
    cudaError_t ce = cudaEventRecord(mesh->wave_start, s);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(mesh->wave_copy, mesh->wave_start, 0);
    for (int w = 0; w < nw && !st && ce == cudaSuccess; ++w) {
        const int b = w & 1;
        const int64_t a = cut[w], e = cut[w + 1];
        // buffer b is refilled once the solves of wave w - 2 are done with it
        if (w >= 2) ce = cudaStreamWaitEvent(mesh->wave_copy, mesh->wave_solved[b], 0);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(buf[b], kappa_host + koff(a), (size_t)(koff(e) - koff(a)) * sizeof(double),
                                 cudaMemcpyHostToDevice, mesh->wave_copy);
        if (ce == cudaSuccess) ce = cudaEventRecord(mesh->wave_copied[b], mesh->wave_copy);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, mesh->wave_copied[b], 0);
        if (ce != cudaSuccess) break;
        mhm_solve_opts ow = o;
        ow.K_begin = a;
        ow.K_end = e;
        // the kernels index kappa by the absolute offset of K: a base koff(a) elements before the buffer
        st = mhm_local_solve_batch(mesh, buf[b] - koff(a), f, precision, &ow, AK, EK, BK, FK, status, iters,
                                   workspace, ws_bytes, stream);
        if (!st) ce = cudaEventRecord(mesh->wave_solved[b], s);
    }
    // every copy queued on the copy stream is ordered before the frees on `s`, whichever
    // call above failed: join the copy stream into `s` first (if even that fails, wait for
    // the copy stream on the host rather than free a buffer a copy may still write)
    cudaError_t je = cudaEventRecord(mesh->wave_start, mesh->wave_copy);
    if (je == cudaSuccess) je = cudaStreamWaitEvent(s, mesh->wave_start, 0);
    if (je != cudaSuccess) cudaStreamSynchronize(mesh->wave_copy);
    for (int b = 0; b < nbuf; ++b) cudaFreeAsync(buf[b], s);
    if (ce != cudaSuccess) return cuda_fail(ce, "mhm_local_solve_waves");
    if (je != cudaSuccess) return cuda_fail(je, "mhm_local_solve_waves: joining the copy stream");
    return st;
}

extern "C" mhm_status mhm_assemble_skeleton(const mhm_mesh* mesh, const double* AK, const double* EK,
                                            const mhm_dirichlet* g, double* A_vals, double* E, void* stream) {
    mhm_status st = enter(mesh, "mhm_assemble_skeleton");
    if (st) return st;
    if (!AK || !EK || !A_vals || !E) return fail(MHM_ERR_INVALID_ARG, "mhm_assemble_skeleton: NULL pointer argument");
    return launch_skeleton(mesh, AK, EK, g, A_vals, E, (cudaStream_t)stream);
}

// ------------------------------------------------------------ pipe peaks ---

namespace {

template <typename T, int CHAINS>
__global__ void k_fma_peak(T* out, int iters, T a, T b) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == (T)12345.678) out[threadIdx.x] = s;  // keeps the chains alive
}

template <typename T, int CHAINS>
double time_fma(int sms, int iters) {
    T* out = nullptr;
    cudaMalloc(&out, 1024 * sizeof(T));
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_peak<T, CHAINS><<<blocks, threads>>>(out, iters / 10, (T)0.999, (T)0.001);
    cudaEventRecord(e0);
    k_fma_peak<T, CHAINS><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const double flops = 2.0 * CHAINS * (double)iters * blocks * threads;
    return flops / (ms * 1e-3) / 1e9;
}

}  // namespace

extern "C" mhm_status mhm_measure_pipes(int32_t device, double* out) {
    if (!out) return fail(MHM_ERR_INVALID_ARG, "mhm_measure_pipes: NULL output");
    if (!device_supported(device)) return fail(MHM_ERR_UNSUPPORTED, "mhm_measure_pipes: not an sm_103 device");
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    out[0] = time_fma<double, 8>(sms, 1 << 12);
    out[1] = time_fma<float, 16>(sms, 1 << 16);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mhm_measure_pipes");
    return MHM_OK;
}

extern "C" mhm_status mhm_sync_status(const mhm_mesh* mesh, void* stream, uint32_t* word_out) {
    if (!mesh || mesh->device < 0 || !mesh->d_sword)
        return fail(MHM_ERR_INVALID_ARG, "mhm_sync_status: NULL or host-only mesh");
    MHM_CUDA_TRY(cudaSetDevice(mesh->device));
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t w = 0;
    MHM_CUDA_TRY(cudaMemcpyAsync(&w, mesh->d_sword, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    MHM_CUDA_TRY(cudaMemsetAsync(mesh->d_sword, 0, sizeof(uint32_t), s));
    MHM_CUDA_TRY(cudaStreamSynchronize(s));
    if (word_out) *word_out = w;
    for (int c : {MHM_ERR_TIMEOUT, MHM_ERR_INVALID_ARG, MHM_ERR_UNSUPPORTED, MHM_ERR_NOT_CONVERGED})
        if (w & (1u << c)) return c;
    return MHM_OK;
}

extern "C" mhm_status mhm_set_timing(mhm_mesh* mesh, int32_t enable) {
    if (!mesh || mesh->device < 0) return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_set_timing: no device mesh");
    mesh->timing = enable != 0;
    mhm::timing_begin(mesh);
    return MHM_OK;
}

extern "C" mhm_status mhm_kernel_times(const mhm_mesh* mesh, int32_t* launches, double* ms) {
    if (!mesh || mesh->device < 0 || !launches || !ms)
        return mhm::fail(MHM_ERR_INVALID_ARG, "mhm_kernel_times: NULL argument or host-only mesh");
    for (int k = 0; k < MHM_N_KERNELS; ++k) {
        launches[k] = 0;
        ms[k] = 0.0;
    }
    for (size_t i = 0; i < mesh->tev_kernel.size() && 2 * i + 1 < mesh->tev_used; ++i) {
        cudaEvent_t a = mesh->tev[2 * i], b = mesh->tev[2 * i + 1];
        cudaError_t e = cudaEventSynchronize(b);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e != cudaSuccess) return mhm::cuda_fail(e, "mhm_kernel_times");
        const int k = mesh->tev_kernel[i];
        if (k >= 0 && k < MHM_N_KERNELS) {
            launches[k] += 1;
            ms[k] += t;
        }
    }
    mhm::timing_begin(mesh);   // the next reading covers the calls from here on
    return MHM_OK;
}
