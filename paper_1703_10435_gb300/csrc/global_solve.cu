// reduceLocalProblems' solve (Alg. 1; Sec. 3, Eq. "mat_global"):
//     [ A  B^T ] [lambda]   [E]
//     [ B  0   ] [u0    ] = [F]
// in FP64 on the GPU.  The saddle-point matrix is filled in CSR by a gather
// kernel from the skeleton values and the per-K blocks B_K, then factored by
// the sparse QR of cuSOLVER (nested-dissection ordering) -- a library direct
// solver for this stage, which is outside the local-problem hot path.
#include <cuda_runtime.h>
#include <cusolverSp.h>
#include <cusparse.h>

#include "mhm_internal.h"

namespace mhm {

namespace {

__global__ void k_fill_saddle(int64_t nnz, const int64_t* src, const double* A_vals, const double* BK, double* out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    const int64_t s = src[t];
    out[t] = s >= 0 ? A_vals[s] : BK[-s - 1];
}

__global__ void k_rhs_saddle(int64_t L, int64_t nK, const double* E, const double* FK, double* rhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < L) rhs[t] = E[t];
    else if (t < L + nK) rhs[t] = FK[t - L];
}

__global__ void k_split(int64_t L, int64_t nK, const double* x, double* lam, double* u0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < L) lam[t] = x[t];
    else if (t < L + nK) u0[t - L] = x[t];
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
    const int64_t n = mesh->nlam + mesh->nK, nnz = mesh->aug_nnz;
    if (n > INT32_MAX || nnz > INT32_MAX) return fail(MHM_ERR_UNSUPPORTED, "mhm_solve_global: system too large");
    double *vals = nullptr, *rhs = nullptr, *x = nullptr;
    cudaError_t e = cudaMallocAsync(&vals, nnz * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&rhs, n * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&x, n * sizeof(double), s);
    mhm_status st = MHM_OK;
    cusolverSpHandle_t h = nullptr;
    cusparseMatDescr_t descr = nullptr;
    if (e != cudaSuccess) {
        st = cuda_fail(e, "mhm_solve_global: cudaMallocAsync");
    } else {
        const int thr = 256;
        k_fill_saddle<<<(unsigned)((nnz + thr - 1) / thr), thr, 0, s>>>(nnz, mesh->d_aug_src, A_vals, BK, vals);
        k_rhs_saddle<<<(unsigned)((n + thr - 1) / thr), thr, 0, s>>>(mesh->nlam, mesh->nK, E, FK, rhs);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "mhm_solve_global: fill");
    }
    if (!st && (cusolverSpCreate(&h) != CUSOLVER_STATUS_SUCCESS || cusolverSpSetStream(h, s) != CUSOLVER_STATUS_SUCCESS))
        st = fail(MHM_ERR_CUDA, "mhm_solve_global: cusolverSpCreate failed");
    if (!st && (cusparseCreateMatDescr(&descr) != CUSPARSE_STATUS_SUCCESS))
        st = fail(MHM_ERR_CUDA, "mhm_solve_global: cusparseCreateMatDescr failed");
    if (!st) {
        cusparseSetMatType(descr, CUSPARSE_MATRIX_TYPE_GENERAL);
        cusparseSetMatIndexBase(descr, CUSPARSE_INDEX_BASE_ZERO);
        int singular = -1;
        const cusolverStatus_t cs = cusolverSpDcsrlsvqr(h, (int)n, (int)nnz, descr, vals, mesh->d_aug_rowptr,
                                                        mesh->d_aug_cols, rhs, 1e-14, 3 /* nested dissection */, x,
                                                        &singular);
        if (cs != CUSOLVER_STATUS_SUCCESS) st = fail(MHM_ERR_CUDA, "mhm_solve_global: cusolverSpDcsrlsvqr failed");
        else if (singular >= 0) st = fail(MHM_ERR_INVALID_ARG, "mhm_solve_global: saddle-point matrix is singular");
        else {
            const int thr = 256;
            k_split<<<(unsigned)((n + thr - 1) / thr), thr, 0, s>>>(mesh->nlam, mesh->nK, x, lambda, u0);
            e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(e, "mhm_solve_global: split");
        }
    }
    if (descr) cusparseDestroyMatDescr(descr);
    if (h) cusolverSpDestroy(h);
    if (vals) cudaFreeAsync(vals, s);
    if (rhs) cudaFreeAsync(rhs, s);
    if (x) cudaFreeAsync(x, s);
    return st;
}
