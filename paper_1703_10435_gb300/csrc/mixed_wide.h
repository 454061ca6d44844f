// Mixed-precision local solves of wide P1 levels (r = 6, 7: lattice rows of 64 and 128
// unknowns), local_mixed_wide.cu; host entry points used by the batch solve.
#pragma once

#include "mhm_internal.h"

namespace mhm {

// True when the level runs on the wide mixed path: P1, N = 64 or 128, at most 16
// right-hand sides (N_I + 1).
bool wide_mixed_level(const mhm_mesh* mesh, const Level& lv);

// Workspace bytes of a wide mixed level: one slot per resident block (FP64 solution,
// residual, direction and product vectors, FP32 level inverses) plus the list of failed
// elements; at least the FP64 path's own need, which the re-solve of failed elements uses.
size_t wide_mixed_workspace(const mhm_mesh* mesh, const Level& lv);

// Launch indices [K0, K1) of the level: factor, preconditioned CG and outputs in one
// persistent launch, then (unless opts.no_fallback) the FP64 re-solve of the elements
// that did not converge.
mhm_status launch_local_mixed_wide(const mhm_mesh* mesh, const Level& lv, const double* kappa, const mhm_source& f,
                                   const mhm_solve_opts& opts, int64_t K0, int64_t K1, double* AK, double* EK,
                                   double* BK, double* FK, int32_t* status, int32_t* iters, void* ws,
                                   size_t ws_bytes, cudaStream_t stream);

// The FP64 path over a device list of elements (count on the device, at most max_n),
// with a workspace for levels whose window lives in global memory (local_fp64.cu).
mhm_status launch_local_fp64_list_ws(const mhm_mesh* mesh, const Level& lv, const double* kappa,
                                     const mhm_source& f, const int32_t* list, const int32_t* count, int64_t max_n,
                                     double* AK, double* EK, double* BK, double* FK, int32_t* status,
                                     int32_t* iters, void* ws, size_t ws_bytes, cudaStream_t stream);

}  // namespace mhm
