// solveLocalProblem in mixed precision (placeholder until the FP32 kernel lands).
#include "mhm_internal.h"

namespace mhm {

size_t mixed_workspace_bytes(const mhm_mesh*) { return 0; }

mhm_status launch_local_mixed(const mhm_mesh*, const double*, const mhm_source&, const mhm_solve_opts&, int64_t,
                              int64_t, double*, double*, double*, double*, int32_t*, int32_t*, void*, size_t,
                              cudaStream_t) {
    return fail(MHM_ERR_UNSUPPORTED, "mhm_local_solve_batch: MIXED precision not built");
}

}  // namespace mhm
