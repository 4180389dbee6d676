// Grouped persistent GEMM (placeholder until the scheduler lands).
#include "pgk_internal.cuh"

namespace pgk {
void grouped_release() {}
}

extern "C" pgk_status pgk_gemm_grouped(int, const pgk_problem*, pgk_dtype, const pgk_params*, int,
                                       int, void*) {
    pgk::set_error("grouped GEMM is not built yet");
    return PGK_ERR_UNSUPPORTED;
}
