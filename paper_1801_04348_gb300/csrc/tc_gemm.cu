// tcgen05 tensor-core variants (placeholder until the kernels land).
#include "pgk_internal.cuh"

namespace pgk {
void register_tc_variants(std::vector<Variant>&) {}
pgk_status tc_select(const pgk_machine*, int, int, int, pgk_dtype, const pgk_params*, pgk_case*) {
    set_error("tensor-core forms are not built yet");
    return PGK_ERR_UNSUPPORTED;
}
pgk_status tc_gemm_fp32_inputs(const pgk_case&, int, int, int, pgk_dtype, const float*, int,
                               const float*, int, float*, int, int, cudaStream_t) {
    set_error("tensor-core forms are not built yet");
    return PGK_ERR_UNSUPPORTED;
}
}  // namespace pgk

extern "C" pgk_status pgk_gemm_lowp(int, int, int, pgk_dtype, const void*, int, const void*, int,
                                    const void*, const void*, const float*, const float*, float*,
                                    int, int, const pgk_params*, void*) {
    pgk::set_error("tensor-core forms are not built yet");
    return PGK_ERR_UNSUPPORTED;
}
