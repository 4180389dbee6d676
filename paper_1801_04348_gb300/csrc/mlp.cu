// Cost-model MLP kernels (placeholder until the kernels land).
#include "pgk_internal.cuh"

extern "C" {
pgk_status pgk_mlp_forward(int, const float*, const float*, float*, void*) {
    pgk::set_error("not built yet");
    return PGK_ERR_UNSUPPORTED;
}
pgk_status pgk_mlp_loss_grad(int, const float*, const float*, const float*, float*, float*, void*) {
    pgk::set_error("not built yet");
    return PGK_ERR_UNSUPPORTED;
}
pgk_status pgk_mlp_adam(int, float*, const float*, float*, float*, int, float, float, float, float,
                        void*) {
    pgk::set_error("not built yet");
    return PGK_ERR_UNSUPPORTED;
}
}
