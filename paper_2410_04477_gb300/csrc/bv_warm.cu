// bv_warm.cu -- learned warm start: dataset features and the MLP that maps them to a
// starting theta for the maximum-likelihood search.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bv_internal.h"

extern "C" int bv_features(bv_ctx* c, int32_t max_points, uint64_t seed, float* out) {
    (void)c; (void)max_points; (void)seed; (void)out;
    return BV_ESTATE;
}

extern "C" int bv_warmstart_load(bv_ctx* c, const char* path) {
    (void)c; (void)path;
    return BV_ESTATE;
}

extern "C" int bv_warmstart_predict(bv_ctx* c, const bv_theta* in, bv_theta* out) {
    (void)c; (void)in; (void)out;
    return BV_ESTATE;
}
