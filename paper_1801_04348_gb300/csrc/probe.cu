// FP32 SIMT throughput probe: the measured denominator beside the derived
// SM count x 128 lanes x 2 flop x clock.  Every thread runs 16 independent
// FMA chains (paired fma.rn.f32x2 or scalar fmaf), enough independent work per
// warp to keep the FMA pipe busy without memory traffic.
#include "pgk_internal.cuh"
#include "simt_rb.cuh"

namespace pgk {

static constexpr int PROBE_THREADS = 256;
static constexpr int PROBE_CHAINS = 16;

template <bool PAIRED>
__global__ void __launch_bounds__(PROBE_THREADS) k_simt_peak_probe(int iters, float* __restrict__ sink) {
    const float seed = 1.0f + 1e-7f * (float)threadIdx.x;
    float out = 0.f;
    if (PAIRED) {
        uint64_t acc[PROBE_CHAINS];
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) acc[c] = pack2(seed + c, seed - c);
        const uint64_t a = pack2(0.999f, 0.998f), b = pack2(1e-3f, 2e-3f);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c) fma2(acc[c], a, b);   // acc += a * b
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) out += lo32(acc[c]) + hi32(acc[c]);
    } else {
        float acc[PROBE_CHAINS];
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) acc[c] = seed + c;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c) acc[c] = fmaf(acc[c], 0.999f, 1e-3f);
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) out += acc[c];
    }
    sink[(size_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = out;
}

}  // namespace pgk

using namespace pgk;

extern "C" {

pgk_status pgk_simt_peak_probe(int blocks, int iters, int paired, float* sink, void* stream) {
    if (blocks < 1 || iters < 1 || !sink) {
        set_error("bad probe arguments (blocks=%d iters=%d)", blocks, iters);
        return PGK_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (paired)
        k_simt_peak_probe<true><<<blocks, PROBE_THREADS, 0, st>>>(iters, sink);
    else
        k_simt_peak_probe<false><<<blocks, PROBE_THREADS, 0, st>>>(iters, sink);
    PGK_CUDA_TRY(cudaGetLastError(), "probe launch");
    return PGK_OK;
}

}  // extern "C"
