// Relative Frobenius error terms in FP64 on the GPU (the only FP64 arithmetic
// on the device): sum (C - Cref)^2 and sum Cref^2, deterministic two-pass
// reduction (fixed per-block partials, then one block sums them in order).
#include <algorithm>

#include "pgk_internal.cuh"

namespace pgk {

static const int RELERR_BLOCKS = 1024;
static const int RELERR_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of (a, b); result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[32], sb[32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = l < nw ? sa[l] : 0.0;
        b = l < nw ? sb[l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

// Block b takes rows b, b + gridDim.x, ...; its threads stride over the columns
// of a row (coalesced, no per-element division).
__global__ void __launch_bounds__(256) k_relerr_partial(int rows, int cols, const float* __restrict__ C,
                                                       int ldc, const double* __restrict__ R, int ldr,
                                                       const int64_t* __restrict__ row_index,
                                                       double* __restrict__ partial) {
    double num = 0.0, den = 0.0;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const long long cr = row_index ? row_index[r] : r;
        const float* crow = C + (size_t)cr * ldc;
        const double* rrow = R + (size_t)r * ldr;
        for (int c = threadIdx.x; c < cols; c += blockDim.x) {
            const double ref = __ldg(rrow + c);
            const double d = (double)__ldg(crow + c) - ref;
            num = fma(d, d, num);
            den = fma(ref, ref, den);
        }
    }
    block_sum2(num, den);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = num;
        partial[2 * blockIdx.x + 1] = den;
    }
}

__global__ void __launch_bounds__(256) k_relerr_final(int nparts, const double* __restrict__ partial,
                                                     double* __restrict__ out) {
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        num += partial[2 * i];
        den += partial[2 * i + 1];
    }
    block_sum2(num, den);
    if (threadIdx.x == 0) {
        out[0] = num;
        out[1] = den;
    }
}

pgk_status relerr_launch(int rows, int cols, const float* C, int ldc, const double* Cref, int ldr,
                         const int64_t* row_index, double* out, double* partial, int max_parts,
                         cudaStream_t st) {
    const int parts = std::max(1, std::min(rows, max_parts));
    k_relerr_partial<<<parts, RELERR_THREADS, 0, st>>>(rows, cols, C, ldc, Cref, ldr, row_index,
                                                       partial);
    k_relerr_final<<<1, RELERR_THREADS, 0, st>>>(parts, partial, out);
    PGK_CUDA_TRY(cudaGetLastError(), "relerr launch");
    return PGK_OK;
}

}  // namespace pgk

using namespace pgk;

extern "C" pgk_status pgk_relerr(int rows, int cols, const float* C, int ldc, const double* Cref,
                                 int ldr, const int64_t* row_index, double* out, void* stream) {
    if (rows < 1 || cols < 1 || !C || !Cref || !out || ldc < cols || ldr < cols) {
        set_error("bad relerr arguments");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_status st;
    double* partial = (double*)workspace(WS_PARTIAL, 2 * sizeof(double) * RELERR_BLOCKS, &st);
    if (!partial) return st;
    return relerr_launch(rows, cols, C, ldc, Cref, ldr, row_index, out, partial, RELERR_BLOCKS,
                         (cudaStream_t)stream);
}
