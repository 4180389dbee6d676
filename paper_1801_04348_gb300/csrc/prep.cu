// Low-precision operand preparation for the tensor-core forms: FP32 -> BF16
// (round to nearest even), the split x = hi + lo with hi = bf16(x),
// lo = bf16(x - hi), and per-128x128-tile scaled FP8 E4M3 (scale = amax / 448,
// q = e4m3_rn_satfinite(x / scale)).  Each kernel optionally writes its output
// transposed, which turns B (K x N) into the K-major N x K operand the
// tensor-core kernels read.  All are HBM-bound streaming kernels.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "pgk_internal.cuh"

namespace pgk {

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float bf16_value(uint16_t b) {
    return __bfloat162float(__ushort_as_bfloat16(b));
}

// MODE 0: dst0 = bf16(x).  MODE 1: dst0 = hi, dst1 = lo.
template <int MODE>
__device__ __forceinline__ void convert_one(float x, uint16_t& h, uint16_t& l) {
    h = bf16_bits(x);
    if (MODE == 1) l = bf16_bits(x - bf16_value(h));
}

// Row-major conversion: each thread handles 4 consecutive columns.
template <int MODE>
__global__ void k_cvt_rows(int rows, int cols, const float* __restrict__ src, int lds,
                           uint16_t* __restrict__ d0, uint16_t* __restrict__ d1, int ldd, int vec) {
    const int cq = (cols + 3) / 4;
    const long long total = (long long)rows * cq;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / cq);
        const int c = (int)(i - (long long)r * cq) * 4;
        const float* s = src + (size_t)r * lds + c;
        float v[4];
        if (vec && c + 3 < cols) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(s));
            v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = (c + u < cols) ? __ldg(s + u) : 0.f;
        }
        uint16_t h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) convert_one<MODE>(v[u], h[u], l[u]);
        uint16_t* o0 = d0 + (size_t)r * ldd + c;
        uint16_t* o1 = MODE == 1 ? d1 + (size_t)r * ldd + c : nullptr;
        if (vec && c + 3 < cols) {
            *reinterpret_cast<uint2*>(o0) =
                make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
            if (MODE == 1)
                *reinterpret_cast<uint2*>(o1) =
                    make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c + u < cols) {
                    o0[u] = h[u];
                    if (MODE == 1) o1[u] = l[u];
                }
        }
    }
}

// Transposed conversion through a 64 x 64 shared tile: src rows are read as
// float4 (coalesced along src rows), each dst row (a src column) is written as
// 32-bit pairs of BF16 values (a full 128-byte segment per warp).
template <int MODE>
__global__ void __launch_bounds__(256) k_cvt_transpose(int rows, int cols,
                                                       const float* __restrict__ src, int lds,
                                                       uint16_t* __restrict__ d0,
                                                       uint16_t* __restrict__ d1, int ldd,
                                                       int vec_in, int pair_out) {
    __shared__ float t[64][65];
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int idx = tid + i * 256;
        const int r = idx >> 4, c = (idx & 15) * 4;
        const int gr = r0 + r, gc = c0 + c;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (gr < rows) {
            const float* sp = src + (size_t)gr * lds + gc;
            if (vec_in && gc + 3 < cols) {
                const float4 f = __ldg(reinterpret_cast<const float4*>(sp));
                v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (gc + u < cols) v[u] = __ldg(sp + u);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) t[r][c + u] = v[u];
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = warp * 8 + j;           // dst row c0 + c
        const int gc = c0 + c;
        if (gc >= cols) break;
        const int gr = r0 + 2 * lane;         // dst columns gr, gr + 1
        uint16_t h0, l0, h1, l1;
        convert_one<MODE>(t[2 * lane][c], h0, l0);
        convert_one<MODE>(t[2 * lane + 1][c], h1, l1);
        uint16_t* o0 = d0 + (size_t)gc * ldd + gr;
        uint16_t* o1 = MODE == 1 ? d1 + (size_t)gc * ldd + gr : nullptr;
        if (pair_out && gr + 1 < rows) {
            *reinterpret_cast<uint32_t*>(o0) = h0 | ((uint32_t)h1 << 16);
            if (MODE == 1) *reinterpret_cast<uint32_t*>(o1) = l0 | ((uint32_t)l1 << 16);
        } else {
            if (gr < rows) {
                o0[0] = h0;
                if (MODE == 1) o1[0] = l0;
            }
            if (gr + 1 < rows) {
                o0[1] = h1;
                if (MODE == 1) o1[1] = l1;
            }
        }
    }
}

// Per-tile FP8 quantisation: one block per 128 x 128 tile of src.
__global__ void __launch_bounds__(256) k_quant_fp8(int rows, int cols, const float* __restrict__ src,
                                                   int lds, uint8_t* __restrict__ dst, int ldd,
                                                   float* __restrict__ scales, int ld_scales,
                                                   int transpose) {
    __shared__ float red[8];
    __shared__ uint8_t tile[128][132];
    const int ti = blockIdx.y, tj = blockIdx.x;
    const int r0 = ti * 128, c0 = tj * 128;
    const int tid = threadIdx.x;
    // pass 1: amax (|x| is exact, max is order independent)
    float amax = 0.f;
    for (int idx = tid; idx < 128 * 128; idx += 256) {
        const int r = r0 + idx / 128, c = c0 + idx % 128;
        if (r < rows && c < cols) amax = fmaxf(amax, fabsf(__ldg(src + (size_t)r * lds + c)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();
    if (tid < 32) {
        float a = tid < 8 ? red[tid] : 0.f;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        if (tid == 0) red[0] = a;
    }
    __syncthreads();
    amax = red[0];
    const float scale = amax == 0.f ? 1.f : amax / 448.f;   // IEEE division
    if (tid == 0) scales[(size_t)ti * ld_scales + tj] = scale;
    // pass 2: quantise (IEEE division, round to nearest even, saturate to +-448)
    for (int idx = tid; idx < 128 * 128; idx += 256) {
        const int rr = idx / 128, cc = idx % 128;
        const int r = r0 + rr, c = c0 + cc;
        uint8_t q = 0;
        if (r < rows && c < cols) {
            const float x = __ldg(src + (size_t)r * lds + c);
            q = (uint8_t)__nv_cvt_float_to_fp8(x / scale, __NV_SATFINITE, __NV_E4M3);
            if (!transpose) dst[(size_t)r * ldd + c] = q;
        }
        tile[rr][cc] = q;
    }
    if (transpose) {
        __syncthreads();
        for (int idx = tid; idx < 128 * 128; idx += 256) {
            const int cc = idx / 128, rr = idx % 128;   // dst row c0+cc, dst col r0+rr
            const int r = r0 + rr, c = c0 + cc;
            if (r < rows && c < cols) dst[(size_t)c * ldd + r] = tile[rr][cc];
        }
    }
}

static bool aligned(const void* p, unsigned a) { return ((uintptr_t)p % a) == 0; }

static pgk_status check_prep(int rows, int cols, const void* src, int lds, const void* dst, int ldd,
                             int transpose) {
    if (rows < 1 || cols < 1 || !src || !dst || lds < cols || ldd < (transpose ? rows : cols)) {
        set_error("bad conversion arguments (rows=%d cols=%d lds=%d ldd=%d)", rows, cols, lds, ldd);
        return PGK_ERR_INVALID_ARG;
    }
    return PGK_OK;
}

template <int MODE>
static pgk_status launch_cvt(int rows, int cols, const float* src, int lds, uint16_t* d0,
                             uint16_t* d1, int ldd, int transpose, cudaStream_t st) {
    if (transpose) {
        dim3 grid((cols + 63) / 64, (rows + 63) / 64);
        if (grid.y > 65535) {
            set_error("too many rows for the transposing conversion");
            return PGK_ERR_INVALID_ARG;
        }
        const int vec_in = aligned(src, 16) && lds % 4 == 0;
        const int pair_out = aligned(d0, 4) && ldd % 2 == 0 && (MODE == 0 || aligned(d1, 4));
        k_cvt_transpose<MODE><<<grid, 256, 0, st>>>(rows, cols, src, lds, d0, d1, ldd, vec_in,
                                                    pair_out);
    } else {
        const int vec = aligned(src, 16) && lds % 4 == 0 && aligned(d0, 8) && ldd % 4 == 0 &&
                        (MODE == 0 || aligned(d1, 8));
        const long long work = (long long)rows * ((cols + 3) / 4);
        const int blocks = (int)std::min<long long>((work + 255) / 256, 152LL * 16);
        k_cvt_rows<MODE><<<blocks, 256, 0, st>>>(rows, cols, src, lds, d0, d1, ldd, vec);
    }
    PGK_CUDA_TRY(cudaGetLastError(), "conversion launch");
    return PGK_OK;
}

pgk_status launch_quant_fp8(int rows, int cols, const float* src, int lds, uint8_t* dst, int ldd,
                            float* scales, int ld_scales, int transpose, cudaStream_t st) {
    dim3 grid((cols + 127) / 128, (rows + 127) / 128);
    if (grid.y > 65535) {
        set_error("too many rows for FP8 quantisation");
        return PGK_ERR_INVALID_ARG;
    }
    k_quant_fp8<<<grid, 256, 0, st>>>(rows, cols, src, lds, dst, ldd, scales, ld_scales, transpose);
    PGK_CUDA_TRY(cudaGetLastError(), "FP8 quantisation launch");
    return PGK_OK;
}

pgk_status launch_cvt_bf16(int rows, int cols, const float* src, int lds, uint16_t* dst, int ldd,
                           int transpose, cudaStream_t st) {
    return launch_cvt<0>(rows, cols, src, lds, dst, nullptr, ldd, transpose, st);
}

pgk_status launch_split_bf16(int rows, int cols, const float* src, int lds, uint16_t* hi,
                             uint16_t* lo, int ldd, int transpose, cudaStream_t st) {
    return launch_cvt<1>(rows, cols, src, lds, hi, lo, ldd, transpose, st);
}

}  // namespace pgk

using namespace pgk;

extern "C" {

pgk_status pgk_cvt_bf16(int rows, int cols, const float* src, int lds, uint16_t* dst, int ldd,
                        int transpose, void* stream) {
    pgk_status st = check_prep(rows, cols, src, lds, dst, ldd, transpose);
    if (st != PGK_OK) return st;
    return launch_cvt_bf16(rows, cols, src, lds, dst, ldd, transpose, (cudaStream_t)stream);
}

pgk_status pgk_split_bf16(int rows, int cols, const float* src, int lds, uint16_t* hi,
                          uint16_t* lo, int ldd, int transpose, void* stream) {
    pgk_status st = check_prep(rows, cols, src, lds, hi, ldd, transpose);
    if (st != PGK_OK) return st;
    if (!lo) {
        set_error("NULL lo output");
        return PGK_ERR_INVALID_ARG;
    }
    return launch_split_bf16(rows, cols, src, lds, hi, lo, ldd, transpose, (cudaStream_t)stream);
}

pgk_status pgk_quant_fp8(int rows, int cols, const float* src, int lds, uint8_t* dst, int ldd,
                         float* scales, int ld_scales, int transpose, void* stream) {
    pgk_status st = check_prep(rows, cols, src, lds, dst, ldd, transpose);
    if (st != PGK_OK) return st;
    if (!scales || ld_scales < (cols + 127) / 128) {
        set_error("bad scale array (ld_scales=%d, need >= %d)", ld_scales, (cols + 127) / 128);
        return PGK_ERR_INVALID_ARG;
    }
    return launch_quant_fp8(rows, cols, src, lds, dst, ldd, scales, ld_scales, transpose,
                            (cudaStream_t)stream);
}

}  // extern "C"
