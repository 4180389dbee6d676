// Low-precision operand preparation for the tensor-core forms: FP32 -> BF16
// (round to nearest even), the split x = hi + lo with hi = bf16(x),
// lo = bf16(x - hi), and per-128x128-tile scaled FP8 E4M3 (scale = amax / 448,
// q = e4m3_rn_satfinite(x / scale)).  Each kernel optionally writes its output
// transposed, which turns B (K x N) into the K-major N x K operand the
// tensor-core kernels read.  All are HBM-bound streaming kernels.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <climits>

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

// Four consecutive elements of row r starting at column c (c a multiple of 4),
// zero outside the matrix; one 128-bit load when the row allows it.
__device__ __forceinline__ float4 load_row4(const float* __restrict__ src, int lds, int rows,
                                            int cols, int r, int c, int vec) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r >= rows || c >= cols) return v;
    const float* p = src + (size_t)r * lds + c;
    if (vec && c + 3 < cols) return __ldg(reinterpret_cast<const float4*>(p));
    v.x = __ldg(p);
    if (c + 1 < cols) v.y = __ldg(p + 1);
    if (c + 2 < cols) v.z = __ldg(p + 2);
    if (c + 3 < cols) v.w = __ldg(p + 3);
    return v;
}

__device__ __forceinline__ uint32_t e4m3(float x, float scale) {
    // binary32 division rounded to nearest, then E4M3 round to nearest even, saturated
    return (uint32_t)__nv_cvt_float_to_fp8(__fdiv_rn(x, scale), __NV_SATFINITE, __NV_E4M3);
}

// Writes the four codes of word w (byte k = element k) to dst + off, or the
// in-range ones among them (n of 4) one by one.
__device__ __forceinline__ void store_codes(uint8_t* __restrict__ dst, size_t off, uint32_t w,
                                            int n, int vec) {
    if (n <= 0) return;
    if (vec && n == 4) {
        *reinterpret_cast<uint32_t*>(dst + off) = w;
        return;
    }
    for (int k = 0; k < n; ++k) dst[off + k] = (uint8_t)(w >> (8 * k));
}

// Per-tile FP8 quantisation: one block of QUANT_THREADS per 128 x 128 tile.  The
// tile is read from global memory once, into registers: warp w, lane l holds rows
// 16 i + w, columns 4 l .. 4 l + 3 (each warp load is one 512-byte row segment).
// The block's amax gives the scale.  Row output: each warp writes 128 contiguous
// bytes of a row.  Transposed output: the codes go through a shared tile with a
// row pitch of 129 bytes (conflict-free both for the row-wise stores and for the
// column-wise reads), and each warp writes whole 128-byte rows of the transpose.
static constexpr int QUANT_THREADS = 512;
static constexpr int QUANT_PITCH = 129;

// Problem of a grouped work item: the largest g with prefix[g] <= item.
__device__ __forceinline__ int grouped_item_problem(const int* __restrict__ prefix, int G, int item) {
    int lo = 0, hi = G - 1;   // largest g with prefix[g] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One 128 x 128 tile at (r0, c0) of src (rows x cols, zero outside): its scale goes
// to *scale_out, its codes to dst, in the source layout for columns below wbound
// (rows mode) or transposed for source rows below wbound (the K extent; entries
// between the source size and wbound are the codes of zeros).  Called by every
// thread of a QUANT_THREADS block; red and tile are the block's shared buffers.
template <bool TRANS>
__device__ __forceinline__ void quant_tile(const float* __restrict__ src, int lds, int rows, int cols,
                                           int wbound, int r0, int c0, uint8_t* __restrict__ dst,
                                           int ldd, float* scale_out, int vec_in, int vec_out,
                                           float* red, uint8_t* tile) {
    constexpr int WARPS = QUANT_THREADS / 32;          // 16
    constexpr int NV = 128 * 128 / 4 / QUANT_THREADS;  // float4 per thread: 8
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = load_row4(src, lds, rows, cols, r0 + i * WARPS + warp, c0 + lane * 4, vec_in);
    // amax (|x| is exact and max is order independent; out-of-range elements are 0)
    float amax = 0.f;
#pragma unroll
    for (int i = 0; i < NV; ++i)
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[i].x), fabsf(v[i].y)),
                                 fmaxf(fabsf(v[i].z), fabsf(v[i].w))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) red[warp] = amax;
    __syncthreads();
    amax = red[0];
#pragma unroll
    for (int w = 1; w < WARPS; ++w) amax = fmaxf(amax, red[w]);
    const float scale = amax == 0.f ? 1.f : __fdiv_rn(amax, 448.f);
    if (threadIdx.x == 0) *scale_out = scale;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int rr = i * WARPS + warp, cc = lane * 4;   // position in the tile
        const uint32_t w = e4m3(v[i].x, scale) | (e4m3(v[i].y, scale) << 8) |
                           (e4m3(v[i].z, scale) << 16) | (e4m3(v[i].w, scale) << 24);
        if (TRANS) {
#pragma unroll
            for (int k = 0; k < 4; ++k) tile[rr * QUANT_PITCH + cc + k] = (uint8_t)(w >> (8 * k));
        } else if (r0 + rr < rows) {
            store_codes(dst, (size_t)(r0 + rr) * ldd + c0 + cc, w, min(4, wbound - c0 - cc), vec_out);
        }
    }
    if (TRANS) {
        __syncthreads();
        // output row j of the tile = source column c0 + j; lane l writes source rows
        // r0 + 4 l .. r0 + 4 l + 3 of it
#pragma unroll
        for (int jj = 0; jj < 128 / WARPS; ++jj) {
            const int j = warp * (128 / WARPS) + jj;
            if (c0 + j >= cols) break;
            const uint8_t* col = tile + (4 * lane) * QUANT_PITCH + j;
            const uint32_t w = (uint32_t)col[0] | ((uint32_t)col[QUANT_PITCH] << 8) |
                               ((uint32_t)col[2 * QUANT_PITCH] << 16) |
                               ((uint32_t)col[3 * QUANT_PITCH] << 24);
            store_codes(dst, (size_t)(c0 + j) * ldd + r0 + 4 * lane, w, min(4, wbound - r0 - 4 * lane),
                        vec_out);
        }
        __syncthreads();   // the shared tile may be reused by the block's next tile
    }
}

template <bool TRANS>
__global__ void __launch_bounds__(QUANT_THREADS) k_quant_fp8(int rows, int cols,
                                                             const float* __restrict__ src, int lds,
                                                             uint8_t* __restrict__ dst, int ldd,
                                                             float* __restrict__ scales, int ld_scales,
                                                             int vec_in, int vec_out) {
    __shared__ float red[QUANT_THREADS / 32];
    __shared__ uint8_t tile[TRANS ? 128 * QUANT_PITCH : 1];
    quant_tile<TRANS>(src, lds, rows, cols, TRANS ? rows : cols, blockIdx.y * 128, blockIdx.x * 128,
                      dst, ldd, scales + (size_t)blockIdx.y * ld_scales + blockIdx.x, vec_in, vec_out,
                      red, tile);
}

// Grouped quantisation: 128 x 128 tile items over every problem (numbered problem
// after problem, prefix[g] = first item of problem g).  Problem g's codes go to
// rows dst_row .. of the packed array (row stride ldd, zero codes up to `width`
// along K), its tile scales to scales + scale_off with row stride ld_scales (A:
// one row per 128-row block, B: one row per 128-deep K chunk).
template <bool TRANS>
__global__ void __launch_bounds__(QUANT_THREADS) k_quant_fp8_grouped(const GQuant* __restrict__ probs,
                                                                     const int* __restrict__ prefix,
                                                                     int G, int total,
                                                                     uint8_t* __restrict__ dst,
                                                                     long long ldd,
                                                                     float* __restrict__ scales,
                                                                     int ld_scales) {
    __shared__ float red[QUANT_THREADS / 32];
    __shared__ uint8_t tile[TRANS ? 128 * QUANT_PITCH : 1];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int g = grouped_item_problem(prefix, G, item);
        const GQuant q = probs[g];
        const int local = item - __ldg(prefix + g);
        // rows mode: tiles over rows x width; transposed: over width x cols
        const int tcols = TRANS ? (q.cols + 127) / 128 : q.width / 128;
        const int ti = local / tcols, tj = local % tcols;
        float* so = TRANS ? scales + (size_t)ti * ld_scales + q.scale_off + tj
                          : scales + (size_t)(q.scale_off + ti) * ld_scales + tj;
        quant_tile<TRANS>(q.src, q.lds, q.rows, q.cols, q.width, ti * 128, tj * 128,
                          dst + (size_t)q.dst_row * ldd, (int)ldd, so, q.vec, 1, red, tile);
        __syncthreads();   // red is reused by the next item
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
    const int vec_in = aligned(src, 16) && lds % 4 == 0;
    const int vec_out = aligned(dst, 4) && ldd % 4 == 0;
    if (transpose)
        k_quant_fp8<true><<<grid, QUANT_THREADS, 0, st>>>(rows, cols, src, lds, dst, ldd, scales,
                                                          ld_scales, vec_in, vec_out);
    else
        k_quant_fp8<false><<<grid, QUANT_THREADS, 0, st>>>(rows, cols, src, lds, dst, ldd, scales,
                                                           ld_scales, vec_in, vec_out);
    PGK_CUDA_TRY(cudaGetLastError(), "FP8 quantisation launch");
    return PGK_OK;
}

// ------------------------------------------------------ grouped conversion
// Every problem of a grouped tensor-core GEMM converted in one launch into a
// packed workspace: problem g's matrix (rows x cols FP32, stride lds) becomes
// destination rows dst_row .. of width `width` (zeros beyond the source), or,
// transposed, destination rows dst_row + c (one per source column) whose first
// `width` entries hold source rows 0 .. width - 1 (zeros beyond `rows`).  The
// work items are 64 x 64 tiles of the (padded) source, numbered problem after
// problem; prefix[g] is the first item of problem g.

// One 64 x 64 work item of problem q (item `local` of that problem).
template <int MODE, bool TRANS>
__device__ __forceinline__ void cvt_grouped_item(const GCvt& q, int local, uint16_t* __restrict__ d0,
                                                 uint16_t* __restrict__ d1, long long ldd,
                                                 float (*t)[65]) {
    const int tid = threadIdx.x;
    // tile grid over the padded source: TRANS covers width x cols, else rows x width
    const int tcols = TRANS ? (q.cols + 63) / 64 : (q.width + 63) / 64;
    const int r0 = (local / tcols) * 64, c0 = (local % tcols) * 64;
    if (!TRANS) {
        // direct: 64 rows x 64 columns, 4 quads per thread, zeros beyond cols
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = tid + i * 256;
            const int r = r0 + (idx >> 4), c = c0 + (idx & 15) * 4;
            if (r >= q.rows || c >= q.width) continue;
            float v[4];
            const float* sp = q.src + (size_t)r * q.lds + c;
            if (q.vec && c + 3 < q.cols) {
                const float4 f = __ldg(reinterpret_cast<const float4*>(sp));
                v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = (c + u < q.cols) ? __ldg(sp + u) : 0.f;
            }
            uint16_t h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) convert_one<MODE>(v[u], h[u], l[u]);
            const size_t o = (size_t)(q.dst_row + r) * ldd + c;   // width is a multiple of 4
            *reinterpret_cast<uint2*>(d0 + o) =
                make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
            if (MODE == 1)
                *reinterpret_cast<uint2*>(d1 + o) =
                    make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
        }
    } else {
        // transposed: source rows r0 .. r0 + 63 (zeros beyond rows), columns c0 .. c0 + 63
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = tid + i * 256;
            const int r = idx >> 4, c = (idx & 15) * 4;
            const int gr = r0 + r, gc = c0 + c;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (gr < q.rows) {
                const float* sp = q.src + (size_t)gr * q.lds + gc;
                if (q.vec && gc + 3 < q.cols) {
                    const float4 f = __ldg(reinterpret_cast<const float4*>(sp));
                    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (gc + u < q.cols) v[u] = __ldg(sp + u);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) t[r][c + u] = v[u];
        }
        __syncthreads();
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = warp * 8 + j;            // destination row dst_row + c0 + c
            const int gc = c0 + c;
            const int gr = r0 + 2 * lane;          // destination columns gr, gr + 1
            if (gc < q.cols && gr < q.width) {     // width is even
                uint16_t h0, l0, h1, l1;
                convert_one<MODE>(t[2 * lane][c], h0, l0);
                convert_one<MODE>(t[2 * lane + 1][c], h1, l1);
                const size_t o = (size_t)(q.dst_row + gc) * ldd + gr;
                *reinterpret_cast<uint32_t*>(d0 + o) = h0 | ((uint32_t)h1 << 16);
                if (MODE == 1) *reinterpret_cast<uint32_t*>(d1 + o) = l0 | ((uint32_t)l1 << 16);
            }
        }
        __syncthreads();   // the tile is reused by the next item
    }
}

// Both operands of every problem in one launch: items [0, totalA) convert the A_g
// (rows), items [totalA, totalA + totalB) the B_g (transposed); a block's item,
// and so its branch, is the same for all its threads.
template <int MODE>
__global__ void __launch_bounds__(256) k_cvt_grouped(const GCvt* __restrict__ pa,
                                                     const int* __restrict__ prefa, int totalA,
                                                     uint16_t* __restrict__ a0, uint16_t* __restrict__ a1,
                                                     const GCvt* __restrict__ pb,
                                                     const int* __restrict__ prefb, int totalB,
                                                     uint16_t* __restrict__ b0, uint16_t* __restrict__ b1,
                                                     int G, long long ldd) {
    __shared__ float t[64][65];
    for (int item = blockIdx.x; item < totalA + totalB; item += gridDim.x) {
        if (item < totalA) {
            const int g = grouped_item_problem(prefa, G, item);
            cvt_grouped_item<MODE, false>(pa[g], item - __ldg(prefa + g), a0, a1, ldd, t);
        } else {
            const int j = item - totalA;
            const int g = grouped_item_problem(prefb, G, j);
            cvt_grouped_item<MODE, true>(pb[g], j - __ldg(prefb + g), b0, b1, ldd, t);
        }
    }
}

pgk_status launch_cvt_grouped(int mode, const GCvt* pa, const int* prefa, int totalA, uint16_t* a0,
                              uint16_t* a1, const GCvt* pb, const int* prefb, int totalB,
                              uint16_t* b0, uint16_t* b1, int G, long long ldd, cudaStream_t st) {
    const long long total = (long long)totalA + totalB;
    if (total < 1) return PGK_OK;
    if (total > INT_MAX) {
        set_error("grouped conversion: too many work items");
        return PGK_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    PGK_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    PGK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int grid = (int)std::min<long long>(total, std::max(sms, 1) * 8);
    if (mode == 0)
        k_cvt_grouped<0><<<grid, 256, 0, st>>>(pa, prefa, totalA, a0, a1, pb, prefb, totalB, b0, b1,
                                               G, ldd);
    else
        k_cvt_grouped<1><<<grid, 256, 0, st>>>(pa, prefa, totalA, a0, a1, pb, prefb, totalB, b0, b1,
                                               G, ldd);
    PGK_CUDA_TRY(cudaGetLastError(), "grouped conversion launch");
    return PGK_OK;
}

pgk_status launch_quant_fp8_grouped(int transpose, const GQuant* probs, const int* prefix, int G,
                                    int total, uint8_t* dst, long long ldd, float* scales,
                                    int ld_scales, cudaStream_t st) {
    if (total < 1) return PGK_OK;
    int dev = 0, sms = 0;
    PGK_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    PGK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int grid = std::min(total, std::max(sms, 1) * 2);
    if (transpose)
        k_quant_fp8_grouped<true><<<grid, QUANT_THREADS, 0, st>>>(probs, prefix, G, total, dst, ldd,
                                                                 scales, ld_scales);
    else
        k_quant_fp8_grouped<false><<<grid, QUANT_THREADS, 0, st>>>(probs, prefix, G, total, dst, ldd,
                                                                  scales, ld_scales);
    PGK_CUDA_TRY(cudaGetLastError(), "grouped FP8 quantisation launch");
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
