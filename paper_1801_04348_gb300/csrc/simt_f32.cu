// FP32 SIMT variants of the parametric GEMM (Section 2, Fig. "cudamul"):
//   * "paper" family: the paper's thread granularity -- thread (t0, t1) of a
//     B0 x B1 block computes s outputs of row b0*B0 + t0, columns strided by
//     B1; shared tiles A: B0 x BK and B: BK x (B1*s) (the paper uses BK = B0).
//     B0, B1, BK are runtime values (blockDim and dynamic shared memory), s is a
//     template parameter (the paper fixes S as a macro for the same reason: a
//     run-time indexed register array would live in local memory).
//     Leaves (4a,3a) and (3b,4a) of the case discussion.
//   * "direct" family: no shared memory, one output per thread; leaf (3b,4b).
//   * "rb" family: register-blocked sr x s micro tiles (simt_rb.cuh).  When the
//     output has fewer tiles than SMs and K >= 4096 the launch splits K into
//     slices (at least 1024 deep); slice partials land in a library workspace and
//     a second kernel adds them in slice order.
// Every variant handles arbitrary M, N, K >= 1 with predicated, zero-filled
// tails (the paper's k loop drops the remainder of n / B0).
#include <algorithm>

#include "pgk_internal.cuh"
#include "simt_rb.cuh"

namespace pgk {

// ----------------------------------------------------------- paper family
template <int S, bool INT>
__device__ __forceinline__ void paper_body(const SimtArgs& p) {
    extern __shared__ float smem_paper[];
    const int B0 = p.B0, B1 = p.B1, BK = p.BK;
    const int t0 = threadIdx.y, t1 = threadIdx.x;
    const int tid = t0 * B1 + t1, nthr = B0 * B1;
    const int BN = B1 * S;
    const int tiles_n = (p.N + BN - 1) / BN;
    const int bm = blockIdx.x / tiles_n, bn = blockIdx.x % tiles_n;
    float* As = smem_paper;            // B0 x BK
    float* Bs = smem_paper + B0 * BK;  // BK x BN
    const int row = bm * B0 + t0;
    const int col0 = bn * BN + t1;
    float acc[S];   // FP32 values, or int32 words for INT
#pragma unroll
    for (int w = 0; w < S; ++w) acc[w] = 0.f;

    for (int k0 = 0; k0 < p.K; k0 += BK) {
        for (int i = tid; i < B0 * BK; i += nthr) {
            const int r = i / BK, c = i - r * BK;
            const int gr = bm * B0 + r, gc = k0 + c;
            As[i] = (gr < p.M && gc < p.K) ? __ldg(p.A + (size_t)gr * p.lda + gc) : 0.f;
        }
        for (int i = tid; i < BK * BN; i += nthr) {
            const int r = i / BN, c = i - r * BN;
            const int gr = k0 + r, gc = bn * BN + c;
            Bs[i] = (gr < p.K && gc < p.N) ? __ldg(p.B + (size_t)gr * p.ldb + gc) : 0.f;
        }
        __syncthreads();
        const int kmax = min(BK, p.K - k0);
        for (int k = 0; k < kmax; ++k) {
            const float a = As[t0 * BK + k];
#pragma unroll
            for (int w = 0; w < S; ++w) {
                const float b = Bs[k * BN + t1 + w * B1];
                acc[w] = INT ? __uint_as_float(__float_as_uint(acc[w]) +
                                               __float_as_uint(a) * __float_as_uint(b))
                             : fmaf(a, b, acc[w]);
            }
        }
        __syncthreads();
    }
    if (row < p.M) {
#pragma unroll
        for (int w = 0; w < S; ++w) {
            const int col = col0 + w * B1;
            if (col < p.N) {
                float* cp = p.C + (size_t)row * p.ldc + col;
                *cp = p.beta ? add32<INT>(*cp, acc[w]) : acc[w];
            }
        }
    }
}

template <int S, bool INT>
__global__ void k_paper(SimtArgs p) { paper_body<S, INT>(p); }

// Register-pressure strategy "1": the same source compiled so that a block of
// 1024 threads fits the 64K register file (at most 64 registers per thread).
template <int S, bool INT>
__global__ void __launch_bounds__(1024, 1) k_paper_cap(SimtArgs p) { paper_body<S, INT>(p); }

template <int S, bool CAP, bool INT>
static cudaError_t launch_paper(const SimtArgs& p, int smem, cudaStream_t st) {
    const int BN = p.B1 * S;
    const long long tiles = (long long)((p.M + p.B0 - 1) / p.B0) * ((p.N + BN - 1) / BN);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const void* f = CAP ? (const void*)k_paper_cap<S, INT> : (const void*)k_paper<S, INT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(p.B1, p.B0);
    if (CAP)
        k_paper_cap<S, INT><<<(unsigned)tiles, block, smem, st>>>(p);
    else
        k_paper<S, INT><<<(unsigned)tiles, block, smem, st>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------- direct family
template <bool INT>
__device__ __forceinline__ void direct_body(const SimtArgs& p) {
    const int B0 = p.B0, B1 = p.B1;
    const int tiles_n = (p.N + B1 - 1) / B1;
    const int bm = blockIdx.x / tiles_n, bn = blockIdx.x % tiles_n;
    const int row = bm * B0 + threadIdx.y, col = bn * B1 + threadIdx.x;
    if (row >= p.M || col >= p.N) return;
    const float* a = p.A + (size_t)row * p.lda;
    const float* b = p.B + col;
    float acc = 0.f;
    for (int k = 0; k < p.K; ++k) {
        const float x = __ldg(a + k), y = __ldg(b + (size_t)k * p.ldb);
        acc = INT ? __uint_as_float(__float_as_uint(acc) + __float_as_uint(x) * __float_as_uint(y))
                  : fmaf(x, y, acc);
    }
    float* cp = p.C + (size_t)row * p.ldc + col;
    *cp = p.beta ? add32<INT>(*cp, acc) : acc;
}

template <bool INT>
__global__ void k_direct(SimtArgs p) { direct_body<INT>(p); }
template <bool INT>
__global__ void __launch_bounds__(1024, 1) k_direct_cap(SimtArgs p) { direct_body<INT>(p); }

template <bool CAP, bool INT>
static cudaError_t launch_direct(const SimtArgs& p, int, cudaStream_t st) {
    const long long tiles = (long long)((p.M + p.B0 - 1) / p.B0) * ((p.N + p.B1 - 1) / p.B1);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 block(p.B1, p.B0);
    if (CAP)
        k_direct_cap<INT><<<(unsigned)tiles, block, 0, st>>>(p);
    else
        k_direct<INT><<<(unsigned)tiles, block, 0, st>>>(p);
    return cudaGetLastError();
}

// -------------------------------------------------------------- rb family
template <class Cfg, bool INT>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB) k_rb(SimtArgs p) {
    extern __shared__ float4 smem_rb4[];
    const int tiles_m = (p.M + Cfg::BM - 1) / Cfg::BM;
    const int tiles_n = (p.N + Cfg::BN - 1) / Cfg::BN;
    int bm, bn;
    grouped_tile_coords(blockIdx.x, tiles_m, tiles_n, bm, bn);
    RbTile<Cfg, INT>::run(p.A, p.lda, p.B, p.ldb, p.C, p.ldc, p.M, p.N, p.K, bm * Cfg::BM,
                          bn * Cfg::BN, p.beta, p.vecA, p.vecB, p.vecC,
                          reinterpret_cast<float*>(smem_rb4));
}

// Split-K: blockIdx.y selects a slice [y * kslice, (y + 1) * kslice) of K; the
// tile's partial product goes to slice y of the workspace P (M x N each).
template <class Cfg, bool INT>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB) k_rb_splitk(SimtArgs p, float* P, int kslice) {
    extern __shared__ float4 smem_sk4[];
    const int tiles_m = (p.M + Cfg::BM - 1) / Cfg::BM;
    const int tiles_n = (p.N + Cfg::BN - 1) / Cfg::BN;
    int bm, bn;
    grouped_tile_coords(blockIdx.x, tiles_m, tiles_n, bm, bn);
    const int k0 = blockIdx.y * kslice;
    const int kn = min(kslice, p.K - k0);
    float* Py = P + (size_t)blockIdx.y * p.M * p.N;
    RbTile<Cfg, INT>::run(p.A + k0, p.lda, p.B + (size_t)k0 * p.ldb, p.ldb, Py, p.N, p.M, p.N, kn,
                          bm * Cfg::BM, bn * Cfg::BN, 0, p.vecA, p.vecB, (p.N & 3) == 0,
                          reinterpret_cast<float*>(smem_sk4));
}

// C = (beta ? C : 0) + sum over slices of P, slices added in order.
template <bool INT>
__global__ void k_splitk_reduce(SimtArgs p, const float* __restrict__ P, int splits) {
    const long long total = (long long)p.M * p.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / p.N), c = (int)(i - (long long)r * p.N);
        float acc = P[i];
        for (int y = 1; y < splits; ++y) acc = add32<INT>(acc, P[(size_t)y * total + i]);
        float* cp = p.C + (size_t)r * p.ldc + c;
        *cp = p.beta ? add32<INT>(*cp, acc) : acc;
    }
}

template <class Cfg, bool INT>
static cudaError_t launch_rb(const SimtArgs& p, int, cudaStream_t st) {
    const long long tiles =
        (long long)((p.M + Cfg::BM - 1) / Cfg::BM) * ((p.N + Cfg::BN - 1) / Cfg::BN);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    // Fewer output tiles than the GPU holds resident blocks, on a long K: split K
    // into as many slices as still fit in one wave of resident blocks (slices of at
    // least 1024, a multiple of BK); a wave and a few blocks would cost two waves.
    pgk_machine m;
    int splits = 1;
    if (p.K >= 4096 && current_machine(&m, NULL) == PGK_OK) {
        if (Cfg::SMEM > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute((const void*)k_rb_splitk<Cfg, INT>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg::SMEM);
            if (e != cudaSuccess) return e;
        }
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_rb_splitk<Cfg, INT>,
                                                          Cfg::NT, Cfg::SMEM) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
        }
        const long long slots = (long long)std::max(per_sm, 1) * m.sm_count;
        if (tiles < slots) {
            splits = (int)std::min<long long>(slots / tiles, 16);
            splits = std::min(splits, p.K / 1024);
        }
    }
    if (splits >= 2) {
        const int kslice = ((p.K + splits - 1) / splits + Cfg::BK - 1) / Cfg::BK * Cfg::BK;
        splits = (p.K + kslice - 1) / kslice;
        pgk_status ws;
        float* P = (float*)workspace(WS_SPLITK, sizeof(float) * (size_t)splits * p.M * p.N, &ws);
        if (!P) return cudaErrorMemoryAllocation;
        k_rb_splitk<Cfg, INT><<<dim3((unsigned)tiles, (unsigned)splits), Cfg::NT, Cfg::SMEM, st>>>(
            p, P, kslice);
        const long long total = (long long)p.M * p.N;
        const int blocks = (int)std::min<long long>((total + 255) / 256, 4LL * m.sm_count);
        k_splitk_reduce<INT><<<blocks, 256, 0, st>>>(p, P, splits);
        return cudaGetLastError();
    }
    if (Cfg::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_rb<Cfg, INT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    k_rb<Cfg, INT><<<(unsigned)tiles, Cfg::NT, Cfg::SMEM, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------ registration
static Variant make_variant(int family, int s, int sr, int B0, int B1, int tile, int regopt,
                            const void* f, simt_launch_fn l, int smem) {
    Variant v;
    v.info.family = family;
    v.info.s = s;
    v.info.sr = sr;
    v.info.B0 = B0;
    v.info.B1 = B1;
    v.info.tile = tile;
    v.info.regopt = regopt;
    v.info.regs = -1;
    v.info.max_threads = -1;
    v.func = f;
    v.launch = l;
    v.smem_fixed = smem;
    return v;
}

template <int B0, int B1, int SR, int S, int BK, bool INT = false>
static void add_rb(std::vector<Variant>& v) {
    typedef RbCfg<B0, B1, SR, S, BK> Cfg;
    v.push_back(make_variant(INT ? PGK_FAM_RB_I32 : PGK_FAM_RB, S, SR, B0, B1, BK, 0,
                             (const void*)k_rb<Cfg, INT>, launch_rb<Cfg, INT>, Cfg::SMEM));
}

template <bool INT>
static void add_paper_and_direct(std::vector<Variant>& v) {
    const int fp = INT ? PGK_FAM_PAPER_I32 : PGK_FAM_PAPER;
    const int fd = INT ? PGK_FAM_DIRECT_I32 : PGK_FAM_DIRECT;
    v.push_back(make_variant(fp, 1, 1, 0, 0, 0, 0, (const void*)k_paper<1, INT>, launch_paper<1, false, INT>, 0));
    v.push_back(make_variant(fp, 2, 1, 0, 0, 0, 0, (const void*)k_paper<2, INT>, launch_paper<2, false, INT>, 0));
    v.push_back(make_variant(fp, 4, 1, 0, 0, 0, 0, (const void*)k_paper<4, INT>, launch_paper<4, false, INT>, 0));
    v.push_back(make_variant(fp, 8, 1, 0, 0, 0, 0, (const void*)k_paper<8, INT>, launch_paper<8, false, INT>, 0));
    v.push_back(make_variant(fp, 1, 1, 0, 0, 0, 1, (const void*)k_paper_cap<1, INT>, launch_paper<1, true, INT>, 0));
    v.push_back(make_variant(fp, 2, 1, 0, 0, 0, 1, (const void*)k_paper_cap<2, INT>, launch_paper<2, true, INT>, 0));
    v.push_back(make_variant(fp, 4, 1, 0, 0, 0, 1, (const void*)k_paper_cap<4, INT>, launch_paper<4, true, INT>, 0));
    v.push_back(make_variant(fp, 8, 1, 0, 0, 0, 1, (const void*)k_paper_cap<8, INT>, launch_paper<8, true, INT>, 0));
    v.push_back(make_variant(fd, 1, 1, 0, 0, 0, 0, (const void*)k_direct<INT>, launch_direct<false, INT>, 0));
    v.push_back(make_variant(fd, 1, 1, 0, 0, 0, 1, (const void*)k_direct_cap<INT>, launch_direct<true, INT>, 0));
}

void register_simt_variants(std::vector<Variant>& v) {
    add_paper_and_direct<false>(v);
    add_paper_and_direct<true>(v);
    // int32 register-blocked variants
    add_rb<16, 16, 8, 8, 8, true>(v);
    add_rb<16, 16, 8, 8, 16, true>(v);
    add_rb<16, 16, 4, 4, 8, true>(v);
    add_rb<8, 8, 8, 8, 8, true>(v);
    // register-blocked variants: (B0, B1, sr, s, BK)
    add_rb<16, 16, 8, 8, 8>(v);
    add_rb<16, 16, 8, 8, 16>(v);
    add_rb<16, 16, 8, 4, 8>(v);
    add_rb<16, 16, 4, 8, 8>(v);
    add_rb<16, 16, 4, 4, 8>(v);
    add_rb<16, 16, 4, 4, 16>(v);
    add_rb<8, 16, 8, 8, 8>(v);
    add_rb<8, 16, 8, 8, 16>(v);
    add_rb<16, 8, 8, 8, 8>(v);
    add_rb<16, 8, 8, 8, 16>(v);
    add_rb<8, 8, 8, 8, 8>(v);
    add_rb<8, 8, 8, 8, 16>(v);
    add_rb<8, 32, 8, 4, 8>(v);
    add_rb<32, 8, 4, 8, 8>(v);
    add_rb<16, 32, 8, 4, 8>(v);
    add_rb<32, 16, 4, 8, 8>(v);
    add_rb<16, 32, 8, 8, 8>(v);
    add_rb<32, 16, 8, 8, 8>(v);
    add_rb<16, 16, 8, 8, 32>(v);
    add_rb<16, 16, 8, 16, 8>(v);
    add_rb<16, 16, 16, 8, 8>(v);
    add_rb<16, 16, 16, 8, 16>(v);
    add_rb<16, 16, 8, 16, 16>(v);
}

}  // namespace pgk
