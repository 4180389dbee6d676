// FP32 SIMT variants of the parametric GEMM (Section 2, Fig. "cudamul"):
//   * "paper" family: the paper's thread granularity -- thread (t0, t1) of a
//     B0 x B1 block computes s outputs of row b0*B0 + t0, columns strided by
//     B1; shared tiles A: B0 x BK and B: BK x (B1*s) (the paper uses BK = B0).
//     B0, B1, BK are runtime values (blockDim and dynamic shared memory), s is a
//     template parameter (the paper fixes S as a macro for the same reason: a
//     run-time indexed register array would live in local memory).
//     Leaves (4a,3a) and (3b,4a) of the case discussion.
//   * "direct" family: no shared memory, one output per thread; leaf (3b,4b).
//   * "rb" family: register-blocked sr x s micro tiles (simt_rb.cuh).
// Every variant handles arbitrary M, N, K >= 1 with predicated, zero-filled
// tails (the paper's k loop drops the remainder of n / B0).
#include "pgk_internal.cuh"
#include "simt_rb.cuh"

namespace pgk {

// ----------------------------------------------------------- paper family
template <int S>
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
    float acc[S];
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
            for (int w = 0; w < S; ++w) acc[w] = fmaf(a, Bs[k * BN + t1 + w * B1], acc[w]);
        }
        __syncthreads();
    }
    if (row < p.M) {
#pragma unroll
        for (int w = 0; w < S; ++w) {
            const int col = col0 + w * B1;
            if (col < p.N) {
                float* cp = p.C + (size_t)row * p.ldc + col;
                *cp = p.beta ? *cp + acc[w] : acc[w];
            }
        }
    }
}

template <int S>
__global__ void k_paper(SimtArgs p) { paper_body<S>(p); }

// Register-pressure strategy "1": the same source compiled so that a block of
// 1024 threads fits the 64K register file (at most 64 registers per thread).
template <int S>
__global__ void __launch_bounds__(1024, 1) k_paper_cap(SimtArgs p) { paper_body<S>(p); }

template <int S, bool CAP>
static cudaError_t launch_paper(const SimtArgs& p, int smem, cudaStream_t st) {
    const int BN = p.B1 * S;
    const long long tiles = (long long)((p.M + p.B0 - 1) / p.B0) * ((p.N + BN - 1) / BN);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const void* f = CAP ? (const void*)k_paper_cap<S> : (const void*)k_paper<S>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(p.B1, p.B0);
    if (CAP)
        k_paper_cap<S><<<(unsigned)tiles, block, smem, st>>>(p);
    else
        k_paper<S><<<(unsigned)tiles, block, smem, st>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------- direct family
__device__ __forceinline__ void direct_body(const SimtArgs& p) {
    const int B0 = p.B0, B1 = p.B1;
    const int tiles_n = (p.N + B1 - 1) / B1;
    const int bm = blockIdx.x / tiles_n, bn = blockIdx.x % tiles_n;
    const int row = bm * B0 + threadIdx.y, col = bn * B1 + threadIdx.x;
    if (row >= p.M || col >= p.N) return;
    const float* a = p.A + (size_t)row * p.lda;
    const float* b = p.B + col;
    float acc = 0.f;
    for (int k = 0; k < p.K; ++k) acc = fmaf(__ldg(a + k), __ldg(b + (size_t)k * p.ldb), acc);
    float* cp = p.C + (size_t)row * p.ldc + col;
    *cp = p.beta ? *cp + acc : acc;
}

__global__ void k_direct(SimtArgs p) { direct_body(p); }
__global__ void __launch_bounds__(1024, 1) k_direct_cap(SimtArgs p) { direct_body(p); }

template <bool CAP>
static cudaError_t launch_direct(const SimtArgs& p, int, cudaStream_t st) {
    const long long tiles = (long long)((p.M + p.B0 - 1) / p.B0) * ((p.N + p.B1 - 1) / p.B1);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 block(p.B1, p.B0);
    if (CAP)
        k_direct_cap<<<(unsigned)tiles, block, 0, st>>>(p);
    else
        k_direct<<<(unsigned)tiles, block, 0, st>>>(p);
    return cudaGetLastError();
}

// -------------------------------------------------------------- rb family
template <class Cfg>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB) k_rb(SimtArgs p) {
    extern __shared__ float4 smem_rb4[];
    const int tiles_m = (p.M + Cfg::BM - 1) / Cfg::BM;
    const int tiles_n = (p.N + Cfg::BN - 1) / Cfg::BN;
    int bm, bn;
    grouped_tile_coords(blockIdx.x, tiles_m, tiles_n, bm, bn);
    RbTile<Cfg>::run(p.A, p.lda, p.B, p.ldb, p.C, p.ldc, p.M, p.N, p.K, bm * Cfg::BM, bn * Cfg::BN,
                     p.beta, p.vecA, p.vecB, p.vecC, reinterpret_cast<float*>(smem_rb4));
}

template <class Cfg>
static cudaError_t launch_rb(const SimtArgs& p, int, cudaStream_t st) {
    const long long tiles =
        (long long)((p.M + Cfg::BM - 1) / Cfg::BM) * ((p.N + Cfg::BN - 1) / Cfg::BN);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (Cfg::SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_rb<Cfg>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
    }
    k_rb<Cfg><<<(unsigned)tiles, Cfg::NT, Cfg::SMEM, st>>>(p);
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

template <int B0, int B1, int SR, int S, int BK>
static void add_rb(std::vector<Variant>& v) {
    typedef RbCfg<B0, B1, SR, S, BK> Cfg;
    v.push_back(make_variant(PGK_FAM_RB, S, SR, B0, B1, BK, 0, (const void*)k_rb<Cfg>,
                             launch_rb<Cfg>, Cfg::SMEM));
}

void register_simt_variants(std::vector<Variant>& v) {
    v.push_back(make_variant(PGK_FAM_PAPER, 1, 1, 0, 0, 0, 0, (const void*)k_paper<1>, launch_paper<1, false>, 0));
    v.push_back(make_variant(PGK_FAM_PAPER, 2, 1, 0, 0, 0, 0, (const void*)k_paper<2>, launch_paper<2, false>, 0));
    v.push_back(make_variant(PGK_FAM_PAPER, 4, 1, 0, 0, 0, 0, (const void*)k_paper<4>, launch_paper<4, false>, 0));
    v.push_back(make_variant(PGK_FAM_PAPER, 8, 1, 0, 0, 0, 0, (const void*)k_paper<8>, launch_paper<8, false>, 0));
    v.push_back(make_variant(PGK_FAM_PAPER, 1, 1, 0, 0, 0, 1, (const void*)k_paper_cap<1>, launch_paper<1, true>, 0));
    v.push_back(make_variant(PGK_FAM_PAPER, 2, 1, 0, 0, 0, 1, (const void*)k_paper_cap<2>, launch_paper<2, true>, 0));
    v.push_back(make_variant(PGK_FAM_PAPER, 4, 1, 0, 0, 0, 1, (const void*)k_paper_cap<4>, launch_paper<4, true>, 0));
    v.push_back(make_variant(PGK_FAM_PAPER, 8, 1, 0, 0, 0, 1, (const void*)k_paper_cap<8>, launch_paper<8, true>, 0));
    v.push_back(make_variant(PGK_FAM_DIRECT, 1, 1, 0, 0, 0, 0, (const void*)k_direct, launch_direct<false>, 0));
    v.push_back(make_variant(PGK_FAM_DIRECT, 1, 1, 0, 0, 0, 1, (const void*)k_direct_cap, launch_direct<true>, 0));
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
