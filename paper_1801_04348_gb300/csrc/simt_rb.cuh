// Register-blocked FP32 SIMT tile (the "rb" family).
//
// Extends the thread granularity of the paper's kernel (Fig. "cudamul": each
// thread of a B0 x B1 block computes s outputs of a row, strided by ub1 = B1)
// to an sr x s micro tile per thread.  Columns are taken in groups of four
// consecutive outputs strided by 4*B1 (rows likewise by 4*B0), so every global
// access stays coalesced, as the paper requires, and every shared-memory
// fragment read is one 128-bit load.  The K loop stages BK-deep tiles of A and B
// through two shared-memory buffers: while one buffer feeds the FFMA loop the
// next tile's global loads are in flight in registers.
#pragma once

#include "pgk_internal.cuh"

namespace pgk {

template <int B0_, int B1_, int SR_, int S_, int BK_>
struct RbCfg {
    static constexpr int B0 = B0_, B1 = B1_, SR = SR_, S = S_, BK = BK_;
    static constexpr int NT = B0 * B1;
    static constexpr int BM = B0 * SR, BN = B1 * S;
    static constexpr int LDAS = BM + 4;            // padded row of A^T in shared memory
    static constexpr int LDBS = BN + 4;            // padded row of B in shared memory
    static constexpr int A_ELEMS = BK * LDAS, B_ELEMS = BK * LDBS;
    static constexpr int SMEM = 2 * (A_ELEMS + B_ELEMS) * 4;   // = 8 BK (BM + BN + 8)
    static constexpr int NA4 = BM * BK / 4, NB4 = BK * BN / 4;
    static constexpr int LA = (NA4 + NT - 1) / NT, LB = (NB4 + NT - 1) / NT;
    static constexpr int MINB = SR * S > 64 ? 1 : (NT <= 128 ? 4 : (NT <= 256 ? 2 : 1));
    static_assert(SR % 4 == 0 && S % 4 == 0 && BK % 4 == 0, "micro tile in float4 groups");
};

// Blackwell's paired FP32 FMA: two IEEE fused multiply-adds (the same rounding
// as fmaf) in one instruction on a 64-bit register pair, which halves the
// issue slots the contraction needs.
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void fma2(uint64_t& c, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(a), "l"(b));
}
__device__ __forceinline__ float lo32(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi32(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// c + x on 32-bit words: FP32 addition, or int32 addition modulo 2^32.
template <bool INT>
__device__ __forceinline__ float add32(float c, float x) {
    if (INT) return __uint_as_float(__float_as_uint(c) + __float_as_uint(x));
    return c + x;
}

// Blocks visit tiles in groups of 8 tile-rows so that concurrently resident
// blocks share panels of A and B in L2.
__device__ __forceinline__ void grouped_tile_coords(int pid, int tiles_m, int tiles_n, int& bm,
                                                    int& bn) {
    const int G = 8;
    const int per_group = G * tiles_n;
    const int g = pid / per_group;
    const int first = g * G;
    const int gm = min(tiles_m - first, G);
    const int r = pid - g * per_group;
    bm = first + r % gm;
    bn = r / gm;
}

// INT = true: the same tile on int32 words (the paper's data type, Fig. "cudamul"):
// the loaders move 32-bit words unchanged and the contraction is an unsigned
// multiply-add, i.e. two's-complement arithmetic modulo 2^32.
template <class Cfg, bool INT = false>
struct RbTile {
    // Global -> registers: A tile rows [row0, row0+BM), cols [k0, k0+BK) as float4 along K.
    static __device__ __forceinline__ void load_a(float4 (&ra)[Cfg::LA], const float* __restrict__ A,
                                                  int lda, int M, int K, int row0, int k0, int tid,
                                                  int vec) {
#pragma unroll
        for (int i = 0; i < Cfg::LA; ++i) {
            const int idx = tid + i * Cfg::NT;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (Cfg::NA4 % Cfg::NT == 0 || idx < Cfg::NA4) {
                const int m = idx / (Cfg::BK / 4);
                const int kq = idx % (Cfg::BK / 4);
                const int gm = row0 + m, gk = k0 + 4 * kq;
                if (gm < M) {
                    const float* p = A + (size_t)gm * lda + gk;
                    if (vec && gk + 3 < K) {
                        v = __ldg(reinterpret_cast<const float4*>(p));
                    } else {
                        if (gk + 0 < K) v.x = __ldg(p + 0);
                        if (gk + 1 < K) v.y = __ldg(p + 1);
                        if (gk + 2 < K) v.z = __ldg(p + 2);
                        if (gk + 3 < K) v.w = __ldg(p + 3);
                    }
                }
            }
            ra[i] = v;
        }
    }
    // Registers -> shared: A stored transposed (As[k][m]) so a thread's rows are contiguous.
    static __device__ __forceinline__ void store_a(const float4 (&ra)[Cfg::LA], float* As, int tid) {
#pragma unroll
        for (int i = 0; i < Cfg::LA; ++i) {
            const int idx = tid + i * Cfg::NT;
            if (Cfg::NA4 % Cfg::NT == 0 || idx < Cfg::NA4) {
                const int m = idx / (Cfg::BK / 4);
                const int kq = idx % (Cfg::BK / 4);
                float* d = As + (4 * kq) * Cfg::LDAS + m;
                d[0] = ra[i].x;
                d[Cfg::LDAS] = ra[i].y;
                d[2 * Cfg::LDAS] = ra[i].z;
                d[3 * Cfg::LDAS] = ra[i].w;
            }
        }
    }
    static __device__ __forceinline__ void load_b(float4 (&rb)[Cfg::LB], const float* __restrict__ B,
                                                  int ldb, int N, int K, int col0, int k0, int tid,
                                                  int vec) {
#pragma unroll
        for (int i = 0; i < Cfg::LB; ++i) {
            const int idx = tid + i * Cfg::NT;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (Cfg::NB4 % Cfg::NT == 0 || idx < Cfg::NB4) {
                const int k = idx / (Cfg::BN / 4);
                const int nq = idx % (Cfg::BN / 4);
                const int gk = k0 + k, gn = col0 + 4 * nq;
                if (gk < K) {
                    const float* p = B + (size_t)gk * ldb + gn;
                    if (vec && gn + 3 < N) {
                        v = __ldg(reinterpret_cast<const float4*>(p));
                    } else {
                        if (gn + 0 < N) v.x = __ldg(p + 0);
                        if (gn + 1 < N) v.y = __ldg(p + 1);
                        if (gn + 2 < N) v.z = __ldg(p + 2);
                        if (gn + 3 < N) v.w = __ldg(p + 3);
                    }
                }
            }
            rb[i] = v;
        }
    }
    static __device__ __forceinline__ void store_b(const float4 (&rb)[Cfg::LB], float* Bs, int tid) {
#pragma unroll
        for (int i = 0; i < Cfg::LB; ++i) {
            const int idx = tid + i * Cfg::NT;
            if (Cfg::NB4 % Cfg::NT == 0 || idx < Cfg::NB4) {
                const int k = idx / (Cfg::BN / 4);
                const int nq = idx % (Cfg::BN / 4);
                *reinterpret_cast<float4*>(Bs + k * Cfg::LDBS + 4 * nq) = rb[i];
            }
        }
    }

    // One BM x BN output tile: C[row0.., col0..] (+)= A[row0.., :] * B[:, col0..].
    static __device__ __forceinline__ void run(const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* C,
                                               int ldc, int M, int N, int K, int row0, int col0,
                                               int beta, int vecA, int vecB, int vecC, float* smem) {
        const int tid = threadIdx.x;
        const int t0 = tid / Cfg::B1, t1 = tid % Cfg::B1;
        float* As = smem;
        float* Bs = smem + 2 * Cfg::A_ELEMS;
        // acc2[i][2 ww + h] holds the outputs of row i, columns 4 ww + 2 h and 4 ww + 2 h + 1
        // (FP32 pairs, or two int32 words for INT)
        uint64_t acc2[Cfg::SR][Cfg::S / 2];
#pragma unroll
        for (int i = 0; i < Cfg::SR; ++i)
#pragma unroll
            for (int j = 0; j < Cfg::S / 2; ++j) acc2[i][j] = 0ull;

        const int nk = (K + Cfg::BK - 1) / Cfg::BK;
        float4 ra[Cfg::LA], rb[Cfg::LB];
        load_a(ra, A, lda, M, K, row0, 0, tid, vecA);
        load_b(rb, B, ldb, N, K, col0, 0, tid, vecB);
        store_a(ra, As, tid);
        store_b(rb, Bs, tid);
        __syncthreads();
        for (int t = 0; t < nk; ++t) {
            const int cur = t & 1;
            if (t + 1 < nk) {
                load_a(ra, A, lda, M, K, row0, (t + 1) * Cfg::BK, tid, vecA);
                load_b(rb, B, ldb, N, K, col0, (t + 1) * Cfg::BK, tid, vecB);
            }
            const float* as = As + cur * Cfg::A_ELEMS;
            const float* bs = Bs + cur * Cfg::B_ELEMS;
#pragma unroll
            for (int k = 0; k < Cfg::BK; ++k) {
                float a[Cfg::SR];
                uint64_t b2[Cfg::S / 2];
#pragma unroll
                for (int rr = 0; rr < Cfg::SR / 4; ++rr) {
                    const float4 v =
                        *reinterpret_cast<const float4*>(as + k * Cfg::LDAS + rr * 4 * Cfg::B0 + 4 * t0);
                    a[4 * rr + 0] = v.x;
                    a[4 * rr + 1] = v.y;
                    a[4 * rr + 2] = v.z;
                    a[4 * rr + 3] = v.w;
                }
#pragma unroll
                for (int ww = 0; ww < Cfg::S / 4; ++ww) {
                    const float4 v =
                        *reinterpret_cast<const float4*>(bs + k * Cfg::LDBS + ww * 4 * Cfg::B1 + 4 * t1);
                    b2[2 * ww + 0] = pack2(v.x, v.y);
                    b2[2 * ww + 1] = pack2(v.z, v.w);
                }
#pragma unroll
                for (int i = 0; i < Cfg::SR; ++i) {
                    if (INT) {
                        const uint32_t ai = __float_as_uint(a[i]);
#pragma unroll
                        for (int j = 0; j < Cfg::S / 2; ++j) {
                            const uint32_t lo = (uint32_t)acc2[i][j] + ai * (uint32_t)b2[j];
                            const uint32_t hi = (uint32_t)(acc2[i][j] >> 32) +
                                                ai * (uint32_t)(b2[j] >> 32);
                            acc2[i][j] = ((uint64_t)hi << 32) | lo;
                        }
                    } else {
                        const uint64_t ai = pack2(a[i], a[i]);
#pragma unroll
                        for (int j = 0; j < Cfg::S / 2; ++j) fma2(acc2[i][j], ai, b2[j]);
                    }
                }
            }
            if (t + 1 < nk) {
                store_a(ra, As + (cur ^ 1) * Cfg::A_ELEMS, tid);
                store_b(rb, Bs + (cur ^ 1) * Cfg::B_ELEMS, tid);
            }
            __syncthreads();
        }

        // Epilogue: C = acc or C += acc, float4 stores where the row allows.
#pragma unroll
        for (int rr = 0; rr < Cfg::SR / 4; ++rr)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int gm = row0 + rr * 4 * Cfg::B0 + 4 * t0 + v;
                if (gm >= M) continue;
#pragma unroll
                for (int ww = 0; ww < Cfg::S / 4; ++ww) {
                    const int gn = col0 + ww * 4 * Cfg::B1 + 4 * t1;
                    float* cp = C + (size_t)gm * ldc + gn;
                    const int i = 4 * rr + v;
                    const float o4[4] = {lo32(acc2[i][2 * ww]), hi32(acc2[i][2 * ww]),
                                         lo32(acc2[i][2 * ww + 1]), hi32(acc2[i][2 * ww + 1])};
                    if (vecC && gn + 3 < N) {
                        float4 o = make_float4(o4[0], o4[1], o4[2], o4[3]);
                        if (beta) {
                            const float4 c = *reinterpret_cast<const float4*>(cp);
                            o.x = add32<INT>(o.x, c.x);
                            o.y = add32<INT>(o.y, c.y);
                            o.z = add32<INT>(o.z, c.z);
                            o.w = add32<INT>(o.w, c.w);
                        }
                        *reinterpret_cast<float4*>(cp) = o;
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (gn + u < N) cp[u] = beta ? add32<INT>(cp[u], o4[u]) : o4[u];
                    }
                }
            }
    }
};

}  // namespace pgk
