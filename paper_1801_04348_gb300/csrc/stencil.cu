// The paper's two other parametric kernels (Section 5), with their own case
// discussion through the same walk as the GEMM (case_walk.cuh):
//
// Matrix transposition (Fig. "transpose"): c = a^T on 32-bit words.  A block of
// B0 x B1 threads owns B0 rows and B1*s columns of a; thread (u0, u1) handles
// columns u1 + k*B1, k < s (the paper's granularity s along j).
//   (4a,3a)  both a and c tile staged in shared memory, granularity s,
//   (3b,4a)  the same with s = 1,
//   (3b,4b)  no shared memory: each thread copies one word directly.
// (The figure prints c[i*N+j] = a[i][j], a copy; the kernel computes the
// transposition the text describes.)
//
// 1D Jacobi (Fig. "1dj"): int32 a[2N]; time step t writes one half from the
// three-point average of the other (t odd: a[p+1] = (a[N+p] + a[N+p+1] +
// a[N+p+2]) / 3, else a[N+p+1] = (a[p] + a[p+1] + a[p+2]) / 3) for every interior
// p in [0, N-2), integer division truncating toward zero.  A block of B threads
// owns s*B consecutive p, thread j handles p = p0 + j + k*B, k < s.
//   (4a,3a)  the read window (s*B + 2 words) and the s*B results are staged in
//            shared memory: 2 s B + 2 words, the figure's first case system,
//   (3b,4a)  the same with s = 1,
//   (3b,4b)  no shared memory.
// One launch per time step (the halves swap roles between steps).
#include <string.h>

#include <algorithm>
#include <vector>

#include "case_walk.cuh"
#include "pgk_internal.cuh"

namespace pgk {

struct TArgs {
    int rows, cols;
    const uint32_t* src;
    int lds;
    uint32_t* dst;
    int ldd;
};

// ------------------------------------------------------------ transposition
template <int S>
__global__ void k_transpose_cached(TArgs p) {
    extern __shared__ uint32_t tile_t[];  // B0 x (B1 S + 1)
    const int B0 = blockDim.y, B1 = blockDim.x;
    const int W = B1 * S, P = W + 1;
    const int tiles_n = (p.cols + W - 1) / W;
    const int r0 = (blockIdx.x / tiles_n) * B0, c0 = (blockIdx.x % tiles_n) * W;
    const int u0 = threadIdx.y, u1 = threadIdx.x;
    const int gi = r0 + u0;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int j = u1 + k * B1;
        const int gj = c0 + j;
        tile_t[u0 * P + j] = (gi < p.rows && gj < p.cols) ? __ldg(p.src + (size_t)gi * p.lds + gj) : 0u;
    }
    __syncthreads();
    // output row c0 + j holds elements r0 .. r0 + B0 - 1: consecutive threads write
    // consecutive elements of one output row.  Thread t writes element i = t mod B0
    // of output rows j = t div B0 + m B1 (m = 0 .. S - 1): one division per thread
    const int tid = u0 * B1 + u1;
    const int i = tid % B0, j0 = tid / B0;
    if (r0 + i < p.rows) {
#pragma unroll
        for (int m = 0; m < S; ++m) {
            const int j = j0 + m * B1;
            if (c0 + j < p.cols) p.dst[(size_t)(c0 + j) * p.ldd + r0 + i] = tile_t[i * P + j];
        }
    }
}

__global__ void k_transpose_direct(TArgs p) {
    const int B0 = blockDim.y, B1 = blockDim.x;
    const int tiles_n = (p.cols + B1 - 1) / B1;
    const int i = (blockIdx.x / tiles_n) * B0 + threadIdx.y;
    const int j = (blockIdx.x % tiles_n) * B1 + threadIdx.x;
    if (i < p.rows && j < p.cols) p.dst[(size_t)j * p.ldd + i] = __ldg(p.src + (size_t)i * p.lds + j);
}

template <int S>
static cudaError_t launch_transpose_cached(const TArgs& a, int B0, int B1, int smem, cudaStream_t st) {
    const long long tiles = (long long)((a.rows + B0 - 1) / B0) * ((a.cols + B1 * S - 1) / (B1 * S));
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_transpose_cached<S>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k_transpose_cached<S><<<(unsigned)tiles, dim3(B1, B0), smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_transpose_direct(const TArgs& a, int B0, int B1, int, cudaStream_t st) {
    const long long tiles = (long long)((a.rows + B0 - 1) / B0) * ((a.cols + B1 - 1) / B1);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_transpose_direct<<<(unsigned)tiles, dim3(B1, B0), 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- 1D Jacobi
template <int S>
__global__ void k_jacobi_cached(int n, int odd, int32_t* a) {
    extern __shared__ int32_t win_j[];  // read window (S B + 2) then results (S B)
    const int B = blockDim.x, j = threadIdx.x;
    const int p0 = blockIdx.x * S * B;
    const int32_t* src = odd ? a + n : a;
    int32_t* dst = odd ? a : a + n;
    int32_t* out = win_j + S * B + 2;
    for (int idx = j; idx < S * B + 2; idx += B) win_j[idx] = (p0 + idx < n) ? src[p0 + idx] : 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int q = j + k * B;
        out[q] = (win_j[q] + win_j[q + 1] + win_j[q + 2]) / 3;
    }
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const int q = j + k * B, pp = p0 + q;
        if (pp < n - 2) dst[pp + 1] = out[q];
    }
}

__global__ void k_jacobi_direct(int n, int odd, int32_t* a) {
    const int pp = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t* src = odd ? a + n : a;
    int32_t* dst = odd ? a : a + n;
    if (pp < n - 2) dst[pp + 1] = (src[pp] + src[pp + 1] + src[pp + 2]) / 3;
}

// ----------------------------------------------------------- variant tables
enum { KIND_TRANSPOSE = 0, KIND_JACOBI = 1 };

struct StencilVariant {
    int kind, cached, s;
    const void* func;
};

static const StencilVariant* stencil_table(int* n) {
    static const StencilVariant t[] = {
        {KIND_TRANSPOSE, 1, 1, (const void*)k_transpose_cached<1>},
        {KIND_TRANSPOSE, 1, 2, (const void*)k_transpose_cached<2>},
        {KIND_TRANSPOSE, 1, 4, (const void*)k_transpose_cached<4>},
        {KIND_TRANSPOSE, 1, 8, (const void*)k_transpose_cached<8>},
        {KIND_TRANSPOSE, 0, 1, (const void*)k_transpose_direct},
        {KIND_JACOBI, 1, 1, (const void*)k_jacobi_cached<1>},
        {KIND_JACOBI, 1, 2, (const void*)k_jacobi_cached<2>},
        {KIND_JACOBI, 1, 4, (const void*)k_jacobi_cached<4>},
        {KIND_JACOBI, 1, 8, (const void*)k_jacobi_cached<8>},
        {KIND_JACOBI, 0, 1, (const void*)k_jacobi_direct},
    };
    *n = (int)(sizeof(t) / sizeof(t[0]));
    return t;
}

static int stencil_base_id = -1;

void register_stencil_variants(std::vector<Variant>& v) {
    int n;
    const StencilVariant* t = stencil_table(&n);
    stencil_base_id = (int)v.size();
    for (int i = 0; i < n; ++i) {
        Variant x;
        memset(&x.info, 0, sizeof(x.info));
        x.info.family = t[i].kind == KIND_TRANSPOSE
                            ? (t[i].cached ? PGK_FAM_TRANSPOSE : PGK_FAM_TRANSPOSE_DIRECT)
                            : (t[i].cached ? PGK_FAM_JACOBI : PGK_FAM_JACOBI_DIRECT);
        x.info.s = t[i].s;
        x.info.sr = 1;
        x.info.regs = -1;
        x.info.max_threads = -1;
        x.func = t[i].func;
        x.launch = nullptr;
        x.smem_fixed = 0;
        v.push_back(x);
    }
}

static int stencil_variant(int kind, int cached, int s) {
    registry();
    int n;
    const StencilVariant* t = stencil_table(&n);
    for (int i = 0; i < n; ++i)
        if (t[i].kind == kind && t[i].cached == cached && (!cached || t[i].s == s))
            return stencil_base_id + i;
    return -1;
}

// Register classes of a caller-supplied table (5 entries): cached s = 1, 2, 4, 8; direct.
static int stencil_reg_class(int cached, int s) {
    if (!cached) return 4;
    return s == 1 ? 0 : s == 2 ? 1 : s == 4 ? 2 : 3;
}

// Program state and evaluation functions of the transposition / Jacobi family
// for walk_cases.  There is no register-capped build: strategy "1" leaves the
// register count unchanged, so a refused register counter stays refused.
struct StencilSpec {
    struct Prog {
        int cache, s, gran, regopt;
    };
    int kind;
    int threads;      // B0 * B1 (transposition) or B (Jacobi)
    int B0, B1;       // transposition tile rows / thread columns
    const int* table; // caller register table or NULL

    long long smem(const Prog& p) const {
        if (!p.cache) return 0;
        if (kind == KIND_TRANSPOSE) return 4LL * B0 * ((long long)B1 * p.s + 1);
        return 4LL * (2LL * p.s * threads + 2);  // 2 s B + 2 words (Fig. "1dj")
    }

    pgk_status regs(const Prog& p, long long* out) const {
        if (table) {
            *out = table[stencil_reg_class(p.cache, p.s)];
            return PGK_OK;
        }
        const int id = stencil_variant(kind, p.cache, p.s);
        if (id < 0) {
            set_error("no compiled variant for s=%d", p.s);
            return PGK_ERR_UNSUPPORTED;
        }
        int r = -1;
        pgk_status st = variant_attrs(id, &r, NULL);
        if (st != PGK_OK) return st;
        *out = r;
        return PGK_OK;
    }

    pgk_status eval(int c, const Prog& p, long long* v) const {
        switch (c) {
            case C_THREADS: *v = threads; return PGK_OK;
            case C_REGS: return regs(p, v);
            case C_REGALLOC: {
                long long r = 0;
                pgk_status st = regs(p, &r);
                if (st != PGK_OK) return st;
                *v = regalloc_bytes(threads, r);
                return PGK_OK;
            }
            default: *v = smem(p); return PGK_OK;
        }
    }

    void apply(int o, Prog& p) const {
        if (o == O_REG) p.regopt = 1;
        else if (o == O_GRAN) { p.s = 1; p.gran = 1; }
        else p.cache = 0;
    }
};

static pgk_status stencil_case(int kind, const pgk_machine* m, const int* table, const pgk_params* prog,
                               pgk_case* out) {
    if (!m || !prog || !out) {
        set_error("NULL argument");
        return PGK_ERR_INVALID_ARG;
    }
    const int s = prog->s;
    const int B0 = prog->B0, B1 = kind == KIND_TRANSPOSE ? prog->B1 : 1;
    if (B0 < 1 || B1 < 1 || s < 1 || B0 > 4096 || B1 > 4096) {
        set_error("program parameters must be positive (B0=%d B1=%d s=%d)", B0, B1, s);
        return PGK_ERR_INVALID_ARG;
    }
    if (!(s == 1 || s == 2 || s == 4 || s == 8)) {
        set_error("variants exist for s in {1,2,4,8}, got %d", s);
        return PGK_ERR_UNSUPPORTED;
    }
    StencilSpec spec;
    spec.kind = kind;
    spec.threads = B0 * B1;
    spec.B0 = B0;
    spec.B1 = B1;
    spec.table = table;
    StencilSpec::Prog p = {1, s, 0, 0};
    pgk_status st = walk_cases(*m, spec, p);
    if (st != PGK_OK) return st;
    pgk_case cs;
    memset(&cs, 0, sizeof(cs));
    cs.leaf = !p.cache ? PGK_LEAF_3B4B : (p.gran ? PGK_LEAF_3B4A : PGK_LEAF_4A3A);
    cs.family = kind == KIND_TRANSPOSE ? (p.cache ? PGK_FAM_TRANSPOSE : PGK_FAM_TRANSPOSE_DIRECT)
                                       : (p.cache ? PGK_FAM_JACOBI : PGK_FAM_JACOBI_DIRECT);
    cs.regopt = p.regopt;
    cs.variant_id = stencil_variant(kind, p.cache, p.s);
    long long r = 0;
    spec.eval(C_REGS, p, &r);
    cs.regs = (int)r;
    cs.smem_bytes = (int)spec.smem(p);
    cs.threads = spec.threads;
    cs.params.B0 = B0;
    cs.params.B1 = B1;
    cs.params.s = p.cache ? p.s : 1;
    cs.params.sr = 1;
    cs.params.tile = 0;
    *out = cs;
    return PGK_OK;
}

static pgk_status run_transpose(const pgk_case& c, int rows, int cols, const void* src, int lds,
                                void* dst, int ldd, cudaStream_t st) {
    TArgs a = {rows, cols, (const uint32_t*)src, lds, (uint32_t*)dst, ldd};
    const int B0 = c.params.B0, B1 = c.params.B1;
    cudaError_t e;
    if (c.family == PGK_FAM_TRANSPOSE_DIRECT) {
        e = launch_transpose_direct(a, B0, B1, 0, st);
    } else if (c.family == PGK_FAM_TRANSPOSE) {
        switch (c.params.s) {
            case 1: e = launch_transpose_cached<1>(a, B0, B1, c.smem_bytes, st); break;
            case 2: e = launch_transpose_cached<2>(a, B0, B1, c.smem_bytes, st); break;
            case 4: e = launch_transpose_cached<4>(a, B0, B1, c.smem_bytes, st); break;
            default: e = launch_transpose_cached<8>(a, B0, B1, c.smem_bytes, st); break;
        }
    } else {
        set_error("case is not a transposition case");
        return PGK_ERR_INVALID_ARG;
    }
    if (e != cudaSuccess) return cuda_fail(e, "transposition launch");
    return PGK_OK;
}

template <int S>
static cudaError_t launch_jacobi_cached(int n, int odd, int32_t* a, int B, int smem, cudaStream_t st) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_jacobi_cached<S>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    const long long blocks = ((long long)n - 2 + (long long)S * B - 1) / ((long long)S * B);
    k_jacobi_cached<S><<<(unsigned)std::max(1LL, blocks), B, smem, st>>>(n, odd, a);
    return cudaGetLastError();
}

static pgk_status run_jacobi(const pgk_case& c, int n, int steps, int32_t* a, cudaStream_t st) {
    const int B = c.params.B0;
    for (int t = 0; t < steps; ++t) {
        const int odd = t & 1;
        cudaError_t e;
        if (c.family == PGK_FAM_JACOBI_DIRECT) {
            const long long blocks = ((long long)n - 2 + B - 1) / B;
            k_jacobi_direct<<<(unsigned)std::max(1LL, blocks), B, 0, st>>>(n, odd, a);
            e = cudaGetLastError();
        } else if (c.family == PGK_FAM_JACOBI) {
            switch (c.params.s) {
                case 1: e = launch_jacobi_cached<1>(n, odd, a, B, c.smem_bytes, st); break;
                case 2: e = launch_jacobi_cached<2>(n, odd, a, B, c.smem_bytes, st); break;
                case 4: e = launch_jacobi_cached<4>(n, odd, a, B, c.smem_bytes, st); break;
                default: e = launch_jacobi_cached<8>(n, odd, a, B, c.smem_bytes, st); break;
            }
        } else {
            set_error("case is not a Jacobi case");
            return PGK_ERR_INVALID_ARG;
        }
        if (e != cudaSuccess) return cuda_fail(e, "Jacobi launch");
    }
    return PGK_OK;
}

}  // namespace pgk

using namespace pgk;

extern "C" {

pgk_status pgk_select_case_transpose(const pgk_machine* machine, const int* regs_by_class, int rows,
                                     int cols, const pgk_params* prog, pgk_case* out) {
    if (rows < 1 || cols < 1) {
        set_error("sizes must be >= 1");
        return PGK_ERR_INVALID_ARG;
    }
    return stencil_case(KIND_TRANSPOSE, machine, regs_by_class, prog, out);
}

pgk_status pgk_transpose_case(const pgk_case* c, int rows, int cols, const void* src, int lds,
                              void* dst, int ldd, void* stream) {
    if (!c || rows < 1 || cols < 1 || !src || !dst || lds < cols || ldd < rows) {
        set_error("bad transposition arguments");
        return PGK_ERR_INVALID_ARG;
    }
    return run_transpose(*c, rows, cols, src, lds, dst, ldd, (cudaStream_t)stream);
}

pgk_status pgk_transpose(int rows, int cols, const void* src, int lds, void* dst, int ldd,
                         const pgk_params* prog, void* stream) {
    if (rows < 1 || cols < 1 || !src || !dst || lds < cols || ldd < rows) {
        set_error("bad transposition arguments");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_machine m;
    pgk_status st = current_machine(&m, NULL);
    if (st != PGK_OK) return st;
    pgk_params p = {8, 32, 2, 1, 0};  // the paper's best block for order 2^14 (Table "transpose")
    if (prog) p = *prog;
    pgk_case c;
    if ((st = stencil_case(KIND_TRANSPOSE, &m, NULL, &p, &c)) != PGK_OK) return st;
    return run_transpose(c, rows, cols, src, lds, dst, ldd, (cudaStream_t)stream);
}

pgk_status pgk_select_case_jacobi(const pgk_machine* machine, const int* regs_by_class, int n,
                                  const pgk_params* prog, pgk_case* out) {
    if (n < 3) {
        set_error("Jacobi needs n >= 3");
        return PGK_ERR_INVALID_ARG;
    }
    return stencil_case(KIND_JACOBI, machine, regs_by_class, prog, out);
}

pgk_status pgk_jacobi_case(const pgk_case* c, int n, int steps, int32_t* a, void* stream) {
    if (!c || n < 3 || steps < 0 || !a) {
        set_error("bad Jacobi arguments");
        return PGK_ERR_INVALID_ARG;
    }
    return run_jacobi(*c, n, steps, a, (cudaStream_t)stream);
}

pgk_status pgk_jacobi(int n, int steps, int32_t* a, const pgk_params* prog, void* stream) {
    if (n < 3 || steps < 0 || !a) {
        set_error("bad Jacobi arguments");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_machine m;
    pgk_status st = current_machine(&m, NULL);
    if (st != PGK_OK) return st;
    pgk_params p = {128, 1, 2, 1, 0};  // the paper's best: block 128, granularity 2 (Table Jacobi)
    if (prog) p = *prog;
    pgk_case c;
    if ((st = stencil_case(KIND_JACOBI, &m, NULL, &p, &c)) != PGK_OK) return st;
    return run_jacobi(c, n, steps, a, (cudaStream_t)stream);
}

}  // extern "C"
