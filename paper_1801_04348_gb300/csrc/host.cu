// Host side of the library: status/error reporting, machine parameters, the
// variant registry, the case discussion (Section 3, Algorithm 2) and the
// FP32 GEMM entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "case_walk.cuh"
#include "pgk_internal.cuh"

namespace pgk {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

pgk_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    return PGK_ERR_CUDA;
}

static std::mutex g_mu;

// ------------------------------------------------------- machine parameters
static bool g_machine_valid[64];
static pgk_machine g_machine[64];

static pgk_status query_machine(int device, pgk_machine* out) {
    if (device < 0 || device >= 64) {
        set_error("device index %d out of range", device);
        return PGK_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_machine_valid[device]) {
        cudaDeviceProp p;
        cudaError_t e = cudaGetDeviceProperties(&p, device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
        pgk_machine m;
        m.max_threads_per_block = p.maxThreadsPerBlock;
        m.smem_per_block = (int)p.sharedMemPerBlock;
        m.smem_per_block_optin = (int)p.sharedMemPerBlockOptin;
        m.regs_per_block = p.regsPerBlock;
        m.regs_per_sm = p.regsPerMultiprocessor;
        m.max_regs_per_thread = 255;
        m.max_threads_per_sm = p.maxThreadsPerMultiProcessor;
        m.sm_count = p.multiProcessorCount;
        m.warp_size = p.warpSize;
        m.cc_major = p.major;
        m.cc_minor = p.minor;
        m.l2_bytes = p.l2CacheSize;
        g_machine[device] = m;
        g_machine_valid[device] = true;
    }
    *out = g_machine[device];
    return PGK_OK;
}

pgk_status current_machine(pgk_machine* m, int* device) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (device) *device = dev;
    return query_machine(dev, m);
}

// --------------------------------------------------------- variant registry
static std::vector<Variant> g_registry;
static bool g_registry_init = false;
// regs cache per device: g_regs[dev][id]
static std::vector<int> g_regs[64];
static std::vector<int> g_maxthr[64];

std::vector<Variant>& registry() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_registry_init) {
        register_simt_variants(g_registry);
        register_tc_variants(g_registry);
        register_stencil_variants(g_registry);
        g_registry_init = true;
    }
    return g_registry;
}

int find_paper_variant(int family, int s, int regopt) {
    std::vector<Variant>& r = registry();
    for (size_t i = 0; i < r.size(); ++i)
        if (r[i].info.family == family && r[i].info.s == s && r[i].info.regopt == regopt)
            return (int)i;
    return -1;
}

int find_direct_variant(int family, int regopt) {
    std::vector<Variant>& r = registry();
    for (size_t i = 0; i < r.size(); ++i)
        if (r[i].info.family == family && r[i].info.regopt == regopt) return (int)i;
    return -1;
}

int find_rb_variant(int family, int B0, int B1, int sr, int s, int tile) {
    std::vector<Variant>& r = registry();
    for (size_t i = 0; i < r.size(); ++i) {
        const pgk_variant_info& v = r[i].info;
        if (v.family == family && v.B0 == B0 && v.B1 == B1 && v.sr == sr && v.s == s &&
            v.tile == tile)
            return (int)i;
    }
    return -1;
}

// Registers per thread of variant `id` on the current device: the evaluation
// function f_regs of step S2 (Section 1), read from the compiled code.
pgk_status variant_attrs(int id, int* regs, int* maxthr) {
    std::vector<Variant>& r = registry();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return PGK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_regs[dev].size() != r.size()) {
        g_regs[dev].assign(r.size(), -1);
        g_maxthr[dev].assign(r.size(), -1);
    }
    if (g_regs[dev][id] < 0) {
        cudaFuncAttributes a;
        e = cudaFuncGetAttributes(&a, r[id].func);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
        g_regs[dev][id] = a.numRegs;
        g_maxthr[dev][id] = a.maxThreadsPerBlock;
    }
    if (regs) *regs = g_regs[dev][id];
    if (maxthr) *maxthr = g_maxthr[dev][id];
    return PGK_OK;
}

int variant_regs(int id) {
    int regs = -1;
    if (variant_attrs(id, &regs, NULL) != PGK_OK) return -1;
    return regs;
}

long long smem_paper(int B0, int B1, int s, int BK) {
    return 4LL * ((long long)B0 * BK + (long long)BK * B1 * s);
}

long long smem_rb(int B0, int B1, int sr, int s, int BK) {
    return 8LL * BK * ((long long)B0 * sr + (long long)B1 * s + 8);
}

// -------------------------------------------------------- case discussion
// The GEMM family's program state and evaluation functions for walk_cases
// (case_walk.cuh): families paper / register-blocked / direct, FP32 or int32.
struct RegSource {
    const int* table;  // PGK_REG_CLASSES entries, or NULL = query the device
};

struct GemmSpec {
    struct Prog {
        int family;  // PGK_FAM_PAPER / RB / DIRECT (logical family; int32 mapped by is_int)
        int is_int;  // int32 variants (PGK_I32)
        int cache;   // (4a) / (4b)
        int s, sr;   // effective granularity
        int regopt;  // strategy "1" applied
        int gran;    // strategy "3b" applied
    };
    int B0, B1, BK;
    RegSource src;

    int variant_of(const Prog& p) const {
        if (p.family == PGK_FAM_DIRECT)
            return find_direct_variant(p.is_int ? PGK_FAM_DIRECT_I32 : PGK_FAM_DIRECT, p.regopt);
        if (p.family == PGK_FAM_PAPER)
            return find_paper_variant(p.is_int ? PGK_FAM_PAPER_I32 : PGK_FAM_PAPER, p.s, p.regopt);
        return find_rb_variant(p.is_int ? PGK_FAM_RB_I32 : PGK_FAM_RB, B0, B1, p.sr, p.s, BK);
    }

    pgk_status regs_of(const Prog& p, long long* out) const {
        if (src.table) {
            int cls;
            if (p.family == PGK_FAM_PAPER) {
                const int si = p.s == 1 ? 0 : p.s == 2 ? 1 : p.s == 4 ? 2 : 3;
                cls = si + (p.regopt ? 4 : 0);
            } else if (p.family == PGK_FAM_DIRECT) {
                cls = p.regopt ? 9 : 8;
            } else {
                cls = 10;
            }
            *out = src.table[cls];
            return PGK_OK;
        }
        const int id = variant_of(p);
        if (id < 0) {
            set_error("no compiled variant for family %d s=%d sr=%d", p.family, p.s, p.sr);
            return PGK_ERR_UNSUPPORTED;
        }
        int regs = -1;
        pgk_status st = variant_attrs(id, &regs, NULL);
        if (st != PGK_OK) return st;
        *out = regs;
        return PGK_OK;
    }

    pgk_status eval(int c, const Prog& p, long long* v) const {
        const long long threads = (long long)B0 * B1;
        switch (c) {
            case C_THREADS: *v = threads; return PGK_OK;
            case C_REGS: return regs_of(p, v);
            case C_REGALLOC: {
                long long r = 0;
                pgk_status st = regs_of(p, &r);
                if (st != PGK_OK) return st;
                *v = regalloc_bytes(threads, r);
                return PGK_OK;
            }
            default:
                if (!p.cache || p.family == PGK_FAM_DIRECT) *v = 0;
                else if (p.family == PGK_FAM_PAPER) *v = smem_paper(B0, B1, p.s, BK);
                else *v = smem_rb(B0, B1, p.sr, p.s, BK);
                return PGK_OK;
        }
    }

    void apply(int o, Prog& p) const {
        if (o == O_REG) {
            p.regopt = 1;
        } else if (o == O_GRAN) {
            p.s = 1;
            p.sr = 1;
            p.gran = 1;
            if (p.family == PGK_FAM_RB) p.family = PGK_FAM_PAPER;
        } else {
            p.cache = 0;
            p.family = PGK_FAM_DIRECT;
        }
    }
};

static pgk_status simt_case(const pgk_machine* m, const RegSource& src, const pgk_params* prog,
                            int is_int, pgk_case* out) {
    const int B0 = prog->B0, B1 = prog->B1, s = prog->s;
    const int sr = prog->sr <= 0 ? 1 : prog->sr;
    const int BK = prog->tile == 0 ? B0 : prog->tile;
    if (B0 < 1 || B1 < 1 || s < 1 || BK < 1 || B0 > 4096 || B1 > 4096 || BK > 4096) {
        set_error("program parameters must be positive (B0=%d B1=%d s=%d tile=%d)", B0, B1, s, BK);
        return PGK_ERR_INVALID_ARG;
    }
    // precondition of the source program: assert(B0 <= ub1 * s), Fig. "metamul"
    if ((long long)B0 > (long long)B1 * s) {
        set_error("precondition B0 <= B1*s fails (B0=%d B1=%d s=%d)", B0, B1, s);
        return PGK_ERR_INFEASIBLE;
    }
    GemmSpec spec;
    spec.B0 = B0;
    spec.B1 = B1;
    spec.BK = BK;
    spec.src = src;
    GemmSpec::Prog p;
    p.family = sr == 1 ? PGK_FAM_PAPER : PGK_FAM_RB;
    p.is_int = is_int;
    p.cache = 1;
    p.s = s;
    p.sr = sr;
    p.regopt = 0;
    p.gran = 0;
    if (p.family == PGK_FAM_PAPER && !(s == 1 || s == 2 || s == 4 || s == 8)) {
        set_error("paper-form variants exist for s in {1,2,4,8}, got %d", s);
        return PGK_ERR_UNSUPPORTED;
    }
    if (p.family == PGK_FAM_RB &&
        find_rb_variant(is_int ? PGK_FAM_RB_I32 : PGK_FAM_RB, B0, B1, sr, s, BK) < 0) {
        set_error("register-blocked variant (B0=%d,B1=%d,sr=%d,s=%d,tile=%d) is not compiled", B0,
                  B1, sr, s, BK);
        return PGK_ERR_UNSUPPORTED;
    }
    pgk_status st = walk_cases(*m, spec, p);
    if (st != PGK_OK) return st;
    pgk_case cs;
    memset(&cs, 0, sizeof(cs));
    cs.leaf = !p.cache ? PGK_LEAF_3B4B : (p.gran ? PGK_LEAF_3B4A : PGK_LEAF_4A3A);
    cs.family = !is_int ? p.family
                        : (p.family == PGK_FAM_PAPER ? PGK_FAM_PAPER_I32
                                                     : p.family == PGK_FAM_RB ? PGK_FAM_RB_I32
                                                                              : PGK_FAM_DIRECT_I32);
    cs.regopt = p.regopt;
    cs.variant_id = spec.variant_of(p);
    long long sm = 0, rg = 0;
    spec.eval(C_SMEM, p, &sm);
    spec.eval(C_REGS, p, &rg);
    cs.smem_bytes = (int)sm;
    cs.regs = (int)rg;
    cs.threads = B0 * B1;
    cs.params.B0 = B0;
    cs.params.B1 = B1;
    cs.params.s = p.s;
    cs.params.sr = p.sr;
    cs.params.tile = BK;
    *out = cs;
    return PGK_OK;
}

static pgk_status check_dims(int M, int N, int K) {
    if (M < 1 || N < 1 || K < 1) {
        set_error("sizes must be >= 1 (M=%d N=%d K=%d)", M, N, K);
        return PGK_ERR_INVALID_ARG;
    }
    return PGK_OK;
}

static pgk_status select_any(const pgk_machine* m, const int* regs_table, int M, int N, int K,
                             pgk_dtype dtype, const pgk_params* prog, pgk_case* out) {
    if (!m || !prog || !out) {
        set_error("NULL argument");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_status st = check_dims(M, N, K);
    if (st != PGK_OK) return st;
    if (dtype == PGK_F32 || dtype == PGK_I32) {
        RegSource src;
        src.table = regs_table;
        return simt_case(m, src, prog, dtype == PGK_I32, out);
    }
    if (dtype == PGK_BF16 || dtype == PGK_FP8_E4M3 || dtype == PGK_SPLIT_BF16)
        return tc_select(m, M, N, K, dtype, prog, out);
    set_error("unknown dtype %d", (int)dtype);
    return PGK_ERR_INVALID_ARG;
}

// ----------------------------------------------------------------- SIMT run
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

pgk_status run_simt_case(const pgk_case& c, int M, int N, int K, const float* A, int lda,
                         const float* B, int ldb, float* C, int ldc, int beta, cudaStream_t st) {
    std::vector<Variant>& r = registry();
    if (c.variant_id < 0 || c.variant_id >= (int)r.size() || !r[c.variant_id].launch) {
        set_error("case does not name a SIMT variant");
        return PGK_ERR_INVALID_ARG;
    }
    SimtArgs a;
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.lda = lda;
    a.B = B;
    a.ldb = ldb;
    a.C = C;
    a.ldc = ldc;
    a.beta = beta ? 1 : 0;
    a.B0 = c.params.B0;
    a.B1 = c.params.B1;
    a.BK = c.params.tile;
    a.vecA = aligned16(A) && lda % 4 == 0;
    a.vecB = aligned16(B) && ldb % 4 == 0;
    a.vecC = aligned16(C) && ldc % 4 == 0;
    cudaError_t e = r[c.variant_id].launch(a, c.smem_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "SIMT GEMM launch");
    return PGK_OK;
}

static pgk_status check_gemm_args(int M, int N, int K, const void* A, int lda, const void* B,
                                  int ldb, const void* C, int ldc) {
    pgk_status st = check_dims(M, N, K);
    if (st != PGK_OK) return st;
    if (!A || !B || !C) {
        set_error("NULL matrix pointer");
        return PGK_ERR_INVALID_ARG;
    }
    if (lda < K || ldb < N || ldc < N) {
        set_error("leading dimension too small (lda=%d ldb=%d ldc=%d for M=%d N=%d K=%d)", lda, ldb,
                  ldc, M, N, K);
        return PGK_ERR_INVALID_ARG;
    }
    return PGK_OK;
}

pgk_params default_params(int M, int N, int K, pgk_dtype dtype) {
    pgk_params p;
    if (dtype == PGK_F32 || dtype == PGK_I32) {
        if ((long long)M * N >= 2048LL * 2048) {
            p.B0 = 16; p.B1 = 16; p.s = 8; p.sr = 8; p.tile = 8;
        } else if ((long long)M * N >= 256LL * 256) {
            p.B0 = 16; p.B1 = 16; p.s = 4; p.sr = 4; p.tile = 8;
        } else {
            p.B0 = 8; p.B1 = 8; p.s = 8; p.sr = 8; p.tile = 8;
        }
        (void)K;
    } else if (dtype == PGK_SPLIT_BF16) {
        p.B0 = 128; p.B1 = 128; p.s = 3; p.sr = 0; p.tile = 0;
    } else if (dtype == PGK_BF16) {
        p.B0 = 128; p.B1 = 256; p.s = 4; p.sr = 0; p.tile = 0;
    } else {
        p.B0 = 128; p.B1 = 128; p.s = 6; p.sr = 0; p.tile = 0;
    }
    return p;
}

}  // namespace pgk

using namespace pgk;

// tensor-core user path (tc_gemm.cu)
namespace pgk {
pgk_status tc_gemm_fp32_inputs(const pgk_case& c, int M, int N, int K, pgk_dtype dtype,
                               const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                               int beta, cudaStream_t st, bool prep_b);

pgk_status gemm_device(int M, int N, int K, pgk_dtype dtype, const float* A, int lda, const float* B,
                       int ldb, float* C, int ldc, int beta, const pgk_params* prog, cudaStream_t stream,
                       bool reuse_b) {
    pgk_status st = check_gemm_args(M, N, K, A, lda, B, ldb, C, ldc);
    if (st != PGK_OK) return st;
    pgk_machine m;
    st = current_machine(&m, NULL);
    if (st != PGK_OK) return st;
    pgk_params p;
    if (prog) {
        p = *prog;
    } else if (pgk_tune_cache_get(M, N, K, dtype, &p) != PGK_OK) {
        // skinny products in the BF16 and split forms: the fused-conversion program
        // (A read once, in FP32, by the GEMM) is the leaf of the case discussion
        // whenever N fits its 64-wide tile and A suits TMA; otherwise the learned
        // selection ranks the tile programs, else the default
        const bool fused = (dtype == PGK_BF16 || dtype == PGK_SPLIT_BF16) && N <= 64 &&
                           ((uintptr_t)A & 15u) == 0 && lda % 4 == 0;
        if (fused) {
            // sr = 0: the program chooses its K slices for the shape
            p = pgk_params{128, 64, dtype == PGK_SPLIT_BF16 ? 3 : 4, 0, 0};
        } else if (learned_select(M, N, K, dtype, A, lda, B, ldb, C, ldc, beta, stream, &p) !=
                   PGK_OK) {
            p = default_params(M, N, K, dtype);
        }
    }
    pgk_case c;
    st = select_any(&m, NULL, M, N, K, dtype, &p, &c);
    if (st != PGK_OK) return st;
    if (dtype == PGK_F32 || dtype == PGK_I32)
        return run_simt_case(c, M, N, K, A, lda, B, ldb, C, ldc, beta, stream);
    return tc_gemm_fp32_inputs(c, M, N, K, dtype, A, lda, B, ldb, C, ldc, beta, stream, !reuse_b);
}
}  // namespace pgk

extern "C" {

int pgk_abi_version(void) { return PGK_ABI_VERSION; }

const char* pgk_status_string(pgk_status s) {
    switch (s) {
        case PGK_OK: return "PGK_OK";
        case PGK_ERR_INVALID_ARG: return "PGK_ERR_INVALID_ARG";
        case PGK_ERR_INFEASIBLE: return "PGK_ERR_INFEASIBLE";
        case PGK_ERR_UNSUPPORTED: return "PGK_ERR_UNSUPPORTED";
        case PGK_ERR_ALIGNMENT: return "PGK_ERR_ALIGNMENT";
        case PGK_ERR_CUDA: return "PGK_ERR_CUDA";
        case PGK_ERR_TIMEOUT: return "PGK_ERR_TIMEOUT";
        case PGK_ERR_NO_MEMORY: return "PGK_ERR_NO_MEMORY";
    }
    return "PGK_ERR_UNKNOWN";
}

const char* pgk_last_error(void) { return g_last_error.c_str(); }

pgk_status pgk_machine_query(int device, pgk_machine* out) {
    if (!out) {
        set_error("NULL output");
        return PGK_ERR_INVALID_ARG;
    }
    return query_machine(device, out);
}

int pgk_num_variants(void) { return (int)registry().size(); }

pgk_status pgk_variant_info_get(int id, pgk_variant_info* out) {
    std::vector<Variant>& r = registry();
    if (!out || id < 0 || id >= (int)r.size()) {
        set_error("bad variant id %d", id);
        return PGK_ERR_INVALID_ARG;
    }
    *out = r[id].info;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) == cudaSuccess && dev_count > 0) {
        int regs = -1, mt = -1;
        if (variant_attrs(id, &regs, &mt) == PGK_OK) {
            out->regs = regs;
            out->max_threads = mt;
        }
    } else {
        cudaGetLastError();
    }
    return PGK_OK;
}

pgk_status pgk_select_case(const pgk_machine* machine, int M, int N, int K, pgk_dtype dtype,
                           const pgk_params* prog, pgk_case* out) {
    return select_any(machine, NULL, M, N, K, dtype, prog, out);
}

pgk_status pgk_select_case_regs(const pgk_machine* machine, const int* regs_by_class, int M,
                                int N, int K, pgk_dtype dtype, const pgk_params* prog,
                                pgk_case* out) {
    if (!regs_by_class) {
        set_error("NULL register table");
        return PGK_ERR_INVALID_ARG;
    }
    return select_any(machine, regs_by_class, M, N, K, dtype, prog, out);
}

pgk_status pgk_gemm_case(const pgk_case* c, int M, int N, int K, const float* A, int lda,
                         const float* B, int ldb, float* C, int ldc, int beta, void* stream) {
    if (!c) {
        set_error("NULL case");
        return PGK_ERR_INVALID_ARG;
    }
    pgk_status st = check_gemm_args(M, N, K, A, lda, B, ldb, C, ldc);
    if (st != PGK_OK) return st;
    if (c->family != PGK_FAM_PAPER && c->family != PGK_FAM_RB && c->family != PGK_FAM_DIRECT &&
        c->family != PGK_FAM_PAPER_I32 && c->family != PGK_FAM_RB_I32 &&
        c->family != PGK_FAM_DIRECT_I32) {
        set_error("pgk_gemm_case runs SIMT cases only");
        return PGK_ERR_INVALID_ARG;
    }
    return run_simt_case(*c, M, N, K, A, lda, B, ldb, C, ldc, beta, (cudaStream_t)stream);
}

pgk_status pgk_gemm(int M, int N, int K, pgk_dtype dtype, const float* A, int lda, const float* B,
                    int ldb, float* C, int ldc, int beta, const pgk_params* prog, void* stream) {
    return gemm_device(M, N, K, dtype, A, lda, B, ldb, C, ldc, beta, prog, (cudaStream_t)stream,
                       false);
}

pgk_status pgk_gemm_i32(int M, int N, int K, const int32_t* A, int lda, const int32_t* B, int ldb,
                        int32_t* C, int ldc, int beta, const pgk_params* prog, void* stream) {
    // int32 words travel through the same 32-bit data paths as FP32
    return pgk_gemm(M, N, K, PGK_I32, reinterpret_cast<const float*>(A), lda,
                    reinterpret_cast<const float*>(B), ldb, reinterpret_cast<float*>(C), ldc, beta,
                    prog, stream);
}

pgk_status pgk_shutdown(void) {
    costmodel_release();
    grouped_release();
    hostio_release();
    tune_cache_release();
    noalloc_release();
    free_workspaces();
    return PGK_OK;
}

}  // extern "C"
