// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pgk.h"

namespace pgk {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
void clear_error();
// Converts a CUDA error into PGK_ERR_CUDA with a message naming `what`.
pgk_status cuda_fail(cudaError_t e, const char* what);

#define PGK_CUDA_TRY(call, what)                    \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return pgk::cuda_fail(e_, what); \
    } while (0)

// -------------------------------------------------------- SIMT arguments
struct SimtArgs {
    int M, N, K;
    const float* A;
    int lda;
    const float* B;
    int ldb;
    float* C;
    int ldc;
    int beta;
    int B0, B1, BK;        // runtime program parameters (paper/direct families)
    int vecA, vecB, vecC;  // 16-byte vector access allowed on A / B / C rows
};

typedef cudaError_t (*simt_launch_fn)(const SimtArgs&, int smem_bytes, cudaStream_t);

// One compiled variant of the registry.
struct Variant {
    pgk_variant_info info;      // regs / max_threads filled lazily
    const void* func;           // __global__ function (for attributes)
    simt_launch_fn launch;      // SIMT launcher (NULL for tensor-core variants)
    int smem_fixed;             // dynamic shared memory of a fixed-shape variant
};

// Registration hooks, one per translation unit that defines variants.
void register_simt_variants(std::vector<Variant>& v);
void register_tc_variants(std::vector<Variant>& v);
void register_stencil_variants(std::vector<Variant>& v);

// Registry access (host.cu).
std::vector<Variant>& registry();
int find_paper_variant(int family, int s, int regopt);
int find_direct_variant(int family, int regopt);
int find_rb_variant(int family, int B0, int B1, int sr, int s, int tile);
// Register count of a variant on the current device (-1 if unavailable).
int variant_regs(int id);
// Registers per thread and max threads per block of a variant (cudaFuncGetAttributes, cached).
pgk_status variant_attrs(int id, int* regs, int* maxthr);

// Shared-memory formulas (bytes) of the SIMT families: the f_smem evaluation.
long long smem_paper(int B0, int B1, int s, int BK);
long long smem_rb(int B0, int B1, int sr, int s, int BK);

// ------------------------------------------------------------- workspace
// Library-owned device memory, grown on demand, freed by pgk_shutdown().
void* workspace(int slot, size_t bytes, pgk_status* st);
enum { WS_A0 = 0, WS_A1, WS_B0, WS_B1, WS_SA, WS_SB, WS_TABLE, WS_COUNTER, WS_PARTIAL, WS_SPLITK, WS_COUNT };
// Device error word set by bounded waits (tensor-core kernels).
unsigned int* device_error_word(pgk_status* st);
void free_workspaces();

// Machine parameters of the current device.
pgk_status current_machine(pgk_machine* m, int* device);

// ------------------------------------------------------- tensor-core path
// Fills the tensor-core case for (dtype, prog) or returns an error.
pgk_status tc_select(const pgk_machine* m, int M, int N, int K, pgk_dtype dtype,
                     const pgk_params* prog, pgk_case* out);
pgk_status tc_gemm_launch(const pgk_case& c, int M, int N, int K, pgk_dtype dtype,
                          const void* A, int lda, const void* Bt, int ldbt, const void* A_lo,
                          const void* Bt_lo, const float* sA, const float* sB, float* C, int ldc,
                          int beta, cudaStream_t stream);

// ------------------------------------------------------------- grouped
void grouped_release();
void hostio_release();

// One problem of a grouped operand conversion (see k_cvt_grouped in prep.cu).
struct GCvt {
    const float* src;
    int lds, rows, cols;
    int width;          // converted width: the padded K (a multiple of 64)
    int vec;            // src 16-byte aligned with lds a multiple of 4
    int pad;
    long long dst_row;  // first destination row in the packed workspace
};
// Grouped GEMM in the BF16 or split form (tc_gemm.cu); the compiled grouped tile
// variants of a form as (128, B1, stages, 0, 64).
pgk_status tc_gemm_grouped(int G, const pgk_problem* pr, pgk_dtype dtype, const pgk_params* prog,
                           int beta, cudaStream_t s);
int tc_grouped_variants(pgk_dtype dtype, pgk_params* out, int cap);
// One problem of a grouped FP8 quantisation (k_quant_fp8_grouped in prep.cu).
struct GQuant {
    const float* src;
    int lds, rows, cols;
    int width;          // padded K (a multiple of 128)
    int vec;
    int scale_off;      // A: first scale row (128-row block); B: first scale column
    long long dst_row;  // first destination row in the packed code array
};
pgk_status launch_quant_fp8_grouped(int transpose, const GQuant* probs, const int* prefix, int G,
                                    int total, uint8_t* dst, long long ldd, float* scales,
                                    int ld_scales, cudaStream_t st);
// mode 0: BF16, mode 1: hi/lo split.  One launch converts every A_g into (a0, a1)
// and every B_g, transposed, into (b0, b1); totalA = prefa[G], totalB = prefb[G]
// tile items.
pgk_status launch_cvt_grouped(int mode, const GCvt* pa, const int* prefa, int totalA, uint16_t* a0,
                              uint16_t* a1, const GCvt* pb, const int* prefb, int totalB,
                              uint16_t* b0, uint16_t* b1, int G, long long ldd, cudaStream_t st);
// pgk_gemm; with reuse_b the tensor-core forms keep the converted B of the
// previous call on the same stream (same B, N and K) instead of converting it again.
pgk_status gemm_device(int M, int N, int K, pgk_dtype dtype, const float* A, int lda, const float* B,
                       int ldb, float* C, int ldc, int beta, const pgk_params* prog, cudaStream_t stream,
                       bool reuse_b);
void tune_cache_release();
void costmodel_release();
// Forgets the cached device addresses of the allocation-free gradient's scratch (mlp.cu).
void noalloc_release();
// Learned selection for pgk_gemm(prog = NULL) on a tuning-cache miss (misc.cu).
pgk_status learned_select(int M, int N, int K, pgk_dtype dtype, const float* A, int lda,
                          const float* B, int ldb, float* C, int ldc, int beta,
                          cudaStream_t stream, pgk_params* out);

}  // namespace pgk
