/*
 * pgk.h -- C ABI of the parametric GEMM kernel library (sm_103a).
 *
 * The library implements the parametric CUDA kernel family for dense matrix
 * multiplication that arXiv 1801.04348 ("Comprehensive Optimization of
 * Parametric Kernels for GPUs") uses as its running example (Section 2,
 * Fig. "metamul" and Fig. "cudamul"), together with the case discussion of
 * Section 3 (Definition 2, Algorithms 1 and 2) that selects, at run time, the
 * variant whose resource constraints hold for the machine parameters read at
 * load time (Section 1: machine parameters "looked up when the generated code
 * is loaded", program parameters chosen by auto-tuning).
 *
 * Conventions for every entry point:
 *  - Matrices are row-major (the paper indexes a[i*n+j], Fig. "compparkern").
 *    A is M x K with leading dimension lda >= K, B is K x N with ldb >= N,
 *    C is M x N FP32 with ldc >= N.
 *  - Matrix pointers are DEVICE pointers owned by the caller unless a parameter
 *    says "host".  The library owns only its own workspaces (conversion
 *    buffers, scheduler tables, error words) and frees them in pgk_shutdown().
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    GEMM and preparation calls are asynchronous on that stream.
 *  - Device memory is per device: a call runs on the calling thread's current
 *    device and uses only that device's workspaces and error word.  Calls that
 *    use library workspaces (pgk_gemm and pgk_gemm_host in the tensor-core
 *    forms or with split K, pgk_gemm_grouped, pgk_relerr, pgk_mlp_loss_grad)
 *    share one set per device, so such calls on one device must not overlap on
 *    different streams: issue them on one stream, or order the streams with
 *    events.  Workspaces grow on demand; a growth synchronises the device.
 *  - No call aborts, traps or prints.  Every failure is returned as a
 *    pgk_status; pgk_last_error() gives a message for the calling thread.
 *  - Sizes are int; M, N, K >= 1 (zero sizes return PGK_ERR_INVALID_ARG).
 */
#ifndef PGK_H_
#define PGK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PGK_ABI_VERSION 1

#if defined(PGK_BUILD) && defined(__GNUC__)
#define PGK_API __attribute__((visibility("default")))
#else
#define PGK_API
#endif

typedef enum {
    PGK_OK = 0,
    PGK_ERR_INVALID_ARG = 1,   /* bad size, leading dimension, pointer or enum   */
    PGK_ERR_INFEASIBLE = 2,    /* no case of the discussion holds (Alg. 2 drop)  */
    PGK_ERR_UNSUPPORTED = 3,   /* parameters valid but no compiled variant       */
    PGK_ERR_ALIGNMENT = 4,     /* a tensor-core operand violates 16-byte rules   */
    PGK_ERR_CUDA = 5,          /* a CUDA runtime call failed (message kept)      */
    PGK_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (error word set) */
    PGK_ERR_NO_MEMORY = 7      /* workspace allocation failed                    */
} pgk_status;

/* Arithmetic form of a GEMM.  For every form the user-facing pgk_gemm takes
 * FP32 A and B and returns FP32 C; the form says how the product is computed:
 *   PGK_F32        FP32 SIMT fused multiply-add (the paper's kernel family),
 *   PGK_BF16       operands rounded to BF16, tcgen05 tensor cores, FP32 accumulate,
 *   PGK_FP8_E4M3   operands quantised to E4M3 with one FP32 scale per 128 x 128
 *                  tile, tcgen05 tensor cores, FP32 accumulate per 128-deep chunk,
 *   PGK_SPLIT_BF16 x = hi + lo with hi = bf16(x), lo = bf16(x - hi); C is the sum
 *                  of the three products lo*hi + hi*lo + hi*hi in one FP32
 *                  accumulator (lo*lo dropped),
 *   PGK_I32        int32 operands and result (the paper's data type, Fig.
 *                  "cudamul"), SIMT multiply-add modulo 2^32 (two's complement);
 *                  with pgk_gemm the A, B, C pointers then hold int32 words
 *                  (pgk_gemm_i32 is the typed form). */
typedef enum { PGK_F32 = 0, PGK_BF16 = 1, PGK_FP8_E4M3 = 2, PGK_SPLIT_BF16 = 3, PGK_I32 = 4 } pgk_dtype;

/* Machine parameters R_1..R_s (Section 3.2), read with cudaGetDeviceProperties.
 * smem_* are in bytes (the paper counts words).  max_regs_per_thread is the
 * architectural 255. */
typedef struct {
    int max_threads_per_block;   /* T                                   */
    int smem_per_block;          /* default dynamic limit (48 KiB)      */
    int smem_per_block_optin;    /* Z_B used by the case discussion     */
    int regs_per_block;          /* R_B                                 */
    int regs_per_sm;
    int max_regs_per_thread;     /* R                                   */
    int max_threads_per_sm;
    int sm_count;
    int warp_size;
    int cc_major;
    int cc_minor;
    int l2_bytes;
} pgk_machine;

/* Program parameters E_1..E_v (Definition 1).
 *  SIMT forms: thread block B0 x B1 (blockDim = (B1, B0) as in the launch of
 *    Fig. "compparkern"), coarsening s (outputs per thread along N), sr (outputs
 *    per thread along M; sr = 1 is the paper's granularity, sr > 1 selects the
 *    register-blocked family), tile = BK, the depth of the shared-memory K tile
 *    (0 = the paper's choice BK = B0).
 *  Tensor-core forms: B0 x B1 is the output tile: B0 = 128 (one CTA per tile,
 *    B1 in {128, 256}) or B0 = 256 (BF16 and split only: B1 = 256, a cluster of
 *    two CTAs on the two SMs of a TPC per tile, each staging its 128 rows of A
 *    and half of the B^T rows, one tcgen05.mma with cta_group::2 and M = 256 for
 *    both); s = number of pipeline stages, sr unused (0) but in the programs
 *    below, tile = K depth per stage (0 = natural: 64 for BF16/split, 128 for FP8).
 *    (128, 64, s, sr): the fused-conversion program of the BF16 (s = 4) and split
 *    (s = 3) forms for skinny products, N <= 64 (INFEASIBLE beyond): the GEMM
 *    reads A in FP32 by TMA and converts it to BF16 (hi and lo) in shared
 *    memory, so A crosses memory once; A must be 16-byte aligned with lda a
 *    multiple of 4 (else ALIGNMENT).  sr >= 2 splits K into sr slices (work
 *    units: 128-row tile x slice) whose partial products a second launch sums
 *    in slice order (deterministic; a library workspace holds sr x M x N
 *    floats); sr = 1: one slice; sr = 0: as many slices as fill the SMs when
 *    the row tiles alone do not, each at least 512 deep.  pgk_gemm without
 *    parameters takes (128, 64, s, 0) for N <= 64 when A qualifies. */
typedef struct { int B0, B1, s, sr, tile; } pgk_params;

/* Leaves of the case discussion, with the paper's labels (Section 5):
 *   PGK_LEAF_4A3A  cache in shared memory, granularity kept,
 *   PGK_LEAF_3B4A  granularity reduced to 1, cache in shared memory,
 *   PGK_LEAF_3B4B  granularity reduced to 1, no shared memory. */
typedef enum { PGK_LEAF_4A3A = 0, PGK_LEAF_3B4A = 1, PGK_LEAF_3B4B = 2 } pgk_leaf;

/* Variant families. */
typedef enum {
    PGK_FAM_PAPER = 0,    /* s outputs per thread strided by B1 (Fig. "cudamul")  */
    PGK_FAM_RB = 1,       /* register-blocked sr x s micro tiles, double-buffered */
    PGK_FAM_DIRECT = 2,   /* no shared memory, one output per thread              */
    PGK_FAM_TC_BF16 = 3,  /* tcgen05 kind::f16, BF16 operands                     */
    PGK_FAM_TC_SPLIT = 4, /* tcgen05 kind::f16, three BF16 products               */
    PGK_FAM_TC_FP8 = 5,   /* tcgen05 kind::f8f6f4, per-tile scaled E4M3           */
    PGK_FAM_PAPER_I32 = 6,  /* the paper family on int32                          */
    PGK_FAM_RB_I32 = 7,     /* the register-blocked family on int32               */
    PGK_FAM_DIRECT_I32 = 8, /* the no-shared-memory leaf on int32                 */
    PGK_FAM_TRANSPOSE = 9,        /* transposition through shared memory (Fig. "transpose") */
    PGK_FAM_TRANSPOSE_DIRECT = 10, /* transposition without shared memory                 */
    PGK_FAM_JACOBI = 11,          /* 1D Jacobi step through shared memory (Fig. "1dj")    */
    PGK_FAM_JACOBI_DIRECT = 12    /* 1D Jacobi step without shared memory                 */
} pgk_family;

/* A leaf chosen by the case discussion: the variant to launch and the values of
 * its resource counters r_i (Section 3.2) at the requested parameters. */
typedef struct {
    int leaf;          /* pgk_leaf                                            */
    int variant_id;    /* index into the variant registry (pgk_variant_info) */
    int family;        /* pgk_family                                          */
    int regopt;        /* 1 if the register-pressure strategy was applied     */
    int smem_bytes;    /* dynamic shared memory per block                     */
    int regs;          /* registers per thread of the variant                 */
    int threads;       /* threads per block                                   */
    pgk_params params; /* effective program parameters of the leaf            */
} pgk_case;

/* A compiled variant (the IR evaluation functions of Section 3.3: registers
 * from cudaFuncGetAttributes, step S2 of Section 1). */
typedef struct {
    int family;        /* pgk_family                                          */
    int s, sr;         /* compile-time coarsening (0 = runtime)               */
    int B0, B1, tile;  /* compile-time block shape / K tile (0 = runtime)     */
    int regopt;        /* compiled with the register cap                      */
    int regs;          /* registers per thread (-1 before a GPU is visible)   */
    int max_threads;   /* cudaFuncAttributes.maxThreadsPerBlock (-1 idem)     */
} pgk_variant_info;

/* Number of register classes accepted by pgk_select_case_regs:
 * [0..3] paper family s = 1, 2, 4, 8; [4..7] the same register-capped;
 * [8] direct; [9] direct capped; [10] every register-blocked variant. */
#define PGK_REG_CLASSES 11

/* One problem of a grouped GEMM: C = A*B (+ C if beta), FP32, device pointers. */
typedef struct {
    int M, N, K, lda, ldb, ldc;
    const float* A;
    const float* B;
    float* C;
} pgk_problem;

/* ---------------------------------------------------------------- machine */

/* Machine parameters of `device` (Section 1 and Section 3.2: looked up when
 * the code is loaded).  Cached per device after the first call.
 * Errors: INVALID_ARG (out == NULL), CUDA (no such device / no driver). */
PGK_API pgk_status pgk_machine_query(int device, pgk_machine* out);

/* ------------------------------------------------------- variant registry */

/* Number of compiled variants. */
PGK_API int pgk_num_variants(void);

/* Describe variant `id`.  regs / max_threads are read with
 * cudaFuncGetAttributes on the current device when one is present, otherwise
 * they are -1.  Errors: INVALID_ARG (bad id or out == NULL). */
PGK_API pgk_status pgk_variant_info_get(int id, pgk_variant_info* out);

/* ------------------------------------------------------ case discussion */

/* Walk the case tree of the GEMM family (Algorithm 2 applied to the counters
 * threads <= T, regs <= R, register file <= R_B, shared memory <= Z_B with the
 * strategies "1" register cap, "3b" reduce granularity, "4b" no shared memory,
 * in that order; the precondition B0 <= B1*s is the assertion of Fig.
 * "metamul").  Pure host code; register counts come from the compiled variants
 * (needs a visible GPU).  Tensor-core forms check their own fixed resources.
 * Returns OK and fills `out`, INFEASIBLE when every branch was refused,
 * UNSUPPORTED when the register-blocked variant was not compiled,
 * INVALID_ARG on bad arguments, CUDA when register counts cannot be read. */
PGK_API pgk_status pgk_select_case(const pgk_machine* machine, int M, int N, int K,
                           pgk_dtype dtype, const pgk_params* prog, pgk_case* out);

/* Same walk with register counts supplied by the caller (host array of
 * PGK_REG_CLASSES ints, see PGK_REG_CLASSES), for mock machines without a GPU.
 * Errors as pgk_select_case (never CUDA). */
PGK_API pgk_status pgk_select_case_regs(const pgk_machine* machine, const int* regs_by_class,
                                int M, int N, int K, pgk_dtype dtype,
                                const pgk_params* prog, pgk_case* out);

/* ----------------------------------------------------------------- GEMM */

/* C = A*B (beta = 0) or C += A*B (beta = 1, the accumulate form c += a*b of
 * Fig. "metamul").  A, B, C are FP32 device matrices (row-major, see top).
 * `dtype` selects the arithmetic form (pgk_dtype).  `prog` = NULL uses the
 * tuned parameters cached for (device, M, N, K, dtype) by pgk_autotune, else a
 * default; otherwise the case discussion runs on `prog` for the current
 * device's machine parameters.  Tensor-core forms convert A and B into library
 * workspaces first (pgk_cvt_bf16 / pgk_split_bf16 / pgk_quant_fp8).
 * Errors: INVALID_ARG, INFEASIBLE, UNSUPPORTED, CUDA, NO_MEMORY. */
PGK_API pgk_status pgk_gemm(int M, int N, int K, pgk_dtype dtype, const float* A, int lda,
                    const float* B, int ldb, float* C, int ldc, int beta,
                    const pgk_params* prog, void* stream);

/* GEMM on host buffers: C = A B (beta = 0) or C += A B (beta = 1) with A, B and
 * C in host memory, row-major FP32 as for pgk_gemm (dtype selects the form;
 * prog = NULL takes the program the tune cache holds for M x N x K for every
 * panel, else each panel's own tuned or selected program).  An extension of the method for callers
 * whose operands live in host memory; the paper's kernels read device memory only.
 * The library copies A and B into one of two device buffer sets that it owns,
 * on a stream of its own, then runs the GEMM on `stream`; consecutive calls
 * alternate the sets, so the input copies of one call run while the GEMM of the
 * previous call computes.  The GEMM runs in row panels (boundaries at multiples
 * of the tile height B0, panels of whole rounds of tiles for the SM count, at most 8; the
 * tensor-core forms convert B once) into a device buffer; each panel's C is
 * copied back on a second library stream while the next panel computes, and
 * `stream` waits for the copies.  Pinned
 * buffers (cudaHostAlloc / cudaMallocHost / cudaHostRegister) copy at the host
 * link's full rate; pageable memory works but the driver stages it.
 * Ordering: the input copies are not ordered after work enqueued on `stream`
 * before the call; A and B must hold their values, and C must not be accessed,
 * from the call until `stream` has completed the work it enqueued.  C is then in
 * host memory.  The buffer sets grow to the largest call and are freed by
 * pgk_shutdown().  Calls from several host threads are serialised.
 * Errors: INVALID_ARG (also for device or managed pointers), NO_MEMORY, and
 * those of pgk_gemm. */
PGK_API pgk_status pgk_gemm_host(int M, int N, int K, pgk_dtype dtype, const float* A, int lda,
                                 const float* B, int ldb, float* C, int ldc, int beta,
                                 const pgk_params* prog, void* stream);

/* C = A*B (beta = 0) or C += A*B (beta = 1) on int32 matrices, modulo 2^32:
 * the paper's own data type (Fig. "cudamul").  Same case discussion, variants
 * and errors as pgk_gemm with dtype PGK_I32 (SIMT only). */
PGK_API pgk_status pgk_gemm_i32(int M, int N, int K, const int32_t* A, int lda, const int32_t* B,
                                int ldb, int32_t* C, int ldc, int beta, const pgk_params* prog,
                                void* stream);

/* Launch the SIMT variant of a case returned by pgk_select_case(_regs) on FP32
 * operands (lets a caller run any leaf, e.g. one chosen for a mock machine).
 * Errors: INVALID_ARG (not a SIMT case / bad sizes), CUDA (launch failed, e.g.
 * cudaErrorLaunchOutOfResources when the case does not fit this device). */
PGK_API pgk_status pgk_gemm_case(const pgk_case* c, int M, int N, int K, const float* A, int lda,
                         const float* B, int ldb, float* C, int ldc, int beta, void* stream);

/* G independent GEMMs C_g = A_g * B_g (C_g += with beta = 1) on FP32 operands.
 * An extension of the method (batching), not in the paper.
 * PGK_F32: ONE persistent launch: the host packs the problems (host array
 * `problems`, device matrix pointers) and the tile prefix sums into a device
 * table; every CTA pulls (problem, tile) work items from an atomic counter
 * until all tiles are done.  `prog` selects the register-blocked tile variant
 * (NULL = tuned/default).  use_graph = 1 captures the counter reset and the
 * launch in a CUDA graph, cached per problem set and replayed on later calls
 * with the same problems.
 * PGK_BF16 / PGK_SPLIT_BF16 / PGK_FP8_E4M3: the operands are converted into
 * library workspaces packed problem after problem (each at a multiple of 128
 * rows, K zero-padded to the K block, 64 or 128 for FP8): for BF16 and split
 * one launch converts every A_g and every B_g (transposed), for FP8 one launch
 * quantises (128 x 128 tile scales) every A_g and one every B_g; then one
 * persistent tensor-core launch runs the tiles of all problems, in decreasing K
 * order.  Each C_g equals, bit for bit, pgk_gemm on that problem with the same
 * tile program.  `prog` = (128, 128, stages, 0, K block): stages 6 for BF16 and
 * FP8, 3 (split) or 6 (split in three passes); NULL = the first.
 * use_graph does not apply.  No alignment condition on the problems.  The packed
 * workspaces hold every problem at the row stride of the largest K: about
 * (sum of M_g and of N_g, each rounded up to 128) x max K x 2 bytes per operand
 * plane (two planes each for split, 1 byte per entry for FP8); a failed
 * allocation returns NO_MEMORY.
 * Errors: INVALID_ARG (G < 1, a bad problem, a set too large for one launch),
 * UNSUPPORTED (no such variant), CUDA, NO_MEMORY. */
PGK_API pgk_status pgk_gemm_grouped(int G, const pgk_problem* problems, pgk_dtype dtype,
                            const pgk_params* prog, int use_graph, int beta, void* stream);

/* ------------------------------------- the paper's other two parametric kernels */

/* Number of register classes of a transposition / Jacobi register table:
 * [0..3] the shared-memory variant with s = 1, 2, 4, 8; [4] the direct variant. */
#define PGK_STENCIL_REG_CLASSES 5

/* Case discussion of the parametric matrix transposition (Section 5, Fig.
 * "transpose"): counters threads = B0*B1 <= T, registers, register file, shared
 * memory 4*B0*(B1*s + 1) bytes (the a tile, padded) <= Z_B; leaves (4a,3a),
 * (3b,4a) and (3b,4b).  prog: B0 x B1 thread block, s = columns per thread
 * (1, 2, 4, 8).  regs_by_class: host array of PGK_STENCIL_REG_CLASSES ints, or
 * NULL to read the compiled variants (needs a GPU).
 * Errors: INVALID_ARG, INFEASIBLE, UNSUPPORTED, CUDA. */
PGK_API pgk_status pgk_select_case_transpose(const pgk_machine* machine, const int* regs_by_class,
                                             int rows, int cols, const pgk_params* prog,
                                             pgk_case* out);

/* dst = src^T on 32-bit words: src rows x cols (lds >= cols), dst cols x rows
 * (ldd >= rows), device pointers.  prog NULL = (B0, B1, s) = (8, 32, 2), the
 * paper's best block for order 2^14.  Errors: INVALID_ARG, INFEASIBLE,
 * UNSUPPORTED, CUDA. */
PGK_API pgk_status pgk_transpose(int rows, int cols, const void* src, int lds, void* dst, int ldd,
                                 const pgk_params* prog, void* stream);

/* Run the variant of a transposition case (any leaf).  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_transpose_case(const pgk_case* c, int rows, int cols, const void* src,
                                      int lds, void* dst, int ldd, void* stream);

/* Case discussion of the 1D Jacobi step (Section 5, Fig. "1dj"): counters
 * threads = B <= T, registers, register file, shared memory 4*(2*s*B + 2)
 * bytes <= Z_B (the figure's 2sB + 2 words).  prog: B0 = B threads per block,
 * s = points per thread (1, 2, 4, 8), B1 ignored.  Errors as for transposition. */
PGK_API pgk_status pgk_select_case_jacobi(const pgk_machine* machine, const int* regs_by_class,
                                          int n, const pgk_params* prog, pgk_case* out);

/* `steps` time steps of 1D Jacobi on the int32 device array a[2n]: step t
 * writes one half from the three-point average of the other (t odd: a[p+1] =
 * (a[n+p] + a[n+p+1] + a[n+p+2]) / 3, else a[n+p+1] = (a[p] + a[p+1] + a[p+2])
 * / 3) for every p in [0, n-2), C integer division.  One launch per step.
 * prog NULL = (B, s) = (128, 2), the paper's best.  n >= 3.
 * Errors: INVALID_ARG, INFEASIBLE, UNSUPPORTED, CUDA. */
PGK_API pgk_status pgk_jacobi(int n, int steps, int32_t* a, const pgk_params* prog, void* stream);

/* Run the variant of a Jacobi case (any leaf).  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_jacobi_case(const pgk_case* c, int n, int steps, int32_t* a, void* stream);

/* ------------------------------------------------ low-precision operands */

/* dst = bf16(src) with round-to-nearest-even, src rows x cols FP32 (lds).
 * transpose = 0: dst is rows x cols (ldd >= cols); transpose = 1: dst is
 * cols x rows (ldd >= rows), i.e. dst[j][i] = bf16(src[i][j]).  dst is uint16
 * bf16 bit patterns.  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_cvt_bf16(int rows, int cols, const float* src, int lds, uint16_t* dst,
                        int ldd, int transpose, void* stream);

/* hi = bf16(src), lo = bf16(src - hi) (round-to-nearest-even), same layout
 * rules as pgk_cvt_bf16 for both outputs.  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_split_bf16(int rows, int cols, const float* src, int lds, uint16_t* hi,
                          uint16_t* lo, int ldd, int transpose, void* stream);

/* Per-tile scaled E4M3: for every 128 x 128 tile (i, j) of src (ragged edge
 * tiles included) scale = amax/448 in FP32 (1 if the tile is all zero),
 * written to scales[i * ld_scales + j]; dst = e4m3_rn_satfinite(src / scale).
 * Layout of dst as in pgk_cvt_bf16 (transpose applies to dst only; scales are
 * always indexed by the tiles of src).  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_quant_fp8(int rows, int cols, const float* src, int lds, uint8_t* dst,
                         int ldd, float* scales, int ld_scales, int transpose, void* stream);

/* Tensor-core GEMM on prepared operands: A is M x K (lda, element type of the
 * form), Bt is N x K (ldbt), i.e. B stored transposed so both operands are
 * K-major.  BF16: A, Bt bf16.  SPLIT: A/A_lo and Bt/Bt_lo are the hi/lo bf16
 * pairs.  FP8: A, Bt E4M3 codes, scaleA is ceil(M/128) x ceil(K/128) and scaleB
 * ceil(K/128) x ceil(N/128) (row-major, dense).  Row strides must be multiples
 * of 16 bytes and pointers 16-byte aligned (else ALIGNMENT).  The
 * fused-conversion programs (B1 = 64) read FP32 A and are not available here
 * (UNSUPPORTED).  The kernel's
 * bounded waits set the device error word on timeout; the call then returns
 * OK and pgk_check_device_error() reports TIMEOUT.
 * Errors: INVALID_ARG, ALIGNMENT, UNSUPPORTED, INFEASIBLE, CUDA. */
PGK_API pgk_status pgk_gemm_lowp(int M, int N, int K, pgk_dtype dtype, const void* A, int lda,
                         const void* Bt, int ldbt, const void* A_lo, const void* Bt_lo,
                         const float* scaleA, const float* scaleB, float* C, int ldc,
                         int beta, const pgk_params* prog, void* stream);

/* ------------------------------------------------------ error measurement */

/* Relative Frobenius error terms in FP64 on the GPU: out[0] = sum (C - Cref)^2,
 * out[1] = sum Cref^2 over `rows` x `cols` entries.  C is FP32 (ldc), Cref FP64
 * (ldr); row r of Cref pairs with row row_index[r] of C (device int64 array),
 * or with row r when row_index is NULL.  `out` is a device double[2],
 * overwritten.  Error = sqrt(out[0] / out[1]).  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_relerr(int rows, int cols, const float* C, int ldc, const double* Cref,
                      int ldr, const int64_t* row_index, double* out, void* stream);

/* ----------------------------------------------------- learned cost model */

/* Number of parameters of the 7 -> 64 -> 64 -> 1 ReLU network, packed as
 * W1 (64x7 row-major), b1 (64), W2 (64x64 row-major), b2 (64), w3 (64), b3. */
#define PGK_MLP_PARAMS 4737

/* y[n] = MLP(X[n][7]) for n samples (device FP32).  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_mlp_forward(int n, const float* X, const float* theta, float* y, void* stream);

/* Mean squared error of n samples and its gradient w.r.t. theta:
 * loss[0] = (1/n) sum (y - t)^2 and grad[PGK_MLP_PARAMS] (device FP32,
 * overwritten).  Sample r is row idx[r] of X / entry idx[r] of t (idx: device
 * int array of n entries, e.g. a minibatch of a shuffled epoch), or row r when
 * idx is NULL.  Deterministic (fixed reduction order).  n <= 65536.
 * Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_mlp_loss_grad(int n, const int* idx, const float* X, const float* t,
                                     const float* theta, float* grad, float* loss, void* stream);

/* Largest sample count accepted by pgk_mlp_loss_grad_noalloc. */
#define PGK_MLP_NOALLOC_MAX_SAMPLES 2048

/* Same result as pgk_mlp_loss_grad, but the call allocates no memory: no
 * cudaMalloc, cudaFree or allocating library routine.  This serves callers
 * that cannot allocate device memory where they need a gradient: real-time
 * training loops that forbid allocation after start-up (an allocation can
 * synchronise the device and stall the loop for milliseconds), and host
 * applications whose device memory belongs to their own pool allocator.  The
 * paper has no counterpart to this entry point.  The per-tile partial gradients live
 * in one static device array of PGK_MLP_NOALLOC_MAX_SAMPLES / 16 tiles
 * (about 2.4 MB), which every GPU that loads the library holds until the
 * process exits.  The first call on a device looks up that array's device
 * address (once per device, with the device current); make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents; every slot a call reads it first writes, so nothing needs
 * clearing.  Calls that overlap on the GPU (different streams, or different
 * host threads) race on the array: serialise them.  Arguments as
 * pgk_mlp_loss_grad.  Errors: INVALID_ARG (n < 1, n > the limit, NULL
 * pointers), CUDA. */
PGK_API pgk_status pgk_mlp_loss_grad_noalloc(int n, const int* idx, const float* X,
                                             const float* t, const float* theta, float* grad,
                                             float* loss, void* stream);

/* One Adam step (step counts from 1) on `count` parameters in place (device).
 * Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_mlp_adam(int count, float* theta, const float* grad, float* m, float* v,
                        int step, float lr, float beta1, float beta2, float eps, void* stream);

/* -------------------------------------------------------------- autotune */

/* Time each candidate (host array of ncand pgk_params; NULL = the built-in
 * feasible set of the form) for C = A*B on the given device buffers (C is
 * overwritten), `reps` timed runs each after one warm-up, CUDA events on
 * `stream`.  ms_out (host, ncand entries, may be NULL) gets each candidate's
 * median time, +inf if infeasible.  The fastest feasible candidate is written
 * to *best and stored in the tuning cache used by pgk_gemm(prog = NULL).
 * If log_path is not NULL one CSV row per candidate is appended there.
 * Synchronises `stream`.  Errors: INVALID_ARG, INFEASIBLE (none feasible), CUDA. */
PGK_API pgk_status pgk_autotune(int M, int N, int K, pgk_dtype dtype, const float* A, int lda,
                        const float* B, int ldb, float* C, int ldc,
                        const pgk_params* candidates, int ncand, int reps,
                        float* ms_out, pgk_params* best, const char* log_path, void* stream);

/* Grouped tile variants compiled for pgk_gemm_grouped (host array of `cap`
 * entries, may be NULL); *count receives the number available. */
PGK_API pgk_status pgk_grouped_variants(pgk_params* out, int cap, int* count);

/* Time each grouped tile variant (candidates NULL = all compiled ones) on the
 * given problems (their C is overwritten) and store the fastest as the
 * default of pgk_gemm_grouped(prog = NULL) for groups of G problems.
 * ms_out (host, may be NULL) gets each candidate's median time.  Synchronises.
 * Errors: INVALID_ARG, INFEASIBLE, CUDA. */
PGK_API pgk_status pgk_autotune_grouped(int G, const pgk_problem* problems,
                                        const pgk_params* candidates, int ncand, int reps,
                                        float* ms_out, pgk_params* best, void* stream);

/* Number of built-in candidates of a form (the autotuner's default set). */
PGK_API int pgk_default_candidates(pgk_dtype dtype, pgk_params* out, int cap);

/* Installs a trained cost model for the learned case selection of one form
 * (PGK_F32, PGK_BF16, PGK_SPLIT_BF16 or PGK_FP8_E4M3): theta (host,
 * PGK_MLP_PARAMS floats), the 7 feature means mu and scales sd (features:
 * log2 M, log2 N, log2 K, log2 B0, log2 B1, log2 s, form code 0 FP32 paper-form,
 * 1 FP32 register-blocked, 2 BF16, 3 split, 4 FP8), the target normalisation
 * (tmu, tsd) of ln(milliseconds), and k.  Afterwards pgk_gemm(prog = NULL) on a
 * shape missing from the tuning cache scores the form's candidate set with
 * pgk_mlp_forward, times the k best predictions on the call's own operands
 * (beta = 0; with beta = 1 the best prediction is taken untimed), stores the
 * winner in the tuning cache and runs it.  That first call on a new shape
 * synchronises its stream.  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_costmodel_load(pgk_dtype dtype, const float* theta, const float* mu,
                                      const float* sd, float tmu, float tsd, int k);
/* Removes the cost model of a form (back to the untuned default on a miss). */
PGK_API pgk_status pgk_costmodel_clear(pgk_dtype dtype);

/* Store / look up the tuned parameters of (current device, M, N, K, dtype). */
PGK_API pgk_status pgk_tune_cache_put(int M, int N, int K, pgk_dtype dtype, const pgk_params* p);
PGK_API pgk_status pgk_tune_cache_get(int M, int N, int K, pgk_dtype dtype, pgk_params* p);
/* Persist / restore the tuning cache as text (one entry per line).  load merges. */
PGK_API pgk_status pgk_tune_cache_save(const char* path);
PGK_API pgk_status pgk_tune_cache_load(const char* path);

/* ------------------------------------------------------------ measurement */

/* FP32 SIMT throughput probe, a measurement utility with no counterpart in the
 * paper: the measured FP32 peak that the GEMM kernels' SIMT fraction can be
 * compared with, beside the derived SM count x 128 lanes x 2 flop x clock.
 * Launches `blocks` blocks of 256 threads; each thread runs `iters` iterations
 * of 16 independent FMA chains, paired (fma.rn.f32x2, 2 FMAs per chain step)
 * when `paired` is nonzero, else scalar.  Flops per launch:
 * blocks x 256 x iters x 16 x (paired ? 2 : 1) x 2.  `sink` is a device float
 * array of blocks x 256 entries that receives one value per thread (written
 * only so that the work is kept).  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_simt_peak_probe(int blocks, int iters, int paired, float* sink, void* stream);

/* ------------------------------------------------------------- status */

/* Reads and clears the device error word that bounded waits set (synchronises
 * the current device).  Returns OK, TIMEOUT, or CUDA. */
PGK_API pgk_status pgk_check_device_error(void);

/* Exercises the bounded device wait the tensor-core kernels use: one thread
 * waits on an mbarrier that nothing arrives at, gives up after limit_ns
 * (at most 2 s), sets the device error word and returns normally; the next
 * pgk_check_device_error() reports PGK_ERR_TIMEOUT and the context stays
 * usable.  No fault, trap or hang is involved.  Errors: INVALID_ARG, CUDA. */
PGK_API pgk_status pgk_selftest_bounded_wait(unsigned long long limit_ns, void* stream);

PGK_API const char* pgk_status_string(pgk_status s);
/* Message for the last failing call on this host thread ("" if none). */
PGK_API const char* pgk_last_error(void);
/* Frees every library workspace and cached graph.  Safe to call repeatedly. */
PGK_API pgk_status pgk_shutdown(void);
PGK_API int pgk_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PGK_H_ */
