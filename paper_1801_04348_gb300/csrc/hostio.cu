// GEMM on host buffers.  The inputs are copied into one of two library-owned
// device buffer sets on a library stream, so that the copies of call i + 1 run
// while call i computes.  The GEMM runs on the caller's stream in row panels
// (boundaries at multiples of 128 rows, so that every tile and FP8 scale block
// is the one of the whole matrix; the tensor-core forms convert B once).  Each
// panel's C is copied back on a second library stream while the next panel
// computes, and the caller's stream waits for the copies; only the last panel's
// copy is not hidden.  Panels hold whole rounds of tiles (a multiple of the SM
// count), so the split costs no extra rounds of the persistent grid and the last
// panel is small.  C stays in device memory until copied: stores from the GEMM
// epilogue straight into host memory stall the tensor-core pipeline on the host link.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "pgk_internal.cuh"

namespace pgk {

namespace {

struct HostSet {
    float* A = nullptr;
    float* B = nullptr;
    float* C = nullptr;
    size_t capA = 0, capB = 0, capC = 0;   // floats
    cudaEvent_t in_done = nullptr;         // inputs landed
    cudaEvent_t comp_done = nullptr;       // last call that used the set finished (C copied out)
};

struct HostIO {
    int device = -1;
    cudaStream_t s_in = nullptr;           // input copies
    cudaStream_t s_out = nullptr;          // copy-back of the first panel
    cudaEvent_t panel_done[8] = {};        // panel computed
    cudaEvent_t out_done = nullptr;        // every panel copied back
    HostSet set[2];
    int next = 0;
};

std::mutex g_hostio_mu;
HostIO g_hostio[64];

pgk_status ensure(float** p, size_t* cap, size_t need, cudaEvent_t busy) {
    if (*cap >= need) return PGK_OK;
    if (*p) {
        // the buffer may still feed a GEMM in flight
        PGK_CUDA_TRY(cudaEventSynchronize(busy), "host-buffer set wait");
        PGK_CUDA_TRY(cudaFree(*p), "cudaFree");
        *p = nullptr;
        *cap = 0;
    }
    if (cudaMalloc(p, need * sizeof(float)) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        set_error("cannot allocate %zu bytes for host-buffer GEMM staging", need * sizeof(float));
        return PGK_ERR_NO_MEMORY;
    }
    *cap = need;
    return PGK_OK;
}

pgk_status state_for_device(int dev, HostIO** out) {
    if (dev < 0 || dev >= 64) {
        set_error("device %d out of range", dev);
        return PGK_ERR_INVALID_ARG;
    }
    HostIO& h = g_hostio[dev];
    if (h.device < 0) {
        PGK_CUDA_TRY(cudaStreamCreateWithFlags(&h.s_in, cudaStreamNonBlocking), "stream create");
        PGK_CUDA_TRY(cudaStreamCreateWithFlags(&h.s_out, cudaStreamNonBlocking), "stream create");
        for (auto& e : h.panel_done)
            PGK_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create");
        PGK_CUDA_TRY(cudaEventCreateWithFlags(&h.out_done, cudaEventDisableTiming), "event create");
        for (auto& s : h.set) {
            PGK_CUDA_TRY(cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming), "event create");
            PGK_CUDA_TRY(cudaEventCreateWithFlags(&s.comp_done, cudaEventDisableTiming), "event create");
        }
        h.device = dev;
    }
    *out = &h;
    return PGK_OK;
}

// Memory type of a pointer (cudaMemoryTypeUnregistered for pageable or unknown memory).
cudaMemoryType memory_type(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return cudaMemoryTypeUnregistered;
    }
    return a.type;
}

// Row panels in tile rows of bm rows (128, or 256 for CTA-pair tiles): the
// smallest panel of at least 1/8 of the tile rows (and at most all but one) whose
// tile count (panel rows x column tiles of width bn) is a multiple of the number
// of tile slots (SMs, or SM pairs), repeated, the remainder last; else two halves.
// Returns the number of panels (<= 8) and their first rows in starts[0..n]
// (starts[n] = M).
int plan_panels(int M, int N, int bm, int bn, int slots, int* starts) {
    const int T = (M + bm - 1) / bm, tn = (N + bn - 1) / bn;
    int r = 0;
    if (T >= 2 && slots > 0)
        for (int c = std::max(1, (T + 7) / 8); c <= T - 1 && !r; ++c)
            if (((long long)c * tn) % slots == 0) r = c;
    if (!r) r = T >= 2 ? (T + 1) / 2 : T;
    int n = 0;
    for (int t = 0; t < T; t += r) starts[n++] = t * bm;
    starts[n] = M;
    return n;
}

}  // namespace

void hostio_release() {
    std::lock_guard<std::mutex> lock(g_hostio_mu);
    int cur = -1;
    (void)cudaGetDevice(&cur);
    for (HostIO& h : g_hostio) {
        if (h.device < 0) continue;
        (void)cudaSetDevice(h.device);
        (void)cudaStreamSynchronize(h.s_in);
        for (auto& s : h.set) {
            if (s.comp_done) (void)cudaEventSynchronize(s.comp_done);
            cudaFree(s.A);
            cudaFree(s.B);
            cudaFree(s.C);
            if (s.in_done) cudaEventDestroy(s.in_done);
            if (s.comp_done) cudaEventDestroy(s.comp_done);
            s = HostSet();
        }
        (void)cudaStreamSynchronize(h.s_out);
        cudaStreamDestroy(h.s_in);
        cudaStreamDestroy(h.s_out);
        for (auto& e : h.panel_done) cudaEventDestroy(e);
        cudaEventDestroy(h.out_done);
        h = HostIO();
    }
    if (cur >= 0) (void)cudaSetDevice(cur);
    (void)cudaGetLastError();
}

}  // namespace pgk

using namespace pgk;

extern "C" {

pgk_status pgk_gemm_host(int M, int N, int K, pgk_dtype dtype, const float* A, int lda, const float* B,
                         int ldb, float* C, int ldc, int beta, const pgk_params* prog, void* stream) {
    if (M < 1 || N < 1 || K < 1) {
        set_error("sizes must be >= 1 (M=%d N=%d K=%d)", M, N, K);
        return PGK_ERR_INVALID_ARG;
    }
    if (!A || !B || !C || lda < K || ldb < N || ldc < N || (beta != 0 && beta != 1)) {
        set_error("bad host GEMM arguments (lda=%d ldb=%d ldc=%d beta=%d)", lda, ldb, ldc, beta);
        return PGK_ERR_INVALID_ARG;
    }
    int dev = 0;
    PGK_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    for (const void* p : {(const void*)A, (const void*)B, (const void*)C}) {
        const cudaMemoryType t = memory_type(p);
        if (t == cudaMemoryTypeDevice || t == cudaMemoryTypeManaged) {
            set_error("pgk_gemm_host takes host buffers (use pgk_gemm for device memory)");
            return PGK_ERR_INVALID_ARG;
        }
    }

    std::lock_guard<std::mutex> lock(g_hostio_mu);
    HostIO* h = nullptr;
    pgk_status s = state_for_device(dev, &h);
    if (s != PGK_OK) return s;
    HostSet& set = h->set[h->next];
    const size_t nA = (size_t)M * K, nB = (size_t)K * N, nC = (size_t)M * N;
    if ((s = ensure(&set.A, &set.capA, nA, set.comp_done)) != PGK_OK) return s;
    if ((s = ensure(&set.B, &set.capB, nB, set.comp_done)) != PGK_OK) return s;
    if ((s = ensure(&set.C, &set.capC, nC, set.comp_done)) != PGK_OK) return s;
    h->next ^= 1;
    const size_t fs = sizeof(float);

    // inputs: after the previous call that used this set, on the library stream
    PGK_CUDA_TRY(cudaStreamWaitEvent(h->s_in, set.comp_done, 0), "stream wait");
    PGK_CUDA_TRY(cudaMemcpy2DAsync(set.A, K * fs, A, lda * fs, K * fs, M, cudaMemcpyHostToDevice, h->s_in),
                 "copy of A");
    PGK_CUDA_TRY(cudaMemcpy2DAsync(set.B, N * fs, B, ldb * fs, N * fs, K, cudaMemcpyHostToDevice, h->s_in),
                 "copy of B");
    if (beta)
        PGK_CUDA_TRY(cudaMemcpy2DAsync(set.C, N * fs, C, ldc * fs, N * fs, M, cudaMemcpyHostToDevice, h->s_in),
                     "copy of C");
    PGK_CUDA_TRY(cudaEventRecord(set.in_done, h->s_in), "event record");
    PGK_CUDA_TRY(cudaStreamWaitEvent(st, set.in_done, 0), "stream wait");

    // row panels; the copy-back of panel i runs while panel i + 1 computes
    int sms = 0;
    PGK_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const bool tc = dtype == PGK_BF16 || dtype == PGK_SPLIT_BF16 || dtype == PGK_FP8_E4M3;
    // without explicit parameters, the program tuned for the whole matrix (if any)
    // plans the panels and runs all of them, as pgk_gemm would run the whole matrix
    pgk_params tuned;
    if (!prog && pgk_tune_cache_get(M, N, K, dtype, &tuned) == PGK_OK) prog = &tuned;
    const int bn = tc ? (prog ? prog->B1 : 256) : (prog ? std::max(1, prog->B1 * prog->s) : 128);
    const int bm = tc && prog && prog->B0 == 256 ? 256 : 128;
    int starts[9];
    const int np = plan_panels(M, N, bm, bn, sms / (bm / 128), starts);
    for (int i = 0; i < np && s == PGK_OK; ++i) {
        const int r0 = starts[i], rows = starts[i + 1] - r0;
        s = gemm_device(rows, N, K, dtype, set.A + (size_t)r0 * K, K, set.B, N, set.C + (size_t)r0 * N, N,
                        beta, prog, st, i > 0);
        if (s != PGK_OK) break;
        cudaError_t e = cudaEventRecord(h->panel_done[i], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->panel_done[i], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(C + (size_t)r0 * ldc, ldc * fs, set.C + (size_t)r0 * N, N * fs, N * fs,
                                  rows, cudaMemcpyDeviceToHost, h->s_out);
        if (e != cudaSuccess) s = cuda_fail(e, "copy-back of a panel");
    }
    {
        cudaError_t e = cudaEventRecord(h->out_done, h->s_out);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->out_done, 0);
        if (e != cudaSuccess && s == PGK_OK) s = cuda_fail(e, "copy-back ordering");
    }
    // the set is free again once the stream passes this point, also after a failure
    PGK_CUDA_TRY(cudaEventRecord(set.comp_done, st), "event record");
    return s;
}

}  // extern "C"
