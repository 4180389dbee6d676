// Grouped GEMM: G independent FP32 problems in ONE persistent launch.
//
// The host packs the problems into a device table, ordered by decreasing K
// (the cost of one tile), with the prefix sums of their tile counts.  Every
// CTA repeatedly takes the next work item from an atomic counter, finds its
// problem by binary search in the prefix sums and runs the register-blocked
// tile (simt_rb.cuh) on it, until all tiles are handed out.  No item waits on
// another, so the kernel has no spin-waits.  With use_graph the counter reset
// and the launch are captured once per problem set and replayed.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "pgk_internal.cuh"
#include "simt_rb.cuh"

namespace pgk {

struct GProb {
    const float* A;
    const float* B;
    float* C;
    int M, N, K, lda, ldb, ldc;
    int tiles_m, tiles_n;
    int vecA, vecB, vecC;
    int beta;
    int pad;
};

template <class Cfg>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MINB)
    k_grouped(const GProb* __restrict__ probs, const int* __restrict__ prefix, int G, int total,
              int* counter) {
    extern __shared__ float4 smem_g4[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) break;
        int lo = 0, hi = G - 1;  // largest g with prefix[g] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(prefix + mid) <= item) lo = mid;
            else hi = mid - 1;
        }
        const GProb p = probs[lo];
        const int local = item - __ldg(prefix + lo);
        int bm, bn;
        grouped_tile_coords(local, p.tiles_m, p.tiles_n, bm, bn);
        RbTile<Cfg>::run(p.A, p.lda, p.B, p.ldb, p.C, p.ldc, p.M, p.N, p.K, bm * Cfg::BM,
                         bn * Cfg::BN, p.beta, p.vecA, p.vecB, p.vecC,
                         reinterpret_cast<float*>(smem_g4));
    }
}

struct GroupedVariant {
    int B0, B1, sr, s, BK;
    int bm, bn, smem, threads;
    const void* func;
    cudaError_t (*launch)(const GProb*, const int*, int, int, int*, int grid, cudaStream_t);
};

template <class Cfg>
static cudaError_t launch_grouped(const GProb* t, const int* prefix, int G, int total, int* counter,
                                  int grid, cudaStream_t st) {
    k_grouped<Cfg><<<grid, Cfg::NT, Cfg::SMEM, st>>>(t, prefix, G, total, counter);
    return cudaGetLastError();
}

template <int B0, int B1, int SR, int S, int BK>
static GroupedVariant gv() {
    typedef RbCfg<B0, B1, SR, S, BK> Cfg;
    GroupedVariant v = {B0, B1, SR, S, BK, Cfg::BM, Cfg::BN, Cfg::SMEM, Cfg::NT,
                        (const void*)k_grouped<Cfg>, launch_grouped<Cfg>};
    return v;
}

static const GroupedVariant* grouped_table(int* n) {
    static const GroupedVariant t[] = {
        gv<16, 16, 8, 8, 8>(),  gv<16, 16, 8, 8, 16>(), gv<16, 16, 4, 4, 8>(),
        gv<16, 16, 8, 4, 8>(),  gv<16, 16, 4, 8, 8>(),  gv<8, 16, 8, 8, 8>(),
        gv<16, 8, 8, 8, 8>(),   gv<8, 8, 8, 8, 8>(),
    };
    *n = (int)(sizeof(t) / sizeof(t[0]));
    return t;
}

// ------------------------------------------------------------ graph cache
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    void* table = nullptr;   // GProb[G] then prefix[G+1] then counter
    int device = 0;          // the graph and its table belong to this device
};

static std::mutex g_gmu;
static std::map<std::vector<long long>, GraphEntry> g_graphs;

void grouped_release() {
    std::lock_guard<std::mutex> lk(g_gmu);
    if (g_graphs.empty()) return;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = -1;
    for (auto& kv : g_graphs) {
        // a replay may still be running on the graph's device
        if (cudaSetDevice(kv.second.device) == cudaSuccess) cudaDeviceSynchronize();
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.table) cudaFree(kv.second.table);
    }
    g_graphs.clear();
    if (cur >= 0) cudaSetDevice(cur);
    cudaGetLastError();
}

static bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Builds the host image of the table: problems sorted by decreasing K, then
// the prefix sums of their tile counts and one int for the counter.
static size_t build_table(int G, const pgk_problem* pr, const GroupedVariant& v, int beta,
                          std::vector<unsigned char>& img, int* total) {
    std::vector<int> order(G);
    for (int i = 0; i < G; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return pr[a].K > pr[b].K; });
    const size_t tbytes = sizeof(GProb) * (size_t)G;
    const size_t pbytes = sizeof(int) * (size_t)(G + 1);
    img.assign(tbytes + pbytes + 16, 0);
    GProb* t = reinterpret_cast<GProb*>(img.data());
    int* prefix = reinterpret_cast<int*>(img.data() + tbytes);
    long long acc = 0;
    for (int j = 0; j < G; ++j) {
        const pgk_problem& p = pr[order[j]];
        GProb g;
        memset(&g, 0, sizeof(g));
        g.A = p.A;
        g.B = p.B;
        g.C = p.C;
        g.M = p.M;
        g.N = p.N;
        g.K = p.K;
        g.lda = p.lda;
        g.ldb = p.ldb;
        g.ldc = p.ldc;
        g.tiles_m = (p.M + v.bm - 1) / v.bm;
        g.tiles_n = (p.N + v.bn - 1) / v.bn;
        g.vecA = al16(p.A) && p.lda % 4 == 0;
        g.vecB = al16(p.B) && p.ldb % 4 == 0;
        g.vecC = al16(p.C) && p.ldc % 4 == 0;
        g.beta = beta ? 1 : 0;
        t[j] = g;
        prefix[j] = (int)acc;
        acc += (long long)g.tiles_m * g.tiles_n;
    }
    prefix[G] = (int)acc;
    *total = (int)acc;
    return tbytes + pbytes + 16;
}

static pgk_status check_problems(int G, const pgk_problem* pr) {
    if (G < 1 || !pr) {
        set_error("grouped GEMM needs G >= 1 problems");
        return PGK_ERR_INVALID_ARG;
    }
    long long tiles = 0;
    for (int i = 0; i < G; ++i) {
        const pgk_problem& p = pr[i];
        if (p.M < 1 || p.N < 1 || p.K < 1 || !p.A || !p.B || !p.C || p.lda < p.K || p.ldb < p.N ||
            p.ldc < p.N) {
            set_error("problem %d is invalid (M=%d N=%d K=%d lda=%d ldb=%d ldc=%d)", i, p.M, p.N,
                      p.K, p.lda, p.ldb, p.ldc);
            return PGK_ERR_INVALID_ARG;
        }
        tiles += (long long)((p.M + 7) / 8) * ((p.N + 7) / 8);
    }
    if (tiles > 0x3fffffffLL) {
        set_error("too many tiles in one grouped launch");
        return PGK_ERR_INVALID_ARG;
    }
    return PGK_OK;
}

static const GroupedVariant* find_grouped(const pgk_params* prog) {
    int n;
    const GroupedVariant* t = grouped_table(&n);
    for (int i = 0; i < n; ++i)
        if (t[i].B0 == prog->B0 && t[i].B1 == prog->B1 && t[i].s == prog->s && t[i].sr == prog->sr &&
            t[i].BK == prog->tile)
            return &t[i];
    return nullptr;
}

static pgk_status grid_for(const GroupedVariant& v, int total, int* grid) {
    pgk_machine m;
    pgk_status st = current_machine(&m, NULL);
    if (st != PGK_OK) return st;
    if (v.smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(v.func, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.func, v.threads, v.smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) {
        set_error("grouped variant does not fit on an SM");
        return PGK_ERR_INFEASIBLE;
    }
    *grid = std::max(1, std::min(total, per_sm * m.sm_count));
    return PGK_OK;
}

static pgk_status enqueue(const GroupedVariant& v, void* dtable, int G, int total, int grid,
                          cudaStream_t s) {
    const size_t tbytes = sizeof(GProb) * (size_t)G;
    const size_t pbytes = sizeof(int) * (size_t)(G + 1);
    int* counter = reinterpret_cast<int*>((char*)dtable + tbytes + pbytes);
    PGK_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), s), "counter reset");
    cudaError_t e = v.launch(reinterpret_cast<const GProb*>(dtable),
                             reinterpret_cast<const int*>((char*)dtable + tbytes), G, total, counter,
                             grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "grouped GEMM launch");
    return PGK_OK;
}

pgk_params default_params(int M, int N, int K, pgk_dtype dtype);

}  // namespace pgk

using namespace pgk;

extern "C" pgk_status pgk_gemm_grouped(int G, const pgk_problem* problems, pgk_dtype dtype,
                                       const pgk_params* prog, int use_graph, int beta,
                                       void* stream) {
    pgk_status st = check_problems(G, problems);
    if (st != PGK_OK) return st;
    if (dtype == PGK_BF16 || dtype == PGK_SPLIT_BF16 || dtype == PGK_FP8_E4M3)
        return tc_gemm_grouped(G, problems, dtype, prog, beta, (cudaStream_t)stream);
    if (dtype != PGK_F32) {
        set_error("the grouped GEMM runs the FP32 SIMT family and the tensor-core forms");
        return PGK_ERR_UNSUPPORTED;
    }
    pgk_params p;
    if (prog) {
        p = *prog;
    } else if (pgk_tune_cache_get(-G, 0, 0, PGK_F32, &p) != PGK_OK) {
        pgk_params d = {16, 16, 4, 4, 8};
        p = d;
    }
    const GroupedVariant* v = find_grouped(&p);
    if (!v) {
        set_error("no grouped variant (B0=%d B1=%d s=%d sr=%d tile=%d)", p.B0, p.B1, p.s, p.sr, p.tile);
        return PGK_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned char> img;
    int total = 0;
    const size_t bytes = build_table(G, problems, *v, beta, img, &total);
    int grid = 0;
    if ((st = grid_for(*v, total, &grid)) != PGK_OK) return st;

    if (!use_graph) {
        void* dt = workspace(WS_TABLE, bytes, &st);
        if (!dt) return st;
        PGK_CUDA_TRY(cudaMemcpyAsync(dt, img.data(), bytes - 16, cudaMemcpyHostToDevice, s),
                     "table upload");
        return enqueue(*v, dt, G, total, grid, s);
    }
    // key: the device, the problem set (sizes, pointers), the variant and beta
    int dev = 0;
    PGK_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    std::vector<long long> key;
    key.reserve(9 * (size_t)G + 9);
    key.push_back(dev);
    key.push_back(G);
    key.push_back(p.B0);
    key.push_back(p.B1);
    key.push_back(p.s);
    key.push_back(p.sr);
    key.push_back(p.tile);
    key.push_back(beta);
    for (int i = 0; i < G; ++i) {
        const pgk_problem& q = problems[i];
        key.push_back(q.M);
        key.push_back(q.N);
        key.push_back(q.K);
        key.push_back(q.lda);
        key.push_back(q.ldb);
        key.push_back(q.ldc);
        key.push_back((long long)(uintptr_t)q.A);
        key.push_back((long long)(uintptr_t)q.B);
        key.push_back((long long)(uintptr_t)q.C);
    }
    std::lock_guard<std::mutex> lk(g_gmu);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        GraphEntry ge;
        ge.device = dev;
        PGK_CUDA_TRY(cudaMalloc(&ge.table, bytes), "graph table allocation");
        cudaError_t e = cudaMemcpy(ge.table, img.data(), bytes - 16, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(ge.table);
            return cuda_fail(e, "graph table upload");
        }
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaFree(ge.table);
            return cuda_fail(e, "capture stream");
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = enqueue(*v, ge.table, G, total, grid, cap);
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (st == PGK_OK && e2 != cudaSuccess) st = cuda_fail(e2, "end capture");
        } else {
            st = cuda_fail(e, "begin capture");
        }
        cudaStreamDestroy(cap);
        if (st == PGK_OK) {
            e = cudaGraphInstantiate(&ge.exec, graph, 0);
            if (e != cudaSuccess) st = cuda_fail(e, "graph instantiate");
        }
        if (graph) cudaGraphDestroy(graph);
        if (st != PGK_OK) {
            cudaFree(ge.table);
            return st;
        }
        it = g_graphs.emplace(key, ge).first;
    }
    PGK_CUDA_TRY(cudaGraphLaunch(it->second.exec, s), "graph launch");
    return PGK_OK;
}

extern "C" pgk_status pgk_grouped_variants(pgk_params* out, int cap, int* count) {
    int n;
    const GroupedVariant* t = grouped_table(&n);
    if (count) *count = n;
    for (int i = 0; i < n && i < cap && out; ++i) {
        pgk_params p = {t[i].B0, t[i].B1, t[i].s, t[i].sr, t[i].BK};
        out[i] = p;
    }
    return PGK_OK;
}

extern "C" pgk_status pgk_autotune_grouped(int G, const pgk_problem* problems,
                                           const pgk_params* candidates, int ncand, int reps,
                                           float* ms_out, pgk_params* best, void* stream) {
    pgk_status st = check_problems(G, problems);
    if (st != PGK_OK) return st;
    std::vector<pgk_params> cand;
    if (candidates && ncand > 0) {
        cand.assign(candidates, candidates + ncand);
    } else {
        int n = 0;
        pgk_grouped_variants(NULL, 0, &n);
        cand.resize(n);
        pgk_grouped_variants(cand.data(), n, NULL);
    }
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    PGK_CUDA_TRY(cudaEventCreate(&e0), "event");
    PGK_CUDA_TRY(cudaEventCreate(&e1), "event");
    float best_ms = 1e30f;
    int bi = -1;
    for (size_t i = 0; i < cand.size(); ++i) {
        float ms = 1e30f;
        st = pgk_gemm_grouped(G, problems, PGK_F32, &cand[i], 0, 0, stream);
        if (st == PGK_OK) {
            std::vector<float> t;
            for (int r = 0; r < reps; ++r) {
                cudaEventRecord(e0, s);
                st = pgk_gemm_grouped(G, problems, PGK_F32, &cand[i], 0, 0, stream);
                cudaEventRecord(e1, s);
                if (st != PGK_OK) break;
                cudaEventSynchronize(e1);
                float x;
                cudaEventElapsedTime(&x, e0, e1);
                t.push_back(x);
            }
            if (!t.empty()) {
                std::sort(t.begin(), t.end());
                ms = t[t.size() / 2];
            }
        }
        if (ms_out) ms_out[i] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            bi = (int)i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bi < 0) {
        set_error("no grouped candidate ran");
        return PGK_ERR_INFEASIBLE;
    }
    if (best) *best = cand[bi];
    // the tuned grouped variant is cached under the key (-G, 0, 0)
    return pgk_tune_cache_put(-G, 0, 0, PGK_F32, &cand[bi]);
}
