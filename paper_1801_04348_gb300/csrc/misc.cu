// Library workspaces, the device error word, the tuning cache and the
// autotuner (the paper leaves program parameters to auto-tuning, Section 1).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pgk_internal.cuh"

namespace pgk {

pgk_params default_params(int M, int N, int K, pgk_dtype dtype);

// -------------------------------------------------------------- workspaces
// One set of workspaces and one error word per device: a call on device d only
// ever receives memory of device d (the current device of the calling thread).
static constexpr int MAX_DEVICES = 64;
static std::mutex g_ws_mu;
static void* g_ws_ptr[MAX_DEVICES][WS_COUNT];
static size_t g_ws_size[MAX_DEVICES][WS_COUNT];
static unsigned int* g_err_word[MAX_DEVICES];

static bool current_device(int* dev, pgk_status* st) {
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "cudaGetDevice");
        return false;
    }
    if (*dev < 0 || *dev >= MAX_DEVICES) {
        set_error("device index %d out of range", *dev);
        *st = PGK_ERR_INVALID_ARG;
        return false;
    }
    return true;
}

void* workspace(int slot, size_t bytes, pgk_status* st) {
    *st = PGK_OK;
    if (slot < 0 || slot >= WS_COUNT) {
        *st = PGK_ERR_INVALID_ARG;
        return nullptr;
    }
    int dev = 0;
    if (!current_device(&dev, st)) return nullptr;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (bytes == 0) bytes = 16;
    void*& ptr = g_ws_ptr[dev][slot];
    size_t& size = g_ws_size[dev][slot];
    if (size < bytes) {
        if (ptr) {
            // earlier work of this device may still use the old buffer
            cudaDeviceSynchronize();
            cudaFree(ptr);
            ptr = nullptr;
            size = 0;
        }
        // grow geometrically so that alternating sizes do not reallocate
        size_t want = bytes + bytes / 4;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
            *st = PGK_ERR_NO_MEMORY;
            return nullptr;
        }
        ptr = p;
        size = want;
    }
    return ptr;
}

unsigned int* device_error_word(pgk_status* st) {
    *st = PGK_OK;
    int dev = 0;
    if (!current_device(&dev, st)) return nullptr;
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (!g_err_word[dev]) {
        unsigned int* w = nullptr;
        cudaError_t e = cudaMalloc(&w, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(w, 0, sizeof(unsigned int));
        if (e != cudaSuccess) {
            if (w) cudaFree(w);
            *st = cuda_fail(e, "error word allocation");
            return nullptr;
        }
        g_err_word[dev] = w;
    }
    return g_err_word[dev];
}

void free_workspaces() {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        cur = -1;
    }
    for (int d = 0; d < MAX_DEVICES; ++d) {
        bool any = g_err_word[d] != nullptr;
        for (int i = 0; i < WS_COUNT; ++i) any = any || g_ws_ptr[d][i] != nullptr;
        if (!any) continue;
        // work still queued on that device may use its buffers
        if (cudaSetDevice(d) == cudaSuccess) cudaDeviceSynchronize();
        for (int i = 0; i < WS_COUNT; ++i) {
            if (g_ws_ptr[d][i]) cudaFree(g_ws_ptr[d][i]);
            g_ws_ptr[d][i] = nullptr;
            g_ws_size[d][i] = 0;
        }
        if (g_err_word[d]) cudaFree(g_err_word[d]);
        g_err_word[d] = nullptr;
    }
    if (cur >= 0) cudaSetDevice(cur);
    cudaGetLastError();
}

// ------------------------------------------------------------ tuning cache
static std::mutex g_tc_mu;
static std::map<std::string, pgk_params> g_tune;

// Device part of the cache key ("<name>_sm<cc>"), looked up once per device.
static std::string device_tag() {
    static std::mutex mu;
    static std::string tags[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return "unknown";
    }
    std::lock_guard<std::mutex> lk(mu);
    if (tags[dev].empty()) {
        cudaDeviceProp p;
        char name[300] = "unknown";
        if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
            snprintf(name, sizeof(name), "%s_sm%d%d", p.name, p.major, p.minor);
        } else {
            cudaGetLastError();
        }
        for (char* c = name; *c; ++c)
            if (*c == ' ' || *c == '\t') *c = '_';
        tags[dev] = name;
    }
    return tags[dev];
}

static std::string tune_key(int M, int N, int K, pgk_dtype dtype) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s %d %d %d %d", device_tag().c_str(), M, N, K, (int)dtype);
    return buf;
}

void tune_cache_release() {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    g_tune.clear();
}

// -------------------------------------------------------- default candidates
static int simt_candidates(int rb_family, pgk_params* out, int cap) {
    // every compiled register-blocked variant plus the paper-form grid of the
    // paper's experiment shapes (B0, B1 in {8,16,32}, s in {1,2,4}, BK = B0)
    std::vector<pgk_params> c;
    std::vector<Variant>& r = registry();
    for (size_t i = 0; i < r.size(); ++i) {
        const pgk_variant_info& v = r[i].info;
        if (v.family != rb_family) continue;
        pgk_params p = {v.B0, v.B1, v.s, v.sr, v.tile};
        c.push_back(p);
    }
    const int bs[3] = {8, 16, 32}, ss[3] = {1, 2, 4};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int s = 0; s < 3; ++s) {
                if (bs[a] > bs[b] * ss[s]) continue;
                pgk_params p = {bs[a], bs[b], ss[s], 1, 0};
                c.push_back(p);
            }
    const int n = (int)c.size();
    for (int i = 0; i < n && i < cap && out; ++i) out[i] = c[i];
    return n;
}

static int tc_candidates(pgk_dtype dtype, pgk_params* out, int cap) {
    std::vector<pgk_params> c;
    // B0 = 256: a CTA pair per 256 x 256 tile (each SM stages half of B)
    // B1 = 64 (last): the fused-conversion program, feasible for N <= 64 only
    if (dtype == PGK_SPLIT_BF16) {
        pgk_params a = {128, 128, 3, 0, 0}, b = {128, 256, 2, 0, 0}, d = {128, 256, 4, 0, 0},
                   e = {128, 128, 6, 0, 0}, f = {256, 256, 3, 0, 0}, g = {256, 256, 6, 0, 0},
                   h = {128, 64, 3, 0, 0};
        c.push_back(a);
        c.push_back(b);
        c.push_back(d);
        c.push_back(e);
        c.push_back(f);
        c.push_back(g);
        c.push_back(h);
    } else if (dtype == PGK_BF16) {
        pgk_params a = {128, 256, 4, 0, 0}, b = {128, 128, 6, 0, 0}, d = {128, 256, 3, 0, 0},
                   e = {128, 128, 4, 0, 0}, f = {256, 256, 6, 0, 0}, h = {128, 64, 4, 0, 0};
        c.push_back(a);
        c.push_back(b);
        c.push_back(d);
        c.push_back(e);
        c.push_back(f);
        c.push_back(h);
    } else {
        pgk_params a = {128, 128, 6, 0, 0}, b = {128, 256, 4, 0, 0};
        c.push_back(a);
        c.push_back(b);
    }
    const int n = (int)c.size();
    for (int i = 0; i < n && i < cap && out; ++i) out[i] = c[i];
    return n;
}

// ---------------------------------------------------- learned selection
// A trained cost model per form: ranks the form's learned candidate set for a
// new shape on the GPU (pgk_mlp_forward), the best k predictions are timed.
struct CostModel {
    bool on = false;
    int k = 3;
    float mu[7], sd[7];
    float tmu = 0.f, tsd = 1.f;
    float* d_theta = nullptr;  // device copy of the parameters
};
static CostModel g_cm[8];
static std::mutex g_cm_mu;

// The learned candidate set: the paper-form grid (B0, B1 in {8, 16, 32},
// s in {1, 2, 4}, B0 <= B1 s, tile = B0) and the register-blocked variants with
// sr = s and tile 8 (F32); the tensor-core candidates of the form otherwise.
static std::vector<pgk_params> learned_candidates(pgk_dtype dtype) {
    std::vector<pgk_params> c;
    if (dtype == PGK_F32) {
        const int bs[3] = {8, 16, 32}, ss[3] = {1, 2, 4};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int s = 0; s < 3; ++s)
                    if (bs[a] <= bs[b] * ss[s]) {
                        pgk_params p = {bs[a], bs[b], ss[s], 1, 0};
                        c.push_back(p);
                    }
        std::vector<Variant>& r = registry();
        for (size_t i = 0; i < r.size(); ++i) {
            const pgk_variant_info& v = r[i].info;
            if (v.family == PGK_FAM_RB && v.sr == v.s && v.tile == 8) {
                pgk_params p = {v.B0, v.B1, v.s, v.sr, v.tile};
                c.push_back(p);
            }
        }
    } else {
        // the tile programs the cost model ranks; the fused-conversion program
        // (B1 = 64) is chosen by the case discussion for N <= 64, not ranked
        const int n = tc_candidates(dtype, NULL, 0);
        std::vector<pgk_params> all(n);
        tc_candidates(dtype, all.data(), n);
        for (const pgk_params& p : all)
            if (p.B1 != 64) c.push_back(p);
    }
    return c;
}

static float form_code(pgk_dtype dtype, const pgk_params& p) {
    if (dtype == PGK_F32) return p.sr > 1 ? 1.f : 0.f;
    return dtype == PGK_BF16 ? 2.f : dtype == PGK_SPLIT_BF16 ? 3.f : 4.f;
}

pgk_status learned_select(int M, int N, int K, pgk_dtype dtype, const float* A, int lda,
                          const float* B, int ldb, float* C, int ldc, int beta,
                          cudaStream_t stream, pgk_params* out) {
    if (dtype < 0 || dtype >= 8) return PGK_ERR_INVALID_ARG;
    CostModel cm;
    {
        std::lock_guard<std::mutex> lk(g_cm_mu);
        if (!g_cm[dtype].on) return PGK_ERR_UNSUPPORTED;
        cm = g_cm[dtype];
    }
    std::vector<pgk_params> cand = learned_candidates(dtype);
    const int n = (int)cand.size();
    if (n == 0) return PGK_ERR_UNSUPPORTED;
    std::vector<float> X((size_t)n * 7), y(n);
    for (int i = 0; i < n; ++i) {
        const float f[7] = {log2f((float)M), log2f((float)N), log2f((float)K), log2f((float)cand[i].B0),
                            log2f((float)cand[i].B1), log2f((float)cand[i].s), form_code(dtype, cand[i])};
        for (int j = 0; j < 7; ++j) X[(size_t)i * 7 + j] = (f[j] - cm.mu[j]) / cm.sd[j];
    }
    pgk_status st;
    float* dX = (float*)workspace(WS_COUNTER, sizeof(float) * (size_t)n * 8, &st);
    if (!dX) return st;
    float* dy = dX + (size_t)n * 7;
    PGK_CUDA_TRY(cudaMemcpyAsync(dX, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, stream),
                 "feature upload");
    if ((st = pgk_mlp_forward(n, dX, cm.d_theta, dy, stream)) != PGK_OK) return st;
    PGK_CUDA_TRY(cudaMemcpyAsync(y.data(), dy, sizeof(float) * n, cudaMemcpyDeviceToHost, stream),
                 "prediction read");
    PGK_CUDA_TRY(cudaStreamSynchronize(stream), "prediction sync");
    // predicted ln(ms) is monotone in the network output: rank by the output
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return y[a] < y[b]; });
    pgk_machine m;
    if ((st = current_machine(&m, NULL)) != PGK_OK) return st;
    std::vector<pgk_params> top;
    for (int i = 0; i < n && (int)top.size() < std::max(1, cm.k); ++i) {
        pgk_case c;
        if (pgk_select_case(&m, M, N, K, dtype, &cand[order[i]], &c) == PGK_OK) top.push_back(cand[order[i]]);
    }
    if (top.empty()) return PGK_ERR_INFEASIBLE;
    if (beta || top.size() == 1) {
        *out = top[0];  // C must not be overwritten by trial runs: take the best prediction
        return pgk_tune_cache_put(M, N, K, dtype, out);
    }
    pgk_params best;
    st = pgk_autotune(M, N, K, dtype, A, lda, B, ldb, C, ldc, top.data(), (int)top.size(), 1, NULL,
                      &best, NULL, stream);
    if (st != PGK_OK) return st;
    *out = best;
    return PGK_OK;
}

void costmodel_release() {
    std::lock_guard<std::mutex> lk(g_cm_mu);
    for (int i = 0; i < 8; ++i) {
        if (g_cm[i].d_theta) cudaFree(g_cm[i].d_theta);
        g_cm[i] = CostModel();
    }
}

}  // namespace pgk

using namespace pgk;

extern "C" {

pgk_status pgk_costmodel_load(pgk_dtype dtype, const float* theta, const float* mu, const float* sd,
                              float tmu, float tsd, int k) {
    if ((int)dtype < 0 || (int)dtype >= 8 || !theta || !mu || !sd || !(tsd > 0.f) || k < 1) {
        set_error("bad cost-model arguments");
        return PGK_ERR_INVALID_ARG;
    }
    for (int j = 0; j < 7; ++j)
        if (!(sd[j] > 0.f)) {
            set_error("feature scales must be positive");
            return PGK_ERR_INVALID_ARG;
        }
    std::lock_guard<std::mutex> lk(g_cm_mu);
    CostModel& cm = g_cm[dtype];
    if (!cm.d_theta) {
        PGK_CUDA_TRY(cudaMalloc(&cm.d_theta, sizeof(float) * PGK_MLP_PARAMS), "cost-model allocation");
    }
    PGK_CUDA_TRY(cudaMemcpy(cm.d_theta, theta, sizeof(float) * PGK_MLP_PARAMS, cudaMemcpyHostToDevice),
                 "cost-model upload");
    for (int j = 0; j < 7; ++j) {
        cm.mu[j] = mu[j];
        cm.sd[j] = sd[j];
    }
    cm.tmu = tmu;
    cm.tsd = tsd;
    cm.k = k;
    cm.on = true;
    return PGK_OK;
}

pgk_status pgk_costmodel_clear(pgk_dtype dtype) {
    if ((int)dtype < 0 || (int)dtype >= 8) {
        set_error("bad dtype");
        return PGK_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_cm_mu);
    if (g_cm[dtype].d_theta) cudaFree(g_cm[dtype].d_theta);
    g_cm[dtype] = CostModel();
    return PGK_OK;
}

pgk_status pgk_tune_cache_put(int M, int N, int K, pgk_dtype dtype, const pgk_params* p) {
    if (!p) {
        set_error("NULL params");
        return PGK_ERR_INVALID_ARG;
    }
    const std::string k = tune_key(M, N, K, dtype);
    std::lock_guard<std::mutex> lk(g_tc_mu);
    g_tune[k] = *p;
    return PGK_OK;
}

pgk_status pgk_tune_cache_get(int M, int N, int K, pgk_dtype dtype, pgk_params* p) {
    if (!p) {
        set_error("NULL params");
        return PGK_ERR_INVALID_ARG;
    }
    const std::string k = tune_key(M, N, K, dtype);
    std::lock_guard<std::mutex> lk(g_tc_mu);
    std::map<std::string, pgk_params>::iterator it = g_tune.find(k);
    if (it == g_tune.end()) return PGK_ERR_INVALID_ARG;
    *p = it->second;
    return PGK_OK;
}

pgk_status pgk_tune_cache_save(const char* path) {
    if (!path) {
        set_error("NULL path");
        return PGK_ERR_INVALID_ARG;
    }
    FILE* f = fopen(path, "w");
    if (!f) {
        set_error("cannot open %s for writing", path);
        return PGK_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tc_mu);
    fprintf(f, "# pgk tuning cache v1: device M N K dtype B0 B1 s sr tile\n");
    for (std::map<std::string, pgk_params>::iterator it = g_tune.begin(); it != g_tune.end(); ++it)
        fprintf(f, "%s %d %d %d %d %d\n", it->first.c_str(), it->second.B0, it->second.B1,
                it->second.s, it->second.sr, it->second.tile);
    fclose(f);
    return PGK_OK;
}

pgk_status pgk_tune_cache_load(const char* path) {
    if (!path) {
        set_error("NULL path");
        return PGK_ERR_INVALID_ARG;
    }
    FILE* f = fopen(path, "r");
    if (!f) {
        set_error("cannot open %s", path);
        return PGK_ERR_INVALID_ARG;
    }
    char line[1024];
    std::lock_guard<std::mutex> lk(g_tc_mu);
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        char dev[512];
        int M, N, K, dt;
        pgk_params p;
        if (sscanf(line, "%511s %d %d %d %d %d %d %d %d %d", dev, &M, &N, &K, &dt, &p.B0, &p.B1,
                   &p.s, &p.sr, &p.tile) == 10) {
            char key[800];
            snprintf(key, sizeof(key), "%s %d %d %d %d", dev, M, N, K, dt);
            g_tune[key] = p;
        }
    }
    fclose(f);
    return PGK_OK;
}

int pgk_default_candidates(pgk_dtype dtype, pgk_params* out, int cap) {
    if (dtype == PGK_F32) return simt_candidates(PGK_FAM_RB, out, cap);
    if (dtype == PGK_I32) return simt_candidates(PGK_FAM_RB_I32, out, cap);
    if (dtype == PGK_BF16 || dtype == PGK_SPLIT_BF16 || dtype == PGK_FP8_E4M3)
        return tc_candidates(dtype, out, cap);
    return 0;
}

pgk_status pgk_autotune(int M, int N, int K, pgk_dtype dtype, const float* A, int lda,
                        const float* B, int ldb, float* C, int ldc, const pgk_params* candidates,
                        int ncand, int reps, float* ms_out, pgk_params* best, const char* log_path,
                        void* stream) {
    if (!A || !B || !C || reps < 1 || (candidates && ncand < 1)) {
        set_error("bad autotune arguments");
        return PGK_ERR_INVALID_ARG;
    }
    std::vector<pgk_params> cand;
    if (candidates) {
        cand.assign(candidates, candidates + ncand);
    } else {
        const int n = pgk_default_candidates(dtype, NULL, 0);
        cand.resize(n);
        pgk_default_candidates(dtype, cand.data(), n);
    }
    pgk_machine m;
    pgk_status st = current_machine(&m, NULL);
    if (st != PGK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    PGK_CUDA_TRY(cudaEventCreate(&e0), "cudaEventCreate");
    PGK_CUDA_TRY(cudaEventCreate(&e1), "cudaEventCreate");
    FILE* log = log_path ? fopen(log_path, "a") : NULL;
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    int best_i = -1;
    float best_ms = INFINITY;
    pgk_status last = PGK_OK;
    for (size_t i = 0; i < cand.size(); ++i) {
        float ms = INFINITY;
        pgk_case c;
        st = pgk_select_case(&m, M, N, K, dtype, &cand[i], &c);
        if (st == PGK_OK) {
            st = pgk_gemm(M, N, K, dtype, A, lda, B, ldb, C, ldc, 0, &cand[i], stream);  // warm-up
            std::vector<float> t;
            for (int r = 0; r < reps && st == PGK_OK; ++r) {
                cudaEventRecord(e0, s);
                st = pgk_gemm(M, N, K, dtype, A, lda, B, ldb, C, ldc, 0, &cand[i], stream);
                cudaEventRecord(e1, s);
                if (st != PGK_OK) break;
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "autotune timing");
                    break;
                }
                float x = 0.f;
                cudaEventElapsedTime(&x, e0, e1);
                t.push_back(x);
            }
            if (st == PGK_OK && !t.empty()) {
                std::sort(t.begin(), t.end());
                ms = t[t.size() / 2];
            }
        }
        if (st == PGK_ERR_CUDA) {
            // a CUDA failure (e.g. out of resources) disqualifies the candidate;
            // a sticky error would fail every later call, so stop there
            cudaError_t sticky = cudaDeviceSynchronize();
            if (sticky != cudaSuccess) {
                last = cuda_fail(sticky, "autotune");
                break;
            }
        }
        if (ms_out) ms_out[i] = ms;
        if (log) {
            const double tflops = isfinite(ms) ? 2.0 * M * (double)N * K / (ms * 1e-3) / 1e12 : 0.0;
            fprintf(log, "%s,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%.6f,%.4f\n", prop.name, M, N, K,
                    (int)dtype, cand[i].B0, cand[i].B1, cand[i].s, cand[i].sr, cand[i].tile,
                    st == PGK_OK ? c.leaf : -1, isfinite(ms) ? ms : -1.0, tflops);
        }
        if (ms < best_ms) {
            best_ms = ms;
            best_i = (int)i;
        }
    }
    if (log) fclose(log);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (last != PGK_OK) return last;
    if (best_i < 0) {
        set_error("no feasible candidate");
        return PGK_ERR_INFEASIBLE;
    }
    if (best) *best = cand[best_i];
    return pgk_tune_cache_put(M, N, K, dtype, &cand[best_i]);
}

pgk_status pgk_check_device_error(void) {
    pgk_status st;
    unsigned int* w = device_error_word(&st);
    if (!w) return st;
    unsigned int h = 0;
    PGK_CUDA_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    PGK_CUDA_TRY(cudaMemcpy(&h, w, sizeof(h), cudaMemcpyDeviceToHost), "error word read");
    if (h) {
        unsigned int z = 0;
        cudaMemcpy(w, &z, sizeof(z), cudaMemcpyHostToDevice);
        set_error("a bounded device wait timed out (code 0x%x)", h);
        return PGK_ERR_TIMEOUT;
    }
    return PGK_OK;
}

}  // extern "C"
