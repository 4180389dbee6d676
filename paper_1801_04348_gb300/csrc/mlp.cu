// Learned cost model: the 7 -> 64 -> 64 -> 1 ReLU network that ranks program
// parameters before the autotuner times the best few (the paper chooses
// program parameters by auto-tuning, Section 1).  Parameters are one packed
// FP32 vector: W1 (64x7), b1 (64), W2 (64x64), b2 (64), w3 (64), b3.
//
//  * forward: one thread per sample, weights staged in shared memory;
//  * loss + gradient: one block per 16-sample tile computes the forward pass,
//    the mean-squared-error gradient and the back-propagated parameter
//    gradient of its tile in shared memory, writes a per-tile partial; a second
//    kernel sums the partials in tile order (deterministic);
//  * Adam: elementwise update with host-computed bias corrections.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "pgk_internal.cuh"

namespace pgk {

static constexpr int D_IN = 7, H = 64;
static constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * D_IN, OFF_W2 = OFF_B1 + H,
                     OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H,
                     NPARAM = OFF_B3 + 1;
static_assert(NPARAM == PGK_MLP_PARAMS, "parameter packing");
static constexpr int TILE = 16;          // samples per gradient block
static constexpr int GTHREADS = 256;

__global__ void __launch_bounds__(128) k_mlp_forward(int n, const float* __restrict__ X,
                                                     const float* __restrict__ theta,
                                                     float* __restrict__ y) {
    __shared__ float w[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = theta[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[D_IN];
#pragma unroll
    for (int k = 0; k < D_IN; ++k) x[k] = X[(size_t)s * D_IN + k];
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float z = w[OFF_B1 + j];
#pragma unroll
        for (int k = 0; k < D_IN; ++k) z = fmaf(w[OFF_W1 + j * D_IN + k], x[k], z);
        h1[j] = z > 0.f ? z : 0.f;
    }
    float out = w[OFF_B3];
    for (int j = 0; j < H; ++j) {
        float z = w[OFF_B2 + j];
#pragma unroll
        for (int i = 0; i < H; ++i) z = fmaf(w[OFF_W2 + j * H + i], h1[i], z);
        if (z > 0.f) out = fmaf(w[OFF_W3 + j], z, out);
    }
    y[s] = out;
}

// Per-tile forward + backward.  partial[tile][NPARAM + 1]: gradient of
// (1/n) sum (y - t)^2 restricted to the tile's samples, then the tile's sum of
// squared residuals.
__global__ void __launch_bounds__(GTHREADS) k_mlp_grad_tile(int n, const int* __restrict__ idx,
                                                           const float* __restrict__ X,
                                                           const float* __restrict__ T,
                                                           const float* __restrict__ theta,
                                                           float* __restrict__ partial) {
    __shared__ float w[NPARAM];
    __shared__ float xs[TILE][D_IN];
    __shared__ float z1[TILE][H + 1];
    __shared__ float z2[TILE][H + 1];
    __shared__ float d2[TILE][H + 1];   // dL/dz2
    __shared__ float d1[TILE][H + 1];   // dL/dz1
    __shared__ float dy[TILE];
    __shared__ float red[GTHREADS / 32];
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * TILE;
    const int cnt = min(TILE, n - s0);
    for (int i = tid; i < NPARAM; i += GTHREADS) w[i] = theta[i];
    for (int i = tid; i < TILE * D_IN; i += GTHREADS) {
        const int r = i / D_IN, k = i % D_IN;
        float v = 0.f;
        if (r < cnt) {
            const int sidx = idx ? idx[s0 + r] : s0 + r;
            v = X[(size_t)sidx * D_IN + k];
        }
        xs[r][k] = v;
    }
    __syncthreads();
    // z1 = W1 x + b1
    for (int i = tid; i < TILE * H; i += GTHREADS) {
        const int r = i / H, j = i % H;
        float z = w[OFF_B1 + j];
#pragma unroll
        for (int k = 0; k < D_IN; ++k) z = fmaf(w[OFF_W1 + j * D_IN + k], xs[r][k], z);
        z1[r][j] = z;
    }
    __syncthreads();
    // z2 = W2 relu(z1) + b2
    for (int i = tid; i < TILE * H; i += GTHREADS) {
        const int r = i / H, j = i % H;
        float z = w[OFF_B2 + j];
        for (int k = 0; k < H; ++k) {
            const float h = z1[r][k];
            z = fmaf(w[OFF_W2 + j * H + k], h > 0.f ? h : 0.f, z);
        }
        z2[r][j] = z;
    }
    __syncthreads();
    // y, residual, dL/dy = 2 (y - t) / n
    if (tid < 32) {
        float sq = 0.f, g = 0.f;
        if (tid < cnt) {
            float yv = w[OFF_B3];
            for (int j = 0; j < H; ++j) {
                const float h = z2[tid][j];
                yv = fmaf(w[OFF_W3 + j], h > 0.f ? h : 0.f, yv);
            }
            const int sidx = idx ? idx[s0 + tid] : s0 + tid;
            const float r = yv - T[sidx];
            sq = r * r;
            g = 2.f * r / (float)n;
        }
        if (tid < TILE) dy[tid] = g;
        // tile sum of squared residuals (fixed order within the warp)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (tid == 0) red[0] = sq;
    }
    __syncthreads();
    // dL/dz2 = dy * w3 * [z2 > 0]
    for (int i = tid; i < TILE * H; i += GTHREADS) {
        const int r = i / H, j = i % H;
        d2[r][j] = z2[r][j] > 0.f ? dy[r] * w[OFF_W3 + j] : 0.f;
    }
    __syncthreads();
    // dL/dz1 = (W2^T dL/dz2) * [z1 > 0]
    for (int i = tid; i < TILE * H; i += GTHREADS) {
        const int r = i / H, k = i % H;
        float g = 0.f;
        if (z1[r][k] > 0.f)
            for (int j = 0; j < H; ++j) g = fmaf(w[OFF_W2 + j * H + k], d2[r][j], g);
        d1[r][k] = g;
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * (NPARAM + 1);
    // parameter gradients summed over the tile's samples in sample order
    for (int p = tid; p < NPARAM; p += GTHREADS) {
        float g = 0.f;
        if (p < OFF_B1) {
            const int j = p / D_IN, k = p % D_IN;
            for (int r = 0; r < TILE; ++r) g = fmaf(d1[r][j], xs[r][k], g);
        } else if (p < OFF_W2) {
            const int j = p - OFF_B1;
            for (int r = 0; r < TILE; ++r) g += d1[r][j];
        } else if (p < OFF_B2) {
            const int j = (p - OFF_W2) / H, k = (p - OFF_W2) % H;
            for (int r = 0; r < TILE; ++r) {
                const float h = z1[r][k];
                g = fmaf(d2[r][j], h > 0.f ? h : 0.f, g);
            }
        } else if (p < OFF_W3) {
            const int j = p - OFF_B2;
            for (int r = 0; r < TILE; ++r) g += d2[r][j];
        } else if (p < OFF_B3) {
            const int j = p - OFF_W3;
            for (int r = 0; r < TILE; ++r) {
                const float h = z2[r][j];
                g = fmaf(dy[r], h > 0.f ? h : 0.f, g);
            }
        } else {
            for (int r = 0; r < TILE; ++r) g += dy[r];
        }
        out[p] = g;
    }
    if (tid == 0) out[NPARAM] = red[0];
}

// Sums the tile partials in tile order: grad[p] = sum_b partial[b][p]; the
// last slot gives the loss (1/n) sum (y - t)^2.
__global__ void __launch_bounds__(256) k_mlp_grad_reduce(int tiles, int n,
                                                         const float* __restrict__ partial,
                                                         float* __restrict__ grad,
                                                         float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NPARAM) return;
    float g = 0.f;
    for (int b = 0; b < tiles; ++b) g += partial[(size_t)b * (NPARAM + 1) + p];
    if (p < NPARAM) grad[p] = g;
    else loss[0] = g / (float)n;
}

__global__ void k_adam(int count, float* __restrict__ theta, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mhat = mi / bc1, vhat = vi / bc2;
    theta[i] -= lr * mhat / (sqrtf(vhat) + eps);
}

}  // namespace pgk

using namespace pgk;

extern "C" {

pgk_status pgk_mlp_forward(int n, const float* X, const float* theta, float* y, void* stream) {
    if (n < 1 || !X || !theta || !y) {
        set_error("bad MLP forward arguments");
        return PGK_ERR_INVALID_ARG;
    }
    k_mlp_forward<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n, X, theta, y);
    PGK_CUDA_TRY(cudaGetLastError(), "MLP forward launch");
    return PGK_OK;
}

pgk_status pgk_mlp_loss_grad(int n, const int* idx, const float* X, const float* t,
                             const float* theta, float* grad, float* loss, void* stream) {
    if (n < 1 || n > 65536 || !X || !t || !theta || !grad || !loss) {
        set_error("bad MLP gradient arguments (1 <= n <= 65536)");
        return PGK_ERR_INVALID_ARG;
    }
    const int tiles = (n + TILE - 1) / TILE;
    pgk_status st;
    float* partial = (float*)workspace(WS_PARTIAL, sizeof(float) * (size_t)tiles * (NPARAM + 1), &st);
    if (!partial) return st;
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_grad_tile<<<tiles, GTHREADS, 0, s>>>(n, idx, X, t, theta, partial);
    k_mlp_grad_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(tiles, n, partial, grad, loss);
    PGK_CUDA_TRY(cudaGetLastError(), "MLP gradient launch");
    return PGK_OK;
}

pgk_status pgk_mlp_adam(int count, float* theta, const float* grad, float* m, float* v, int step,
                        float lr, float beta1, float beta2, float eps, void* stream) {
    if (count < 1 || step < 1 || !theta || !grad || !m || !v) {
        set_error("bad Adam arguments");
        return PGK_ERR_INVALID_ARG;
    }
    const float bc1 = (float)(1.0 - pow((double)beta1, (double)step));
    const float bc2 = (float)(1.0 - pow((double)beta2, (double)step));
    k_adam<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(count, theta, grad, m, v, lr, beta1,
                                                                  beta2, eps, bc1, bc2);
    PGK_CUDA_TRY(cudaGetLastError(), "Adam launch");
    return PGK_OK;
}

}  // extern "C"

// ------------------------------------------------ allocation-free gradient
// Some callers cannot allocate device memory at the point where they need a
// gradient: real-time or embedded training loops that forbid allocation after
// start-up (a cudaMalloc can synchronise the device and take milliseconds), and
// host applications whose device memory is owned by their own pool allocator.  For them the per-tile partials live
// in a file-scope device array sized for PGK_MLP_NOALLOC_MAX_SAMPLES samples.
// Every GPU that loads the library holds this array until the process exits.
namespace pgk {
static constexpr int NOALLOC_TILES = PGK_MLP_NOALLOC_MAX_SAMPLES / TILE;
static __device__ __align__(256) float g_mlp_noalloc_partial[NOALLOC_TILES * (NPARAM + 1)];

static std::mutex g_noalloc_mu;
static float* g_noalloc_ptr[64];  // device address of the array, per device

// In host code the array's name is only a host-side stand-in, so its device
// address is looked up once per device (with that device current) and cached.
static pgk_status noalloc_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("device index %d out of range", dev);
        return PGK_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mlp_noalloc_partial);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the gradient scratch");
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return PGK_OK;
}

// pgk_shutdown forgets the cached addresses, so that the next call looks them up
// again (after a device reset the array may sit at another address)
void noalloc_release() {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (int d = 0; d < 64; ++d) g_noalloc_ptr[d] = nullptr;
}
}  // namespace pgk

extern "C" pgk_status pgk_mlp_loss_grad_noalloc(int n, const int* idx, const float* X,
                                                const float* t, const float* theta, float* grad,
                                                float* loss, void* stream) {
    if (n < 1 || !X || !t || !theta || !grad || !loss) {
        set_error("bad MLP gradient arguments");
        return PGK_ERR_INVALID_ARG;
    }
    if (n > PGK_MLP_NOALLOC_MAX_SAMPLES) {
        set_error("pgk_mlp_loss_grad_noalloc: %d samples exceed the static scratch limit of %d "
                  "(split the batch, or use pgk_mlp_loss_grad, which takes up to 65536)",
                  n, PGK_MLP_NOALLOC_MAX_SAMPLES);
        return PGK_ERR_INVALID_ARG;
    }
    float* partial = nullptr;
    pgk_status st = noalloc_scratch(&partial);
    if (st != PGK_OK) return st;
    const int tiles = (n + TILE - 1) / TILE;
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_grad_tile<<<tiles, GTHREADS, 0, s>>>(n, idx, X, t, theta, partial);
    k_mlp_grad_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(tiles, n, partial, grad, loss);
    PGK_CUDA_TRY(cudaGetLastError(), "MLP gradient launch");
    return PGK_OK;
}
