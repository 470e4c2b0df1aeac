// leea_surrogate.cu -- the surrogate form's learned part: an MLP
// d_in -> h1 -> h2 -> 1 (ReLU) that scores offspring descriptors, with its
// own forward, backward (mean squared error) and Adam kernels.  The paper has
// no counterpart; it is the pre-screen that lets only the most promising
// offspring be made and evaluated.
//
// Parameters, flat FP32: W1 [h1][d_in], b1 [h1], W2 [h2][h1], b2 [h2],
// w3 [h2], b3.  Every reduction runs in a fixed order, so results do not
// depend on scheduling.
#include "leea_internal.h"
#include "philox.cuh"

#include <cmath>

namespace leea {

namespace {

constexpr uint32_t kTagSurrInit = 6;
constexpr int kRows = 32;      // rows per forward CTA at most (fewer for small n: more CTAs)
constexpr int kFwdThreads = 256;

struct MlpView {
    const float *W1, *b1, *W2, *b2, *w3, *b3;
};

__device__ __forceinline__ MlpView view(const float* theta, int32_t d_in, int32_t h1, int32_t h2)
{
    MlpView v;
    v.W1 = theta;
    v.b1 = v.W1 + static_cast<int64_t>(h1) * d_in;
    v.W2 = v.b1 + h1;
    v.b2 = v.W2 + static_cast<int64_t>(h2) * h1;
    v.w3 = v.b2 + h2;
    v.b3 = v.w3 + h2;
    return v;
}

// Glorot-uniform U(-a, a), a = sqrt(6 / (fan_in + fan_out)), from Philox
// stream (SURR_INIT, 0, 0) draw = parameter index; zero biases.
__global__ void surr_init_kernel(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, float* __restrict__ theta)
{
    const int64_t n1 = static_cast<int64_t>(h1) * d_in, n2 = static_cast<int64_t>(h2) * h1;
    const int64_t total = n1 + h1 + n2 + h2 + h2 + 1;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int32_t fin = 0, fout = 0;
        bool bias = false;
        if (i < n1) { fin = d_in; fout = h1; }
        else if (i < n1 + h1) bias = true;
        else if (i < n1 + h1 + n2) { fin = h1; fout = h2; }
        else if (i < n1 + h1 + n2 + h2) bias = true;
        else if (i < n1 + h1 + n2 + h2 + h2) { fin = h2; fout = 1; }
        else bias = true;
        float v = 0.0f;
        if (!bias) {
            const uint4 blk = stream_block(seed, kTagSurrInit, 0u, 0u, static_cast<uint32_t>(i >> 2));
            const float u = u01(word_of(blk, static_cast<uint32_t>(i & 3)));
            v = sqrtf(6.0f / static_cast<float>(fin + fout)) * (2.0f * u - 1.0f);
        }
        theta[i] = v;
    }
}

// Forward for `rpc` rows per CTA; a1 / a2 (the ReLU outputs) are kept for
// the backward pass when not NULL.  Dot products run over k in order.
__global__ void __launch_bounds__(kFwdThreads)
surr_forward_kernel(int32_t n, int32_t d_in, int32_t h1, int32_t h2, int32_t rpc, const float* __restrict__ theta,
                    const float* __restrict__ x, float* __restrict__ y, float* __restrict__ a1_out,
                    float* __restrict__ a2_out)
{
    extern __shared__ float sm[];
    float* xs = sm;                       // [rpc][d_in]
    float* s1 = xs + rpc * d_in;          // [rpc][h1]
    float* s2 = s1 + rpc * h1;            // [rpc][h2]
    const MlpView p = view(theta, d_in, h1, h2);
    const int32_t r0 = blockIdx.x * rpc;
    const int32_t rows = n - r0 < rpc ? n - r0 : rpc;
    for (int i = threadIdx.x; i < rpc * d_in; i += kFwdThreads) {
        const int r = i / d_in;
        xs[i] = r < rows ? x[static_cast<int64_t>(r0 + r) * d_in + (i - r * d_in)] : 0.0f;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < rpc * h1; o += kFwdThreads) {
        const int r = o / h1, u = o - r * h1;
        const float* w = p.W1 + static_cast<int64_t>(u) * d_in;
        const float* xr = xs + r * d_in;
        float z = p.b1[u];
        for (int k = 0; k < d_in; ++k) z = fmaf(w[k], xr[k], z);
        s1[o] = fmaxf(z, 0.0f);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < rpc * h2; o += kFwdThreads) {
        const int r = o / h2, u = o - r * h2;
        const float* w = p.W2 + static_cast<int64_t>(u) * h1;
        const float* ar = s1 + r * h1;
        float z = p.b2[u];
        for (int k = 0; k < h1; ++k) z = fmaf(w[k], ar[k], z);
        s2[o] = fmaxf(z, 0.0f);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += kFwdThreads) {
        float z = p.b3[0];
        for (int u = 0; u < h2; ++u) z = fmaf(p.w3[u], s2[r * h2 + u], z);
        y[r0 + r] = z;
    }
    if (a1_out)
        for (int o = threadIdx.x; o < rows * h1; o += kFwdThreads) a1_out[static_cast<int64_t>(r0) * h1 + o] = s1[o];
    if (a2_out)
        for (int o = threadIdx.x; o < rows * h2; o += kFwdThreads) a2_out[static_cast<int64_t>(r0) * h2 + o] = s2[o];
}

// Per row: dy = 2 (y - t) / n, d2 = dy w3 (.) [a2 > 0], d1 = (W2^T d2) (.) [a1 > 0].
__global__ void surr_backrow_kernel(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* __restrict__ theta,
                                    const float* __restrict__ y, const float* __restrict__ t,
                                    const float* __restrict__ a1, const float* __restrict__ a2,
                                    float* __restrict__ dy, float* __restrict__ d1, float* __restrict__ d2)
{
    const MlpView p = view(theta, d_in, h1, h2);
    const int32_t r = blockIdx.x;
    extern __shared__ float sd2[];  // [h2]
    const float g = 2.0f * (y[r] - t[r]) / static_cast<float>(n);
    for (int u = threadIdx.x; u < h2; u += blockDim.x) {
        const float v = a2[static_cast<int64_t>(r) * h2 + u] > 0.0f ? g * p.w3[u] : 0.0f;
        sd2[u] = v;
        d2[static_cast<int64_t>(r) * h2 + u] = v;
    }
    if (threadIdx.x == 0) dy[r] = g;
    __syncthreads();
    for (int k = threadIdx.x; k < h1; k += blockDim.x) {
        float s = 0.0f;
        for (int u = 0; u < h2; ++u) s = fmaf(sd2[u], p.W2[static_cast<int64_t>(u) * h1 + k], s);
        d1[static_cast<int64_t>(r) * h1 + k] = a1[static_cast<int64_t>(r) * h1 + k] > 0.0f ? s : 0.0f;
    }
}

// One thread per parameter: its gradient summed over the rows in order.
__global__ void surr_grad_kernel(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* __restrict__ x,
                                 const float* __restrict__ a1, const float* __restrict__ a2,
                                 const float* __restrict__ dy, const float* __restrict__ d1,
                                 const float* __restrict__ d2, float* __restrict__ grad)
{
    const int64_t n1 = static_cast<int64_t>(h1) * d_in, n2 = static_cast<int64_t>(h2) * h1;
    const int64_t total = n1 + h1 + n2 + h2 + h2 + 1;
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= total) return;
    float s = 0.0f;
    if (i < n1) {  // W1[u][k]: sum_r d1[r][u] x[r][k]
        const int64_t u = i / d_in, k = i - u * d_in;
        for (int32_t r = 0; r < n; ++r) s = fmaf(d1[static_cast<int64_t>(r) * h1 + u], x[static_cast<int64_t>(r) * d_in + k], s);
    } else if (i < n1 + h1) {
        const int64_t u = i - n1;
        for (int32_t r = 0; r < n; ++r) s += d1[static_cast<int64_t>(r) * h1 + u];
    } else if (i < n1 + h1 + n2) {  // W2[u][k]: sum_r d2[r][u] a1[r][k]
        const int64_t j = i - n1 - h1, u = j / h1, k = j - u * h1;
        for (int32_t r = 0; r < n; ++r)
            s = fmaf(d2[static_cast<int64_t>(r) * h2 + u], a1[static_cast<int64_t>(r) * h1 + k], s);
    } else if (i < n1 + h1 + n2 + h2) {
        const int64_t u = i - n1 - h1 - n2;
        for (int32_t r = 0; r < n; ++r) s += d2[static_cast<int64_t>(r) * h2 + u];
    } else if (i < n1 + h1 + n2 + h2 + h2) {  // w3[u]: sum_r dy_r a2[r][u]
        const int64_t u = i - n1 - h1 - n2 - h2;
        for (int32_t r = 0; r < n; ++r) s = fmaf(dy[r], a2[static_cast<int64_t>(r) * h2 + u], s);
    } else {
        for (int32_t r = 0; r < n; ++r) s += dy[r];
    }
    grad[i] = s;
}

// Mean squared error over the rows, one CTA, fixed-order tree.
__global__ void surr_loss_kernel(int32_t n, const float* __restrict__ y, const float* __restrict__ t,
                                 float* __restrict__ loss)
{
    __shared__ float red[256];
    float s = 0.0f;
    for (int32_t r = threadIdx.x; r < n; r += 256) {
        const float e = y[r] - t[r];
        s = fmaf(e, e, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / static_cast<float>(n);
}

__global__ void surr_adam_kernel(int64_t n, float* __restrict__ theta, const float* __restrict__ grad,
                                 float* __restrict__ m, float* __restrict__ v, float lr, float beta1, float beta2,
                                 float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float g = grad[i];
        const float mi = fmaf(beta1, m[i], (1.0f - beta1) * g);
        const float vi = fmaf(beta2, v[i], (1.0f - beta2) * g * g);
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace

int64_t surrogate_num_params(int32_t d_in, int32_t h1, int32_t h2)
{
    return static_cast<int64_t>(h1) * d_in + h1 + static_cast<int64_t>(h2) * h1 + h2 + h2 + 1;
}

size_t surrogate_forward_smem(int32_t d_in, int32_t h1, int32_t h2)
{
    return sizeof(float) * kRows * static_cast<size_t>(d_in + h1 + h2);
}

cudaError_t launch_surrogate_init(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, float* theta,
                                  cudaStream_t stream)
{
    const int64_t total = surrogate_num_params(d_in, h1, h2);
    surr_init_kernel<<<static_cast<int>((total + 255) / 256), 256, 0, stream>>>(d_in, h1, h2, seed, theta);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_forward(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta,
                                     const float* x, float* y, float* a1, float* a2, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = surrogate_forward_smem(d_in, h1, h2);
    cudaError_t err = cudaFuncSetAttribute(surr_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    // rows per CTA: 32 when the rows fill the GPU several times, fewer otherwise
    const int32_t rpc = n >= 32 * 512 ? 32 : (n >= 8 * 512 ? 8 : 2);
    surr_forward_kernel<<<(n + rpc - 1) / rpc, kFwdThreads, smem, stream>>>(n, d_in, h1, h2, rpc, theta, x, y, a1, a2);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_loss_grad(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta,
                                       const float* x, const float* t, float* loss, float* grad, float* work,
                                       cudaStream_t stream)
{
    // work: y [n], dy [n], a1 [n][h1], a2 [n][h2], d1 [n][h1], d2 [n][h2]
    float* yv = work;
    float* dy = yv + n;
    float* a1 = dy + n;
    float* a2 = a1 + static_cast<int64_t>(n) * h1;
    float* d1 = a2 + static_cast<int64_t>(n) * h2;
    float* d2 = d1 + static_cast<int64_t>(n) * h1;
    cudaError_t err = launch_surrogate_forward(n, d_in, h1, h2, theta, x, yv, a1, a2, stream);
    if (err != cudaSuccess) return err;
    surr_loss_kernel<<<1, 256, 0, stream>>>(n, yv, t, loss);
    surr_backrow_kernel<<<n, 64, sizeof(float) * h2, stream>>>(n, d_in, h1, h2, theta, yv, t, a1, a2, dy, d1, d2);
    const int64_t total = surrogate_num_params(d_in, h1, h2);
    surr_grad_kernel<<<static_cast<int>((total + 127) / 128), 128, 0, stream>>>(n, d_in, h1, h2, x, a1, a2, dy, d1,
                                                                              d2, grad);
    return cudaGetLastError();
}

size_t surrogate_work_floats(int32_t n, int32_t h1, int32_t h2)
{
    return static_cast<size_t>(n) * (2 + 2 * static_cast<size_t>(h1) + 2 * static_cast<size_t>(h2));
}

cudaError_t launch_surrogate_adam(int64_t n_params, float* theta, const float* grad, float* m, float* v, int64_t step,
                                  float lr, float beta1, float beta2, float eps, cudaStream_t stream)
{
    const float c1 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta1), static_cast<double>(step)));
    const float c2 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta2), static_cast<double>(step)));
    const int grid = static_cast<int>((n_params + 255) / 256 < 1024 ? (n_params + 255) / 256 : 1024);
    surr_adam_kernel<<<grid > 0 ? grid : 1, 256, 0, stream>>>(n_params, theta, grad, m, v, lr, beta1, beta2, eps, c1,
                                                              c2);
    return cudaGetLastError();
}

}  // namespace leea
