// leea_surrogate.cu -- the surrogate form's learned part: an MLP
// d_in -> h1 -> h2 -> 1 (ReLU) that scores offspring descriptors, with its
// own forward, backward (mean squared error) and Adam kernels.  The paper has
// no counterpart; it is the pre-screen that lets only the most promising
// offspring be made and evaluated.
//
// Parameters, flat FP32: W1 [h1][d_in], b1 [h1], W2 [h2][h1], b2 [h2],
// w3 [h2], b3.  Every reduction runs in a fixed order (a dot product: lane l
// of a warp sums k = l, l + 32, ... in order, then a fixed butterfly over the
// lanes; a gradient: 8 row segments in order, then the segments in order),
// so results do not depend on scheduling.
#include "leea_internal.h"
#include "philox.cuh"

#include <cmath>

namespace leea {

namespace {

constexpr uint32_t kTagSurrInit = 6;
constexpr int kRows = 32;      // rows per forward CTA at most (fewer for small n: more CTAs)
constexpr int kFwdWarps = 8;
constexpr int kFwdThreads = 32 * kFwdWarps;
constexpr int kSegs = 8;       // row segments of the gradient
constexpr int kGradParams = 32;  // parameters per gradient CTA (one per lane, a warp per segment)

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

// Sum of v over the 32 lanes, the same fixed butterfly in every lane.
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}

// out[r][u] = act(b[u] + sum_k W[u][k] in[r][k]) for R rows: warp w takes
// units u = w, w + 8, ...; lane l sums k = l, l + 32, ... (coalesced rows of
// W), then the lanes combine.
template <int R>
__device__ __forceinline__ void dense_rows(const float* __restrict__ W, const float* __restrict__ b, int32_t n_in,
                                           int32_t n_out, const float* in, float* out, bool relu, int warp, int lane)
{
    for (int u = warp; u < n_out; u += kFwdWarps) {
        float acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.0f;
        const float* w = W + static_cast<int64_t>(u) * n_in;
        for (int k = lane; k < n_in; k += 32) {
            const float wk = __ldg(w + k);
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fmaf(wk, in[r * n_in + k], acc[r]);
        }
        const float bu = __ldg(b + u);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float z = warp_sum(acc[r]) + bu;
            if (lane == 0) out[r * n_out + u] = relu ? fmaxf(z, 0.0f) : z;
        }
    }
}

// Forward for R rows per CTA; a1 / a2 (the ReLU outputs) are kept for the
// backward pass when not NULL.  With targets t (then a1, a2, dy, d1, d2 are
// all given) the same CTA also takes its rows' backward pass up to the
// per-row deltas: dy = 2 (y - t) / n, d2 = dy w3 (.) [a2 > 0],
// d1 = (W2^T d2) (.) [a1 > 0] (sums over the h2 units in order).
template <int R>
__global__ void __launch_bounds__(kFwdThreads)
surr_forward_kernel(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* __restrict__ theta,
                    const float* __restrict__ x, float* __restrict__ y, float* __restrict__ a1_out,
                    float* __restrict__ a2_out, const float* __restrict__ t, float* __restrict__ dy,
                    float* __restrict__ d1, float* __restrict__ d2)
{
    extern __shared__ float sm[];
    float* xs = sm;                     // [R][d_in]
    float* s1 = xs + R * d_in;          // [R][h1]
    float* s2 = s1 + R * h1;            // [R][h2]
    float* s3 = s2 + R * h2;            // [R]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const MlpView p = view(theta, d_in, h1, h2);
    const int32_t r0 = blockIdx.x * R;
    const int32_t rows = n - r0 < R ? n - r0 : R;
    for (int i = threadIdx.x; i < R * d_in; i += kFwdThreads) {
        const int r = i / d_in;
        xs[i] = r < rows ? x[static_cast<int64_t>(r0 + r) * d_in + (i - r * d_in)] : 0.0f;
    }
    __syncthreads();
    dense_rows<R>(p.W1, p.b1, d_in, h1, xs, s1, true, warp, lane);
    __syncthreads();
    dense_rows<R>(p.W2, p.b2, h1, h2, s1, s2, true, warp, lane);
    __syncthreads();
    if (warp == 0) dense_rows<R>(p.w3, p.b3, h2, 1, s2, s3, false, 0, lane);
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += kFwdThreads) y[r0 + r] = s3[r];
    if (a1_out)
        for (int o = threadIdx.x; o < rows * h1; o += kFwdThreads) a1_out[static_cast<int64_t>(r0) * h1 + o] = s1[o];
    if (a2_out)
        for (int o = threadIdx.x; o < rows * h2; o += kFwdThreads) a2_out[static_cast<int64_t>(r0) * h2 + o] = s2[o];
    if (!t) return;
    // deltas: s3 <- dy, s2 <- d2 (in place), then d1 per (row, hidden unit)
    __syncthreads();
    for (int r = threadIdx.x; r < rows; r += kFwdThreads) {
        const float g = 2.0f * (s3[r] - t[r0 + r]) / static_cast<float>(n);
        s3[r] = g;
        dy[r0 + r] = g;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < rows * h2; o += kFwdThreads) {
        const int r = o / h2, u = o - r * h2;
        const float v = s2[o] > 0.0f ? s3[r] * p.w3[u] : 0.0f;
        s2[o] = v;
        d2[static_cast<int64_t>(r0) * h2 + o] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < rows * h1; o += kFwdThreads) {
        const int r = o / h1, k = o - r * h1;
        float sum = 0.0f;
        for (int u = 0; u < h2; ++u) sum = fmaf(s2[r * h2 + u], p.W2[static_cast<int64_t>(u) * h1 + k], sum);
        d1[static_cast<int64_t>(r0) * h1 + o] = s1[o] > 0.0f ? sum : 0.0f;
    }
}

struct AdamArgs {
    float* theta;
    float *m, *v;
    float lr, beta1, beta2, eps, c1, c2;
};

// One Adam update of parameter i with gradient g (Kingma & Ba).
__device__ __forceinline__ void adam_update(const AdamArgs& ad, int64_t i, float g)
{
    const float mi = fmaf(ad.beta1, ad.m[i], (1.0f - ad.beta1) * g);
    const float vi = fmaf(ad.beta2, ad.v[i], (1.0f - ad.beta2) * g * g);
    ad.m[i] = mi;
    ad.v[i] = vi;
    ad.theta[i] -= ad.lr * (mi / ad.c1) / (sqrtf(vi / ad.c2) + ad.eps);
}

// Gradient: parameter i's sum over the rows, in kSegs segments of rows
// (warp = segment, lane = parameter: coalesced rows of x / a1 / a2), each
// summed in row order, then the segments in order.  ADAM: the parameter is
// updated at once instead of writing its gradient (the gradient reads no
// parameter, so the update cannot race with another CTA).
template <bool ADAM>
__global__ void __launch_bounds__(32 * kSegs)
surr_grad_kernel(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* __restrict__ x,
                 const float* __restrict__ a1, const float* __restrict__ a2, const float* __restrict__ dy,
                 const float* __restrict__ d1, const float* __restrict__ d2, float* __restrict__ grad,
                 const AdamArgs ad)
{
    __shared__ float part[kSegs][kGradParams];
    const int seg = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n1 = static_cast<int64_t>(h1) * d_in, n2 = static_cast<int64_t>(h2) * h1;
    const int64_t total = n1 + h1 + n2 + h2 + h2 + 1;
    const int64_t i = blockIdx.x * static_cast<int64_t>(kGradParams) + lane;
    const int32_t per = (n + kSegs - 1) / kSegs;
    const int32_t ra = seg * per, rb = ra + per < n ? ra + per : n;
    float s = 0.0f;
    if (i < total) {
        if (i < n1) {  // W1[u][k]: sum_r d1[r][u] x[r][k]
            const int64_t u = i / d_in, k = i - u * d_in;
            for (int32_t r = ra; r < rb; ++r)
                s = fmaf(d1[static_cast<int64_t>(r) * h1 + u], x[static_cast<int64_t>(r) * d_in + k], s);
        } else if (i < n1 + h1) {
            const int64_t u = i - n1;
            for (int32_t r = ra; r < rb; ++r) s += d1[static_cast<int64_t>(r) * h1 + u];
        } else if (i < n1 + h1 + n2) {  // W2[u][k]: sum_r d2[r][u] a1[r][k]
            const int64_t j = i - n1 - h1, u = j / h1, k = j - u * h1;
            for (int32_t r = ra; r < rb; ++r)
                s = fmaf(d2[static_cast<int64_t>(r) * h2 + u], a1[static_cast<int64_t>(r) * h1 + k], s);
        } else if (i < n1 + h1 + n2 + h2) {
            const int64_t u = i - n1 - h1 - n2;
            for (int32_t r = ra; r < rb; ++r) s += d2[static_cast<int64_t>(r) * h2 + u];
        } else if (i < n1 + h1 + n2 + h2 + h2) {  // w3[u]: sum_r dy_r a2[r][u]
            const int64_t u = i - n1 - h1 - n2 - h2;
            for (int32_t r = ra; r < rb; ++r) s = fmaf(dy[r], a2[static_cast<int64_t>(r) * h2 + u], s);
        } else {
            for (int32_t r = ra; r < rb; ++r) s += dy[r];
        }
    }
    part[seg][lane] = s;
    __syncthreads();
    if (seg == 0 && i < total) {
        float g = part[0][lane];
#pragma unroll
        for (int t = 1; t < kSegs; ++t) g += part[t][lane];
        if (ADAM)
            adam_update(ad, i, g);
        else
            grad[i] = g;
    }
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
        adam_update(AdamArgs{ theta, m, v, lr, beta1, beta2, eps, c1, c2 }, i, grad[i]);
    }
}

}  // namespace

int64_t surrogate_num_params(int32_t d_in, int32_t h1, int32_t h2)
{
    return static_cast<int64_t>(h1) * d_in + h1 + static_cast<int64_t>(h2) * h1 + h2 + h2 + 1;
}

size_t surrogate_forward_smem(int32_t d_in, int32_t h1, int32_t h2)
{
    return sizeof(float) * kRows * static_cast<size_t>(d_in + h1 + h2 + 1);
}

cudaError_t launch_surrogate_init(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, float* theta,
                                  cudaStream_t stream)
{
    const int64_t total = surrogate_num_params(d_in, h1, h2);
    surr_init_kernel<<<static_cast<int>((total + 255) / 256), 256, 0, stream>>>(d_in, h1, h2, seed, theta);
    return cudaGetLastError();
}

namespace {

cudaError_t forward_rows(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta, const float* x, float* y,
                         float* a1, float* a2, const float* t, float* dy, float* d1, float* d2, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    // rows per CTA: enough CTAs to spread over the SMs, as many rows as that
    // allows (each CTA streams all of W1 once)
    const int32_t rpc = n >= 32 * 128 ? 32 : (n >= 8 * 128 ? 8 : 2);
    const size_t smem = sizeof(float) * rpc * static_cast<size_t>(d_in + h1 + h2 + 1);
    const int grid = (n + rpc - 1) / rpc;
    cudaError_t err;
    if (rpc == 32) {
        err = cudaFuncSetAttribute(surr_forward_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(smem));
        if (err == cudaSuccess)
            surr_forward_kernel<32><<<grid, kFwdThreads, smem, stream>>>(n, d_in, h1, h2, theta, x, y, a1, a2, t, dy,
                                                                         d1, d2);
    } else if (rpc == 8) {
        err = cudaFuncSetAttribute(surr_forward_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(smem));
        if (err == cudaSuccess)
            surr_forward_kernel<8><<<grid, kFwdThreads, smem, stream>>>(n, d_in, h1, h2, theta, x, y, a1, a2, t, dy,
                                                                         d1, d2);
    } else {
        err = cudaFuncSetAttribute(surr_forward_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(smem));
        if (err == cudaSuccess)
            surr_forward_kernel<2><<<grid, kFwdThreads, smem, stream>>>(n, d_in, h1, h2, theta, x, y, a1, a2, t, dy,
                                                                         d1, d2);
    }
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_surrogate_forward(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta,
                                     const float* x, float* y, float* a1, float* a2, cudaStream_t stream)
{
    return forward_rows(n, d_in, h1, h2, theta, x, y, a1, a2, nullptr, nullptr, nullptr, nullptr, stream);
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
    cudaError_t err = forward_rows(n, d_in, h1, h2, theta, x, yv, a1, a2, t, dy, d1, d2, stream);
    if (err != cudaSuccess) return err;
    surr_loss_kernel<<<1, 256, 0, stream>>>(n, yv, t, loss);
    const int64_t total = surrogate_num_params(d_in, h1, h2);
    surr_grad_kernel<false><<<static_cast<int>((total + kGradParams - 1) / kGradParams), 32 * kSegs, 0, stream>>>(
        n, d_in, h1, h2, x, a1, a2, dy, d1, d2, grad, AdamArgs{});
    return cudaGetLastError();
}

cudaError_t launch_surrogate_train_step(int32_t n, int32_t d_in, int32_t h1, int32_t h2, float* theta, const float* x,
                                        const float* t, float* loss, float* work, float* m, float* v, int64_t step,
                                        float lr, float beta1, float beta2, float eps, cudaStream_t stream)
{
    float* yv = work;
    float* dy = yv + n;
    float* a1 = dy + n;
    float* a2 = a1 + static_cast<int64_t>(n) * h1;
    float* d1 = a2 + static_cast<int64_t>(n) * h2;
    float* d2 = d1 + static_cast<int64_t>(n) * h1;
    cudaError_t err = forward_rows(n, d_in, h1, h2, theta, x, yv, a1, a2, t, dy, d1, d2, stream);
    if (err != cudaSuccess) return err;
    if (loss) surr_loss_kernel<<<1, 256, 0, stream>>>(n, yv, t, loss);
    AdamArgs ad{ theta, m, v, lr, beta1, beta2, eps,
                 static_cast<float>(1.0 - std::pow(static_cast<double>(beta1), static_cast<double>(step))),
                 static_cast<float>(1.0 - std::pow(static_cast<double>(beta2), static_cast<double>(step))) };
    const int64_t total = surrogate_num_params(d_in, h1, h2);
    surr_grad_kernel<true><<<static_cast<int>((total + kGradParams - 1) / kGradParams), 32 * kSegs, 0, stream>>>(
        n, d_in, h1, h2, x, a1, a2, dy, d1, d2, nullptr, ad);
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
