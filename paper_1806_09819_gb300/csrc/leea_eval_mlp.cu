// leea_eval_mlp.cu -- fitness (Eq. 1) of nets with several hidden layers, such
// as the paper's own 196-256-128-64-10 behind 2x2 max-pooling (Section 4.1),
// exact FP32 on the CUDA cores; and the max-pooling input stage itself.
//
// One CTA per individual walks the batch in tiles of 64 samples.  Each layer
// is a [64 x K] x [K x N] product: the activations stay in shared memory,
// k-major (act[k][s], so a thread reads 4 samples of one input with one
// 128-bit load), and the weights W_l (N rows of K, the gene order) pass
// through shared memory transposed in chunks of 32 inputs, double-buffered
// through registers.  A thread owns 4 samples x TO outputs (TO = N / 32
// rounded up), so 512 threads cover 64 samples x up to 256 outputs in one pass.
// Hidden layers add the bias and apply ReLU into the other activation
// buffer; the last layer leaves the logits in shared memory, where the first
// two warps take the softmax cross-entropy of the tile's 64 samples, a thread
// per sample (maximum subtracted, FP32), and the argmax.  Each tile's two warp
// sums are added in order, the tiles in order: identical individuals give
// bitwise identical fitness.
#include "leea_internal.h"

namespace leea {

namespace {

constexpr int kMlpThreads = 512;
constexpr int kTS = 64;         // samples per tile
constexpr int kKC = 32;         // inputs per weight chunk
constexpr int kMaxWidth = 256;  // widest layer input / hidden layer
constexpr int kMaxOutMlp = 32;
constexpr int kActStride = kTS + 4;          // act[k][s] row stride (floats)
constexpr int kWStride = kMaxWidth + 4;      // WT[kk][o] row stride (floats)
constexpr int kLogitStride = kMaxOutMlp + 1;

struct MlpArgs {
    int32_t n_layers, batch;
    int32_t dims[kMaxLayers + 1];
    int64_t w_off[kMaxLayers], b_off[kMaxLayers];
    int64_t c_pad;
    float alpha, x_div;
};

constexpr size_t kMlpSmemBytes =
    sizeof(float) * (2 * kMaxWidth * kActStride + 2 * kKC * kWStride + kTS * kLogitStride) + 64;

__device__ __forceinline__ float mlp_input(float v, float) { return v; }
__device__ __forceinline__ float mlp_input(uint8_t k, float div) { return static_cast<float>(k) / div; }

// One layer on the current tile: out = act_in (32 x K) x W^T (K x N) + b,
// ReLU into act_out[o][s] (hidden) or the logits[s][o] (last layer).
template <int TO>
__device__ __forceinline__ void mlp_layer(const float* __restrict__ W, const float* __restrict__ b, int K, int N,
                                          bool last, const float* act_in, float* act_out, float* logits, float* wt)
{
    const int tid = threadIdx.x;
    const int sg = tid & 15;  // samples 4 sg .. 4 sg + 3
    const int og = tid >> 4;  // outputs og TO .. og TO + TO - 1
    float acc[4][TO];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TO; ++j) acc[i][j] = 0.0f;

    // Weight chunk c: WT[kk][o] = W[o][32 c + kk]; thread t stages rows o = t / 32
    // + 16 u of input kk = t % 32 (a warp's loads cover one row's 128 contiguous
    // bytes), double-buffered through registers.  Inputs past K get zeros.
    constexpr int kRowsPerPass = kMlpThreads / kKC;  // 16
    const int n_chunks = (K + kKC - 1) / kKC;
    const int kk_l = tid % kKC, o_l = tid / kKC;
    float stage[kMaxWidth / kRowsPerPass];
    auto load_chunk = [&](int c) {
        const int k = c * kKC + kk_l;
#pragma unroll
        for (int u = 0; u < kMaxWidth / kRowsPerPass; ++u) {
            const int o = o_l + kRowsPerPass * u;
            stage[u] = (o < N && k < K) ? __ldg(W + static_cast<int64_t>(o) * K + k) : 0.0f;
        }
    };
    auto store_chunk = [&](int buf) {
        float* dst = wt + buf * kKC * kWStride + kk_l * kWStride;
#pragma unroll
        for (int u = 0; u < kMaxWidth / kRowsPerPass; ++u) {
            const int o = o_l + kRowsPerPass * u;
            if (o < N) dst[o] = stage[u];
        }
    };
    load_chunk(0);
    store_chunk(0);
    __syncthreads();
    for (int c = 0; c < n_chunks; ++c) {
        const int buf = c & 1;
        if (c + 1 < n_chunks) load_chunk(c + 1);
        const float* wb = wt + buf * kKC * kWStride;
        const float* ab = act_in + c * kKC * kActStride + 4 * sg;
        // Inputs past K (up to K rounded to 32) hold zero weights and zero
        // activations: the input tile and every hidden layer write zeros there.
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(ab + kk * kActStride);
            float w[TO];
            if constexpr (TO % 4 == 0) {
#pragma unroll
                for (int j = 0; j < TO; j += 4) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wb + kk * kWStride + og * TO + j);
                    w[j] = w4.x;
                    w[j + 1] = w4.y;
                    w[j + 2] = w4.z;
                    w[j + 3] = w4.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < TO; ++j) w[j] = wb[kk * kWStride + og * TO + j];
            }
#pragma unroll
            for (int j = 0; j < TO; ++j) {
                acc[0][j] = fmaf(a.x, w[j], acc[0][j]);
                acc[1][j] = fmaf(a.y, w[j], acc[1][j]);
                acc[2][j] = fmaf(a.z, w[j], acc[2][j]);
                acc[3][j] = fmaf(a.w, w[j], acc[3][j]);
            }
        }
        if (c + 1 < n_chunks) store_chunk(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TO; ++j) {
        const int o = og * TO + j;
        if (!last && o >= N && o < ((N + kKC - 1) / kKC) * kKC) {
            *reinterpret_cast<float4*>(act_out + o * kActStride + 4 * sg) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (o < N) {
            const float bo = __ldg(b + o);
            if (last) {
#pragma unroll
                for (int i = 0; i < 4; ++i) logits[(4 * sg + i) * kLogitStride + o] = acc[i][j] + bo;
            } else {  // 4 samples of output o: one 16-byte store
                *reinterpret_cast<float4*>(act_out + o * kActStride + 4 * sg) =
                    make_float4(fmaxf(acc[0][j] + bo, 0.0f), fmaxf(acc[1][j] + bo, 0.0f),
                                fmaxf(acc[2][j] + bo, 0.0f), fmaxf(acc[3][j] + bo, 0.0f));
            }
        }
    }
    __syncthreads();
}

template <typename XT>
__global__ void __launch_bounds__(kMlpThreads, 1)
eval_mlp_kernel(const MlpArgs e, const float* __restrict__ popv, const XT* __restrict__ x,
                const int32_t* __restrict__ y, const float* __restrict__ f_inh, float* __restrict__ f_raw,
                float* __restrict__ f_adj, int32_t* __restrict__ correct, const int32_t* __restrict__ only)
{
    if (only && only[blockIdx.x] == 0) return;  // only the marked individuals
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    float* act[2] = { smem, smem + kMaxWidth * kActStride };
    float* wt = smem + 2 * kMaxWidth * kActStride;  // [2][kKC][kWStride]
    float* logits = wt + 2 * kKC * kWStride;        // [kTS][kLogitStride]
    float* red = logits + kTS * kLogitStride;        // [2]: per-warp loss sums of a tile
    int32_t* red_ok = reinterpret_cast<int32_t*>(red + 2);
    const int tid = threadIdx.x;
    const int p = blockIdx.x;
    const float* net = popv + static_cast<int64_t>(p) * e.c_pad;
    const int d0 = e.dims[0], d_out = e.dims[e.n_layers];
    float total = 0.0f;
    int32_t n_ok = 0;
    for (int b0 = 0; b0 < e.batch; b0 += kTS) {
        // Input tile, k-major; samples past the batch are zero.
        const int d0r = (d0 + kKC - 1) / kKC * kKC;  // rows up to the chunk boundary: zero past d0
        for (int sk = tid; sk < kTS * kMaxWidth; sk += kMlpThreads) {
            const int s = sk / kMaxWidth, k = sk % kMaxWidth;  // powers of two: shifts
            if (k < d0r)
                act[0][k * kActStride + s] = (b0 + s < e.batch && k < d0)
                                                 ? mlp_input(x[static_cast<int64_t>(b0 + s) * d0 + k], e.x_div)
                                                 : 0.0f;
        }
        __syncthreads();
        for (int l = 0; l < e.n_layers; ++l) {
            const int K = e.dims[l], N = e.dims[l + 1];
            const bool last = l == e.n_layers - 1;
            const float* W = net + e.w_off[l];
            const float* b = net + e.b_off[l];
            const float* in = act[l & 1];
            float* out = act[(l + 1) & 1];
            const int to = (N + 31) / 32;
            if (to <= 1) mlp_layer<1>(W, b, K, N, last, in, out, logits, wt);
            else if (to <= 2) mlp_layer<2>(W, b, K, N, last, in, out, logits, wt);
            else if (to <= 4) mlp_layer<4>(W, b, K, N, last, in, out, logits, wt);
            else mlp_layer<8>(W, b, K, N, last, in, out, logits, wt);
        }
        if (tid < kTS) {  // one sample per thread of the first two warps
            const int s = tid;
            float loss = 0.0f;
            int32_t good = 0;
            if (b0 + s < e.batch) {
                const float* z = logits + s * kLogitStride;
                float zmax = z[0];
                int arg = 0;
                for (int o = 1; o < d_out; ++o)
                    if (z[o] > zmax) { zmax = z[o]; arg = o; }
                float se = 0.0f;
                for (int o = 0; o < d_out; ++o) se += expf(z[o] - zmax);
                const int32_t lbl = y[b0 + s];
                if (lbl >= 0 && lbl < d_out) {
                    loss = logf(se) + zmax - z[lbl];
                    good = arg == lbl ? 1 : 0;
                } else {
                    loss = __int_as_float(0x7FC00000);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
                good += __shfl_xor_sync(0xFFFFFFFFu, good, off);
            }
            if ((tid & 31) == 0) {
                red[tid >> 5] = loss;
                red_ok[tid >> 5] = good;
            }
        }
        __syncthreads();  // the logits and activations are rewritten by the next tile
        if (tid == 0) {   // the tile's two warp sums, in order
            total += red[0] + red[1];
            n_ok += red_ok[0] + red_ok[1];
        }
    }
    if (tid == 0) {
        const float f = -(total / static_cast<float>(e.batch));
        f_raw[p] = f;
        if (f_adj) f_adj[p] = f_inh ? (1.0f - e.alpha) * f_inh[p] + e.alpha * f : f;
        if (correct) correct[p] = n_ok;
    }
}

template <typename XT>
__global__ void maxpool2x2_kernel(int32_t batch, int32_t h, int32_t w, const XT* __restrict__ x, XT* __restrict__ out)
{
    const int32_t ho = h >> 1, wo = w >> 1;
    const int64_t n = static_cast<int64_t>(batch) * ho * wo;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < n;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = t / (ho * wo);
        const int32_t r = static_cast<int32_t>(t - b * ho * wo);
        const int32_t i = r / wo, j = r - i * wo;
        const XT* img = x + b * h * w + static_cast<int64_t>(2 * i) * w + 2 * j;
        XT m = img[0];
        if (img[1] > m) m = img[1];
        if (img[w] > m) m = img[w];
        if (img[w + 1] > m) m = img[w + 1];
        out[t] = m;
    }
}

MlpArgs mlp_args(const NetLayout& net, int32_t batch, float alpha, float x_div)
{
    MlpArgs e{};
    e.n_layers = net.n_layers;
    e.batch = batch;
    for (int l = 0; l <= net.n_layers; ++l) e.dims[l] = net.dims[l];
    for (int l = 0; l < net.n_layers; ++l) {
        e.w_off[l] = net.w_off[l];
        e.b_off[l] = net.b_off[l];
    }
    e.c_pad = net.c_pad;
    e.alpha = alpha;
    e.x_div = x_div;
    return e;
}

template <typename XT>
cudaError_t launch_mlp(const NetLayout& net, int32_t pop, const float* pop_dev, const XT* x, float x_div,
                       const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw, float* f_adj,
                       int32_t* correct, cudaStream_t stream, const int32_t* only = nullptr)
{
    cudaError_t err = cudaFuncSetAttribute(eval_mlp_kernel<XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(kMlpSmemBytes));
    if (err != cudaSuccess) return err;
    eval_mlp_kernel<XT><<<pop, kMlpThreads, kMlpSmemBytes, stream>>>(mlp_args(net, batch, alpha, x_div), pop_dev, x, y,
                                                                    f_inh, f_raw, f_adj, correct, only);
    return cudaGetLastError();
}

}  // namespace

bool eval_mlp_supported(const NetLayout& net)
{
    if (net.n_layers < 2 || net.dims[net.n_layers] > kMaxOutMlp) return false;
    for (int l = 0; l < net.n_layers; ++l)
        if (net.dims[l] > kMaxWidth) return false;
    return true;
}

cudaError_t launch_eval_mlp(const NetLayout& net, int32_t pop, const float* pop_dev, const float* x, const int32_t* y,
                            int32_t batch, float alpha, const float* f_inh, float* f_raw, float* f_adj,
                            int32_t* correct, cudaStream_t stream)
{
    return launch_mlp<float>(net, pop, pop_dev, x, 1.0f, y, batch, alpha, f_inh, f_raw, f_adj, correct, stream);
}

cudaError_t launch_eval_mlp_u8(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x, float x_div,
                               const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                               float* f_adj, int32_t* correct, cudaStream_t stream)
{
    return launch_mlp<uint8_t>(net, pop, pop_dev, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct, stream);
}

cudaError_t launch_eval_mlp_u8_only(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                                    float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                    float* f_raw, float* f_adj, int32_t* correct, const int32_t* only,
                                    cudaStream_t stream)
{
    return launch_mlp<uint8_t>(net, pop, pop_dev, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct, stream,
                               only);
}

template <typename XT>
static cudaError_t launch_pool(int32_t batch, int32_t h, int32_t w, const XT* x, XT* out, cudaStream_t stream)
{
    const int64_t n = static_cast<int64_t>(batch) * (h / 2) * (w / 2);
    if (n == 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    maxpool2x2_kernel<XT><<<static_cast<int>(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(batch, h, w, x, out);
    return cudaGetLastError();
}

cudaError_t launch_maxpool2x2(int32_t batch, int32_t h, int32_t w, const float* x, float* out, cudaStream_t stream)
{
    return launch_pool<float>(batch, h, w, x, out, stream);
}

cudaError_t launch_maxpool2x2_u8(int32_t batch, int32_t h, int32_t w, const uint8_t* x, uint8_t* out,
                                 cudaStream_t stream)
{
    return launch_pool<uint8_t>(batch, h, w, x, out, stream);
}

}  // namespace leea
