// leea_eval_simt.cu -- fitness of every individual on one shared minibatch
// (Eq. 1; Section 3.3's population-batched forward pass), exact FP32 on the
// CUDA cores.  General in d_0, h, d_out <= 32 and batch.
//
// One CTA per individual p.  The hidden layer H = ReLU(W1_p X^T + b1_p) is
// computed tile by tile (BM hidden units x BN samples, K-loop over d_0 with
// double-buffered shared-memory tiles and a TM x TN register micro-tile per
// thread); each finished tile goes straight through layer 2 into per-sample
// logits kept in shared memory, so neither H nor the logits reach HBM.  The
// per-sample cross-entropy (maximum subtracted, FP32) and the sum over the
// batch use fixed reduction orders: identical individuals give bitwise
// identical fitness.
#include "leea_internal.h"

namespace leea {

constexpr int kEvalThreads = 256;  // 16 x 16 thread grid
constexpr int kBK = 16;
constexpr int kMaxOut = 32;

struct EvalSimtArgs {
    int32_t d_in, h, d_out, batch;
    int64_t c_pad;
    float alpha;
    float x_div;  // 8-bit inputs: x = k / x_div
};

__device__ __forceinline__ float input_value(float v, float) { return v; }
__device__ __forceinline__ float input_value(uint8_t k, float div) { return static_cast<float>(k) / div; }

template <int TM, int TN>
struct SimtTile {
    static constexpr int BM = 16 * TM;
    static constexpr int BN = 16 * TN;
    static constexpr int AS = BM + 4;  // padded row of the k-major A tile
    static constexpr int BS = BN + 4;
    static constexpr int HS = BN + 4;
    static size_t smem_bytes(int d_out)
    {
        return sizeof(float) * (2 * kBK * AS + 2 * kBK * BS + BM * HS + d_out * BM + d_out * BN + BN) +
               sizeof(int32_t) * (BN + 32);
    }
};

template <int TM, int TN, typename XT>
__global__ void __launch_bounds__(kEvalThreads, 2)
eval_simt_kernel(EvalSimtArgs e, const float* __restrict__ popv, const XT* __restrict__ x,
                 const int32_t* __restrict__ y, const float* __restrict__ f_inh,
                 float* __restrict__ f_raw, float* __restrict__ f_adj, int32_t* __restrict__ correct)
{
    using T = SimtTile<TM, TN>;
    constexpr int BM = T::BM, BN = T::BN, AS = T::AS, BS = T::BS, HS = T::HS;
    extern __shared__ float4 smem4[];
    float* smem = reinterpret_cast<float*>(smem4);
    float* As = smem;                      // [2][kBK][AS]
    float* Bs = As + 2 * kBK * AS;         // [2][kBK][BS]
    float* Hs = Bs + 2 * kBK * BS;         // [BM][HS]
    float* W2s = Hs + BM * HS;             // [d_out][BM]
    float* Ls = W2s + e.d_out * BM;        // [d_out][BN]
    float* lossv = Ls + e.d_out * BN;      // [BN]
    int32_t* corv = reinterpret_cast<int32_t*>(lossv + BN);  // [BN]
    float* warp_sums = reinterpret_cast<float*>(corv + BN);  // [32]

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int p = blockIdx.x;
    const int K = e.d_in, H = e.h, D = e.d_out, Bt = e.batch;
    const float* W1 = popv + static_cast<int64_t>(p) * e.c_pad;
    const float* b1 = W1 + static_cast<int64_t>(H) * K;
    const float* W2 = b1 + H;
    const float* b2 = W2 + static_cast<int64_t>(D) * H;

    const int nk = (K + kBK - 1) / kBK;
    float total = 0.0f;  // meaningful in thread 0 only
    int32_t n_correct = 0;

    for (int b0 = 0; b0 < Bt; b0 += BN) {
        for (int t = tid; t < D * BN; t += kEvalThreads) Ls[t] = 0.0f;

        for (int h0 = 0; h0 < H; h0 += BM) {
            float acc[TM][TN];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int jn = 0; jn < TN; ++jn) acc[i][jn] = 0.0f;

            // Register staging of one K-tile: TM elements of A, TN of B per thread.
            float ra[TM], rb[TN];
            auto load_tile = [&](int kt) {
                const int k0 = kt * kBK;
#pragma unroll
                for (int u = 0; u < TM; ++u) {
                    const int idx = tid + u * kEvalThreads;  // < BM * kBK
                    const int r = idx / kBK, k = idx % kBK;
                    const int gr = h0 + r, gk = k0 + k;
                    ra[u] = (gr < H && gk < K) ? W1[static_cast<int64_t>(gr) * K + gk] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < TN; ++u) {
                    const int idx = tid + u * kEvalThreads;  // < BN * kBK
                    const int n = idx / kBK, k = idx % kBK;
                    const int gn = b0 + n, gk = k0 + k;
                    rb[u] = (gn < Bt && gk < K) ? input_value(x[static_cast<int64_t>(gn) * K + gk], e.x_div) : 0.0f;
                }
            };
            auto store_tile = [&](int buf) {
                float* a = As + buf * kBK * AS;
                float* b = Bs + buf * kBK * BS;
#pragma unroll
                for (int u = 0; u < TM; ++u) {
                    const int idx = tid + u * kEvalThreads;
                    a[(idx % kBK) * AS + idx / kBK] = ra[u];
                }
#pragma unroll
                for (int u = 0; u < TN; ++u) {
                    const int idx = tid + u * kEvalThreads;
                    b[(idx % kBK) * BS + idx / kBK] = rb[u];
                }
            };

            load_tile(0);
            store_tile(0);
            __syncthreads();
            for (int kt = 0; kt < nk; ++kt) {
                const int buf = kt & 1;
                if (kt + 1 < nk) load_tile(kt + 1);
                const float* a = As + buf * kBK * AS + ty * TM;
                const float* b = Bs + buf * kBK * BS + tx * TN;
#pragma unroll
                for (int k = 0; k < kBK; ++k) {
                    float av[TM], bv[TN];
#pragma unroll
                    for (int i = 0; i < TM; ++i) av[i] = a[k * AS + i];
#pragma unroll
                    for (int jn = 0; jn < TN; ++jn) bv[jn] = b[k * BS + jn];
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int jn = 0; jn < TN; ++jn) acc[i][jn] = fmaf(av[i], bv[jn], acc[i][jn]);
                }
                if (kt + 1 < nk) store_tile(buf ^ 1);
                __syncthreads();
            }

            // Bias + ReLU into the hidden tile; stage the matching W2 columns.
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const int r = ty * TM + i;
                const float bias = (h0 + r < H) ? b1[h0 + r] : 0.0f;
#pragma unroll
                for (int jn = 0; jn < TN; ++jn) Hs[r * HS + tx * TN + jn] = fmaxf(acc[i][jn] + bias, 0.0f);
            }
            for (int t = tid; t < D * BM; t += kEvalThreads) {
                const int o = t / BM, r = t % BM;
                W2s[t] = (h0 + r < H) ? W2[static_cast<int64_t>(o) * H + h0 + r] : 0.0f;
            }
            __syncthreads();
            // Layer 2 on this tile: logits[o][n] += sum_r W2[o][r] H[r][n], r ascending.
            for (int t = tid; t < D * BN; t += kEvalThreads) {
                const int o = t / BN, n = t % BN;
                float s = Ls[t];
                const float* w = W2s + o * BM;
#pragma unroll 8
                for (int r = 0; r < BM; ++r) s = fmaf(w[r], Hs[r * HS + n], s);
                Ls[t] = s;
            }
            __syncthreads();
        }

        // Per-sample cross-entropy of the softmax output (Eq. 1) and argmax.
        if (tid < BN) {
            const int n = tid, gn = b0 + n;
            float loss = 0.0f;
            int32_t ok = 0;
            if (gn < Bt) {
                float zmax = Ls[n] + b2[0];
                int arg = 0;
                for (int o = 1; o < D; ++o) {
                    const float z = Ls[o * BN + n] + b2[o];
                    if (z > zmax) { zmax = z; arg = o; }
                }
                float s = 0.0f;
                for (int o = 0; o < D; ++o) s += expf(Ls[o * BN + n] + b2[o] - zmax);
                const int32_t lbl = y[gn];
                if (lbl >= 0 && lbl < D) {
                    loss = logf(s) + zmax - (Ls[lbl * BN + n] + b2[lbl]);
                    ok = (arg == lbl) ? 1 : 0;
                } else {
                    loss = __int_as_float(0x7FC00000);  // NaN: label out of range
                }
            }
            lossv[n] = loss;
            corv[n] = ok;
        }
        __syncthreads();
        // Fixed-order reduction over the tile's samples: warp xor-tree, then
        // warp sums in order.
        if (tid < BN) {
            float v = lossv[tid];
            int32_t cv = corv[tid];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
                cv += __shfl_xor_sync(0xFFFFFFFFu, cv, off);
            }
            if ((tid & 31) == 0) {
                warp_sums[tid >> 5] = v;
                corv[tid] = cv;  // lane 0 of each warp keeps the warp's count
            }
        }
        __syncthreads();
        if (tid == 0) {
            float s = 0.0f;
            for (int w = 0; w < (BN + 31) / 32; ++w) {
                s += warp_sums[w];
                n_correct += corv[w * 32];
            }
            total += s;
        }
        __syncthreads();
    }

    if (tid == 0) {
        const float f = -(total / static_cast<float>(Bt));
        f_raw[p] = f;
        if (f_adj) f_adj[p] = f_inh ? (1.0f - e.alpha) * f_inh[p] + e.alpha * f : f;
        if (correct) correct[p] = n_correct;
    }
}

template <int TM, int TN, typename XT>
static cudaError_t launch_simt_t(const EvalSimtArgs& e, int32_t pop, const float* popv, const XT* x,
                                 const int32_t* y, const float* f_inh, float* f_raw, float* f_adj,
                                 int32_t* correct, cudaStream_t stream)
{
    const size_t smem = SimtTile<TM, TN>::smem_bytes(e.d_out);
    cudaError_t err = cudaFuncSetAttribute(eval_simt_kernel<TM, TN, XT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    eval_simt_kernel<TM, TN, XT><<<pop, kEvalThreads, smem, stream>>>(e, popv, x, y, f_inh, f_raw, f_adj,
                                                                       correct);
    return cudaGetLastError();
}

static int pick_micro(int extent)
{
    return extent <= 32 ? 2 : extent <= 64 ? 4 : 8;
}

template <typename XT>
static cudaError_t launch_simt_any(const NetLayout& net, int32_t pop, const float* pop_dev, const XT* x,
                                   float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                   float* f_raw, float* f_adj, int32_t* correct, cudaStream_t stream)
{
    if (net.n_layers != 2 || net.dims[2] > kMaxOut) return cudaErrorInvalidValue;
    EvalSimtArgs e{ net.dims[0], net.dims[1], net.dims[2], batch, net.c_pad, alpha, x_div };
    const int tm = pick_micro(e.h), tn = pick_micro(batch);
#define LEEA_SIMT_CASE(A, B)                                                                      \
    if (tm == A && tn == B)                                                                       \
        return launch_simt_t<A, B, XT>(e, pop, pop_dev, x, y, f_inh, f_raw, f_adj, correct, stream);
    LEEA_SIMT_CASE(2, 2) LEEA_SIMT_CASE(2, 4) LEEA_SIMT_CASE(2, 8)
    LEEA_SIMT_CASE(4, 2) LEEA_SIMT_CASE(4, 4) LEEA_SIMT_CASE(4, 8)
    LEEA_SIMT_CASE(8, 2) LEEA_SIMT_CASE(8, 4) LEEA_SIMT_CASE(8, 8)
#undef LEEA_SIMT_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_eval_simt(const NetLayout& net, int32_t pop, const float* pop_dev,
                             const float* x, const int32_t* y, int32_t batch, float alpha,
                             const float* f_inh, float* f_raw, float* f_adj, int32_t* correct,
                             cudaStream_t stream)
{
    return launch_simt_any<float>(net, pop, pop_dev, x, 1.0f, y, batch, alpha, f_inh, f_raw, f_adj, correct,
                                  stream);
}

cudaError_t launch_eval_simt_u8(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                                float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                float* f_raw, float* f_adj, int32_t* correct, cudaStream_t stream)
{
    return launch_simt_any<uint8_t>(net, pop, pop_dev, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct,
                                    stream);
}

}  // namespace leea
