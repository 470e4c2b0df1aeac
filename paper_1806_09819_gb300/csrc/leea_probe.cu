// leea_probe.cu -- the surrogate form's fused breed + probe pass: for each
// recipe (a virtual offspring: kind, parents and the Philox entity whose
// streams make its genes, Section 3.2's operators) it regenerates the child's
// genes from the parents without writing them, runs the child (d_0-h-d_out,
// ReLU) on a small probe batch and writes the recipe's descriptor:
//   [f_adj of parent 1, f_adj of parent 2, f_inh, crossover fraction,
//    mutation step length sigma ||z (.) m||, probe logits (n_probe x d_out)].
//
// One CTA per recipe.  Layer 1 runs over K tiles of 64 inputs: the child's W1
// tile (h x 64 genes, 8 genes per thread and Philox block) and the probe
// tile go to shared memory transposed, and each thread accumulates a 4 x 4
// block of (sample, hidden unit) sums in registers (FP32, k in order).
#include "leea_internal.h"
#include "philox.cuh"

namespace leea {

namespace {

constexpr uint32_t kTagXo = 3, kTagMutMask = 4, kTagNormal = 5;
constexpr int kProbeThreads = 256;
constexpr int kKT = 64;          // inputs per K tile
constexpr int kMaxProbe = 32;    // probe samples
constexpr int kMaxHidden = 256;

__device__ __forceinline__ uint32_t draws8_mask(const uint4& r, uint32_t thr)
{
    const uint32_t w[4] = { r.x, r.y, r.z, r.w };
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t u = (k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xFFFFu);
        m |= (u < thr ? 1u : 0u) << k;
    }
    return m;
}

// Genes i .. i+7 (i % 8 == 0) of a child of the given kind: out[8] and, for
// the descriptor, the XO hits and the sum of z^2 over masked genes (genes
// >= c excluded).
__device__ __forceinline__ void child_genes8(const ProbeArgs& a, const PhiloxKeys& key, int32_t kind, uint32_t ent,
                                             const float* __restrict__ pa, const float* __restrict__ pb, int64_t i,
                                             float (&out)[8], uint32_t& xo_hits, float& zz)
{
    const float4 a0 = *reinterpret_cast<const float4*>(pa + i), a1 = *reinterpret_cast<const float4*>(pa + i + 4);
    float v[8] = { a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w };
    const int64_t live = a.c - i;  // genes of this unit below c (may exceed 8)
    const uint32_t in_c = live >= 8 ? 0xFFu : (live > 0 ? ((1u << live) - 1u) : 0u);
    if (kind == 1) {
        const float4 b0 = *reinterpret_cast<const float4*>(pb + i), b1 = *reinterpret_cast<const float4*>(pb + i + 4);
        const float w[8] = { b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w };
        if (a.xo_op == 0) {
            const uint32_t m = draws8_mask(philox_keyed(make_uint4(static_cast<uint32_t>(i >> 3), ent, a.gen, kTagXo), key),
                                           a.thr_xo);
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = ((m >> t) & 1u) ? w[t] : v[t];
            xo_hits += __popc(m & in_c);
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = 0.5f * (v[t] + w[t]);
        }
    } else if (kind == 2) {
        const uint32_t m =
            draws8_mask(philox_keyed(make_uint4(static_cast<uint32_t>(i >> 3), ent, a.gen, kTagMutMask), key),
                        a.thr_mut);
        if (m) {
#pragma unroll
            for (int pr = 0; pr < 4; ++pr) {  // Box-Muller pairs (i + 2 pr, i + 2 pr + 1)
                if ((m >> (2 * pr)) & 3u) {
                    const uint32_t g = static_cast<uint32_t>(i) + 2u * pr;  // even gene of the pair
                    const uint4 n = philox_keyed(make_uint4(g >> 2, ent, a.gen, kTagNormal), key);
                    const float2 z = (g & 2u) ? box_muller(n.z, n.w) : box_muller(n.x, n.y);
                    if ((m >> (2 * pr)) & 1u) {
                        v[2 * pr] = fmaf(a.sigma, z.x, v[2 * pr]);
                        if ((in_c >> (2 * pr)) & 1u) zz = fmaf(z.x, z.x, zz);
                    }
                    if ((m >> (2 * pr + 1)) & 1u) {
                        v[2 * pr + 1] = fmaf(a.sigma, z.y, v[2 * pr + 1]);
                        if ((in_c >> (2 * pr + 1)) & 1u) zz = fmaf(z.y, z.y, zz);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) out[t] = v[t];
}

__global__ void __launch_bounds__(kProbeThreads)
probe_kernel(const __grid_constant__ ProbeArgs a)
{
    extern __shared__ float smp[];
    const int h = a.h, k_in = a.k, d_out = a.d_out, np = a.n_probe;
    float* wt = smp;                          // [kKT][h]       W1 tile, transposed
    float* xt = wt + kKT * h;                 // [kKT][kMaxProbe] probe tile, transposed
    float* hs = xt + kKT * kMaxProbe;         // [kMaxProbe][h] hidden activations
    float* w2 = hs + kMaxProbe * h;           // [d_out][h] + b2 [d_out] (+ padding)
    float* red = w2 + d_out * h + 16;         // [kProbeThreads] reductions
    __shared__ int32_t s_kind, s_p1, s_p2;
    __shared__ uint32_t s_ent;

    const int r = blockIdx.x;
    if (threadIdx.x == 0) {
        s_kind = a.kind[r];
        s_p1 = a.par1[r];
        s_p2 = a.par2[r];
        s_ent = a.entity ? a.entity[r] : static_cast<uint32_t>(r);
    }
    __syncthreads();
    const int32_t kind = s_kind;
    const uint32_t ent = s_ent;
    const float* pa = a.parents + static_cast<int64_t>(s_p1) * a.c_pad;
    const float* pb = a.parents + static_cast<int64_t>(s_p2) * a.c_pad;
    const PhiloxKeys key = philox_keys(a.seed);
    uint32_t xo_hits = 0;
    float zz = 0.0f;

    // register block: 4 samples x 4 hidden units per (thread, block)
    const int n_sb = kMaxProbe / 4, n_hb = h / 4, n_blk = n_sb * n_hb;
    constexpr int kMaxBlk = (kMaxProbe / 4) * (kMaxHidden / 4) / kProbeThreads;  // blocks per thread, at most
    float acc[kMaxBlk][4][4];
#pragma unroll
    for (int b = 0; b < kMaxBlk; ++b)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[b][s][o] = 0.0f;

    const int units_per_row = kKT / 8;
    for (int k0 = 0; k0 < k_in; k0 += kKT) {
        const int kw = k_in - k0 < kKT ? k_in - k0 : kKT;  // multiple of 16
        __syncthreads();  // previous tile consumed
        for (int u = threadIdx.x; u < h * units_per_row; u += kProbeThreads) {
            const int o = u / units_per_row, k8 = (u - o * units_per_row) * 8;
            float g[8] = { 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f };
            if (k8 < kw)
                child_genes8(a, key, kind, ent, pa, pb, static_cast<int64_t>(o) * k_in + k0 + k8, g, xo_hits, zz);
#pragma unroll
            for (int t = 0; t < 8; ++t) wt[(k8 + t) * h + o] = g[t];
        }
        for (int e = threadIdx.x; e < kKT * kMaxProbe; e += kProbeThreads) {
            const int s = e / kKT, kk = e - s * kKT;
            xt[kk * kMaxProbe + s] = (s < np && kk < kw) ? a.probe[static_cast<int64_t>(s) * k_in + k0 + kk] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < kMaxBlk; ++b) {
            const int blk = threadIdx.x + b * kProbeThreads;
            if (blk < n_blk) {
                const int sb = blk / n_hb, hb = blk - sb * n_hb;
                for (int kk = 0; kk < kw; ++kk) {
                    const float4 xv = *reinterpret_cast<const float4*>(xt + kk * kMaxProbe + 4 * sb);
                    const float4 wv = *reinterpret_cast<const float4*>(wt + kk * h + 4 * hb);
                    const float xs[4] = { xv.x, xv.y, xv.z, xv.w }, ws[4] = { wv.x, wv.y, wv.z, wv.w };
#pragma unroll
                    for (int s = 0; s < 4; ++s)
#pragma unroll
                        for (int o = 0; o < 4; ++o) acc[b][s][o] = fmaf(xs[s], ws[o], acc[b][s][o]);
                }
            }
        }
    }
    __syncthreads();
    // b1 (genes k h .. k h + h - 1), then H = ReLU(acc + b1)
    const int64_t g_b1 = static_cast<int64_t>(k_in) * h;
    for (int u = threadIdx.x; u < h / 8; u += kProbeThreads) {
        float g[8];
        child_genes8(a, key, kind, ent, pa, pb, g_b1 + 8 * u, g, xo_hits, zz);
#pragma unroll
        for (int t = 0; t < 8; ++t) wt[8 * u + t] = g[t];  // b1 into the (free) tile buffer
    }
    // W2 and b2 (genes g_b1 + h .. c - 1): d_out h + d_out genes, in units of 8
    const int64_t g_w2 = g_b1 + h;
    const int n_tail = (d_out * h + d_out + 7) / 8;
    for (int u = threadIdx.x; u < n_tail; u += kProbeThreads) {
        float g[8];
        child_genes8(a, key, kind, ent, pa, pb, g_w2 + 8 * u, g, xo_hits, zz);
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (8 * u + t < d_out * h + d_out) w2[8 * u + t] = g[t];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < kMaxBlk; ++b) {
        const int blk = threadIdx.x + b * kProbeThreads;
        if (blk < n_blk) {
            const int sb = blk / n_hb, hb = blk - sb * n_hb;
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int oo = 4 * hb + o;
                    hs[(4 * sb + s) * h + oo] = fmaxf(acc[b][s][o] + wt[oo], 0.0f);
                }
        }
    }
    __syncthreads();
    float* row = a.desc + static_cast<int64_t>(r) * a.width;
    for (int e = threadIdx.x; e < np * d_out; e += kProbeThreads) {
        const int s = e / d_out, cl = e - s * d_out;
        float z = w2[d_out * h + cl];  // b2
        const float* wr = w2 + static_cast<int64_t>(cl) * h;
        const float* hr = hs + s * h;
        for (int o = 0; o < h; ++o) z = fmaf(wr[o], hr[o], z);
        row[5 + e] = z;
    }
    // crossover fraction and mutation step length over all c genes
    red[threadIdx.x] = static_cast<float>(xo_hits);
    __syncthreads();
    for (int w = kProbeThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const float hits = red[0];
    __syncthreads();
    red[threadIdx.x] = zz;
    __syncthreads();
    for (int w = kProbeThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        row[0] = a.f_adj[s_p1];
        row[1] = a.f_adj[s_p2];
        row[2] = a.f_inh[r];
        row[3] = kind == 1 ? (a.xo_op == 0 ? hits / static_cast<float>(a.c) : 0.5f) : 0.0f;
        row[4] = kind == 2 ? a.sigma * sqrtf(red[0]) : 0.0f;
    }
}

}  // namespace

bool probe_supported(int32_t k, int32_t h, int32_t d_out, int32_t n_probe, int32_t precision)
{
    if (precision >= 1) return probe_tc_supported(k, h, d_out, n_probe);
    return k % 16 == 0 && h % 16 == 0 && h >= 16 && h <= kMaxHidden && d_out >= 1 && d_out <= 16 && n_probe >= 1 &&
           n_probe <= kMaxProbe;
}

cudaError_t launch_descriptors(const ProbeArgs& a, int32_t n_recipes, cudaStream_t stream)
{
    if (n_recipes <= 0) return cudaSuccess;
    if (a.precision >= 1) return launch_descriptors_tc(a, n_recipes, stream);
    const size_t smem = sizeof(float) * (static_cast<size_t>(kKT) * a.h + kKT * kMaxProbe + kMaxProbe * a.h +
                                         static_cast<size_t>(a.d_out) * a.h + 16 + kProbeThreads);
    cudaError_t err = cudaFuncSetAttribute(probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    probe_kernel<<<n_recipes, kProbeThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace leea
