// leea_small_gen.cu -- one whole generation of Algorithm 1 (ranking and
// selection, Section 3.1; crossover and mutation, Section 3.2; the fitness of
// Eq. 1 with inheritance, Section 3.3) in a single launch, for populations so
// small that the usual chain of kernels spends its time in launch and
// dependency latency rather than in moving bytes (P = 32 nets of 784-32-10 on
// 16 samples are 3 MB).
//
// Grid: one CTA per (child i, slice q of kSlice = 8 hidden units), no waiting
// between CTAs.  Each CTA
//   1. ranks the whole previous population itself (a bitonic sort of the
//      64-bit rank keys in shared memory) and selects child i with the
//      selection kernels' code (select_ops.cuh), so that no CTA depends on
//      another's selection;
//   2. breeds the genes its slice owns -- W1 rows 8q .. 8q+7, b1[8q .. 8q+7],
//      the column block 8q .. 8q+7 of every W2 row and (slice 0) b2 -- with
//      the breeding kernel's per-unit code (breed_ops.cuh), writes them to
//      the new population and keeps the slice's W1 rows and b1 in shared
//      memory (8-gene units never straddle slices: 8 rows of d_0 genes are
//      d_0 units, and h % 8 == 0 aligns b1, W2 and b2);
//   3. forms the slice's layer 1 for the whole batch on the CUDA cores and
//      writes ReLU(.) to a scratch buffer;
//   4. counts itself in with an atomic add after a memory fence; the last of
//      child i's CTAs to arrive (the others simply exit) reads every slice's
//      activations and the child's W2 and b2 back through L2 and forms layer
//      2, the softmax cross-entropy (Eq. 1), the batch sum and the
//      inheritance blend, then zeroes the counter for the next launch.
// Arithmetic order: layer 1 is one FMA chain per (hidden unit, sample) over
// the inputs in ascending order, layer 2 one chain per (output, sample) over
// the hidden units in ascending order, and the loss and batch reduction are
// those of eval_simt_kernel, so the fitness is bit-identical to the CUDA-core
// evaluation's and the children bit-identical to breed_kernel's.
#include "breed_ops.cuh"
#include "leea_internal.h"
#include "philox.cuh"
#include "select_ops.cuh"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kSmallThreads = 512;
constexpr int kSlice = 8;  // hidden units per CTA
constexpr int kSmallMaxPop = 1024;
constexpr int kSmallMaxBatch = 128;
constexpr int kSmallMaxIn = 2048;
constexpr int kSmallMaxHidden = 256;
constexpr int kSmallMaxOut = 32;
constexpr size_t kSmallMaxSmem = 200 * 1024;

int pow2_at_least(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Floats of the region shared by the two phases: the batch and the slice's
// W1 rows (steps 1-3), then the last arriver's activations, W2, b2, logits
// and reduction buffers (step 4).  A multiple of 4 floats.
int64_t small_region_floats(int32_t d_in, int32_t h, int32_t d_out, int32_t batch)
{
    const int64_t r1 = static_cast<int64_t>(batch) * d_in + static_cast<int64_t>(kSlice) * (d_in + 4) + kSlice;
    const int64_t r2 = static_cast<int64_t>(batch) * (h + 1) + static_cast<int64_t>(d_out) * h + d_out +
                       static_cast<int64_t>(d_out) * batch + 2 * kSmallMaxBatch + 32;
    const int64_t r = r1 > r2 ? r1 : r2;
    return (r + 3) & ~int64_t(3);
}

// Batch tile of eval_simt_kernel for this batch (16 x its TN): the reduction
// over samples below follows the same tiles.
__device__ __forceinline__ int simt_batch_tile(int batch)
{
    return 16 * (batch <= 32 ? 2 : batch <= 64 ? 4 : 8);
}

__global__ void __launch_bounds__(kSmallThreads, 1) small_gen_kernel(const __grid_constant__ SmallGenArgs a)
{
    extern __shared__ float4 smem_small[];
    __shared__ ChildSelection sel_s;
    __shared__ int last_s;
    float* R = reinterpret_cast<float*>(smem_small);
    uint64_t* keys = reinterpret_cast<uint64_t*>(R + a.region_floats);
    int32_t* ord = reinterpret_cast<int32_t*>(keys + a.n_pow2);
    const int K = a.d_in, H = a.h, D = a.d_out, Bt = a.batch;
    const int i = static_cast<int>(blockIdx.x) / a.n_slices;
    const int q = static_cast<int>(blockIdx.x) - i * a.n_slices;
    const int tid = threadIdx.x;
    float* xs = R;                       // [Bt][K]: the batch as k / x_div
    float* w1s = xs + Bt * K;            // [kSlice][K + 4]: the slice's W1 rows
    float* b1s = w1s + kSlice * (K + 4);  // [kSlice]

    ptx::grid_dep_launch();
    ptx::grid_dep_wait();  // the previous generation's fitness and population

    // The batch, as the FP32 values k / x_div of its 8-bit levels (four per word).
    {
        const uint32_t* x4 = reinterpret_cast<const uint32_t*>(a.x);
        float4* xs4 = reinterpret_cast<float4*>(xs);
        const int n4 = Bt * K / 4;
        for (int t = tid; t < n4; t += kSmallThreads) {
            const uint32_t v = x4[t];
            xs4[t] = make_float4(static_cast<float>(v & 0xFFu) / a.x_div,
                                 static_cast<float>((v >> 8) & 0xFFu) / a.x_div,
                                 static_cast<float>((v >> 16) & 0xFFu) / a.x_div,
                                 static_cast<float>(v >> 24) / a.x_div);
        }
    }

    // 1. Ranking of the previous population and child i's selection.
    if (a.breed) {
        const int P = a.pop, n2 = a.n_pow2;
        for (int t = tid; t < n2; t += kSmallThreads) keys[t] = t < P ? rank_key(a.f_adj_in[t], t) : ~0ull;
        __syncthreads();
        for (int size = 2; size <= n2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = tid; t < (n2 >> 1); t += kSmallThreads) {
                    const int lo = 2 * stride * (t / stride) + (t % stride);
                    const int hi = lo + stride;
                    const bool ascending = (lo & size) == 0;
                    const uint64_t x = keys[lo], y = keys[hi];
                    if ((x > y) == ascending) {
                        keys[lo] = y;
                        keys[hi] = x;
                    }
                }
                __syncthreads();
            }
        }
        for (int r = tid; r < P; r += kSmallThreads) {
            const int32_t idx = static_cast<int32_t>(keys[r] & 0xFFFFFFFFu);
            ord[r] = idx;
            if (blockIdx.x == 0) a.order[r] = idx;
        }
        __syncthreads();
        if (tid == 0) {
            const ChildSelection c = select_child_of(a.sel, a.f_adj_in, ord, i);
            sel_s = c;
            if (q == 0) store_child_selection(a.sel, c, i, a.par1, a.par2, a.kind, a.f_inh);
        }
    }
    __syncthreads();

    // 2. The slice's genes: bred (children) or read (the first evaluation).
    {
        const int b2_units = static_cast<int>((a.c - a.b2_off + 7) / 8);
        const int n_units = a.breed ? K + 1 + D + (q == 0 ? b2_units : 0) : K + 1;
        const ChildSelection c = sel_s;
        const uint32_t gen = a.br.gen, ent = static_cast<uint32_t>(i);
        const PhiloxKeys key = philox_keys(a.br.seed);
        float* child = a.popv + static_cast<int64_t>(i) * a.c_pad;
        for (int t = tid; t < n_units; t += kSmallThreads) {
            int64_t g0;
            if (t < K) g0 = static_cast<int64_t>(q) * kSlice * K + 8 * t;  // W1 rows 8q .. 8q+7
            else if (t == K) g0 = a.b1_off + kSlice * q;
            else if (t < K + 1 + D) g0 = a.w2_off + static_cast<int64_t>(t - K - 1) * H + kSlice * q;
            else g0 = a.b2_off + 8 * (t - K - 1 - D);
            float4 v[2];
            if (a.breed) {
                const float4* p1 = reinterpret_cast<const float4*>(a.parents + static_cast<int64_t>(c.p1) * a.c_pad + g0);
                v[0] = p1[0];
                v[1] = p1[1];
                const uint32_t u = static_cast<uint32_t>(g0 >> 3);
                if (c.kind == kKindMut) {
                    const uint32_t hit = mask8(philox_keyed(make_uint4(u, ent, gen, kTagMutMask), key), a.br.thr_mut);
                    mutate8_direct(c.sigma, gen, key, ent, u, hit, v);
                } else if (c.kind == kKindCross) {
                    const float4* p2 =
                        reinterpret_cast<const float4*>(a.parents + static_cast<int64_t>(c.p2) * a.c_pad + g0);
                    const float4 b0 = p2[0], b1 = p2[1];
                    if (a.br.xo_op == 0) {
                        const uint32_t msk = mask8(philox_keyed(make_uint4(u, ent, gen, kTagXo), key), a.br.thr_xo);
                        v[0] = select4(msk, v[0], b0);
                        v[1] = select4(msk >> 4, v[1], b1);
                    } else {
                        v[0] = mean4(v[0], b0);
                        v[1] = mean4(v[1], b1);
                    }
                }
                if (g0 + 8 > a.c) {  // the last unit of b2 holds the padding
                    v[0] = clear_padding(v[0], g0, a.c);
                    v[1] = clear_padding(v[1], g0 + 4, a.c);
                }
                reinterpret_cast<float4*>(child + g0)[0] = v[0];
                reinterpret_cast<float4*>(child + g0)[1] = v[1];
            } else {
                v[0] = reinterpret_cast<const float4*>(child + g0)[0];
                v[1] = reinterpret_cast<const float4*>(child + g0)[1];
            }
            if (t < K) {
                const float e[8] = { v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w };
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const int l = 8 * t + s;  // gene of the slice's rows: row l / K, input l % K
                    const int r = l / K;
                    w1s[r * (K + 4) + (l - r * K)] = e[s];
                }
            } else if (t == K) {
                b1s[0] = v[0].x; b1s[1] = v[0].y; b1s[2] = v[0].z; b1s[3] = v[0].w;
                b1s[4] = v[1].x; b1s[5] = v[1].y; b1s[6] = v[1].z; b1s[7] = v[1].w;
            }
        }
    }
    __syncthreads();

    // 3. Layer 1 of the slice: hidden unit jj, sample n; inputs in ascending order.
    {
        float* hid = a.hid + static_cast<int64_t>(i) * Bt * H;
        for (int ch = tid; ch < kSlice * Bt; ch += kSmallThreads) {
            const int jj = ch & (kSlice - 1), n = ch / kSlice;
            const float4* w = reinterpret_cast<const float4*>(w1s + jj * (K + 4));
            const float4* xv = reinterpret_cast<const float4*>(xs + n * K);
            float acc = 0.0f;
#pragma unroll 4
            for (int k4 = 0; k4 < K / 4; ++k4) {
                const float4 wv = w[k4], xx = xv[k4];
                acc = fmaf(wv.x, xx.x, acc);
                acc = fmaf(wv.y, xx.y, acc);
                acc = fmaf(wv.z, xx.z, acc);
                acc = fmaf(wv.w, xx.w, acc);
            }
            hid[n * H + kSlice * q + jj] = fmaxf(acc + b1s[jj], 0.0f);
        }
    }

    // 4. Arrival: the last of child i's CTAs finishes the evaluation.
    __threadfence();
    __syncthreads();
    if (tid == 0) last_s = atomicAdd(a.count + i, 1u) == static_cast<uint32_t>(a.n_slices - 1) ? 1 : 0;
    __syncthreads();
    if (!last_s) return;
    __threadfence();

    const int HS = H + 1;                 // padded rows: chains of consecutive samples hit distinct banks
    float* Hs = R;                        // [Bt][H + 1]
    float* W2s = Hs + Bt * HS;            // [D][H]
    float* b2s = W2s + D * H;             // [D]
    float* Ls = b2s + D;                  // [D][Bt]
    float* lossv = Ls + D * Bt;           // [kSmallMaxBatch]
    int32_t* corv = reinterpret_cast<int32_t*>(lossv + kSmallMaxBatch);  // [kSmallMaxBatch]
    float* warp_sums = reinterpret_cast<float*>(corv + kSmallMaxBatch);  // [32]
    {
        const float* hid = a.hid + static_cast<int64_t>(i) * Bt * H;
        for (int t = tid; t < Bt * H; t += kSmallThreads) {
            const int n = t / H;
            Hs[n * HS + (t - n * H)] = __ldcg(hid + t);
        }
        const float* gi = a.popv + static_cast<int64_t>(i) * a.c_pad;
        for (int t = tid; t < D * H; t += kSmallThreads) W2s[t] = __ldcg(gi + a.w2_off + t);
        for (int t = tid; t < D; t += kSmallThreads) b2s[t] = __ldcg(gi + a.b2_off + t);
    }
    __syncthreads();
    for (int ch = tid; ch < D * Bt; ch += kSmallThreads) {
        const int o = ch / Bt, n = ch - o * Bt;
        const float* w = W2s + o * H;
        const float* hv = Hs + n * HS;
        float s = 0.0f;
        for (int r = 0; r < H; ++r) s = fmaf(w[r], hv[r], s);
        Ls[ch] = s;
    }
    __syncthreads();

    // Per-sample softmax cross-entropy and argmax, then the fixed-order batch
    // sum: per tile of BN samples a warp xor-tree over each 32 samples, the
    // warp sums added in order, the tile sums added in order.
    const int BN = simt_batch_tile(Bt);
    float total = 0.0f;  // meaningful in thread 0 only
    int32_t n_correct = 0;
    for (int b0 = 0; b0 < Bt; b0 += BN) {
        if (tid < BN) {
            const int gn = b0 + tid;
            float loss = 0.0f;
            int32_t ok = 0;
            if (gn < Bt) {
                float zmax = Ls[gn] + b2s[0];
                int arg = 0;
                for (int o = 1; o < D; ++o) {
                    const float z = Ls[o * Bt + gn] + b2s[o];
                    if (z > zmax) { zmax = z; arg = o; }
                }
                float s = 0.0f;
                for (int o = 0; o < D; ++o) s += expf(Ls[o * Bt + gn] + b2s[o] - zmax);
                const int32_t lbl = a.y[gn];
                if (lbl >= 0 && lbl < D) {
                    loss = logf(s) + zmax - (Ls[lbl * Bt + gn] + b2s[lbl]);
                    ok = (arg == lbl) ? 1 : 0;
                } else {
                    loss = __int_as_float(0x7FC00000);  // NaN: label out of range
                }
            }
            lossv[tid] = loss;
            corv[tid] = ok;
        }
        __syncthreads();
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
                corv[tid] = cv;
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
        a.f_raw[i] = f;
        a.f_adj[i] = a.breed ? (1.0f - a.alpha) * sel_s.f_inh + a.alpha * f : f;
        if (a.correct) a.correct[i] = n_correct;
        a.count[i] = 0u;  // for the next launch
    }
}

}  // namespace

size_t small_gen_smem_bytes(int32_t d_in, int32_t h, int32_t d_out, int32_t batch, int32_t pop)
{
    return sizeof(float) * static_cast<size_t>(small_region_floats(d_in, h, d_out, batch)) +
           sizeof(uint64_t) * static_cast<size_t>(pow2_at_least(pop)) + sizeof(int32_t) * static_cast<size_t>(pop);
}

bool small_gen_supported(const NetLayout& net, int32_t pop, int32_t batch)
{
    if (net.n_layers != 2) return false;
    const int32_t d_in = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    if (pop < 1 || pop > kSmallMaxPop || batch < 1 || batch > kSmallMaxBatch) return false;
    if (d_in % 4 != 0 || d_in > kSmallMaxIn || h % kSlice != 0 || h > kSmallMaxHidden || d_out < 1 ||
        d_out > kSmallMaxOut)
        return false;
    return small_gen_smem_bytes(d_in, h, d_out, batch, pop) <= kSmallMaxSmem;
}

int32_t small_gen_ctas(const NetLayout& net, int32_t pop)
{
    return pop * (net.dims[1] / kSlice);
}

cudaError_t launch_small_gen(SmallGenArgs a, cudaStream_t stream)
{
    a.n_slices = a.h / kSlice;
    a.n_pow2 = pow2_at_least(a.pop);
    a.region_floats = small_region_floats(a.d_in, a.h, a.d_out, a.batch);
    const size_t smem = small_gen_smem_bytes(a.d_in, a.h, a.d_out, a.batch, a.pop);
    cudaError_t err =
        cudaFuncSetAttribute(small_gen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    return launch_pdl(small_gen_kernel, dim3(a.pop * a.n_slices), dim3(kSmallThreads), smem, stream, a);
}

}  // namespace leea
