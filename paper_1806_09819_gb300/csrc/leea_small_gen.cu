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
//      64-bit rank keys: in one warp's registers up to 32 keys, else in
//      shared memory) and selects child i with the
//      selection kernels' code (select_ops.cuh), so that no CTA depends on
//      another's selection;
//   2. breeds the genes its slice owns -- W1 rows 8q .. 8q+7, b1[8q .. 8q+7],
//      the column block 8q .. 8q+7 of every W2 row and (slice 0) b2 -- with
//      the breeding kernel's per-unit code (breed_ops.cuh), writes them to
//      the new population and keeps the slice's W1 rows and b1 in shared
//      memory (8-gene units never straddle slices: 8 rows of d_0 genes are
//      d_0 units, and h % 8 == 0 aligns b1, W2 and b2);
//   3. forms the slice's layer 1 for the whole batch on the CUDA cores (4 x 4
//      register blocks over pieces of the inputs), and from it the slice's share of
//      layer 2 (the partial logits of its 8 hidden units), written to a
//      scratch buffer;
//   4. counts itself in with an atomic add after a memory fence; the last of
//      child i's CTAs to arrive (the others simply exit) adds the slices'
//      partial logits and b2, and forms the softmax cross-entropy (Eq. 1),
//      the batch sum and the inheritance blend, then zeroes the counter for
//      the next launch.
// Arithmetic order (fixed, so identical individuals get identical bits):
// layer 1 sums w k (k the exact 8-bit level) over each of up to 16 pieces of
// the inputs in an FMA chain in ascending order, adds the pieces in order and
// divides by x_div; layer 2 is one FMA chain per slice over its hidden units in
// ascending order, the slices added in order, then b2; the loss (softmax
// cross-entropy with the maximum subtracted, exponentials added in class
// order) and the batch reduction are eval_simt_kernel's.  The fitness is
// thus within FP32 rounding of the CUDA-core evaluation's, and the children
// are bit-identical to breed_kernel's.
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

// Layer 1 is computed in 4 x 4 register blocks (4 hidden units x 4 samples)
// over `pieces` consecutive pieces of the inputs, enough threads for the CTA.
constexpr int kBlk = 4;
constexpr int kMaxPieces = 16;
__host__ __device__ inline int layer1_pieces(int batch)
{
    const int blocks = (kSlice / kBlk) * ((batch + kBlk - 1) / kBlk);
    const int p = kSmallThreads / blocks;
    return p < 1 ? 1 : (p > kMaxPieces ? kMaxPieces : p);
}

// Floats of the region shared by the two phases: the batch, the slice's W1
// rows, b1, W2 columns and activations (steps 1-3), then the last arriver's
// logits, b2 and reduction buffers (step 4).  A multiple of 4 floats.
int64_t small_region_floats(int32_t d_in, int32_t h, int32_t d_out, int32_t batch)
{
    (void)h;
    const int64_t r1 = static_cast<int64_t>(batch) * (d_in + 4) + static_cast<int64_t>(kSlice) * (d_in + 4) + kSlice +
                       static_cast<int64_t>(kSlice) * d_out +
                       static_cast<int64_t>(1 + layer1_pieces(batch)) * kSlice * batch;
    const int64_t r2 = 2 * static_cast<int64_t>(d_out) * batch + 2 * static_cast<int64_t>(batch) +
                       2 * kSmallMaxBatch + 32;
    const int64_t r = r1 > r2 ? r1 : r2;
    return (r + 3) & ~int64_t(3);
}

// Batch tile of eval_simt_kernel for this batch (16 x its TN): the reduction
// over samples below follows the same tiles.
__device__ __forceinline__ int simt_batch_tile(int batch)
{
    return 16 * (batch <= 32 ? 2 : batch <= 64 ? 4 : 8);
}

// Bitonic sort of one key per lane (n2 <= 32 keys, padding keys ~0 sort
// last): afterwards lane r holds the r-th smallest key.
__device__ __forceinline__ uint64_t warp_sort_keys(uint64_t key, int lane, int n2)
{
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t other = __shfl_xor_sync(0xFFFFFFFFu, key, stride);
            const bool ascending = (lane & size) == 0;
            const bool lower = (lane & stride) == 0;
            const uint64_t lo = key < other ? key : other, hi = key < other ? other : key;
            key = (lower == ascending) ? lo : hi;
        }
    }
    return key;
}

constexpr int kSmallJobs = 4 * 32;  // Box-Muller pairs of a warp's 32 units
constexpr int kXWords = 8;  // words of the batch a thread holds in registers while it selects and breeds

// A read-only load issued where it stands in the program (the memory clobber
// keeps the compiler from sinking it to its first use), so that its latency
// overlaps the work in between.
__device__ __forceinline__ uint32_t ld_u32_now(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Four 8-bit levels k as FP32 (exact).
__device__ __forceinline__ float4 levels_to_float4(uint32_t v)
{
    return make_float4(static_cast<float>(v & 0xFFu), static_cast<float>((v >> 8) & 0xFFu),
                       static_cast<float>((v >> 16) & 0xFFu), static_cast<float>(v >> 24));
}

__global__ void __launch_bounds__(kSmallThreads, 1) small_gen_kernel(const __grid_constant__ SmallGenArgs a)
{
    extern __shared__ float4 smem_small[];
    __shared__ ChildSelection sel_s;
    __shared__ int last_s;
    __shared__ float2 job_z[kSmallThreads / 32 * kSmallJobs];     // per warp: normals of its job list
    __shared__ uint8_t job_code[kSmallThreads / 32 * kSmallJobs];  // per warp: owner lane << 2 | pair slot
    float* R = reinterpret_cast<float*>(smem_small);
    uint64_t* keys = reinterpret_cast<uint64_t*>(R + a.region_floats);
    int32_t* ord = reinterpret_cast<int32_t*>(keys + a.n_pow2);
    float* fs = reinterpret_cast<float*>(ord + a.pop);  // the previous fitness, for the selection
    const int K = a.d_in, H = a.h, D = a.d_out, Bt = a.batch;
    const int i = static_cast<int>(blockIdx.x) / a.n_slices;
    const int q = static_cast<int>(blockIdx.x) - i * a.n_slices;
    const int tid = threadIdx.x;
    float* xs = R;                       // [Bt][K + 4]: the batch's levels k (rows padded: distinct banks)
    float* w1s = xs + Bt * (K + 4);      // [kSlice][K + 4]: the slice's W1 rows
    float* b1s = w1s + kSlice * (K + 4);  // [kSlice]
    float* w2s = b1s + kSlice;            // [D][kSlice]: the slice's columns of W2
    float* hs = w2s + D * kSlice;         // [Bt][kSlice]: the slice's activations
    float* qs = hs + Bt * kSlice;         // [pieces][Bt * kSlice]: layer 1's sums over the pieces

    ptx::grid_dep_launch();
    ptx::grid_dep_wait();  // the previous generation's fitness and population

    // The previous fitness, then the batch's 8-bit levels (four per word):
    // a small batch is held in registers until layer 1 needs it, so that its
    // loads overlap the selection and the breed.
    const int P = a.pop, n2 = a.n_pow2;
    float f_mine = 0.0f;
    if (a.breed && tid < P) f_mine = __ldcg(a.f_adj_in + tid);
    const uint32_t* x4 = reinterpret_cast<const uint32_t*>(a.x);
    const int n4 = Bt * K / 4;
    const bool x_in_regs = n4 <= kXWords * kSmallThreads;
    uint32_t xw[kXWords];
#pragma unroll
    for (int j = 0; j < kXWords; ++j) {
        const int t = tid + j * kSmallThreads;
        xw[j] = (x_in_regs && t < n4) ? ld_u32_now(x4 + t) : 0u;
    }

    // 1. Ranking of the previous population and child i's selection.
    if (a.breed) {
        if (n2 <= 32) {  // one warp sorts the keys in registers
            if (tid < 32) {
                if (tid < P) fs[tid] = f_mine;
                const uint64_t k = warp_sort_keys(tid < P ? rank_key(f_mine, tid) : ~0ull, tid, n2);
                if (tid < P) {
                    const int32_t idx = static_cast<int32_t>(k & 0xFFFFFFFFu);
                    ord[tid] = idx;
                    if (blockIdx.x == 0) a.order[tid] = idx;
                }
            }
            __syncthreads();
        } else {
        for (int t = tid; t < n2; t += kSmallThreads) {
            const float f = t < P ? (t < kSmallThreads ? f_mine : __ldcg(a.f_adj_in + t)) : 0.0f;
            if (t < P) fs[t] = f;
            keys[t] = t < P ? rank_key(f, t) : ~0ull;
        }
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
        }
        if (tid == 0) {
            const ChildSelection c = select_child_of(a.sel, fs, ord, i);
            sel_s = c;
            if (q == 0) store_child_selection(a.sel, c, i, a.par1, a.par2, a.kind, a.f_inh);
        }
    }
    __syncthreads();

    // 2. The slice's genes: bred (children) or read (the first evaluation),
    // two units per thread at a time so that their loads are in flight together.
    {
        const int b2_units = static_cast<int>((a.c - a.b2_off + 7) / 8);
        const int n_units = K + 1 + D + ((a.breed && q == 0) ? b2_units : 0);
        const ChildSelection c = sel_s;
        const uint32_t gen = a.br.gen, ent = static_cast<uint32_t>(i);
        const PhiloxKeys key = philox_keys(a.br.seed);
        float* child = a.popv + static_cast<int64_t>(i) * a.c_pad;
        const float* par1 = a.parents + static_cast<int64_t>(c.p1) * a.c_pad;
        const float* par2 = a.parents + static_cast<int64_t>(c.p2) * a.c_pad;
        auto first_gene = [&](int t) -> int64_t {
            if (t < K) return static_cast<int64_t>(q) * kSlice * K + 8 * t;  // W1 rows 8q .. 8q+7
            if (t == K) return a.b1_off + kSlice * q;
            if (t < K + 1 + D) return a.w2_off + static_cast<int64_t>(t - K - 1) * H + kSlice * q;
            return a.b2_off + 8 * (t - K - 1 - D);
        };
        // Parent genes of a unit (a.breed), or the individual's own (the first evaluation).
        auto load = [&](int64_t g0, float4 (&v)[2], float4 (&w)[2]) {
            const float4* src = reinterpret_cast<const float4*>((a.breed ? par1 : child) + g0);
            v[0] = __ldcg(src);
            v[1] = __ldcg(src + 1);
            if (a.breed && c.kind == kKindCross) {
                const float4* src2 = reinterpret_cast<const float4*>(par2 + g0);
                w[0] = __ldcg(src2);
                w[1] = __ldcg(src2 + 1);
            }
        };
        // Called by every lane of a warp that holds a unit (ok: this lane's
        // unit exists): the mutation normals go through the warp's job list.
        auto finish = [&](int t, bool ok, int64_t g0, float4 (&v)[2], const float4 (&w)[2]) {
            if (a.breed) {
                const uint32_t u = static_cast<uint32_t>(g0 >> 3);
                if (c.kind == kKindMut) {  // the same for the whole CTA
                    const int lane = tid & 31, t0 = t - lane;
                    const uint32_t hit =
                        ok ? mask8(philox_keyed(make_uint4(u, ent, gen, kTagMutMask), key), a.br.thr_mut) : 0u;
                    mutate8(c.sigma, gen, key, ent, hit, v, lane, job_z + (tid >> 5) * kSmallJobs,
                            job_code + (tid >> 5) * kSmallJobs,
                            [&](uint32_t o) { return static_cast<uint32_t>(first_gene(t0 + static_cast<int>(o)) >> 3); });
                } else if (ok && c.kind == kKindCross) {
                    if (a.br.xo_op == 0) {
                        const uint32_t msk = mask8(philox_keyed(make_uint4(u, ent, gen, kTagXo), key), a.br.thr_xo);
                        v[0] = select4(msk, v[0], w[0]);
                        v[1] = select4(msk >> 4, v[1], w[1]);
                    } else {
                        v[0] = mean4(v[0], w[0]);
                        v[1] = mean4(v[1], w[1]);
                    }
                }
                if (g0 + 8 > a.c) {  // the last unit of b2 holds the padding
                    v[0] = clear_padding(v[0], g0, a.c);
                    v[1] = clear_padding(v[1], g0 + 4, a.c);
                }
                if (!ok) return;
                reinterpret_cast<float4*>(child + g0)[0] = v[0];
                reinterpret_cast<float4*>(child + g0)[1] = v[1];
            } else if (!ok) {
                return;
            }
            if (t < K) {  // genes 8t .. 8t+7 of the slice's rows: row l / K, input l % K
                const float e8[8] = { v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w };
                int r = (8 * t) / K, col = 8 * t - r * K;
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    w1s[r * (K + 4) + col] = e8[s];
                    if (++col == K) { col = 0; ++r; }
                }
            } else if (t <= K + D) {  // b1, or column block 8q .. 8q+7 of W2 row t - K - 1
                float* dst = t == K ? b1s : w2s + (t - K - 1) * kSlice;
                reinterpret_cast<float4*>(dst)[0] = v[0];
                reinterpret_cast<float4*>(dst)[1] = v[1];
            }
        };
        // The batch's levels as FP32, while the first units' parent loads are
        // in flight (word t holds inputs 4t .. 4t+3 of the row-major batch).
        auto convert_batch = [&]() {
            const int kw = K / 4;
            auto dst = [&](int t) {
                const int n = t / kw;
                return reinterpret_cast<float4*>(xs + n * (K + 4) + 4 * (t - n * kw));
            };
            if (x_in_regs) {
#pragma unroll
                for (int j = 0; j < kXWords; ++j) {
                    const int t = tid + j * kSmallThreads;
                    if (t < n4) *dst(t) = levels_to_float4(xw[j]);
                }
            } else {
                for (int t0 = tid; t0 < n4; t0 += 4 * kSmallThreads) {
                    uint32_t w4[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t = t0 + j * kSmallThreads;
                        w4[j] = t < n4 ? __ldg(x4 + t) : 0u;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int t = t0 + j * kSmallThreads;
                        if (t < n4) *dst(t) = levels_to_float4(w4[j]);
                    }
                }
            }
        };
        for (int base = 0; base < n_units; base += 2 * kSmallThreads) {
            const int tA = base + tid, tB = tA + kSmallThreads;
            const bool okA = tA < n_units, okB = tB < n_units;
            const int64_t gA = okA ? first_gene(tA) : 0, gB = okB ? first_gene(tB) : 0;
            float4 vA[2], wA[2], vB[2], wB[2];
            if (okA) load(gA, vA, wA);
            if (okB) load(gB, vB, wB);
            if (base == 0) convert_batch();
            const int wbase = base + (tid & ~31);  // the warp's first unit of this round
            if (wbase < n_units) finish(tA, okA, gA, vA, wA);
            if (wbase + kSmallThreads < n_units) finish(tB, okB, gB, vB, wB);
        }
    }
    __syncthreads();

    // 3. Layer 1 of the slice (hidden unit jj, sample n): the sum of w k (k the
    // exact 8-bit level, each product exact in the FMA) over each piece of the
    // inputs in ascending order, the pieces added in order, divided by x_div;
    // then bias and ReLU.  A thread holds a 4 x 4 block of sums (4 rows of W1,
    // 4 samples) for one piece: 8 vector loads per 64 FMAs.
    {
        const int n_pc = layer1_pieces(Bt);
        const int kp = ((K + 4 * n_pc - 1) / (4 * n_pc)) * 4;  // piece length, a multiple of 4
        const int n_nb = (Bt + kBlk - 1) / kBlk, n_blk = (kSlice / kBlk) * n_nb;
        const int n_ch = kSlice * Bt;
        for (int ct = tid; ct < n_pc * n_blk; ct += kSmallThreads) {
            const int z = ct / n_blk, blk = ct - z * n_blk;
            // rows j0 .. j0+3 of the slice; samples nb, nb + n_nb, nb + 2 n_nb, nb + 3 n_nb
            // (interleaved, so that a load's 8 threads of a phase hit distinct banks)
            const int j0 = kBlk * (blk % (kSlice / kBlk)), nb = blk / (kSlice / kBlk);
            const int k0 = z * kp, k1 = min(K, k0 + kp);
            const float* wr[kBlk];
            const float* xr[kBlk];
#pragma unroll
            for (int r = 0; r < kBlk; ++r) {
                wr[r] = w1s + (j0 + r) * (K + 4);
                xr[r] = xs + min(nb + r * n_nb, Bt - 1) * (K + 4);  // samples past the batch: computed, not kept
            }
            float acc[kBlk][kBlk];
#pragma unroll
            for (int r = 0; r < kBlk; ++r)
#pragma unroll
                for (int s = 0; s < kBlk; ++s) acc[r][s] = 0.0f;
            for (int k = k0; k < k1; k += 4) {
                float4 wv[kBlk], xv[kBlk];
#pragma unroll
                for (int r = 0; r < kBlk; ++r) {
                    wv[r] = *reinterpret_cast<const float4*>(wr[r] + k);
                    xv[r] = *reinterpret_cast<const float4*>(xr[r] + k);
                }
#pragma unroll
                for (int r = 0; r < kBlk; ++r)
#pragma unroll
                    for (int s = 0; s < kBlk; ++s) {
                        acc[r][s] = fmaf(wv[r].x, xv[s].x, acc[r][s]);
                        acc[r][s] = fmaf(wv[r].y, xv[s].y, acc[r][s]);
                        acc[r][s] = fmaf(wv[r].z, xv[s].z, acc[r][s]);
                        acc[r][s] = fmaf(wv[r].w, xv[s].w, acc[r][s]);
                    }
            }
#pragma unroll
            for (int s = 0; s < kBlk; ++s)
                if (nb + s * n_nb < Bt)
#pragma unroll
                    for (int r = 0; r < kBlk; ++r) qs[z * n_ch + (nb + s * n_nb) * kSlice + j0 + r] = acc[r][s];
        }
        __syncthreads();
        for (int ch = tid; ch < n_ch; ch += kSmallThreads) {
            float v = qs[ch];
#pragma unroll 4
            for (int z = 1; z < n_pc; ++z) v += qs[z * n_ch + ch];
            hs[ch] = fmaxf(v / a.x_div + b1s[ch & (kSlice - 1)], 0.0f);
        }
    }
    __syncthreads();
    // The slice's share of layer 2: partial logit o of sample n over hidden
    // units 8q .. 8q+7 in ascending order.
    {
        float* part = a.part + (static_cast<int64_t>(i) * a.n_slices + q) * Bt * D;  // [Bt][D]
        for (int ch = tid; ch < Bt * D; ch += kSmallThreads) {
            const int n = ch / D, o = ch - n * D;
            const float* wv = w2s + o * kSlice;
            const float* hv = hs + n * kSlice;
            float s = 0.0f;
#pragma unroll
            for (int r = 0; r < kSlice; ++r) s = fmaf(wv[r], hv[r], s);
            part[ch] = s;
        }
    }

    // 4. Arrival: the last of child i's CTAs finishes the evaluation.  The
    // barrier orders the CTA's partial logits before thread 0's fence, which
    // releases them with its count (and, in the last arriver, acquires the
    // other slices' before the barrier that follows).
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const bool last = atomicAdd(a.count + i, 1u) == static_cast<uint32_t>(a.n_slices - 1);
        if (last) __threadfence();
        last_s = last ? 1 : 0;
    }
    __syncthreads();
    if (!last_s) return;

    float* Ls = R;                        // [D][Bt]: the logits z
    float* Es = Ls + D * Bt;              // [D][Bt]: exp(z - max z)
    float* zm = Es + D * Bt;              // [Bt]: max z of the sample
    int32_t* am = reinterpret_cast<int32_t*>(zm + Bt);  // [Bt]: its argmax (lowest class on ties)
    float* lossv = reinterpret_cast<float*>(am + Bt);   // [kSmallMaxBatch]
    int32_t* corv = reinterpret_cast<int32_t*>(lossv + kSmallMaxBatch);  // [kSmallMaxBatch]
    float* warp_sums = reinterpret_cast<float*>(corv + kSmallMaxBatch);  // [32]
    {  // z = the slices' partial logits added in slice order, then b2
        const float* b2 = a.popv + static_cast<int64_t>(i) * a.c_pad + a.b2_off;
        const float* part = a.part + static_cast<int64_t>(i) * a.n_slices * Bt * D;
        const int64_t slice_stride = static_cast<int64_t>(Bt) * D;
        for (int ch = tid; ch < Bt * D; ch += kSmallThreads) {
            const int n = ch / D, o = ch - n * D;
            const float bias = __ldcg(b2 + o);
            float s = __ldcg(part + ch);
#pragma unroll 4
            for (int qq = 1; qq < a.n_slices; ++qq) s += __ldcg(part + qq * slice_stride + ch);
            Ls[o * Bt + n] = s + bias;
        }
    }
    __syncthreads();
    for (int n = tid; n < Bt; n += kSmallThreads) {
        float zmax = Ls[n];
        int arg = 0;
        for (int o = 1; o < D; ++o) {
            const float z = Ls[o * Bt + n];
            if (z > zmax) { zmax = z; arg = o; }
        }
        zm[n] = zmax;
        am[n] = arg;
    }
    __syncthreads();
    for (int ch = tid; ch < D * Bt; ch += kSmallThreads) Es[ch] = expf(Ls[ch] - zm[ch % Bt]);
    __syncthreads();

    // Per-sample softmax cross-entropy (Eq. 1): log sum exp(z - max z) + max z
    // - z[label], the exponentials summed over the classes in ascending order;
    // then the fixed-order batch sum: per tile of BN samples a warp xor-tree
    // over each 32 samples, the warp sums added in order, the tile sums added
    // in order.
    const int BN = simt_batch_tile(Bt);
    float total = 0.0f;  // meaningful in thread 0 only
    int32_t n_correct = 0;
    for (int b0 = 0; b0 < Bt; b0 += BN) {
        if (tid < BN) {
            const int gn = b0 + tid;
            float loss = 0.0f;
            int32_t ok = 0;
            if (gn < Bt) {
                float s = 0.0f;
                for (int o = 0; o < D; ++o) s += Es[o * Bt + gn];
                const int32_t lbl = a.y[gn];
                if (lbl >= 0 && lbl < D) {
                    loss = logf(s) + zm[gn] - Ls[lbl * Bt + gn];
                    ok = (am[gn] == lbl) ? 1 : 0;
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
           sizeof(uint64_t) * static_cast<size_t>(pow2_at_least(pop)) +
           (sizeof(int32_t) + sizeof(float)) * static_cast<size_t>(pop);
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
