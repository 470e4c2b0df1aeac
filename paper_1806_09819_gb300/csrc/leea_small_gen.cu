// leea_small_gen.cu -- one whole generation of Algorithm 1 (ranking and
// selection, Section 3.1; crossover and mutation, Section 3.2; the fitness of
// Eq. 1 with inheritance, Section 3.3) in a single launch, for populations so
// small that the usual chain of kernels spends its time in launch and
// dependency latency rather than in moving bytes (P = 32 nets of 784-32-10 on
// 16 samples are 3 MB).
//
// Grid: one CTA per (child i, slice q of kSlice = 8 hidden units); a child's
// slices form a thread-block cluster (up to 8 of them), no other CTA waits for
// another.  Each CTA
//   0. draws the random numbers of the genes its slice owns -- the crossover
//      or mutation masks and the mutation normals (through the warps' job
//      lists) -- which depend on the child's index and kind, not on its
//      parents, while the batch is copied to shared memory;
//   1. meanwhile ranks the whole previous population itself and selects child
//      i with the selection kernels' code (select_ops.cuh): up to 32
//      individuals the last warp counts, for each, the rank keys below its
//      own; beyond, the whole CTA sorts the keys in shared memory after the
//      draws;
//   2. breeds the slice's genes -- W1 rows 8q .. 8q+7, b1[8q .. 8q+7], the
//      column block 8q .. 8q+7 of every W2 row and (slice 0) b2 -- from the
//      parents' genes and the drawn numbers with the breeding kernel's
//      per-unit operators (breed_ops.cuh), writes them to the new population
//      and keeps the slice in shared memory (8-gene units never straddle
//      slices: 8 rows of d_0 genes are d_0 units, and h % 8 == 0 aligns b1,
//      W2 and b2);
//   3. forms the slice's layer 1 for the whole batch (m16n8k8 tensor-core
//      tiles, the warps splitting the inputs) and from it the slice's share
//      of layer 2, the partial logits of its 8 hidden units;
//   4. hands them to slice 0: in a cluster by writing them into slice 0's
//      shared memory before a cluster barrier, otherwise through L2 with an
//      arrival counter (the last slice to count itself in finishes and zeroes
//      the counter for the next launch).  The finishing CTA adds the partial
//      logits and b2 and forms the softmax cross-entropy (Eq. 1), the batch
//      sum and the inheritance blend.
// Arithmetic order (fixed, so identical individuals get identical bits):
// layer 1 accumulates the exact products k w_hi and k w_lo (k the 8-bit
// level, w_hi + w_lo the weight to 22 bits) in FP32 on the tensor cores over
// each warp's input group, adds the groups in order and divides by x_div;
// layer 2 is one FMA chain per slice over its hidden units in ascending
// order, the slices added in order, then b2; the loss (softmax cross-entropy
// with the maximum subtracted, exponentials added in class order) and the
// batch reduction are eval_simt_kernel's.  The fitness is thus within the
// evaluation tolerance of the CUDA-core evaluation's (as the 8-bit
// tensor-core evaluation is), and the children are bit-identical to
// breed_kernel's.  A single CTA's layer 1 is 16 samples x 8 units x d_0
// inputs: mma.sync tiles in registers serve it without the setup of the
// tcgen05 path (tensor memory, descriptors, barriers) that the large
// evaluations amortise.
#include "breed_ops.cuh"
#include "leea_internal.h"
#include "philox.cuh"
#include "select_ops.cuh"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kSmallThreads = 512;
constexpr int kUnitThreads = kSmallThreads - 32;  // warps 0-14 breed; warp 15 selects (populations up to 32)
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

// Layer 1 runs as m16n8k8 TF32 tensor-core tiles (16 samples x the slice's 8
// hidden units x 8 inputs); the warps split the inputs, and their partial
// tiles ([input groups][16 * tiles][8] floats) are added in order.
constexpr int kWarps = kSmallThreads / 32;
constexpr int kPartialFloats = kWarps * 16 * kSlice;  // the largest [groups][16 tiles][8] over batch <= 128

// Floats of the region shared by the two phases: the batch, the slice's W1
// rows, b1, W2 columns and activations (steps 1-3), then the last arriver's
// logits, b2 and reduction buffers (step 4).  A multiple of 4 floats.
int64_t small_region_floats(int32_t d_in, int32_t h, int32_t d_out, int32_t batch)
{
    (void)h;
    const int64_t r1 = static_cast<int64_t>(batch) * (d_in + 4) + static_cast<int64_t>(kSlice) * (d_in + 4) + kSlice +
                       static_cast<int64_t>(kSlice) * d_out + static_cast<int64_t>(kSlice) * batch + kPartialFloats +
                       static_cast<int64_t>(batch) * d_in / 4;
    const int64_t r2 = static_cast<int64_t>(d_out) * batch + 2 * kSmallMaxBatch + 32;
    const int64_t r = r1 > r2 ? r1 : r2;
    return (r + 3) & ~int64_t(3);
}

// Offset in floats of b2 (and the cluster's gather buffer) behind the region,
// the rank keys, the order and the fitness: a multiple of 4 (16 bytes).
__host__ __device__ inline int64_t small_tail_floats(int64_t region_floats, int n_pow2, int pop)
{
    return (region_floats + 2 * static_cast<int64_t>(n_pow2) + 2 * static_cast<int64_t>(pop) + 3) & ~int64_t(3);
}

// Batch tile of eval_simt_kernel for this batch (16 x its TN): the reduction
// over samples below follows the same tiles.
__device__ __forceinline__ int simt_batch_tile(int batch)
{
    return 16 * (batch <= 32 ? 2 : batch <= 64 ? 4 : 8);
}

constexpr int kSmallJobs = 4 * 32;  // Box-Muller pairs of a warp's 32 units

// 4-byte asynchronous copy global -> shared (completion per thread by cp.async groups).
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(ptx::smem_u32(dst)), "l"(src) : "memory");
}

// Thread-block cluster of one child's slices (cluster rank q = slice q).
__device__ __forceinline__ void cluster_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The address of this CTA's shared variable p in the shared memory of cluster CTA `rank`.
__device__ __forceinline__ uint32_t cluster_map(const void* p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(ptx::smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// FP32 -> TF32 (round to nearest, ties away), the bits of a TF32 operand.
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// d += a b for one m16n8k8 tile: A 16 x 8 (row-major fragment), B 8 x 8
// (column-major fragment), TF32 operands, FP32 accumulators.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                 "{%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four 8-bit levels k as FP32 (exact).
__device__ __forceinline__ float4 levels_to_float4(uint32_t v)
{
    return make_float4(static_cast<float>(v & 0xFFu), static_cast<float>((v >> 8) & 0xFFu),
                       static_cast<float>((v >> 16) & 0xFFu), static_cast<float>(v >> 24));
}

// CLUSTER: child i's slices form a thread-block cluster; each slice writes its
// partial logits into slice 0's shared memory and one cluster barrier hands
// them over.  Otherwise the partial logits go through L2 and the last slice to
// count itself in (atomic add) finishes.
template <bool CLUSTER>
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
    float* b2s = R + small_tail_floats(a.region_floats, a.n_pow2, a.pop);  // slice 0: b2 (padded to 8), 16-byte aligned
    float* gather = b2s + 8 * a.b2_units;               // CLUSTER, slice 0: [n_slices][Bt][D] partial logits
    const int K = a.d_in, H = a.h, D = a.d_out, Bt = a.batch;
    const int i = static_cast<int>(blockIdx.x) / a.n_slices;
    const int q = static_cast<int>(blockIdx.x) - i * a.n_slices;
    const int tid = threadIdx.x;
    float* xs = R;                       // [Bt][K + 4]: the batch's levels k (rows padded: distinct banks)
    float* w1s = xs + Bt * (K + 4);      // [kSlice][K + 4]: the slice's W1 rows
    float* b1s = w1s + kSlice * (K + 4);  // [kSlice]
    float* w2s = b1s + kSlice;            // [D][kSlice]: the slice's columns of W2
    float* hs = w2s + D * kSlice;         // [Bt][kSlice]: the slice's activations
    float* qs = hs + Bt * kSlice;         // layer 1's partial tiles of the input groups
    uint32_t* xraw = reinterpret_cast<uint32_t*>(qs + kPartialFloats);  // [Bt * K / 4]: the batch's levels as copied

    ptx::grid_dep_launch();
    if (CLUSTER) cluster_arrive_relaxed();  // every CTA of the cluster has started before any writes to slice 0
    ptx::grid_dep_wait();  // the previous generation's fitness and population

    // The batch's 8-bit levels are copied to shared memory four at a time
    // (cp.async) by the unit threads while the work below proceeds.  For
    // populations up to 32 the last warp ranks the previous population and
    // selects child i meanwhile (step 1); larger ones are ranked by the whole
    // CTA after the draws.
    const int P = a.pop, n2 = a.n_pow2;
    const bool sel_warp = a.breed && P <= 32;
    const int n4 = Bt * K / 4;  // 4-input groups of the batch
    if (tid < kUnitThreads) {
        if (a.xf) {  // FP32 inputs: 16-byte copies straight into the padded rows
            const int kw = K / 4;
            for (int t = tid; t < n4; t += kUnitThreads) {
                const int n = t / kw;
                ptx::cp_async16(xs + n * (K + 4) + 4 * (t - n * kw), a.xf + 4 * static_cast<int64_t>(t));
            }
        } else {
            const uint32_t* x4 = reinterpret_cast<const uint32_t*>(a.x);
            for (int t = tid; t < n4; t += kUnitThreads) cp_async4(xraw + t, x4 + t);
        }
        ptx::cp_async_commit();
    }

    // 1a. Ranking and selection by the last warp: the rank of individual l is
    // the number of rank keys below its own (the keys are distinct).
    if (sel_warp && tid >= kUnitThreads) {
        const int l = tid - kUnitThreads;
        SelStream sel_st(a.sel.seed, a.sel.gen, static_cast<uint32_t>(i));
        if (l == 0) sel_st.draw(0);  // child i's first SEL block, while the fitness loads are in flight
        const float f = l < P ? __ldcg(a.f_adj_in + l) : 0.0f;
        const uint64_t mine = l < P ? rank_key(f, l) : ~0ull;
        if (l < P) {
            fs[l] = f;
            keys[l] = mine;
        }
        __syncwarp();
        int r = 0;
        for (int m = 0; m < P; ++m) r += keys[m] < mine ? 1 : 0;
        if (l < P) {
            ord[r] = l;
            if (blockIdx.x == 0) a.order[r] = l;
        }
        __syncwarp();
        if (l == 0) {
            const ChildSelection c = select_child_of(a.sel, fs, ord, i, sel_st);
            sel_s = c;
            if (q == 0) store_child_selection(a.sel, c, i, a.par1, a.par2, a.kind, a.f_inh);
        }
    }

    // The slice's units (8 genes each) and, ahead of the selection, their
    // random numbers: the crossover and mutation masks and the mutation
    // normals depend on the child's index (its kind too), not on its parents.
    const int n_units = K + 1 + D + (q == 0 ? a.b2_units : 0);
    const int kind = i < a.sel.n_elite ? kKindElite : (i < a.sel.n_elite + a.sel.n_cross ? kKindCross : kKindMut);
    const uint32_t gen = a.br.gen, ent = static_cast<uint32_t>(i);
    const PhiloxKeys key = philox_keys(a.br.seed);
    const int lane = tid & 31;
    auto first_gene = [&](int t) -> int64_t {
        if (t < K) return static_cast<int64_t>(q) * kSlice * K + 8 * t;  // W1 rows 8q .. 8q+7
        if (t == K) return a.b1_off + kSlice * q;
        if (t < K + 1 + D) return a.w2_off + static_cast<int64_t>(t - K - 1) * H + kSlice * q;
        return a.b2_off + 8 * (t - K - 1 - D);
    };
    // The mask of unit t (mutation or crossover); for a mutation child also its
    // normals, through the warp's job list (every lane of the warp calls it).
    auto draw_unit = [&](int t, bool ok, uint32_t& msk, float2 (&z)[4]) {
        const uint32_t u = ok ? static_cast<uint32_t>(first_gene(t) >> 3) : 0u;
        if (kind == kKindMut) {
            msk = ok ? mask8(philox_keyed(make_uint4(u, ent, gen, kTagMutMask), key), a.br.thr_mut) : 0u;
            const int t0 = t - lane;
            normals8(gen, key, ent, msk, z, lane, job_z + (tid >> 5) * kSmallJobs, job_code + (tid >> 5) * kSmallJobs,
                     [&](uint32_t o) { return static_cast<uint32_t>(first_gene(t0 + static_cast<int>(o)) >> 3); });
        } else if (kind == kKindCross && a.br.xo_op == 0) {
            msk = ok ? mask8(philox_keyed(make_uint4(u, ent, gen, kTagXo), key), a.br.thr_xo) : 0u;
        }
    };
    // Unit round r of a thread: units t = r * 2 * kUnitThreads + tid (A) and
    // + kUnitThreads (B); the first round's numbers are drawn here.
    const bool drawn = a.breed && n_units <= 2 * kUnitThreads;
    uint32_t mskA = 0u, mskB = 0u;
    float2 zA[4], zB[4];
    if (tid < kUnitThreads) {
        if (drawn && kind != kKindElite) {
            if ((tid & ~31) < n_units) draw_unit(tid, tid < n_units, mskA, zA);
            if (kUnitThreads + (tid & ~31) < n_units)
                draw_unit(kUnitThreads + tid, kUnitThreads + tid < n_units, mskB, zB);
        }
    }
    // The batch's levels as FP32 in the padded layout (word t holds inputs
    // 4t .. 4t+3 of the row-major batch); a unit thread converts the words it
    // copied, while the first units' parent loads are in flight (step 2).
    auto convert_batch = [&]() {
        ptx::cp_async_wait_group<0>();
        if (a.xf) return;  // FP32 inputs arrive in place
        const int kw = K / 4;
        for (int t = tid; t < n4; t += kUnitThreads) {
            const int n = t / kw;
            *reinterpret_cast<float4*>(xs + n * (K + 4) + 4 * (t - n * kw)) = levels_to_float4(xraw[t]);
        }
    };

    // 1b. Larger populations: the whole CTA ranks (a bitonic sort of the keys
    // in shared memory, padding keys last), then thread 0 selects.
    if (a.breed && !sel_warp) {
        for (int t = tid; t < n2; t += kSmallThreads) {
            const float f = t < P ? __ldcg(a.f_adj_in + t) : 0.0f;
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
        const ChildSelection c = sel_s;
        float* child = a.popv + static_cast<int64_t>(i) * a.c_pad;
        const float* par1 = a.parents + static_cast<int64_t>(c.p1) * a.c_pad;
        const float* par2 = a.parents + static_cast<int64_t>(c.p2) * a.c_pad;
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
        // The unit's genes from its parents' and its drawn numbers; then stored
        // (children) and kept in shared memory.  ok: this lane's unit exists.
        auto finish = [&](int t, bool ok, int64_t g0, float4 (&v)[2], const float4 (&w)[2], uint32_t msk,
                          const float2 (&z)[4]) {
            if (!ok) return;
            if (a.breed) {
                if (c.kind == kKindMut) {
                    apply_mutation8(c.sigma, msk, z, v);
                } else if (c.kind == kKindCross) {
                    if (a.br.xo_op == 0) {
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
                reinterpret_cast<float4*>(child + g0)[0] = v[0];
                reinterpret_cast<float4*>(child + g0)[1] = v[1];
            }
            if (t < K) {  // genes 8t .. 8t+7 of the slice's rows: row l / K, input l % K
                // (K % 4 == 0: each half of the unit is 4 genes of one row, 16-byte aligned)
                const int r = (8 * t) / K, col = 8 * t - r * K;
                *reinterpret_cast<float4*>(w1s + r * (K + 4) + col) = v[0];
                const int r1 = col + 4 < K ? r : r + 1, col1 = col + 4 < K ? col + 4 : col + 4 - K;
                *reinterpret_cast<float4*>(w1s + r1 * (K + 4) + col1) = v[1];
            } else {  // b1, column block 8q .. 8q+7 of W2 row t - K - 1, or (slice 0) 8 genes of b2
                float* dst = t == K ? b1s : (t <= K + D ? w2s + (t - K - 1) * kSlice : b2s + 8 * (t - K - 1 - D));
                reinterpret_cast<float4*>(dst)[0] = v[0];
                reinterpret_cast<float4*>(dst)[1] = v[1];
            }
        };
        for (int base = 0; tid < kUnitThreads && base < n_units; base += 2 * kUnitThreads) {
            const int tA = base + tid, tB = tA + kUnitThreads;
            const bool okA = tA < n_units, okB = tB < n_units;
            const int64_t gA = okA ? first_gene(tA) : 0, gB = okB ? first_gene(tB) : 0;
            float4 vA[2], wA[2], vB[2], wB[2];
            if (okA) load(gA, vA, wA);
            if (okB) load(gB, vB, wB);
            if (base == 0) convert_batch();
            if (a.breed && !(drawn && base == 0) && kind != kKindElite) {  // later rounds draw here
                const int wbase = base + (tid & ~31);
                if (wbase < n_units) draw_unit(tA, okA, mskA, zA);
                if (wbase + kUnitThreads < n_units) draw_unit(tB, okB, mskB, zB);
            }
            finish(tA, okA, gA, vA, wA, mskA, zA);
            finish(tB, okB, gB, vB, wB, mskB, zB);
        }
    }
    __syncthreads();

    // 3. Layer 1 of the slice (hidden unit jj, sample n) on the tensor cores:
    // the levels k are exact TF32 operands and each weight enters as two TF32
    // pieces (w_hi = tf32(w), w_lo = tf32(w - w_hi): 22 of FP32's 24 bits), so
    // every product is exact and only the FP32 accumulation rounds; FP32
    // inputs are split the same way and enter as x_hi w_hi + x_hi w_lo +
    // x_lo w_hi (x_div = 1).  Warp w
    // takes sample tile w / groups and every groups-th 8-input step from
    // w % groups on; the groups' partial tiles are added in order, divided by
    // x_div; then bias and ReLU.
    {
        const int n_tiles = (Bt + 15) / 16, T16 = 16 * n_tiles;
        const int groups = kWarps / n_tiles > 1 ? kWarps / n_tiles : 1;
        const int n_steps = (K + 7) / 8;
        const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
        const bool float_x = a.xf != nullptr;
        if (warp < groups * n_tiles) {
            const int tile = warp / groups, kg = warp - tile * groups;
            const float* x_lo = xs + min(16 * tile + g, Bt - 1) * (K + 4);      // sample rows g and g + 8
            const float* x_hi = xs + min(16 * tile + g + 8, Bt - 1) * (K + 4);  // (past the batch: not kept)
            const float* wrow = w1s + g * (K + 4);                               // hidden unit g of the slice
            float d[4] = { 0.0f, 0.0f, 0.0f, 0.0f };
            for (int st = kg; st < n_steps; st += groups) {
                const int k0 = 8 * st + tq, k1 = k0 + 4;
                const bool in0 = k0 < K, in1 = k1 < K;
                const float xv[4] = { in0 ? x_lo[k0] : 0.0f, in0 ? x_hi[k0] : 0.0f, in1 ? x_lo[k1] : 0.0f,
                                      in1 ? x_hi[k1] : 0.0f };
                const float w0 = in0 ? wrow[k0] : 0.0f, w1 = in1 ? wrow[k1] : 0.0f;
                const uint32_t h0 = to_tf32(w0), h1 = to_tf32(w1);
                const uint32_t l0 = to_tf32(w0 - __uint_as_float(h0)), l1 = to_tf32(w1 - __uint_as_float(h1));
                if (!float_x) {  // the levels are exact TF32 operands
                    const uint32_t av[4] = { __float_as_uint(xv[0]), __float_as_uint(xv[1]), __float_as_uint(xv[2]),
                                             __float_as_uint(xv[3]) };
                    mma_tf32(d, av, h0, h1);
                    mma_tf32(d, av, l0, l1);
                } else {  // x_hi w_hi + x_hi w_lo + x_lo w_hi
                    uint32_t ah[4], al[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        ah[e] = to_tf32(xv[e]);
                        al[e] = to_tf32(xv[e] - __uint_as_float(ah[e]));
                    }
                    mma_tf32(d, ah, h0, h1);
                    mma_tf32(d, ah, l0, l1);
                    mma_tf32(d, al, h0, h1);
                }
            }
            float* part = qs + (kg * T16 + 16 * tile) * kSlice;  // [16 samples][8 hidden units]
            part[g * kSlice + 2 * tq] = d[0];
            part[g * kSlice + 2 * tq + 1] = d[1];
            part[(g + 8) * kSlice + 2 * tq] = d[2];
            part[(g + 8) * kSlice + 2 * tq + 1] = d[3];
        }
        __syncthreads();
        for (int ch = tid; ch < kSlice * Bt; ch += kSmallThreads) {
            float v = qs[ch];
            for (int kg = 1; kg < groups; ++kg) v += qs[kg * T16 * kSlice + ch];
            hs[ch] = fmaxf(v / a.x_div + b1s[ch & (kSlice - 1)], 0.0f);
        }
    }
    __syncthreads();
    // The slice's share of layer 2: partial logit o of sample n over hidden
    // units 8q .. 8q+7 in ascending order.
    {
        float* part = a.part + (static_cast<int64_t>(i) * a.n_slices + q) * Bt * D;  // [Bt][D]
        if (CLUSTER) cluster_wait_acquire();
        const uint32_t dst = CLUSTER ? cluster_map(gather + q * Bt * D, 0) : 0u;
        for (int ch = tid; ch < Bt * D; ch += kSmallThreads) {
            const int n = ch / D, o = ch - n * D;
            const float* wv = w2s + o * kSlice;
            const float* hv = hs + n * kSlice;
            float s = 0.0f;
#pragma unroll
            for (int r = 0; r < kSlice; ++r) s = fmaf(wv[r], hv[r], s);
            if (CLUSTER) st_cluster_f32(dst + 4u * static_cast<uint32_t>(ch), s);
            else part[ch] = s;
        }
    }

    // 4. Hand-over.  Cluster: the barrier releases every slice's partial logits
    // to slice 0, which finishes.  Otherwise: the block barrier orders the
    // CTA's partial logits before thread 0's fence, which releases them with
    // its count (and, in the last arriver, acquires the other slices' before
    // the barrier that follows).
    if (CLUSTER) {
        cluster_arrive_release();
        cluster_wait_acquire();
        if (q != 0) return;
    } else {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const bool last = atomicAdd(a.count + i, 1u) == static_cast<uint32_t>(a.n_slices - 1);
            if (last) __threadfence();
            last_s = last ? 1 : 0;
        }
        __syncthreads();
        if (!last_s) return;
    }

    float* Ls = R;                        // [D][Bt]: the logits z
    float* lossv = Ls + D * Bt;           // [kSmallMaxBatch]
    int32_t* corv = reinterpret_cast<int32_t*>(lossv + kSmallMaxBatch);  // [kSmallMaxBatch]
    float* warp_sums = reinterpret_cast<float*>(corv + kSmallMaxBatch);  // [32]
    {  // z = the slices' partial logits added in slice order, then b2
        const float* b2 = a.popv + static_cast<int64_t>(i) * a.c_pad + a.b2_off;
        const float* part = a.part + static_cast<int64_t>(i) * a.n_slices * Bt * D;
        const int slice_stride = Bt * D;
        for (int ch = tid; ch < Bt * D; ch += kSmallThreads) {
            const int n = ch / D, o = ch - n * D;
            float s, bias;
            if (CLUSTER) {  // slice 0 holds b2 and every slice's partial logits
                bias = b2s[o];
                s = gather[ch];
                for (int qq = 1; qq < a.n_slices; ++qq) s += gather[qq * slice_stride + ch];
            } else {
                bias = __ldcg(b2 + o);
                s = __ldcg(part + ch);
#pragma unroll 4
                for (int qq = 1; qq < a.n_slices; ++qq) s += __ldcg(part + static_cast<int64_t>(qq) * slice_stride + ch);
            }
            Ls[o * Bt + n] = s + bias;
        }
    }
    __syncthreads();

    // Per-sample softmax cross-entropy (Eq. 1): log sum exp(z - max z) + max z
    // - z[label], the exponentials summed over the classes in ascending order,
    // and the argmax (the lowest class on ties); then the fixed-order batch
    // sum: per tile of BN samples a warp xor-tree over each 32 samples, the
    // warp sums added in order, the tile sums added in order.
    auto sample_loss = [&](int n, float& loss, int32_t& ok) {
        float zmax = Ls[n];
        int arg = 0;
        for (int o = 1; o < D; ++o) {
            const float z = Ls[o * Bt + n];
            if (z > zmax) { zmax = z; arg = o; }
        }
        float s = 0.0f;
#pragma unroll 4
        for (int o = 0; o < D; ++o) s += expf(Ls[o * Bt + n] - zmax);
        const int32_t lbl = a.y[n];
        if (lbl >= 0 && lbl < D) {
            loss = logf(s) + zmax - Ls[lbl * Bt + n];
            ok = (arg == lbl) ? 1 : 0;
        } else {
            loss = __int_as_float(0x7FC00000);  // NaN: label out of range
        }
    };
    auto write_out = [&](float total, int32_t n_correct) {
        const float f = -(total / static_cast<float>(Bt));
        a.f_raw[i] = f;
        a.f_adj[i] = a.breed ? (1.0f - a.alpha) * sel_s.f_inh + a.alpha * f : f;
        if (a.correct) a.correct[i] = n_correct;
        if (!CLUSTER) a.count[i] = 0u;  // for the next launch
    };
    const int BN = simt_batch_tile(Bt);
    if (Bt <= 32) {  // one tile, one warp: a lane per sample, no block barriers
        if (tid < 32) {
            float v = 0.0f;
            int32_t cv = 0;
            if (tid < Bt) sample_loss(tid, v, cv);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
                cv += __shfl_xor_sync(0xFFFFFFFFu, cv, off);
            }
            if (tid == 0) {
                float s = 0.0f, total = 0.0f;
                s += v;
                total += s;
                write_out(total, cv);
            }
        }
        return;
    }
    float total = 0.0f;  // meaningful in thread 0 only
    int32_t n_correct = 0;
    for (int b0 = 0; b0 < Bt; b0 += BN) {
        if (tid < BN) {
            const int gn = b0 + tid;
            float loss = 0.0f;
            int32_t ok = 0;
            if (gn < Bt) sample_loss(gn, loss, ok);
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
    if (tid == 0) write_out(total, n_correct);
}

}  // namespace

namespace {

size_t smem_bytes_of(int32_t d_in, int32_t h, int32_t d_out, int32_t batch, int32_t pop, bool cluster)
{
    const size_t gather = cluster ? static_cast<size_t>(h / kSlice) * batch * d_out : 0;
    const int64_t tail = small_tail_floats(small_region_floats(d_in, h, d_out, batch), pow2_at_least(pop), pop);
    return sizeof(float) * (static_cast<size_t>(tail) + 8 * static_cast<size_t>((d_out + 7) / 8) + gather);
}

constexpr int kMaxClusterSlices = 8;  // portable cluster size

}  // namespace

size_t small_gen_smem_bytes(int32_t d_in, int32_t h, int32_t d_out, int32_t batch, int32_t pop)
{
    return smem_bytes_of(d_in, h, d_out, batch, pop, false);
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
    a.b2_units = (a.d_out + 7) / 8;
    a.region_floats = small_region_floats(a.d_in, a.h, a.d_out, a.batch);
    const size_t smem_c = smem_bytes_of(a.d_in, a.h, a.d_out, a.batch, a.pop, true);
    const bool cluster = a.n_slices <= kMaxClusterSlices && smem_c <= kSmallMaxSmem;
    const size_t smem = cluster ? smem_c : smem_bytes_of(a.d_in, a.h, a.d_out, a.batch, a.pop, false);
    auto kernel = cluster ? small_gen_kernel<true> : small_gen_kernel<false>;
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(a.pop * a.n_slices);
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = static_cast<unsigned>(a.n_slices);
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cluster ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

}  // namespace leea
