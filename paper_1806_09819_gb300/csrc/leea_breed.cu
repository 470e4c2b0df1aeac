// leea_breed.cu -- crossover and mutation (Section 3.2) fused into one
// streaming pass over every child's genes.
//
// The pass is HBM-bound: per gene it reads one (mutation, elite) or two
// (crossover) parent floats and writes one child float.  To keep HBM busy
// while the generator arithmetic runs, the kernel is persistent (one CTA per
// SM) and decoupled:
//   warp 0               streams parent chunks (6144 genes = 24 KB per parent
//                        for one run, 4096 for many) into a ring of
//                        shared-memory stages with cp.async.bulk, tracked by
//                        transaction-count mbarriers;
//   warps 1-24 (1-16)    take a stage, compute the child chunk and write it
//                        with 128-bit stores, then release the stage.
// Work items walk the children alternately from the front (elites, crossover
// children) and the back (mutation children), so every SM mixes the
// HBM-heavier crossover items with the arithmetic-heavier mutation items;
// with one run they go chunk by chunk over all children, so that parents
// shared by several children are read from HBM about once.  The producer
// warp resolves 32 items' children and parents at a time.
// With many runs each CTA takes a contiguous range of items, so that it
// meets few run boundaries (each one reloads the run's arguments).
// A consumer thread owns 8 consecutive genes of the chunk: one Philox block
// of 16-bit mask draws (crossover or mutation mask) and two Philox blocks of
// normals.  In mutation children only the Box-Muller pairs that hold a masked
// gene are generated, and a warp first gathers them into a dense job list in
// shared memory (one ballot per pair slot) so that normals are computed by
// consecutive lanes instead of by whichever lane happens to own a masked
// gene; the normals go back through the same list.  Every mbarrier
// wait is bounded in time; on expiry the kernel sets kStatusBreedTimeout.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "breed_ops.cuh"
#include "leea_internal.h"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace leea {

namespace {

// Shape of the kernel: one run takes 24 consumer warps (about six per
// scheduler, to hide the Philox and Box-Muller dependency chains) over
// 6144-gene chunks in a 4-deep ring; many runs keep 16 warps over 4096-gene
// chunks in a 6-deep ring (their per-run state needs more registers).
template <bool MULTI>
struct BreedShape {
    static constexpr int kConsumerWarps = MULTI ? 16 : 24;
    static constexpr int kThreads = 32 * (1 + kConsumerWarps);
    static constexpr int kChunk = 8 * 32 * kConsumerWarps;  // genes per work item: 8 per consumer thread
    static constexpr int kStages = MULTI ? 6 : 4;           // ring depth (2 parent chunks per stage)
    static constexpr uint32_t kChunkBytes = kChunk * 4;
};
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;
constexpr int32_t kKindInvalid = -1;

struct StageMeta {
    int32_t j;       // child
    int32_t kind;    // 0 elite, 1 crossover, 2 mutation, -1 invalid parent index
    int32_t g0;      // first gene of the chunk
    int32_t len;     // genes in the chunk (multiple of 32)
    int32_t sexp;    // precision form, FP8: exponent of the child's scale
    int32_t run;     // many runs: index of the child's run
    float sigma;     // the child's mutation strength
    int32_t pad;
};

constexpr int kJobSlots = 4 * 32;  // Box-Muller pairs of a warp's 32 units

// An item's source as the producer warp resolves it, 32 items at a time.
struct ItemSrc {
    const float* p1;  // parent chunks (NULL for an invalid parent index)
    const float* p2;
    StageMeta m;
};

struct BreedSmem {
    uint8_t* base;   // stage i: parent 1 at base + 2i chunks, parent 2 at base + (2i+1) chunks
    StageMeta* meta;
    ItemSrc* batch;  // [32]: the producer warp's next 32 items
    float2* job_z;      // [consumer warps][kJobSlots]: normals of a warp's job list
    uint8_t* job_code;  // [consumer warps][kJobSlots]: owner lane << 2 | pair slot
    uint64_t* full;
    uint64_t* empty;
    volatile int* abort_flag;
};

template <bool MULTI>
__device__ __forceinline__ BreedSmem carve(uint8_t* raw)
{
    using S = BreedShape<MULTI>;
    constexpr int kStages = S::kStages, kConsumerWarps = S::kConsumerWarps;
    constexpr uint32_t kChunkBytes = S::kChunkBytes;
    BreedSmem s;
    uint8_t* base = raw + ((128u - (ptx::smem_u32(raw) & 127u)) & 127u);
    s.base = base;
    uint8_t* p = base + 2 * kStages * kChunkBytes;
    s.meta = reinterpret_cast<StageMeta*>(p);
    p += sizeof(StageMeta) * kStages;
    s.batch = reinterpret_cast<ItemSrc*>(p);
    p += sizeof(ItemSrc) * 32;
    s.job_z = reinterpret_cast<float2*>(p);
    p += sizeof(float2) * kConsumerWarps * kJobSlots;
    s.job_code = p;
    p += kConsumerWarps * kJobSlots;
    s.full = reinterpret_cast<uint64_t*>(p);
    s.empty = s.full + kStages;
    s.abort_flag = reinterpret_cast<volatile int*>(s.empty + kStages);
    return s;
}

template <bool MULTI>
constexpr size_t breed_smem_bytes()
{
    using S = BreedShape<MULTI>;
    return 128 + 2 * S::kStages * S::kChunkBytes + sizeof(StageMeta) * S::kStages + sizeof(ItemSrc) * 32 +
           (sizeof(float2) + 1) * S::kConsumerWarps * kJobSlots + 16 * S::kStages + 16;
}
static_assert(breed_smem_bytes<false>() <= 227 * 1024 && breed_smem_bytes<true>() <= 227 * 1024,
              "breed ring must fit in shared memory");

// The shadow of 8 child genes i0 .. i0+7 of W1: 8 BF16 (16 bytes) or 8 FP8-e4m3
// of w / 2^sexp with saturation (8 bytes).  Returns max |w| of the 8 genes.
__device__ __forceinline__ float write_shadow8(const BreedArgs& a, int32_t j, int32_t sexp, int64_t i0,
                                               const float4 (&v)[2])
{
    const float mx = fmaxf(fmaxf(fmaxf(fabsf(v[0].x), fabsf(v[0].y)), fmaxf(fabsf(v[0].z), fabsf(v[0].w))),
                           fmaxf(fmaxf(fabsf(v[1].x), fabsf(v[1].y)), fmaxf(fabsf(v[1].z), fabsf(v[1].w))));
    // Eight genes of one row: d_0 % 16 == 0 keeps them in one 16-byte (BF16)
    // or 8-byte (FP8) piece of a chunk.
    const int32_t i32 = static_cast<int32_t>(i0);  // a W1 gene: i0 < h d_0 < 2^31
    const int32_t o = i32 / a.sh_k;
    const int32_t k = i32 - o * a.sh_k;
    uint8_t* dst = a.shadow + static_cast<int64_t>(j) * a.sh_stride +
                   shadow_offset(a.sh_h, a.precision == 1 ? 2 : 1, o, k);
    if (a.precision == 1) {
        const __nv_bfloat162 b0 = __floats2bfloat162_rn(v[0].x, v[0].y);
        const __nv_bfloat162 b1 = __floats2bfloat162_rn(v[0].z, v[0].w);
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[1].x, v[1].y);
        const __nv_bfloat162 b3 = __floats2bfloat162_rn(v[1].z, v[1].w);
        uint4 w;
        w.x = *reinterpret_cast<const uint32_t*>(&b0);
        w.y = *reinterpret_cast<const uint32_t*>(&b1);
        w.z = *reinterpret_cast<const uint32_t*>(&b2);
        w.w = *reinterpret_cast<const uint32_t*>(&b3);
        *reinterpret_cast<uint4*>(dst) = w;
    } else {
        const float inv = ldexpf(1.0f, -sexp);  // exact: a power of two
        const __nv_fp8x2_storage_t q0 =
            __nv_cvt_float2_to_fp8x2(make_float2(v[0].x * inv, v[0].y * inv), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t q1 =
            __nv_cvt_float2_to_fp8x2(make_float2(v[0].z * inv, v[0].w * inv), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t q2 =
            __nv_cvt_float2_to_fp8x2(make_float2(v[1].x * inv, v[1].y * inv), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t q3 =
            __nv_cvt_float2_to_fp8x2(make_float2(v[1].z * inv, v[1].w * inv), __NV_SATFINITE, __NV_E4M3);
        uint2 w;
        w.x = static_cast<uint32_t>(q0) | (static_cast<uint32_t>(q1) << 16);
        w.y = static_cast<uint32_t>(q2) | (static_cast<uint32_t>(q3) << 16);
        *reinterpret_cast<uint2*>(dst) = w;
    }
    return mx;
}

__device__ __forceinline__ float* stage_a(const BreedSmem& s, uint32_t stage, uint32_t chunk_bytes)
{
    return reinterpret_cast<float*>(s.base + (2u * stage) * chunk_bytes);
}

__device__ __forceinline__ float* stage_b(const BreedSmem& s, uint32_t stage, uint32_t chunk_bytes)
{
    return reinterpret_cast<float*>(s.base + (2u * stage + 1u) * chunk_bytes);
}

__device__ __forceinline__ void raise_abort(volatile int* abort_flag, unsigned int* status)
{
    *abort_flag = 1;
    atomicOr(status, kStatusBreedTimeout);
}

constexpr int kGenesPerLane = 8;  // one Philox block of 16-bit mask draws per lane and chunk
static_assert(BreedShape<false>::kChunk == kGenesPerLane * 32 * BreedShape<false>::kConsumerWarps &&
                  BreedShape<true>::kChunk == kGenesPerLane * 32 * BreedShape<true>::kConsumerWarps,
              "consumers must tile a chunk exactly");

// The run owning global work item `it`: the last one whose first item is <= it.
__device__ __forceinline__ int32_t run_of_item(const BreedRun* runs, int32_t n_runs, int64_t it)
{
    int32_t lo = 0, hi = n_runs - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (runs[mid].item0 <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// MULTI = false: one run (run0), generation in run0.a.gen.  MULTI = true: the
// runs of a device table, whose work items are numbered consecutively, and
// the generation read from gen_dev.
template <bool MULTI>
__global__ void __launch_bounds__(BreedShape<MULTI>::kThreads, 1)
breed_kernel(const __grid_constant__ BreedRun run0, const BreedRun* __restrict__ runs, int32_t n_runs,
             int64_t n_items, const uint32_t* __restrict__ gen_dev, unsigned int* __restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    ptx::grid_dep_launch();  // the evaluation that follows may stage its batch meanwhile
    ptx::grid_dep_wait();    // the selection comes from the previous kernel
    using S = BreedShape<MULTI>;
    constexpr int kStages = S::kStages, kConsumerWarps = S::kConsumerWarps, kChunk = S::kChunk;
    constexpr uint32_t kChunkBytes = S::kChunkBytes;
    const BreedSmem s = carve<MULTI>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Items of this CTA: many runs, a contiguous range; one run, every gridDim.x-th
    // (neighbouring CTAs then work on neighbouring children, which share parents in L2).
    const int64_t it_begin = MULTI ? n_items * blockIdx.x / gridDim.x : blockIdx.x;
    const int64_t it_end = MULTI ? n_items * (blockIdx.x + 1) / gridDim.x : n_items;
    const int64_t it_step = MULTI ? 1 : gridDim.x;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            ptx::mbar_init(&s.full[i], 1);
            ptx::mbar_init(&s.empty[i], kConsumerWarps);
        }
        *s.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // The warp resolves 32 items at a time (lane l: the item's child,
        // kind, parents, scale and sigma; loads of all lanes in flight
        // together), then lane 0 streams their parent chunks into the ring.
        uint32_t stage = 0, phase = 0;
        uint32_t issued_mask = 0, parity_mask = 0;  // per stage: issued at all / parity of the last issue
        bool ok = true;
        for (int64_t base = it_begin; ok && base < it_end; base += 32 * it_step) {
            {
                const int64_t it = base + lane * it_step;
                ItemSrc src{};
                src.m.kind = kKindInvalid;
                src.m.len = 0;
                if (it < it_end) {
                    const int32_t ri = MULTI ? run_of_item(runs, n_runs, it) : 0;
                    const BreedRun& R = MULTI ? runs[ri] : run0;
                    const BreedArgs& a = R.a;
                    const int64_t li = it - R.item0;
                    // One run: chunk-major (all children's chunk 0, then chunk
                    // 1, ...), so the parents' chunk (pool x 16 KB) stays in L2
                    // while every child that reads it is made: each parent
                    // chunk comes from HBM about once however many children
                    // share it.  Many runs: child-major within each CTA's
                    // contiguous range.
                    const int32_t ci = MULTI ? static_cast<int32_t>(li / R.chunks) : static_cast<int32_t>(li % a.pop);
                    const int32_t ck = MULTI ? static_cast<int32_t>(li - static_cast<int64_t>(ci) * R.chunks)
                                             : static_cast<int32_t>(li / a.pop);
                    // Front (elites, crossover) and back (mutation) children
                    // alternate along a CTA's items; with an even grid a CTA's
                    // ci keep one parity, so alternate rounds swap ci with its
                    // pair partner (a bijection on each chunk's children).
                    int32_t x = ci;
                    if (!MULTI && (gridDim.x & 1u) == 0u) {
                        const int32_t y = ci ^ static_cast<int32_t>((static_cast<uint32_t>(ci) / gridDim.x) & 1u);
                        if (y < a.pop) x = y;
                    }
                    const int32_t j = (x & 1) ? a.pop - 1 - (x >> 1) : (x >> 1);
                    int32_t kind = R.kind[j];
                    const int32_t p1 = R.par1[j], p2 = R.par2[j];
                    const int32_t n_par = a.n_parents > 0 ? a.n_parents : a.pop;
                    if (p1 < 0 || p1 >= n_par || p2 < 0 || p2 >= n_par) kind = kKindInvalid;
                    const int64_t g0 = static_cast<int64_t>(ck) * kChunk;
                    const int32_t len = static_cast<int32_t>(a.c_pad - g0 < kChunk ? a.c_pad - g0 : kChunk);
                    src.m = StageMeta{ j, kind, static_cast<int32_t>(g0), len,
                                       (a.precision == 2) ? a.scale_exp[j] : 0, ri,
                                       a.sigma_child ? a.sigma_child[j] : a.sigma, 0 };
                    if (kind != kKindInvalid) {
                        src.p1 = R.parents + static_cast<int64_t>(p1) * a.c_pad + g0;
                        src.p2 = R.parents + static_cast<int64_t>(p2) * a.c_pad + g0;
                    }
                }
                s.batch[lane] = src;
            }
            __syncwarp();
            if (lane == 0) {
                for (int l = 0; l < 32 && base + l * it_step < it_end; ++l) {
                    if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s.abort_flag, status);
                        ok = false;
                        break;
                    }
                    const ItemSrc src = s.batch[l];
                    s.meta[stage] = src.m;
                    const uint32_t bytes = static_cast<uint32_t>(src.m.len) * 4u;
                    if (src.m.kind == kKindInvalid) {
                        ptx::mbar_arrive(&s.full[stage]);
                    } else {
                        const bool two = (src.m.kind == 1);
                        ptx::mbar_arrive_expect_tx(&s.full[stage], two ? 2u * bytes : bytes);
                        ptx::bulk_load(stage_a(s, stage, kChunkBytes), src.p1, bytes, &s.full[stage]);
                        if (two) ptx::bulk_load(stage_b(s, stage, kChunkBytes), src.p2, bytes, &s.full[stage]);
                    }
                    issued_mask |= 1u << stage;
                    parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                    if (++stage == kStages) { stage = 0; phase ^= 1u; }
                }
            }
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);  // also: lane 0 is done with the batch
        }
        if (!ok && lane == 0) {  // let copies in flight land before the CTA exits
            volatile int never = 0;
            for (int i = 0; i < kStages; ++i)
                if (issued_mask & (1u << i))
                    ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int ct = threadIdx.x - 32;
        const uint32_t gen = MULTI ? *gen_dev : run0.a.gen;
        PhiloxKeys key = philox_keys(run0.a.seed);
        // The current run's arguments and generator keys, held in registers
        // while consecutive items belong to the same run (many runs: the
        // table lives in global memory).
        BreedArgs a = run0.a;
        float* children = run0.children;
        int32_t cur_run = MULTI ? -1 : 0;
        uint32_t stage = 0, phase = 0;
        for (int64_t it = it_begin; it < it_end; it += it_step) {
            if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                raise_abort(s.abort_flag, status);
                break;
            }
            const StageMeta m = s.meta[stage];
            if (MULTI && m.run != cur_run) {
                a = runs[m.run].a;
                children = runs[m.run].children;
                key = philox_keys(a.seed);
                cur_run = m.run;
            }
            const float4* A = reinterpret_cast<const float4*>(stage_a(s, stage, kChunkBytes));
            const float4* B = reinterpret_cast<const float4*>(stage_b(s, stage, kChunkBytes));
            float4* O = reinterpret_cast<float4*>(children + static_cast<int64_t>(m.j) * a.c_pad + m.g0);
            const uint32_t j = a.entity ? a.entity[m.j] : static_cast<uint32_t>(m.j);  // Philox entity
            const bool live = ct * kGenesPerLane < m.len;
            const uint32_t u = (static_cast<uint32_t>(m.g0) >> 3) + static_cast<uint32_t>(ct);  // 8-gene unit
            float4 v[2] = { make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f) };
            if (live && m.kind >= 0) {
                v[0] = A[2 * ct];
                v[1] = A[2 * ct + 1];
            }
            if (m.kind == 2) {
                // Lanes of a warp own consecutive units: lane o owns u - lane + o.
                const int cw = warp - 1;  // consumer warp
                const uint32_t hit = live ? mask8(philox_keyed(make_uint4(u, j, gen, kTagMutMask), key), a.thr_mut) : 0u;
                mutate8(m.sigma, gen, key, j, hit, v, lane, s.job_z + cw * kJobSlots, s.job_code + cw * kJobSlots,
                        [&](uint32_t o) { return u - static_cast<uint32_t>(lane) + o; });
            } else if (live && m.kind == 1) {
                const float4 b0 = B[2 * ct], b1 = B[2 * ct + 1];
                if (a.xo_op == 0) {
                    const uint32_t msk = mask8(philox_keyed(make_uint4(u, j, gen, kTagXo), key), a.thr_xo);
                    v[0] = select4(msk, v[0], b0);
                    v[1] = select4(msk >> 4, v[1], b1);
                } else {
                    v[0] = mean4(v[0], b0);
                    v[1] = mean4(v[1], b1);
                }
            } else if (m.kind == kKindInvalid) {
                const float nan = __int_as_float(0x7FC00000);
                v[0] = v[1] = make_float4(nan, nan, nan, nan);
            }
            if (live) {
                const int64_t i0 = static_cast<int64_t>(m.g0) + kGenesPerLane * ct;
                if (i0 + kGenesPerLane > a.c) {  // only a child's last chunk holds padding
                    v[0] = clear_padding(v[0], i0, a.c);
                    v[1] = clear_padding(v[1], i0 + 4, a.c);
                }
                O[2 * ct] = v[0];
                O[2 * ct + 1] = v[1];
            }
            if (a.precision > 0 && static_cast<int64_t>(m.g0) < a.n_w1) {  // warp-uniform
                const int64_t i0 = static_cast<int64_t>(m.g0) + kGenesPerLane * ct;
                float mx = 0.0f;
                if (live && i0 < a.n_w1) mx = write_shadow8(a, m.j, m.sexp, i0, v);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
                if (lane == 0 && mx > 0.0f) atomicMax(reinterpret_cast<int*>(a.amax_out + m.j), __float_as_int(mx));
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.empty[stage]);
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
    }
    __syncthreads();
}

}  // namespace

int32_t breed_chunks(int64_t c_pad)
{
    return static_cast<int32_t>((c_pad + BreedShape<true>::kChunk - 1) / BreedShape<true>::kChunk);
}

namespace {

cudaError_t breed_grid(int64_t items, int* grid)
{
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    *grid = static_cast<int>(items < sms ? (items > 0 ? items : 1) : sms);
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_breed(const BreedArgs& a, const float* parents, const int32_t* par1, const int32_t* par2,
                         const int32_t* kind, float* children, unsigned int* status, cudaStream_t stream)
{
    BreedRun r{};
    r.a = a;
    r.parents = parents;
    r.par1 = par1;
    r.par2 = par2;
    r.kind = kind;
    r.children = children;
    r.chunks = static_cast<int32_t>((a.c_pad + BreedShape<false>::kChunk - 1) / BreedShape<false>::kChunk);
    r.item0 = 0;
    const int64_t items = static_cast<int64_t>(a.pop) * r.chunks;
    int grid = 0;
    cudaError_t err = breed_grid(items, &grid);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(breed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(breed_smem_bytes<false>()));
    if (err != cudaSuccess) return err;
    return launch_pdl(breed_kernel<false>, dim3(grid), dim3(BreedShape<false>::kThreads), breed_smem_bytes<false>(),
                      stream, r,
                      static_cast<const BreedRun*>(nullptr), 1, items, static_cast<const uint32_t*>(nullptr), status);
}

cudaError_t launch_breed_runs(const BreedRun* runs_dev, int32_t n_runs, int64_t n_items, const uint32_t* gen_dev,
                              unsigned int* status, cudaStream_t stream)
{
    int grid = 0;
    cudaError_t err = breed_grid(n_items, &grid);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(breed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(breed_smem_bytes<true>()));
    if (err != cudaSuccess) return err;
    const BreedRun none{};
    breed_kernel<true><<<grid, BreedShape<true>::kThreads, breed_smem_bytes<true>(), stream>>>(
        none, runs_dev, n_runs, n_items, gen_dev, status);
    return cudaGetLastError();
}

}  // namespace leea
