// leea_breed.cu -- crossover and mutation (Section 3.2) fused into one
// streaming pass over every child's genes.
//
// The pass is HBM-bound: per gene it reads one (mutation, elite) or two
// (crossover) parent floats and writes one child float.  To keep HBM busy
// while the generator arithmetic runs, the kernel is persistent (one CTA per
// SM) and decoupled:
//   warp 0 (one thread)  streams parent chunks (4096 genes = 16 KB per parent)
//                        into a ring of shared-memory stages with
//                        cp.async.bulk, tracked by transaction-count mbarriers;
//   warps 1-16           take a stage, compute the child chunk and write it
//                        with 128-bit stores, then release the stage.
// Work items walk the children alternately from the front (elites, crossover
// children) and the back (mutation children), so every SM mixes the
// HBM-heavier crossover items with the arithmetic-heavier mutation items.
// A consumer thread owns blocks of four consecutive genes (two per chunk),
// which is exactly one Philox block of each per-gene stream.  In mutation
// children only the Box-Muller pairs that hold a masked gene are generated,
// and a warp first gathers them into a dense job list (ballot-free prefix
// scan over the lanes) so that normals are computed by consecutive lanes
// instead of by whichever lane happens to own a masked gene.  Every mbarrier
// wait is bounded in time; on expiry the kernel sets kStatusBreedTimeout.
#include "leea_internal.h"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr uint32_t kTagXo = 3, kTagMutMask = 4, kTagNormal = 5;
constexpr int kConsumerWarps = 16;
constexpr int kBreedThreads = 32 * (1 + kConsumerWarps);
constexpr int kChunk = 4096;                // genes per work item
constexpr int kStages = 6;                  // ring depth (2 x 16 KB per stage)
constexpr uint32_t kChunkBytes = kChunk * 4;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;
constexpr int32_t kKindInvalid = -1;

struct StageMeta {
    int32_t j;       // child
    int32_t kind;    // 0 elite, 1 crossover, 2 mutation, -1 invalid parent index
    int32_t g0;      // first gene of the chunk
    int32_t len;     // genes in the chunk (multiple of 32)
};

struct BreedSmem {
    uint8_t* base;   // stage i: parent 1 at base + 2i chunks, parent 2 at base + (2i+1) chunks
    StageMeta* meta;
    uint64_t* full;
    uint64_t* empty;
    volatile int* abort_flag;
};

__device__ __forceinline__ BreedSmem carve(uint8_t* raw)
{
    BreedSmem s;
    uint8_t* base = raw + ((128u - (ptx::smem_u32(raw) & 127u)) & 127u);
    s.base = base;
    uint8_t* p = base + 2 * kStages * kChunkBytes;
    s.meta = reinterpret_cast<StageMeta*>(p);
    p += sizeof(StageMeta) * kStages;
    s.full = reinterpret_cast<uint64_t*>(p);
    s.empty = s.full + kStages;
    s.abort_flag = reinterpret_cast<volatile int*>(s.empty + kStages);
    return s;
}

constexpr size_t kBreedSmemBytes =
    128 + 2 * kStages * kChunkBytes + sizeof(StageMeta) * kStages + 16 * kStages + 16;

__device__ __forceinline__ float* stage_a(const BreedSmem& s, uint32_t stage)
{
    return reinterpret_cast<float*>(s.base + (2u * stage) * kChunkBytes);
}

__device__ __forceinline__ float* stage_b(const BreedSmem& s, uint32_t stage)
{
    return reinterpret_cast<float*>(s.base + (2u * stage + 1u) * kChunkBytes);
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(ptx::smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(ptx::smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void raise_abort(volatile int* abort_flag, unsigned int* status)
{
    *abort_flag = 1;
    atomicOr(status, kStatusBreedTimeout);
}

constexpr int kBlocksPerLane = 2;  // 4096-gene chunk = 1024 blocks = 512 consumers x 2
static_assert(kChunk / 4 == kBlocksPerLane * 32 * kConsumerWarps, "consumers must tile a chunk exactly");

// Zero the padding genes (>= c) of block q.
__device__ __forceinline__ float4 clear_padding(float4 v, uint32_t q, int64_t c)
{
    const int64_t i0 = 4 * static_cast<int64_t>(q);
    if (i0 + 3 >= c) {
        if (i0 + 0 >= c) v.x = 0.0f;
        if (i0 + 1 >= c) v.y = 0.0f;
        if (i0 + 2 >= c) v.z = 0.0f;
        if (i0 + 3 >= c) v.w = 0.0f;
    }
    return v;
}

// Elite copy, uniform or arithmetic crossover of block q.
__device__ __forceinline__ float4 cross_block(const BreedArgs& a, const PhiloxKeys& key, int32_t kind, uint32_t j,
                                              uint32_t q, float4 va, float4 vb)
{
    if (kind == 1) {
        if (a.xo_op == 0) {
            const uint4 r = philox_keyed(make_uint4(q, j, a.gen, kTagXo), key);
            va.x = hits(r.x, a.thr_xo) ? vb.x : va.x;
            va.y = hits(r.y, a.thr_xo) ? vb.y : va.y;
            va.z = hits(r.z, a.thr_xo) ? vb.z : va.z;
            va.w = hits(r.w, a.thr_xo) ? vb.w : va.w;
        } else {
            va = make_float4(0.5f * (va.x + vb.x), 0.5f * (va.y + vb.y), 0.5f * (va.z + vb.z), 0.5f * (va.w + vb.w));
        }
    } else if (kind == kKindInvalid) {
        const float nan = __int_as_float(0x7FC00000);
        va = make_float4(nan, nan, nan, nan);
    }
    return va;
}

// Mutation of this lane's kBlocksPerLane blocks q[g] (valid where live[g]).
// Slot s = 2 g + pair names the Box-Muller pair (genes 4q + 2 pair, +1).
__device__ __forceinline__ void mutate_blocks(const BreedArgs& a, const PhiloxKeys& key, uint32_t j,
                                              const uint32_t (&q)[kBlocksPerLane], const bool (&live)[kBlocksPerLane],
                                              float4 (&v)[kBlocksPerLane], int lane)
{
    constexpr int kSlots = 2 * kBlocksPerLane;
    uint32_t hit[kBlocksPerLane];  // 4 bits: which genes of the block mutate
    uint32_t need = 0;             // kSlots bits: which pairs need normals
#pragma unroll
    for (int g = 0; g < kBlocksPerLane; ++g) {
        hit[g] = 0;
        if (live[g]) {
            const uint4 r = philox_keyed(make_uint4(q[g], j, a.gen, kTagMutMask), key);
            hit[g] = (hits(r.x, a.thr_mut) ? 1u : 0u) | (hits(r.y, a.thr_mut) ? 2u : 0u) |
                     (hits(r.z, a.thr_mut) ? 4u : 0u) | (hits(r.w, a.thr_mut) ? 8u : 0u);
        }
        need |= ((hit[g] & 3u) ? 1u : 0u) << (2 * g);
        need |= ((hit[g] & 12u) ? 1u : 0u) << (2 * g + 1);
    }
    // Exclusive prefix of the per-lane job counts: jobs are numbered by lane,
    // then by slot.
    const uint32_t cnt = __popc(need);
    uint32_t incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += o;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);

    float2 z[kSlots];
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) z[sl] = make_float2(0.f, 0.f);
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t job = base + static_cast<uint32_t>(lane);
        // Owner lane o: the last lane whose exclusive prefix is <= job.
        int o = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int cand = o + step;
            const uint32_t e = __shfl_sync(0xFFFFFFFFu, excl, cand & 31);
            if (cand < 32 && e <= job) o = cand;
        }
        const uint32_t mo = __shfl_sync(0xFFFFFFFFu, need, o);
        const uint32_t eo = __shfl_sync(0xFFFFFFFFu, excl, o);
        float2 zz = make_float2(0.f, 0.f);
        if (job < total) {
            // The (job - eo)-th set slot of the owner.
            uint32_t nth = job - eo, slot = 0, mm = mo;
#pragma unroll
            for (int sl = 0; sl < kSlots; ++sl) {
                if (mm & 1u) {
                    if (nth == 0) { slot = sl; break; }
                    --nth;
                }
                mm >>= 1;
            }
            // Lanes of a warp own consecutive blocks (q[g] - lane is the same
            // for every lane): shift this lane's block g to the owner's.
            uint32_t qg = q[0];
#pragma unroll
            for (int g = 1; g < kBlocksPerLane; ++g)
                if (static_cast<uint32_t>(g) == (slot >> 1)) qg = q[g];
            const uint32_t qb = qg - static_cast<uint32_t>(lane) + static_cast<uint32_t>(o);
            const uint4 n = philox_keyed(make_uint4(qb, j, a.gen, kTagNormal), key);
            zz = (slot & 1u) ? box_muller(n.z, n.w) : box_muller(n.x, n.y);
        }
        // Every lane fetches the normals of its own slots numbered in this pass.
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) {
            const uint32_t id = excl + __popc(need & ((1u << sl) - 1u));
            const bool mine = ((need >> sl) & 1u) && id >= base && id < base + 32;
            const int src = mine ? static_cast<int>(id - base) : lane;
            const float zx = __shfl_sync(0xFFFFFFFFu, zz.x, src);
            const float zy = __shfl_sync(0xFFFFFFFFu, zz.y, src);
            if (mine) z[sl] = make_float2(zx, zy);
        }
    }
#pragma unroll
    for (int g = 0; g < kBlocksPerLane; ++g) {
        const float2 z0 = z[2 * g], z1 = z[2 * g + 1];
        if (hit[g] & 1u) v[g].x = fmaf(a.sigma, z0.x, v[g].x);
        if (hit[g] & 2u) v[g].y = fmaf(a.sigma, z0.y, v[g].y);
        if (hit[g] & 4u) v[g].z = fmaf(a.sigma, z1.x, v[g].z);
        if (hit[g] & 8u) v[g].w = fmaf(a.sigma, z1.y, v[g].w);
    }
}

__global__ void __launch_bounds__(kBreedThreads, 1)
breed_kernel(BreedArgs a, int32_t chunks_per_child, const float* __restrict__ parents,
             const int32_t* __restrict__ par1, const int32_t* __restrict__ par2, const int32_t* __restrict__ kind,
             float* __restrict__ children, unsigned int* __restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    const BreedSmem s = carve(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            ptx::mbar_init(&s.full[i], 1);
            ptx::mbar_init(&s.empty[i], kConsumerWarps);
        }
        *s.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();

    const int64_t n_items = static_cast<int64_t>(a.pop) * chunks_per_child;
    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            uint32_t issued_mask = 0, parity_mask = 0;  // per stage: issued at all / parity of the last issue
            int32_t cur_j = -1, cur_kind = 0, cur_p1 = 0, cur_p2 = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
                if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s.abort_flag, status);
                    ok = false;
                    break;
                }
                const int32_t ci = static_cast<int32_t>(it / chunks_per_child);
                const int32_t ck = static_cast<int32_t>(it - static_cast<int64_t>(ci) * chunks_per_child);
                const int32_t j = (ci & 1) ? a.pop - 1 - (ci >> 1) : (ci >> 1);
                if (j != cur_j) {
                    cur_j = j;
                    cur_kind = kind[j];
                    cur_p1 = par1[j];
                    cur_p2 = par2[j];
                    if (cur_p1 < 0 || cur_p1 >= a.pop || cur_p2 < 0 || cur_p2 >= a.pop) cur_kind = kKindInvalid;
                }
                const int64_t g0 = static_cast<int64_t>(ck) * kChunk;
                const int32_t len = static_cast<int32_t>(a.c_pad - g0 < kChunk ? a.c_pad - g0 : kChunk);
                s.meta[stage] = StageMeta{ j, cur_kind, static_cast<int32_t>(g0), len };
                const uint32_t bytes = static_cast<uint32_t>(len) * 4u;
                if (cur_kind == kKindInvalid) {
                    ptx::mbar_arrive(&s.full[stage]);
                } else {
                    const bool two = (cur_kind == 1);
                    ptx::mbar_arrive_expect_tx(&s.full[stage], two ? 2u * bytes : bytes);
                    bulk_load(stage_a(s, stage), parents + static_cast<int64_t>(cur_p1) * a.c_pad + g0, bytes, &s.full[stage]);
                    if (two)
                        bulk_load(stage_b(s, stage), parents + static_cast<int64_t>(cur_p2) * a.c_pad + g0, bytes,
                                  &s.full[stage]);
                }
                issued_mask |= 1u << stage;
                parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                for (int i = 0; i < kStages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
            }
        }
    } else {
        // ------------------------------------------------------------ consumers
        const int ct = threadIdx.x - 32;
        const PhiloxKeys key = philox_keys(a.seed);
        uint32_t stage = 0, phase = 0;
        for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
            if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                raise_abort(s.abort_flag, status);
                break;
            }
            const StageMeta m = s.meta[stage];
            const float4* A = reinterpret_cast<const float4*>(stage_a(s, stage));
            const float4* B = reinterpret_cast<const float4*>(stage_b(s, stage));
            float4* O = reinterpret_cast<float4*>(children + static_cast<int64_t>(m.j) * a.c_pad + m.g0);
            const int nq = m.len >> 2;
            const uint32_t q0 = static_cast<uint32_t>(m.g0) >> 2;
            const uint32_t j = static_cast<uint32_t>(m.j);
            uint32_t q[kBlocksPerLane];
            bool live[kBlocksPerLane];
            float4 v[kBlocksPerLane];
#pragma unroll
            for (int g = 0; g < kBlocksPerLane; ++g) {
                const int t = ct + g * 32 * kConsumerWarps;
                live[g] = t < nq;
                q[g] = q0 + static_cast<uint32_t>(t);
                v[g] = (live[g] && m.kind >= 0) ? A[t] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (m.kind == 2) {
                mutate_blocks(a, key, j, q, live, v, lane);
            } else {
#pragma unroll
                for (int g = 0; g < kBlocksPerLane; ++g) {
                    const int t = ct + g * 32 * kConsumerWarps;
                    if (live[g]) {
                        const float4 vb = (m.kind == 1) ? B[t] : v[g];
                        v[g] = cross_block(a, key, m.kind, j, q[g], v[g], vb);
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < kBlocksPerLane; ++g) {
                const int t = ct + g * 32 * kConsumerWarps;
                if (live[g]) O[t] = clear_padding(v[g], q[g], a.c);
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.empty[stage]);
            if (++stage == kStages) { stage = 0; phase ^= 1u; }
        }
    }
    __syncthreads();
}

}  // namespace

cudaError_t launch_breed(const BreedArgs& a, const float* parents, const int32_t* par1, const int32_t* par2,
                         const int32_t* kind, float* children, unsigned int* status, cudaStream_t stream)
{
    const int32_t chunks = static_cast<int32_t>((a.c_pad + kChunk - 1) / kChunk);
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(breed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(kBreedSmemBytes));
    if (err != cudaSuccess) return err;
    const int64_t items = static_cast<int64_t>(a.pop) * chunks;
    const int grid = static_cast<int>(items < sms ? items : sms);
    breed_kernel<<<grid, kBreedThreads, kBreedSmemBytes, stream>>>(a, chunks, parents, par1, par2, kind, children,
                                                                 status);
    return cudaGetLastError();
}

}  // namespace leea
