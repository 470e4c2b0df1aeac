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
// A consumer thread owns blocks of four consecutive genes, which is exactly
// one Philox block of each per-gene stream.  Normals are only generated for
// blocks in which some gene is masked for mutation.  Every mbarrier wait is
// bounded in time; on expiry the kernel sets kStatusBreedTimeout and exits.
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

// The four child genes of block q (genes 4q .. 4q+3).
__device__ __forceinline__ float4 breed_block(const BreedArgs& a, int32_t kind, uint32_t j, uint32_t q, float4 va,
                                              float4 vb)
{
    float v[4] = { va.x, va.y, va.z, va.w };
    if (kind == 1) {
        const float w2[4] = { vb.x, vb.y, vb.z, vb.w };
        if (a.xo_op == 0) {
            const uint4 r = stream_block(a.seed, kTagXo, a.gen, j, q);
            const uint32_t rw[4] = { r.x, r.y, r.z, r.w };
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = hits(rw[k], a.thr_xo) ? w2[k] : v[k];
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = 0.5f * (v[k] + w2[k]);
        }
    } else if (kind == 2) {
        const uint4 r = stream_block(a.seed, kTagMutMask, a.gen, j, q);
        const bool m0 = hits(r.x, a.thr_mut), m1 = hits(r.y, a.thr_mut);
        const bool m2 = hits(r.z, a.thr_mut), m3 = hits(r.w, a.thr_mut);
        if (m0 | m1 | m2 | m3) {
            const uint4 n = stream_block(a.seed, kTagNormal, a.gen, j, q);
            if (m0 | m1) {
                const float2 z = box_muller(n.x, n.y);
                if (m0) v[0] = fmaf(a.sigma, z.x, v[0]);
                if (m1) v[1] = fmaf(a.sigma, z.y, v[1]);
            }
            if (m2 | m3) {
                const float2 z = box_muller(n.z, n.w);
                if (m2) v[2] = fmaf(a.sigma, z.x, v[2]);
                if (m3) v[3] = fmaf(a.sigma, z.y, v[3]);
            }
        }
    } else if (kind == kKindInvalid) {
        const float nan = __int_as_float(0x7FC00000);
        v[0] = v[1] = v[2] = v[3] = nan;
    }
    // Genes past c are padding and stay zero whatever the operator.
    const int64_t i0 = 4 * static_cast<int64_t>(q);
    if (i0 + 3 >= a.c) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k >= a.c) v[k] = 0.0f;
    }
    return make_float4(v[0], v[1], v[2], v[3]);
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
                const int32_t j = static_cast<int32_t>(it / chunks_per_child);
                const int32_t ck = static_cast<int32_t>(it - static_cast<int64_t>(j) * chunks_per_child);
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
#pragma unroll 2
            for (int t = ct; t < nq; t += 32 * kConsumerWarps) {
                const float4 va = (m.kind >= 0) ? A[t] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 vb = (m.kind == 1) ? B[t] : va;
                O[t] = breed_block(a, m.kind, static_cast<uint32_t>(m.j), q0 + static_cast<uint32_t>(t), va, vb);
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
