// leea_probe_tc.cu -- the surrogate form's fused breed + probe pass with the
// child's first layer on the tensor cores: for each recipe (a virtual
// offspring: kind, parents and the Philox entity whose streams make its
// genes, Section 3.2's operators) the child's genes are regenerated from the
// parents and never written to global memory; W1 goes to shared memory in
// BF16 (round to nearest even, as the precision form evaluates children) and
// meets the probe inputs in a tcgen05 MMA with FP32 accumulation; b1, W2, b2
// stay FP32 for layer 2 on the CUDA cores.  Descriptor row:
//   [f_adj of parent 1, f_adj of parent 2, f_inh, crossover fraction,
//    mutation step length sigma ||z (.) m||, probe logits (n_probe x d_out)].
//
// The probe inputs enter as two BF16 pieces x = x_hi + x_lo (x_lo rounds the
// exact remainder), so they carry 16 significant bits: the MMA is
// D[o][s] = sum_k W1[o][k] x_hi[s][k] (columns s < 32) and the same with x_lo
// (columns 32 + s), one instruction of N = 64, summed in the epilogue.
//
// Persistent CTA (one per SM), recipes strided by gridDim.x.  Warp roles:
//   warps 0-15   producers: the child's genes, 8 per lane and Philox block,
//                for one 64-input K block of W1 at a time (128 rows x 128 B
//                in the 128-byte swizzled K-major layout, rows >= h unused),
//                then b1, W2, b2 into a tail buffer, and per-thread crossover
//                hits and sums of z^2 for the descriptor
//   warp 16      TMEM allocation; one thread issues the MMAs
//   warps 17-20  stage the probe pieces once; then per recipe the epilogue:
//                accumulator (TMEM lane = hidden unit) + b1, ReLU into shared
//                memory, layer 2 in FP32, the descriptor row
// Accumulators and tail buffers are double-buffered, so a recipe's epilogue
// overlaps the next recipe's genes and MMAs.  Mutation normals are computed
// only for Box-Muller pairs that hold a masked gene, gathered per warp into a
// shared-memory job list.  Every mbarrier wait is bounded in time; on expiry
// the kernel sets kStatusProbeTimeout, drains its MMAs and exits.
#include <cuda_bf16.h>

#include "leea_internal.h"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr uint32_t kTagXo = 3, kTagMutMask = 4, kTagNormal = 5;
constexpr int kProducerWarps = 16;
constexpr int kPT = 32 * kProducerWarps;         // producer threads
constexpr int kMmaWarp = kProducerWarps;
constexpr int kFirstEpiWarp = kProducerWarps + 1;
constexpr int kTcThreads = 32 * (kProducerWarps + 5);
constexpr int kKB = 64;                          // inputs per K block: 128 B of BF16
constexpr int kStages = 4;
constexpr int kMaxProbeTc = 32;
constexpr int kMaxHiddenTc = 128;
constexpr int kN = 2 * kMaxProbeTc;              // MMA N: x_hi samples, then x_lo samples
constexpr uint32_t kStageBytes = 128u * 128u;    // M = 128 rows of 128 B
constexpr uint32_t kXBlockBytes = kN * 128u;     // one K block of the probe pieces
constexpr uint32_t kTmemCols = 2 * kN;           // two accumulators
constexpr int kJobSlots = 4 * 32;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct TcSmem {
    uint8_t* ring;       // kStages x kStageBytes (1024-aligned)
    uint8_t* xb;         // n_kb x kXBlockBytes (1024-aligned)
    float* tail;         // 2 x tail_len: b1 [h], W2 [d_out][h], b2 [d_out]
    float* hs;           // [kMaxProbeTc][h + 1]: hidden activations
    uint32_t* part_hits; // 2 x kPT
    float* part_zz;      // 2 x kPT
    float2* job_z;       // kProducerWarps x kJobSlots
    uint8_t* job_code;   // kProducerWarps x kJobSlots: owner lane << 2 | pair slot
    uint32_t* lane_gene; // kProducerWarps x 32: first gene of each lane's unit
    uint64_t *full, *empty, *dfull, *dempty, *tfull, *tempty, *x_ready, *drain;
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
};

__host__ __device__ inline int32_t tc_n_kb(int32_t k) { return (k + kKB - 1) / kKB; }
__host__ __device__ inline int32_t tc_tail_len(int32_t h, int32_t d_out)
{
    return (h + d_out * h + d_out + 3) / 4 * 4;
}

__host__ __device__ inline size_t tc_smem_bytes(int32_t k, int32_t h, int32_t d_out)
{
    return 1024 + static_cast<size_t>(kStages) * kStageBytes + static_cast<size_t>(tc_n_kb(k)) * kXBlockBytes +
           sizeof(float) * (2 * static_cast<size_t>(tc_tail_len(h, d_out)) + kMaxProbeTc * (h + 1)) +
           2 * kPT * (sizeof(uint32_t) + sizeof(float)) +
           kProducerWarps * (kJobSlots * (sizeof(float2) + 1) + 32 * sizeof(uint32_t)) +
           8 * (2 * kStages + 8 + 2) + 64;
}

__device__ __forceinline__ TcSmem carve(uint8_t* raw, const ProbeArgs& a)
{
    TcSmem s;
    uint8_t* p = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    s.ring = p;
    p += kStages * kStageBytes;
    s.xb = p;
    p += tc_n_kb(a.k) * kXBlockBytes;
    s.tail = reinterpret_cast<float*>(p);
    p += sizeof(float) * 2 * tc_tail_len(a.h, a.d_out);
    s.hs = reinterpret_cast<float*>(p);
    p += sizeof(float) * kMaxProbeTc * (a.h + 1);
    s.part_hits = reinterpret_cast<uint32_t*>(p);
    p += sizeof(uint32_t) * 2 * kPT;
    s.part_zz = reinterpret_cast<float*>(p);
    p += sizeof(float) * 2 * kPT;
    s.job_z = reinterpret_cast<float2*>(p);
    p += sizeof(float2) * kProducerWarps * kJobSlots;
    s.lane_gene = reinterpret_cast<uint32_t*>(p);
    p += sizeof(uint32_t) * kProducerWarps * 32;
    s.job_code = p;
    p += kProducerWarps * kJobSlots;
    p += (8u - (ptx::smem_u32(p) & 7u)) & 7u;
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.empty = bars + kStages;
    s.dfull = bars + 2 * kStages;
    s.dempty = s.dfull + 2;
    s.tfull = s.dfull + 4;
    s.tempty = s.dfull + 6;
    s.x_ready = s.dfull + 8;
    s.drain = s.dfull + 9;
    uint32_t* w = reinterpret_cast<uint32_t*>(s.dfull + 10);
    s.tmem_holder = w;
    s.abort_flag = reinterpret_cast<volatile int*>(w + 1);
    s.ep_go = reinterpret_cast<int*>(w + 2);
    return s;
}

__device__ __forceinline__ void raise_abort(const TcSmem& s, unsigned int* status)
{
    *s.abort_flag = 1;
    atomicOr(status, kStatusProbeTimeout);
}

// Bit t of the result: the 16-bit draw t (t = 0..7) of block r is below thr.
__device__ __forceinline__ uint32_t mask8(const uint4& r, uint32_t thr)
{
    const uint32_t w[4] = { r.x, r.y, r.z, r.w };
    uint32_t m = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const uint32_t u = (t & 1) ? (w[t >> 1] >> 16) : (w[t >> 1] & 0xFFFFu);
        m |= (u < thr ? 1u : 0u) << t;
    }
    return m;
}

__device__ __forceinline__ void prefetch_l2(const float* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<uint64_t>(p)));
}

// Prefetches into L2 the parent genes of this thread's units of K block kb
// (the producers' loads then wait on L2, not on HBM).
__device__ __forceinline__ void prefetch_kb(const ProbeArgs& a, int kb, const float* pa, const float* pb, bool two,
                                            int pt)
{
    const int kw = a.k - kb * kKB < kKB ? a.k - kb * kKB : kKB;
    for (int u = pt; u < 8 * a.h; u += kPT) {
        const int o = u >> 3, jc = u & 7;
        if (8 * jc < kw) {
            const int64_t i = static_cast<int64_t>(o) * a.k + kb * kKB + 8 * jc;
            prefetch_l2(pa + i);
            if (two) prefetch_l2(pb + i);
        }
    }
}

__device__ __forceinline__ uint32_t bf162_bits(__nv_bfloat162 v)
{
    return *reinterpret_cast<uint32_t*>(&v);
}

// Genes i .. i+7 (i % 8 == 0) of the child of a recipe of kind `kind`
// (1 crossover, 2 mutation, else a copy of parent 1), warp-collective: every
// lane of the warp calls it, `live` marks lanes with a unit.  Adds the unit's
// crossover hits and sum of z^2 over masked genes below c to hits and zz.
__device__ __forceinline__ void child8(const ProbeArgs& a, const PhiloxKeys& key, int32_t kind, uint32_t ent,
                                       const float* __restrict__ pa, const float* __restrict__ pb, uint32_t i,
                                       bool live, float (&v)[8], uint32_t& hits, float& zz, int lane, float2* job_z,
                                       uint8_t* job_code, uint32_t* lane_gene)
{
    if (live) {
        const float4 a0 = __ldg(reinterpret_cast<const float4*>(pa + i));
        const float4 a1 = __ldg(reinterpret_cast<const float4*>(pa + i + 4));
        v[0] = a0.x; v[1] = a0.y; v[2] = a0.z; v[3] = a0.w;
        v[4] = a1.x; v[5] = a1.y; v[6] = a1.z; v[7] = a1.w;
    } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = 0.0f;
    }
    const int64_t left = a.c - static_cast<int64_t>(i);  // genes of this unit below c
    const uint32_t in_c = !live ? 0u : (left >= 8 ? 0xFFu : (left > 0 ? ((1u << left) - 1u) : 0u));
    if (kind == 1) {
        if (!live) return;
        const float4 b0 = __ldg(reinterpret_cast<const float4*>(pb + i));
        const float4 b1 = __ldg(reinterpret_cast<const float4*>(pb + i + 4));
        const float w[8] = { b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w };
        if (a.xo_op == 0) {
            const uint32_t m = mask8(philox_keyed(make_uint4(i >> 3, ent, a.gen, kTagXo), key), a.thr_xo);
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = ((m >> t) & 1u) ? w[t] : v[t];
            hits += __popc(m & in_c);
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = 0.5f * (v[t] + w[t]);
        }
    } else if (kind == 2) {
        // Slot sl = Box-Muller pair (i + 2 sl, i + 2 sl + 1): words (0,1) or
        // (2,3) of NORMAL block (i + 2 sl) >> 2.  The warp lists the needed
        // slots (one ballot per slot), consecutive lanes compute them.
        uint32_t hit = 0;
        if (live) hit = mask8(philox_keyed(make_uint4(i >> 3, ent, a.gen, kTagMutMask), key), a.thr_mut);
        lane_gene[lane] = i;
        const uint32_t lt = (1u << lane) - 1u;
        uint32_t idx[4], total = 0;
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            const bool need = ((hit >> (2 * sl)) & 3u) != 0u;
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, need);
            idx[sl] = total + __popc(b & lt);
            if (need) job_code[idx[sl]] = static_cast<uint8_t>((lane << 2) | sl);
            total += __popc(b);
        }
        __syncwarp();
        for (uint32_t job = static_cast<uint32_t>(lane); job < total; job += 32) {
            const uint32_t code = job_code[job];
            const uint32_t g = lane_gene[code >> 2] + 2u * (code & 3u);  // even gene of the pair
            const uint4 n = philox_keyed(make_uint4(g >> 2, ent, a.gen, kTagNormal), key);
            job_z[job] = (g & 2u) ? box_muller(n.z, n.w) : box_muller(n.x, n.y);
        }
        __syncwarp();
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            if ((hit >> (2 * sl)) & 3u) {
                const float2 z = job_z[idx[sl]];
                if ((hit >> (2 * sl)) & 1u) {
                    v[2 * sl] = fmaf(a.sigma, z.x, v[2 * sl]);
                    if ((in_c >> (2 * sl)) & 1u) zz = fmaf(z.x, z.x, zz);
                }
                if ((hit >> (2 * sl + 1)) & 1u) {
                    v[2 * sl + 1] = fmaf(a.sigma, z.y, v[2 * sl + 1]);
                    if ((in_c >> (2 * sl + 1)) & 1u) zz = fmaf(z.y, z.y, zz);
                }
            }
        }
        __syncwarp();  // the list is reused by the next unit
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
probe_tc_kernel(const __grid_constant__ ProbeArgs a, int32_t n)
{
    extern __shared__ uint8_t smem_raw[];
    const TcSmem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_kb = tc_n_kb(a.k);
    const int tail_len = tc_tail_len(a.h, a.d_out);

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            ptx::mbar_init(&s.full[i], kProducerWarps);
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.dfull[i], 1);
            ptx::mbar_init(&s.dempty[i], 128);
            ptx::mbar_init(&s.tfull[i], kProducerWarps);
            ptx::mbar_init(&s.tempty[i], 128);
        }
        ptx::mbar_init(s.x_ready, 128);
        ptx::mbar_init(s.drain, 1);
        *s.abort_flag = 0;
        *s.ep_go = 0;
        ptx::fence_mbar_init();
    }
    if (warp == kMmaWarp) ptx::tmem_alloc(s.tmem_holder, kTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *s.tmem_holder;

    if (warp < kProducerWarps) {
        // ------------------------------------------------------------ producers
        const int pt = threadIdx.x;
        float2* job_z = s.job_z + warp * kJobSlots;
        uint8_t* job_code = s.job_code + warp * kJobSlots;
        uint32_t* lane_gene = s.lane_gene + warp * 32;
        const PhiloxKeys key = philox_keys(a.seed);
        const int units_kb = 8 * a.h;  // units of one K block (a multiple of 128)
        const uint32_t t0 = static_cast<uint32_t>(a.h) * static_cast<uint32_t>(a.k) / 8u;  // first tail unit
        const int n_tail = static_cast<int>((a.c + 7) / 8 - t0);
        uint32_t stage = 0, phase = 0;
        bool ok = true;
        int q = 0;
        for (int r = blockIdx.x; ok && r < n; r += gridDim.x, ++q) {
            const int32_t kind = a.kind[r];
            const uint32_t ent = a.entity ? a.entity[r] : static_cast<uint32_t>(r);
            const float* pa = a.parents + static_cast<int64_t>(a.par1[r]) * a.c_pad;
            const float* pb = a.parents + static_cast<int64_t>(a.par2[r]) * a.c_pad;
            uint32_t hits = 0;
            float zz = 0.0f;
            if (q == 0) {
                prefetch_kb(a, 0, pa, pb, kind == 1, pt);
                if (n_kb > 1) prefetch_kb(a, 1, pa, pb, kind == 1, pt);
            }
            for (int kb = 0; kb < n_kb; ++kb) {
                if (kb + 2 < n_kb) prefetch_kb(a, kb + 2, pa, pb, kind == 1, pt);
                if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a.status);
                    ok = false;
                    break;
                }
                uint8_t* sb = s.ring + stage * kStageBytes;
                const int kw = a.k - kb * kKB < kKB ? a.k - kb * kKB : kKB;  // a multiple of 16
                for (int u = pt; u < units_kb; u += kPT) {
                    const int o = u >> 3, jc = u & 7;
                    const bool live = 8 * jc < kw;
                    float v[8];
                    child8(a, key, kind, ent, pa, pb, static_cast<uint32_t>(o * a.k + kb * kKB + 8 * jc), live, v,
                           hits, zz, lane, job_z, job_code, lane_gene);
                    if (live) {
                        uint4 w;
                        w.x = bf162_bits(__floats2bfloat162_rn(v[0], v[1]));
                        w.y = bf162_bits(__floats2bfloat162_rn(v[2], v[3]));
                        w.z = bf162_bits(__floats2bfloat162_rn(v[4], v[5]));
                        w.w = bf162_bits(__floats2bfloat162_rn(v[6], v[7]));
                        *reinterpret_cast<uint4*>(sb + o * 128 + ((jc ^ (o & 7)) << 4)) = w;
                    }
                }
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&s.full[stage]);
                if (++stage == kStages) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            const int rn = r + gridDim.x;  // the next recipe's first K blocks
            if (rn < n) {
                const int32_t kn = a.kind[rn];
                const float* pan = a.parents + static_cast<int64_t>(a.par1[rn]) * a.c_pad;
                const float* pbn = a.parents + static_cast<int64_t>(a.par2[rn]) * a.c_pad;
                prefetch_kb(a, 0, pan, pbn, kn == 1, pt);
                if (n_kb > 1) prefetch_kb(a, 1, pan, pbn, kn == 1, pt);
            }
            // b1, W2, b2 (genes h k .. c - 1) into tail buffer q & 1
            const uint32_t tb = static_cast<uint32_t>(q) & 1u, tpar = (static_cast<uint32_t>(q) >> 1) & 1u;
            if (!ptx::mbar_wait_bounded(&s.tempty[tb], tpar ^ 1u, s.abort_flag, kWaitLimitNs)) {
                raise_abort(s, a.status);
                break;
            }
            float* tail = s.tail + tb * tail_len;
            for (int base = 0; base < n_tail; base += kPT) {
                const int u = base + pt;
                const bool live = u < n_tail;
                float v[8];
                child8(a, key, kind, ent, pa, pb, 8u * (t0 + static_cast<uint32_t>(live ? u : 0)), live, v, hits,
                       zz, lane, job_z, job_code, lane_gene);
                if (live) {
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        if (8 * u + t < tail_len) tail[8 * u + t] = v[t];
                }
            }
            s.part_hits[tb * kPT + pt] = hits;
            s.part_zz[tb * kPT + pt] = zz;
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.tfull[tb]);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_bf16(128, kN);
            bool ok = ptx::mbar_wait_bounded(s.x_ready, 0u, s.abort_flag, kWaitLimitNs);
            if (!ok) raise_abort(s, a.status);
            ptx::tc_fence_after();
            const uint32_t ring = ptx::smem_u32(s.ring), xb = ptx::smem_u32(s.xb);
            uint32_t stage = 0, phase = 0;
            int q = 0;
            for (int r = blockIdx.x; ok && r < n; r += gridDim.x, ++q) {
                const uint32_t db = static_cast<uint32_t>(q) & 1u, dpar = (static_cast<uint32_t>(q) >> 1) & 1u;
                if (!ptx::mbar_wait_bounded(&s.dempty[db], dpar ^ 1u, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a.status);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d_tmem = tmem_base + db * kN;
                for (int kb = 0; kb < n_kb; ++kb) {
                    if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a.status);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const int kw = a.k - kb * kKB < kKB ? a.k - kb * kKB : kKB;
                    for (int kk = 0; kk < kw / 16; ++kk) {
                        const uint64_t ad = ptx::smem_desc_sw128(ring + stage * kStageBytes + kk * 32u);
                        const uint64_t bd = ptx::smem_desc_sw128(xb + kb * kXBlockBytes + kk * 32u);
                        ptx::mma_f16(d_tmem, ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
                    }
                    ptx::mma_commit(&s.empty[stage]);
                    if (++stage == kStages) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                ptx::mma_commit(&s.dfull[db]);
            }
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kWaitLimitNs : kDrainLimitNs);
        }
    } else {
        // ------------------------------------------------------------ probe pieces, then epilogue
        const int et = threadIdx.x - 32 * kFirstEpiWarp;
        // Row rr of the B operand: sample rr & 31, piece rr >> 5 (hi, lo); K
        // block kb, 16-byte chunk c at chunk position c ^ (rr & 7).
        for (int e = et; e < kN * n_kb * 8; e += 128) {
            const int rr = e / (n_kb * 8), rest = e - rr * (n_kb * 8), kb = rest >> 3, c = rest & 7;
            const int smp = rr & 31, piece = rr >> 5;
            uint32_t wd[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                float f[2];
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int kk = kb * kKB + 8 * c + 2 * t + h2;
                    const float x = (smp < a.n_probe && kk < a.k) ? a.probe[static_cast<int64_t>(smp) * a.k + kk] : 0.0f;
                    const float hi = __bfloat162float(__float2bfloat16_rn(x));
                    f[h2] = piece == 0 ? hi : x - hi;  // the remainder is exact in FP32
                }
                wd[t] = bf162_bits(__floats2bfloat162_rn(f[0], f[1]));
            }
            *reinterpret_cast<uint4*>(s.xb + kb * kXBlockBytes + rr * 128 + ((c ^ (rr & 7)) << 4)) =
                make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
        ptx::fence_proxy_async_smem();
        ptx::mbar_arrive(s.x_ready);

        const int qd = warp & 3;                  // TMEM lane quarter
        const int o = qd * 32 + lane;             // hidden unit = accumulator row
        const uint32_t lane_addr = static_cast<uint32_t>(qd * 32) << 16;
        const int hp = a.h + 1;
        int q = 0;
        for (int r = blockIdx.x; r < n; r += gridDim.x, ++q) {
            const uint32_t db = static_cast<uint32_t>(q) & 1u, dpar = (static_cast<uint32_t>(q) >> 1) & 1u;
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(&s.dfull[db], dpar, s.abort_flag, kWaitLimitNs) &&
                                 ptx::mbar_wait_bounded(&s.tfull[db], dpar, s.abort_flag, kWaitLimitNs);
                if (!got) raise_abort(s, a.status);
                *s.ep_go = got ? 1 : 0;
            }
            ptx::named_barrier_sync(1, 128);  // accumulator and tail ready (or abort)
            if (!*s.ep_go) break;
            ptx::tc_fence_after();
            uint32_t d[kN];
#pragma unroll
            for (int c0 = 0; c0 < kN; c0 += 16)
                ptx::tmem_ld16_nowait(tmem_base + lane_addr + db * kN + static_cast<uint32_t>(c0), d + c0);
            ptx::tmem_ld_wait();
            ptx::tc_fence_before();
            ptx::mbar_arrive(&s.dempty[db]);
            const float* tail = s.tail + db * tail_len;
            if (o < a.h) {
                const float b1 = tail[o];
#pragma unroll
                for (int smp = 0; smp < kMaxProbeTc; ++smp)
                    if (smp < a.n_probe)
                        s.hs[smp * hp + o] =
                            fmaxf(__uint_as_float(d[smp]) + __uint_as_float(d[kMaxProbeTc + smp]) + b1, 0.0f);
            }
            ptx::named_barrier_sync(1, 128);  // hidden activations complete
            float* row = a.desc + static_cast<int64_t>(r) * a.width;
            const float* w2 = tail + a.h;
            for (int e = et; e < a.n_probe * a.d_out; e += 128) {
                const int smp = e / a.d_out, cl = e - smp * a.d_out;
                float z = w2[a.d_out * a.h + cl];  // b2
                const float* wr = w2 + cl * a.h;
                const float* hr = s.hs + smp * hp;
                for (int oo = 0; oo < a.h; ++oo) z = fmaf(wr[oo], hr[oo], z);
                row[5 + e] = z;
            }
            if (et == 0) {
                float hsum = 0.0f, zsum = 0.0f;  // fixed order over the producer threads
                for (int t = 0; t < kPT; ++t) {
                    hsum += static_cast<float>(s.part_hits[db * kPT + t]);
                    zsum += s.part_zz[db * kPT + t];
                }
                const int32_t kind = a.kind[r];
                row[0] = a.f_adj[a.par1[r]];
                row[1] = a.f_adj[a.par2[r]];
                row[2] = a.f_inh[r];
                row[3] = kind == 1 ? (a.xo_op == 0 ? hsum / static_cast<float>(a.c) : 0.5f) : 0.0f;
                row[4] = kind == 2 ? a.sigma * sqrtf(zsum) : 0.0f;
            }
            ptx::named_barrier_sync(1, 128);  // tail, activations and partials read
            ptx::mbar_arrive(&s.tempty[db]);
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, kTmemCols);
    }
}

}  // namespace

bool probe_tc_supported(int32_t k, int32_t h, int32_t d_out, int32_t n_probe)
{
    return k % 16 == 0 && h % 16 == 0 && h >= 16 && h <= kMaxHiddenTc && d_out >= 1 && d_out <= 16 &&
           n_probe >= 1 && n_probe <= kMaxProbeTc && tc_smem_bytes(k, h, d_out) <= 227u * 1024u;
}

cudaError_t launch_descriptors_tc(const ProbeArgs& a, int32_t n_recipes, cudaStream_t stream)
{
    if (n_recipes <= 0) return cudaSuccess;
    if (!probe_tc_supported(a.k, a.h, a.d_out, a.n_probe) || !a.status) return cudaErrorInvalidValue;
    const size_t smem = tc_smem_bytes(a.k, a.h, a.d_out);
    cudaError_t err = cudaFuncSetAttribute(probe_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    const int grid = n_recipes < sms ? n_recipes : sms;
    probe_tc_kernel<<<grid, kTcThreads, smem, stream>>>(a, n_recipes);
    return cudaGetLastError();
}

}  // namespace leea
