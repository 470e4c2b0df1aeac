// leea_eval_u8.cu -- fitness of every individual (Eq. 1; Section 3.3) for
// minibatches of 8-bit image levels, x = k / x_div with k in [0, 255] (MNIST's
// encoding), on the tcgen05 tensor cores with FP32-class accuracy.
//
// Numerics.  The integers k are exact in FP16, and every FP32 weight, scaled
// by 2^8, is split into two FP16 pieces: w1 = fp16(2^8 w) and
// w2 = fp16(2^8 w - w1), with the remainder exact in FP32.  So
// |2^8 w - w1 - w2| <= max(2^-22 2^8 |w|, 2^-25): a 22-bit significand
// against FP32's 24, and D = K (w1 + w2)^T is formed from exact products; only
// the FP32 accumulation in the tensor core rounds.  The epilogue scales by
// 2^-8 / x_div.  An individual with a weight |w| >= 128 (its scaled w1 could
// overflow FP16) is flagged by the converters, and the epilogue forms its
// layer 1 with FP32 FFMA from global memory instead of the accumulator.
//
// Shape.  A tcgen05.mma of M = 128 and K = 16 costs about the same time for any
// N up to 256, so two individuals share every MMA: the batch tile (<= 128
// samples, the M side) is the A operand and the stacked W1 pieces of two
// individuals (N = 2h) the B operand, and 2 x 49 MMAs evaluate a pair at
// d_0 = 784.  The batch, staged once per evaluation as FP16 in global memory
// (stage_x16_kernel; it stays in L2), arrives by TMA in 32-input tiles next to
// the weights.
//
// Pipeline (persistent CTA, one per SM; each CTA takes a contiguous range of
// individuals, as pairs, the last one alone when the range is odd):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      producer: per stage, one TMA of the batch tile (128 x 32
//               FP16, 64-byte swizzle, from L2) and one TMA per individual of
//               its FP32 W1 slice (h x 32); per unit, b1/W2/b2 by one bulk
//               copy per individual
//   warps 2-9   converters: each 8-row group of a raw FP32 slice (1 KB) is
//               read by one warp and overwritten in place by its two FP16
//               pieces in the 64-byte swizzled K-major layout (piece q at
//               +512 bytes, so the pieces of all 2h rows form two operands
//               with 8-row groups 1 KB apart); a warp reads all its groups of
//               the stage before it writes any.  (Measured with no compute:
//               tile loads of these 32-input slices stream the population at
//               4.5 TB/s; 128-bit loads from many threads at 5.1-5.5 TB/s but
//               only with 64-128 KB in flight per SM, more registers than this
//               kernel has; cp.async into the ring at 4.1-4.8 TB/s.)
//   warps 10-17 epilogue, 4 warps (one per TMEM lane quarter = 32 samples)
//               per individual: bias, ReLU, layer 2 (W2 staged transposed in
//               shared memory), softmax cross-entropy, fixed-order batch sum,
//               inheritance blend; accumulators are double-buffered in TMEM
//               (columns 0 and 256), so a pair's epilogue overlaps the next
//               pair's MMAs
// Every mbarrier wait is bounded in time; on expiry the kernel sets
// kStatusEvalTimeout, lets its copies and MMAs in flight finish and exits.
#include <cuda.h>

#include <algorithm>
#include <cuda_fp16.h>

#include "leea_internal.h"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kConvWarps = 8;
constexpr int kFirstConvWarp = 2;
constexpr int kGroupsPerWarp = 4;           // 8-row groups per converter warp and stage: 2 x 128 rows / 8 / 8
constexpr int kFirstEpiWarp = kFirstConvWarp + kConvWarps;
constexpr int kEpiWarps = 8;
constexpr int kU8Threads = 32 * (kFirstEpiWarp + kEpiWarps);
constexpr int kKStage = 32;             // K elements per stage: 128-byte FP32 rows, 64-byte FP16 rows
constexpr uint32_t kATileBytes = 128u * 64u;  // batch tile: 128 samples x 32 levels as FP16
constexpr int kMinStages = 3;
constexpr int kMaxStages = 6;
constexpr int kMaxOutU8 = 16;
constexpr int kFlagSlots = 16;          // unit-tagged range flags; converters run at most a few units ahead
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;    // the two accumulators: columns 0 and 256
constexpr float kPieceScale = 256.0f;   // 2^8: weights enter the pieces as 2^8 w
constexpr float kPieceRange = 128.0f;   // |w| below this: 2^8 |w| < 2^15, finite in FP16
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct EvalU8Args {
    int32_t pop, k, h, d_out, dpad, batch, k16, k_stages, n_stages;
    int32_t per_cta, extra;  // individuals per CTA: per_cta, one more for the first `extra` CTAs
    uint32_t prm_bytes;      // b1, W2, b2 of one individual, rounded up to 16 bytes
    uint32_t slot_bytes;     // one individual's slice of a stage: h rows x 128 bytes (FP32, then its two FP16 pieces)
    uint32_t stage_bytes;    // two slots and the batch tile
    int64_t c_pad;
    float inv_div, alpha;
    const float* popv;
    const uint8_t* x;        // the levels, for the FP32 fallback
    const int32_t* y;
    const float* f_inh;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    unsigned int* status;
};

struct U8Smem {
    uint8_t* ring;       // n_stages x stage_bytes, 1024-aligned: W1 slices (raw, then pieces), then the batch tile
    uint8_t* prm_raw;    // [2 buffers][2 slots] x prm_bytes: b1, W2 (row-major), b2 as stored
    float* w2t;          // [2 slots][h][dpad]
    float* b1;           // [2 slots][h]
    float* b2;           // [2 slots][16]
    float* red_loss;     // [2 slots][4 quarters]
    int32_t* red_ok;     // [2 slots][4 quarters]
    uint32_t* flag;      // [kFlagSlots][2]: u + 1 if unit u's individual in that slot has |w| >= 128
    uint32_t* accflag;   // [2]: the flags of the unit in that accumulator, for the epilogue
    int* ep_go;          // [2 slots][2]: the epilogue groups' go words (parameters, accumulator)
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    uint64_t *full, *a_full, *empty, *prm_full, *prm_empty, *acc_full, *acc_empty, *drain;
};

__host__ __device__ inline size_t u8_tail_bytes(int32_t h, int32_t dpad, uint32_t prm_bytes, int32_t n_stages)
{
    return 4u * static_cast<size_t>(prm_bytes) + sizeof(float) * (2u * h * dpad + 2u * h + 32u + 8u) +
           sizeof(int32_t) * 8u + sizeof(uint32_t) * (2u * kFlagSlots + 2u) + sizeof(int) * 4u + 16u +
           8u * (3u * n_stages + 9u) + 64u;
}

__device__ __forceinline__ U8Smem carve(uint8_t* raw, const EvalU8Args& a)
{
    U8Smem s;
    s.ring = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    uint8_t* p = s.ring + static_cast<size_t>(a.n_stages) * a.stage_bytes;
    s.prm_raw = p;
    p += 4u * a.prm_bytes;
    s.w2t = reinterpret_cast<float*>(p);
    p += sizeof(float) * 2 * a.h * a.dpad;
    s.b1 = reinterpret_cast<float*>(p);
    p += sizeof(float) * 2 * a.h;
    s.b2 = reinterpret_cast<float*>(p);
    p += sizeof(float) * 32;
    s.red_loss = reinterpret_cast<float*>(p);
    p += sizeof(float) * 8;
    s.red_ok = reinterpret_cast<int32_t*>(p);
    p += sizeof(int32_t) * 8;
    s.flag = reinterpret_cast<uint32_t*>(p);
    p += sizeof(uint32_t) * 2 * kFlagSlots;
    s.accflag = reinterpret_cast<uint32_t*>(p);
    p += sizeof(uint32_t) * 2;
    s.ep_go = reinterpret_cast<int*>(p);
    p += sizeof(int) * 4;
    s.tmem_holder = reinterpret_cast<uint32_t*>(p);
    s.abort_flag = reinterpret_cast<volatile int*>(p + 4);
    p += 16;
    p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 7u) & ~uintptr_t(7));
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.a_full = bars + a.n_stages;
    s.empty = bars + 2 * a.n_stages;
    s.prm_full = bars + 3 * a.n_stages;
    s.prm_empty = s.prm_full + 2;
    s.acc_full = s.prm_empty + 2;
    s.acc_empty = s.acc_full + 2;
    s.drain = s.acc_empty + 2;
    return s;
}

uint32_t u8_prm_bytes(int32_t h, int32_t d_out)
{
    return (static_cast<uint32_t>(h + d_out * h + d_out) * 4u + 15u) & ~15u;
}

uint32_t u8_stage_bytes(int32_t h)
{
    return 2u * static_cast<uint32_t>(h) * 128u + kATileBytes;
}

size_t u8_smem_bytes(int32_t h, int32_t d_out, int32_t n_stages)
{
    const int32_t dpad = (d_out + 3) / 4 * 4;
    return 1024 + static_cast<size_t>(n_stages) * u8_stage_bytes(h) +
           u8_tail_bytes(h, dpad, u8_prm_bytes(h, d_out), n_stages);
}

// The deepest ring that fits in 227 KB of shared memory; 0 if not even kMinStages do.
int32_t u8_stages(int32_t h, int32_t d_out)
{
    for (int32_t ns = kMaxStages; ns >= kMinStages; --ns)
        if (u8_smem_bytes(h, d_out, ns) <= 227u * 1024u) return ns;
    return 0;
}

__device__ __forceinline__ void raise_abort(const U8Smem& s, const EvalU8Args& a)
{
    *s.abort_flag = 1;
    atomicOr(a.status, kStatusEvalTimeout);
}

__device__ __forceinline__ uint32_t half2_bits(__half2 v)
{
    return *reinterpret_cast<uint32_t*>(&v);
}

// Two FP32 weights (lower K index in the low half) as packed FP16 pieces of
// 2^8 w: p1 rounds 2^8 w to nearest, p2 rounds the remainder, which is exact
// in FP32.
__device__ __forceinline__ void split2x2(float w0, float w1, uint32_t& p1, uint32_t& p2)
{
    const float s0 = w0 * kPieceScale, s1 = w1 * kPieceScale;
    const __half2 h1 = __floats2half2_rn(s0, s1);
    const float2 f1 = __half22float2(h1);
    p1 = half2_bits(h1);
    p2 = half2_bits(__floats2half2_rn(s0 - f1.x, s1 - f1.y));
}

__device__ __forceinline__ bool out_of_piece_range(const float4& v)
{
    return fabsf(v.x) >= kPieceRange || fabsf(v.y) >= kPieceRange || fabsf(v.z) >= kPieceRange ||
           fabsf(v.w) >= kPieceRange;
}

// Four weights of row r (0..7) of an 8-row group, K offset 4 c8 within the
// stage, as FP16 pieces at their 64-byte-swizzle positions: piece q of the
// group occupies bytes 512 q .. 512 q + 511 of the group.
__device__ __forceinline__ void put_pieces(uint8_t* group, int r, int c8, const float4& f)
{
    uint32_t lo[2], hi[2];
    split2x2(f.x, f.y, lo[0], lo[1]);
    split2x2(f.z, f.w, hi[0], hi[1]);
    const uint32_t off = static_cast<uint32_t>(r) * 64u +
                         ((static_cast<uint32_t>(c8 >> 1) ^ (static_cast<uint32_t>(r >> 1) & 3u)) << 4) +
                         (static_cast<uint32_t>(c8 & 1) << 3);
    *reinterpret_cast<uint2*>(group + off) = make_uint2(lo[0], hi[0]);
    *reinterpret_cast<uint2*>(group + 512 + off) = make_uint2(lo[1], hi[1]);
}

// This CTA's individuals: [first, first + count).
__device__ __forceinline__ void cta_range(const EvalU8Args& a, int& first, int& count)
{
    const int b = static_cast<int>(blockIdx.x);
    first = b * a.per_cta + min(b, a.extra);
    count = a.per_cta + (b < a.extra ? 1 : 0);
}

__global__ void __launch_bounds__(kU8Threads, 1)
eval_u8_kernel(const __grid_constant__ CUtensorMap tmap_w, const __grid_constant__ CUtensorMap tmap_x,
               const EvalU8Args a)
{
    extern __shared__ uint8_t smem_raw[];
    const U8Smem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int first = 0, count = 0;
    cta_range(a, first, count);
    const uint32_t a_off = 2u * a.slot_bytes;  // batch tile within a stage

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.n_stages; ++i) {
            ptx::mbar_init(&s.full[i], kConvWarps);  // converted
            ptx::mbar_init(&s.a_full[i], 1);         // the stage's tiles landed
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.prm_full[i], 1);
            ptx::mbar_init(&s.prm_empty[i], kEpiWarps);
            ptx::mbar_init(&s.acc_full[i], 2);  // the MMAs' commit and the issuer's flag hand-over
            ptx::mbar_init(&s.acc_empty[i], kEpiWarps);
        }
        ptx::mbar_init(s.drain, 1);
        ptx::tma_prefetch_map(&tmap_w);
        ptx::tma_prefetch_map(&tmap_x);
        for (int i = 0; i < 2 * kFlagSlots; ++i) s.flag[i] = 0u;
        s.accflag[0] = s.accflag[1] = 0u;
        for (int i = 0; i < 4; ++i) s.ep_go[i] = 0;
        *s.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 0) ptx::tmem_alloc(s.tmem_holder, kTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *s.tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc1 = ptx::idesc_f16(128, static_cast<uint32_t>(a.h));
            const uint32_t idesc2 = ptx::idesc_f16(128, 2u * static_cast<uint32_t>(a.h));
            const uint32_t ring = ptx::smem_u32(s.ring);
            uint32_t stage = 0, phase = 0;
            bool ok = true;
            for (int u = 0; ok && 2 * u < count; ++u) {
                const int n = min(2, count - 2 * u);
                const uint32_t buf = static_cast<uint32_t>(u) & 1u;
                if (!ptx::mbar_wait_bounded(&s.acc_empty[buf], ((static_cast<uint32_t>(u) >> 1) & 1u) ^ 1u,
                                            s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + buf * kAccStride;
                const uint32_t idesc = n == 2 ? idesc2 : idesc1;
                for (int kc = 0; kc < a.k_stages; ++kc) {
                    if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t sb = ring + stage * a.stage_bytes;
#pragma unroll
                    for (int kk = 0; kk < kKStage / 16; ++kk) {
                        if (kc * kKStage + kk * 16 >= a.k16) break;
                        const uint64_t ad = ptx::smem_desc_sw64(sb + a_off + 32u * kk, 512u);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const uint64_t bd = ptx::smem_desc_sw64(sb + 512u * q + 32u * kk, 1024u);
                            ptx::mma_f16(d, ad, bd, idesc, (kc | kk | q) != 0 ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit(&s.empty[stage]);
                    if (++stage == static_cast<uint32_t>(a.n_stages)) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                ptx::mma_commit(&s.acc_full[buf]);
                // Every converter arrival of this unit was acquired above, so
                // its range flags are final; hand them to the epilogue with a
                // releasing arrival on the same barrier.
                const volatile uint32_t* fl = s.flag + 2 * (u % kFlagSlots);
                const uint32_t tag = static_cast<uint32_t>(u) + 1u;
                s.accflag[buf] = (fl[0] == tag ? 1u : 0u) | (fl[1] == tag ? 2u : 0u);
                ptx::mbar_arrive(&s.acc_full[buf]);
            }
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kWaitLimitNs : kDrainLimitNs);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            ptx::grid_dep_wait();  // the population (breeding) and the staged batch come from earlier kernels
            uint32_t stage = 0, phase = 0, issued_mask = 0, parity_mask = 0, prm_issued = 0;
            bool ok = true;
            for (int u = 0; ok && 2 * u < count; ++u) {
                const int n = min(2, count - 2 * u), p0 = first + 2 * u;
                const uint32_t pb = static_cast<uint32_t>(u) & 1u, pph = (static_cast<uint32_t>(u) >> 1) & 1u;
                if (!ptx::mbar_wait_bounded(&s.prm_empty[pb], pph ^ 1u, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                ptx::mbar_arrive_expect_tx(&s.prm_full[pb], static_cast<uint32_t>(n) * a.prm_bytes);
                for (int j = 0; j < n; ++j)
                    ptx::bulk_load(s.prm_raw + (2 * pb + j) * a.prm_bytes,
                                   a.popv + static_cast<int64_t>(p0 + j) * a.c_pad + static_cast<int64_t>(a.h) * a.k,
                                   a.prm_bytes, &s.prm_full[pb]);
                ++prm_issued;
                for (int kc = 0; kc < a.k_stages; ++kc) {
                    if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    uint8_t* sb = s.ring + stage * a.stage_bytes;
                    ptx::mbar_arrive_expect_tx(&s.a_full[stage], kATileBytes + static_cast<uint32_t>(n) * a.slot_bytes);
                    ptx::tma_load_2d(sb + a_off, &tmap_x, &s.a_full[stage], kc * kKStage, 0);
                    for (int j = 0; j < n; ++j)
                        ptx::tma_load_3d(sb + j * a.slot_bytes, &tmap_w, &s.a_full[stage], kc * kKStage, 0, p0 + j);
                    issued_mask |= 1u << stage;
                    parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                    if (++stage == static_cast<uint32_t>(a.n_stages)) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                for (int i = 0; i < a.n_stages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.a_full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
                for (uint32_t u = prm_issued > 2 ? prm_issued - 2 : 0; u < prm_issued; ++u)
                    ptx::mbar_wait_bounded(&s.prm_full[u & 1u], (u >> 1) & 1u, &never, kDrainLimitNs);
            }
        }
    } else if (warp < kFirstEpiWarp) {
        // ------------------------------------------------------------ converters (in place)
        const int cw = warp - kFirstConvWarp;
        const int gps = a.h >> 3;  // 8-row groups per individual
        uint32_t stage = 0, phase = 0;
        bool ok = true;
        for (int u = 0; ok && 2 * u < count; ++u) {
            const int n = min(2, count - 2 * u);
            const int groups = n * gps;
            for (int kc = 0; kc < a.k_stages; ++kc) {
                if (!ptx::mbar_wait_bounded(&s.a_full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                uint8_t* sb = s.ring + stage * a.stage_bytes;
                bool bad0 = false, bad1 = false;
                // All of this warp's groups are read first (their loads in
                // flight together), then overwritten: lane l holds rows l/8
                // and 4 + l/8 of each group, K-elements 4 (l % 8) .. + 3.
                float4 f0[kGroupsPerWarp], f1[kGroupsPerWarp];
#pragma unroll
                for (int j = 0; j < kGroupsPerWarp; ++j) {
                    const int g = cw + kConvWarps * j;
                    if (g < groups) {
                        const uint8_t* gp = sb + g * 1024;
                        f0[j] = *reinterpret_cast<const float4*>(gp + lane * 16);
                        f1[j] = *reinterpret_cast<const float4*>(gp + 512 + lane * 16);
                    }
                }
                __syncwarp();  // every group is read before any of it is overwritten
#pragma unroll
                for (int j = 0; j < kGroupsPerWarp; ++j) {
                    const int g = cw + kConvWarps * j;
                    if (g < groups) {
                        uint8_t* gp = sb + g * 1024;
                        put_pieces(gp, lane >> 3, lane & 7, f0[j]);
                        put_pieces(gp, 4 + (lane >> 3), lane & 7, f1[j]);
                        const bool b = out_of_piece_range(f0[j]) || out_of_piece_range(f1[j]);
                        if (g < gps) bad0 |= b; else bad1 |= b;
                    }
                }
                const bool any0 = __any_sync(0xFFFFFFFFu, bad0), any1 = __any_sync(0xFFFFFFFFu, bad1);
                if (lane == 0) {
                    const uint32_t tag = static_cast<uint32_t>(u) + 1u;
                    if (any0) atomicExch(&s.flag[2 * (u % kFlagSlots)], tag);
                    if (any1) atomicExch(&s.flag[2 * (u % kFlagSlots) + 1], tag);
                }
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&s.full[stage]);
                if (++stage == static_cast<uint32_t>(a.n_stages)) { stage = 0; phase ^= 1u; }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - kFirstEpiWarp;
        const int g = ew >> 2;        // slot: the pair's first or second individual
        const int q = warp & 3;       // TMEM lane quarter of this warp
        const int et = (ew & 3) * 32 + lane;
        const int row = q * 32 + lane;
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        const uint32_t bar_id = 1u + static_cast<uint32_t>(g);
        const int32_t label = row < a.batch ? a.y[row] : 0;
        float* b1 = s.b1 + g * a.h;
        float* b2 = s.b2 + g * 16;
        float* w2t = s.w2t + g * a.h * a.dpad;
        int* go_prm = s.ep_go + 2 * g;
        int* go_acc = s.ep_go + 2 * g + 1;
        for (int u = 0; 2 * u < count; ++u) {
            const int n = min(2, count - 2 * u);
            const int p = first + 2 * u + g;
            const uint32_t buf = static_cast<uint32_t>(u) & 1u, bph = (static_cast<uint32_t>(u) >> 1) & 1u;
            // Parameters of this slot's individual: wait for the bulk copy,
            // then stage b1, W2 transposed (rows padded to dpad) and b2.
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(&s.prm_full[buf], bph, s.abort_flag, kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *go_prm = got ? 1 : 0;
            }
            ptx::named_barrier_sync(bar_id, 128);  // A1: parameters landed (or abort)
            if (!*go_prm) break;
            if (g < n) {
                const float* src = reinterpret_cast<const float*>(s.prm_raw + (2 * buf + g) * a.prm_bytes);
                for (int i = et; i < a.h; i += 128) b1[i] = src[i];
                for (int i = et; i < a.d_out * a.h; i += 128) {
                    const int o = i / a.h, col = i - o * a.h;
                    w2t[col * a.dpad + o] = src[a.h + i];
                }
                const int pad = a.dpad - a.d_out;
                for (int i = et; i < a.h * pad; i += 128) w2t[(i / pad) * a.dpad + a.d_out + i % pad] = 0.0f;
                if (et < 16) b2[et] = et < a.d_out ? src[a.h + a.d_out * a.h + et] : 0.0f;
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.prm_empty[buf]);
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(&s.acc_full[buf], bph, s.abort_flag, kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *go_acc = !got ? 0 : (((s.accflag[buf] >> g) & 1u) ? 2 : 1);
            }
            ptx::named_barrier_sync(bar_id, 128);  // A2: accumulator ready (or abort); parameters staged
            const int go = *go_acc;
            if (!go) break;
            ptx::tc_fence_after();

            float loss = 0.0f;
            int32_t good = 0;
            if (g < n) {
                // Individuals with a weight outside the piece range: layer 1 by
                // FP32 FFMA from global memory, k in order, in the accumulator's units.
                const float* w1p = a.popv + static_cast<int64_t>(p) * a.c_pad;
                const uint8_t* xrow = a.x + static_cast<int64_t>(row < a.batch ? row : 0) * a.k;
                const uint32_t col0 = tmem_base + lane_addr + buf * kAccStride + static_cast<uint32_t>(g * a.h);
                float logit[kMaxOutU8];
#pragma unroll
                for (int o = 0; o < kMaxOutU8; ++o) logit[o] = 0.0f;
                for (int c = 0; c < a.h; c += 16) {
                    float v[16];
                    ptx::tmem_ld16(col0 + static_cast<uint32_t>(c), v);
                    if (row < a.batch) {
                        if (go == 2) {
                            ptx::grid_dep_wait();
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float* wr = w1p + static_cast<int64_t>(c + j) * a.k;
                                float acc = 0.0f;
                                for (int kk = 0; kk < a.k; ++kk) acc = fmaf(wr[kk], static_cast<float>(xrow[kk]), acc);
                                v[j] = acc * kPieceScale;
                            }
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int col = c + j;
                            const float hv = fmaxf(fmaf(v[j], a.inv_div, b1[col]), 0.0f);
                            const float4* wr = reinterpret_cast<const float4*>(w2t + col * a.dpad);
#pragma unroll
                            for (int o4 = 0; o4 < kMaxOutU8 / 4; ++o4) {
                                if (4 * o4 < a.d_out) {
                                    const float4 w = wr[o4];
                                    logit[4 * o4 + 0] = fmaf(w.x, hv, logit[4 * o4 + 0]);
                                    logit[4 * o4 + 1] = fmaf(w.y, hv, logit[4 * o4 + 1]);
                                    logit[4 * o4 + 2] = fmaf(w.z, hv, logit[4 * o4 + 2]);
                                    logit[4 * o4 + 3] = fmaf(w.w, hv, logit[4 * o4 + 3]);
                                }
                            }
                        }
                    }
                }
                if (row < a.batch) {
                    float zmax = logit[0] + b2[0];
                    int arg = 0;
#pragma unroll
                    for (int o = 1; o < kMaxOutU8; ++o) {
                        if (o < a.d_out) {
                            const float z = logit[o] + b2[o];
                            if (z > zmax) { zmax = z; arg = o; }
                        }
                    }
                    float se = 0.0f;
#pragma unroll
                    for (int o = 0; o < kMaxOutU8; ++o)
                        if (o < a.d_out) se += expf(logit[o] + b2[o] - zmax);
                    if (label >= 0 && label < a.d_out) {
                        float zl = 0.0f;
#pragma unroll
                        for (int o = 0; o < kMaxOutU8; ++o)
                            if (o == label) zl = logit[o] + b2[o];
                        loss = logf(se) + zmax - zl;
                        good = (arg == label) ? 1 : 0;
                    } else {
                        loss = __int_as_float(0x7FC00000);
                    }
                }
            }
            // The accumulator is read: release it to the next unit's MMAs.
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.acc_empty[buf]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
                good += __shfl_xor_sync(0xFFFFFFFFu, good, off);
            }
            if (lane == 0) {
                s.red_loss[g * 4 + q] = loss;
                s.red_ok[g * 4 + q] = good;
            }
            ptx::named_barrier_sync(bar_id, 128);  // B: quarter sums written; staged parameters no longer read
            if (g < n && et == 0) {
                const float* rl = s.red_loss + g * 4;
                const int32_t* ro = s.red_ok + g * 4;
                const float total = ((rl[0] + rl[1]) + rl[2]) + rl[3];
                const int32_t n_ok = ro[0] + ro[1] + ro[2] + ro[3];
                const float f = -(total / static_cast<float>(a.batch));
                a.f_raw[p] = f;
                if (a.f_adj) a.f_adj[p] = a.f_inh ? (1.0f - a.alpha) * a.f_inh[p] + a.alpha * f : f;
                if (a.correct) a.correct[p] = n_ok;
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, kTmemCols);
    }
}

// The batch's levels as FP16 (exact), row-major [batch][kp], kp = round_up(k,
// 8) with zero padding: the A operand tiles of eval_u8_kernel.  It reads only
// the caller's levels, so it lets the next kernel start at once; before it
// ends it waits for its own predecessor, so that a successor that waits for it
// also sees everything earlier on the stream complete.
__global__ void __launch_bounds__(256) stage_x16_kernel(const uint8_t* __restrict__ x, int32_t batch, int32_t k,
                                                        int32_t kp, __half* __restrict__ x16)
{
    ptx::grid_dep_launch();
    const int32_t per_row = kp >> 3;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < static_cast<int64_t>(batch) * per_row) {
        const int32_t b = static_cast<int32_t>(i / per_row), k0 = static_cast<int32_t>(i % per_row) * 8;
        const uint8_t* src = x + static_cast<int64_t>(b) * k;
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float l0 = k0 + 2 * j < k ? static_cast<float>(src[k0 + 2 * j]) : 0.0f;
            const float l1 = k0 + 2 * j + 1 < k ? static_cast<float>(src[k0 + 2 * j + 1]) : 0.0f;
            w[j] = half2_bits(__floats2half2_rn(l0, l1));
        }
        *reinterpret_cast<uint4*>(x16 + static_cast<int64_t>(b) * kp + k0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    ptx::grid_dep_wait();
}

typedef CUresult (*U8EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

U8EncodeTiledFn u8_encode_fn()
{
    static U8EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<U8EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

bool eval_u8_tc_supported(const NetLayout& net, int32_t batch, const float* pop_dev)
{
    if (net.n_layers != 2) return false;
    const int32_t k = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    if (k % 4 != 0 || h % 16 != 0 || h > 128 || d_out > kMaxOutU8 || batch < 1 || batch > 128) return false;
    if (reinterpret_cast<uintptr_t>(pop_dev) & 15u) return false;
    return u8_stages(h, d_out) > 0 && u8_encode_fn() != nullptr;
}

size_t eval_u8_x16_bytes(const NetLayout& net, int32_t batch)
{
    const int64_t kp = (net.dims[0] + 7) / 8 * 8;
    return static_cast<size_t>(batch) * static_cast<size_t>(kp) * 2u;
}

cudaError_t launch_stage_x16(const NetLayout& net, const uint8_t* x, int32_t batch, void* x16, cudaStream_t stream)
{
    const int32_t k = net.dims[0], kp = (k + 7) / 8 * 8;
    const int64_t items = static_cast<int64_t>(batch) * (kp / 8);
    if (items <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>((items + 255) / 256));
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, stage_x16_kernel, x, batch, k, kp, static_cast<__half*>(x16));
}

cudaError_t launch_eval_u8_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                              const void* x16, float x_div, const int32_t* y, int32_t batch, float alpha,
                              const float* f_inh, float* f_raw, float* f_adj, int32_t* correct, unsigned int* status,
                              cudaStream_t stream)
{
    EvalU8Args a{};
    a.pop = pop;
    a.k = net.dims[0];
    a.h = net.dims[1];
    a.d_out = net.dims[2];
    a.dpad = (a.d_out + 3) / 4 * 4;
    a.batch = batch;
    a.k16 = (a.k + 15) / 16 * 16;
    a.k_stages = (a.k + kKStage - 1) / kKStage;
    a.n_stages = u8_stages(a.h, a.d_out);
    if (a.n_stages == 0) return cudaErrorInvalidValue;
    a.c_pad = net.c_pad;
    a.inv_div = static_cast<float>(1.0 / (static_cast<double>(x_div) * kPieceScale));
    a.alpha = alpha;
    a.popv = pop_dev;
    a.x = x;
    a.y = y;
    a.f_inh = f_inh;
    a.f_raw = f_raw;
    a.f_adj = f_adj;
    a.correct = correct;
    a.status = status;
    a.prm_bytes = u8_prm_bytes(a.h, a.d_out);
    a.slot_bytes = static_cast<uint32_t>(a.h) * 128u;
    a.stage_bytes = u8_stage_bytes(a.h);
    const size_t smem = u8_smem_bytes(a.h, a.d_out, a.n_stages);
    U8EncodeTiledFn enc = u8_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tw, tx;
    {
        // W1 of every individual: [pop][h][k] FP32, rows k * 4 bytes apart.
        const cuuint64_t dims[3] = { static_cast<cuuint64_t>(a.k), static_cast<cuuint64_t>(a.h),
                                     static_cast<cuuint64_t>(pop) };
        const cuuint64_t strides[2] = { static_cast<cuuint64_t>(a.k) * 4u, static_cast<cuuint64_t>(net.c_pad) * 4u };
        const cuuint32_t box[3] = { static_cast<cuuint32_t>(kKStage), static_cast<cuuint32_t>(a.h), 1 };
        const cuuint32_t es[3] = { 1, 1, 1 };
        if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(pop_dev), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // The staged batch: [batch][kp] FP16; rows past the batch and levels
        // past k read as zero.
        const int32_t kp = (a.k + 7) / 8 * 8;
        const cuuint64_t dims[2] = { static_cast<cuuint64_t>(a.k), static_cast<cuuint64_t>(batch) };
        const cuuint64_t strides[1] = { static_cast<cuuint64_t>(kp) * 2u };
        const cuuint32_t box[2] = { static_cast<cuuint32_t>(kKStage), 128 };
        const cuuint32_t es[2] = { 1, 1 };
        if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(x16), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(eval_u8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int grid = pop < sms ? pop : sms;
    a.per_cta = pop / grid;
    a.extra = pop % grid;
    // Programmatic stream serialisation: CTAs may start (barriers, TMEM) while
    // the previous kernel finishes; the producer waits for it before it reads
    // the population or the staged batch.
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kU8Threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, eval_u8_kernel, tw, tx, a);
}

}  // namespace leea
