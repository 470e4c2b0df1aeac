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
// (stage_x16_kernel; it stays in L2), arrives by TMA in K-stage tiles next to
// the weights.  A K stage is 64 inputs (128-byte swizzled FP16 rows, 256-byte
// FP32 rows) when three such stages fit in shared memory (h <= 112), else 32
// (64-byte swizzle): the wider slices stream HBM faster (measured with no
// compute: 4.8 against 4.0-4.4 TB/s for the same 351 MB).
//
// Pipeline (persistent CTA, one per SM; each CTA takes a contiguous range of
// individuals, as pairs, the last one alone when the range is odd):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      producer: per stage, one TMA of the batch tile (the batch's
//               rows rounded up to 8, from L2) and one TMA per individual of
//               its FP32 W1 slice.  A stage is [batch tile][slot 0][slot 1]:
//               the MMA reads 128 rows of A, and rows past the tile fall on
//               the slots' data, which only accumulator rows past the batch see
//   warps 2-9   converters: each 8-row group of a raw FP32 slice is read by
//               one warp and overwritten in place by its two FP16 pieces in
//               the swizzled K-major layout (piece q in the group's q-th half,
//               so the pieces of all 2h rows form two operands whose 8-row
//               groups are one group apart); a warp reads the groups of a
//               batch before it writes any of them
//   warps 10-17 epilogue, 4 warps (one per TMEM lane quarter = 32 samples)
//               per individual: while the unit's MMAs run, b1, W2 (transposed)
//               and b2 are loaded into shared memory; then bias, ReLU, layer
//               2, softmax cross-entropy, fixed-order batch sum, inheritance
//               blend; accumulators are double-buffered in TMEM (columns 0
//               and 256), so a pair's epilogue overlaps the next pair's MMAs
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
constexpr int kFirstEpiWarp = kFirstConvWarp + kConvWarps;
constexpr int kEpiWarps = 8;
constexpr int kU8Threads = 32 * (kFirstEpiWarp + kEpiWarps);
constexpr int kMinStages = 3;
constexpr int kMaxStages = 6;
constexpr int kMaxOutU8 = 16;
constexpr int kMaxGroups = 2 * 128 / 8;  // 8-row groups of the widest pair
constexpr int kFlagSlots = 16;          // unit-tagged range flags; converters run at most a few units ahead
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;    // the two accumulators: columns 0 and 256
constexpr float kPieceScale = 256.0f;   // 2^8: weights enter the pieces as 2^8 w
constexpr float kPieceRange = 128.0f;   // |w| below this: 2^8 |w| < 2^15, finite in FP16
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

// Layout of one K stage of KS inputs.
template <int KS>
struct StageShape {
    static constexpr uint32_t kRawRow = 4u * KS;            // FP32 bytes per row
    static constexpr uint32_t kPieceRow = 2u * KS;          // FP16 bytes per row: one swizzle atom row
    static constexpr uint32_t kGroup = 8u * kRawRow;        // an 8-row group: raw, then both pieces
    static constexpr uint32_t kPieceOff = 8u * kPieceRow;   // piece 1 within a group
    static constexpr int kF4 = KS / 16;                     // float4 per lane and group
    static constexpr int kBatch = KS == 64 ? 2 : 4;         // groups a converter warp reads before it writes
    static constexpr uint32_t kSwizzle = KS == 64 ? 2u : 4u;  // descriptor swizzle code: 128 or 64 bytes
};

struct EvalU8Args {
    int32_t pop, k, h, d_out, dpad, batch, k16, k_stages, n_stages;
    int32_t per_cta, extra;  // individuals per CTA: per_cta, one more for the first `extra` CTAs
    uint32_t slot_bytes;     // one individual's slice of a stage: h raw rows
    uint32_t a_bytes;        // the batch tile: round_up(batch, 8) rows of FP16 levels
    uint32_t stage_bytes;    // the batch tile and two slots, rounded up to 1 KB
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
    uint8_t* ring;       // n_stages x stage_bytes, 1024-aligned: the batch tile, then W1 slices (raw, then pieces)
    float* w2t;          // [2 slots][h][dpad]
    float* b1;           // [2 slots][h]
    float* b2;           // [2 slots][16]
    float* red_loss;     // [2 slots][4 quarters]
    int32_t* red_ok;     // [2 slots][4 quarters]
    uint32_t* flag;      // [kFlagSlots][2]: u + 1 if unit u's individual in that slot has |w| >= 128
    uint32_t* accflag;   // [2]: the flags of the unit in that accumulator, for the epilogue
    int* ep_go;          // [2 slots]: the epilogue groups' go words
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    uint64_t *full, *a_full, *empty, *acc_full, *acc_empty, *drain;
};

constexpr size_t kTailFixed = sizeof(float) * 8 + sizeof(int32_t) * 8 + sizeof(uint32_t) * (2 * kFlagSlots + 2) +
                              sizeof(int) * 2 + 16 + 16;

size_t u8_tail_bytes(int32_t h, int32_t dpad, int32_t n_stages)
{
    return sizeof(float) * (2u * h * dpad + 2u * h + 32u) + kTailFixed + 8u * (3u * n_stages + 5u);
}

__device__ __forceinline__ U8Smem carve(uint8_t* raw, const EvalU8Args& a)
{
    U8Smem s;
    s.ring = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    uint8_t* p = s.ring + static_cast<size_t>(a.n_stages) * a.stage_bytes;
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
    p += sizeof(int) * 2;
    s.tmem_holder = reinterpret_cast<uint32_t*>(p);
    s.abort_flag = reinterpret_cast<volatile int*>(p + 4);
    p += 16;
    p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 15u) & ~uintptr_t(15));
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.a_full = bars + a.n_stages;
    s.empty = bars + 2 * a.n_stages;
    s.acc_full = bars + 3 * a.n_stages;
    s.acc_empty = s.acc_full + 2;
    s.drain = s.acc_empty + 2;
    return s;
}

uint32_t u8_a_bytes(int32_t batch, int32_t ks)
{
    return static_cast<uint32_t>((batch + 7) / 8 * 8) * 2u * static_cast<uint32_t>(ks);
}

// A stage holds the batch tile and two slots, and at least the 128 rows of A
// the MMA reads from its start.
uint32_t u8_stage_bytes(int32_t h, int32_t batch, int32_t ks)
{
    const uint32_t b = u8_a_bytes(batch, ks) + 2u * static_cast<uint32_t>(h) * 4u * static_cast<uint32_t>(ks);
    return std::max((b + 1023u) & ~1023u, 128u * 2u * static_cast<uint32_t>(ks));
}

size_t u8_smem_bytes(int32_t h, int32_t d_out, int32_t batch, int32_t ks, int32_t n_stages)
{
    const int32_t dpad = (d_out + 3) / 4 * 4;
    return 1024 + static_cast<size_t>(n_stages) * u8_stage_bytes(h, batch, ks) + u8_tail_bytes(h, dpad, n_stages);
}

// The deepest ring of K stage `ks` that fits in 227 KB of shared memory; 0 if
// not even kMinStages do.
int32_t u8_stages(int32_t h, int32_t d_out, int32_t batch, int32_t ks)
{
    for (int32_t ns = kMaxStages; ns >= kMinStages; --ns)
        if (u8_smem_bytes(h, d_out, batch, ks, ns) <= 227u * 1024u) return ns;
    return 0;
}

// K stage of a net: 64 inputs when kMinStages of them fit, else 32 (0: neither).
int32_t u8_kstage(int32_t h, int32_t d_out, int32_t batch)
{
    return u8_stages(h, d_out, batch, 64) > 0 ? 64 : (u8_stages(h, d_out, batch, 32) > 0 ? 32 : 0);
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

// Four weights of row r (0..7) of an 8-row group, inputs 4 c4 .. 4 c4 + 3 of
// the stage, as FP16 pieces at their swizzled positions (the 16-byte chunk
// index XORed with r for the 128-byte swizzle, with r / 2 for the 64-byte one).
template <int KS>
__device__ __forceinline__ void put_pieces(uint8_t* group, int r, int c4, const float4& f)
{
    using S = StageShape<KS>;
    uint32_t lo[2], hi[2];
    split2x2(f.x, f.y, lo[0], lo[1]);
    split2x2(f.z, f.w, hi[0], hi[1]);
    const uint32_t chunk = static_cast<uint32_t>(c4 >> 1) ^
                           (KS == 64 ? static_cast<uint32_t>(r & 7) : (static_cast<uint32_t>(r >> 1) & 3u));
    const uint32_t off = static_cast<uint32_t>(r) * S::kPieceRow + (chunk << 4) + (static_cast<uint32_t>(c4 & 1) << 3);
    *reinterpret_cast<uint2*>(group + off) = make_uint2(lo[0], hi[0]);
    *reinterpret_cast<uint2*>(group + S::kPieceOff + off) = make_uint2(lo[1], hi[1]);
}

// This CTA's individuals: [first, first + count).
__device__ __forceinline__ void cta_range(const EvalU8Args& a, int& first, int& count)
{
    const int b = static_cast<int>(blockIdx.x);
    first = b * a.per_cta + min(b, a.extra);
    count = a.per_cta + (b < a.extra ? 1 : 0);
}

template <int KS>
__global__ void __launch_bounds__(kU8Threads, 1)
eval_u8_kernel(const __grid_constant__ CUtensorMap tmap_w, const __grid_constant__ CUtensorMap tmap_x,
               const EvalU8Args a)
{
    using S = StageShape<KS>;
    extern __shared__ uint8_t smem_raw[];
    const U8Smem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int first = 0, count = 0;
    cta_range(a, first, count);

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.n_stages; ++i) {
            ptx::mbar_init(&s.full[i], kConvWarps);  // converted
            ptx::mbar_init(&s.a_full[i], 1);         // the stage's tiles landed
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.acc_full[i], 2);  // the MMAs' commit and the issuer's flag hand-over
            ptx::mbar_init(&s.acc_empty[i], kEpiWarps);
        }
        ptx::mbar_init(s.drain, 1);
        ptx::tma_prefetch_map(&tmap_w);
        ptx::tma_prefetch_map(&tmap_x);
        for (int i = 0; i < 2 * kFlagSlots; ++i) s.flag[i] = 0u;
        s.accflag[0] = s.accflag[1] = 0u;
        s.ep_go[0] = s.ep_go[1] = 0;
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
                    for (int kk = 0; kk < KS / 16; ++kk) {
                        if (kc * KS + kk * 16 >= a.k16) break;
                        const uint64_t ad = ptx::smem_desc(sb + 32u * kk, 8u * S::kPieceRow, S::kSwizzle);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const uint64_t bd =
                                ptx::smem_desc(sb + a.a_bytes + S::kPieceOff * q + 32u * kk, S::kGroup, S::kSwizzle);
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
            uint32_t stage = 0, phase = 0, issued_mask = 0, parity_mask = 0;
            bool ok = true;
            for (int u = 0; ok && 2 * u < count; ++u) {
                const int n = min(2, count - 2 * u), p0 = first + 2 * u;
                for (int kc = 0; kc < a.k_stages; ++kc) {
                    if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    uint8_t* sb = s.ring + stage * a.stage_bytes;
                    ptx::mbar_arrive_expect_tx(&s.a_full[stage], a.a_bytes + static_cast<uint32_t>(n) * a.slot_bytes);
                    ptx::tma_load_2d(sb, &tmap_x, &s.a_full[stage], kc * KS, 0);
                    for (int j = 0; j < n; ++j)
                        ptx::tma_load_3d(sb + a.a_bytes + j * a.slot_bytes, &tmap_w, &s.a_full[stage], kc * KS, 0,
                                         p0 + j);
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
            }
        }
    } else if (warp < kFirstEpiWarp) {
        // ------------------------------------------------------------ converters (in place)
        // Lane l handles float4 f = l + 32 m (m < kF4) of each of its groups:
        // row f / (KS / 4), inputs 4 (f % (KS / 4)) .. + 3.
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
                uint8_t* sb = s.ring + stage * a.stage_bytes + a.a_bytes;  // the slots
                bool bad0 = false, bad1 = false;
#pragma unroll
                for (int g0 = 0; g0 < kMaxGroups / kConvWarps; g0 += S::kBatch) {
                    // Read a batch of this warp's groups, then overwrite them.
                    float4 f[S::kBatch][S::kF4];
#pragma unroll
                    for (int b = 0; b < S::kBatch; ++b) {
                        const int g = cw + kConvWarps * (g0 + b);
                        if (g < groups) {
#pragma unroll
                            for (int m = 0; m < S::kF4; ++m)
                                f[b][m] = *reinterpret_cast<const float4*>(sb + g * S::kGroup + (lane + 32 * m) * 16);
                        }
                    }
                    __syncwarp();  // the batch is read before any of it is overwritten
#pragma unroll
                    for (int b = 0; b < S::kBatch; ++b) {
                        const int g = cw + kConvWarps * (g0 + b);
                        if (g < groups) {
                            bool bad = false;
#pragma unroll
                            for (int m = 0; m < S::kF4; ++m) {
                                const int fi = lane + 32 * m;
                                put_pieces<KS>(sb + g * S::kGroup, fi / (KS / 4), fi % (KS / 4), f[b][m]);
                                bad |= out_of_piece_range(f[b][m]);
                            }
                            if (g < gps) bad0 |= bad; else bad1 |= bad;
                        }
                    }
                    __syncwarp();
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
        float* b1s = s.b1 + g * a.h;
        float* b2s = s.b2 + g * 16;
        float* w2t = s.w2t + g * a.h * a.dpad;
        int* go = s.ep_go + g;
        ptx::grid_dep_wait();  // b1, W2, b2 come from the previous kernel (breeding)
        for (int u = 0; 2 * u < count; ++u) {
            const int n = min(2, count - 2 * u);
            const int p = first + 2 * u + g;
            const uint32_t buf = static_cast<uint32_t>(u) & 1u, bph = (static_cast<uint32_t>(u) >> 1) & 1u;
            if (g < n) {
                // While this unit's MMAs run: b1, W2 transposed (rows padded to
                // dpad with zeros) and b2 of this slot's individual, as stored
                // after W1, into shared memory.  The group finished reading the
                // previous ones at its barrier B.  Loads go through L2
                // (ld.global.cg), not the read-only path: this grid starts while
                // the breeding kernel that writes the masters still runs, and the
                // read-only path assumes data no grid changes during the kernel.
                const float* src = a.popv + static_cast<int64_t>(p) * a.c_pad + static_cast<int64_t>(a.h) * a.k;
                for (int i = et; i < a.h; i += 128) b1s[i] = __ldcg(src + i);
                for (int i = et; i < a.d_out * a.h; i += 128) {
                    const int o = i / a.h, col = i - o * a.h;
                    w2t[col * a.dpad + o] = __ldcg(src + a.h + i);
                }
                const int pad = a.dpad - a.d_out;
                for (int i = et; i < a.h * pad; i += 128) w2t[(i / pad) * a.dpad + a.d_out + i % pad] = 0.0f;
                if (et < 16) b2s[et] = et < a.d_out ? __ldcg(src + a.h + a.d_out * a.h + et) : 0.0f;
            }
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(&s.acc_full[buf], bph, s.abort_flag, kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *go = !got ? 0 : (((s.accflag[buf] >> g) & 1u) ? 2 : 1);
            }
            ptx::named_barrier_sync(bar_id, 128);  // A: accumulator ready (or abort); parameters staged
            const int gov = *go;
            if (!gov) break;
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
                        if (gov == 2) {
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
                            const float hv = fmaxf(fmaf(v[j], a.inv_div, b1s[col]), 0.0f);
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
                    float bo[kMaxOutU8];
#pragma unroll
                    for (int o = 0; o < kMaxOutU8; ++o) bo[o] = b2s[o];
                    float zmax = logit[0] + bo[0];
                    int arg = 0;
#pragma unroll
                    for (int o = 1; o < kMaxOutU8; ++o) {
                        if (o < a.d_out) {
                            const float z = logit[o] + bo[o];
                            if (z > zmax) { zmax = z; arg = o; }
                        }
                    }
                    float se = 0.0f;
#pragma unroll
                    for (int o = 0; o < kMaxOutU8; ++o)
                        if (o < a.d_out) se += expf(logit[o] + bo[o] - zmax);
                    if (label >= 0 && label < a.d_out) {
                        float zl = 0.0f;
#pragma unroll
                        for (int o = 0; o < kMaxOutU8; ++o)
                            if (o == label) zl = logit[o] + bo[o];
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
    return u8_kstage(h, d_out, batch) > 0 && u8_encode_fn() != nullptr;
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
    a.batch = batch;
    a.k16 = (a.k + 15) / 16 * 16;
    a.dpad = (a.d_out + 3) / 4 * 4;
    const int32_t ks = u8_kstage(a.h, a.d_out, batch);
    if (ks == 0) return cudaErrorInvalidValue;
    a.k_stages = (a.k + ks - 1) / ks;
    a.n_stages = u8_stages(a.h, a.d_out, batch, ks);
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
    a.slot_bytes = static_cast<uint32_t>(a.h) * 4u * static_cast<uint32_t>(ks);
    a.a_bytes = u8_a_bytes(batch, ks);
    a.stage_bytes = u8_stage_bytes(a.h, batch, ks);
    const size_t smem = u8_smem_bytes(a.h, a.d_out, batch, ks, a.n_stages);
    U8EncodeTiledFn enc = u8_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tw, tx;
    {
        // W1 of every individual: [pop][h][k] FP32, rows k * 4 bytes apart.
        const cuuint64_t dims[3] = { static_cast<cuuint64_t>(a.k), static_cast<cuuint64_t>(a.h),
                                     static_cast<cuuint64_t>(pop) };
        const cuuint64_t strides[2] = { static_cast<cuuint64_t>(a.k) * 4u, static_cast<cuuint64_t>(net.c_pad) * 4u };
        const cuuint32_t box[3] = { static_cast<cuuint32_t>(ks), static_cast<cuuint32_t>(a.h), 1 };
        const cuuint32_t es[3] = { 1, 1, 1 };
        if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(pop_dev), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // The staged batch: [batch][kp] FP16, tiles of round_up(batch, 8)
        // rows; rows past the batch and levels past k read as zero.
        const int32_t kp = (a.k + 7) / 8 * 8;
        const cuuint64_t dims[2] = { static_cast<cuuint64_t>(a.k), static_cast<cuuint64_t>(batch) };
        const cuuint64_t strides[1] = { static_cast<cuuint64_t>(kp) * 2u };
        const cuuint32_t box[2] = { static_cast<cuuint32_t>(ks), static_cast<cuuint32_t>((batch + 7) / 8 * 8) };
        const cuuint32_t es[2] = { 1, 1 };
        if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(x16), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, ks == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    const void* kern = ks == 64 ? reinterpret_cast<const void*>(eval_u8_kernel<64>)
                                : reinterpret_cast<const void*>(eval_u8_kernel<32>);
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int grid = pop < sms ? pop : sms;
    a.per_cta = pop / grid;
    a.extra = pop % grid;
    // Programmatic stream serialisation: CTAs may start (barriers, TMEM) while
    // the previous kernel finishes; the producer and the epilogue wait for it
    // before they read the population or the staged batch.
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
    return ks == 64 ? cudaLaunchKernelEx(&cfg, eval_u8_kernel<64>, tw, tx, a)
                    : cudaLaunchKernelEx(&cfg, eval_u8_kernel<32>, tw, tx, a);
}

}  // namespace leea
