// leea_eval_u8.cu -- fitness of every individual (Eq. 1; Section 3.3) for
// minibatches of 8-bit image levels, x = k / x_div with k in [0, 255] (MNIST's
// encoding), on the tcgen05 tensor cores with FP32-class accuracy.
//
// The integers k are exact in FP16, and every FP32 weight, scaled by 2^8, is
// split into two FP16 pieces: w1 = fp16(2^8 w) and w2 = fp16(2^8 w - w1), with
// the remainder exact in FP32.  So |2^8 w - w1 - w2| <= max(2^-22 2^8 |w|,
// 2^-25): a 22-bit significand against FP32's 24, and D = K (w1 + w2)^T is
// formed from exact products; only the FP32 accumulation in the tensor core
// rounds.  The epilogue scales by 2^-8 / x_div.  An individual with a weight
// |w| >= 128 (its scaled w1 could overflow FP16) is flagged by the converters,
// and the epilogue forms its layer 1 with FP32 FFMA from global memory instead
// of the accumulator, so every weight range is evaluated in FP32 accuracy.
//
// The batch (<= 128 samples) is written once per CTA into tensor memory as
// the MMA's A operand (lane = sample, two FP16 per column), so shared memory
// only carries the weight pieces: per 64-wide K stage, 2 x h rows of 128
// bytes in the 128-byte swizzled K-major layout.  Two pieces cost two MMAs per
// 16 inputs (the tensor core's per-instruction cost, not its FLOP rate, bounds
// this kernel at h = 112).
//
// Warp roles (persistent CTA, one per SM, individuals strided by gridDim.x):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      TMA producer: FP32 W1 tiles (h rows x 64 K) into a raw ring
//   warps 2-9   converters: split each raw tile into two FP16 pieces and
//               store them swizzled into the piece ring the MMAs read
//   warps 10-13 write the batch into TMEM once; then the epilogue (bias,
//               ReLU, layer 2 with W2 staged transposed in shared memory,
//               softmax cross-entropy, fixed-order batch sum, inheritance)
// Every mbarrier wait is bounded in time; on expiry the kernel sets
// kStatusEvalTimeout, drains its MMAs and exits.
#include <cuda.h>

#include <algorithm>
#include <cuda_fp16.h>

#include "leea_internal.h"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kLoaderWarps = 8;    // converter warps
constexpr int kFirstLoaderWarp = 2;
constexpr int kFirstEpilogueWarp = kFirstLoaderWarp + kLoaderWarps;
constexpr int kU8Threads = 32 * (kFirstEpilogueWarp + 4);
constexpr int kKStage = 64;        // K elements per stage: one 128-byte BF16 row
constexpr int kPieces = 2;          // FP16 pieces per weight
constexpr int kMaxPieceStages = 3;  // piece ring
constexpr int kMaxRawStages = 6;    // FP32 raw ring (TMA)
constexpr int kMaxOutU8 = 16;
constexpr int kRowBatch = 8;       // 16-row groups a loader thread holds in registers at once
constexpr int kXGroups = 7;        // 32-level groups of the batch row loaded at once
constexpr uint32_t kTmemCols = 512;
constexpr float kPieceScale = 256.0f;   // 2^8: weights enter the pieces as 2^8 w
constexpr float kPieceRange = 128.0f;   // |w| below this: 2^8 |w| < 2^15, finite in FP16
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct EvalU8Args {
    int32_t pop, k, h, d_out, dpad, batch, k_stages, k16, raw_stages, piece_stages;
    uint32_t prm_bytes;  // b1, W2, b2 of one individual, rounded up to 16 bytes
    int64_t c_pad;
    float inv_div, alpha;
    uint32_t a_col;  // first TMEM column of the A operand (the accumulator uses 0 .. h-1)
    // Batch staging: chunks of x_kc levels per row at stride x_stride, from
    // byte x_off of the rings (the tail of the region: the piece ring and the
    // last raw stages); raw stages below x_off may load before the batch is in.
    int32_t x_staged, x_kc, x_stride, x_off, n_early;
    const float* popv;
    const uint8_t* x;
    const int32_t* y;
    const float* f_inh;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    unsigned int* status;
};

struct U8Smem {
    uint8_t* raw;         // raw_stages x h x 256 B (FP32 rows of 64 K-elements), 1024-aligned
    uint8_t* ring;        // piece_stages x kPieces x h x 128 B, right after (1024-aligned: h % 4 == 0)
    uint32_t piece_bytes, raw_bytes;
    uint8_t* prm_raw;     // 2 x prm_bytes: b1, W2 (row-major), b2 as stored, bulk-copied
    float* w2t;           // [h][dpad]
    float* b1;            // [h]
    float* b2;            // [16]
    float* hbuf;          // [batch][h + 4]: the accumulator, staged so TMEM is released early
    uint64_t *full, *empty, *raw_full, *raw_empty, *prm_full, *prm_empty, *acc_full, *acc_empty, *a_ready, *drain;
    uint64_t* conv_done;  // [2]: the converters finished individual (unit) u, by u & 1
    uint64_t* x_loaded;   // the epilogue warps have read the batch (rings free for the weights)
    uint64_t* x_full;     // a chunk of the batch landed in the staging area (the idle rings)
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
    uint32_t* flag_unit;  // [2]: u + 1 if individual (unit) u has a weight outside the piece range
    float* red_loss;
    int32_t* red_ok;
};

__device__ __forceinline__ U8Smem carve(uint8_t* raw, const EvalU8Args& a)
{
    U8Smem s;
    s.raw = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    s.piece_bytes = static_cast<uint32_t>(a.h) * 128u;
    s.raw_bytes = static_cast<uint32_t>(a.h) * 256u;
    s.ring = s.raw + a.raw_stages * s.raw_bytes;
    uint8_t* p = s.ring + a.piece_stages * kPieces * s.piece_bytes;
    s.prm_raw = p;
    p += 2u * a.prm_bytes;
    s.w2t = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.h * a.dpad;
    s.b1 = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.h;
    s.b2 = reinterpret_cast<float*>(p);
    p += sizeof(float) * 16;
    s.hbuf = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.batch * (a.h + 4);
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.empty = bars + a.piece_stages;
    s.raw_full = bars + 2 * a.piece_stages;
    s.raw_empty = s.raw_full + a.raw_stages;
    s.prm_full = s.raw_empty + a.raw_stages;
    s.prm_empty = s.prm_full + 2;
    s.acc_full = s.prm_empty + 2;
    s.acc_empty = s.acc_full + 1;
    s.a_ready = s.acc_full + 2;
    s.drain = s.acc_full + 3;
    s.conv_done = s.acc_full + 4;
    s.x_loaded = s.acc_full + 6;
    s.x_full = s.acc_full + 7;
    uint32_t* w = reinterpret_cast<uint32_t*>(s.acc_full + 8);
    s.tmem_holder = w;
    s.abort_flag = reinterpret_cast<volatile int*>(w + 1);
    s.ep_go = reinterpret_cast<int*>(w + 2);
    s.flag_unit = w + 12;
    s.red_loss = reinterpret_cast<float*>(w + 4);
    s.red_ok = reinterpret_cast<int32_t*>(w + 8);
    return s;
}

uint32_t u8_prm_bytes(int32_t h, int32_t d_out)
{
    return (static_cast<uint32_t>(h + d_out * h + d_out) * 4u + 15u) & ~15u;
}

size_t u8_smem_bytes(int32_t h, int32_t dpad, int32_t batch, int32_t piece_stages, int32_t raw_stages)
{
    const int32_t d_out = dpad;  // upper bound for the raw parameter area
    return 1024 + static_cast<size_t>(piece_stages) * kPieces * h * 128 + static_cast<size_t>(raw_stages) * h * 256 +
           2 * u8_prm_bytes(h, d_out) + sizeof(float) * (h * dpad + h + 16) +
           sizeof(float) * static_cast<size_t>(batch) * (h + 4) + 8 * (2 * piece_stages + 2 * raw_stages + 4 + 8) +
           64;
}

// Ring depths (piece, raw) that fit in 227 KB of shared memory, deepest raw
// ring first (the raw ring holds the HBM loads in flight, the piece ring only
// decouples converters from MMAs); false if not even (2, 2) fits.
bool u8_stages(int32_t h, int32_t dpad, int32_t batch, int32_t* piece, int32_t* raw)
{
    for (int32_t rs = kMaxRawStages; rs >= 2; --rs)
        for (int32_t ps = kMaxPieceStages; ps >= 2; --ps)
            if (u8_smem_bytes(h, dpad, batch, ps, rs) <= 227u * 1024u) {
                *piece = ps;
                *raw = rs;
                return true;
            }
    return false;
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

__global__ void __launch_bounds__(kU8Threads, 1)
eval_u8_kernel(const __grid_constant__ CUtensorMap tmap_w, const EvalU8Args a)
{
    extern __shared__ uint8_t smem_raw[];
    const U8Smem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.piece_stages; ++i) {
            ptx::mbar_init(&s.full[i], kLoaderWarps);
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < a.raw_stages; ++i) {
            ptx::mbar_init(&s.raw_full[i], 1);
            ptx::mbar_init(&s.raw_empty[i], kLoaderWarps);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.prm_full[i], 1);
            ptx::mbar_init(&s.prm_empty[i], 128);
        }
        ptx::tma_prefetch_map(&tmap_w);
        ptx::mbar_init(s.acc_full, 1);
        ptx::mbar_init(s.acc_empty, 128);
        ptx::mbar_init(s.a_ready, 128);
        ptx::mbar_init(s.drain, 1);
        ptx::mbar_init(&s.conv_done[0], kLoaderWarps);
        ptx::mbar_init(&s.conv_done[1], kLoaderWarps);
        ptx::mbar_init(s.x_loaded, 128);
        ptx::mbar_init(s.x_full, 1);
        *s.abort_flag = 0;
        *s.ep_go = 0;
        s.flag_unit[0] = 0;
        s.flag_unit[1] = 0;
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
            const uint32_t idesc = ptx::idesc_f16(128, static_cast<uint32_t>(a.h));
            bool ok = ptx::mbar_wait_bounded(s.a_ready, 0u, s.abort_flag, kWaitLimitNs);
            if (!ok) raise_abort(s, a);
            ptx::tc_fence_after();
            uint32_t stage = 0, phase = 0, acc_phase = 0;
            const uint32_t ring = ptx::smem_u32(s.ring);
            for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
                if (!ptx::mbar_wait_bounded(s.acc_empty, acc_phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                for (int kc = 0; kc < a.k_stages; ++kc) {
                    if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t sb = ring + stage * kPieces * s.piece_bytes;
#pragma unroll
                    for (int kk = 0; kk < kKStage / 16; ++kk) {
                        const int kg = kc * kKStage + kk * 16;
                        if (kg >= a.k16) break;
                        const uint32_t a_tmem = tmem_base + a.a_col + static_cast<uint32_t>(kg >> 1);
#pragma unroll
                        for (int piece = 0; piece < kPieces; ++piece) {
                            const uint64_t bd = ptx::smem_desc_sw128(sb + piece * s.piece_bytes + kk * 32u);
                            ptx::mma_f16_tmem_a(tmem_base, a_tmem, bd, idesc, (kc | kk | piece) != 0 ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit(&s.empty[stage]);
                    if (++stage == static_cast<uint32_t>(a.piece_stages)) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                ptx::mma_commit(s.acc_full);
                acc_phase ^= 1u;
            }
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kWaitLimitNs : kDrainLimitNs);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ TMA producer (raw FP32 tiles)
        if (lane == 0) {
            ptx::grid_dep_wait();  // the population comes from the previous kernel (breeding)
            uint32_t stage = 0, phase = 0;
            uint32_t issued_mask = 0, parity_mask = 0;
            uint32_t prm_issued = 0;  // units whose parameters were requested
            // Raw stages that overlap the batch staging area wait until the
            // batch is in TMEM (without staging, all do: the batch's own loads
            // queued behind every SM's first weight tiles took several times
            // as long).
            uint32_t raw_issued = 0;
            bool ok = true;
            for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
                {
                    // b1, W2, b2 of individual p into parameter buffer (unit & 1).
                    const uint32_t pb = prm_issued & 1u, pphase = (prm_issued >> 1) & 1u;
                    if (!ptx::mbar_wait_bounded(&s.prm_empty[pb], pphase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&s.prm_full[pb], a.prm_bytes);
                    ptx::bulk_load(s.prm_raw + pb * a.prm_bytes,
                                   a.popv + static_cast<int64_t>(p) * a.c_pad + static_cast<int64_t>(a.h) * a.k,
                                   a.prm_bytes, &s.prm_full[pb]);
                    ++prm_issued;
                }
                for (int kc = 0; kc < a.k_stages; ++kc) {
                    if (raw_issued == static_cast<uint32_t>(a.n_early) &&
                        !ptx::mbar_wait_bounded(s.x_loaded, 0u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ++raw_issued;
                    if (!ptx::mbar_wait_bounded(&s.raw_empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&s.raw_full[stage], s.raw_bytes);
                    ptx::tma_load_3d(s.raw + stage * s.raw_bytes, &tmap_w, &s.raw_full[stage], kc * kKStage, 0, p);
                    issued_mask |= 1u << stage;
                    parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                    if (++stage == static_cast<uint32_t>(a.raw_stages)) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                for (int i = 0; i < a.raw_stages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.raw_full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
                for (uint32_t u = prm_issued > 2 ? prm_issued - 2 : 0; u < prm_issued; ++u)
                    ptx::mbar_wait_bounded(&s.prm_full[u & 1u], (u >> 1) & 1u, &never, kDrainLimitNs);
            }
        }
    } else if (warp < kFirstEpilogueWarp) {
        // ------------------------------------------------------------ converters
        // Thread (row0, c4) converts K-elements 4 c4 .. 4 c4 + 3 of rows row0 + 16 u.
        const int lt = threadIdx.x - 32 * kFirstLoaderWarp;
        const int row0 = lt >> 4, c4 = lt & 15;
        const int groups = a.h >> 4;
        uint32_t rstage = 0, rphase = 0, stage = 0, phase = 0, unit = 0;
        // the piece ring doubles as the batch staging area until the batch is in
        bool ok = ptx::mbar_wait_bounded(s.x_loaded, 0u, s.abort_flag, kWaitLimitNs);
        if (!ok) raise_abort(s, a);
        for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x, ++unit) {
            for (int kc = 0; kc < a.k_stages; ++kc) {
                if (!ptx::mbar_wait_bounded(&s.raw_full[rstage], rphase, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                const uint8_t* rb = s.raw + rstage * s.raw_bytes;
                float4 v[kRowBatch];
#pragma unroll
                for (int u = 0; u < kRowBatch; ++u)
                    v[u] = u < groups ? *reinterpret_cast<const float4*>(rb + (row0 + 16 * u) * 256 + c4 * 16)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&s.raw_empty[rstage]);
                if (++rstage == static_cast<uint32_t>(a.raw_stages)) { rstage = 0; rphase ^= 1u; }
                if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                uint8_t* sb = s.ring + stage * kPieces * s.piece_bytes;
                bool bad = false;
#pragma unroll
                for (int u = 0; u < kRowBatch; ++u) {
                    if (u < groups) {
                        const int r = row0 + 16 * u;
                        uint32_t lo[kPieces], hi[kPieces];  // pieces of (x, y) and of (z, w)
                        split2x2(v[u].x, v[u].y, lo[0], lo[1]);
                        split2x2(v[u].z, v[u].w, hi[0], hi[1]);
                        bad |= out_of_piece_range(v[u]);
                        const uint32_t off = static_cast<uint32_t>(r) * 128u +
                                             ((static_cast<uint32_t>(c4 >> 1) ^ static_cast<uint32_t>(r & 7)) << 4) +
                                             (static_cast<uint32_t>(c4 & 1) << 3);
#pragma unroll
                        for (int piece = 0; piece < kPieces; ++piece)
                            *reinterpret_cast<uint2*>(sb + piece * s.piece_bytes + off) = make_uint2(lo[piece], hi[piece]);
                    }
                }
                if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) s.flag_unit[unit & 1u] = unit + 1u;
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    ptx::mbar_arrive(&s.full[stage]);
                    // the flag (if any) is released to the epilogue with this arrival
                    if (kc == a.k_stages - 1) ptx::mbar_arrive(&s.conv_done[unit & 1u]);
                }
                if (++stage == static_cast<uint32_t>(a.piece_stages)) { stage = 0; phase ^= 1u; }
            }
        }
    } else {
        // ------------------------------------------------------------ batch into TMEM, then epilogue
        const int et = threadIdx.x - 32 * kFirstEpilogueWarp;
        const int q = warp & 3;  // TMEM lane quarter of this warp
        const int row = q * 32 + lane;
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        {
            // Row `row` of the batch into TMEM as FP16 pairs (lower k in the low
            // half); group g = levels 32 g .. 32 g + 31 = columns 16 g .. 16 g + 15.
            // The last group may reach 8 columns past k16 / 2; levels >= k are 0.
            // A level k < 1024 is exact in FP16 as (1024 + k) - 1024, and 1024 + k
            // has the bit pattern 0x6400 | k: one byte permute builds two of
            // them, one packed subtraction makes the pair exact.
            auto put_group = [&](int g, const uint32_t (&bytes)[8]) {
                const __half2 k1024 = __floats2half2_rn(1024.0f, 1024.0f);
                uint32_t cols[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const uint32_t biased = __byte_perm(bytes[i >> 1], 0x64646464u, (i & 1) ? 0x4342u : 0x4140u);
                    cols[i] = half2_bits(__hsub2(*reinterpret_cast<const __half2*>(&biased), k1024));
                }
                ptx::tmem_st16(tmem_base + lane_addr + a.a_col + static_cast<uint32_t>(16 * g), cols);
            };
            const uint8_t* xr = a.x + static_cast<int64_t>(row) * a.k;
            const bool live = row < a.batch;
            const int n_groups = (a.k16 + 31) / 32;
            // Staged: chunks of every row land by bulk copies in the tail of
            // the rings, which stays idle until the batch is in TMEM (one
            // memory latency per chunk; one chunk at d_0 = 784 and h = 112).
            if (a.x_staged) {
                const int kc = a.x_kc, stride = a.x_stride;
                uint8_t* xs = s.raw + a.x_off;
                uint32_t xphase = 0;
                for (int k0 = 0; k0 < a.k16; k0 += kc, xphase ^= 1u) {
                    const int bytes = min(kc, a.k - k0);  // multiple of 16
                    if (et == 0) ptx::mbar_arrive_expect_tx(s.x_full, static_cast<uint32_t>(a.batch * bytes));
                    if (live) ptx::bulk_load(xs + row * stride, xr + k0, static_cast<uint32_t>(bytes), s.x_full);
                    const bool got = ptx::mbar_wait_bounded(s.x_full, xphase, s.abort_flag, kWaitLimitNs);
                    if (!got) {  // let this chunk's copies land before anything reuses the rings
                        raise_abort(s, a);
                        volatile int never = 0;
                        ptx::mbar_wait_bounded(s.x_full, xphase, &never, kDrainLimitNs);
                    }
                    const uint8_t* src = xs + (live ? row : 0) * stride;
                    for (int g = 0; g < kc / 32 && k0 + 32 * g < a.k16; ++g) {
                        uint32_t wds[8] = { 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u };
                        if (live && got) {
                            const uint4 v0 = *reinterpret_cast<const uint4*>(src + 32 * g);
                            const uint4 v1 = *reinterpret_cast<const uint4*>(src + 32 * g + 16);
                            wds[0] = v0.x; wds[1] = v0.y; wds[2] = v0.z; wds[3] = v0.w;
                            if (k0 + 32 * g + 16 < a.k) { wds[4] = v1.x; wds[5] = v1.y; wds[6] = v1.z; wds[7] = v1.w; }
                        }
                        put_group(k0 / 32 + g, wds);
                    }
                    ptx::named_barrier_sync(1, 128);  // staging area read before the next chunk lands
                }
            } else {
                // Direct: kXGroups groups per round, their loads all in flight.
                for (int g0 = 0; g0 < n_groups; g0 += kXGroups) {
                    uint32_t lv[kXGroups][8];
#pragma unroll
                    for (int b = 0; b < kXGroups; ++b) {
                        const int k0 = 32 * (g0 + b);
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            uint32_t word = 0;
                            if (live && g0 + b < n_groups) {
#pragma unroll
                                for (int q8 = 0; q8 < 4; ++q8) {
                                    const int kk = k0 + 4 * w + q8;
                                    if (kk < a.k) word |= static_cast<uint32_t>(__ldg(xr + kk)) << (8 * q8);
                                }
                            }
                            lv[b][w] = word;
                        }
                    }
#pragma unroll
                    for (int b = 0; b < kXGroups; ++b)
                        if (g0 + b < n_groups) put_group(g0 + b, lv[b]);
                }
            }
            ptx::mbar_arrive(s.x_loaded);
            ptx::tmem_st_wait();
            ptx::tc_fence_before();
            ptx::mbar_arrive(s.a_ready);
        }

        const int32_t label = row < a.batch ? a.y[row] : 0;
        uint32_t acc_phase = 0, unit = 0;
        bool ok = true;
        for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x, ++unit) {
            // Parameters of individual p: wait for the bulk copy, then stage
            // b1, W2 transposed (rows padded to dpad) and b2.
            const uint32_t pb = unit & 1u, pphase = (unit >> 1) & 1u;
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(&s.prm_full[pb], pphase, s.abort_flag, kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *s.ep_go = got ? 1 : 0;
            }
            ptx::named_barrier_sync(1, 128);  // A1: parameters landed (or abort)
            if (!*s.ep_go) { ok = false; break; }
            const float* src = reinterpret_cast<const float*>(s.prm_raw + pb * a.prm_bytes);
            for (int i = et; i < a.h; i += 128) s.b1[i] = src[i];
            for (int i = et; i < a.d_out * a.h; i += 128) {
                const int o = i / a.h, col = i - o * a.h;
                s.w2t[col * a.dpad + o] = src[a.h + i];
            }
            for (int i = et; i < a.h * (a.dpad - a.d_out); i += 128) {
                const int pad = a.dpad - a.d_out;
                s.w2t[(i / pad) * a.dpad + a.d_out + i % pad] = 0.0f;
            }
            if (et < 16) s.b2[et] = et < a.d_out ? src[a.h + a.d_out * a.h + et] : 0.0f;
            ptx::mbar_arrive(&s.prm_empty[pb]);
            if (et == 0) {
                bool got = ptx::mbar_wait_bounded(s.acc_full, acc_phase, s.abort_flag, kWaitLimitNs) &&
                           ptx::mbar_wait_bounded(&s.conv_done[unit & 1u], (unit >> 1) & 1u, s.abort_flag,
                                                  kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *s.ep_go = !got ? 0 : (s.flag_unit[unit & 1u] == unit + 1u ? 2 : 1);
            }
            ptx::named_barrier_sync(1, 128);  // A2: accumulator ready (or abort); parameters staged
            const int go = *s.ep_go;
            if (!go) { ok = false; break; }
            ptx::tc_fence_after();
            // Individuals with a weight outside the piece range: layer 1 by FP32
            // FFMA from global memory, k in order, in the accumulator's units.
            const float* w1p = a.popv + static_cast<int64_t>(p) * a.c_pad;
            const uint8_t* xrow = a.x + static_cast<int64_t>(row < a.batch ? row : 0) * a.k;

            // Stage this lane's accumulator row in shared memory and release
            // TMEM, so the next individual's MMAs overlap the rest of the
            // epilogue (rows >= batch take part in the collective loads only).
            float* hrow = s.hbuf + (row < a.batch ? row : 0) * (a.h + 4);
            for (int c = 0; c < a.h; c += 16) {
                float v[16];
                ptx::tmem_ld16(tmem_base + lane_addr + static_cast<uint32_t>(c), v);
                if (row < a.batch) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(hrow + c + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(s.acc_empty);
            acc_phase ^= 1u;

            float logit[kMaxOutU8];
#pragma unroll
            for (int o = 0; o < kMaxOutU8; ++o) logit[o] = 0.0f;
            for (int c = 0; row < a.batch && c < a.h; c += 16) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    const float4 t4 = *reinterpret_cast<const float4*>(hrow + c + j);
                    v[j] = t4.x;
                    v[j + 1] = t4.y;
                    v[j + 2] = t4.z;
                    v[j + 3] = t4.w;
                }
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
                    const float hv = fmaxf(fmaf(v[j], a.inv_div, s.b1[col]), 0.0f);
                    const float4* wr = reinterpret_cast<const float4*>(s.w2t + col * a.dpad);
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

            float loss = 0.0f;
            int32_t good = 0;
            if (row < a.batch) {
                float zmax = logit[0] + s.b2[0];
                int arg = 0;
#pragma unroll
                for (int o = 1; o < kMaxOutU8; ++o) {
                    if (o < a.d_out) {
                        const float z = logit[o] + s.b2[o];
                        if (z > zmax) { zmax = z; arg = o; }
                    }
                }
                float se = 0.0f;
#pragma unroll
                for (int o = 0; o < kMaxOutU8; ++o)
                    if (o < a.d_out) se += expf(logit[o] + s.b2[o] - zmax);
                const int32_t lbl = label;
                if (lbl >= 0 && lbl < a.d_out) {
                    float zl = 0.0f;
#pragma unroll
                    for (int o = 0; o < kMaxOutU8; ++o)
                        if (o == lbl) zl = logit[o] + s.b2[o];
                    loss = logf(se) + zmax - zl;
                    good = (arg == lbl) ? 1 : 0;
                } else {
                    loss = __int_as_float(0x7FC00000);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
                good += __shfl_xor_sync(0xFFFFFFFFu, good, off);
            }
            if (lane == 0) {
                s.red_loss[q] = loss;
                s.red_ok[q] = good;
            }
            ptx::named_barrier_sync(1, 128);  // B: quarter sums written; staged parameters no longer read
            if (et == 0) {
                const float total = ((s.red_loss[0] + s.red_loss[1]) + s.red_loss[2]) + s.red_loss[3];
                const int32_t n_ok = s.red_ok[0] + s.red_ok[1] + s.red_ok[2] + s.red_ok[3];
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
    if (k % 4 != 0 || h % 16 != 0 || h > 16 * kRowBatch || d_out > kMaxOutU8 || batch < 1 || batch > 128) return false;
    const int32_t k16 = (k + 15) / 16 * 16;
    const int32_t a_cols = (k16 / 2 + 15) / 16 * 16;
    if (h + a_cols > static_cast<int32_t>(kTmemCols)) return false;
    if (reinterpret_cast<uintptr_t>(pop_dev) & 15u) return false;
    const int32_t dpad = (d_out + 3) / 4 * 4;
    int32_t ps = 0, rs = 0;
    return u8_stages(h, dpad, batch, &ps, &rs) && u8_encode_fn() != nullptr;
}

cudaError_t launch_eval_u8_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                              float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                              float* f_raw, float* f_adj, int32_t* correct, unsigned int* status,
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
    a.c_pad = net.c_pad;
    a.inv_div = static_cast<float>(1.0 / (static_cast<double>(x_div) * kPieceScale));
    a.alpha = alpha;
    a.a_col = static_cast<uint32_t>(a.h);
    a.popv = pop_dev;
    a.x = x;
    a.y = y;
    a.f_inh = f_inh;
    a.f_raw = f_raw;
    a.f_adj = f_adj;
    a.correct = correct;
    a.status = status;
    a.prm_bytes = u8_prm_bytes(a.h, a.d_out);
    if (!u8_stages(a.h, a.dpad, a.batch, &a.piece_stages, &a.raw_stages)) return cudaErrorInvalidValue;
    const size_t smem = u8_smem_bytes(a.h, a.dpad, a.batch, a.piece_stages, a.raw_stages);
    {
        // Batch staging in the tail of the rings: row stride kc + 16 bytes
        // (kc a multiple of 32) keeps the per-row 16-byte reads conflict-free.
        const int32_t raw_bytes = a.h * 256;
        const int32_t region = a.piece_stages * kPieces * a.h * 128 + a.raw_stages * raw_bytes;
        const int32_t n_groups = (a.k16 + 31) / 32;
        const int32_t kc = std::min(32 * n_groups, (region / a.batch - 16) / 32 * 32);
        a.x_staged = (a.k % 16 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) && kc >= 32;
        a.x_kc = kc;
        a.x_stride = kc + 16;
        a.x_off = region - a.batch * a.x_stride;
        a.n_early = a.x_staged ? std::min(a.raw_stages, a.x_off / raw_bytes) : 0;
    }
    U8EncodeTiledFn enc = u8_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tw;
    {
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
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(eval_u8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int grid = pop < sms ? pop : sms;
    // Programmatic stream serialisation: CTAs may start (barriers, TMEM, the
    // batch into TMEM) while the previous kernel finishes; the producer waits
    // for it before it reads the population.
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
    return cudaLaunchKernelEx(&cfg, eval_u8_kernel, tw, a);
}

}  // namespace leea
