// leea_eval_u8.cu -- fitness of every individual (Eq. 1; Section 3.3) for
// minibatches of 8-bit image levels, x = k / x_div with k in [0, 255] (MNIST's
// encoding), on the tcgen05 tensor cores with FP32-class accuracy.
//
// The integers k are exact in BF16, and every FP32 weight is split exactly into
// three BF16 pieces w = w1 + w2 + w3 (8 significant bits each).  So
// D = K W1_p^T = sum_i K w_i is formed from exact products, and only the FP32
// accumulation in the tensor core rounds.  The epilogue scales by 1 / x_div.
//
// The batch (<= 128 samples) is written once per CTA into tensor memory as
// the MMA's A operand (lane = sample, two BF16 per column), so shared memory
// only carries the weight pieces: per 64-wide K stage, 3 x h rows of 128
// bytes in the 128-byte swizzled K-major layout.
//
// Warp roles (persistent CTA, one per SM, individuals strided by gridDim.x):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      TMA producer: FP32 W1 tiles (h rows x 64 K) into a raw ring
//   warps 2-9   converters: split each raw tile into three BF16 pieces and
//               store them swizzled into the piece ring the MMAs read
//   warps 10-13 write the batch into TMEM once; then the epilogue (bias,
//               ReLU, layer 2 with W2 staged transposed in shared memory,
//               softmax cross-entropy, fixed-order batch sum, inheritance)
// Every mbarrier wait is bounded in time; on expiry the kernel sets
// kStatusEvalTimeout, drains its MMAs and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include "leea_internal.h"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kLoaderWarps = 8;    // converter warps
constexpr int kFirstLoaderWarp = 2;
constexpr int kFirstEpilogueWarp = kFirstLoaderWarp + kLoaderWarps;
constexpr int kU8Threads = 32 * (kFirstEpilogueWarp + 4);
constexpr int kKStage = 64;        // K elements per stage: one 128-byte BF16 row
constexpr int kMaxPieceStages = 3;  // BF16 piece ring
constexpr int kMaxRawStages = 4;    // FP32 raw ring (TMA)
constexpr int kMaxOutU8 = 16;
constexpr int kRowBatch = 8;       // 16-row groups a loader thread holds in registers at once
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct EvalU8Args {
    int32_t pop, k, h, d_out, dpad, batch, k_stages, k16, raw_stages, piece_stages;
    uint32_t prm_bytes;  // b1, W2, b2 of one individual, rounded up to 16 bytes
    int64_t c_pad;
    float inv_div, alpha;
    uint32_t a_col;  // first TMEM column of the A operand (the accumulator uses 0 .. h-1)
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
    uint8_t* ring;        // piece_stages x 3 pieces x h x 128 B (1024-aligned)
    uint8_t* raw;         // raw_stages x h x 256 B (FP32 rows of 64 K-elements)
    uint32_t piece_bytes, raw_bytes;
    uint8_t* prm_raw;     // 2 x prm_bytes: b1, W2 (row-major), b2 as stored, bulk-copied
    float* w2t;           // [h][dpad]
    float* b1;            // [h]
    float* b2;            // [16]
    uint64_t *full, *empty, *raw_full, *raw_empty, *prm_full, *prm_empty, *acc_full, *acc_empty, *a_ready, *drain;
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
    float* red_loss;
    int32_t* red_ok;
};

__device__ __forceinline__ U8Smem carve(uint8_t* raw, const EvalU8Args& a)
{
    U8Smem s;
    s.ring = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    s.piece_bytes = static_cast<uint32_t>(a.h) * 128u;
    s.raw_bytes = static_cast<uint32_t>(a.h) * 256u;
    s.raw = s.ring + a.piece_stages * 3u * s.piece_bytes;
    uint8_t* p = s.raw + a.raw_stages * s.raw_bytes;
    s.prm_raw = p;
    p += 2u * a.prm_bytes;
    s.w2t = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.h * a.dpad;
    s.b1 = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.h;
    s.b2 = reinterpret_cast<float*>(p);
    p += sizeof(float) * 16;
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
    uint32_t* w = reinterpret_cast<uint32_t*>(s.acc_full + 4);
    s.tmem_holder = w;
    s.abort_flag = reinterpret_cast<volatile int*>(w + 1);
    s.ep_go = reinterpret_cast<int*>(w + 2);
    s.red_loss = reinterpret_cast<float*>(w + 4);
    s.red_ok = reinterpret_cast<int32_t*>(w + 8);
    return s;
}

uint32_t u8_prm_bytes(int32_t h, int32_t d_out)
{
    return (static_cast<uint32_t>(h + d_out * h + d_out) * 4u + 15u) & ~15u;
}

size_t u8_smem_bytes(int32_t h, int32_t dpad, int32_t piece_stages, int32_t raw_stages)
{
    const int32_t d_out = dpad;  // upper bound for the raw parameter area
    return 1024 + static_cast<size_t>(piece_stages) * 3 * h * 128 + static_cast<size_t>(raw_stages) * h * 256 +
           2 * u8_prm_bytes(h, d_out) + sizeof(float) * (h * dpad + h + 16) +
           8 * (2 * piece_stages + 2 * raw_stages + 4 + 4) + 64;
}

// Ring depths (piece, raw) that fit in 227 KB of shared memory, deepest piece
// ring first; false if not even (2, 2) fits.
bool u8_stages(int32_t h, int32_t dpad, int32_t* piece, int32_t* raw)
{
    for (int32_t ps = kMaxPieceStages; ps >= 2; --ps)
        for (int32_t rs = kMaxRawStages; rs >= 2; --rs)
            if (u8_smem_bytes(h, dpad, ps, rs) <= 227u * 1024u) {
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

__device__ __forceinline__ uint32_t bf162_bits(__nv_bfloat162 v)
{
    return *reinterpret_cast<uint32_t*>(&v);
}

// Exact three-way split of two FP32 values into packed BF16 pairs (lower K
// index in the low half): each piece rounds the remainder of the previous
// ones to nearest, and the remainders are exact in FP32.
__device__ __forceinline__ void split3x2(float w0, float w1, uint32_t& p1, uint32_t& p2, uint32_t& p3)
{
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(w0, w1);
    const float2 f1 = __bfloat1622float2(h1);
    const float r0 = w0 - f1.x, r1 = w1 - f1.y;
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(r0, r1);
    const float2 f2 = __bfloat1622float2(h2);
    const __nv_bfloat162 h3 = __floats2bfloat162_rn(r0 - f2.x, r1 - f2.y);
    p1 = bf162_bits(h1);
    p2 = bf162_bits(h2);
    p3 = bf162_bits(h3);
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
        *s.abort_flag = 0;
        *s.ep_go = 0;
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
            const uint32_t idesc = ptx::idesc_bf16(128, static_cast<uint32_t>(a.h));
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
                    const uint32_t sb = ring + stage * 3u * s.piece_bytes;
#pragma unroll
                    for (int kk = 0; kk < kKStage / 16; ++kk) {
                        const int kg = kc * kKStage + kk * 16;
                        if (kg >= a.k16) break;
                        const uint32_t a_tmem = tmem_base + a.a_col + static_cast<uint32_t>(kg >> 1);
#pragma unroll
                        for (int piece = 0; piece < 3; ++piece) {
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
            uint32_t stage = 0, phase = 0;
            uint32_t issued_mask = 0, parity_mask = 0;
            uint32_t prm_issued = 0;  // units whose parameters were requested
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
        uint32_t rstage = 0, rphase = 0, stage = 0, phase = 0;
        bool ok = true;
        for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
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
                uint8_t* sb = s.ring + stage * 3u * s.piece_bytes;
#pragma unroll
                for (int u = 0; u < kRowBatch; ++u) {
                    if (u < groups) {
                        const int r = row0 + 16 * u;
                        uint32_t lo[3], hi[3];  // pieces of (x, y) and of (z, w)
                        split3x2(v[u].x, v[u].y, lo[0], lo[1], lo[2]);
                        split3x2(v[u].z, v[u].w, hi[0], hi[1], hi[2]);
                        const uint32_t off = static_cast<uint32_t>(r) * 128u +
                                             ((static_cast<uint32_t>(c4 >> 1) ^ static_cast<uint32_t>(r & 7)) << 4) +
                                             (static_cast<uint32_t>(c4 & 1) << 3);
#pragma unroll
                        for (int piece = 0; piece < 3; ++piece)
                            *reinterpret_cast<uint2*>(sb + piece * s.piece_bytes + off) = make_uint2(lo[piece], hi[piece]);
                    }
                }
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&s.full[stage]);
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
            // Row `row` of the batch as BF16 pairs (k even in the low half).
            const uint8_t* xr = a.x + static_cast<int64_t>(row) * a.k;
            const bool live = row < a.batch;
            const bool vec = (a.k % 16 == 0) && ((reinterpret_cast<uintptr_t>(a.x) & 15u) == 0);
#pragma unroll 2
            for (int c0 = 0; c0 < a.k16 / 2; c0 += 16) {
                uint32_t bytes[8];  // the 32 levels of columns c0 .. c0+15
                const int k0 = 2 * c0;
                if (vec && live && k0 + 32 <= a.k) {
                    const uint4 lo4 = __ldg(reinterpret_cast<const uint4*>(xr + k0));
                    const uint4 hi4 = __ldg(reinterpret_cast<const uint4*>(xr + k0 + 16));
                    bytes[0] = lo4.x; bytes[1] = lo4.y; bytes[2] = lo4.z; bytes[3] = lo4.w;
                    bytes[4] = hi4.x; bytes[5] = hi4.y; bytes[6] = hi4.z; bytes[7] = hi4.w;
                } else {
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        uint32_t word = 0;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int kk = k0 + 4 * w + b;
                            if (live && kk < a.k) word |= static_cast<uint32_t>(xr[kk]) << (8 * b);
                        }
                        bytes[w] = word;
                    }
                }
                uint32_t cols[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const uint32_t pair = bytes[i >> 1] >> (16 * (i & 1));
                    const uint32_t lo = pair & 0xFFu, hi = (pair >> 8) & 0xFFu;
                    cols[i] = (__float_as_uint(static_cast<float>(lo)) >> 16) |
                              (__float_as_uint(static_cast<float>(hi)) & 0xFFFF0000u);
                }
                ptx::tmem_st16(tmem_base + lane_addr + a.a_col + static_cast<uint32_t>(c0), cols);
            }
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
                const bool got = ptx::mbar_wait_bounded(s.acc_full, acc_phase, s.abort_flag, kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *s.ep_go = got ? 1 : 0;
            }
            ptx::named_barrier_sync(1, 128);  // A2: accumulator ready (or abort); parameters staged
            if (!*s.ep_go) { ok = false; break; }
            ptx::tc_fence_after();

            float logit[kMaxOutU8];
#pragma unroll
            for (int o = 0; o < kMaxOutU8; ++o) logit[o] = 0.0f;
            for (int c = 0; c < a.h; c += 16) {
                float v[16];
                ptx::tmem_ld16(tmem_base + lane_addr + static_cast<uint32_t>(c), v);
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
            ptx::tc_fence_before();
            ptx::mbar_arrive(s.acc_empty);
            acc_phase ^= 1u;

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
    return u8_stages(h, dpad, &ps, &rs) && u8_encode_fn() != nullptr;
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
    a.inv_div = static_cast<float>(1.0 / static_cast<double>(x_div));
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
    if (!u8_stages(a.h, a.dpad, &a.piece_stages, &a.raw_stages)) return cudaErrorInvalidValue;
    const size_t smem = u8_smem_bytes(a.h, a.dpad, a.piece_stages, a.raw_stages);
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
    eval_u8_kernel<<<grid, kU8Threads, smem, stream>>>(tw, a);
    return cudaGetLastError();
}

}  // namespace leea
