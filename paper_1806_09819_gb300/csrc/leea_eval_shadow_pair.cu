// leea_eval_shadow_pair.cu -- the precision form's fitness evaluation (Eq. 1;
// Section 3.3) in the state object: layer 1 on the BF16 or FP8-e4m3 shadow
// of W1 with FP32 accumulation, two individuals per tcgen05 MMA; b1, W2, b2
// and the softmax cross-entropy in FP32 from the master.
//
// A tcgen05.mma of M = 128 costs about the same time for any N up to 256,
// and the shadows carry half (BF16) or a quarter (FP8) of the master's bytes,
// so the MMA rate bounds this evaluation unless two individuals share every
// MMA: the batch tile is the A operand (128 samples, the M side) and the
// pair's shadow blocks, side by side, the B operand (N = 2h).  The batch is
// staged once per evaluation as operand tiles in global memory, in the
// 128-byte-swizzled K-major image the tensor core reads (stage_xop_kernel:
// BF16 levels, exact; or the two exact FP8 pieces 16 floor(k / 16) and
// k mod 16, whose products add to k w); the shadows are stored pre-tiled
// (shadow_offset), so every operand of a stage is one contiguous bulk copy.
// A batch above 128 samples is split into 128-sample tiles on different CTAs;
// their partial sums meet in scratch memory and are combined in tile order.
//
// Warp roles (persistent CTA, one per SM; CTA b takes tile b % m_tiles and a
// contiguous range of individuals, as pairs, the last one alone when the
// range is odd):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      producer of the shadows: per stage each individual's shadow
//               block, by bulk copy
//   warp 18     producer of the batch: per stage its block (one or two
//               pieces), by bulk copy from L2.  One thread's bulk copies
//               complete about one at a time (measured from L2: 16 KB copies
//               at 50 GB/s per issuing thread, 100 with two), so the two
//               streams get their own threads.
//   warps 2-17  epilogue, 8 warps per individual: for each TMEM lane quarter
//               one warp runs layer-2 chains 0 and 1, another chains 2 and 3
//               and the softmax cross-entropy.  b1, W2 and b2 are loaded into
//               registers one unit ahead and staged in shared memory; scale
//               (1 / x_div, times the FP8 factor 2^e), bias, ReLU, layer 2 in
//               packed FP32 FMAs, fixed-order sums; accumulators
//               double-buffered in TMEM (columns 0 and 256).  Eight warps
//               per individual rather than four: the epilogue is bound by
//               instruction latency (shared-memory loads feeding FMA chains),
//               not by any pipe, so it needs the warps to hide it.
// Every mbarrier wait is bounded in time; on expiry the kernel sets
// kStatusEvalTimeout, lets its copies and MMAs in flight finish and exits.
#include <cuda.h>

#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "leea_internal.h"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kFirstEpiWarp = 2;
constexpr int kEpiWarps = 16;      // 8 per individual of a pair: 2 per TMEM lane quarter
constexpr int kGroupThreads = 256;  // epilogue threads per individual
constexpr int kPrmRegs = 9;        // b1, W2, b2 floats per epilogue thread: ceil((128 + 16 * 128 + 16) / 256)
constexpr int kBatchWarp = kFirstEpiWarp + kEpiWarps;  // the batch's producer
constexpr int kPairThreads = 32 * (kBatchWarp + 1);
constexpr int kMaxOut = 16;
constexpr int kSegGroups = 4;  // 8-column groups in a quarter of a chunk of at most 128 hidden units
constexpr int kMinStages = 3;
constexpr int kMaxStages = 6;
constexpr uint32_t kBlockBytes = 128u * 128u;  // a 128-row operand block of 128-byte rows
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct PairArgs {
    int32_t pop, k, h, d_out, dpad, batch, m_tiles, k_blocks, k_mma, n_stages, n_prm;
    int32_t cw, n_chunks;  // the hidden-unit chunks whose summation order the epilogue keeps
    int32_t per_grp, extra, groups;  // individuals per CTA group: per_grp, one more for the first `extra`
    uint32_t a_bytes, slot_bytes, stage_bytes;
    int64_t c_pad, sh_stride;
    float inv_div, alpha;
    const float* popv;
    const uint8_t* shadow;
    const int32_t* scale_exp;
    const uint8_t* xop;  // staged batch tiles: [m_tiles][k_blocks][pieces][128 rows][128 B]
    const int32_t* y;
    const float* f_inh;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    float* scratch;  // m_tiles > 1: [2][m_tiles][pop] partial loss sums and correct counts
    unsigned int* status;
};

struct PairSmem {
    uint8_t* ring;       // n_stages x stage_bytes: the batch block(s), then the pair's shadow blocks
    float* w2t;          // [2 slots][h][dpad]
    float* b1;           // [2 slots][h]
    float* b2;           // [2 slots][16]
    float* red_loss;     // [2 slots][4]
    float* part;         // [2 slots][128 rows][dpad]: the first half's sum of chains 0 and 1
    int32_t* red_ok;     // [2 slots][4]
    int* ep_go;          // [2 slots]
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    uint64_t *full, *empty, *acc_full, *acc_empty, *drain;
};

size_t pair_tail_bytes(int32_t h, int32_t d_out, int32_t n_stages)
{
    const int32_t dpad = (d_out + 3) / 4 * 4;
    return sizeof(float) * (2u * h * dpad + 2u * h + 32u + 8u + 2u * 128u * dpad) + sizeof(int32_t) * 8u +
           sizeof(int) * 2u + 16u + 8u * (2u * n_stages + 5u) + 64u;
}

uint32_t pair_stage_bytes(int32_t precision, int32_t h)
{
    return (precision == 1 ? 1u : 2u) * kBlockBytes + 2u * static_cast<uint32_t>(h) * 128u;
}

size_t pair_smem_bytes(int32_t precision, int32_t h, int32_t d_out, int32_t n_stages)
{
    return 1024 + static_cast<size_t>(n_stages) * pair_stage_bytes(precision, h) + pair_tail_bytes(h, d_out, n_stages);
}

int32_t pair_stages(int32_t precision, int32_t h, int32_t d_out)
{
    for (int32_t ns = kMaxStages; ns >= kMinStages; --ns)
        if (pair_smem_bytes(precision, h, d_out, ns) <= 227u * 1024u) return ns;
    return 0;
}

__device__ __forceinline__ PairSmem carve(uint8_t* raw, const PairArgs& a)
{
    PairSmem s;
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
    s.part = reinterpret_cast<float*>(p);
    p += sizeof(float) * 2 * 128 * a.dpad;
    s.red_ok = reinterpret_cast<int32_t*>(p);
    p += sizeof(int32_t) * 8;
    s.ep_go = reinterpret_cast<int*>(p);
    p += sizeof(int) * 2;
    s.tmem_holder = reinterpret_cast<uint32_t*>(p);
    s.abort_flag = reinterpret_cast<volatile int*>(p + 4);
    p += 16;
    p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 7u) & ~uintptr_t(7));
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.empty = bars + a.n_stages;
    s.acc_full = bars + 2 * a.n_stages;
    s.acc_empty = s.acc_full + 2;
    s.drain = s.acc_empty + 2;
    return s;
}

__device__ __forceinline__ void raise_abort(const PairSmem& s, const PairArgs& a)
{
    *s.abort_flag = 1;
    atomicOr(a.status, kStatusEvalTimeout);
}

// This CTA's sample tile and individuals [first, first + count).
__device__ __forceinline__ void cta_work(const PairArgs& a, int& mt, int& first, int& count)
{
    const int b = static_cast<int>(blockIdx.x);
    mt = b % a.m_tiles;
    const int g = b / a.m_tiles;
    first = g * a.per_grp + min(g, a.extra);
    count = a.per_grp + (g < a.extra ? 1 : 0);
}

template <int PREC, int DOUT>  // DOUT: d_out when fixed at compile time (10), else 0
__global__ void __launch_bounds__(kPairThreads, 1) eval_shadow_pair_kernel(const PairArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const PairSmem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int mt = 0, first = 0, count = 0;
    cta_work(a, mt, first, count);
    constexpr uint32_t kPieces = PREC == 1 ? 1u : 2u;
    const uint32_t b_off = kPieces * kBlockBytes;  // the pair's shadow blocks within a stage

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.n_stages; ++i) {
            ptx::mbar_init(&s.full[i], 2);  // the shadows' and the batch's producers
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.acc_full[i], 1);
            ptx::mbar_init(&s.acc_empty[i], kEpiWarps);
        }
        ptx::mbar_init(s.drain, 1);
        s.ep_go[0] = s.ep_go[1] = 0;
        // W2's padding outputs (d_out .. dpad - 1) stay zero
        const int pad = a.dpad - a.d_out;
        for (int i = 0; i < 2 * a.h * pad; ++i) s.w2t[(i / pad) * a.dpad + a.d_out + i % pad] = 0.0f;
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
            const uint32_t ring = ptx::smem_u32(s.ring);
            uint32_t stage = 0, phase = 0;
            bool ok = true;
            for (int u = 0; ok && 2 * u < count; ++u) {
                const uint32_t n = static_cast<uint32_t>(min(2, count - 2 * u));
                const uint32_t buf = static_cast<uint32_t>(u) & 1u;
                const uint32_t idesc = PREC == 1 ? ptx::idesc_bf16(128, n * static_cast<uint32_t>(a.h))
                                                 : ptx::idesc_e4m3(128, n * static_cast<uint32_t>(a.h));
                if (!ptx::mbar_wait_bounded(&s.acc_empty[buf], ((static_cast<uint32_t>(u) >> 1) & 1u) ^ 1u,
                                            s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t d = tmem_base + buf * kAccStride;
                bool first_mma = true;
                for (int kb = 0; kb < a.k_blocks; ++kb) {
                    if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t sb = ring + stage * a.stage_bytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {  // 32-byte K steps of the 128-byte rows
                        const int kg = kb * (PREC == 1 ? 64 : 128) + kk * (PREC == 1 ? 16 : 32);
                        if (kg >= a.k_mma) break;
                        const uint64_t bd = ptx::smem_desc_sw128(sb + b_off + 32u * kk);
#pragma unroll
                        for (uint32_t q = 0; q < kPieces; ++q) {
                            const uint64_t ad = ptx::smem_desc_sw128(sb + q * kBlockBytes + 32u * kk);
                            if (PREC == 1)
                                ptx::mma_f16(d, ad, bd, idesc, first_mma ? 0u : 1u);
                            else
                                ptx::mma_f8(d, ad, bd, idesc, first_mma ? 0u : 1u);
                            first_mma = false;
                        }
                    }
                    ptx::mma_commit(&s.empty[stage]);
                    if (++stage == static_cast<uint32_t>(a.n_stages)) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                ptx::mma_commit(&s.acc_full[buf]);
            }
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kWaitLimitNs : kDrainLimitNs);
        }
    } else if (warp == 1 || warp == kBatchWarp) {
        // ------------------------------------------------------------ producers
        if (lane == 0) {
            const bool batch = warp == kBatchWarp;
            ptx::grid_dep_wait();  // shadows and masters (breeding) and the staged batch come from earlier kernels
            uint32_t stage = 0, phase = 0, issued_mask = 0, parity_mask = 0;
            bool ok = true;
            const uint8_t* xt = a.xop + static_cast<int64_t>(mt) * a.k_blocks * a.a_bytes;
            for (int u = 0; ok && 2 * u < count; ++u) {
                const int n = min(2, count - 2 * u), p0 = first + 2 * u;
                for (int kb = 0; kb < a.k_blocks; ++kb) {
                    if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    uint8_t* sb = s.ring + stage * a.stage_bytes;
                    if (batch) {
                        ptx::mbar_arrive_expect_tx(&s.full[stage], a.a_bytes);
                        ptx::bulk_load(sb, xt + static_cast<int64_t>(kb) * a.a_bytes, a.a_bytes, &s.full[stage]);
                    } else {
                        ptx::mbar_arrive_expect_tx(&s.full[stage], static_cast<uint32_t>(n) * a.slot_bytes);
                    }
                    for (int j = 0; j < (batch ? 0 : n); ++j)
                        ptx::bulk_load(sb + b_off + j * a.slot_bytes,
                                       a.shadow + static_cast<int64_t>(p0 + j) * a.sh_stride +
                                           static_cast<int64_t>(kb) * a.slot_bytes,
                                       a.slot_bytes, &s.full[stage]);
                    issued_mask |= 1u << stage;
                    parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                    if (++stage == static_cast<uint32_t>(a.n_stages)) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                for (int i = 0; i < a.n_stages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // Per individual of the pair 8 warps: for each TMEM lane quarter one
        // warp of the first half (chains 0 and 1 of layer 2) and one of the
        // second (chains 2 and 3, then the softmax cross-entropy).
        const int ew = warp - kFirstEpiWarp;
        const int g = (ew >> 2) & 1;  // slot: the pair's first or second individual
        const int hh = ew >> 3;       // half: chains 2 hh and 2 hh + 1
        const int q = warp & 3;       // TMEM lane quarter of this warp
        const int et = (hh * 4 + (ew & 3)) * 32 + lane;
        const int row = q * 32 + lane;
        const int srow = mt * 128 + row;  // the sample of this TMEM lane
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        const uint32_t bar_id = 1u + static_cast<uint32_t>(g);
        const int32_t label = hh == 1 && srow < a.batch ? a.y[srow] : 0;
        // Output slots the chains run over, and W2's row stride in shared memory
        // (10 exactly for 10 outputs; else d_out rounded up to 4).
        constexpr int kOutP = DOUT == 0 ? kMaxOut : DOUT;
        static_assert(DOUT == 0 || DOUT == 10, "the fixed-output form is written for 10 outputs");
        const int d_out = DOUT == 0 ? a.d_out : DOUT;
        const int dpad = DOUT == 0 ? a.dpad : 10;
        float* b1 = s.b1 + g * a.h;
        float* b2 = s.b2 + g * 16;
        float* w2t = s.w2t + g * a.h * dpad;
        float* part = s.part + (g * 128 + row) * dpad;
        int* go = s.ep_go + g;
        ptx::grid_dep_wait();  // b1, W2, b2 come from the previous kernel (breeding)
        // b1, W2, b2 of this slot's individual of unit u (as stored after W1),
        // element et + 256 j of each thread, into registers.  Loaded through
        // L2 (ld.global.cg), not the read-only path: this grid starts while
        // the breeding kernel that writes them still runs, and the read-only
        // path assumes data that no grid changes during the kernel's lifetime.
        float prm[kPrmRegs];
        auto load_prm = [&](int u) {
            const int n = min(2, count - 2 * u);
            const float* src =
                a.popv + static_cast<int64_t>(first + 2 * u + g) * a.c_pad + static_cast<int64_t>(a.h) * a.k;
#pragma unroll
            for (int j = 0; j < kPrmRegs; ++j) {
                const int i = et + kGroupThreads * j;
                prm[j] = (2 * u < count && g < n && i < a.n_prm) ? __ldcg(src + i) : 0.0f;
            }
        };
        // The chain of quarter sl: in column order over quarter sl (whole
        // 8-unit groups) of every chunk of cw hidden units, ReLU(D scale + b1)
        // times W2.  A quarter's groups of a chunk are read from TMEM at once;
        // two outputs share each packed FMA (each half an ordinary
        // round-to-nearest FMA, so every chain keeps its bits).
        auto chain = [&](int sl, uint32_t col0, float2 scale2, float2 (&acc)[kOutP / 2]) {
#pragma unroll
            for (int o2 = 0; o2 < kOutP / 2; ++o2) acc[o2] = make_float2(0.0f, 0.0f);
            for (int c = 0; c < a.n_chunks; ++c) {
                const int r0 = c * a.cw, n8 = min(a.cw, a.h - r0) / 8;
                const int g0 = n8 * sl / 4, g1 = n8 * (sl + 1) / 4;
                for (int gg = g0; gg < g1; gg += 2) {
                    const int ng = min(2, g1 - gg);
                    uint32_t d[16];
                    ptx::tmem_ld8_nowait(col0 + static_cast<uint32_t>(r0 + 8 * gg), *reinterpret_cast<uint32_t(*)[8]>(d));
                    if (ng > 1)
                        ptx::tmem_ld8_nowait(col0 + static_cast<uint32_t>(r0 + 8 * gg + 8),
                                             *reinterpret_cast<uint32_t(*)[8]>(d + 8));
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int jj = 0; jj < 16; jj += 4) {
                        if (jj < 8 * ng) {
                            const int col = r0 + 8 * gg + jj;
                            const float4 bb = *reinterpret_cast<const float4*>(b1 + col);
                            const float2 h01 = __ffma2_rn(make_float2(__uint_as_float(d[jj]), __uint_as_float(d[jj + 1])),
                                                          scale2, make_float2(bb.x, bb.y));
                            const float2 h23 = __ffma2_rn(
                                make_float2(__uint_as_float(d[jj + 2]), __uint_as_float(d[jj + 3])), scale2,
                                make_float2(bb.z, bb.w));
                            const float hv[4] = {fmaxf(h01.x, 0.0f), fmaxf(h01.y, 0.0f), fmaxf(h23.x, 0.0f),
                                                 fmaxf(h23.y, 0.0f)};
                            if (DOUT == 10) {
                                // two columns of 10 outputs: five 16-byte loads
#pragma unroll
                                for (int e = 0; e < 4; e += 2) {
                                    const float4* wr = reinterpret_cast<const float4*>(w2t + (col + e) * 10);
                                    float wv[20];
#pragma unroll
                                    for (int v = 0; v < 5; ++v) {
                                        const float4 w = wr[v];
                                        wv[4 * v] = w.x;
                                        wv[4 * v + 1] = w.y;
                                        wv[4 * v + 2] = w.z;
                                        wv[4 * v + 3] = w.w;
                                    }
#pragma unroll
                                    for (int half = 0; half < 2; ++half) {
                                        const float2 hh2 = make_float2(hv[e + half], hv[e + half]);
#pragma unroll
                                        for (int o2 = 0; o2 < 5; ++o2)
                                            acc[o2] = __ffma2_rn(make_float2(wv[10 * half + 2 * o2], wv[10 * half + 2 * o2 + 1]),
                                                                 hh2, acc[o2]);
                                    }
                                }
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const float4* wr = reinterpret_cast<const float4*>(w2t + (col + e) * dpad);
                                    const float2 hh2 = make_float2(hv[e], hv[e]);
#pragma unroll
                                    for (int o4 = 0; o4 < kOutP / 4; ++o4) {
                                        if (4 * o4 < d_out) {
                                            const float4 w = wr[o4];
                                            acc[2 * o4] = __ffma2_rn(make_float2(w.x, w.y), hh2, acc[2 * o4]);
                                            acc[2 * o4 + 1] = __ffma2_rn(make_float2(w.z, w.w), hh2, acc[2 * o4 + 1]);
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
            }
        };
        load_prm(0);
        for (int u = 0; 2 * u < count; ++u) {
            const int n = min(2, count - 2 * u);
            const int p = first + 2 * u + g;
            const uint32_t buf = static_cast<uint32_t>(u) & 1u, bph = (static_cast<uint32_t>(u) >> 1) & 1u;
            if (g < n) {
                // The group finished reading the previous unit's parameters at its barrier B.
#pragma unroll
                for (int j = 0; j < kPrmRegs; ++j) {
                    const int i = et + kGroupThreads * j;
                    if (i < a.h) {
                        b1[i] = prm[j];
                    } else if (i < a.h + d_out * a.h) {
                        const int o = (i - a.h) / a.h, col = (i - a.h) - o * a.h;
                        w2t[col * dpad + o] = prm[j];
                    } else if (i < a.n_prm) {
                        b2[i - a.h - d_out * a.h] = prm[j];
                    }
                }
            }
            load_prm(u + 1);  // in flight while this unit is evaluated
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(&s.acc_full[buf], bph, s.abort_flag, kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *go = got ? 1 : 0;
            }
            ptx::named_barrier_sync(bar_id, kGroupThreads);  // A: accumulator ready (or abort); parameters staged
            if (!*go) break;
            ptx::tc_fence_after();

            // Layer 2 in the order of the chunked shadow evaluation (the
            // batching form's kernel), so that both give the same bits: each
            // output is ((chain 0 + chain 1) + chain 2) + chain 3, then b2.
            float2 c_a[kOutP / 2], c_b[kOutP / 2];
            if (g < n) {
                // D * (w scale / x_div): the FP8 shadow stores w / 2^e.
                const float scale = PREC == 2 ? ldexpf(a.inv_div, a.scale_exp[p]) : a.inv_div;
                const float2 scale2 = make_float2(scale, scale);
                const uint32_t col0 = tmem_base + lane_addr + buf * kAccStride + static_cast<uint32_t>(g * a.h);
                chain(2 * hh, col0, scale2, c_a);
                chain(2 * hh + 1, col0, scale2, c_b);
            }
            // The accumulator is read: release it to the next unit's MMAs.
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.acc_empty[buf]);
            if (hh == 0 && g < n) {
#pragma unroll
                for (int o2 = 0; o2 < kOutP / 2; ++o2)
                    if (DOUT != 0 || 2 * o2 < d_out)
                        reinterpret_cast<float2*>(part)[o2] = make_float2(c_a[o2].x + c_b[o2].x, c_a[o2].y + c_b[o2].y);
            }
            ptx::named_barrier_sync(bar_id, kGroupThreads);  // C: the first half's sums written
            float loss = 0.0f;
            int32_t good = 0;
            if (hh == 1 && g < n && srow < a.batch) {
                float logit[kOutP];
#pragma unroll
                for (int o2 = 0; o2 < kOutP / 2; ++o2) {
                    if (DOUT != 0 || 2 * o2 < d_out) {
                        const float2 v = reinterpret_cast<const float2*>(part)[o2];
                        logit[2 * o2] = ((v.x + c_a[o2].x) + c_b[o2].x) + b2[2 * o2];
                        logit[2 * o2 + 1] = ((v.y + c_a[o2].y) + c_b[o2].y) + b2[2 * o2 + 1];
                    } else {
                        logit[2 * o2] = logit[2 * o2 + 1] = 0.0f;
                    }
                }
                float zmax = logit[0];
                int arg = 0;
#pragma unroll
                for (int o = 1; o < kOutP; ++o)
                    if (o < d_out && logit[o] > zmax) { zmax = logit[o]; arg = o; }
                float se = 0.0f;
#pragma unroll
                for (int o = 0; o < kOutP; ++o)
                    if (o < d_out) se += expf(logit[o] - zmax);
                if (label >= 0 && label < d_out) {
                    float zl = 0.0f;
#pragma unroll
                    for (int o = 0; o < kOutP; ++o)
                        if (o == label) zl = logit[o];
                    loss = logf(se) + zmax - zl;
                    good = (arg == label) ? 1 : 0;
                } else {
                    loss = __int_as_float(0x7FC00000);
                }
            }
            if (hh == 1) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
                    good += __shfl_xor_sync(0xFFFFFFFFu, good, off);
                }
                if (lane == 0) {
                    s.red_loss[g * 4 + q] = loss;
                    s.red_ok[g * 4 + q] = good;
                }
            }
            ptx::named_barrier_sync(bar_id, kGroupThreads);  // B: quarter sums written; staged data no longer read
            if (g < n && et == 128) {
                const float* rl = s.red_loss + g * 4;
                const int32_t* ro = s.red_ok + g * 4;
                const float total = ((rl[0] + rl[1]) + rl[2]) + rl[3];
                const int32_t n_ok = ro[0] + ro[1] + ro[2] + ro[3];
                if (a.m_tiles == 1) {
                    const float f = -(total / static_cast<float>(a.batch));
                    a.f_raw[p] = f;
                    if (a.f_adj) a.f_adj[p] = a.f_inh ? (1.0f - a.alpha) * a.f_inh[p] + a.alpha * f : f;
                    if (a.correct) a.correct[p] = n_ok;
                } else {
                    a.scratch[static_cast<int64_t>(mt) * a.pop + p] = total;
                    a.scratch[static_cast<int64_t>(a.m_tiles + mt) * a.pop + p] = static_cast<float>(n_ok);
                }
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

// Sums each individual's per-tile partial losses in tile order.
__global__ void combine_pair_tiles_kernel(const PairArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.pop) return;
    float total = 0.0f, ok = 0.0f;
    for (int mt = 0; mt < a.m_tiles; ++mt) {
        total += a.scratch[static_cast<int64_t>(mt) * a.pop + p];
        ok += a.scratch[static_cast<int64_t>(a.m_tiles + mt) * a.pop + p];
    }
    const float f = -(total / static_cast<float>(a.batch));
    a.f_raw[p] = f;
    if (a.f_adj) a.f_adj[p] = a.f_inh ? (1.0f - a.alpha) * a.f_inh[p] + a.alpha * f : f;
    if (a.correct) a.correct[p] = static_cast<int32_t>(ok);
}

// The batch as A operand tiles: tile mt, K block kb, piece q at
// xop + ((mt * k_blocks + kb) * pieces + q) * 16 KB; row r (sample mt 128 + r,
// zero past the batch) at 128 r, its 16-byte chunk c at chunk position
// c ^ (r & 7).  BF16: 64 levels per row of a block; FP8: 128 levels, piece 0
// holding 16 floor(k / 16), piece 1 k mod 16, both exact in e4m3.  One thread
// per 16-byte chunk.  It reads only the caller's levels, so it lets the next
// kernel start at once; it waits for its own predecessor before it ends.
template <int PREC>
__global__ void __launch_bounds__(256) stage_xop_kernel(const uint8_t* __restrict__ x, int32_t batch, int32_t k,
                                                        int32_t m_tiles, int32_t k_blocks, uint8_t* __restrict__ xop)
{
    ptx::grid_dep_launch();
    constexpr int kPieces = PREC == 1 ? 1 : 2;
    const int64_t chunks = static_cast<int64_t>(m_tiles) * k_blocks * kPieces * 128 * 8;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < chunks) {
        const int c = static_cast<int>(i & 7);
        const int r = static_cast<int>((i >> 3) & 127);
        const int64_t blk = i >> 10;  // (mt * k_blocks + kb) * pieces + piece
        const int q = static_cast<int>(blk % kPieces);
        const int64_t tb = blk / kPieces;
        const int kb = static_cast<int>(tb % k_blocks);
        const int mt = static_cast<int>(tb / k_blocks);
        const int sample = mt * 128 + r;
        const bool live = sample < batch;
        const uint8_t* xr = x + static_cast<int64_t>(live ? sample : 0) * k;
        uint32_t w[4];
        if (PREC == 1) {
            const int k0 = kb * 64 + c * 8;  // 8 BF16 levels
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float l0 = live && k0 + 2 * e < k ? static_cast<float>(xr[k0 + 2 * e]) : 0.0f;
                const float l1 = live && k0 + 2 * e + 1 < k ? static_cast<float>(xr[k0 + 2 * e + 1]) : 0.0f;
                const __nv_bfloat162 b2v = __floats2bfloat162_rn(l0, l1);
                w[e] = *reinterpret_cast<const uint32_t*>(&b2v);
            }
        } else {
            const int k0 = kb * 128 + c * 16;  // 16 FP8 pieces
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int kk = k0 + 4 * e + b;
                    const uint32_t lv = live && kk < k ? xr[kk] : 0u;
                    const float pv = q == 0 ? static_cast<float>(lv & 0xF0u) : static_cast<float>(lv & 15u);
                    word |= static_cast<uint32_t>(__nv_cvt_float_to_fp8(pv, __NV_SATFINITE, __NV_E4M3)) << (8 * b);
                }
                w[e] = word;
            }
        }
        *reinterpret_cast<uint4*>(xop + blk * kBlockBytes + r * 128 + ((c ^ (r & 7)) << 4)) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
    ptx::grid_dep_wait();
}

}  // namespace

bool eval_shadow_pair_supported(const NetLayout& net, int32_t precision, int32_t batch)
{
    if (net.n_layers != 2 || (precision != 1 && precision != 2) || batch < 1) return false;
    const int32_t k = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    if (k % 16 != 0 || h % 16 != 0 || h > 128 || d_out > kMaxOut) return false;
    // The layer-2 order follows the chunked kernel's chunks, which must exist.
    if (eval_shadow_max_chunk(precision, k) < 16) return false;
    return pair_stages(precision, h, d_out) > 0;
}

size_t eval_shadow_pair_xop_bytes(const NetLayout& net, int32_t precision, int32_t batch)
{
    const int32_t m_tiles = (batch + 127) / 128;
    const int32_t k_blocks = (net.dims[0] + (precision == 1 ? 63 : 127)) / (precision == 1 ? 64 : 128);
    return static_cast<size_t>(m_tiles) * k_blocks * (precision == 1 ? 1 : 2) * kBlockBytes;
}

cudaError_t launch_stage_xop(const NetLayout& net, int32_t precision, const uint8_t* x, int32_t batch, void* xop,
                             cudaStream_t stream)
{
    const int32_t m_tiles = (batch + 127) / 128;
    const int32_t k_blocks = (net.dims[0] + (precision == 1 ? 63 : 127)) / (precision == 1 ? 64 : 128);
    const int64_t chunks = static_cast<int64_t>(m_tiles) * k_blocks * (precision == 1 ? 1 : 2) * 128 * 8;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>((chunks + 255) / 256));
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    uint8_t* dst = static_cast<uint8_t*>(xop);
    return precision == 1 ? cudaLaunchKernelEx(&cfg, stage_xop_kernel<1>, x, batch, net.dims[0], m_tiles, k_blocks, dst)
                          : cudaLaunchKernelEx(&cfg, stage_xop_kernel<2>, x, batch, net.dims[0], m_tiles, k_blocks, dst);
}

cudaError_t launch_eval_shadow_pair(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                                    const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp,
                                    const void* xop, float x_div, const int32_t* y, int32_t batch, float alpha,
                                    const float* f_inh, float* f_raw, float* f_adj, int32_t* correct, float* scratch,
                                    unsigned int* status, cudaStream_t stream)
{
    PairArgs a{};
    a.pop = pop;
    a.k = net.dims[0];
    a.h = net.dims[1];
    a.d_out = net.dims[2];
    // W2's row stride in shared memory: 10 for the fixed 10-output kernel, else
    // d_out rounded up to 4 (16-byte rows).
    a.dpad = a.d_out == 10 ? 10 : (a.d_out + 3) / 4 * 4;
    a.batch = batch;
    a.m_tiles = (batch + 127) / 128;
    a.k_blocks = (a.k + (precision == 1 ? 63 : 127)) / (precision == 1 ? 64 : 128);
    a.k_mma = precision == 1 ? (a.k + 15) / 16 * 16 : (a.k + 31) / 32 * 32;
    a.n_stages = pair_stages(precision, a.h, a.d_out);
    if (a.n_stages == 0) return cudaErrorInvalidValue;
    if (a.m_tiles > 1 && !scratch) return cudaErrorInvalidValue;
    a.n_prm = a.h + a.d_out * a.h + a.d_out;
    {
        // The widest chunk the chunked kernel takes for this net, split evenly (its rule).
        int32_t cw = std::min(eval_shadow_max_chunk(precision, a.k), a.h);
        if (cw < 16) return cudaErrorInvalidValue;
        const int32_t n = (a.h + cw - 1) / cw;
        a.cw = ((a.h + n - 1) / n + 15) / 16 * 16;
        a.n_chunks = (a.h + a.cw - 1) / a.cw;
    }
    a.a_bytes = (precision == 1 ? 1u : 2u) * kBlockBytes;
    a.slot_bytes = static_cast<uint32_t>(a.h) * 128u;
    a.stage_bytes = pair_stage_bytes(precision, a.h);
    a.c_pad = net.c_pad;
    a.sh_stride = sh_stride;
    a.inv_div = static_cast<float>(1.0 / static_cast<double>(x_div));
    a.alpha = alpha;
    a.popv = pop_dev;
    a.shadow = shadow;
    a.scale_exp = scale_exp;
    a.xop = static_cast<const uint8_t*>(xop);
    a.y = y;
    a.f_inh = f_inh;
    a.f_raw = f_raw;
    a.f_adj = f_adj;
    a.correct = correct;
    a.scratch = scratch;
    a.status = status;
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    // Whole groups of m_tiles CTAs (one per tile), no more groups than individuals.
    int groups = sms / a.m_tiles;
    if (groups < 1) groups = 1;
    if (groups > pop) groups = pop;
    a.groups = groups;
    a.per_grp = pop / groups;
    a.extra = pop % groups;
    const size_t smem = pair_smem_bytes(precision, a.h, a.d_out, a.n_stages);
    // The usual 10 outputs get a kernel with d_out fixed at compile time.
    const bool ten = a.d_out == 10;
    const void* kern = precision == 1 ? (ten ? reinterpret_cast<const void*>(eval_shadow_pair_kernel<1, 10>)
                                             : reinterpret_cast<const void*>(eval_shadow_pair_kernel<1, 0>))
                                      : (ten ? reinterpret_cast<const void*>(eval_shadow_pair_kernel<2, 10>)
                                             : reinterpret_cast<const void*>(eval_shadow_pair_kernel<2, 0>));
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    // Programmatic stream serialisation: CTAs may start (barriers, TMEM) while
    // the previous kernel finishes; the producer waits for it before it reads.
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(groups * a.m_tiles);
    cfg.blockDim = dim3(kPairThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (precision == 1)
        err = ten ? cudaLaunchKernelEx(&cfg, eval_shadow_pair_kernel<1, 10>, a)
                  : cudaLaunchKernelEx(&cfg, eval_shadow_pair_kernel<1, 0>, a);
    else
        err = ten ? cudaLaunchKernelEx(&cfg, eval_shadow_pair_kernel<2, 10>, a)
                  : cudaLaunchKernelEx(&cfg, eval_shadow_pair_kernel<2, 0>, a);
    if (err != cudaSuccess || a.m_tiles == 1) return err;
    combine_pair_tiles_kernel<<<(pop + 255) / 256, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace leea
