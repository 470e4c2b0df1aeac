// leea_eval_shadow.cu -- precision form of the fitness evaluation (Eq. 1;
// Section 3.3): layer 1 reads the BF16 or FP8-e4m3 shadow of W1 that
// breeding writes next to the FP32 master, with FP32 accumulation; the rest
// of the net (b1, W2, b2) and the softmax cross-entropy use the FP32 master.
//
// Inputs are 8-bit levels x = k / x_div.  The A operand (a tile of 128
// samples) is written once per CTA into tensor memory: for BF16 shadows the
// levels themselves (exact), for FP8 shadows two exact pieces 16 floor(k/16)
// and k mod 16 accumulated by two MMAs.  The B operand, the shadow of W1, is
// stored pre-tiled and pre-swizzled (shadow_offset), so each pipeline stage is
// one contiguous bulk copy of h x 128 bytes straight into the layout the
// tensor core reads.  FP8 products are scaled by the child's power-of-two
// factor 2^scale_exp in the epilogue.
//
// A batch above 128 samples is split over groups of CTAs, one 128-sample tile
// per group (each keeps its tile resident in TMEM); the groups write partial
// loss sums to scratch memory and a second kernel combines them in tile order.
//
// Warp roles (persistent CTAs, one per SM):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      copy producer: the batch tile (once), then per individual its
//               b1, W2, b2 and the shadow blocks, by bulk copy
//   warps 2-17  batch tile into TMEM once; then the epilogue, four warps per
//               TMEM lane quarter, each taking a quarter of the hidden units.
//               The accumulator goes to registers at once (h <= 128) so that
//               the next individual's MMAs overlap the epilogue's arithmetic.
// Every mbarrier wait is bounded in time (kStatusEvalTimeout on expiry).
#include <cuda.h>
#include <cuda_fp8.h>

#include "leea_internal.h"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kShSlots = 4;  // epilogue warps per TMEM lane quarter
constexpr int kShEpiWarps = 4 * kShSlots;
constexpr int kShEpiThreads = 32 * kShEpiWarps;
constexpr int kShThreads = 32 * (2 + kShEpiWarps);
constexpr int kFirstEpiWarp = 2;
constexpr int kShMaxOut = 16;
constexpr int kShStages = 8;
constexpr int kShRegCols = 32;  // accumulator columns a thread holds in registers (h <= 128)
constexpr uint32_t kShTmemCols = 512;
constexpr uint64_t kShWaitNs = 2000000000ull;
constexpr uint64_t kShDrainNs = 200000000ull;

struct EvalShArgs {
    int32_t pop, k, h, d_out, dpad, batch, precision, k_elems_stage, k_stages, k_mma, m_tiles, stages;
    int64_t c_pad, sh_stride;
    float inv_div, alpha;
    uint32_t a_col, a_piece_cols, a_total_cols, prm_bytes, ring_bytes;
    const float* popv;
    const uint8_t* shadow;
    const uint8_t* x;
    const int32_t* y;
    const float* f_inh;
    const int32_t* scale_exp;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    float* scratch;  // m_tiles > 1: [m_tiles][pop] loss sums, then [m_tiles][pop] correct counts
    unsigned int* status;
};

struct ShSmem {
    uint8_t* ring;  // also holds the batch tile before the first stage
    uint32_t stage_bytes;
    uint8_t* prm_raw;
    float *w2t, *b2, *part;
    uint64_t *full, *empty, *prm_full, *prm_empty, *acc_full, *acc_empty, *a_ready, *drain, *x_full;
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
    float* red_loss;
    int32_t* red_ok;
};

uint32_t sh_prm_bytes(int32_t h, int32_t d_out)
{
    return (static_cast<uint32_t>(h + d_out * h + d_out) * 4u + 15u) & ~15u;
}

uint32_t sh_ring_bytes(int32_t h, int32_t k, int32_t stages)
{
    const uint32_t ring = static_cast<uint32_t>(stages) * h * 128u, xtile = 128u * static_cast<uint32_t>(k);
    return ring > xtile ? ring : xtile;
}

size_t sh_smem_bytes(int32_t h, int32_t k, int32_t dpad, int32_t stages)
{
    return 1024 + sh_ring_bytes(h, k, stages) + 2 * sh_prm_bytes(h, dpad) +
           sizeof(float) * (h * dpad + 16 + (kShSlots - 1) * 128 * kShMaxOut) + 8 * (2 * stages + 9) + 64;
}

__device__ __forceinline__ ShSmem carve(uint8_t* raw, const EvalShArgs& a)
{
    ShSmem s;
    s.ring = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    s.stage_bytes = static_cast<uint32_t>(a.h) * 128u;
    uint8_t* p = s.ring + a.ring_bytes;
    s.prm_raw = p;
    p += 2u * a.prm_bytes;
    s.w2t = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.h * a.dpad;
    s.b2 = reinterpret_cast<float*>(p);
    p += sizeof(float) * 16;
    s.part = reinterpret_cast<float*>(p);  // [slot 1..3][128][kShMaxOut] partial logits
    p += sizeof(float) * (kShSlots - 1) * 128 * kShMaxOut;
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.empty = bars + a.stages;
    s.prm_full = bars + 2 * a.stages;
    s.prm_empty = s.prm_full + 2;
    s.acc_full = s.prm_empty + 2;
    s.acc_empty = s.acc_full + 1;
    s.a_ready = s.acc_full + 2;
    s.drain = s.acc_full + 3;
    s.x_full = s.acc_full + 4;
    uint32_t* w = reinterpret_cast<uint32_t*>(s.acc_full + 5);
    s.tmem_holder = w;
    s.abort_flag = reinterpret_cast<volatile int*>(w + 1);
    s.ep_go = reinterpret_cast<int*>(w + 2);
    s.red_loss = reinterpret_cast<float*>(w + 4);
    s.red_ok = reinterpret_cast<int32_t*>(w + 8);
    return s;
}

// TMEM columns the A operand needs, rounded to whole 16-column stores: BF16
// holds two levels per column; FP8 two pieces of four levels per column.
uint32_t sh_a_cols(int32_t precision, int32_t k, uint32_t* piece_cols)
{
    if (precision == 1) {
        *piece_cols = 0;
        return ((static_cast<uint32_t>((k + 15) / 16) * 8u) + 15u) & ~15u;
    }
    *piece_cols = static_cast<uint32_t>((k + 31) / 32) * 8u;
    return (2u * *piece_cols + 15u) & ~15u;
}

__device__ __forceinline__ void raise_abort(const ShSmem& s, const EvalShArgs& a)
{
    *s.abort_flag = 1;
    atomicOr(a.status, kStatusEvalTimeout);
}

__device__ __forceinline__ uint32_t e4m3_bits(float v)
{
    return static_cast<uint32_t>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
}

template <int PREC>
__global__ void __launch_bounds__(kShThreads, 1)
eval_shadow_kernel(const EvalShArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const ShSmem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x % a.m_tiles;  // this CTA's 128-sample tile
    const int g = blockIdx.x / a.m_tiles;   // individuals g, g + groups, ...
    const int groups = gridDim.x / a.m_tiles;
    const int tile_rows = min(128, a.batch - mt * 128);

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.stages; ++i) {
            ptx::mbar_init(&s.full[i], 1);
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.prm_full[i], 1);
            ptx::mbar_init(&s.prm_empty[i], kShEpiThreads);
        }
        ptx::mbar_init(s.acc_full, 1);
        ptx::mbar_init(s.acc_empty, kShEpiThreads);
        ptx::mbar_init(s.a_ready, kShEpiThreads);
        ptx::mbar_init(s.drain, 1);
        ptx::mbar_init(s.x_full, 1);
        *s.abort_flag = 0;
        *s.ep_go = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 0) ptx::tmem_alloc(s.tmem_holder, kShTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *s.tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = PREC == 1 ? ptx::idesc_bf16(128, static_cast<uint32_t>(a.h))
                                             : ptx::idesc_e4m3(128, static_cast<uint32_t>(a.h));
            bool ok = ptx::mbar_wait_bounded(s.a_ready, 0u, s.abort_flag, kShWaitNs);
            if (!ok) raise_abort(s, a);
            ptx::tc_fence_after();
            uint32_t stage = 0, phase = 0, acc_phase = 0;
            const uint32_t ring = ptx::smem_u32(s.ring);
            for (int p = g; ok && p < a.pop; p += groups) {
                if (!ptx::mbar_wait_bounded(s.acc_empty, acc_phase ^ 1u, s.abort_flag, kShWaitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                bool first = true;
                for (int kc = 0; kc < a.k_stages; ++kc) {
                    // The stage was filled by the copy engine (async proxy, like the
                    // MMA's operand reads): the mbarrier completion orders it.
                    if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kShWaitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    const uint32_t sb = ring + stage * s.stage_bytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {  // 4 MMA K-steps of 32 bytes per 128-byte row
                        const int kg = kc * a.k_elems_stage + kk * (a.k_elems_stage / 4);
                        if (kg >= a.k_mma) break;
                        const uint64_t bd = ptx::smem_desc_sw128(sb + kk * 32u);
                        if (PREC == 1) {
                            ptx::mma_f16_tmem_a(tmem_base, tmem_base + a.a_col + static_cast<uint32_t>(kg >> 1), bd,
                                                idesc, first ? 0u : 1u);
                            first = false;
                        } else {
#pragma unroll
                            for (int piece = 0; piece < 2; ++piece) {
                                const uint32_t at = tmem_base + a.a_col + piece * a.a_piece_cols +
                                                    static_cast<uint32_t>(kg >> 2);
                                ptx::mma_f8_tmem_a(tmem_base, at, bd, idesc, first ? 0u : 1u);
                                first = false;
                            }
                        }
                    }
                    ptx::mma_commit(&s.empty[stage]);
                    if (++stage == static_cast<uint32_t>(a.stages)) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                ptx::mma_commit(s.acc_full);
                acc_phase ^= 1u;
            }
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kShWaitNs : kShDrainNs);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ copy producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, issued_mask = 0, parity_mask = 0, prm_issued = 0;
            bool ok = true;
            // The batch tile (rows mt*128 .. +tile_rows, d_0 bytes each) into the ring.
            const uint32_t x_bytes = static_cast<uint32_t>(tile_rows) * static_cast<uint32_t>(a.k);
            ptx::mbar_arrive_expect_tx(s.x_full, x_bytes);
            ptx::bulk_load(s.ring, a.x + static_cast<int64_t>(mt) * 128 * a.k, x_bytes, s.x_full);
            // The ring is free again once the tile sits in TMEM.
            if (!ptx::mbar_wait_bounded(s.a_ready, 0u, s.abort_flag, kShWaitNs)) {
                raise_abort(s, a);
                ok = false;
            }
            for (int p = g; ok && p < a.pop; p += groups) {
                {
                    const uint32_t pb = prm_issued & 1u, pphase = (prm_issued >> 1) & 1u;
                    if (!ptx::mbar_wait_bounded(&s.prm_empty[pb], pphase ^ 1u, s.abort_flag, kShWaitNs)) {
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
                const uint8_t* src = a.shadow + static_cast<int64_t>(p) * a.sh_stride;
                for (int kc = 0; kc < a.k_stages; ++kc) {
                    if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kShWaitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&s.full[stage], s.stage_bytes);
                    ptx::bulk_load(s.ring + stage * s.stage_bytes, src + static_cast<int64_t>(kc) * s.stage_bytes,
                                   s.stage_bytes, &s.full[stage]);
                    issued_mask |= 1u << stage;
                    parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                    if (++stage == static_cast<uint32_t>(a.stages)) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                ptx::mbar_wait_bounded(s.x_full, 0u, &never, kShDrainNs);
                for (int i = 0; i < a.stages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kShDrainNs);
                for (uint32_t u = prm_issued > 2 ? prm_issued - 2 : 0; u < prm_issued; ++u)
                    ptx::mbar_wait_bounded(&s.prm_full[u & 1u], (u >> 1) & 1u, &never, kShDrainNs);
            }
        }
    } else {
        // ------------------------------------------------------------ batch tile into TMEM, then epilogue
        const int et = threadIdx.x - 32 * kFirstEpiWarp;  // 0 .. kShEpiThreads-1
        const int q = warp & 3;                           // TMEM lane quarter
        const int slot = (warp - kFirstEpiWarp) >> 2;     // which quarter of the columns
        const int row = q * 32 + lane;
        const int srow = mt * 128 + row;  // sample held by this TMEM lane
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        bool ok = ptx::mbar_wait_bounded(s.x_full, 0u, s.abort_flag, kShWaitNs);
        if (!ok) raise_abort(s, a);
        {
            // Levels 4i .. 4i+3 of this row from the staged tile (zero outside).
            const uint32_t* xrow = reinterpret_cast<const uint32_t*>(s.ring + static_cast<size_t>(row) * a.k);
            const bool live = ok && row < tile_rows;
            const uint32_t n16 = a.a_total_cols / 16, c16_0 = n16 * slot / kShSlots,
                           c16_1 = n16 * (slot + 1) / kShSlots;
            for (uint32_t c16 = c16_0; c16 < c16_1; ++c16) {
                const uint32_t c0 = 16 * c16;
                uint32_t cols[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const uint32_t c = c0 + i;
                    uint32_t word = 0;
                    if (PREC == 1) {  // levels 2c, 2c+1 as BF16 (exact)
                        const uint32_t wi = c >> 1;
                        const uint32_t lw = (live && 4 * wi < static_cast<uint32_t>(a.k)) ? xrow[wi] : 0u;
                        const uint32_t pr = lw >> (16 * (c & 1u));
                        word = (__float_as_uint(static_cast<float>(pr & 0xFFu)) >> 16) |
                               (__float_as_uint(static_cast<float>((pr >> 8) & 0xFFu)) & 0xFFFF0000u);
                    } else if (c < 2u * a.a_piece_cols) {  // piece 0: 16 floor(k/16); piece 1: k mod 16
                        const uint32_t piece = c >= a.a_piece_cols ? 1u : 0u;
                        const uint32_t wi = c - piece * a.a_piece_cols;
                        const uint32_t lw = (live && 4 * wi < static_cast<uint32_t>(a.k)) ? xrow[wi] : 0u;
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const uint32_t lv = (lw >> (8 * t)) & 0xFFu;
                            const float pv = piece == 0 ? static_cast<float>(lv & 0xF0u) : static_cast<float>(lv & 15u);
                            word |= e4m3_bits(pv) << (8 * t);
                        }
                    }
                    cols[i] = word;
                }
                ptx::tmem_st16(tmem_base + lane_addr + a.a_col + c0, cols);
            }
        }
        ptx::tmem_st_wait();
        ptx::tc_fence_before();
        ptx::mbar_arrive(s.a_ready);

        const int32_t label = srow < a.batch ? a.y[srow] : 0;
        // This thread's accumulator columns: 8-column chunks [j0, j1) of the h / 8.
        const int n8 = a.h / 8, j0 = n8 * slot / kShSlots, j1 = n8 * (slot + 1) / kShSlots;
        uint32_t acc_phase = 0, unit = 0;
        for (int p = g; ok && p < a.pop; p += groups, ++unit) {
            const uint32_t pb = unit & 1u, pphase = (unit >> 1) & 1u;
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(&s.prm_full[pb], pphase, s.abort_flag, kShWaitNs);
                if (!got) raise_abort(s, a);
                *s.ep_go = got ? 1 : 0;
            }
            ptx::named_barrier_sync(1, kShEpiThreads);  // A1: parameters landed (or abort)
            if (!*s.ep_go) { ok = false; break; }
            // b1 is read in place; W2 (d_out rows of h) is staged transposed,
            // one hidden unit (column) per thread.
            const float* src = reinterpret_cast<const float*>(s.prm_raw + pb * a.prm_bytes);
            const float* b1 = src;
            for (int col = et; col < a.h; col += kShEpiThreads) {
                float4* dst = reinterpret_cast<float4*>(s.w2t + col * a.dpad);
                for (int o4 = 0; o4 < a.dpad / 4; ++o4) {
                    float v[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int o = 4 * o4 + t;
                        v[t] = o < a.d_out ? src[a.h + o * a.h + col] : 0.0f;
                    }
                    dst[o4] = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
            if (et < 16) s.b2[et] = et < a.d_out ? src[a.h + a.d_out * a.h + et] : 0.0f;
            if (et == 0) {
                const bool got = ptx::mbar_wait_bounded(s.acc_full, acc_phase, s.abort_flag, kShWaitNs);
                if (!got) raise_abort(s, a);
                *s.ep_go = got ? 1 : 0;
            }
            ptx::named_barrier_sync(1, kShEpiThreads);  // A2: accumulator ready (or abort); parameters staged
            if (!*s.ep_go) { ok = false; break; }
            ptx::tc_fence_after();

            // D * (w_scale / x_div): the FP8 shadow stores w / 2^e.
            const float scale = PREC == 2 ? ldexpf(a.inv_div, a.scale_exp[p]) : a.inv_div;
            float logit[kShMaxOut];
#pragma unroll
            for (int o = 0; o < kShMaxOut; ++o) logit[o] = 0.0f;
            // hidden unit col: ReLU(D * scale + b1), then its layer-2 contributions
            auto hidden = [&](int col, float d) {
                const float hv = fmaxf(fmaf(d, scale, b1[col]), 0.0f);
                const float4* wr = reinterpret_cast<const float4*>(s.w2t + col * a.dpad);
#pragma unroll
                for (int o4 = 0; o4 < kShMaxOut / 4; ++o4) {
                    if (4 * o4 < a.d_out) {
                        const float4 w = wr[o4];
                        logit[4 * o4 + 0] = fmaf(w.x, hv, logit[4 * o4 + 0]);
                        logit[4 * o4 + 1] = fmaf(w.y, hv, logit[4 * o4 + 1]);
                        logit[4 * o4 + 2] = fmaf(w.z, hv, logit[4 * o4 + 2]);
                        logit[4 * o4 + 3] = fmaf(w.w, hv, logit[4 * o4 + 3]);
                    }
                }
            };
            if (j1 - j0 <= kShRegCols / 8) {
                // This thread's accumulator columns into registers, then hand the
                // accumulator back so the next individual's MMAs overlap this math.
                uint32_t dreg[kShRegCols];
#pragma unroll
                for (int j = 0; j < kShRegCols / 8; ++j)
                    if (j0 + j < j1)
                        ptx::tmem_ld8_nowait(tmem_base + lane_addr + static_cast<uint32_t>(8 * (j0 + j)),
                                             *reinterpret_cast<uint32_t(*)[8]>(dreg + 8 * j));
                ptx::tmem_ld_wait();
                ptx::tc_fence_before();
                ptx::mbar_arrive(s.acc_empty);
#pragma unroll
                for (int c = 0; c < kShRegCols; ++c)
                    if (j0 + c / 8 < j1) hidden(8 * j0 + c, __uint_as_float(dreg[c]));
            } else {
                for (int j = j0; j < j1; ++j) {
                    uint32_t r8[8];
                    ptx::tmem_ld8_nowait(tmem_base + lane_addr + static_cast<uint32_t>(8 * j), r8);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int t = 0; t < 8; ++t) hidden(8 * j + t, __uint_as_float(r8[t]));
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(s.acc_empty);
            }
            acc_phase ^= 1u;
            ptx::mbar_arrive(&s.prm_empty[pb]);  // b1 no longer read

            if (slot) {
                float4* dst = reinterpret_cast<float4*>(s.part + ((slot - 1) * 128 + row) * kShMaxOut);
#pragma unroll
                for (int o4 = 0; o4 < kShMaxOut / 4; ++o4)
                    dst[o4] = make_float4(logit[4 * o4], logit[4 * o4 + 1], logit[4 * o4 + 2], logit[4 * o4 + 3]);
            }
            ptx::named_barrier_sync(1, kShEpiThreads);  // C: partial logits of slots 1..3 written
            if (!slot) {
                float loss = 0.0f;
                int32_t good = 0;
                if (srow < a.batch) {
#pragma unroll
                    for (int o = 0; o < kShMaxOut; ++o) {
                        float z = logit[o];
#pragma unroll
                        for (int r = 0; r < kShSlots - 1; ++r) z += s.part[(r * 128 + row) * kShMaxOut + o];
                        logit[o] = z + s.b2[o];
                    }
                    float zmax = logit[0];
                    int arg = 0;
#pragma unroll
                    for (int o = 1; o < kShMaxOut; ++o) {
                        if (o < a.d_out && logit[o] > zmax) { zmax = logit[o]; arg = o; }
                    }
                    float se = 0.0f;
#pragma unroll
                    for (int o = 0; o < kShMaxOut; ++o)
                        if (o < a.d_out) se += expf(logit[o] - zmax);
                    if (label >= 0 && label < a.d_out) {
                        float zl = 0.0f;
#pragma unroll
                        for (int o = 0; o < kShMaxOut; ++o)
                            if (o == label) zl = logit[o];
                        loss = logf(se) + zmax - zl;
                        good = (arg == label) ? 1 : 0;
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
            }
            ptx::named_barrier_sync(1, kShEpiThreads);  // B: quarter sums written; staged data no longer read
            if (et == 0) {
                const float total = ((s.red_loss[0] + s.red_loss[1]) + s.red_loss[2]) + s.red_loss[3];
                const int32_t n_ok = s.red_ok[0] + s.red_ok[1] + s.red_ok[2] + s.red_ok[3];
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
        ptx::tmem_dealloc(tmem_base, kShTmemCols);
    }
}

// Sums the per-tile partial losses of each individual in tile order.
__global__ void combine_tiles_kernel(int32_t pop, int32_t m_tiles, int32_t batch, float alpha,
                                     const float* __restrict__ scratch, const float* __restrict__ f_inh,
                                     float* __restrict__ f_raw, float* __restrict__ f_adj,
                                     int32_t* __restrict__ correct)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pop) return;
    float total = 0.0f, ok = 0.0f;
    for (int mt = 0; mt < m_tiles; ++mt) {
        total += scratch[static_cast<int64_t>(mt) * pop + p];
        ok += scratch[static_cast<int64_t>(m_tiles + mt) * pop + p];
    }
    const float f = -(total / static_cast<float>(batch));
    f_raw[p] = f;
    if (f_adj) f_adj[p] = f_inh ? (1.0f - alpha) * f_inh[p] + alpha * f : f;
    if (correct) correct[p] = static_cast<int32_t>(ok);
}

int32_t sh_stages_for(int32_t h, int32_t k, int32_t dpad)
{
    int32_t stages = kShStages;
    while (stages > 2 && sh_smem_bytes(h, k, dpad, stages) > 227u * 1024u) --stages;
    return stages;
}

}  // namespace

bool eval_shadow_supported(const NetLayout& net, int32_t precision, int32_t batch)
{
    if (net.n_layers != 2 || (precision != 1 && precision != 2)) return false;
    const int32_t k = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    if (k % 16 != 0 || h % 16 != 0 || h > 256 || d_out > kShMaxOut || batch < 1) return false;
    uint32_t piece = 0;
    if (static_cast<uint32_t>(h) + sh_a_cols(precision, k, &piece) > kShTmemCols) return false;
    const int32_t dpad = (d_out + 3) / 4 * 4;
    return sh_smem_bytes(h, k, dpad, sh_stages_for(h, k, dpad)) <= 227u * 1024u;
}

size_t eval_shadow_scratch_bytes(int32_t pop, int32_t batch)
{
    const int32_t m_tiles = (batch + 127) / 128;
    return m_tiles > 1 ? sizeof(float) * 2 * static_cast<size_t>(m_tiles) * pop : 0;
}

cudaError_t launch_eval_shadow(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                               const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp,
                               const uint8_t* x, float x_div, const int32_t* y, int32_t batch, float alpha,
                               const float* f_inh, float* f_raw, float* f_adj, int32_t* correct, float* scratch,
                               unsigned int* status, cudaStream_t stream)
{
    EvalShArgs a{};
    a.pop = pop;
    a.k = net.dims[0];
    a.h = net.dims[1];
    a.d_out = net.dims[2];
    a.dpad = (a.d_out + 3) / 4 * 4;
    a.batch = batch;
    a.precision = precision;
    a.k_elems_stage = precision == 1 ? 64 : 128;
    a.k_stages = (a.k + a.k_elems_stage - 1) / a.k_elems_stage;
    a.k_mma = precision == 1 ? (a.k + 15) / 16 * 16 : (a.k + 31) / 32 * 32;
    a.m_tiles = (batch + 127) / 128;
    a.c_pad = net.c_pad;
    a.sh_stride = sh_stride;
    a.inv_div = static_cast<float>(1.0 / static_cast<double>(x_div));
    a.alpha = alpha;
    a.a_col = static_cast<uint32_t>(a.h);
    a.a_total_cols = sh_a_cols(precision, a.k, &a.a_piece_cols);
    a.prm_bytes = sh_prm_bytes(a.h, a.d_out);
    a.popv = pop_dev;
    a.shadow = shadow;
    a.x = x;
    a.y = y;
    a.f_inh = f_inh;
    a.scale_exp = scale_exp;
    a.f_raw = f_raw;
    a.f_adj = f_adj;
    a.correct = correct;
    a.scratch = scratch;
    a.status = status;
    if (a.m_tiles > 1 && !scratch) return cudaErrorInvalidValue;
    a.stages = sh_stages_for(a.h, a.k, a.dpad);
    a.ring_bytes = sh_ring_bytes(a.h, a.k, a.stages);
    // At least half of the shared memory, so that one CTA (which holds all 512
    // TMEM columns) is resident per SM.
    size_t smem = sh_smem_bytes(a.h, a.k, a.dpad, a.stages);
    if (smem < 116u * 1024u) smem = 116u * 1024u;

    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    auto kernel = precision == 1 ? eval_shadow_kernel<1> : eval_shadow_kernel<2>;
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    // Whole groups of m_tiles CTAs, no more groups than individuals.
    int groups = sms / a.m_tiles;
    if (groups < 1) groups = 1;
    if (groups > pop) groups = pop;
    kernel<<<groups * a.m_tiles, kShThreads, smem, stream>>>(a);
    err = cudaGetLastError();
    if (err != cudaSuccess || a.m_tiles == 1) return err;
    combine_tiles_kernel<<<(pop + 255) / 256, 256, 0, stream>>>(pop, a.m_tiles, batch, alpha, scratch, f_inh, f_raw,
                                                               f_adj, correct);
    return cudaGetLastError();
}

}  // namespace leea
