// leea_eval_shadow.cu -- precision form of the fitness evaluation (Eq. 1;
// Section 3.3): layer 1 reads the BF16 or FP8-e4m3 shadow of W1 that
// breeding writes next to the FP32 master, with FP32 accumulation; the rest
// of the net (b1, W2, b2) and the softmax cross-entropy use the FP32 master.
//
// Inputs are 8-bit levels x = k / x_div.  The A operand (a tile of 128
// samples) is written into tensor memory: for BF16 shadows the levels
// themselves (exact), for FP8 shadows two exact pieces 16 floor(k/16) and
// k mod 16 accumulated by two MMAs.  The B operand, the shadow of W1, is
// stored pre-tiled and pre-swizzled (shadow_offset), so each pipeline stage is
// one contiguous bulk copy of (hidden rows) x 128 bytes straight into the
// layout the tensor core reads.  FP8 products are scaled by the child's
// power-of-two factor 2^scale_exp in the epilogue.
//
// The hidden units are processed in chunks of at most 128 (the accumulator
// shares the 512 TMEM columns with the batch tile); the epilogue keeps each
// sample's partial logits in registers across an individual's chunks.  A
// batch above 128 samples is split into 128-sample tiles handled by
// different CTAs, whose partial loss sums go to scratch memory and are
// combined in tile order by a second kernel.
//
// One kernel serves a single run (the work split arithmetically over the
// grid) and many independent runs at once (the batching form): then each
// CTA walks its own list of segments -- (run, sample tile, range of
// individuals) -- from a device table, reloading the batch tile into TMEM
// when the run or the tile changes.
//
// Warp roles (persistent CTAs, one per SM):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      copy producer: per individual its b1, W2, b2, then per hidden
//               chunk the shadow blocks, by bulk copy
//   warps 2-17  batch tile into TMEM (per segment that needs it); then the
//               epilogue, four warps per TMEM lane quarter, each taking a
//               quarter of a chunk's hidden units.  The accumulator goes to
//               registers at once so that the next chunk's MMAs overlap the
//               epilogue's arithmetic.
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
constexpr int kShPartStride = kShMaxOut + 4;  // floats per sample row of partial logits: 16-byte
                                              // accesses of 8 consecutive rows hit distinct banks
constexpr int kShMaxChunk = 128;   // hidden units per chunk at most
constexpr int kShStageBlocks = 2;  // shadow blocks (128 bytes of every row) per pipeline stage
constexpr int kShRegCols = kShMaxChunk / kShSlots;  // accumulator columns a thread holds
constexpr uint32_t kShTmemCols = 512;
constexpr uint64_t kShWaitNs = 2000000000ull;
constexpr uint64_t kShDrainNs = 200000000ull;

struct EvalShArgs {
    int32_t k, d_out, dpad, k_elems_stage, k_stages, k_mma, stages;
    uint32_t a_col, a_piece_cols, a_total_cols, prm_bytes_max, stage_bytes;
    const ShadowRun* runs;   // many runs: device table; NULL: the single run run0
    const ShadowSeg* segs;   // many runs: CTA b walks segs[seg_off[b] .. seg_off[b+1])
    const int32_t* seg_off;
    ShadowRun run0;
    unsigned int* status;
};

struct ShSmem {
    uint8_t* ring;
    uint8_t* prm_raw;
    float *b2, *part;
    uint64_t *full, *empty, *prm_full, *prm_empty, *acc_full, *acc_empty, *a_ready, *drain;
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
    float* red_loss;
    int32_t* red_ok;
};

__host__ __device__ inline uint32_t sh_prm_bytes(int32_t h, int32_t d_out)
{
    return (static_cast<uint32_t>(h + d_out * h + d_out) * 4u + 15u) & ~15u;
}

size_t sh_smem_bytes(int32_t h_max, int32_t cw_max, int32_t dpad, int32_t stages)
{
    return 1024 + static_cast<size_t>(stages) * kShStageBlocks * cw_max * 128 + 2 * sh_prm_bytes(h_max, dpad) +
           sizeof(float) * (16 + (kShSlots - 1) * 128 * kShPartStride) + 8 * (2 * stages + 8) + 64;
}

__device__ __forceinline__ ShSmem carve(uint8_t* raw, const EvalShArgs& a, int32_t h_max)
{
    ShSmem s;
    s.ring = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    uint8_t* p = s.ring + a.stages * a.stage_bytes;
    s.prm_raw = p;
    p += 2u * a.prm_bytes_max;
    s.b2 = reinterpret_cast<float*>(p);
    p += sizeof(float) * 16;
    s.part = reinterpret_cast<float*>(p);  // [slot 1..3][128][kShPartStride] partial logits
    p += sizeof(float) * (kShSlots - 1) * 128 * kShPartStride;
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.empty = bars + a.stages;
    s.prm_full = bars + 2 * a.stages;
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

__device__ __forceinline__ const ShadowRun& run_of(const EvalShArgs& a, int32_t r)
{
    return a.runs ? a.runs[r] : a.run0;
}

__device__ __forceinline__ int32_t seg_count(const EvalShArgs& a)
{
    return a.runs ? a.seg_off[blockIdx.x + 1] - a.seg_off[blockIdx.x] : 1;
}

// Segment i of this CTA.  A single run splits its m_tiles x pop work over the
// grid: CTA b takes tile b % m_tiles and a contiguous share of the individuals.
__device__ __forceinline__ ShadowSeg seg_at(const EvalShArgs& a, int32_t i)
{
    if (a.runs) return a.segs[a.seg_off[blockIdx.x] + i];
    const int32_t mt = blockIdx.x % a.run0.m_tiles, g = blockIdx.x / a.run0.m_tiles;
    const int32_t groups = gridDim.x / a.run0.m_tiles;
    const int64_t pop = a.run0.pop;
    return ShadowSeg{ 0, mt, static_cast<int32_t>(pop * g / groups), static_cast<int32_t>(pop * (g + 1) / groups) };
}

// Whether segment i needs a batch tile other than the one in TMEM: the first
// non-empty segment, or one whose run or tile differs from the last non-empty one.
__device__ __forceinline__ bool new_tile(const EvalShArgs& a, int32_t i, const ShadowSeg& sg)
{
    for (int32_t j = i - 1; j >= 0; --j) {
        const ShadowSeg prev = seg_at(a, j);
        if (prev.p0 < prev.p1) return prev.run != sg.run || prev.mt != sg.mt;
    }
    return true;
}

__device__ __forceinline__ int32_t chunk_width(const ShadowRun& r, int32_t c)
{
    const int32_t r0 = c * r.cw;
    return r.h - r0 < r.cw ? r.h - r0 : r.cw;
}

// Writes this thread's share of the batch tile (TMEM lane `row`) into the A
// region: 16-column groups [c16_0, c16_1), levels read from global memory 16
// bytes at a time.
template <int PREC>
__device__ __forceinline__ void fill_tile(const EvalShArgs& a, const ShadowRun& r, int32_t mt, int row,
                                          uint32_t c16_0, uint32_t c16_1, uint32_t taddr)
{
    const int32_t srow = mt * 128 + row;
    const bool live = srow < r.batch;
    const uint4* xrow = reinterpret_cast<const uint4*>(r.x + static_cast<int64_t>(live ? srow : 0) * a.k);
    const uint32_t kw = static_cast<uint32_t>(a.k) / 4;  // 32-bit words of levels in a row
    for (uint32_t c16 = c16_0; c16 < c16_1; ++c16) {
        const uint32_t c0 = 16 * c16;
        uint32_t cols[16];
        if (PREC == 1) {
            // columns c0 .. c0+15 hold levels 2 c0 .. 2 c0 + 31: words c0/2 .. c0/2 + 7
            const uint32_t w0 = c0 >> 1;
            uint4 q[2];
#pragma unroll
            for (int t = 0; t < 2; ++t)
                q[t] = (live && w0 + 4 * t < kw) ? __ldg(xrow + (w0 >> 2) + t) : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t wd[8] = { q[0].x, q[0].y, q[0].z, q[0].w, q[1].x, q[1].y, q[1].z, q[1].w };
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const uint32_t pr = wd[i >> 1] >> (16 * (i & 1));
                cols[i] = (__float_as_uint(static_cast<float>(pr & 0xFFu)) >> 16) |
                          (__float_as_uint(static_cast<float>((pr >> 8) & 0xFFu)) & 0xFFFF0000u);
            }
        } else {
            // column c: piece (c >= piece_cols), levels of word c - piece * piece_cols;
            // groups of 4 columns never straddle a piece boundary (piece_cols % 8 == 0).
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4) {
                const uint32_t c = c0 + 4 * g4;
                const bool valid = c < 2u * a.a_piece_cols;
                const uint32_t piece = c >= a.a_piece_cols ? 1u : 0u;
                const uint32_t wi = c - piece * a.a_piece_cols;
                const uint4 q = (live && valid && wi < kw) ? __ldg(xrow + (wi >> 2)) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t wd[4] = { q.x, q.y, q.z, q.w };
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    uint32_t word = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t lv = (wd[t] >> (8 * b)) & 0xFFu;
                        const float pv = piece == 0 ? static_cast<float>(lv & 0xF0u) : static_cast<float>(lv & 15u);
                        word |= e4m3_bits(pv) << (8 * b);
                    }
                    cols[4 * g4 + t] = word;
                }
            }
        }
        ptx::tmem_st16(taddr + c0, cols);
    }
}

template <int PREC>
__global__ void __launch_bounds__(kShThreads, 1)
eval_shadow_kernel(const __grid_constant__ EvalShArgs a, int32_t h_max)
{
    extern __shared__ uint8_t smem_raw[];
    const ShSmem s = carve(smem_raw, a, h_max);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t nseg = seg_count(a);

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
            bool ok = true;
            uint32_t stage = 0, phase = 0, acc_phase = 0, tiles = 0;
            const uint32_t ring = ptx::smem_u32(s.ring);
            for (int32_t si = 0; ok && si < nseg; ++si) {
                const ShadowSeg sg = seg_at(a, si);
                const ShadowRun& r = run_of(a, sg.run);
                if (sg.p0 >= sg.p1) continue;
                if (new_tile(a, si, sg)) {  // the epilogue wrote this segment's batch tile
                    if (!ptx::mbar_wait_bounded(s.a_ready, tiles & 1u, s.abort_flag, kShWaitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ++tiles;
                    ptx::tc_fence_after();
                }
                for (int32_t p = sg.p0; ok && p < sg.p1; ++p) {
                    for (int32_t c = 0; ok && c < r.n_chunks; ++c) {
                        const uint32_t width = static_cast<uint32_t>(chunk_width(r, c));
                        const uint32_t idesc = PREC == 1 ? ptx::idesc_bf16(128, width) : ptx::idesc_e4m3(128, width);
                        if (!ptx::mbar_wait_bounded(s.acc_empty, acc_phase ^ 1u, s.abort_flag, kShWaitNs)) {
                            raise_abort(s, a);
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        bool first = true;
                        for (int kc = 0; kc < a.k_stages; kc += kShStageBlocks) {
                            // Stages are filled by the copy engine (async proxy, like the
                            // MMA's operand reads): the mbarrier completion orders them.
                            if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kShWaitNs)) {
                                raise_abort(s, a);
                                ok = false;
                                break;
                            }
                            for (int blk = 0; blk < kShStageBlocks && kc + blk < a.k_stages; ++blk) {
                            const uint32_t sb = ring + stage * a.stage_bytes + blk * width * 128u;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {  // 4 MMA K-steps of 32 bytes per 128-byte row
                                const int kg = (kc + blk) * a.k_elems_stage + kk * (a.k_elems_stage / 4);
                                if (kg >= a.k_mma) break;
                                const uint64_t bd = ptx::smem_desc_sw128(sb + kk * 32u);
                                if (PREC == 1) {
                                    ptx::mma_f16_tmem_a(tmem_base, tmem_base + a.a_col + static_cast<uint32_t>(kg >> 1),
                                                        bd, idesc, first ? 0u : 1u);
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
                            }
                            ptx::mma_commit(&s.empty[stage]);
                            if (++stage == static_cast<uint32_t>(a.stages)) { stage = 0; phase ^= 1u; }
                        }
                        if (!ok) break;
                        ptx::mma_commit(s.acc_full);
                        acc_phase ^= 1u;
                    }
                }
            }
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kShWaitNs : kShDrainNs);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ copy producer
        if (lane == 0) {
            ptx::grid_dep_wait();  // shadows and masters come from the previous kernel (breeding)
            uint32_t stage = 0, phase = 0, issued_mask = 0, parity_mask = 0, prm_issued = 0;
            bool ok = true;
            for (int32_t si = 0; ok && si < nseg; ++si) {
                const ShadowSeg sg = seg_at(a, si);
                const ShadowRun& r = run_of(a, sg.run);
                const uint32_t prm_bytes = sh_prm_bytes(r.h, a.d_out);
                for (int32_t p = sg.p0; ok && p < sg.p1; ++p) {
                    {
                        const uint32_t pb = prm_issued & 1u, pphase = (prm_issued >> 1) & 1u;
                        if (!ptx::mbar_wait_bounded(&s.prm_empty[pb], pphase ^ 1u, s.abort_flag, kShWaitNs)) {
                            raise_abort(s, a);
                            ok = false;
                            break;
                        }
                        ptx::mbar_arrive_expect_tx(&s.prm_full[pb], prm_bytes);
                        ptx::bulk_load(s.prm_raw + pb * a.prm_bytes_max,
                                       r.popv + static_cast<int64_t>(p) * r.c_pad + static_cast<int64_t>(r.h) * a.k,
                                       prm_bytes, &s.prm_full[pb]);
                        ++prm_issued;
                    }
                    const uint8_t* src = r.shadow + static_cast<int64_t>(p) * r.sh_stride;
                    for (int32_t c = 0; ok && c < r.n_chunks; ++c) {
                        const uint32_t bytes = static_cast<uint32_t>(chunk_width(r, c)) * 128u;
                        for (int kc = 0; kc < a.k_stages; kc += kShStageBlocks) {
                            if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kShWaitNs)) {
                                raise_abort(s, a);
                                ok = false;
                                break;
                            }
                            // rows [c cw, c cw + width) of blocks kc, kc + 1: each contiguous in
                            // the tiled layout, one after the other in the stage
                            const int nb = kc + kShStageBlocks <= a.k_stages ? kShStageBlocks : a.k_stages - kc;
                            ptx::mbar_arrive_expect_tx(&s.full[stage], bytes * static_cast<uint32_t>(nb));
                            for (int blk = 0; blk < nb; ++blk)
                                ptx::bulk_load(s.ring + stage * a.stage_bytes + blk * bytes,
                                               src + (static_cast<int64_t>(kc + blk) * r.h +
                                                      static_cast<int64_t>(c) * r.cw) * 128,
                                               bytes, &s.full[stage]);
                            issued_mask |= 1u << stage;
                            parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                            if (++stage == static_cast<uint32_t>(a.stages)) { stage = 0; phase ^= 1u; }
                        }
                    }
                }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                for (int i = 0; i < a.stages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kShDrainNs);
                for (uint32_t u = prm_issued > 2 ? prm_issued - 2 : 0; u < prm_issued; ++u)
                    ptx::mbar_wait_bounded(&s.prm_full[u & 1u], (u >> 1) & 1u, &never, kShDrainNs);
            }
        }
    } else {
        // ------------------------------------------------------------ batch tiles into TMEM, epilogue
        const int et = threadIdx.x - 32 * kFirstEpiWarp;  // 0 .. kShEpiThreads-1
        const int q = warp & 3;                           // TMEM lane quarter
        const int slot = (warp - kFirstEpiWarp) >> 2;     // which quarter of a chunk's columns
        const int row = q * 32 + lane;
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        const uint32_t n16 = a.a_total_cols / 16;
        bool ok = true;
        uint32_t acc_phase = 0, unit = 0;
        for (int32_t si = 0; ok && si < nseg; ++si) {
            const ShadowSeg sg = seg_at(a, si);
            const ShadowRun& r = run_of(a, sg.run);
            if (sg.p0 >= sg.p1) continue;
            if (new_tile(a, si, sg)) {
                // Every MMA that read the previous tile has completed: its last
                // accumulator was handed over before this point.
                fill_tile<PREC>(a, r, sg.mt, row, n16 * slot / kShSlots, n16 * (slot + 1) / kShSlots,
                                tmem_base + lane_addr + a.a_col);
                ptx::tmem_st_wait();
                ptx::tc_fence_before();
                ptx::mbar_arrive(s.a_ready);
            }
            const int32_t srow = sg.mt * 128 + row;  // sample held by this TMEM lane
            const int32_t label = srow < r.batch ? r.y[srow] : 0;
            for (int32_t p = sg.p0; ok && p < sg.p1; ++p, ++unit) {
                const uint32_t pb = unit & 1u, pphase = (unit >> 1) & 1u;
                if (et == 0) {
                    const bool got = ptx::mbar_wait_bounded(&s.prm_full[pb], pphase, s.abort_flag, kShWaitNs);
                    if (!got) raise_abort(s, a);
                    *s.ep_go = got ? 1 : 0;
                }
                ptx::named_barrier_sync(1, kShEpiThreads);  // A1: parameters landed (or abort)
                if (!*s.ep_go) { ok = false; break; }
                // b1 and W2 (d_out rows of h) are read in place: a thread's columns
                // are contiguous, so 16-byte loads serve 4 hidden units (h % 16 == 0).
                const float* src = reinterpret_cast<const float*>(s.prm_raw + pb * a.prm_bytes_max);
                const float* b1 = src;
                const float* w2 = src + r.h;
                if (et < 16) s.b2[et] = et < a.d_out ? src[r.h + a.d_out * r.h + et] : 0.0f;

                // D * (w_scale / x_div): the FP8 shadow stores w / 2^e.
                const float scale = PREC == 2 ? ldexpf(r.inv_div, r.scale_exp[p]) : r.inv_div;
                float logit[kShMaxOut];
#pragma unroll
                for (int o = 0; o < kShMaxOut; ++o) logit[o] = 0.0f;
                for (int32_t c = 0; ok && c < r.n_chunks; ++c) {
                    if (et == 0) {
                        const bool got = ptx::mbar_wait_bounded(s.acc_full, acc_phase, s.abort_flag, kShWaitNs);
                        if (!got) raise_abort(s, a);
                        *s.ep_go = got ? 1 : 0;
                    }
                    ptx::named_barrier_sync(1, kShEpiThreads);  // A2: accumulator ready; parameters staged
                    if (!*s.ep_go) { ok = false; break; }
                    ptx::tc_fence_after();
                    // This thread's columns: 8-column groups [j0, j1) of the chunk's width / 8,
                    // read into registers at once; then the accumulator is handed back.
                    const int32_t r0 = c * r.cw, n8 = chunk_width(r, c) / 8;
                    const int32_t j0 = n8 * slot / kShSlots, j1 = n8 * (slot + 1) / kShSlots;
                    uint32_t dreg[kShRegCols];
#pragma unroll
                    for (int j = 0; j < kShRegCols / 8; ++j)
                        if (j0 + j < j1)
                            ptx::tmem_ld8_nowait(tmem_base + lane_addr + static_cast<uint32_t>(8 * (j0 + j)),
                                                 *reinterpret_cast<uint32_t(*)[8]>(dreg + 8 * j));
                    ptx::tmem_ld_wait();
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(s.acc_empty);
                    acc_phase ^= 1u;
                    // hidden units col0 .. col0 + ncol - 1: ReLU(D * scale + b1), then
                    // per output its layer-2 sum over them in column order (each
                    // logit accumulates over the hidden units in order across chunks)
                    const int32_t col0 = r0 + 8 * j0, ncol = 8 * (j1 - j0);
                    // (the activations replace the accumulator values in place)
#pragma unroll
                    for (int cc = 0; cc < kShRegCols; cc += 4) {
                        if (cc < ncol) {
                            const float4 b4 = *reinterpret_cast<const float4*>(b1 + col0 + cc);
                            dreg[cc] = __float_as_uint(fmaxf(fmaf(__uint_as_float(dreg[cc]), scale, b4.x), 0.0f));
                            dreg[cc + 1] = __float_as_uint(fmaxf(fmaf(__uint_as_float(dreg[cc + 1]), scale, b4.y), 0.0f));
                            dreg[cc + 2] = __float_as_uint(fmaxf(fmaf(__uint_as_float(dreg[cc + 2]), scale, b4.z), 0.0f));
                            dreg[cc + 3] = __float_as_uint(fmaxf(fmaf(__uint_as_float(dreg[cc + 3]), scale, b4.w), 0.0f));
                        }
                    }
#pragma unroll
                    for (int o = 0; o < kShMaxOut; ++o) {
                        if (o < a.d_out) {
                            const float* wr = w2 + o * r.h + col0;
                            float acc = logit[o];
#pragma unroll
                            for (int cc = 0; cc < kShRegCols; cc += 4) {
                                if (cc < ncol) {
                                    const float4 w = *reinterpret_cast<const float4*>(wr + cc);
                                    acc = fmaf(w.x, __uint_as_float(dreg[cc]), acc);
                                    acc = fmaf(w.y, __uint_as_float(dreg[cc + 1]), acc);
                                    acc = fmaf(w.z, __uint_as_float(dreg[cc + 2]), acc);
                                    acc = fmaf(w.w, __uint_as_float(dreg[cc + 3]), acc);
                                }
                            }
                            logit[o] = acc;
                        }
                    }
                }
                if (!ok) break;
                ptx::mbar_arrive(&s.prm_empty[pb]);  // b1 no longer read

                if (slot) {
                    float4* dst = reinterpret_cast<float4*>(s.part + ((slot - 1) * 128 + row) * kShPartStride);
#pragma unroll
                    for (int o4 = 0; o4 < kShMaxOut / 4; ++o4)
                        dst[o4] = make_float4(logit[4 * o4], logit[4 * o4 + 1], logit[4 * o4 + 2], logit[4 * o4 + 3]);
                }
                ptx::named_barrier_sync(1, kShEpiThreads);  // C: partial logits of slots 1..3 written
                if (!slot) {
                    float loss = 0.0f;
                    int32_t good = 0;
                    if (srow < r.batch) {
#pragma unroll
                        for (int t = 0; t < kShSlots - 1; ++t) {  // slot order 1, 2, 3 per output
                            const float4* srcp = reinterpret_cast<const float4*>(s.part + (t * 128 + row) * kShPartStride);
#pragma unroll
                            for (int o4 = 0; o4 < kShMaxOut / 4; ++o4) {
                                if (4 * o4 < a.d_out) {
                                    const float4 v = srcp[o4];
                                    logit[4 * o4] += v.x;
                                    logit[4 * o4 + 1] += v.y;
                                    logit[4 * o4 + 2] += v.z;
                                    logit[4 * o4 + 3] += v.w;
                                }
                            }
                        }
#pragma unroll
                        for (int o = 0; o < kShMaxOut; ++o) logit[o] += s.b2[o];
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
                    if (r.m_tiles == 1) {
                        const float f = -(total / static_cast<float>(r.batch));
                        r.f_raw[p] = f;
                        if (r.f_adj) r.f_adj[p] = r.f_inh ? (1.0f - r.alpha) * r.f_inh[p] + r.alpha * f : f;
                        if (r.correct) r.correct[p] = n_ok;
                    } else {
                        r.scratch[static_cast<int64_t>(sg.mt) * r.pop + p] = total;
                        r.scratch[static_cast<int64_t>(r.m_tiles + sg.mt) * r.pop + p] = static_cast<float>(n_ok);
                    }
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

// Sums the per-tile partial losses of each individual in tile order; one
// grid row (blockIdx.y) per run, runs with a single tile skipped.
__global__ void combine_tiles_kernel(const __grid_constant__ EvalShArgs a)
{
    const ShadowRun& r = run_of(a, blockIdx.y);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (r.m_tiles < 2 || p >= r.pop) return;
    float total = 0.0f, ok = 0.0f;
    for (int mt = 0; mt < r.m_tiles; ++mt) {
        total += r.scratch[static_cast<int64_t>(mt) * r.pop + p];
        ok += r.scratch[static_cast<int64_t>(r.m_tiles + mt) * r.pop + p];
    }
    const float f = -(total / static_cast<float>(r.batch));
    r.f_raw[p] = f;
    if (r.f_adj) r.f_adj[p] = r.f_inh ? (1.0f - r.alpha) * r.f_inh[p] + r.alpha * f : f;
    if (r.correct) r.correct[p] = static_cast<int32_t>(ok);
}

int32_t sh_stages_for(int32_t h_max, int32_t cw_max, int32_t dpad)
{
    int32_t stages = 8 / kShStageBlocks;
    while (stages > 2 && sh_smem_bytes(h_max, cw_max, dpad, stages) > 227u * 1024u) --stages;
    return stages;
}

// The shared part of the arguments for k = d_0 inputs.
EvalShArgs common_args(int32_t k, int32_t d_out, int32_t precision, int32_t h_max, int32_t cw_max)
{
    EvalShArgs a{};
    a.k = k;
    a.d_out = d_out;
    a.dpad = (d_out + 3) / 4 * 4;
    a.k_elems_stage = precision == 1 ? 64 : 128;
    a.k_stages = (k + a.k_elems_stage - 1) / a.k_elems_stage;
    a.k_mma = precision == 1 ? (k + 15) / 16 * 16 : (k + 31) / 32 * 32;
    a.a_col = static_cast<uint32_t>(cw_max);
    a.a_total_cols = sh_a_cols(precision, k, &a.a_piece_cols);
    a.prm_bytes_max = sh_prm_bytes(h_max, d_out);
    a.stage_bytes = static_cast<uint32_t>(kShStageBlocks * cw_max) * 128u;
    a.stages = sh_stages_for(h_max, cw_max, a.dpad);
    return a;
}

cudaError_t launch(const EvalShArgs& a, int32_t precision, int32_t h_max, int32_t cw_max, int grid,
                   int32_t n_runs, int32_t pop_max, bool any_tiles, cudaStream_t stream)
{
    // At least half of the shared memory, so that one CTA (which holds all 512
    // TMEM columns) is resident per SM.
    size_t smem = sh_smem_bytes(h_max, cw_max, a.dpad, a.stages);
    if (smem < 116u * 1024u) smem = 116u * 1024u;
    auto kernel = precision == 1 ? eval_shadow_kernel<1> : eval_shadow_kernel<2>;
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    // Programmatic stream serialisation: CTAs may start (barriers, TMEM, the
    // batch tile) while the previous kernel finishes; the copy producer waits
    // for it before it reads shadows and masters.
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kShThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    err = cudaLaunchKernelEx(&cfg, kernel, a, h_max);
    if (err != cudaSuccess || !any_tiles) return err;
    combine_tiles_kernel<<<dim3((pop_max + 255) / 256, n_runs), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

int32_t eval_shadow_max_chunk(int32_t precision, int32_t k)
{
    uint32_t piece = 0;
    const uint32_t a_cols = sh_a_cols(precision, k, &piece);
    if (a_cols >= kShTmemCols) return 0;
    int32_t cw = static_cast<int32_t>(kShTmemCols - a_cols) / 16 * 16;
    return cw > kShMaxChunk ? kShMaxChunk : cw;
}

bool eval_shadow_supported(const NetLayout& net, int32_t precision, int32_t batch)
{
    if (net.n_layers != 2 || (precision != 1 && precision != 2)) return false;
    const int32_t k = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    if (k % 16 != 0 || h % 16 != 0 || h > 256 || d_out > kShMaxOut || batch < 1) return false;
    const int32_t cw = eval_shadow_max_chunk(precision, k);
    if (cw < 16) return false;
    const int32_t dpad = (d_out + 3) / 4 * 4;
    return sh_smem_bytes(h, cw, dpad, sh_stages_for(h, cw, dpad)) <= 227u * 1024u;
}

size_t eval_shadow_scratch_bytes(int32_t pop, int32_t batch)
{
    const int32_t m_tiles = (batch + 127) / 128;
    return m_tiles > 1 ? sizeof(float) * 2 * static_cast<size_t>(m_tiles) * pop : 0;
}

ShadowRun shadow_run(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                     const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp, const uint8_t* x,
                     float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                     float* f_adj, int32_t* correct, float* scratch, int32_t chunk)
{
    ShadowRun r{};
    r.pop = pop;
    r.h = net.dims[1];
    r.batch = batch;
    r.m_tiles = (batch + 127) / 128;
    const int32_t cw_max = eval_shadow_max_chunk(precision, net.dims[0]);
    int32_t cw = chunk > 0 && chunk <= cw_max ? chunk : cw_max;
    if (cw > r.h) cw = r.h;
    // Equal chunks when the hidden units need several: ceil(h / n) rounded up to 16.
    const int32_t n = (r.h + cw - 1) / cw;
    r.cw = ((r.h + n - 1) / n + 15) / 16 * 16;
    r.n_chunks = (r.h + r.cw - 1) / r.cw;
    r.c_pad = net.c_pad;
    r.sh_stride = sh_stride;
    r.inv_div = static_cast<float>(1.0 / static_cast<double>(x_div));
    r.alpha = alpha;
    r.popv = pop_dev;
    r.shadow = shadow;
    r.x = x;
    r.y = y;
    r.f_inh = f_inh;
    r.scale_exp = scale_exp;
    r.f_raw = f_raw;
    r.f_adj = f_adj;
    r.correct = correct;
    r.scratch = scratch;
    return r;
}

cudaError_t launch_eval_shadow(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                               const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp,
                               const uint8_t* x, float x_div, const int32_t* y, int32_t batch, float alpha,
                               const float* f_inh, float* f_raw, float* f_adj, int32_t* correct, float* scratch,
                               unsigned int* status, cudaStream_t stream, int32_t chunk)
{
    const ShadowRun r = shadow_run(net, pop, pop_dev, precision, shadow, sh_stride, scale_exp, x, x_div, y, batch,
                                   alpha, f_inh, f_raw, f_adj, correct, scratch, chunk);
    if (r.m_tiles > 1 && !scratch) return cudaErrorInvalidValue;
    EvalShArgs a = common_args(net.dims[0], net.dims[2], precision, r.h, r.cw);
    a.run0 = r;
    a.status = status;
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    // Whole groups of m_tiles CTAs, no more groups than individuals.
    int groups = sms / r.m_tiles;
    if (groups < 1) groups = 1;
    if (groups > pop) groups = pop;
    return launch(a, precision, r.h, r.cw, groups * r.m_tiles, 1, pop, r.m_tiles > 1, stream);
}

cudaError_t launch_combine_shadow_tiles(const ShadowRun* runs_dev, int32_t n_runs, int32_t pop_max,
                                        cudaStream_t stream)
{
    EvalShArgs a{};
    a.runs = runs_dev;
    combine_tiles_kernel<<<dim3((pop_max + 255) / 256, n_runs), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_combine_shadow_run_tiles(const ShadowRun& run, cudaStream_t stream)
{
    EvalShArgs a{};
    a.run0 = run;
    combine_tiles_kernel<<<dim3((run.pop + 255) / 256, 1), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_eval_shadow_runs(int32_t k, int32_t d_out, int32_t precision, int32_t h_max, int32_t cw_max,
                                    int32_t n_runs, int32_t pop_max, bool any_tiles, const ShadowRun* runs_dev,
                                    const ShadowSeg* segs_dev, const int32_t* seg_off_dev, int32_t grid,
                                    unsigned int* status, cudaStream_t stream)
{
    EvalShArgs a = common_args(k, d_out, precision, h_max, cw_max);
    a.runs = runs_dev;
    a.segs = segs_dev;
    a.seg_off = seg_off_dev;
    a.status = status;
    return launch(a, precision, h_max, cw_max, grid, n_runs, pop_max, any_tiles, stream);
}

}  // namespace leea
