// leea_eval_shadow_group.cu -- the batching form's fitness evaluation (Eq. 1;
// Sections 3.3 and 3.3's batched evaluation extended to many runs): layer 1
// on the BF16 or FP8-e4m3 shadows of W1 with FP32 accumulation, several
// individuals of a run per tcgen05 MMA; b1, W2, b2 and the softmax
// cross-entropy in FP32 from the masters.
//
// A tcgen05.mma of M = 128 costs about the same for any N up to 256, so a
// run of hidden width h puts group = min(16, 256 / h) individuals side by
// side in N (their pre-tiled shadow blocks stacked as the B operand); the
// 128-sample batch tile is the A operand, staged once per evaluation as
// 128-byte-swizzled operand tiles (launch_stage_xop_tiles) and streamed from
// L2.  An individual of h up to 256 thus needs one pass over K (the chunked
// kernel, whose batch tile sits in TMEM, needs up to three).
//
// Work: one launch over a table of runs and a table of units (at most
// `group` individuals of a run on one sample tile, the tiles of a group
// next to each other so that the second tile finds the shadows in L2).
// CTAs take units dynamically: the shadow producer's lane 0 claims the next
// unit index with an atomic add, one unit ahead of its own work, and hands
// it to the CTA's other roles through a ring of unit slots in shared memory
// (each slot with a full and an empty mbarrier).  A single run (the state
// object's precision form for h above 128) comes by value, its units
// computed from their index.
// Warp roles (one CTA per SM):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      shadow producer: lane j copies individual j's block of each
//               stage (one thread's bulk copies complete about one at a
//               time, so each individual's stream gets its own lane)
//   warp 18     batch producer: the tile's block of each stage
//   warps 2-17  epilogue, 4 per TMEM lane quarter.  Layer 2 runs as four
//               FP32 chains per output, chain sl over quarter sl (whole
//               8-unit groups) of every hidden chunk the chunked kernel would
//               use, added in quarter order, then b2 -- the chunked kernel's
//               order, so both give the same bits.  A unit of three or more
//               individuals gives each warp whole individuals; a unit of one
//               or two splits each individual's chains over two warps: one
//               sums chains 0 and 1 and finishes the individual, the other
//               passes chains 2 and 3 through shared memory.  Accumulators
//               double-buffered in TMEM (columns 0 and 256).  Registers (96
//               per thread at 608 threads) decide the shapes here: weights
//               are read one column at a time and TMEM one 8-column group at
//               a time, so that nothing spills; spilled values went to L2,
//               since shared memory leaves the L1 little room.
// Batches above 128 samples: tiles on different CTAs, partial sums through
// scratch, combined in tile order by launch_combine_shadow_tiles.  Every
// mbarrier wait is bounded in time; on expiry the kernel sets
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
constexpr int kEpiWarps = 16;                           // 4 per TMEM lane quarter
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kBatchWarp = kFirstEpiWarp + kEpiWarps;  // the batch's producer
constexpr int kGroupThreads = 32 * (kBatchWarp + 1);
constexpr int kMaxOut = 16;
constexpr int kMaxN = 256;    // accumulator columns of one unit
constexpr int kMaxGroup = 16;  // individuals of one unit (h >= 16)
constexpr int kMaxSplit = 2;   // units of at most this many individuals split each one's chains
constexpr int kPrmRegs = 9;    // b1, W2, b2 floats per epilogue thread: ceil((256 (1 + 16) + 16 16) / 512)
constexpr int kFullArrivals = 33;  // the shadow producer's 32 lanes and the batch producer
constexpr int kURing = 8;          // unit slots
constexpr int kUnitReaders = 3;    // the MMA thread, the batch producer, the epilogue
constexpr int kMinStages = 2;
constexpr int kMaxStages = 6;
constexpr uint32_t kBlockBytes = 128u * 128u;  // a 128-row operand block of 128-byte rows
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct GroupArgs {
    int32_t k, d_out, dpad, k_blocks, k_mma, n_stages;
    uint32_t a_bytes, stage_bytes;
    const ShadowRun* runs;    // many runs: device table; NULL: the single run run0
    ShadowRun run0;
    const GroupUnit* units;   // many runs: device table; NULL: unit i of run0 is (i / m_tiles, i % m_tiles)
    int32_t n_units;
    int32_t* sched;  // [0] next unit, [1] CTAs that found no more
    unsigned int* status;
};

struct GroupSmem {
    uint8_t* ring;       // n_stages x stage_bytes: the batch block(s), then the unit's shadow blocks
    float* w2t;          // [kMaxN columns of the unit][dpad]
    float* b1;           // [kMaxN]
    float* b2;           // [kMaxGroup][16]
    float* part;         // [kMaxSplit][128 rows][2][dpad]: the second half's chains (split units)
    float* red_loss;     // [kMaxGroup][4]
    int32_t* red_ok;     // [kMaxGroup][4]
    int* ep_go;
    int32_t* ep_next;    // [2]: the epilogue's unit indices, slot = unit parity
    int32_t* uidx;       // [kURing] unit slots
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    uint64_t *full, *empty, *acc_full, *acc_empty, *drain, *ufull, *uempty;
};

size_t group_tail_bytes(int32_t dpad, int32_t n_stages)
{
    return sizeof(float) * (static_cast<size_t>(kMaxN) * dpad + kMaxN + kMaxGroup * 16 +
                            static_cast<size_t>(kMaxSplit) * 128 * 2 * dpad + kMaxGroup * 4) +
           sizeof(int32_t) * kMaxGroup * 4 + 48u + sizeof(int32_t) * kURing + 8u * (2u * n_stages + 5u + 2u * kURing) +
           64u;
}

uint32_t group_stage_bytes(int32_t precision, int32_t n_max)
{
    return (precision == 1 ? 1u : 2u) * kBlockBytes + static_cast<uint32_t>(n_max) * 128u;
}

size_t group_smem_bytes(int32_t precision, int32_t n_max, int32_t dpad, int32_t n_stages)
{
    return 1024 + static_cast<size_t>(n_stages) * group_stage_bytes(precision, n_max) +
           group_tail_bytes(dpad, n_stages);
}

int32_t group_dpad(int32_t d_out) { return d_out == 10 ? 10 : (d_out + 3) / 4 * 4; }

int32_t group_stages(int32_t precision, int32_t n_max, int32_t d_out)
{
    for (int32_t ns = kMaxStages; ns >= kMinStages; --ns)
        if (group_smem_bytes(precision, n_max, group_dpad(d_out), ns) <= 227u * 1024u) return ns;
    return 0;
}

__device__ __forceinline__ GroupSmem carve(uint8_t* raw, const GroupArgs& a)
{
    GroupSmem s;
    s.ring = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    uint8_t* p = s.ring + static_cast<size_t>(a.n_stages) * a.stage_bytes;
    s.w2t = reinterpret_cast<float*>(p);
    p += sizeof(float) * kMaxN * a.dpad;
    s.b1 = reinterpret_cast<float*>(p);
    p += sizeof(float) * kMaxN;
    s.b2 = reinterpret_cast<float*>(p);
    p += sizeof(float) * kMaxGroup * 16;
    s.part = reinterpret_cast<float*>(p);
    p += sizeof(float) * kMaxSplit * 128 * 2 * a.dpad;
    s.red_loss = reinterpret_cast<float*>(p);
    p += sizeof(float) * kMaxGroup * 4;
    s.red_ok = reinterpret_cast<int32_t*>(p);
    p += sizeof(int32_t) * kMaxGroup * 4;
    s.ep_go = reinterpret_cast<int*>(p);
    s.tmem_holder = reinterpret_cast<uint32_t*>(p + 4);
    s.abort_flag = reinterpret_cast<volatile int*>(p + 8);
    s.ep_next = reinterpret_cast<int32_t*>(p + 12);
    p += 32;
    s.uidx = reinterpret_cast<int32_t*>(p);
    p += sizeof(int32_t) * kURing;
    p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 7u) & ~uintptr_t(7));
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.empty = bars + a.n_stages;
    s.acc_full = bars + 2 * a.n_stages;
    s.acc_empty = s.acc_full + 2;
    s.drain = s.acc_empty + 2;
    s.ufull = s.drain + 1;
    s.uempty = s.ufull + kURing;
    return s;
}

__device__ __forceinline__ void raise_abort(const GroupSmem& s, const GroupArgs& a)
{
    *s.abort_flag = 1;
    atomicOr(a.status, kStatusEvalTimeout);
}

__device__ __forceinline__ const ShadowRun& run_of(const GroupArgs& a, int32_t r)
{
    return a.runs ? a.runs[r] : a.run0;
}

// Unit idx of the table, or of run0's groups in order, each on all its tiles.
__device__ __forceinline__ GroupUnit unit_at(const GroupArgs& a, int32_t idx)
{
    if (a.units) return a.units[idx];
    const int32_t p0 = (idx / a.run0.m_tiles) * a.run0.group;
    return GroupUnit{ 0, idx % a.run0.m_tiles, p0, min(a.run0.group, a.run0.pop - p0) };
}

// The index of unit ui of this CTA (-1: no more), from the ring; false when
// the wait gives up.  Each reader releases the slot once it has the index.
__device__ __forceinline__ bool take_unit(const GroupSmem& s, uint32_t ui, int32_t& idx)
{
    const uint32_t slot = ui % kURing;
    if (!ptx::mbar_wait_bounded(&s.ufull[slot], (ui / kURing) & 1u, s.abort_flag, kWaitLimitNs)) return false;
    idx = s.uidx[slot];
    ptx::mbar_arrive(&s.uempty[slot]);
    return true;
}

// Claims the CTA's unit ui and publishes its index; the CTA that is last to
// find the table exhausted leaves the counters at zero for the next launch.
__device__ __forceinline__ bool publish_unit(const GroupSmem& s, const GroupArgs& a, uint32_t ui, int32_t& idx)
{
    const uint32_t slot = ui % kURing;
    if (!ptx::mbar_wait_bounded(&s.uempty[slot], ((ui / kURing) & 1u) ^ 1u, s.abort_flag, kWaitLimitNs)) return false;
    idx = atomicAdd(&a.sched[0], 1);
    if (idx >= a.n_units) {
        idx = -1;
        if (atomicAdd(&a.sched[1], 1) == static_cast<int>(gridDim.x) - 1) {
            atomicExch(&a.sched[0], 0);
            atomicExch(&a.sched[1], 0);
        }
    }
    s.uidx[slot] = idx;
    ptx::mbar_arrive(&s.ufull[slot]);
    return true;
}

template <int PREC, int DOUT>  // DOUT: d_out when fixed at compile time (10), else 0
__global__ void __launch_bounds__(kGroupThreads, 1) eval_shadow_group_kernel(const GroupArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const GroupSmem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t kPieces = PREC == 1 ? 1u : 2u;
    const uint32_t b_off = kPieces * kBlockBytes;  // the unit's shadow blocks within a stage

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.n_stages; ++i) {
            ptx::mbar_init(&s.full[i], kFullArrivals);
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.acc_full[i], 1);
            ptx::mbar_init(&s.acc_empty[i], kEpiWarps);
        }
        ptx::mbar_init(s.drain, 1);
        for (int i = 0; i < kURing; ++i) {
            ptx::mbar_init(&s.ufull[i], 1);
            ptx::mbar_init(&s.uempty[i], kUnitReaders);
        }
        *s.ep_go = 0;
        *s.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    // W2's padding outputs (d_out .. dpad - 1) stay zero: the staging writes only o < d_out.
    if (a.dpad > a.d_out) {
        const int pad = a.dpad - a.d_out;
        for (int i = threadIdx.x; i < kMaxN * pad; i += blockDim.x)
            s.w2t[(i / pad) * a.dpad + a.d_out + i % pad] = 0.0f;
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
            for (uint32_t ui = 0; ok; ++ui) {
                int32_t idx = -1;
                if (!take_unit(s, ui, idx)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                if (idx < 0) break;
                const GroupUnit u = unit_at(a, idx);
                const uint32_t n_cols = static_cast<uint32_t>(u.n * run_of(a, u.run).h);
                const uint32_t buf = ui & 1u;
                const uint32_t idesc = PREC == 1 ? ptx::idesc_bf16(128, n_cols) : ptx::idesc_e4m3(128, n_cols);
                if (!ptx::mbar_wait_bounded(&s.acc_empty[buf], ((ui >> 1) & 1u) ^ 1u, s.abort_flag, kWaitLimitNs)) {
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
    } else if (warp == 1) {
        // ------------------------------------------------------------ shadow producer (all lanes)
        ptx::grid_dep_wait();  // shadows and masters come from the previous kernel (breeding)
        uint32_t stage = 0, phase = 0, issued_mask = 0, parity_mask = 0;
        bool ok = true;
        int32_t idx = -1;
        if (lane == 0) ok = publish_unit(s, a, 0, idx);
        for (uint32_t ui = 0; ; ++ui) {
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            idx = __shfl_sync(0xFFFFFFFFu, idx, 0);
            if (!ok || idx < 0) break;
            const GroupUnit u = unit_at(a, idx);
            if (lane == 0) ok = publish_unit(s, a, ui + 1, idx);  // one unit ahead
            if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) break;
            const ShadowRun& r = run_of(a, u.run);
            const uint32_t slot = static_cast<uint32_t>(r.h) * 128u;
            const uint8_t* src = r.shadow + static_cast<int64_t>(u.p + (lane < u.n ? lane : 0)) * r.sh_stride;
            for (int kb = 0; kb < a.k_blocks; ++kb) {
                bool got = true;
                if (lane == 0) got = ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs);
                got = __shfl_sync(0xFFFFFFFFu, got, 0);
                if (!got) {
                    if (lane == 0) raise_abort(s, a);
                    ok = false;
                    break;
                }
                uint8_t* sb = s.ring + stage * a.stage_bytes;
                if (lane < u.n) {
                    ptx::mbar_arrive_expect_tx(&s.full[stage], slot);
                    ptx::bulk_load(sb + b_off + lane * slot, src + static_cast<int64_t>(kb) * slot, slot,
                                   &s.full[stage]);
                } else {
                    ptx::mbar_arrive(&s.full[stage]);
                }
                issued_mask |= 1u << stage;
                parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                if (++stage == static_cast<uint32_t>(a.n_stages)) { stage = 0; phase ^= 1u; }
            }
        }
        if (!ok && lane == 0) {  // let copies in flight land before the CTA exits
            raise_abort(s, a);
            volatile int never = 0;
            for (int i = 0; i < a.n_stages; ++i)
                if (issued_mask & (1u << i))
                    ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
        }
    } else if (warp == kBatchWarp) {
        // ------------------------------------------------------------ batch producer
        if (lane == 0) {
            ptx::grid_dep_wait();  // the staged batch comes from an earlier kernel
            uint32_t stage = 0, phase = 0, issued_mask = 0, parity_mask = 0;
            bool ok = true;
            for (uint32_t ui = 0; ok; ++ui) {
                int32_t idx = -1;
                if (!take_unit(s, ui, idx)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                if (idx < 0) break;
                const GroupUnit u = unit_at(a, idx);
                const uint8_t* xt = run_of(a, u.run).xop + static_cast<int64_t>(u.mt) * a.k_blocks * a.a_bytes;
                for (int kb = 0; kb < a.k_blocks; ++kb) {
                    if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    uint8_t* sb = s.ring + stage * a.stage_bytes;
                    ptx::mbar_arrive_expect_tx(&s.full[stage], a.a_bytes);
                    ptx::bulk_load(sb, xt + static_cast<int64_t>(kb) * a.a_bytes, a.a_bytes, &s.full[stage]);
                    issued_mask |= 1u << stage;
                    parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                    if (++stage == static_cast<uint32_t>(a.n_stages)) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {
                volatile int never = 0;
                for (int i = 0; i < a.n_stages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - kFirstEpiWarp;
        const int wq = ew >> 2;      // this warp's index among the 4 of its lane quarter
        const int q = warp & 3;      // TMEM lane quarter of this warp
        const int et = ew * 32 + lane;
        const int row = q * 32 + lane;
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        constexpr uint32_t kBar = 1u;
        // Output slots the chains run over, and W2's row stride in shared memory
        // (10 exactly for 10 outputs; else d_out rounded up to 4).
        constexpr int kOutP = DOUT == 0 ? kMaxOut : DOUT;
        static_assert(DOUT == 0 || DOUT == 10, "the fixed-output form is written for 10 outputs");
        const int d_out = DOUT == 0 ? a.d_out : DOUT;
        const int dpad = DOUT == 0 ? a.dpad : 10;
        ptx::grid_dep_wait();  // b1, W2, b2 come from the previous kernel (breeding)

        // b1, W2, b2 of the unit's individuals (as stored after W1), element
        // et + 512 j, into registers one unit ahead.  Loaded through L2
        // (ld.global.cg), not the read-only path: this grid starts while the
        // breeding kernel that writes them still runs.
        float prm[kPrmRegs];
        auto load_prm = [&](const GroupUnit& u) {
            const ShadowRun& r = run_of(a, u.run);
            const int n_prm = r.h + d_out * r.h + d_out;
            const int total = u.n * n_prm;
#pragma unroll
            for (int j = 0; j < kPrmRegs; ++j) {
                const int i = et + kEpiThreads * j;
                float v = 0.0f;
                if (i < total) {
                    const int g = i / n_prm, e = i - g * n_prm;
                    v = __ldcg(r.popv + static_cast<int64_t>(u.p + g) * r.c_pad + static_cast<int64_t>(r.h) * a.k +
                               e);
                }
                prm[j] = v;
            }
        };
        auto stage_prm = [&](const GroupUnit& u) {
            const int h = run_of(a, u.run).h;
            const int n_prm = h + d_out * h + d_out;
            const int total = u.n * n_prm;
#pragma unroll
            for (int j = 0; j < kPrmRegs; ++j) {
                const int i = et + kEpiThreads * j;
                if (i < total) {
                    const int g = i / n_prm, e = i - g * n_prm;
                    if (e < h) {
                        s.b1[g * h + e] = prm[j];
                    } else if (e < h + d_out * h) {
                        const int o = (e - h) / h, col = (e - h) - o * h;
                        s.w2t[(g * h + col) * dpad + o] = prm[j];
                    } else {
                        s.b2[g * 16 + (e - h - d_out * h)] = prm[j];
                    }
                }
            }
        };
        // The chain of quarter sl for the individual whose accumulator starts
        // at TMEM column col0: in column order over quarter sl (whole 8-unit
        // groups) of every chunk of cw hidden units, ReLU(D scale + b1) times
        // W2.  Two outputs share each packed FMA (each half an ordinary
        // round-to-nearest FMA, so every chain keeps its bits).
        auto chain = [&](int sl, uint32_t col0, int h, int cw, int n_chunks, const float* b1, const float* w2t,
                         float2 scale2, float2 (&acc)[kOutP / 2]) {
#pragma unroll
            for (int o2 = 0; o2 < kOutP / 2; ++o2) acc[o2] = make_float2(0.0f, 0.0f);
            for (int c = 0; c < n_chunks; ++c) {
                const int r0 = c * cw, n8 = min(cw, h - r0) / 8;
                const int g0 = n8 * sl / 4, g1 = n8 * (sl + 1) / 4;
                for (int gg = g0; gg < g1; ++gg) {
                    uint32_t d[8];
                    ptx::tmem_ld8_nowait(col0 + static_cast<uint32_t>(r0 + 8 * gg), d);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int jj = 0; jj < 8; jj += 4) {
                        const int col = r0 + 8 * gg + jj;
                        const float4 bb = *reinterpret_cast<const float4*>(b1 + col);
                        const float2 h01 = __ffma2_rn(make_float2(__uint_as_float(d[jj]), __uint_as_float(d[jj + 1])),
                                                      scale2, make_float2(bb.x, bb.y));
                        const float2 h23 = __ffma2_rn(make_float2(__uint_as_float(d[jj + 2]), __uint_as_float(d[jj + 3])),
                                                      scale2, make_float2(bb.z, bb.w));
                        const float hv[4] = {fmaxf(h01.x, 0.0f), fmaxf(h01.y, 0.0f), fmaxf(h23.x, 0.0f),
                                             fmaxf(h23.y, 0.0f)};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 hh2 = make_float2(hv[e], hv[e]);
                            if (DOUT == 10) {
                                // a column of 10 outputs: five 8-byte loads
                                const float2* wr = reinterpret_cast<const float2*>(w2t + (col + e) * 10);
#pragma unroll
                                for (int o2 = 0; o2 < 5; ++o2) acc[o2] = __ffma2_rn(wr[o2], hh2, acc[o2]);
                            } else {
                                const float4* wr = reinterpret_cast<const float4*>(w2t + (col + e) * dpad);
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
        };
        // acc += add, output by output (the chains' fixed order of addition).
        auto add_to = [&](float2 (&acc)[kOutP / 2], const float2 (&add)[kOutP / 2]) {
#pragma unroll
            for (int o2 = 0; o2 < kOutP / 2; ++o2) acc[o2] = make_float2(acc[o2].x + add[o2].x, acc[o2].y + add[o2].y);
        };
        // Softmax cross-entropy and the hit of this thread's sample from the
        // sum of the four chains, ((c0 + c1) + c2) + c3.
        auto loss_of = [&](const float2 (&sum)[kOutP / 2], const float* b2, int label, float& loss, int32_t& good) {
            float logit[kOutP];
#pragma unroll
            for (int o2 = 0; o2 < kOutP / 2; ++o2) {
                if (DOUT != 0 || 2 * o2 < d_out) {
                    logit[2 * o2] = sum[o2].x + b2[2 * o2];
                    logit[2 * o2 + 1] = sum[o2].y + b2[2 * o2 + 1];
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
                good = 0;
            }
        };
        auto reduce_store = [&](int g, float loss, int32_t good) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
                good += __shfl_xor_sync(0xFFFFFFFFu, good, off);
            }
            if (lane == 0) {
                s.red_loss[g * 4 + q] = loss;
                s.red_ok[g * 4 + q] = good;
            }
        };

        GroupUnit u{}, un{};
        if (et == 0) {
            int32_t idx = -1;
            if (!take_unit(s, 0, idx)) {
                raise_abort(s, a);
                idx = -1;
            }
            s.ep_next[0] = idx;
        }
        ptx::named_barrier_sync(kBar, kEpiThreads);
        const int32_t idx0 = s.ep_next[0];
        bool have = idx0 >= 0;
        if (have) {
            u = unit_at(a, idx0);
            load_prm(u);
        }
        int32_t cur_run = -1, cur_mt = -1, label = 0;
        for (uint32_t ui = 0; have; ++ui) {
            // The previous unit's readers finished with the staged parameters at barrier B.
            stage_prm(u);
            const uint32_t buf = ui & 1u, bph = (ui >> 1) & 1u;
            if (et == 0) {
                bool got = ptx::mbar_wait_bounded(&s.acc_full[buf], bph, s.abort_flag, kWaitLimitNs);
                int32_t nx = -1;
                if (got) got = take_unit(s, ui + 1, nx);
                if (!got) raise_abort(s, a);
                *s.ep_go = got ? 1 : 0;
                s.ep_next[(ui + 1) & 1u] = nx;  // its previous value was read after barrier A of unit ui - 2
            }
            ptx::named_barrier_sync(kBar, kEpiThreads);  // A: accumulator ready (or abort); parameters staged
            if (!*s.ep_go) break;
            const int32_t idx_n = s.ep_next[(ui + 1) & 1u];
            const bool have_n = idx_n >= 0;
            if (have_n) {
                un = unit_at(a, idx_n);
                load_prm(un);  // in flight while this unit is evaluated
            }
            ptx::tc_fence_after();

            const ShadowRun& r = run_of(a, u.run);
            const int h = r.h, cw = r.cw, n_chunks = r.n_chunks, n = u.n;
            const int srow = u.mt * 128 + row;  // the sample of this TMEM lane
            const bool live = srow < r.batch;
            if (u.run != cur_run || u.mt != cur_mt) {
                label = live ? r.y[srow] : 0;
                cur_run = u.run;
                cur_mt = u.mt;
            }
            const uint32_t acc0 = tmem_base + lane_addr + buf * kAccStride;
            auto scale_of = [&](int g) {
                // D * (w scale / x_div): the FP8 shadow stores w / 2^e.
                const float sc = PREC == 2 ? ldexpf(r.inv_div, r.scale_exp[u.p + g]) : r.inv_div;
                return make_float2(sc, sc);
            };
            // Layer 2 in the chunked kernel's order (see the file comment).
            const bool split = n <= kMaxSplit;
            int g_keep = -1;  // split units: the individual whose chains 0 and 1 this warp holds
            float2 k01[kOutP / 2];
            if (split) {
                // items: (g, chains 0-1) for it < n, (it - n, chains 2-3) after
                for (int it = wq; it < 2 * n; it += 4) {
                    const int g = it < n ? it : it - n;
                    const int hh = it < n ? 0 : 1;
                    const uint32_t col0 = acc0 + static_cast<uint32_t>(g * h);
                    const float* b1 = s.b1 + g * h;
                    const float* w2t = s.w2t + g * h * dpad;
                    const float2 sc2 = scale_of(g);
                    float2 cc[kOutP / 2];
                    if (hh == 0) {
                        chain(0, col0, h, cw, n_chunks, b1, w2t, sc2, k01);
                        chain(1, col0, h, cw, n_chunks, b1, w2t, sc2, cc);
                        add_to(k01, cc);
                        g_keep = g;
                    } else {
                        float* part = s.part + (g * 128 + row) * (2 * dpad);
#pragma unroll 1
                        for (int sl = 2; sl < 4; ++sl) {
                            chain(sl, col0, h, cw, n_chunks, b1, w2t, sc2, cc);
#pragma unroll
                            for (int o2 = 0; o2 < kOutP / 2; ++o2)
                                if (DOUT != 0 || 2 * o2 < d_out)
                                    reinterpret_cast<float2*>(part + (sl - 2) * dpad)[o2] = cc[o2];
                        }
                    }
                }
            } else {
                for (int g = wq; g < n; g += 4) {
                    const uint32_t col0 = acc0 + static_cast<uint32_t>(g * h);
                    const float* b1 = s.b1 + g * h;
                    const float* w2t = s.w2t + g * h * dpad;
                    const float2 sc2 = scale_of(g);
                    float2 sum[kOutP / 2], cc[kOutP / 2];
                    chain(0, col0, h, cw, n_chunks, b1, w2t, sc2, sum);
#pragma unroll 1
                    for (int sl = 1; sl < 4; ++sl) {
                        chain(sl, col0, h, cw, n_chunks, b1, w2t, sc2, cc);
                        add_to(sum, cc);
                    }
                    float loss = 0.0f;
                    int32_t good = 0;
                    if (live) loss_of(sum, s.b2 + g * 16, label, loss, good);
                    reduce_store(g, loss, good);
                }
            }
            // The accumulator is read: release it to the next unit's MMAs.
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&s.acc_empty[buf]);
            ptx::named_barrier_sync(kBar, kEpiThreads);  // C: the second halves' chains written
            if (split && g_keep >= 0) {
                const float* part = s.part + (g_keep * 128 + row) * (2 * dpad);
#pragma unroll 1
                for (int sl = 0; sl < 2; ++sl) {
                    float2 cc[kOutP / 2];
#pragma unroll
                    for (int o2 = 0; o2 < kOutP / 2; ++o2)
                        cc[o2] = (DOUT != 0 || 2 * o2 < d_out) ? reinterpret_cast<const float2*>(part + sl * dpad)[o2]
                                                               : make_float2(0.0f, 0.0f);
                    add_to(k01, cc);
                }
                float loss = 0.0f;
                int32_t good = 0;
                if (live) loss_of(k01, s.b2 + g_keep * 16, label, loss, good);
                reduce_store(g_keep, loss, good);
            }
            ptx::named_barrier_sync(kBar, kEpiThreads);  // B: quarter sums written; staged data no longer read
            if (et < n) {
                const int g = et, p = u.p + g;
                const float* rl = s.red_loss + g * 4;
                const int32_t* ro = s.red_ok + g * 4;
                const float total = ((rl[0] + rl[1]) + rl[2]) + rl[3];
                const int32_t n_ok = ro[0] + ro[1] + ro[2] + ro[3];
                if (r.m_tiles == 1) {
                    const float f = -(total / static_cast<float>(r.batch));
                    r.f_raw[p] = f;
                    if (r.f_adj) r.f_adj[p] = r.f_inh ? (1.0f - r.alpha) * r.f_inh[p] + r.alpha * f : f;
                    if (r.correct) r.correct[p] = n_ok;
                } else {
                    r.scratch[static_cast<int64_t>(u.mt) * r.pop + p] = total;
                    r.scratch[static_cast<int64_t>(r.m_tiles + u.mt) * r.pop + p] = static_cast<float>(n_ok);
                }
            }
            u = un;
            have = have_n;
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

// The batch as A operand tiles, as in the state object's staging: tile t of
// the table, K block kb, piece q at dst + (kb * pieces + q) * 16 KB; row r
// (zero past the tile's rows) at 128 r, its 16-byte chunk c at chunk position
// c ^ (r & 7).  BF16: 64 levels per row of a block; FP8: 128 levels, piece 0
// holding 16 floor(k / 16), piece 1 k mod 16, both exact in e4m3.  One thread
// per 16-byte chunk.
template <int PREC>
__global__ void __launch_bounds__(256) stage_xop_tiles_kernel(const XopTile* __restrict__ tiles, int32_t n_tiles,
                                                              int32_t k, int32_t k_blocks)
{
    ptx::grid_dep_launch();
    constexpr int kPieces = PREC == 1 ? 1 : 2;
    const int64_t per_tile = static_cast<int64_t>(k_blocks) * kPieces * 128 * 8;
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < per_tile * n_tiles) {
        const int t = static_cast<int>(i / per_tile);
        const int64_t w = i - t * per_tile;
        const XopTile tile = tiles[t];
        const int c = static_cast<int>(w & 7);
        const int r = static_cast<int>((w >> 3) & 127);
        const int64_t blk = w >> 10;  // kb * pieces + piece
        const int pc = static_cast<int>(blk % kPieces);
        const int kb = static_cast<int>(blk / kPieces);
        const bool live = r < tile.rows;
        const uint8_t* xr = tile.x + static_cast<int64_t>(live ? r : 0) * k;
        uint32_t wd[4];
        if (PREC == 1) {
            const int k0 = kb * 64 + c * 8;  // 8 BF16 levels
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float l0 = live && k0 + 2 * e < k ? static_cast<float>(xr[k0 + 2 * e]) : 0.0f;
                const float l1 = live && k0 + 2 * e + 1 < k ? static_cast<float>(xr[k0 + 2 * e + 1]) : 0.0f;
                const __nv_bfloat162 b2v = __floats2bfloat162_rn(l0, l1);
                wd[e] = *reinterpret_cast<const uint32_t*>(&b2v);
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
                    const float pv = pc == 0 ? static_cast<float>(lv & 0xF0u) : static_cast<float>(lv & 15u);
                    word |= static_cast<uint32_t>(__nv_cvt_float_to_fp8(pv, __NV_SATFINITE, __NV_E4M3)) << (8 * b);
                }
                wd[e] = word;
            }
        }
        *reinterpret_cast<uint4*>(tile.dst + blk * kBlockBytes + r * 128 + ((c ^ (r & 7)) << 4)) =
            make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
    ptx::grid_dep_wait();
}

}  // namespace

int32_t eval_shadow_group_size(int32_t h)
{
    const int32_t g = h > 0 ? kMaxN / h : 1;
    return g < 1 ? 1 : (g > kMaxGroup ? kMaxGroup : g);
}

bool eval_shadow_group_supported(int32_t k, int32_t d_out, int32_t precision, int32_t h, int32_t n_max)
{
    if ((precision != 1 && precision != 2) || k % 16 != 0 || h % 16 != 0 || h < 16 || h > kMaxN ||
        d_out < 1 || d_out > kMaxOut || n_max < h || n_max > kMaxN || n_max % 16 != 0)
        return false;
    // The layer-2 order follows the chunked kernel's chunks, which must exist.
    if (eval_shadow_max_chunk(precision, k) < 16) return false;
    return group_stages(precision, n_max, d_out) > 0;
}

size_t eval_shadow_group_xop_bytes(int32_t k, int32_t precision, int32_t batch)
{
    const int32_t m_tiles = (batch + 127) / 128;
    const int32_t k_blocks = (k + (precision == 1 ? 63 : 127)) / (precision == 1 ? 64 : 128);
    return static_cast<size_t>(m_tiles) * k_blocks * (precision == 1 ? 1 : 2) * kBlockBytes;
}

cudaError_t launch_stage_xop_tiles(const XopTile* tiles_dev, int32_t n_tiles, int32_t k, int32_t precision,
                                   cudaStream_t stream)
{
    if (n_tiles < 1) return cudaSuccess;
    const int32_t k_blocks = (k + (precision == 1 ? 63 : 127)) / (precision == 1 ? 64 : 128);
    const int64_t chunks = static_cast<int64_t>(n_tiles) * k_blocks * (precision == 1 ? 1 : 2) * 128 * 8;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>((chunks + 255) / 256));
    cfg.blockDim = dim3(256);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return precision == 1 ? cudaLaunchKernelEx(&cfg, stage_xop_tiles_kernel<1>, tiles_dev, n_tiles, k, k_blocks)
                          : cudaLaunchKernelEx(&cfg, stage_xop_tiles_kernel<2>, tiles_dev, n_tiles, k, k_blocks);
}

namespace {

cudaError_t launch_group(GroupArgs& a, int32_t precision, int32_t n_max, int32_t grid, cudaStream_t stream)
{
    a.dpad = group_dpad(a.d_out);
    a.k_blocks = (a.k + (precision == 1 ? 63 : 127)) / (precision == 1 ? 64 : 128);
    a.k_mma = precision == 1 ? (a.k + 15) / 16 * 16 : (a.k + 31) / 32 * 32;
    a.n_stages = group_stages(precision, n_max, a.d_out);
    if (a.n_stages == 0 || grid < 1) return cudaErrorInvalidValue;
    a.a_bytes = (precision == 1 ? 1u : 2u) * kBlockBytes;
    a.stage_bytes = group_stage_bytes(precision, n_max);
    const size_t smem = group_smem_bytes(precision, n_max, a.dpad, a.n_stages);
    const bool ten = a.d_out == 10;
    const void* kern = precision == 1 ? (ten ? reinterpret_cast<const void*>(eval_shadow_group_kernel<1, 10>)
                                             : reinterpret_cast<const void*>(eval_shadow_group_kernel<1, 0>))
                                      : (ten ? reinterpret_cast<const void*>(eval_shadow_group_kernel<2, 10>)
                                             : reinterpret_cast<const void*>(eval_shadow_group_kernel<2, 0>));
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    // Programmatic stream serialisation: CTAs may start (barriers, TMEM) while
    // the previous kernel finishes; the producers and the epilogue wait for it
    // before they read.
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kGroupThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (precision == 1)
        return ten ? cudaLaunchKernelEx(&cfg, eval_shadow_group_kernel<1, 10>, a)
                   : cudaLaunchKernelEx(&cfg, eval_shadow_group_kernel<1, 0>, a);
    return ten ? cudaLaunchKernelEx(&cfg, eval_shadow_group_kernel<2, 10>, a)
               : cudaLaunchKernelEx(&cfg, eval_shadow_group_kernel<2, 0>, a);
}

}  // namespace

cudaError_t launch_eval_shadow_group_run(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                                         const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp,
                                         const void* xop, float x_div, const int32_t* y, int32_t batch, float alpha,
                                         const float* f_inh, float* f_raw, float* f_adj, int32_t* correct,
                                         float* scratch, int32_t* sched, unsigned int* status, cudaStream_t stream)
{
    if (precision != 1 && precision != 2) return cudaErrorInvalidValue;
    GroupArgs a{};
    a.k = net.dims[0];
    a.d_out = net.dims[2];
    a.run0 = shadow_run(net, pop, pop_dev, precision, shadow, sh_stride, scale_exp, nullptr, x_div, y, batch, alpha,
                        f_inh, f_raw, f_adj, correct, scratch, 0);
    a.run0.xop = static_cast<const uint8_t*>(xop);
    a.run0.group = eval_shadow_group_size(net.dims[1]);
    if (a.run0.m_tiles > 1 && !scratch) return cudaErrorInvalidValue;
    a.n_units = (pop + a.run0.group - 1) / a.run0.group * a.run0.m_tiles;
    a.sched = sched;
    a.status = status;
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = launch_group(a, precision, a.run0.group * net.dims[1], sms, stream);
    if (err != cudaSuccess || a.run0.m_tiles == 1) return err;
    return launch_combine_shadow_run_tiles(a.run0, stream);
}

cudaError_t launch_eval_shadow_group(int32_t k, int32_t d_out, int32_t precision, int32_t n_max,
                                     const ShadowRun* runs_dev, int32_t n_runs, int32_t pop_max, bool any_tiles,
                                     const GroupUnit* units_dev, int32_t n_units, int32_t* sched_dev, int32_t grid,
                                     unsigned int* status, cudaStream_t stream)
{
    if (precision != 1 && precision != 2) return cudaErrorInvalidValue;
    GroupArgs a{};
    a.k = k;
    a.d_out = d_out;
    a.runs = runs_dev;
    a.units = units_dev;
    a.n_units = n_units;
    a.sched = sched_dev;
    a.status = status;
    cudaError_t err = launch_group(a, precision, n_max, grid, stream);
    if (err != cudaSuccess || !any_tiles) return err;
    return launch_combine_shadow_tiles(runs_dev, n_runs, pop_max, stream);
}

}  // namespace leea
