// leea_breed_eval.cu -- crossover, mutation and evaluation of every child in
// one pass (Section 3.2 and Eq. 1, for minibatches of 8-bit levels x = k /
// x_div).  A child's first-layer weights are made in shared memory from its
// parents' tiles, written to HBM once and handed to the tcgen05 tensor cores
// from there, so the evaluation does not read the new population back: per
// child the pass moves what breeding alone moves (one or two parent floats in,
// one child float out per gene), and the evaluation's weight stream is gone.
//
// The children are bit-identical to the breeding kernel's (same streams, same
// operators: breed_ops.cuh).  The evaluation numerics are those of the 8-bit
// tensor-core evaluation: each child weight, scaled by 2^8, as two FP16 pieces
// against the exact FP16 levels held in TMEM, FP32 accumulation, and an FP32
// FFMA fallback for a child with a weight |w| >= 128.
//
// Warp roles (persistent CTA, one per SM; CTA b takes children
// pop - 1 - (b + n gridDim.x), n = 0, 1, ...):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      TMA producer: per 64-wide K stage the parents' W1 tiles
//               (h rows x 64 FP32 each) into a ring of slots, one slot per
//               parent tile (two for a crossover child)
//   warps 2-15  breeders: per stage a thread makes 8 consecutive genes of some
//               rows (crossover mask or mean; mutation with a warp job list of
//               normals), stores them to HBM and splits them into the two FP16
//               pieces, written swizzled into the ring the MMAs read
//   warps 16-19 the batch into TMEM once; then per child: breed the remaining
//               genes (b1, W2, b2, padding) from HBM and stage them, read the
//               accumulator row by row (one sample per thread), layer 2,
//               softmax cross-entropy, fixed-order batch sum, inheritance
// Every mbarrier wait is bounded in time; on expiry the kernel sets
// kStatusEvalTimeout, drains what it has in flight and exits.
#include <cuda.h>

#include <algorithm>
#include <cuda_fp16.h>

#include "breed_ops.cuh"
#include "leea_internal.h"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kBreedWarps = 14;
constexpr int kFirstBreedWarp = 2;
constexpr int kFirstEpiWarp = kFirstBreedWarp + kBreedWarps;
constexpr int kEpiWarps = 4;
constexpr int kBreedThreads = 32 * kBreedWarps;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kFusedThreads = 32 * (kFirstEpiWarp + kEpiWarps);
constexpr int kKStage = 64;            // K elements per stage: one 128-byte FP16 row per piece
constexpr int kPieces = 2;             // FP16 pieces per weight
constexpr int kPieceStages = 2;
constexpr int kMaxSlots = 6;           // parent tiles in flight
constexpr int kMaxOut = 16;
constexpr int kJobs = 4 * 32;          // Box-Muller pairs of a warp's 32 units
constexpr uint32_t kTmemCols = 512;
constexpr float kPieceScale = 256.0f;  // 2^8: weights enter the pieces as 2^8 w
constexpr float kPieceRange = 128.0f;  // |w| below this: 2^8 |w| < 2^15, finite in FP16
constexpr int32_t kKindInvalid = -1;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct FusedArgs {
    int32_t pop, k, h, d_out, dpad, batch, k_stages, k16, slots;
    int64_t c, c_pad;
    int32_t xo_op;
    uint32_t thr_xo, thr_mut;
    float sigma;
    const float* sigma_child;  // NULL: sigma for every child
    uint64_t seed;
    uint32_t gen;
    float inv_div, alpha;
    uint32_t a_col;  // first TMEM column of the batch operand (the accumulator uses 0 .. h-1)
    // batch staging in the tail of the rings (as in the 8-bit evaluation)
    int32_t x_staged, x_kc, x_stride, x_off, n_early;
    const float* parents;
    float* children;
    const int32_t *par1, *par2, *kind;
    const uint8_t* x;
    const int32_t* y;
    const float* f_inh;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    unsigned int* status;
};

struct FusedSmem {
    uint8_t* raw;       // slots x h x 256 B: one parent's W1 tile each, 1024-aligned
    uint8_t* ring;      // kPieceStages x kPieces x h x 128 B, right after
    uint32_t raw_bytes, piece_bytes;
    float* w2t;         // [h][dpad]: the child's W2, transposed
    float* b1;          // [h]
    float* b2;          // [16]
    float2* job_z;      // [kBreedWarps][kJobs]
    uint8_t* job_code;  // [kBreedWarps][kJobs]
    uint64_t *slot_full, *slot_empty, *full, *empty, *acc_full, *acc_empty, *a_ready, *drain, *conv_done, *x_loaded,
        *x_full;
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
    uint32_t* flag_unit;  // [2]: u + 1 if child (unit) u has a weight outside the piece range
    float* red_loss;      // [4]
    int32_t* red_ok;      // [4]
};

__host__ __device__ inline size_t fused_smem_bytes(int32_t h, int32_t dpad, int32_t batch, int32_t slots)
{
    return 1024 + static_cast<size_t>(slots) * h * 256 + static_cast<size_t>(kPieceStages) * kPieces * h * 128 +
           sizeof(float) * (static_cast<size_t>(h) * dpad + h + 16) +
           (sizeof(float2) + 1) * kBreedWarps * kJobs + 8 * (2 * slots + 2 * kPieceStages + 8) + 64;
}

__device__ __forceinline__ FusedSmem carve(uint8_t* raw, const FusedArgs& a)
{
    FusedSmem s;
    s.raw = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    s.raw_bytes = static_cast<uint32_t>(a.h) * 256u;
    s.piece_bytes = static_cast<uint32_t>(a.h) * 128u;
    s.ring = s.raw + a.slots * s.raw_bytes;
    uint8_t* p = s.ring + kPieceStages * kPieces * s.piece_bytes;
    s.w2t = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.h * a.dpad;
    s.b1 = reinterpret_cast<float*>(p);
    p += sizeof(float) * a.h;
    s.b2 = reinterpret_cast<float*>(p);
    p += sizeof(float) * 16;
    // an even number of floats so far (h even): 8-byte aligned
    s.job_z = reinterpret_cast<float2*>(p);
    p += sizeof(float2) * kBreedWarps * kJobs;
    s.job_code = p;
    p += kBreedWarps * kJobs;
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.slot_full = bars;
    s.slot_empty = bars + a.slots;
    s.full = bars + 2 * a.slots;
    s.empty = s.full + kPieceStages;
    s.acc_full = s.empty + kPieceStages;
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
    s.flag_unit = w + 3;
    s.red_loss = reinterpret_cast<float*>(w + 5);
    s.red_ok = reinterpret_cast<int32_t*>(w + 9);
    return s;
}

// Deepest slot ring that fits in 227 KB next to everything else (at least 2:
// a crossover stage holds two slots at once).
bool fused_slots(int32_t h, int32_t dpad, int32_t batch, int32_t* slots)
{
    for (int32_t n = kMaxSlots; n >= 2; --n)
        if (fused_smem_bytes(h, dpad, batch, n) <= 227u * 1024u) {
            *slots = n;
            return true;
        }
    return false;
}

__device__ __forceinline__ void raise_abort(const FusedSmem& s, const FusedArgs& a)
{
    *s.abort_flag = 1;
    atomicOr(a.status, kStatusEvalTimeout);
}

// The n-th child a CTA sequence visits: children in reverse index order, so
// that mutation children (the most work per gene) come first and the last
// round, which only some CTAs take, holds crossover children and elites.
__device__ __forceinline__ int child_of(const FusedArgs& a, int n)
{
    return a.pop - 1 - n;
}

struct ChildInfo {
    int32_t kind, p1, p2;
};

// Kind and parents of child j; a parent index outside [0, pop) makes an invalid
// child (NaN genes), as in the breeding kernel.
__device__ __forceinline__ ChildInfo child_info(const FusedArgs& a, int32_t j)
{
    ChildInfo ci{ a.kind[j], a.par1[j], a.par2[j] };
    if (ci.p1 < 0 || ci.p1 >= a.pop || ci.p2 < 0 || ci.p2 >= a.pop || ci.kind < 0 || ci.kind > 2)
        ci.kind = kKindInvalid;
    return ci;
}

__device__ __forceinline__ uint32_t half2_bits(__half2 v)
{
    return *reinterpret_cast<uint32_t*>(&v);
}

// Two FP32 weights as packed FP16 pieces of 2^8 w (lower K index in the low
// half): p1 rounds 2^8 w to nearest, p2 rounds the remainder, exact in FP32.
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

// Eight genes of a shared-memory tile row at float offset off (a multiple of 8).
__device__ __forceinline__ void load8(const float* tile, int32_t off, float4 (&v)[2])
{
    v[0] = *reinterpret_cast<const float4*>(tile + off);
    v[1] = *reinterpret_cast<const float4*>(tile + off + 4);
}

__global__ void __launch_bounds__(kFusedThreads, 1)
breed_eval_u8_kernel(const __grid_constant__ CUtensorMap tmap_par, const FusedArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const FusedSmem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.slots; ++i) {
            ptx::mbar_init(&s.slot_full[i], 1);
            ptx::mbar_init(&s.slot_empty[i], kBreedWarps);
        }
        for (int i = 0; i < kPieceStages; ++i) {
            ptx::mbar_init(&s.full[i], kBreedWarps);
            ptx::mbar_init(&s.empty[i], 1);
        }
        ptx::tma_prefetch_map(&tmap_par);
        ptx::mbar_init(s.acc_full, 1);
        ptx::mbar_init(s.acc_empty, kEpiThreads);
        ptx::mbar_init(s.a_ready, kEpiThreads);
        ptx::mbar_init(s.drain, 1);
        ptx::mbar_init(&s.conv_done[0], kBreedWarps);
        ptx::mbar_init(&s.conv_done[1], kBreedWarps);
        ptx::mbar_init(s.x_loaded, kEpiThreads);
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
            for (int j = blockIdx.x; ok && j < a.pop; j += gridDim.x) {
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
                    if (++stage == static_cast<uint32_t>(kPieceStages)) { stage = 0; phase ^= 1u; }
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
        // ------------------------------------------------------------ TMA producer (parent tiles)
        if (lane == 0) {
            ptx::grid_dep_wait();  // kinds and parents come from the selection kernel
            uint32_t slot = 0, sphase = 0, issued = 0;
            uint32_t issued_mask = 0, parity_mask = 0;
            bool ok = true;
            for (int n = blockIdx.x; ok && n < a.pop; n += gridDim.x) {
                const int j = child_of(a, n);
                const ChildInfo ci = child_info(a, j);
                const int need = ci.kind == 1 ? 2 : 1;
                for (int kc = 0; ok && kc < a.k_stages; ++kc) {
                    for (int t = 0; t < need; ++t) {
                        // Slots that overlap the batch staging area wait until
                        // the batch is in TMEM.
                        if (issued == static_cast<uint32_t>(a.n_early) &&
                            !ptx::mbar_wait_bounded(s.x_loaded, 0u, s.abort_flag, kWaitLimitNs)) {
                            raise_abort(s, a);
                            ok = false;
                            break;
                        }
                        ++issued;
                        if (!ptx::mbar_wait_bounded(&s.slot_empty[slot], sphase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                            raise_abort(s, a);
                            ok = false;
                            break;
                        }
                        if (ci.kind == kKindInvalid) {
                            ptx::mbar_arrive(&s.slot_full[slot]);
                        } else {
                            ptx::mbar_arrive_expect_tx(&s.slot_full[slot], s.raw_bytes);
                            ptx::tma_load_3d(s.raw + slot * s.raw_bytes, &tmap_par, &s.slot_full[slot], kc * kKStage, 0,
                                             t ? ci.p2 : ci.p1);
                            issued_mask |= 1u << slot;
                            parity_mask = (parity_mask & ~(1u << slot)) | (sphase << slot);
                        }
                        if (++slot == static_cast<uint32_t>(a.slots)) { slot = 0; sphase ^= 1u; }
                    }
                }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                for (int i = 0; i < a.slots; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.slot_full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
            }
        }
    } else if (warp < kFirstEpiWarp) {
        // ------------------------------------------------------------ breeders
        // Per stage, item t = lt + kBreedThreads v is (row t >> 3, genes
        // 8 (t & 7) .. 8 (t & 7) + 7 of the stage's 64).
        const int lt = threadIdx.x - 32 * kFirstBreedWarp;
        const int bw = warp - kFirstBreedWarp;
        float2* job_z = s.job_z + bw * kJobs;
        uint8_t* job_code = s.job_code + bw * kJobs;
        const int items = (a.h * 8 + kBreedThreads - 1) / kBreedThreads;
        ptx::grid_dep_wait();  // kinds, parents and sigma genes come from the selection kernel
        const PhiloxKeys key = philox_keys(a.seed);
        uint32_t slot = 0, sphase = 0, stage = 0, phase = 0, unit = 0;
        // the piece ring doubles as the batch staging area until the batch is in
        bool ok = ptx::mbar_wait_bounded(s.x_loaded, 0u, s.abort_flag, kWaitLimitNs);
        if (!ok) raise_abort(s, a);
        for (int n = blockIdx.x; ok && n < a.pop; n += gridDim.x, ++unit) {
            const int j = child_of(a, n);
            const ChildInfo ci = child_info(a, j);
            const float sigma = a.sigma_child ? a.sigma_child[j] : a.sigma;
            const uint32_t ent = static_cast<uint32_t>(j);
            float* child = a.children + static_cast<int64_t>(j) * a.c_pad;
            for (int kc = 0; kc < a.k_stages; ++kc) {
                const uint32_t sa = slot, pa = sphase;
                if (++slot == static_cast<uint32_t>(a.slots)) { slot = 0; sphase ^= 1u; }
                uint32_t sb = sa, pb = pa;
                if (ci.kind == 1) {
                    sb = slot;
                    pb = sphase;
                    if (++slot == static_cast<uint32_t>(a.slots)) { slot = 0; sphase ^= 1u; }
                }
                if (!ptx::mbar_wait_bounded(&s.slot_full[sa], pa, s.abort_flag, kWaitLimitNs) ||
                    (sb != sa && !ptx::mbar_wait_bounded(&s.slot_full[sb], pb, s.abort_flag, kWaitLimitNs)) ||
                    !ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                    raise_abort(s, a);
                    ok = false;
                    break;
                }
                const float* A = reinterpret_cast<const float*>(s.raw + sa * s.raw_bytes);
                const float* B = reinterpret_cast<const float*>(s.raw + sb * s.raw_bytes);
                uint8_t* pr = s.ring + stage * kPieces * s.piece_bytes;
                bool bad = false;
                for (int v = 0; v < items; ++v) {
                    const int t = lt + kBreedThreads * v;
                    const int r = t >> 3, c8 = t & 7;
                    const int kk = kc * kKStage + 8 * c8;
                    const bool row_ok = r < a.h;
                    const bool live = row_ok && kk < a.k;
                    const uint32_t gi = static_cast<uint32_t>(r * a.k + kk);  // gene index (< h d_0 < 2^31)
                    const uint32_t u = gi >> 3;
                    float4 x[2] = { make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f) };
                    if (live && ci.kind >= 0) load8(A, r * kKStage + 8 * c8, x);
                    if (ci.kind == 2) {
                        const uint32_t hit =
                            live ? mask8(philox_keyed(make_uint4(u, ent, a.gen, kTagMutMask), key), a.thr_mut) : 0u;
                        const int tb = lt - lane + kBreedThreads * v;  // item of lane 0
                        mutate8(sigma, a.gen, key, ent, hit, x, lane, job_z, job_code, [&](uint32_t o) {
                            const int to = tb + static_cast<int>(o);
                            return static_cast<uint32_t>((to >> 3) * a.k + kc * kKStage + 8 * (to & 7)) >> 3;
                        });
                    } else if (ci.kind == 1 && live) {
                        float4 y2[2];
                        load8(B, r * kKStage + 8 * c8, y2);
                        if (a.xo_op == 0) {
                            const uint32_t m = mask8(philox_keyed(make_uint4(u, ent, a.gen, kTagXo), key), a.thr_xo);
                            x[0] = select4(m, x[0], y2[0]);
                            x[1] = select4(m >> 4, x[1], y2[1]);
                        } else {
                            x[0] = mean4(x[0], y2[0]);
                            x[1] = mean4(x[1], y2[1]);
                        }
                    } else if (ci.kind == kKindInvalid && live) {
                        const float nan = __int_as_float(0x7FC00000);
                        x[0] = x[1] = make_float4(nan, nan, nan, nan);
                    }
                    if (live) {
                        float4* dst = reinterpret_cast<float4*>(child + gi);
                        dst[0] = x[0];
                        dst[1] = x[1];
                        bad |= out_of_piece_range(x[0]) || out_of_piece_range(x[1]);
                    }
                    if (row_ok) {
                        uint32_t p1[4], p2[4];
                        split2x2(x[0].x, x[0].y, p1[0], p2[0]);
                        split2x2(x[0].z, x[0].w, p1[1], p2[1]);
                        split2x2(x[1].x, x[1].y, p1[2], p2[2]);
                        split2x2(x[1].z, x[1].w, p1[3], p2[3]);
                        const uint32_t off = static_cast<uint32_t>(r) * 128u +
                                             ((static_cast<uint32_t>(c8) ^ static_cast<uint32_t>(r & 7)) << 4);
                        *reinterpret_cast<uint4*>(pr + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
                        *reinterpret_cast<uint4*>(pr + s.piece_bytes + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
                    }
                }
                if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) s.flag_unit[unit & 1u] = unit + 1u;
                ptx::fence_proxy_async_smem();
                if (kc == a.k_stages - 1) __threadfence_block();  // the child's W1 before the epilogue may read it
                __syncwarp();
                if (lane == 0) {
                    ptx::mbar_arrive(&s.slot_empty[sa]);
                    if (sb != sa) ptx::mbar_arrive(&s.slot_empty[sb]);
                    ptx::mbar_arrive(&s.full[stage]);
                    // the flag (if any) is released to the epilogue with this arrival
                    if (kc == a.k_stages - 1) ptx::mbar_arrive(&s.conv_done[unit & 1u]);
                }
                if (++stage == static_cast<uint32_t>(kPieceStages)) { stage = 0; phase ^= 1u; }
            }
        }
    } else {
        // ------------------------------------------------------------ batch into TMEM, then epilogue
        const int et = threadIdx.x - 32 * kFirstEpiWarp;
        const int q = warp & 3;  // TMEM lane quarter of this warp
        const int row = q * 32 + lane;
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        {
            // Row `row` of the batch into TMEM as FP16 pairs (lower k in the low
            // half); group g = levels 32 g .. 32 g + 31 = columns 16 g .. 16 g + 15.
            // A level k < 1024 is exact in FP16 as (1024 + k) - 1024, and
            // 1024 + k has the bit pattern 0x6400 | k.
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
                    ptx::named_barrier_sync(1, kEpiThreads);  // staging area read before the next chunk lands
                }
            } else {
                for (int g = 0; g < n_groups; ++g) {
                    uint32_t wds[8];
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        uint32_t word = 0;
                        if (live) {
#pragma unroll
                            for (int q8 = 0; q8 < 4; ++q8) {
                                const int kk = 32 * g + 4 * w + q8;
                                if (kk < a.k) word |= static_cast<uint32_t>(__ldg(xr + kk)) << (8 * q8);
                            }
                        }
                        wds[w] = word;
                    }
                    put_group(g, wds);
                }
            }
            ptx::mbar_arrive(s.x_loaded);
            ptx::tmem_st_wait();
            ptx::tc_fence_before();
            ptx::mbar_arrive(s.a_ready);
        }
        // Padding of the staged layer-2 parameters (never overwritten).
        for (int i = et; i < a.h * (a.dpad - a.d_out); i += kEpiThreads) {
            const int pad = a.dpad - a.d_out;
            s.w2t[(i / pad) * a.dpad + a.d_out + i % pad] = 0.0f;
        }
        if (et < 16 && et >= a.d_out) s.b2[et] = 0.0f;

        ptx::grid_dep_wait();  // kinds, parents, sigma genes and f_inh come from the selection kernel
        const PhiloxKeys key = philox_keys(a.seed);
        const int32_t label = row < a.batch ? a.y[row] : 0;
        const int64_t g_tail = static_cast<int64_t>(a.h) * a.k;  // first gene after W1 (a multiple of 16)
        const int32_t n_tail_units = static_cast<int32_t>((a.c_pad - g_tail) >> 3);
        const int32_t n_w2 = a.d_out * a.h;
        uint32_t acc_phase = 0, unit = 0;
        for (int n = blockIdx.x; n < a.pop; n += gridDim.x, ++unit) {
            const int j = child_of(a, n);
            const ChildInfo ci = child_info(a, j);
            const float sigma = a.sigma_child ? a.sigma_child[j] : a.sigma;
            const uint32_t ent = static_cast<uint32_t>(j);
            float* child = a.children + static_cast<int64_t>(j) * a.c_pad;
            // b1, W2, b2 and the padding of child j: bred here from the parents
            // in HBM (8 genes per thread), stored, and staged for layer 2.
            for (int ut = et; ut < n_tail_units; ut += kEpiThreads) {
                const int64_t i0 = g_tail + 8 * static_cast<int64_t>(ut);
                const uint32_t u = static_cast<uint32_t>(i0 >> 3);
                float4 x[2] = { make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f) };
                if (ci.kind >= 0) {
                    const float4* src = reinterpret_cast<const float4*>(a.parents + static_cast<int64_t>(ci.p1) * a.c_pad + i0);
                    x[0] = __ldg(src);
                    x[1] = __ldg(src + 1);
                }
                if (ci.kind == 1) {
                    const float4* src = reinterpret_cast<const float4*>(a.parents + static_cast<int64_t>(ci.p2) * a.c_pad + i0);
                    const float4 y0 = __ldg(src), y1 = __ldg(src + 1);
                    if (a.xo_op == 0) {
                        const uint32_t m = mask8(philox_keyed(make_uint4(u, ent, a.gen, kTagXo), key), a.thr_xo);
                        x[0] = select4(m, x[0], y0);
                        x[1] = select4(m >> 4, x[1], y1);
                    } else {
                        x[0] = mean4(x[0], y0);
                        x[1] = mean4(x[1], y1);
                    }
                } else if (ci.kind == 2) {
                    const uint32_t hit = mask8(philox_keyed(make_uint4(u, ent, a.gen, kTagMutMask), key), a.thr_mut);
                    mutate8_direct(sigma, a.gen, key, ent, u, hit, x);
                } else if (ci.kind == kKindInvalid) {
                    const float nan = __int_as_float(0x7FC00000);
                    x[0] = x[1] = make_float4(nan, nan, nan, nan);
                }
                float g8[8] = { x[0].x, x[0].y, x[0].z, x[0].w, x[1].x, x[1].y, x[1].z, x[1].w };
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if (i0 + e >= a.c) g8[e] = 0.0f;  // padding stays zero
                    const int32_t t = static_cast<int32_t>(i0 + e - g_tail);
                    if (t < a.h) {
                        s.b1[t] = g8[e];
                    } else if (t < a.h + n_w2) {
                        const int32_t tt = t - a.h, o = tt / a.h;
                        s.w2t[(tt - o * a.h) * a.dpad + o] = g8[e];
                    } else if (t < a.h + n_w2 + a.d_out) {
                        s.b2[t - a.h - n_w2] = g8[e];
                    }
                }
                float4* dst = reinterpret_cast<float4*>(child + i0);
                dst[0] = make_float4(g8[0], g8[1], g8[2], g8[3]);
                dst[1] = make_float4(g8[4], g8[5], g8[6], g8[7]);
            }
            ptx::named_barrier_sync(1, kEpiThreads);  // A1: the tail genes are staged
            if (et == 0) {
                bool got = ptx::mbar_wait_bounded(s.acc_full, acc_phase, s.abort_flag, kWaitLimitNs) &&
                           ptx::mbar_wait_bounded(&s.conv_done[unit & 1u], (unit >> 1) & 1u, s.abort_flag,
                                                  kWaitLimitNs);
                if (!got) raise_abort(s, a);
                *s.ep_go = !got ? 0 : (s.flag_unit[unit & 1u] == unit + 1u ? 2 : 1);
            }
            ptx::named_barrier_sync(1, kEpiThreads);  // A2: accumulator ready (or abort)
            const int go = *s.ep_go;
            if (!go) break;
            ptx::tc_fence_after();
            // Layer 1 from the accumulator (or, for a child with a weight
            // outside the piece range, by FP32 FFMA from HBM, k in order), 8
            // hidden units at a time, each folded into layer 2 at once.
            const float* w1p = child;
            const uint8_t* xrow = a.x + static_cast<int64_t>(row < a.batch ? row : 0) * a.k;
            float logit[kMaxOut];
#pragma unroll
            for (int o = 0; o < kMaxOut; ++o) logit[o] = 0.0f;
            for (int c = 0; c < a.h; c += 8) {
                uint32_t r8[8];
                ptx::tmem_ld8_nowait(tmem_base + lane_addr + static_cast<uint32_t>(c), r8);
                ptx::tmem_ld_wait();
                float v[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) v[jj] = __uint_as_float(r8[jj]);
                if (go == 2 && row < a.batch) {
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const float* wr = w1p + static_cast<int64_t>(c + jj) * a.k;
                        float acc = 0.0f;
                        for (int kk = 0; kk < a.k; ++kk) acc = fmaf(wr[kk], static_cast<float>(xrow[kk]), acc);
                        v[jj] = acc * kPieceScale;
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int col = c + jj;
                    const float hv = fmaxf(fmaf(v[jj], a.inv_div, s.b1[col]), 0.0f);
                    const float4* wr = reinterpret_cast<const float4*>(s.w2t + col * a.dpad);
#pragma unroll
                    for (int o4 = 0; o4 < kMaxOut / 4; ++o4) {
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
            ptx::mbar_arrive(s.acc_empty);  // the next child's MMAs may overwrite the accumulator
            acc_phase ^= 1u;
            float loss = 0.0f;
            int32_t good = 0;
            if (row < a.batch) {
                float z[kMaxOut];
#pragma unroll
                for (int o = 0; o < kMaxOut; ++o) z[o] = o < a.d_out ? logit[o] + s.b2[o] : 0.0f;
                float zmax = z[0];
                int arg = 0;
#pragma unroll
                for (int o = 1; o < kMaxOut; ++o)
                    if (o < a.d_out && z[o] > zmax) { zmax = z[o]; arg = o; }
                float se = 0.0f;
#pragma unroll
                for (int o = 0; o < kMaxOut; ++o)
                    if (o < a.d_out) se += expf(z[o] - zmax);
                if (label >= 0 && label < a.d_out) {
                    float zl = 0.0f;
#pragma unroll
                    for (int o = 0; o < kMaxOut; ++o)
                        if (o == label) zl = z[o];
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
            ptx::named_barrier_sync(1, kEpiThreads);  // B2: quarter sums written; staged parameters no longer read
            if (et == 0) {
                const float total = ((s.red_loss[0] + s.red_loss[1]) + s.red_loss[2]) + s.red_loss[3];
                const int32_t n_ok = s.red_ok[0] + s.red_ok[1] + s.red_ok[2] + s.red_ok[3];
                const float f = -(total / static_cast<float>(a.batch));
                a.f_raw[j] = f;
                if (a.f_adj) a.f_adj[j] = a.f_inh ? (1.0f - a.alpha) * a.f_inh[j] + a.alpha * f : f;
                if (a.correct) a.correct[j] = n_ok;
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

typedef CUresult (*FusedEncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                       const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

FusedEncodeTiledFn fused_encode_fn()
{
    static FusedEncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<FusedEncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

bool breed_eval_u8_supported(const NetLayout& net, int32_t batch, const float* parents, const float* children)
{
    if (net.n_layers != 2) return false;
    const int32_t k = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    if (k % 16 != 0 || h % 16 != 0 || h > 128 || d_out > kMaxOut || batch < 1 || batch > 128) return false;
    const int32_t a_cols = (k / 2 + 15) / 16 * 16;
    if (h + a_cols > static_cast<int32_t>(kTmemCols)) return false;
    if ((reinterpret_cast<uintptr_t>(parents) | reinterpret_cast<uintptr_t>(children)) & 15u) return false;
    int32_t slots = 0;
    return fused_slots(h, (d_out + 3) / 4 * 4, batch, &slots) && fused_encode_fn() != nullptr;
}

cudaError_t launch_breed_eval_u8(const BreedArgs& b, const NetLayout& net, const float* parents, const int32_t* par1,
                                 const int32_t* par2, const int32_t* kind, float* children, const uint8_t* x,
                                 float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                 float* f_raw, float* f_adj, int32_t* correct, unsigned int* status,
                                 cudaStream_t stream)
{
    FusedArgs a{};
    a.pop = b.pop;
    a.k = net.dims[0];
    a.h = net.dims[1];
    a.d_out = net.dims[2];
    a.dpad = (a.d_out + 3) / 4 * 4;
    a.batch = batch;
    a.k16 = a.k;  // k % 16 == 0
    a.k_stages = (a.k + kKStage - 1) / kKStage;
    a.c = net.c;
    a.c_pad = net.c_pad;
    a.xo_op = b.xo_op;
    a.thr_xo = b.thr_xo;
    a.thr_mut = b.thr_mut;
    a.sigma = b.sigma;
    a.sigma_child = b.sigma_child;
    a.seed = b.seed;
    a.gen = b.gen;
    a.inv_div = static_cast<float>(1.0 / (static_cast<double>(x_div) * kPieceScale));
    a.alpha = alpha;
    a.a_col = static_cast<uint32_t>(a.h);
    a.parents = parents;
    a.children = children;
    a.par1 = par1;
    a.par2 = par2;
    a.kind = kind;
    a.x = x;
    a.y = y;
    a.f_inh = f_inh;
    a.f_raw = f_raw;
    a.f_adj = f_adj;
    a.correct = correct;
    a.status = status;
    if (!fused_slots(a.h, a.dpad, a.batch, &a.slots)) return cudaErrorInvalidValue;
    const size_t smem = fused_smem_bytes(a.h, a.dpad, a.batch, a.slots);
    {
        // Batch staging in the tail of the rings: row stride kc + 16 bytes
        // (kc a multiple of 32) keeps the per-row 16-byte reads conflict-free.
        const int32_t raw_bytes = a.h * 256;
        const int32_t region = kPieceStages * kPieces * a.h * 128 + a.slots * raw_bytes;
        const int32_t n_groups = (a.k16 + 31) / 32;
        const int32_t kc = std::min(32 * n_groups, (region / a.batch - 16) / 32 * 32);
        a.x_staged = ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) && kc >= 32;
        a.x_kc = kc;
        a.x_stride = kc + 16;
        a.x_off = region - a.batch * a.x_stride;
        a.n_early = a.x_staged ? std::min(a.slots, a.x_off / raw_bytes) : 0;
    }
    FusedEncodeTiledFn enc = fused_encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tp;
    {
        const cuuint64_t dims[3] = { static_cast<cuuint64_t>(a.k), static_cast<cuuint64_t>(a.h),
                                     static_cast<cuuint64_t>(a.pop) };
        const cuuint64_t strides[2] = { static_cast<cuuint64_t>(a.k) * 4u, static_cast<cuuint64_t>(net.c_pad) * 4u };
        const cuuint32_t box[3] = { static_cast<cuuint32_t>(kKStage), static_cast<cuuint32_t>(a.h), 1 };
        const cuuint32_t es[3] = { 1, 1, 1 };
        if (enc(&tp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(parents), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(breed_eval_u8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int grid = a.pop < sms ? a.pop : sms;
    // Programmatic stream serialisation: barriers, TMEM and the batch may be
    // set up while the selection kernel finishes; every role waits for it
    // before it reads kinds, parents, sigma genes or f_inh.
    return launch_pdl(breed_eval_u8_kernel, dim3(grid), dim3(kFusedThreads), smem, stream, tp, a);
}

}  // namespace leea
