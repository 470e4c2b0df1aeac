// leea_eval_mlp_tc.cu -- fitness (Eq. 1) of nets with three hidden layers such
// as the paper's 196-256-128-64-10 (Section 4.1), on the tcgen05 tensor cores
// with FP32-class accuracy, for minibatches of 8-bit levels x = k / x_div.
//
// A unit is one individual on one 128-sample tile.  Layers 1-3 are MMAs with
// the samples as M = 128 and FP32 accumulation in tensor memory (layer 1 in
// columns [0, d1), layers 2 and 3 both from column d1: layer 3 starts after
// the epilogue has read layer 2):
//   layer 1     A = the tile's levels k, exact in FP16; B = 2^8 W1 as two FP16
//               pieces hi = fp16(2^8 w), lo = fp16(2^8 w - hi) (the remainder is
//               exact in FP32): 2 MMAs per 16 inputs, only the accumulation rounds
//   layers 2, 3 A = 2^8 h of the layer below and B = 2^8 W, both as two FP16
//               pieces: hi.hi + hi.lo + lo.hi; the dropped lo.lo term is below
//               2^-21 of the product.  For widths N <= 128 the two products of
//               the hi activations are one MMA of width 2N against the stacked
//               [W_hi; W_lo] block (its rows are contiguous), lo.hi adds onto
//               the second half, and the epilogue sums the halves: 2 MMAs per
//               16 inputs (an MMA of N = 256 costs little more than one of
//               N = 128), else 3
// The epilogue adds the bias and applies ReLU in FP32, splits the activations
// for the next layer, and computes layer 4 (d3 -> d_out), the softmax
// cross-entropy and the loss sums in FP32, tiles in order.  A weight or an
// activation with |v| >= 128 (2^8 |v| could overflow its FP16 piece) marks the
// individual; the CUDA-core kernel then recomputes its fitness in FP32.
// The weights are split once per evaluation (split_weights_kernel), and the
// batch's levels are converted once per evaluation into FP16 operand tiles
// (stage_levels_kernel), so a unit's layer-1 operands arrive by bulk copies and
// its layer-1 MMAs run while the epilogue finishes the previous unit.
//
// Warp roles (persistent CTA, one per SM; individuals strided by gridDim.x,
// their tiles in order):
//   warp 0      TMEM allocation and the single MMA-issuing thread
//   warp 1      producer: per unit, the tile's levels (one bulk copy into the
//               activation region), then one bulk copy per 64-input block of
//               W1, W2, W3, already split into FP16 pieces and swizzled by
//               split_weights_kernel, into one of two weight buffers
//   warps 2-9   the epilogue (TMEM lane = sample, two warps per lane
//               quarter, each with half of a layer's 16-column groups): the
//               activations of layers 1 and 2 as the next operands, layer 4
//               (the halves' partial logits added through shared memory) and
//               the loss
// The layers of a unit share one activation region, each layer's weight
// blocks double-buffered.  Layer 1's activations go to the layer-2 MMAs one
// 64-column block at a time (the epilogue halves take two of each block's four
// column groups); layer 3 starts after all of layer 2's; the next unit's
// levels and layer-1 MMAs start as soon as this unit's layer-3 MMAs are done.
// Every wait is bounded; on expiry the kernel sets kStatusEvalTimeout and exits.
#include <cuda.h>

#include <cuda_fp16.h>

#include <mutex>

#include "leea_internal.h"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kFirstEpiWarp = 2;
constexpr int kEpiWarps = 8;  // two per TMEM lane quarter: half of a layer's columns each
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kTcThreads = 32 * (kFirstEpiWarp + kEpiWarps);
constexpr int kTile = 128;                      // samples per unit (MMA M)
constexpr uint32_t kBlockBytes = kTile * 128;   // one 64-input block of a 128-row operand
constexpr uint32_t kHalfRegion = 4 * kBlockBytes;  // 64 KB: one piece of up to 256 inputs
constexpr uint32_t kRegionBytes = 2 * kHalfRegion;  // activations: hi piece, lo piece
constexpr uint32_t kSlotBytes = 2 * 256 * 128;      // weights: two pieces of up to 256 rows
constexpr int kMaxOutTc = 16;
constexpr uint32_t kTmemCols = 512;
constexpr float kPieceScale = 256.0f;
constexpr float kPieceRange = 128.0f;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr uint64_t kDrainLimitNs = 200000000ull;

struct MlpTcArgs {
    int32_t pop, batch, n_tiles;
    int32_t dims[5];     // d0, d1, d2, d3, d_out
    int32_t k16[3];      // inputs of layers 1-3 rounded up to 16
    int64_t c_pad;
    int64_t w_off[4], b_off[4];
    float inv_div;       // 2^-8 / x_div: layer-1 accumulator units to x units
    float alpha;
    const float* popv;
    const uint8_t* x;
    const int32_t* y;
    const float* f_inh;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    int32_t* flagged;    // [pop], zeroed before the launch: 1 = recompute in FP32
    // the batch's levels as FP16 layer-1 operand tiles: tile t (128 samples)
    // at byte t * x_bytes, its 64-input blocks of 128 swizzled 128-byte rows
    const uint8_t* xtiles;
    uint32_t x_bytes;
    unsigned int* status;
    // the weights of layers 1-3 as FP16 pieces, per individual (piece_stride
    // bytes): layer l's 64-input blocks from byte layer_off[l], each block the
    // hi piece (N rows of 128 bytes, swizzled) then the lo piece
    const uint8_t* pieces;
    int64_t piece_stride;
    int64_t layer_off[3];
};

struct TcSmem {
    uint8_t* region;  // activations: hi piece [0, 64 KB), lo piece [64 KB, 128 KB); the levels in the hi part
    uint8_t* slot;    // weights: hi piece then lo piece, N x 128 bytes each per 64-input block
    float *b1, *b2, *b3, *w4t, *b4;
    float* plog;  // [128][16]: the second half's partial layer-4 logits
    uint64_t *buf_full, *buf_empty, *x_full, *d_full, *h_blk, *h2_ready, *drain;
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
    float* red_loss;
    int32_t* red_ok;
};

__host__ __device__ inline size_t tc_param_floats(const int32_t* dims)
{
    return static_cast<size_t>(dims[1] + dims[2] + dims[3] + dims[3] * kMaxOutTc + kMaxOutTc + kTile * kMaxOutTc);
}

__host__ __device__ inline size_t tc_smem_bytes(const int32_t* dims)
{
    // room for 16 barriers (14 used) and 16 words (11 used)
    return 1024 + kRegionBytes + kSlotBytes + sizeof(float) * tc_param_floats(dims) + 8 * 16 + 64;
}

__device__ __forceinline__ TcSmem carve(uint8_t* raw, const MlpTcArgs& a)
{
    TcSmem s;
    s.region = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    s.slot = s.region + kRegionBytes;
    float* f = reinterpret_cast<float*>(s.slot + kSlotBytes);
    s.b1 = f;
    s.b2 = s.b1 + a.dims[1];
    s.b3 = s.b2 + a.dims[2];
    s.w4t = s.b3 + a.dims[3];
    s.b4 = s.w4t + a.dims[3] * kMaxOutTc;
    s.plog = s.b4 + kMaxOutTc;
    uint8_t* p = reinterpret_cast<uint8_t*>(s.plog + kTile * kMaxOutTc);
    p += (8u - (reinterpret_cast<uintptr_t>(p) & 7u)) & 7u;
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.buf_full = bars;       // [2]
    s.buf_empty = bars + 2;  // [2]
    s.x_full = bars + 4;
    s.d_full = bars + 5;     // [3]
    s.h_blk = bars + 8;      // [4]: a 64-column block of layer 1's activations is in
    s.h2_ready = bars + 12;  // layer 2's activations are in
    s.drain = bars + 13;
    uint32_t* w = reinterpret_cast<uint32_t*>(bars + 14);
    s.tmem_holder = w;
    s.abort_flag = reinterpret_cast<volatile int*>(w + 1);
    s.ep_go = reinterpret_cast<int*>(w + 2);
    s.red_loss = reinterpret_cast<float*>(w + 3);
    s.red_ok = reinterpret_cast<int32_t*>(w + 7);
    return s;
}

__device__ __forceinline__ void raise_abort(const TcSmem& s, const MlpTcArgs& a)
{
    *s.abort_flag = 1;
    atomicOr(a.status, kStatusEvalTimeout);
}

__device__ __forceinline__ uint32_t half2_bits(__half2 v)
{
    return *reinterpret_cast<uint32_t*>(&v);
}

// Two FP32 values as packed FP16 pieces of 2^8 v (lower index in the low half).
__device__ __forceinline__ void split2x2(float v0, float v1, uint32_t& p1, uint32_t& p2)
{
    const float s0 = v0 * kPieceScale, s1 = v1 * kPieceScale;
    const __half2 h1 = __floats2half2_rn(s0, s1);
    const float2 f1 = __half22float2(h1);
    p1 = half2_bits(h1);
    p2 = half2_bits(__floats2half2_rn(s0 - f1.x, s1 - f1.y));
}

// Byte offset of 16-byte chunk `ch` (inputs 8 ch .. 8 ch + 7 of a 64-input
// block) of row r in the 128-byte swizzled K-major layout.
__device__ __forceinline__ uint32_t swz(int r, int ch)
{
    return static_cast<uint32_t>(r) * 128u + ((static_cast<uint32_t>(ch) ^ static_cast<uint32_t>(r & 7)) << 4);
}

__device__ __forceinline__ int layer_blocks(const MlpTcArgs& a, int l) { return (a.k16[l] + 63) / 64; }

// The weight blocks of a layer alternate between two buffers, so that one is
// converted while the MMAs read the other.  Layer 1: the slot, and the lo half
// of the activation region (it holds nothing while layer 1 runs: the levels
// use the hi half).  Layers 2 and 3 with N <= 128 (blocks of <= 32 KB): the
// slot's two halves; wider ones take the whole slot for every block.
__device__ __forceinline__ int buffer_of(const MlpTcArgs& a, int l, int kb)
{
    return (l == 0 || a.dims[l + 1] <= 128) ? (kb & 1) : 0;
}

// Offset of weight buffer b of layer l from the start of the region.
__device__ __forceinline__ uint32_t buffer_offset(int l, int b)
{
    if (b == 0) return kRegionBytes;
    return l == 0 ? kHalfRegion : kRegionBytes + kSlotBytes / 2;
}

// 16 accumulator columns of this thread's lane from TMEM address taddr; for a
// merged layer the sum of the two halves (hi.hi + (hi.lo + lo.hi)).
__device__ __forceinline__ void load_acc16(uint32_t taddr, uint32_t half_cols, bool merged, float (&v)[16])
{
    uint32_t r[16];
    ptx::tmem_ld16_nowait(taddr, r);
    if (merged) {
        uint32_t r2[16];
        ptx::tmem_ld16_nowait(taddr + half_cols, r2);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]) + __uint_as_float(r2[i]);
    } else {
        ptx::tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
    }
}

// Layers 2 and 3 (width n, layer 1 of width d1 in the columns below them) take
// the hi activations' two products as one MMA of width 2n where 2n fits both
// the MMA (N <= 256) and tensor memory.
__host__ __device__ inline bool merged_layer(int32_t d1, int32_t n)
{
    return 2 * n <= 256 && d1 + 2 * n <= static_cast<int32_t>(kTmemCols);
}

__global__ void __launch_bounds__(kTcThreads, 1) eval_mlp_tc_kernel(const MlpTcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const TcSmem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d1 = a.dims[1], d2 = a.dims[2], d3 = a.dims[3], d_out = a.dims[4];
    // Layer 3 reuses layer 2's columns; a merged layer (2N columns: hi.hi, then
    // hi.lo + lo.hi) where its width allows.
    const bool merged2 = merged_layer(d1, d2), merged3 = merged_layer(d1, d3);
    auto col = [&](int l) { return l == 0 ? 0u : static_cast<uint32_t>(d1); };
    auto merged = [&](int l) { return l == 1 ? merged2 : (l == 2 && merged3); };

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.buf_full[i], 1);
            ptx::mbar_init(&s.buf_empty[i], 1);
        }
        ptx::mbar_init(s.x_full, 1);
        for (int i = 0; i < 3; ++i) ptx::mbar_init(&s.d_full[i], 1);
        for (int i = 0; i < 4; ++i) ptx::mbar_init(&s.h_blk[i], kEpiThreads);
        ptx::mbar_init(s.h2_ready, kEpiThreads);
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
            const uint32_t region = ptx::smem_u32(s.region);
            uint32_t unit = 0, bphase = 0;  // bit b: phase of weight buffer b
            bool ok = true;
            for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
                for (int t = 0; ok && t < a.n_tiles; ++t, ++unit) {
                    if (!ptx::mbar_wait_bounded(s.x_full, unit & 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    for (int l = 0; ok && l < 3; ++l) {
                        // layer 3 after all of layer 2's activations (it reuses layer 2's
                        // columns); layer 2 block by block below
                        if (l == 2 && !ptx::mbar_wait_bounded(s.h2_ready, unit & 1u, s.abort_flag, kWaitLimitNs)) {
                            raise_abort(s, a);
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t n = static_cast<uint32_t>(a.dims[l + 1]);
                        const uint32_t idesc = ptx::idesc_f16(kTile, n);
                        const uint32_t idesc2 = ptx::idesc_f16(kTile, 2u * n);
                        const uint32_t d_tmem = tmem_base + col(l);
                        const int blocks = layer_blocks(a, l);
                        for (int kb = 0; kb < blocks; ++kb) {
                            const int b = buffer_of(a, l, kb);
                            if (!ptx::mbar_wait_bounded(&s.buf_full[b], (bphase >> b) & 1u, s.abort_flag,
                                                        kWaitLimitNs)) {
                                raise_abort(s, a);
                                ok = false;
                                break;
                            }
                            bphase ^= 1u << b;
                            if (l == 1 &&
                                !ptx::mbar_wait_bounded(&s.h_blk[kb], unit & 1u, s.abort_flag, kWaitLimitNs)) {
                                raise_abort(s, a);
                                ok = false;
                                break;
                            }
                            const uint32_t slot = region + buffer_offset(l, b);
                            ptx::tc_fence_after();
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const int kg = kb * 64 + kk * 16;
                                if (kg >= a.k16[l]) break;
                                const uint32_t a_hi = region + kb * kBlockBytes + kk * 32u;
                                const uint32_t b_hi = slot + kk * 32u;
                                const uint32_t b_lo = slot + n * 128u + kk * 32u;
                                const uint32_t first = (kb | kk) == 0 ? 0u : 1u;
                                if (merged(l)) {
                                    // [hi.hi | hi.lo] against the stacked block, then lo.hi onto the second half
                                    ptx::mma_f16(d_tmem, ptx::smem_desc_sw128(a_hi), ptx::smem_desc_sw128(b_hi),
                                                 idesc2, first);
                                    ptx::mma_f16(d_tmem + n, ptx::smem_desc_sw128(a_hi + kHalfRegion),
                                                 ptx::smem_desc_sw128(b_hi), idesc, 1u);
                                    continue;
                                }
                                ptx::mma_f16(d_tmem, ptx::smem_desc_sw128(a_hi), ptx::smem_desc_sw128(b_hi), idesc,
                                             first);
                                ptx::mma_f16(d_tmem, ptx::smem_desc_sw128(a_hi), ptx::smem_desc_sw128(b_lo), idesc,
                                             1u);
                                if (l > 0)
                                    ptx::mma_f16(d_tmem, ptx::smem_desc_sw128(a_hi + kHalfRegion),
                                                 ptx::smem_desc_sw128(b_hi), idesc, 1u);
                            }
                            ptx::mma_commit(&s.buf_empty[b]);
                        }
                        if (ok) ptx::mma_commit(&s.d_full[l]);
                    }
                }
            }
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kWaitLimitNs : kDrainLimitNs);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ producer
        // One bulk copy per 64-input weight block: the pieces are already in
        // the swizzled operand layout (split_weights_kernel).
        if (lane == 0) {
            uint32_t bphase = 0, unit = 0;
            uint32_t issued = 0, parity = 0;  // per buffer: a copy was issued / the parity it completes
            uint32_t x_issued = 0;            // level copies issued (at most the last one in flight)
            bool ok = true;
            for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
                const uint8_t* src_p = a.pieces + static_cast<int64_t>(p) * a.piece_stride;
                for (int t = 0; ok && t < a.n_tiles; ++t, ++unit) {
                    // The activation region and the buffers of this unit's layer 1
                    // (the slot, the region's lo half) are free once the previous
                    // unit's last MMAs are done: the tile's levels into the hi half.
                    if (unit > 0 &&
                        !ptx::mbar_wait_bounded(&s.d_full[2], (unit - 1) & 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(s.x_full, a.x_bytes);
                    ptx::bulk_load(s.region, a.xtiles + static_cast<int64_t>(t) * a.x_bytes, a.x_bytes, s.x_full);
                    ++x_issued;
                    for (int l = 0; ok && l < 3; ++l) {
                        const uint32_t bytes = static_cast<uint32_t>(a.dims[l + 1]) * 256u;
                        const int blocks = layer_blocks(a, l);
                        for (int kb = 0; kb < blocks; ++kb) {
                            const int b = buffer_of(a, l, kb);
                            if (!ptx::mbar_wait_bounded(&s.buf_empty[b], ((bphase >> b) & 1u) ^ 1u, s.abort_flag,
                                                        kWaitLimitNs)) {
                                raise_abort(s, a);
                                ok = false;
                                break;
                            }
                            ptx::mbar_arrive_expect_tx(&s.buf_full[b], bytes);
                            ptx::bulk_load(s.region + buffer_offset(l, b),
                                           src_p + a.layer_off[l] + static_cast<int64_t>(kb) * bytes, bytes,
                                           &s.buf_full[b]);
                            issued |= 1u << b;
                            parity = (parity & ~(1u << b)) | (((bphase >> b) & 1u) << b);
                            bphase ^= 1u << b;
                        }
                    }
                }
            }
            if (!ok) {  // let copies in flight land before the CTA exits
                volatile int never = 0;
                for (int b = 0; b < 2; ++b)
                    if (issued & (1u << b))
                        ptx::mbar_wait_bounded(&s.buf_full[b], (parity >> b) & 1u, &never, kDrainLimitNs);
                if (x_issued) ptx::mbar_wait_bounded(s.x_full, (x_issued - 1) & 1u, &never, kDrainLimitNs);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int et = threadIdx.x - 32 * kFirstEpiWarp;
        const int q = warp & 3;
        const int half = (warp - kFirstEpiWarp) >> 2;
        const int row = q * 32 + lane;
        const uint32_t lane_addr = static_cast<uint32_t>(q * 32) << 16;
        uint32_t unit = 0;
        bool ok = true;
        for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
            const float* net = a.popv + static_cast<int64_t>(p) * a.c_pad;
            // Biases and layer 4 of individual p (row-major W4 -> [d3][16]).
            ptx::named_barrier_sync(1, kEpiThreads);  // the previous individual's parameters are no longer read
            for (int i = et; i < d1; i += kEpiThreads) s.b1[i] = net[a.b_off[0] + i];
            for (int i = et; i < d2; i += kEpiThreads) s.b2[i] = net[a.b_off[1] + i];
            for (int i = et; i < d3; i += kEpiThreads) s.b3[i] = net[a.b_off[2] + i];
            for (int i = et; i < d3 * kMaxOutTc; i += kEpiThreads) {
                const int c = i / kMaxOutTc, o = i % kMaxOutTc;
                s.w4t[i] = o < d_out ? net[a.w_off[3] + static_cast<int64_t>(o) * d3 + c] : 0.0f;
            }
            if (et < kMaxOutTc) s.b4[et] = et < d_out ? net[a.b_off[3] + et] : 0.0f;
            ptx::named_barrier_sync(1, kEpiThreads);
            float total = 0.0f;
            int32_t n_ok = 0;
            bool bad = false;
            for (int t = 0; t < a.n_tiles; ++t, ++unit) {
                const int smp = t * kTile + row;
                const bool live = smp < a.batch;
                // layers 1 and 2: bias, ReLU, split for the next layer; layer 3: ReLU, layer 4, loss
                for (int l = 0; l < 3; ++l) {
                    if (et == 0) {
                        const bool got = ptx::mbar_wait_bounded(&s.d_full[l], unit & 1u, s.abort_flag, kWaitLimitNs);
                        if (!got) raise_abort(s, a);
                        *s.ep_go = got ? 1 : 0;
                    }
                    ptx::named_barrier_sync(1, kEpiThreads);
                    if (!*s.ep_go) { ok = false; break; }
                    ptx::tc_fence_after();
                    const int N = a.dims[l + 1];
                    const float* bias = l == 0 ? s.b1 : (l == 1 ? s.b2 : s.b3);
                    const float scale = l == 0 ? a.inv_div : 1.0f / (kPieceScale * kPieceScale);
                    // this half's 16-column groups
                    const int groups = N / 16, g0 = half ? groups / 2 : 0, g1 = half ? groups : groups / 2;
                    if (l < 2) {
                        // 64-column blocks in order, two of each block's four groups per
                        // half; layer 1's blocks go to the layer-2 MMAs one by one
                        for (int gi = 0; gi < 2 * ((N + 63) / 64); ++gi) {
                            const int kb = gi >> 1, g = 4 * kb + 2 * half + (gi & 1);
                            const int c = 16 * g;
                            if (g < groups) {
                                float v[16];
                                load_acc16(tmem_base + lane_addr + col(l) + static_cast<uint32_t>(c),
                                           static_cast<uint32_t>(N), merged(l), v);
                                uint32_t hi[8], lo[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    const float h0 = fmaxf(fmaf(v[2 * e], scale, bias[c + 2 * e]), 0.0f);
                                    const float h1 = fmaxf(fmaf(v[2 * e + 1], scale, bias[c + 2 * e + 1]), 0.0f);
                                    bad |= h0 >= kPieceRange || h1 >= kPieceRange;
                                    split2x2(h0, h1, hi[e], lo[e]);
                                }
                                uint8_t* dst = s.region + (c >> 6) * kBlockBytes;
                                const int ch = (c & 63) >> 3;
                                *reinterpret_cast<uint4*>(dst + swz(row, ch)) =
                                    make_uint4(hi[0], hi[1], hi[2], hi[3]);
                                *reinterpret_cast<uint4*>(dst + swz(row, ch + 1)) =
                                    make_uint4(hi[4], hi[5], hi[6], hi[7]);
                                *reinterpret_cast<uint4*>(dst + kHalfRegion + swz(row, ch)) =
                                    make_uint4(lo[0], lo[1], lo[2], lo[3]);
                                *reinterpret_cast<uint4*>(dst + kHalfRegion + swz(row, ch + 1)) =
                                    make_uint4(lo[4], lo[5], lo[6], lo[7]);
                            }
                            if (l == 0 && (gi & 1)) {
                                ptx::fence_proxy_async_smem();
                                ptx::tc_fence_before();
                                ptx::mbar_arrive(&s.h_blk[kb]);
                            }
                        }
                        if (l == 1) {
                            ptx::fence_proxy_async_smem();
                            ptx::tc_fence_before();
                            ptx::mbar_arrive(s.h2_ready);
                        }
                    } else {
                        // layer 3's ReLU, then layer 4 and the loss in FP32
                        float logit[kMaxOutTc];
#pragma unroll
                        for (int o = 0; o < kMaxOutTc; ++o) logit[o] = 0.0f;
                        for (int c = 16 * g0; c < 16 * g1; c += 16) {
                            float v[16];
                            load_acc16(tmem_base + lane_addr + col(l) + static_cast<uint32_t>(c),
                                       static_cast<uint32_t>(N), merged(l), v);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float h = fmaxf(fmaf(v[j], scale, bias[c + j]), 0.0f);
                                const float4* wr = reinterpret_cast<const float4*>(s.w4t + (c + j) * kMaxOutTc);
#pragma unroll
                                for (int o4 = 0; o4 < kMaxOutTc / 4; ++o4) {
                                    if (4 * o4 < d_out) {
                                        const float4 w4 = wr[o4];
                                        logit[4 * o4 + 0] = fmaf(w4.x, h, logit[4 * o4 + 0]);
                                        logit[4 * o4 + 1] = fmaf(w4.y, h, logit[4 * o4 + 1]);
                                        logit[4 * o4 + 2] = fmaf(w4.z, h, logit[4 * o4 + 2]);
                                        logit[4 * o4 + 3] = fmaf(w4.w, h, logit[4 * o4 + 3]);
                                    }
                                }
                            }
                        }
                        ptx::tc_fence_before();
                        if (half == 1) {
#pragma unroll
                            for (int o = 0; o < kMaxOutTc; ++o) s.plog[row * kMaxOutTc + o] = logit[o];
                        }
                        ptx::named_barrier_sync(1, kEpiThreads);  // the second half's partial logits are in
                        float loss = 0.0f;
                        int32_t good = 0;
                        if (live && half == 0) {
                            float z[kMaxOutTc];
#pragma unroll
                            for (int o = 0; o < kMaxOutTc; ++o)
                                z[o] = o < d_out ? (logit[o] + s.plog[row * kMaxOutTc + o]) + s.b4[o] : 0.0f;
                            float zmax = z[0];
                            int arg = 0;
#pragma unroll
                            for (int o = 1; o < kMaxOutTc; ++o)
                                if (o < d_out && z[o] > zmax) { zmax = z[o]; arg = o; }
                            float se = 0.0f;
#pragma unroll
                            for (int o = 0; o < kMaxOutTc; ++o)
                                if (o < d_out) se += expf(z[o] - zmax);
                            const int32_t lbl = a.y[smp];
                            if (lbl >= 0 && lbl < d_out) {
                                float zl = 0.0f;
#pragma unroll
                                for (int o = 0; o < kMaxOutTc; ++o)
                                    if (o == lbl) zl = z[o];
                                loss = logf(se) + zmax - zl;
                                good = arg == lbl ? 1 : 0;
                            } else {
                                loss = __int_as_float(0x7FC00000);
                            }
                        }
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) {
                            loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
                            good += __shfl_xor_sync(0xFFFFFFFFu, good, off);
                        }
                        if (lane == 0 && half == 0) {
                            s.red_loss[q] = loss;
                            s.red_ok[q] = good;
                        }
                        ptx::named_barrier_sync(1, kEpiThreads);
                        if (et == 0) {
                            total += ((s.red_loss[0] + s.red_loss[1]) + s.red_loss[2]) + s.red_loss[3];
                            n_ok += s.red_ok[0] + s.red_ok[1] + s.red_ok[2] + s.red_ok[3];
                        }
                    }
                }
                if (!ok) break;
            }
            if (!ok) break;
            if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) a.flagged[p] = 1;
            if (et == 0) {
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

// Each individual's weights of layers 1-3 as FP16 pieces of 2^8 w in the
// swizzled operand layout (individuals strided over blockIdx.y); a weight
// |w| >= 128 marks the individual for the FP32 recomputation.
__global__ void __launch_bounds__(256) split_weights_kernel(const MlpTcArgs a)
{
    for (int p = blockIdx.y; p < a.pop; p += gridDim.y) {
        const float* net = a.popv + static_cast<int64_t>(p) * a.c_pad;
        uint8_t* dst_p = const_cast<uint8_t*>(a.pieces) + static_cast<int64_t>(p) * a.piece_stride;
        int n_items[3];
        for (int l = 0; l < 3; ++l) n_items[l] = layer_blocks(a, l) * a.dims[l + 1] * 8;
        const int total = n_items[0] + n_items[1] + n_items[2];
        bool bad = false;
        for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
            int l = 0, r = it;
            while (r >= n_items[l]) r -= n_items[l++];
            const int K = a.dims[l], N = a.dims[l + 1];
            const int kb = r / (N * 8), rem = r - kb * N * 8;
            const int n = rem >> 3, ch = rem & 7;
            const int k = kb * 64 + 8 * ch;
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
            if (k < K) {
                const float4* src = reinterpret_cast<const float4*>(net + a.w_off[l] + static_cast<int64_t>(n) * K + k);
                v0 = __ldg(src);
                if (k + 4 < K) v1 = __ldg(src + 1);
            }
            const float w[8] = { v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w };
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                split2x2(w[2 * e], w[2 * e + 1], hi[e], lo[e]);
                bad |= fabsf(w[2 * e]) >= kPieceRange || fabsf(w[2 * e + 1]) >= kPieceRange;
            }
            uint8_t* blk = dst_p + a.layer_off[l] + static_cast<int64_t>(kb) * N * 256;
            const uint32_t off = swz(n, ch);
            *reinterpret_cast<uint4*>(blk + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(blk + N * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        if (bad) a.flagged[p] = 1;
    }
}

// The batch's levels as FP16 layer-1 operand tiles (exact: integers below 2048
// are FP16 values).  Item = (tile t, 64-input block kb, row r, 16-byte chunk
// ch): levels kb * 64 + 8 ch .. + 7 of sample t * 128 + r, swizzled like the
// weight pieces; levels past d0 and samples past the batch are 0.
__global__ void __launch_bounds__(256) stage_levels_kernel(const MlpTcArgs a, const uint8_t* __restrict__ x)
{
    const int blocks = layer_blocks(a, 0), d0 = a.dims[0];
    const int items = a.n_tiles * blocks * kTile * 8;
    uint8_t* out = const_cast<uint8_t*>(a.xtiles);
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        const int ch = it & 7, r = (it >> 3) % kTile, tb = (it >> 3) / kTile;
        const int t = tb / blocks, kb = tb - t * blocks;
        const int smp = t * kTile + r, k0 = kb * 64 + 8 * ch;
        const uint8_t* xr = x + static_cast<int64_t>(smp) * d0;
        uint32_t h[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + 2 * e;
            const float v0 = (smp < a.batch && k < d0) ? static_cast<float>(xr[k]) : 0.0f;
            const float v1 = (smp < a.batch && k + 1 < d0) ? static_cast<float>(xr[k + 1]) : 0.0f;
            h[e] = half2_bits(__floats2half2_rn(v0, v1));
        }
        *reinterpret_cast<uint4*>(out + static_cast<int64_t>(t) * a.x_bytes + kb * kBlockBytes + swz(r, ch)) =
            make_uint4(h[0], h[1], h[2], h[3]);
    }
}

// Library-owned scratch (weight pieces, marks), grown on demand, for callers
// that bring none: one buffer per device, for the device current at the call
// (a buffer of another device would be another GPU's memory).
uint8_t* shared_scratch(size_t bytes)
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static uint8_t* buf[kMaxDevices] = { nullptr };
    static size_t cap[kMaxDevices] = { 0 };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (bytes > cap[dev]) {
        if (buf[dev]) cudaFree(buf[dev]);  // synchronises the device: earlier calls' kernels are done with it
        buf[dev] = nullptr;
        cap[dev] = 0;
        if (cudaMalloc(&buf[dev], bytes) != cudaSuccess) {
            buf[dev] = nullptr;
            return nullptr;
        }
        cap[dev] = bytes;
    }
    return buf[dev];
}

// Bytes of one individual's weight pieces; byte offset of each layer's blocks.
int64_t piece_layout(const NetLayout& net, int64_t* layer_off)
{
    int64_t off = 0;
    for (int l = 0; l < 3; ++l) {
        layer_off[l] = off;
        const int64_t k16 = (net.dims[l] + 15) / 16 * 16;
        off += (k16 + 63) / 64 * net.dims[l + 1] * 256;
    }
    return off;
}

// Bytes of one tile's levels (64-input blocks of 128 rows of 128 bytes).
uint32_t level_tile_bytes(const NetLayout& net)
{
    return static_cast<uint32_t>((net.dims[0] + 63) / 64) * kBlockBytes;
}

// Scratch layout: the pieces (a multiple of 256 bytes), the marks (rounded up
// to 256 bytes), the level tiles.
size_t marks_bytes(int32_t pop)
{
    return (sizeof(int32_t) * static_cast<size_t>(pop) + 255) / 256 * 256;
}

}  // namespace

size_t eval_mlp_tc_scratch_bytes(const NetLayout& net, int32_t pop, int32_t batch)
{
    int64_t layer_off[3];
    const size_t pieces = static_cast<size_t>(piece_layout(net, layer_off)) * static_cast<size_t>(pop);
    const size_t tiles = static_cast<size_t>((batch + kTile - 1) / kTile);
    return pieces + marks_bytes(pop) + tiles * level_tile_bytes(net);
}

bool eval_mlp_tc_supported(const NetLayout& net, const float* pop_dev)
{
    if (net.n_layers != 4) return false;
    const int32_t d0 = net.dims[0], d1 = net.dims[1], d2 = net.dims[2], d3 = net.dims[3], d_out = net.dims[4];
    if (d0 % 4 != 0 || d0 > 256 || d_out > kMaxOutTc) return false;
    for (int32_t n : { d1, d2, d3 })
        if (n % 16 != 0 || n < 16 || n > 256) return false;
    // layer 1 in [0, d1), layers 2 and 3 from column d1 (2n columns if merged)
    for (int32_t n : { d2, d3 })
        if (d1 + (merged_layer(d1, n) ? 2 * n : n) > static_cast<int32_t>(kTmemCols)) return false;
    for (int l = 0; l < 3; ++l)
        if (net.w_off[l] % 4 != 0) return false;
    if (reinterpret_cast<uintptr_t>(pop_dev) & 15u) return false;
    return tc_smem_bytes(net.dims) <= 227u * 1024u;
}

cudaError_t launch_eval_mlp_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x, float x_div,
                               const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                               float* f_adj, int32_t* correct, unsigned int* status, cudaStream_t stream,
                               void* scratch)
{
    MlpTcArgs a{};
    a.pop = pop;
    a.batch = batch;
    a.n_tiles = (batch + kTile - 1) / kTile;
    for (int l = 0; l <= 4; ++l) a.dims[l] = net.dims[l];
    for (int l = 0; l < 3; ++l) a.k16[l] = (net.dims[l] + 15) / 16 * 16;
    a.c_pad = net.c_pad;
    for (int l = 0; l < 4; ++l) {
        a.w_off[l] = net.w_off[l];
        a.b_off[l] = net.b_off[l];
    }
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
    a.piece_stride = piece_layout(net, a.layer_off);
    const size_t pieces = static_cast<size_t>(a.piece_stride) * static_cast<size_t>(pop);
    uint8_t* base =
        scratch ? static_cast<uint8_t*>(scratch) : shared_scratch(eval_mlp_tc_scratch_bytes(net, pop, batch));
    if (!base) return cudaErrorMemoryAllocation;
    a.pieces = base;
    a.flagged = reinterpret_cast<int32_t*>(base + pieces);  // pieces: a multiple of 256 bytes
    a.x_bytes = level_tile_bytes(net);
    a.xtiles = base + pieces + marks_bytes(pop);
    cudaError_t err = cudaMemsetAsync(a.flagged, 0, sizeof(int32_t) * static_cast<size_t>(pop), stream);
    if (err != cudaSuccess) return err;
    {
        int items = 0;
        for (int l = 0; l < 3; ++l) items += ((a.k16[l] + 63) / 64) * net.dims[l + 1] * 8;
        split_weights_kernel<<<dim3((items + 255) / 256, pop < 65535 ? pop : 65535), 256, 0, stream>>>(a);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        const int level_items = a.n_tiles * ((a.dims[0] + 63) / 64) * kTile * 8;
        stage_levels_kernel<<<(level_items + 255) / 256, 256, 0, stream>>>(a, x);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    const size_t smem = tc_smem_bytes(net.dims);
    err = cudaFuncSetAttribute(eval_mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    const int grid = pop < sms ? pop : sms;
    eval_mlp_tc_kernel<<<grid, kTcThreads, smem, stream>>>(a);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    // Individuals with a weight or activation outside the FP16 pieces' range:
    // their fitness again, in FP32 on the CUDA cores.
    return launch_eval_mlp_u8_only(net, pop, pop_dev, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct,
                                   a.flagged, stream);
}

}  // namespace leea
