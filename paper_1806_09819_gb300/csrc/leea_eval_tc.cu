// leea_eval_tc.cu -- fitness of every individual on one shared minibatch
// (Eq. 1; Section 3.3's population-batched forward pass) on the tcgen05 tensor
// cores, FP32-class accuracy by a three-term TF32 split.
//
// Per individual p the hidden pre-activations are D = X W1_p^T: A = X (a tile
// of 128 samples x K), B = W1_p (h rows x K), both K-major, D (128 x h, FP32)
// in tensor memory.  Every operand is split in shared memory into
// hi = TF32 truncation and lo = x - hi, and D accumulates
// X_hi W_hi + X_hi W_lo + X_lo W_hi (the dropped lo*lo term is ~2^-22
// relative).  With a TMEM lane per sample, the epilogue thread of sample b
// reads its h accumulators, applies bias + ReLU, layer 2 (d_out <= 16) and
// the softmax cross-entropy in registers; the batch sum uses a fixed order.
//
// Warp roles (persistent CTA, one per SM, individuals strided by gridDim.x):
//   warp 0      TMA producer: X tile (128 x 32 floats) and W1 tile (h x 32)
//               per stage, 128-byte swizzle, zero fill past K, h and batch
//   warp 1      TMEM allocation and the single MMA-issuing thread
//   warps 2-5   hi/lo split of each stage (in place + lo buffers)
//   warps 6-9   epilogue from the double-buffered TMEM accumulators
// Every mbarrier wait is bounded in time; on expiry the kernel records
// kStatusEvalTimeout in the status word, drains its async work and exits.
#include <cuda.h>

#include "leea_internal.h"
#include "tc_ptx.cuh"

namespace leea {

namespace {

constexpr int kTcThreads = 320;
constexpr int kKChunk = 32;                       // floats of K per stage (one 128-byte row)
constexpr int kMTile = 128;                       // samples per accumulator
constexpr int kMaxOutTc = 16;
constexpr uint32_t kXTileBytes = kMTile * kKChunk * 4;
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait
constexpr uint64_t kDrainLimitNs = 200000000ull;  // 0.2 s when draining after an abort

struct EvalTcArgs {
    int32_t pop, h, npad, d_out, batch, k_chunks, m_tiles, stages;
    int64_t c_pad;
    int32_t k;
    float alpha;
    uint32_t acc_stride, tmem_cols, params_floats, params_bytes;
    const float* popv;
    const int32_t* y;
    const float* f_inh;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    unsigned int* status;
};

struct TcSmem {
    uint8_t* base;
    uint32_t stage_bytes, w_bytes;
    float* prm;
    uint64_t *full, *split, *empty, *acc_full, *acc_empty, *drain;
    uint32_t* tmem_holder;
    volatile int* abort_flag;
    int* ep_go;
    float* red_loss;
    int32_t* red_ok;
};

__device__ __forceinline__ TcSmem carve(uint8_t* raw, const EvalTcArgs& a)
{
    TcSmem s;
    s.base = raw + ((1024u - (ptx::smem_u32(raw) & 1023u)) & 1023u);
    s.w_bytes = static_cast<uint32_t>(a.npad) * 128u;
    s.stage_bytes = 2u * kXTileBytes + 2u * s.w_bytes;
    uint8_t* p = s.base + a.stages * s.stage_bytes;
    s.prm = reinterpret_cast<float*>(p);
    p += a.params_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(p);
    s.full = bars;
    s.split = bars + a.stages;
    s.empty = bars + 2 * a.stages;
    s.acc_full = bars + 3 * a.stages;
    s.acc_empty = s.acc_full + 2;
    s.drain = s.acc_empty + 2;
    uint32_t* w = reinterpret_cast<uint32_t*>(s.drain + 1);
    s.tmem_holder = w;
    s.abort_flag = reinterpret_cast<volatile int*>(w + 1);
    s.ep_go = reinterpret_cast<int*>(w + 2);
    s.red_loss = reinterpret_cast<float*>(w + 4);
    s.red_ok = reinterpret_cast<int32_t*>(w + 8);
    return s;
}

__device__ __forceinline__ void raise_abort(const TcSmem& s, const EvalTcArgs& a)
{
    *s.abort_flag = 1;
    atomicOr(a.status, kStatusEvalTimeout);
}

__device__ __forceinline__ float tf32_hi(float v)
{
    return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
}

__global__ void __launch_bounds__(kTcThreads, 1)
eval_tc_kernel(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_w,
               const EvalTcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const TcSmem s = carve(smem_raw, a);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.stages; ++i) {
            ptx::mbar_init(&s.full[i], 1);
            ptx::mbar_init(&s.split[i], 128);
            ptx::mbar_init(&s.empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&s.acc_full[i], 1);
            ptx::mbar_init(&s.acc_empty[i], 128);
        }
        ptx::mbar_init(s.drain, 1);
        *s.abort_flag = 0;
        *s.ep_go = 0;
        ptx::fence_mbar_init();
        ptx::tma_prefetch_map(&tmap_x);
        ptx::tma_prefetch_map(&tmap_w);
    }
    if (warp == 1) ptx::tmem_alloc(s.tmem_holder, a.tmem_cols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem_base = *s.tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            uint32_t issued_mask = 0, parity_mask = 0;  // per stage: issued at all / parity of the last issue
            bool ok = true;
            for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
                for (int mt = 0; ok && mt < a.m_tiles; ++mt) {
                    for (int kc = 0; kc < a.k_chunks; ++kc) {
                        if (!ptx::mbar_wait_bounded(&s.empty[stage], phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                            raise_abort(s, a);
                            ok = false;
                            break;
                        }
                        uint8_t* st = s.base + stage * s.stage_bytes;
                        ptx::mbar_arrive_expect_tx(&s.full[stage], kXTileBytes + s.w_bytes);
                        ptx::tma_load_2d(st, &tmap_x, &s.full[stage], kc * kKChunk, mt * kMTile);
                        ptx::tma_load_3d(st + 2 * kXTileBytes, &tmap_w, &s.full[stage], kc * kKChunk, 0, p);
                        issued_mask |= 1u << stage;
                        parity_mask = (parity_mask & ~(1u << stage)) | (phase << stage);
                        if (++stage == static_cast<uint32_t>(a.stages)) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            if (!ok) {  // let every copy already in flight land before the CTA exits
                volatile int never = 0;
                for (int i = 0; i < a.stages; ++i)
                    if (issued_mask & (1u << i))
                        ptx::mbar_wait_bounded(&s.full[i], (parity_mask >> i) & 1u, &never, kDrainLimitNs);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_tf32(kMTile, static_cast<uint32_t>(a.npad));
            uint32_t stage = 0, phase = 0, acc = 0, acc_phase = 0;
            bool ok = true;
            for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
                for (int mt = 0; ok && mt < a.m_tiles; ++mt) {
                    if (!ptx::mbar_wait_bounded(&s.acc_empty[acc], acc_phase ^ 1u, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint32_t d = tmem_base + acc * a.acc_stride;
                    for (int kc = 0; kc < a.k_chunks; ++kc) {
                        if (!ptx::mbar_wait_bounded(&s.split[stage], phase, s.abort_flag, kWaitLimitNs)) {
                            raise_abort(s, a);
                            ok = false;
                            break;
                        }
                        ptx::tc_fence_after();
                        const uint32_t sb = ptx::smem_u32(s.base + stage * s.stage_bytes);
                        const uint32_t ax = sb, axl = sb + kXTileBytes;
                        const uint32_t bw = sb + 2 * kXTileBytes, bwl = bw + s.w_bytes;
#pragma unroll
                        for (int k = 0; k < kKChunk / 8; ++k) {
                            const uint32_t off = static_cast<uint32_t>(k) * 32u;  // 8 TF32 = 32 bytes of K
                            const uint64_t a_hi = ptx::smem_desc_sw128(ax + off);
                            const uint64_t a_lo = ptx::smem_desc_sw128(axl + off);
                            const uint64_t b_hi = ptx::smem_desc_sw128(bw + off);
                            const uint64_t b_lo = ptx::smem_desc_sw128(bwl + off);
                            ptx::mma_tf32(d, a_hi, b_hi, idesc, (kc | k) != 0 ? 1u : 0u);
                            ptx::mma_tf32(d, a_hi, b_lo, idesc, 1u);
                            ptx::mma_tf32(d, a_lo, b_hi, idesc, 1u);
                        }
                        ptx::mma_commit(&s.empty[stage]);
                        if (++stage == static_cast<uint32_t>(a.stages)) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    ptx::mma_commit(&s.acc_full[acc]);
                    acc ^= 1u;
                    if (acc == 0) acc_phase ^= 1u;
                }
            }
            // Wait until every MMA issued by this thread has finished reading
            // shared memory and writing TMEM.
            ptx::mma_commit(s.drain);
            volatile int never = 0;
            ptx::mbar_wait_bounded(s.drain, 0u, &never, ok ? kWaitLimitNs : kDrainLimitNs);
        }
    } else if (warp < 6) {
        // ------------------------------------------------------------ hi/lo split
        const int tt = threadIdx.x - 64;
        uint32_t stage = 0, phase = 0;
        bool ok = true;
        for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
            for (int mt = 0; ok && mt < a.m_tiles; ++mt) {
                for (int kc = 0; kc < a.k_chunks; ++kc) {
                    if (!ptx::mbar_wait_bounded(&s.full[stage], phase, s.abort_flag, kWaitLimitNs)) {
                        raise_abort(s, a);
                        ok = false;
                        break;
                    }
                    uint8_t* st = s.base + stage * s.stage_bytes;
                    float4* xh = reinterpret_cast<float4*>(st);
                    float4* xl = reinterpret_cast<float4*>(st + kXTileBytes);
                    for (uint32_t i = tt; i < kXTileBytes / 16u; i += 128u) {
                        const float4 v = xh[i];
                        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
                        xh[i] = h;
                        xl[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                    }
                    float4* wh = reinterpret_cast<float4*>(st + 2 * kXTileBytes);
                    float4* wl = reinterpret_cast<float4*>(st + 2 * kXTileBytes + s.w_bytes);
                    for (uint32_t i = tt; i < s.w_bytes / 16u; i += 128u) {
                        const float4 v = wh[i];
                        const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
                        wh[i] = h;
                        wl[i] = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                    }
                    ptx::fence_proxy_async_smem();
                    ptx::mbar_arrive(&s.split[stage]);
                    if (++stage == static_cast<uint32_t>(a.stages)) { stage = 0; phase ^= 1u; }
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int et = threadIdx.x - 192;
        const int q = warp & 3;  // the TMEM lane quarter this warp may access
        const int row = q * 32 + lane;
        const float* b1 = s.prm;
        const float* W2 = s.prm + a.h;
        const float* b2 = s.prm + a.h + a.d_out * a.h;
        uint32_t acc = 0, acc_phase = 0;
        float total = 0.0f;
        int32_t n_ok = 0;
        bool ok = true;
        for (int p = blockIdx.x; ok && p < a.pop; p += gridDim.x) {
            for (int mt = 0; mt < a.m_tiles; ++mt) {
                if (mt == 0) {
                    const float* src = a.popv + static_cast<int64_t>(p) * a.c_pad + static_cast<int64_t>(a.h) * a.k;
                    for (uint32_t i = et; i < a.params_floats; i += 128u) s.prm[i] = src[i];
                }
                if (et == 0) {
                    const bool got = ptx::mbar_wait_bounded(&s.acc_full[acc], acc_phase, s.abort_flag, kWaitLimitNs);
                    if (!got) raise_abort(s, a);
                    *s.ep_go = got ? 1 : 0;
                }
                ptx::named_barrier_sync(1, 128);  // A: accumulator ready (or abort), params loaded
                if (!*s.ep_go) { ok = false; break; }
                ptx::tc_fence_after();

                float logit[kMaxOutTc];
#pragma unroll
                for (int o = 0; o < kMaxOutTc; ++o) logit[o] = 0.0f;
                const uint32_t tbase = tmem_base + acc * a.acc_stride + (static_cast<uint32_t>(q * 32) << 16);
                for (int c = 0; c < a.npad; c += 16) {
                    float v[16];
                    ptx::tmem_ld16(tbase + static_cast<uint32_t>(c), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = c + j;
                        if (col < a.h) {
                            const float hv = fmaxf(v[j] + b1[col], 0.0f);
#pragma unroll
                            for (int o = 0; o < kMaxOutTc; ++o)
                                if (o < a.d_out) logit[o] = fmaf(W2[o * a.h + col], hv, logit[o]);
                        }
                    }
                }
                ptx::tc_fence_before();
                ptx::mbar_arrive(&s.acc_empty[acc]);
                acc ^= 1u;
                if (acc == 0) acc_phase ^= 1u;

                const int sample = mt * kMTile + row;
                float loss = 0.0f;
                int32_t good = 0;
                if (sample < a.batch) {
                    float zmax = logit[0] + b2[0];
                    int arg = 0;
#pragma unroll
                    for (int o = 1; o < kMaxOutTc; ++o) {
                        if (o < a.d_out) {
                            const float z = logit[o] + b2[o];
                            if (z > zmax) { zmax = z; arg = o; }
                        }
                    }
                    float se = 0.0f;
#pragma unroll
                    for (int o = 0; o < kMaxOutTc; ++o)
                        if (o < a.d_out) se += expf(logit[o] + b2[o] - zmax);
                    const int32_t lbl = a.y[sample];
                    if (lbl >= 0 && lbl < a.d_out) {
                        float zl = 0.0f;
#pragma unroll
                        for (int o = 0; o < kMaxOutTc; ++o)
                            if (o == lbl) zl = logit[o] + b2[o];
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
                ptx::named_barrier_sync(1, 128);  // B: quarter sums written
                if (et == 0) {
                    total += ((s.red_loss[0] + s.red_loss[1]) + s.red_loss[2]) + s.red_loss[3];
                    n_ok += s.red_ok[0] + s.red_ok[1] + s.red_ok[2] + s.red_ok[3];
                    if (mt == a.m_tiles - 1) {
                        const float f = -(total / static_cast<float>(a.batch));
                        a.f_raw[p] = f;
                        if (a.f_adj) a.f_adj[p] = a.f_inh ? (1.0f - a.alpha) * a.f_inh[p] + a.alpha * f : f;
                        if (a.correct) a.correct[p] = n_ok;
                        total = 0.0f;
                        n_ok = 0;
                    }
                }
            }
        }
    }

    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem_base, a.tmem_cols);
    }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

uint32_t next_pow2(uint32_t v)
{
    uint32_t r = 32;
    while (r < v) r <<= 1;
    return r;
}

}  // namespace

bool eval_tc_supported(const NetLayout& net, int32_t batch, const float* pop_dev, const float* x)
{
    if (net.n_layers != 2) return false;
    const int32_t k = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    if (k % 4 != 0 || h % 16 != 0 || h > 256 || d_out > kMaxOutTc || batch < 1) return false;
    if ((reinterpret_cast<uintptr_t>(pop_dev) | reinterpret_cast<uintptr_t>(x)) & 15u) return false;
    return encode_fn() != nullptr;
}

cudaError_t launch_eval_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const float* x,
                           const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                           float* f_adj, int32_t* correct, unsigned int* status, cudaStream_t stream)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int32_t k = net.dims[0], h = net.dims[1], d_out = net.dims[2];
    const int32_t npad = h;  // h % 16 == 0 on this path

    CUtensorMap tx, tw;
    {
        const cuuint64_t dims[2] = { static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(batch) };
        const cuuint64_t strides[1] = { static_cast<cuuint64_t>(k) * 4u };
        const cuuint32_t box[2] = { static_cast<cuuint32_t>(kKChunk), static_cast<cuuint32_t>(kMTile) };
        const cuuint32_t es[2] = { 1, 1 };
        if (enc(&tx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        const cuuint64_t dims[3] = { static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(h),
                                     static_cast<cuuint64_t>(pop) };
        const cuuint64_t strides[2] = { static_cast<cuuint64_t>(k) * 4u, static_cast<cuuint64_t>(net.c_pad) * 4u };
        const cuuint32_t box[3] = { static_cast<cuuint32_t>(kKChunk), static_cast<cuuint32_t>(npad), 1 };
        const cuuint32_t es[3] = { 1, 1, 1 };
        if (enc(&tw, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(pop_dev), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }

    EvalTcArgs a{};
    a.pop = pop;
    a.h = h;
    a.npad = npad;
    a.d_out = d_out;
    a.batch = batch;
    a.k = k;
    a.k_chunks = (k + kKChunk - 1) / kKChunk;
    a.m_tiles = (batch + kMTile - 1) / kMTile;
    a.c_pad = net.c_pad;
    a.alpha = alpha;
    a.tmem_cols = next_pow2(2u * static_cast<uint32_t>(npad));
    a.acc_stride = a.tmem_cols / 2u;
    a.params_floats = static_cast<uint32_t>(h + d_out * h + d_out);
    a.params_bytes = (a.params_floats * 4u + 15u) & ~15u;
    a.popv = pop_dev;
    a.y = y;
    a.f_inh = f_inh;
    a.f_raw = f_raw;
    a.f_adj = f_adj;
    a.correct = correct;
    a.status = status;

    const uint32_t stage_bytes = 2u * kXTileBytes + 2u * static_cast<uint32_t>(npad) * 128u;
    const uint32_t fixed = 1024u + a.params_bytes + 8u * (3u * 8u + 5u) + 64u;
    const uint32_t budget = 227u * 1024u;
    int stages = static_cast<int>((budget - fixed) / stage_bytes);
    if (stages > 4) stages = 4;
    if (stages < 2) return cudaErrorInvalidValue;
    a.stages = stages;
    const size_t smem = 1024u + stages * stage_bytes + a.params_bytes + 8u * (3u * stages + 5u) + 64u;

    int dev = 0, sms = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(eval_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int grid = pop < sms ? pop : sms;
    eval_tc_kernel<<<grid, kTcThreads, smem, stream>>>(tx, tw, a);
    return cudaGetLastError();
}

}  // namespace leea
