// leea_shadow.cu -- precision form: BF16 / FP8-e4m3 shadows of W1 made from a
// whole FP32 master population (after initialisation or when the caller
// replaces the population), in the tiled layout of shadow_offset, padding
// included.  Breeding writes the shadows of its children itself.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "leea_internal.h"

namespace leea {

namespace {

constexpr int kShadowThreads = 256;

// One CTA per individual: exact max |W1| (fixed-order tree reduction), the FP8
// exponent from it, then the shadow.
__global__ void __launch_bounds__(kShadowThreads) make_shadow_kernel(int32_t k, int32_t h, int64_t c_pad,
                                                                     const float* __restrict__ popv,
                                                                     int32_t precision, uint8_t* __restrict__ shadow,
                                                                     int64_t sh_stride, int32_t* __restrict__ scale_exp,
                                                                     float* __restrict__ amax)
{
    __shared__ float red[kShadowThreads / 32];
    __shared__ int32_t sexp_s;
    const int p = blockIdx.x;
    const float* wp = popv + static_cast<int64_t>(p) * c_pad;
    const float4* w = reinterpret_cast<const float4*>(wp);
    const int64_t n8 = static_cast<int64_t>(k) * h / 8;  // units of 8 genes
    float mx = 0.0f;
    for (int64_t u = threadIdx.x; u < n8; u += kShadowThreads) {
        const float4 a = w[2 * u], b = w[2 * u + 1];
        mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                             fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w)))));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int i = 0; i < kShadowThreads / 32; ++i) m = fmaxf(m, red[i]);
        amax[p] = m;
        sexp_s = precision == 2 ? fp8_scale_exp(m) : 0;
        if (precision == 2) scale_exp[p] = sexp_s;
    }
    __syncthreads();
    const int32_t sexp = sexp_s;
    const float inv = ldexpf(1.0f, -sexp);
    const int32_t elem = precision == 1 ? 2 : 1;
    uint4* dst = reinterpret_cast<uint4*>(shadow + static_cast<int64_t>(p) * sh_stride);
    // One 16-byte chunk of the tiled layout per step (coalesced stores); its
    // source is 8 BF16 or 16 FP8 consecutive inputs of one row, or zero padding.
    const int64_t n16 = shadow_stride_bytes(k, h, elem) / 16;
    for (int64_t t = threadIdx.x; t < n16; t += kShadowThreads) {
        const int64_t blk = t / (8 * h);
        const int32_t rem = static_cast<int32_t>(t - blk * 8 * h);
        const int32_t o = rem >> 3, c = (rem & 7) ^ (o & 7);
        const int32_t k0 = static_cast<int32_t>((blk * 128 + c * 16) / elem);
        uint4 out = make_uint4(0u, 0u, 0u, 0u);
        if (k0 < k) {
            const float4* src = reinterpret_cast<const float4*>(wp + static_cast<int64_t>(o) * k + k0);
            if (precision == 1) {
                const float4 a = src[0], b = src[1];
                const __nv_bfloat162 b0 = __floats2bfloat162_rn(a.x, a.y), b1 = __floats2bfloat162_rn(a.z, a.w);
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(b.x, b.y), b3 = __floats2bfloat162_rn(b.z, b.w);
                out.x = *reinterpret_cast<const uint32_t*>(&b0);
                out.y = *reinterpret_cast<const uint32_t*>(&b1);
                out.z = *reinterpret_cast<const uint32_t*>(&b2);
                out.w = *reinterpret_cast<const uint32_t*>(&b3);
            } else {
                uint32_t word[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 a = src[q];
                    const __nv_fp8x2_storage_t lo =
                        __nv_cvt_float2_to_fp8x2(make_float2(a.x * inv, a.y * inv), __NV_SATFINITE, __NV_E4M3);
                    const __nv_fp8x2_storage_t hi =
                        __nv_cvt_float2_to_fp8x2(make_float2(a.z * inv, a.w * inv), __NV_SATFINITE, __NV_E4M3);
                    word[q] = static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
                }
                out = make_uint4(word[0], word[1], word[2], word[3]);
            }
        }
        dst[t] = out;
    }
}

}  // namespace

cudaError_t launch_make_shadow(int32_t pop, int32_t k, int32_t h, int64_t c_pad, const float* pop_dev,
                               int32_t precision, uint8_t* shadow, int64_t sh_stride, int32_t* scale_exp, float* amax,
                               cudaStream_t stream)
{
    make_shadow_kernel<<<pop, kShadowThreads, 0, stream>>>(k, h, c_pad, pop_dev, precision, shadow, sh_stride,
                                                           scale_exp, amax);
    return cudaGetLastError();
}

}  // namespace leea
