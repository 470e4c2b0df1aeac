// leea_breed.cu -- crossover and mutation (Section 3.2) fused into one
// streaming pass over every child's genes.
//
// The pass is HBM-bound: per gene it reads one (mutation, elite) or two
// (crossover) parent floats and writes one child float.  A thread owns blocks
// of four consecutive genes, which is exactly one Philox block of each
// per-gene stream, so one generator call serves one 128-bit load and store.
// Normals are only generated for blocks in which some gene is masked for
// mutation.
#include "leea_internal.h"
#include "philox.cuh"

namespace leea {

constexpr uint32_t kTagXo = 3, kTagMutMask = 4, kTagNormal = 5;
constexpr int kBreedThreads = 256;
constexpr int kBreedUnroll = 4;  // float4 per thread per trip: 64 B in flight per parent

__device__ __forceinline__ float4 ldg_stream(const float4* p)
{
    return __ldg(p);
}

__global__ void __launch_bounds__(kBreedThreads) breed_kernel(BreedArgs a, int32_t chunks,
                                                              const float* __restrict__ parents,
                                                              const int32_t* __restrict__ par1,
                                                              const int32_t* __restrict__ par2,
                                                              const int32_t* __restrict__ kind,
                                                              float* __restrict__ children)
{
    const int32_t j = blockIdx.x / chunks;
    const int32_t chunk = blockIdx.x - j * chunks;
    const int32_t kd = kind[j];
    const int32_t i1 = par1[j], i2 = par2[j];
    float4* O = reinterpret_cast<float4*>(children + static_cast<int64_t>(j) * a.c_pad);
    const int64_t nq = a.c_pad >> 2;
    const int64_t q0 = static_cast<int64_t>(chunk) * (kBreedThreads * kBreedUnroll) + threadIdx.x;
    if (i1 < 0 || i1 >= a.pop || i2 < 0 || i2 >= a.pop) {
        // A parent index outside the population: the child becomes NaN (its
        // fitness then ranks last) instead of reading out of bounds.
        const float nan = __int_as_float(0x7FC00000);
        for (int u = 0; u < kBreedUnroll; ++u)
            if (q0 + u * kBreedThreads < nq) O[q0 + u * kBreedThreads] = make_float4(nan, nan, nan, nan);
        return;
    }
    const float4* A = reinterpret_cast<const float4*>(parents + static_cast<int64_t>(i1) * a.c_pad);
    const float4* B = reinterpret_cast<const float4*>(parents + static_cast<int64_t>(i2) * a.c_pad);

    float4 va[kBreedUnroll], vb[kBreedUnroll];
#pragma unroll
    for (int u = 0; u < kBreedUnroll; ++u) {
        const int64_t q = q0 + u * kBreedThreads;
        if (q < nq) {
            va[u] = ldg_stream(A + q);
            if (kd == 1) vb[u] = ldg_stream(B + q);
        }
    }
#pragma unroll
    for (int u = 0; u < kBreedUnroll; ++u) {
        const int64_t q = q0 + u * kBreedThreads;
        if (q >= nq) continue;
        const uint32_t blk = static_cast<uint32_t>(q);
        float v[4] = { va[u].x, va[u].y, va[u].z, va[u].w };
        if (kd == 1) {
            const float w2[4] = { vb[u].x, vb[u].y, vb[u].z, vb[u].w };
            if (a.xo_op == 0) {
                const uint4 r = stream_block(a.seed, kTagXo, a.gen, static_cast<uint32_t>(j), blk);
                const uint32_t rw[4] = { r.x, r.y, r.z, r.w };
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = hits(rw[k], a.thr_xo) ? w2[k] : v[k];
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = 0.5f * (v[k] + w2[k]);
            }
        } else if (kd == 2) {
            const uint4 r = stream_block(a.seed, kTagMutMask, a.gen, static_cast<uint32_t>(j), blk);
            const bool m0 = hits(r.x, a.thr_mut), m1 = hits(r.y, a.thr_mut);
            const bool m2 = hits(r.z, a.thr_mut), m3 = hits(r.w, a.thr_mut);
            if (m0 | m1 | m2 | m3) {
                const uint4 n = stream_block(a.seed, kTagNormal, a.gen, static_cast<uint32_t>(j), blk);
                if (m0 | m1) {
                    const float2 z = box_muller(n.x, n.y);
                    if (m0) v[0] = fmaf(a.sigma, z.x, v[0]);
                    if (m1) v[1] = fmaf(a.sigma, z.y, v[1]);
                }
                if (m2 | m3) {
                    const float2 z = box_muller(n.z, n.w);
                    if (m2) v[2] = fmaf(a.sigma, z.x, v[2]);
                    if (m3) v[3] = fmaf(a.sigma, z.y, v[3]);
                }
            }
        }
        // Genes past c are padding and stay zero whatever the operator.
        const int64_t i0 = 4 * q;
        if (i0 + 3 >= a.c) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i0 + k >= a.c) v[k] = 0.0f;
        }
        O[q] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

cudaError_t launch_breed(const BreedArgs& a, const float* parents, const int32_t* par1,
                         const int32_t* par2, const int32_t* kind, float* children,
                         cudaStream_t stream)
{
    const int64_t nq = a.c_pad >> 2;
    const int64_t per_cta = kBreedThreads * kBreedUnroll;
    const int32_t chunks = static_cast<int32_t>((nq + per_cta - 1) / per_cta);
    const int64_t grid = static_cast<int64_t>(chunks) * a.pop;
    if (grid > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
    breed_kernel<<<static_cast<unsigned>(grid), kBreedThreads, 0, stream>>>(a, chunks, parents, par1, par2,
                                                                          kind, children);
    return cudaGetLastError();
}

}  // namespace leea
