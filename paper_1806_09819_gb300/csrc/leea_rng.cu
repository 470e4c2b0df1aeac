// leea_rng.cu -- population initialisation (Algorithm 1's initial population; Section
// 4.1) and the diagnostic stream dumps.
#include "leea_internal.h"
#include "philox.cuh"
#include "tc_ptx.cuh"

namespace leea {

constexpr uint32_t kTagInit = 1;

// One thread per block of 4 genes: one Philox call yields the four uniforms
// (Glorot) or, through two Box-Muller pairs, the four normals (N(0,1/fan_in)).
__global__ void __launch_bounds__(256) init_kernel(NetLayout net, int32_t init, uint64_t seed,
                                                   uint32_t p_base, float* __restrict__ pop)
{
    const uint32_t p = p_base + blockIdx.y;
    const int64_t nq = net.c_pad >> 2;
    float4* out = reinterpret_cast<float4*>(pop + static_cast<int64_t>(p) * net.c_pad);
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < nq;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint4 w = stream_block(seed, kTagInit, 0u, p, static_cast<uint32_t>(q));
        float z[4];
        if (init == 0) {
            const float2 za = box_muller(w.x, w.y);
            const float2 zb = box_muller(w.z, w.w);
            z[0] = za.x; z[1] = za.y; z[2] = zb.x; z[3] = zb.y;
        } else {
            z[0] = fmaf(2.0f, u01(w.x), -1.0f);
            z[1] = fmaf(2.0f, u01(w.y), -1.0f);
            z[2] = fmaf(2.0f, u01(w.z), -1.0f);
            z[3] = fmaf(2.0f, u01(w.w), -1.0f);
        }
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = 4 * q + k;
            v[k] = 0.0f;  // biases and padding
            for (int l = 0; l < net.n_layers; ++l) {
                if (i >= net.w_off[l] && i < net.b_off[l]) {
                    v[k] = z[k] * net.init_scale[l];
                    break;
                }
            }
        }
        out[q] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

cudaError_t launch_init(const NetLayout& net, int32_t pop, int32_t init, uint64_t seed,
                        float* pop_dev, cudaStream_t stream)
{
    const int64_t nq = net.c_pad >> 2;
    const unsigned gx = static_cast<unsigned>((nq + 255) / 256 < 1024 ? (nq + 255) / 256 : 1024);
    for (int32_t p0 = 0; p0 < pop; p0 += 65535) {
        const int32_t n = pop - p0 < 65535 ? pop - p0 : 65535;
        init_kernel<<<dim3(gx, n), 256, 0, stream>>>(net, init, seed, static_cast<uint32_t>(p0),
                                                     pop_dev);
    }
    return cudaGetLastError();
}

__global__ void philox_fill_kernel(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                                   uint32_t n0, int64_t count, uint32_t* __restrict__ out)
{
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t n = n0 + static_cast<uint32_t>(t);
        out[t] = word_of(stream_block(seed, tag, gen, ent, n >> 2), n & 3u);
    }
}

__global__ void normal_fill_kernel(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                                   uint32_t n0, int64_t count, float* __restrict__ out)
{
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < count;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t i = n0 + static_cast<uint32_t>(t);
        const uint4 w = stream_block(seed, tag, gen, ent, i >> 2);
        const float2 z = (i & 2u) ? box_muller(w.z, w.w) : box_muller(w.x, w.y);
        out[t] = (i & 1u) ? z.y : z.x;
    }
}

cudaError_t launch_philox_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                               uint32_t n0, int64_t count, uint32_t* out, cudaStream_t stream)
{
    const int64_t blocks = (count + 255) / 256;
    philox_fill_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(
        seed, tag, gen, ent, n0, count, out);
    return cudaGetLastError();
}

cudaError_t launch_normal_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                               uint32_t n0, int64_t count, float* out, cudaStream_t stream)
{
    const int64_t blocks = (count + 255) / 256;
    normal_fill_kernel<<<static_cast<unsigned>(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(
        seed, tag, gen, ent, n0, count, out);
    return cudaGetLastError();
}

// A bounded wait on an mbarrier that nothing completes (phase 0 of a fresh
// barrier with one expected arrival): the same wait the pipelines use, run
// to its limit, then the status bit the host reads.
__global__ void wait_timeout_probe_kernel(uint64_t limit_ns, unsigned int* status)
{
    __shared__ uint64_t bar;
    __shared__ int never;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        never = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !ptx::mbar_wait_bounded(&bar, 0u, &never, limit_ns))
        atomicOr(status, kStatusSelftestTimeout);
}

cudaError_t launch_wait_timeout_probe(uint64_t limit_ns, unsigned int* status, cudaStream_t stream)
{
    wait_timeout_probe_kernel<<<1, 32, 0, stream>>>(limit_ns, status);
    return cudaGetLastError();
}

}  // namespace leea
