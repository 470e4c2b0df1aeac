// philox.cuh -- device-side counter-based random numbers for the LEEA kernels.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds, each two 32x32->64-bit multiplies whose
// high halves are xored with the other counter words and the round key, and a
// Weyl bump of the key.  Stream layout: key = (seed lo, seed hi), counter =
// (n >> 2, entity, generation, tag); draw n is word n & 3.
#pragma once
#include <cstdint>

namespace leea {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * ctr.x;
        const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * ctr.z;
        ctr = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ ctr.y ^ k0,
                         static_cast<uint32_t>(p1),
                         static_cast<uint32_t>(p0 >> 32) ^ ctr.w ^ k1,
                         static_cast<uint32_t>(p0));
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return ctr;
}

// Block `blk` (= n >> 2) of stream (tag, gen, ent).
__device__ __forceinline__ uint4 stream_block(uint64_t seed, uint32_t tag, uint32_t gen,
                                              uint32_t ent, uint32_t blk)
{
    return philox4x32_10(make_uint4(blk, ent, gen, tag), static_cast<uint32_t>(seed),
                         static_cast<uint32_t>(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(const uint4& w, uint32_t lane)
{
    return lane == 0 ? w.x : lane == 1 ? w.y : lane == 2 ? w.z : w.w;
}

// Open-interval uniform (2k+1) / 2^24 from the top 23 bits, exact in FP32.
__device__ __forceinline__ float u01(uint32_t u)
{
    return static_cast<float>(((u >> 9) << 1) | 1u) * 5.9604644775390625e-08f;
}

// Two standard normals from one pair of words (Box-Muller): radius from the
// first word, angle from the second; cosine for the even gene, sine for the odd.
__device__ __forceinline__ float2 box_muller(uint32_t ua, uint32_t ub)
{
    const float r = sqrtf(-2.0f * logf(u01(ua)));
    float s, c;
    sincospif(2.0f * u01(ub), &s, &c);
    return make_float2(r * c, r * s);
}

// Uniform index in [0, m): floor(u m / 2^32).
__device__ __forceinline__ uint32_t index_of(uint32_t u, uint32_t m)
{
    return static_cast<uint32_t>((static_cast<uint64_t>(u) * m) >> 32);
}

// A draw hits with probability q iff u < thr, thr = floor(q 2^32) (2^32 when q >= 1).
__device__ __forceinline__ bool hits(uint32_t u, uint64_t thr)
{
    return static_cast<uint64_t>(u) < thr;
}

}  // namespace leea

namespace leea {

// The ten round keys of Philox4x32-10 for one seed, computed once per thread
// so that the rounds themselves are two wide multiplies and two xors.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys k;
    uint32_t a = static_cast<uint32_t>(seed), b = static_cast<uint32_t>(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = a;
        k.k1[r] = b;
        a += kPhiloxW0;
        b += kPhiloxW1;
    }
    return k;
}

__device__ __forceinline__ uint4 philox_keyed(uint4 ctr, const PhiloxKeys& k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = static_cast<uint64_t>(kPhiloxM0) * ctr.x;
        const uint64_t p1 = static_cast<uint64_t>(kPhiloxM1) * ctr.z;
        ctr = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ ctr.y ^ k.k0[round], static_cast<uint32_t>(p1),
                         static_cast<uint32_t>(p0 >> 32) ^ ctr.w ^ k.k1[round], static_cast<uint32_t>(p0));
    }
    return ctr;
}

}  // namespace leea
