// breed_ops.cuh -- per-gene operators of crossover and mutation (Section 3.2)
// shared by the breeding kernel and the fused breed + evaluate kernel, so that
// both make bit-identical children from the same streams.
//
// Genes are handled in units of 8 consecutive genes 8u .. 8u+7: one Philox
// block of the XO or MUTMASK stream holds their 16-bit mask draws (draw16 i
// is half i & 1 of word (i >> 1) & 3 of block i >> 3), and NORMAL blocks 2u and
// 2u + 1 hold their Box-Muller pairs (block i >> 2, words (0,1) for genes
// i & 3 in {0, 1}, words (2,3) for {2, 3}).
#pragma once
#include <cstdint>

#include "philox.cuh"

namespace leea {

constexpr uint32_t kTagXo = 3, kTagMutMask = 4, kTagNormal = 5;

// Bit k of the result: the 16-bit draw k (k = 0..7) of block r is below thr.
__device__ __forceinline__ uint32_t mask8(const uint4& r, uint32_t thr)
{
    const uint32_t w[4] = { r.x, r.y, r.z, r.w };
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t u = (k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xFFFFu);
        m |= (u < thr ? 1u : 0u) << k;
    }
    return m;
}

__device__ __forceinline__ float4 select4(uint32_t m, float4 a, float4 b)
{
    return make_float4((m & 1u) ? b.x : a.x, (m & 2u) ? b.y : a.y, (m & 4u) ? b.z : a.z, (m & 8u) ? b.w : a.w);
}

__device__ __forceinline__ float4 mean4(float4 a, float4 b)
{
    return make_float4(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z), 0.5f * (a.w + b.w));
}

// Zero the padding genes (>= c) among genes i0 .. i0+3.
__device__ __forceinline__ float4 clear_padding(float4 v, int64_t i0, int64_t c)
{
    if (i0 + 0 >= c) v.x = 0.0f;
    if (i0 + 1 >= c) v.y = 0.0f;
    if (i0 + 2 >= c) v.z = 0.0f;
    if (i0 + 3 >= c) v.w = 0.0f;
    return v;
}

// Normals of one lane's unit (8 genes) whose mask bits are `hit`.  Slot
// s = 0..3 names the Box-Muller pair of genes 8u + 2s, 8u + 2s + 1, i.e. pair
// s & 1 of NORMAL block 2u + (s >> 1).  The warp lists the slots that hold a
// masked gene, slot by slot (one ballot each), in its shared-memory job list
// (kJobs = 4 x 32 entries); consecutive lanes compute the listed normals and
// every lane reads its own back into z (zero for slots without a masked
// gene).  unit_of(o) is the unit owned by lane o.  Every lane of the warp
// calls it (hit = 0 for a lane without a unit).
template <typename UnitOf>
__device__ __forceinline__ void normals8(uint32_t gen, const PhiloxKeys& key, uint32_t ent, uint32_t hit,
                                         float2 (&z)[4], int lane, float2* job_z, uint8_t* job_code, UnitOf unit_of)
{
    constexpr int kSlots = 4;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t idx[kSlots], total = 0;
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
        const bool need = ((hit >> (2 * sl)) & 3u) != 0u;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, need);
        idx[sl] = total + __popc(b & lt);
        if (need) job_code[idx[sl]] = static_cast<uint8_t>((lane << 2) | sl);
        total += __popc(b);
    }
    __syncwarp();
    for (uint32_t job = static_cast<uint32_t>(lane); job < total; job += 32) {
        const uint32_t code = job_code[job];
        const uint32_t o = code >> 2, slot = code & 3u;
        const uint32_t uo = unit_of(o);
        const uint4 n = philox_keyed(make_uint4(2u * uo + (slot >> 1), ent, gen, kTagNormal), key);
        job_z[job] = (slot & 1u) ? box_muller(n.z, n.w) : box_muller(n.x, n.y);
    }
    __syncwarp();
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl)
        z[sl] = ((hit >> (2 * sl)) & 3u) ? job_z[idx[sl]] : make_float2(0.f, 0.f);
    __syncwarp();  // the list is reused by the next unit
}

// The mutation step of the masked genes: v += sigma z.
__device__ __forceinline__ void apply_mutation8(float sigma, uint32_t hit, const float2 (&z)[4], float4 (&v)[2])
{
    if (hit & 0x01u) v[0].x = fmaf(sigma, z[0].x, v[0].x);
    if (hit & 0x02u) v[0].y = fmaf(sigma, z[0].y, v[0].y);
    if (hit & 0x04u) v[0].z = fmaf(sigma, z[1].x, v[0].z);
    if (hit & 0x08u) v[0].w = fmaf(sigma, z[1].y, v[0].w);
    if (hit & 0x10u) v[1].x = fmaf(sigma, z[2].x, v[1].x);
    if (hit & 0x20u) v[1].y = fmaf(sigma, z[2].y, v[1].y);
    if (hit & 0x40u) v[1].z = fmaf(sigma, z[3].x, v[1].z);
    if (hit & 0x80u) v[1].w = fmaf(sigma, z[3].y, v[1].w);
}

// Mutation of one lane's unit (8 genes in v) whose mask bits are `hit`: the
// normals of normals8 (the same job list, the same draws), the step applied
// before the warp lets the list go.
template <typename UnitOf>
__device__ __forceinline__ void mutate8(float sigma, uint32_t gen, const PhiloxKeys& key, uint32_t ent, uint32_t hit,
                                        float4 (&v)[2], int lane, float2* job_z, uint8_t* job_code, UnitOf unit_of)
{
    constexpr int kSlots = 4;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t idx[kSlots], total = 0;
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
        const bool need = ((hit >> (2 * sl)) & 3u) != 0u;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, need);
        idx[sl] = total + __popc(b & lt);
        if (need) job_code[idx[sl]] = static_cast<uint8_t>((lane << 2) | sl);
        total += __popc(b);
    }
    __syncwarp();
    for (uint32_t job = static_cast<uint32_t>(lane); job < total; job += 32) {
        const uint32_t code = job_code[job];
        const uint32_t o = code >> 2, slot = code & 3u;
        const uint32_t uo = unit_of(o);
        const uint4 n = philox_keyed(make_uint4(2u * uo + (slot >> 1), ent, gen, kTagNormal), key);
        job_z[job] = (slot & 1u) ? box_muller(n.z, n.w) : box_muller(n.x, n.y);
    }
    __syncwarp();
    float2 z[kSlots];
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl)
        z[sl] = ((hit >> (2 * sl)) & 3u) ? job_z[idx[sl]] : make_float2(0.f, 0.f);
    apply_mutation8(sigma, hit, z, v);
    __syncwarp();  // the list is reused by the next unit
}

// The same mutation of one unit by a single thread (no job list): each masked
// pair's normals are generated where they are needed.  Bit-identical to
// mutate8 for the same unit.
__device__ __forceinline__ void mutate8_direct(float sigma, uint32_t gen, const PhiloxKeys& key, uint32_t ent,
                                               uint32_t u, uint32_t hit, float4 (&v)[2])
{
    float2 z[4];
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
        z[sl] = make_float2(0.f, 0.f);
        if ((hit >> (2 * sl)) & 3u) {
            const uint4 n = philox_keyed(make_uint4(2u * u + (sl >> 1), ent, gen, kTagNormal), key);
            z[sl] = (sl & 1) ? box_muller(n.z, n.w) : box_muller(n.x, n.y);
        }
    }
    apply_mutation8(sigma, hit, z, v);
}

}  // namespace leea
