// select_ops.cuh -- the selection of one child (Algorithm 1; Section 3.1:
// elites, truncation selection from the top rho*lambda, fitness inheritance
// values; the tournament alternative), shared by the selection kernels and
// the single-launch generation of small populations so that both pick the
// same parents from the same streams.
#pragma once
#include <cstdint>

#include "leea_internal.h"
#include "philox.cuh"

namespace leea {

constexpr uint32_t kTagSel = 2;
constexpr uint32_t kTagSigma = 7;
constexpr int32_t kKindElite = 0, kKindCross = 1, kKindMut = 2;

// A 64-bit key whose ascending order is: fitness descending (NaN as -inf,
// -0 as +0), then index ascending.  Comparing keys is exact, so the order is
// the same total order any correct sort of the same FP32 vector produces.
__device__ __forceinline__ uint64_t rank_key(float f, int32_t idx)
{
    uint32_t b = __float_as_uint(f);
    if (f != f) b = 0xFF800000u;       // NaN -> -inf
    if (b == 0x80000000u) b = 0u;      // -0 -> +0
    const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // grows with f
    return (static_cast<uint64_t>(~asc) << 32) | static_cast<uint32_t>(idx);
}

// Draw n of child j's SEL stream, caching the current Philox block.
struct SelStream {
    uint64_t seed;
    uint32_t gen, ent, blk;
    uint4 w;
    __device__ SelStream(uint64_t s, uint32_t g, uint32_t e) : seed(s), gen(g), ent(e), blk(0xFFFFFFFFu) {}
    __device__ uint32_t draw(uint32_t n)
    {
        if ((n >> 2) != blk) {
            blk = n >> 2;
            w = stream_block(seed, kTagSel, gen, ent, blk);
        }
        return word_of(w, n & 3u);
    }
};

__device__ __forceinline__ int32_t pick_parent(const SelectArgs& a, const float* f_adj,
                                               const int32_t* order, SelStream& st, uint32_t first)
{
    if (a.sel_op == 0)
        return order[index_of(st.draw(first), static_cast<uint32_t>(a.pool))];
    int32_t best = -1;
    uint64_t best_key = 0;
    for (int32_t t = 0; t < a.tour_k; ++t) {
        const int32_t cand = static_cast<int32_t>(index_of(st.draw(first + t), static_cast<uint32_t>(a.pop)));
        const uint64_t k = rank_key(f_adj[cand], cand);
        if (best < 0 || k < best_key) { best = cand; best_key = k; }
    }
    return best;
}

// Kind, parents, inherited fitness and mutation strength of child j
// (Algorithm 1; Section 3.1).
struct ChildSelection {
    int32_t kind, p1, p2;
    float f_inh, sigma;
};

// st: child j's SEL stream (its first block may already be drawn).
__device__ __forceinline__ ChildSelection select_child_of(const SelectArgs& a, const float* f_adj,
                                                          const int32_t* order, int32_t j, SelStream st)
{
    ChildSelection c;
    if (j < a.n_elite) {
        c.kind = kKindElite;
        c.p1 = c.p2 = order[j];
        c.f_inh = f_adj[c.p1];
    } else if (j < a.n_elite + a.n_cross) {
        c.kind = kKindCross;
        const uint32_t draws = a.sel_op == 0 ? 1u : static_cast<uint32_t>(a.tour_k);
        c.p1 = pick_parent(a, f_adj, order, st, 0u);
        c.p2 = pick_parent(a, f_adj, order, st, draws);
        c.f_inh = 0.5f * (f_adj[c.p1] + f_adj[c.p2]);
    } else {
        c.kind = kKindMut;
        c.p1 = c.p2 = pick_parent(a, f_adj, order, st, 0u);
        c.f_inh = f_adj[c.p1];
    }
    // Mutation strength of the child (Section 3.2): constant or scheduled, or
    // under self-adaptation its sigma gene -- the elite's own, the mean of the
    // crossover parents', or the mutation parent's times exp(tau z), z from
    // draw 0 of the child's SIGMA stream.
    c.sigma = a.sigma;
    if (a.sigma_out) {
        c.sigma = a.sigma_in[c.p1];
        if (c.kind == kKindCross) {
            c.sigma = 0.5f * (c.sigma + a.sigma_in[c.p2]);
        } else if (c.kind == kKindMut) {
            const uint4 w = stream_block(a.seed, kTagSigma, a.gen, static_cast<uint32_t>(j), 0u);
            c.sigma *= expf(a.tau * box_muller(w.x, w.y).x);
        }
    }
    return c;
}

__device__ __forceinline__ ChildSelection select_child_of(const SelectArgs& a, const float* f_adj,
                                                          const int32_t* order, int32_t j)
{
    return select_child_of(a, f_adj, order, j, SelStream(a.seed, a.gen, static_cast<uint32_t>(j)));
}

// Writes child j's selection (and, in the precision form, its scale bounds).
__device__ __forceinline__ void store_child_selection(const SelectArgs& a, const ChildSelection& c, int32_t j,
                                                      int32_t* par1, int32_t* par2, int32_t* kind, float* f_inh)
{
    kind[j] = c.kind;
    par1[j] = c.p1;
    par2[j] = c.p2;
    f_inh[j] = c.f_inh;
    if (a.sigma_out) a.sigma_out[j] = c.sigma;
    if (a.precision > 0) {
        a.amax_out[j] = 0.0f;
        if (a.precision == 2) {
            // Upper bound on the child's max |W1|: a crossover gene (either
            // parent's, or their mean) is bounded by the larger parent bound; a
            // mutation adds at most sigma * kNormalBound.
            float bound = a.amax_in[c.p1];
            if (c.kind == kKindCross) bound = fmaxf(bound, a.amax_in[c.p2]);
            else if (c.kind == kKindMut) bound = fmaf(c.sigma, kNormalBound, bound);
            a.scale_exp_out[j] = fp8_scale_exp(bound);
        }
    }
}

__device__ __forceinline__ void select_child(const SelectArgs& a, const float* f_adj, const int32_t* order, int32_t j,
                                             int32_t* par1, int32_t* par2, int32_t* kind, float* f_inh)
{
    store_child_selection(a, select_child_of(a, f_adj, order, j), j, par1, par2, kind, f_inh);
}

}  // namespace leea
