// leea_select.cu -- sort by fitness and parent selection (Algorithm 1;
// Section 3.1: elites, truncation selection from the top rho*lambda, fitness
// inheritance values) plus the tournament alternative.
#include "leea_internal.h"
#include "philox.cuh"
#include "select_ops.cuh"
#include "tc_ptx.cuh"

namespace leea {

// Rank by counting: the rank of i is the number of keys below its own.  A
// warp owns one individual: its lanes scan the keys of a shared tile (the
// CTA's 8 warps share it), then the counts are summed over the lanes.  At
// the population sizes of the method (<= a few 10^4) this is a few
// microseconds spread over many SMs and needs no scratch memory.
constexpr int kRankTile = 2048;
constexpr int kRankWarps = 8;

__global__ void __launch_bounds__(32 * kRankWarps) rank_kernel(int32_t pop, const float* __restrict__ f_adj,
                                                              int32_t* __restrict__ order)
{
    __shared__ uint64_t tile[kRankTile];
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();  // f_adj comes from the previous kernel
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t i = blockIdx.x * kRankWarps + warp;
    const uint64_t mine = i < pop ? rank_key(f_adj[i], i) : 0ull;
    int32_t r = 0;
    for (int32_t base = 0; base < pop; base += kRankTile) {
        const int32_t n = pop - base < kRankTile ? pop - base : kRankTile;
        __syncthreads();
        for (int32_t t = threadIdx.x; t < n; t += blockDim.x) tile[t] = rank_key(f_adj[base + t], base + t);
        __syncthreads();
#pragma unroll 4
        for (int32_t t = lane; t < n; t += 32) r += tile[t] < mine ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, off);
    if (lane == 0 && i < pop) order[r] = i;
}

cudaError_t launch_rank(int32_t pop, const float* f_adj, int32_t* order, cudaStream_t stream)
{
    return launch_pdl(rank_kernel, dim3((pop + kRankWarps - 1) / kRankWarps), dim3(32 * kRankWarps), 0, stream, pop,
                      f_adj, order);
}

// Recipe r of the surrogate form: a crossover (r < mult n_cross) or a
// mutation, parents picked as for a child of that kind from the streams of
// entity kRecipeEntity0 + r.
__global__ void __launch_bounds__(256) select_recipes_kernel(SelectArgs a, int32_t mult, const float* __restrict__ f_adj,
                                                             const int32_t* __restrict__ order,
                                                             int32_t* __restrict__ par1, int32_t* __restrict__ par2,
                                                             int32_t* __restrict__ kind, float* __restrict__ f_inh,
                                                             uint32_t* __restrict__ entity)
{
    const int32_t n = mult * (a.pop - a.n_elite);
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t ent = kRecipeEntity0 + static_cast<uint32_t>(r);
    SelStream st(a.seed, a.gen, ent);
    const uint32_t draws = a.sel_op == 0 ? 1u : static_cast<uint32_t>(a.tour_k);
    int32_t p1, p2, k;
    float fi;
    if (r < mult * a.n_cross) {
        k = kKindCross;
        p1 = pick_parent(a, f_adj, order, st, 0u);
        p2 = pick_parent(a, f_adj, order, st, draws);
        fi = 0.5f * (f_adj[p1] + f_adj[p2]);
    } else {
        k = kKindMut;
        p1 = p2 = pick_parent(a, f_adj, order, st, 0u);
        fi = f_adj[p1];
    }
    kind[r] = k;
    par1[r] = p1;
    par2[r] = p2;
    f_inh[r] = fi;
    entity[r] = ent;
}

__global__ void __launch_bounds__(256) select_kernel(SelectArgs a, const float* __restrict__ f_adj,
                                                     const int32_t* __restrict__ order,
                                                     int32_t* __restrict__ par1, int32_t* __restrict__ par2,
                                                     int32_t* __restrict__ kind, float* __restrict__ f_inh)
{
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();  // the ranking comes from the previous kernel
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < a.pop) select_child(a, f_adj, order, j, par1, par2, kind, f_inh);
}

cudaError_t launch_select(const SelectArgs& a, const float* f_adj, const int32_t* order,
                          int32_t* par1, int32_t* par2, int32_t* kind, float* f_inh,
                          cudaStream_t stream)
{
    return launch_pdl(select_kernel, dim3((a.pop + 255) / 256), dim3(256), 0, stream, a, f_adj, order, par1, par2, kind,
                      f_inh);
}

// Rank and select in one CTA for populations up to kFusedMaxPop: a bitonic
// sort of the 64-bit rank keys in shared memory (padding keys sort last),
// then one thread per child runs the selection against the sorted order.
constexpr int kFusedThreads = 1024;
constexpr int kFusedMaxPop = 4096;
constexpr int kSplitMinPop = 512;  // from here on: rank_kernel + select_kernel (measured at P = 1000)

__device__ __forceinline__ void rank_select_body(const SelectArgs& a, const float* __restrict__ f_adj,
                                                 int32_t* __restrict__ order_out, int32_t* __restrict__ par1,
                                                 int32_t* __restrict__ par2, int32_t* __restrict__ kind,
                                                 float* __restrict__ f_inh)
{
    __shared__ uint64_t keys[kFusedMaxPop];
    __shared__ int32_t order[kFusedMaxPop];
    int n = 1;
    while (n < a.pop) n <<= 1;
    for (int i = threadIdx.x; i < n; i += kFusedThreads) keys[i] = i < a.pop ? rank_key(f_adj[i], i) : ~0ull;
    __syncthreads();
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (n >> 1); t += kFusedThreads) {
                // t-th compare-exchange pair of this pass
                const int lo = 2 * stride * (t / stride) + (t % stride);
                const int hi = lo + stride;
                const bool ascending = (lo & size) == 0;
                const uint64_t x = keys[lo], y = keys[hi];
                if ((x > y) == ascending) {
                    keys[lo] = y;
                    keys[hi] = x;
                }
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < a.pop; r += kFusedThreads) {
        const int32_t idx = static_cast<int32_t>(keys[r] & 0xFFFFFFFFu);
        order[r] = idx;
        order_out[r] = idx;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < a.pop; j += kFusedThreads) select_child(a, f_adj, order, j, par1, par2, kind, f_inh);
}

__global__ void __launch_bounds__(kFusedThreads, 1)
rank_select_kernel(SelectArgs a, const float* __restrict__ f_adj, int32_t* __restrict__ order_out,
                   int32_t* __restrict__ par1, int32_t* __restrict__ par2, int32_t* __restrict__ kind,
                   float* __restrict__ f_inh)
{
    rank_select_body(a, f_adj, order_out, par1, par2, kind, f_inh);
}

// Many runs at once: CTA r ranks and selects run r; the generation is read
// from device memory (so that a captured graph can be replayed).
__global__ void __launch_bounds__(kFusedThreads, 1)
rank_select_runs_kernel(const SelectRun* __restrict__ runs, const uint32_t* __restrict__ gen_dev)
{
    const SelectRun& r = runs[blockIdx.x];
    SelectArgs a = r.a;
    a.gen = *gen_dev;
    rank_select_body(a, r.f_adj, r.order, r.par1, r.par2, r.kind, r.f_inh);
}

cudaError_t launch_rank_select(const SelectArgs& a, const float* f_adj, int32_t* order, int32_t* par1, int32_t* par2,
                               int32_t* kind, float* f_inh, cudaStream_t stream)
{
    // The fused single-CTA kernel serves small populations, where one launch
    // beats two; above kSplitMinPop the ranking spread over many SMs wins.
    if (a.pop > kFusedMaxPop || a.pop >= kSplitMinPop) {
        cudaError_t err = launch_rank(a.pop, f_adj, order, stream);
        if (err != cudaSuccess) return err;
        return launch_select(a, f_adj, order, par1, par2, kind, f_inh, stream);
    }
    rank_select_kernel<<<1, kFusedThreads, 0, stream>>>(a, f_adj, order, par1, par2, kind, f_inh);
    return cudaGetLastError();
}

cudaError_t launch_select_recipes(const SelectArgs& a, int32_t mult, const float* f_adj, const int32_t* order,
                                  int32_t* par1, int32_t* par2, int32_t* kind, float* f_inh, uint32_t* entity,
                                  cudaStream_t stream)
{
    const int32_t n = mult * (a.pop - a.n_elite);
    if (n <= 0) return cudaSuccess;
    select_recipes_kernel<<<(n + 255) / 256, 256, 0, stream>>>(a, mult, f_adj, order, par1, par2, kind, f_inh, entity);
    return cudaGetLastError();
}

cudaError_t launch_rank_select_runs(const SelectRun* runs_dev, int32_t n_runs, const uint32_t* gen_dev,
                                    cudaStream_t stream)
{
    rank_select_runs_kernel<<<n_runs, kFusedThreads, 0, stream>>>(runs_dev, gen_dev);
    return cudaGetLastError();
}

}  // namespace leea
