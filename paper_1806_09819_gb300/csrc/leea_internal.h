// leea_internal.h -- launch interface between the C ABI (leea_capi.cu) and the
// kernels.  Host-only declarations; every launcher enqueues on `stream` and
// returns the launch error (cudaSuccess when the launch was accepted).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace leea {

constexpr int kMaxLayers = 15;

// Bits of the device status word (set by kernels, read and cleared by the host).
constexpr unsigned int kStatusEvalTimeout = 1u;   // a bounded mbarrier wait of the tensor-core eval gave up
constexpr unsigned int kStatusBreedTimeout = 2u;  // a bounded mbarrier wait of the breed kernel gave up

// Per-layer offsets of a net, computed on the host (logical gene order of
// Section 3.2: W_l rows out x in, then b_l).
struct NetLayout {
    int32_t n_layers;                  // L = n_dims - 1
    int32_t dims[kMaxLayers + 1];
    int64_t w_off[kMaxLayers];         // first gene of W_l
    int64_t b_off[kMaxLayers];         // first gene of b_l
    float init_scale[kMaxLayers];      // N(0,1/fan_in): 1/sqrt(d_l); Glorot: a
    int64_t c;                         // genes
    int64_t c_pad;                     // device stride, multiple of 32
};

struct SelectArgs {
    int32_t pop, n_elite, n_cross, pool;
    int32_t sel_op, tour_k;
    uint64_t seed;
    uint32_t gen;
};

struct BreedArgs {
    int32_t pop;
    int64_t c, c_pad;
    int32_t xo_op;
    uint32_t thr_xo, thr_mut;  // 16-bit draw thresholds floor(q 2^16), 2^16 when q >= 1
    float sigma;
    uint64_t seed;
    uint32_t gen;
};

cudaError_t launch_init(const NetLayout& net, int32_t pop, int32_t init, uint64_t seed,
                        float* pop_dev, cudaStream_t stream);
cudaError_t launch_rank(int32_t pop, const float* f_adj, int32_t* order, cudaStream_t stream);
cudaError_t launch_select(const SelectArgs& a, const float* f_adj, const int32_t* order,
                          int32_t* par1, int32_t* par2, int32_t* kind, float* f_inh,
                          cudaStream_t stream);
// Ranking and selection in one launch (one CTA, bitonic sort in shared
// memory) when pop <= 4096; otherwise the two kernels above in sequence.
cudaError_t launch_rank_select(const SelectArgs& a, const float* f_adj, int32_t* order, int32_t* par1,
                               int32_t* par2, int32_t* kind, float* f_inh, cudaStream_t stream);
cudaError_t launch_breed(const BreedArgs& a, const float* parents, const int32_t* par1,
                         const int32_t* par2, const int32_t* kind, float* children,
                         unsigned int* status, cudaStream_t stream);
// Evaluation of d_0-h-d_out nets (one hidden layer), SIMT FP32.
cudaError_t launch_eval_simt(const NetLayout& net, int32_t pop, const float* pop_dev,
                             const float* x, const int32_t* y, int32_t batch, float alpha,
                             const float* f_inh, float* f_raw, float* f_adj, int32_t* correct,
                             cudaStream_t stream);
// Evaluation on the tcgen05 tensor cores (3xTF32), d_0-h-d_out with d_0 % 4 == 0,
// h % 16 == 0, h <= 256, d_out <= 16 and 16-byte aligned population and x.
bool eval_tc_supported(const NetLayout& net, int32_t batch, const float* pop_dev, const float* x);
cudaError_t launch_eval_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const float* x,
                           const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                           float* f_adj, int32_t* correct, unsigned int* status, cudaStream_t stream);
// 8-bit inputs x = k / x_div: CUDA-core FP32 evaluation of any shape, and the
// tensor-core evaluation (batch in TMEM, exact BF16 pieces) for batch <= 128,
// d_0 % 4 == 0, h % 16 == 0, h + d_0/2 (rounded) <= 512 TMEM columns, d_out <= 16.
cudaError_t launch_eval_simt_u8(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                                float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                float* f_raw, float* f_adj, int32_t* correct, cudaStream_t stream);
bool eval_u8_tc_supported(const NetLayout& net, int32_t batch, const float* pop_dev);
cudaError_t launch_eval_u8_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                              float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                              float* f_raw, float* f_adj, int32_t* correct, unsigned int* status,
                              cudaStream_t stream);
cudaError_t launch_philox_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                               uint32_t n0, int64_t count, uint32_t* out, cudaStream_t stream);
cudaError_t launch_normal_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                               uint32_t n0, int64_t count, float* out, cudaStream_t stream);

}  // namespace leea
