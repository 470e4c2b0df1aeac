// capi_common.h -- helpers the C ABI's translation units share: error
// reporting, argument checks, layout and the per-step kernel arguments.
#pragma once
#include "leea.h"
#include "leea_internal.h"

#include <cuda_runtime.h>

namespace leea {
namespace capi {

// Records a message for leea_last_error() and returns st.
leea_status fail(leea_status st, const char* fmt, ...);
// LEEA_ENOMEM for an allocation failure, LEEA_ECUDA otherwise.
leea_status cuda_fail(cudaError_t err, const char* what);

// Section 3.2's gene offsets and Section 4.1's init scales of a net.
bool make_layout(const int32_t* dims, int32_t n_dims, int32_t init, NetLayout* net);
// floor(q 2^16), 2^16 when q >= 1: the 16-bit draw threshold of probability q.
uint32_t threshold16(double q);
leea_status check_params(const leea_params* p);
// LEEA_EINVAL unless p->sigma_ctl is LEEA_SIGMA_CONST (calls outside the state object).
leea_status require_const_sigma(const leea_params* p, const char* what);
leea_status check_pop(int32_t pop);
// Elites, crossover and mutation children and the truncation pool (Algorithm 1).
void counts_of(int32_t pop, const leea_params* p, int32_t* ne, int32_t* nc, int32_t* nm, int32_t* pool);
// This device's status word (bounded waits report here).
unsigned int* device_status_ptr();
// Synchronises the stream, then reads and clears the status word.
leea_status check_device_status(cudaStream_t stream, uint32_t* flags_out);

int64_t shadow_stride_of(const NetLayout& net, int32_t precision);
leea_status check_shadow_shape(const NetLayout& net, int32_t precision);

// The evaluation kernel `path` selects (LEEA_EVAL_*) for 8-bit inputs x = k / x_div;
// mlp_scratch: the caller's scratch of the tensor-core evaluation of deeper nets
// (eval_mlp_tc_scratch_bytes), or NULL for the library's shared buffer.
// x16: the caller's buffer for the batch as FP16 (eval_u8_x16_bytes), already
// filled when x16_staged; NULL takes a stream-ordered allocation for the call.
leea_status dispatch_eval_u8(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x, float x_div,
                             const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                             float* f_adj, int32_t* correct, int32_t path, cudaStream_t stream,
                             void* mlp_scratch = nullptr, void* x16 = nullptr, bool x16_staged = false);
// The precision form's evaluation on W1 shadows (scratch: batch > 128).
leea_status dispatch_eval_shadow(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                                 const uint8_t* shadow, const int32_t* scale_exp, const uint8_t* x, float x_div,
                                 const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                                 float* f_adj, int32_t* correct, float* scratch, cudaStream_t stream);

SelectArgs select_args(int32_t pop, const leea_params* p, uint64_t seed, uint32_t gen);
BreedArgs breed_args(int32_t pop, const NetLayout& net, const leea_params* p, uint64_t seed, uint32_t gen);

}  // namespace capi
}  // namespace leea

#define LEEA_CUDA_TRY(expr, what)                                      \
    do {                                                               \
        cudaError_t err_ = (expr);                                     \
        if (err_ != cudaSuccess) return leea::capi::cuda_fail(err_, what); \
    } while (0)
