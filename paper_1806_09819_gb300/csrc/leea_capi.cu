// leea_capi.cu -- the C ABI declared in include/leea.h: argument checking,
// layout arithmetic, the step entry points and the state object that strings
// them together in the order of Algorithm 1.
#include "leea.h"
#include "leea_internal.h"
#include "capi_common.h"

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

using namespace leea;

namespace leea {
namespace capi {

thread_local char g_error[1024] = "";

leea_status fail(leea_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_error, sizeof(g_error), fmt, ap);
    va_end(ap);
    return st;
}

leea_status cuda_fail(cudaError_t err, const char* what)
{
    if (err == cudaErrorMemoryAllocation)
        return fail(LEEA_ENOMEM, "%s: %s", what, cudaGetErrorString(err));
    return fail(LEEA_ECUDA, "%s: %s", what, cudaGetErrorString(err));
}


// Offsets of Section 3.2's direct encoding, plus the initialisation scale of
// each weight matrix (Section 4.1).
bool make_layout(const int32_t* dims, int32_t n_dims, int32_t init, NetLayout* net)
{
    if (!dims || n_dims < 2 || n_dims > kMaxLayers + 1) return false;
    std::memset(net, 0, sizeof(*net));
    net->n_layers = n_dims - 1;
    int64_t off = 0;
    for (int l = 0; l < n_dims; ++l) {
        if (dims[l] <= 0 || dims[l] > (1 << 20)) return false;
        net->dims[l] = dims[l];
    }
    for (int l = 0; l + 1 < n_dims; ++l) {
        const int64_t fan_in = dims[l], fan_out = dims[l + 1];
        net->w_off[l] = off;
        off += fan_in * fan_out;
        net->b_off[l] = off;
        off += fan_out;
        net->init_scale[l] = init == 1 ? static_cast<float>(std::sqrt(6.0 / static_cast<double>(fan_in + fan_out)))
                                       : static_cast<float>(std::sqrt(1.0 / static_cast<double>(fan_in)));
    }
    net->c = off;
    net->c_pad = (off + 31) / 32 * 32;
    return off < (int64_t{1} << 32);  // gene indices feed 32-bit Philox counters
}

// Threshold of the 16-bit per-gene mask draws: a draw hits iff below it.
uint32_t threshold16(double q)
{
    if (!(q > 0.0)) return 0;
    if (q >= 1.0) return 65536u;
    return static_cast<uint32_t>(std::floor(q * 65536.0));
}

leea_status check_params(const leea_params* p)
{
    if (!p) return fail(LEEA_EINVAL, "params is NULL");
    if (p->xo_op != 0 && p->xo_op != 1) return fail(LEEA_EINVAL, "xo_op must be 0 or 1");
    if (p->sel_op != 0 && p->sel_op != 1) return fail(LEEA_EINVAL, "sel_op must be 0 or 1");
    if (!(p->xo_gene_p >= 0.0f && p->xo_gene_p <= 1.0f)) return fail(LEEA_EINVAL, "xo_gene_p not in [0,1]");
    if (!(p->rho > 0.0f && p->rho <= 1.0f)) return fail(LEEA_EINVAL, "rho not in (0,1]");
    if (p->sel_op == 1 && p->tour_k < 1) return fail(LEEA_EINVAL, "tour_k must be >= 1");
    if (!(p->p_e >= 0.0f && p->p_e <= 1.0f)) return fail(LEEA_EINVAL, "p_e not in [0,1]");
    if (!(p->p_c >= 0.0f && p->p_c <= 1.0f)) return fail(LEEA_EINVAL, "p_c not in [0,1]");
    if (!(p->sigma >= 0.0f) || std::isinf(p->sigma)) return fail(LEEA_EINVAL, "sigma must be finite and >= 0");
    if (!(p->mut_rate >= 0.0f && p->mut_rate <= 1.0f)) return fail(LEEA_EINVAL, "mut_rate not in [0,1]");
    if (!(p->alpha >= 0.0f && p->alpha <= 1.0f)) return fail(LEEA_EINVAL, "alpha not in [0,1]");
    if (p->init != 0 && p->init != 1) return fail(LEEA_EINVAL, "init must be 0 or 1");
    if (p->precision < 0 || p->precision > 2) return fail(LEEA_EINVAL, "precision must be 0, 1 or 2");
    if (p->eval_path < LEEA_EVAL_AUTO || p->eval_path > LEEA_EVAL_SMALL)
        return fail(LEEA_EINVAL, "eval_path must be LEEA_EVAL_AUTO, _SIMT, _TENSOR, _FUSED or _SMALL");
    if (p->eval_path == LEEA_EVAL_FUSED && p->precision != 0)
        return fail(LEEA_EINVAL, "the fused breed + evaluate path takes precision 0");
    if (p->eval_path == LEEA_EVAL_SMALL && p->precision != 0)
        return fail(LEEA_EINVAL, "the single-launch generation takes precision 0");
    if (p->sigma_ctl < LEEA_SIGMA_CONST || p->sigma_ctl > LEEA_SIGMA_SELF)
        return fail(LEEA_EINVAL, "sigma_ctl must be LEEA_SIGMA_CONST, _DECAY or _SELF");
    if (p->sigma_ctl == LEEA_SIGMA_DECAY && !(p->sigma_k > 0.0f && !std::isinf(p->sigma_k)))
        return fail(LEEA_EINVAL, "sigma_k must be finite and > 0");
    if (p->sigma_ctl == LEEA_SIGMA_SELF && !(p->tau >= 0.0f && !std::isinf(p->tau)))
        return fail(LEEA_EINVAL, "tau must be finite and >= 0");
    return LEEA_OK;
}

leea_status require_const_sigma(const leea_params* p, const char* what)
{
    if (p->sigma_ctl != LEEA_SIGMA_CONST)
        return fail(LEEA_EINVAL, "%s takes sigma_ctl LEEA_SIGMA_CONST; sigma control runs in the state object", what);
    return LEEA_OK;
}

// Same rounding rules as the paper's proportions demand (Algorithm 1): round()
// for elites and crossover children, the rest mutate; pool = max(1, floor(rho pop)).
void counts_of(int32_t pop, const leea_params* p, int32_t* ne, int32_t* nc, int32_t* nm, int32_t* pool)
{
    int32_t e = p->n_elite >= 0 ? p->n_elite
                                : static_cast<int32_t>(std::round(static_cast<double>(p->p_e) * pop));
    e = e > pop ? pop : (e < 0 ? 0 : e);
    int32_t c = static_cast<int32_t>(std::round(static_cast<double>(p->p_c) * pop));
    c = c > pop - e ? pop - e : (c < 0 ? 0 : c);
    int32_t pl = static_cast<int32_t>(std::floor(static_cast<double>(p->rho) * pop));
    pl = pl < 1 ? 1 : (pl > pop ? pop : pl);
    *ne = e;
    *nc = c;
    *nm = pop - e - c;
    *pool = pl;
}

constexpr int32_t kMaxPop = 1 << 24;

// Status word written by kernels whose waits are bounded (one per device).
__device__ unsigned int g_device_status = 0;

// Device address of g_device_status on the current device (looked up once per
// device, with that device current).
// Host threads may race on the first lookup; each stores the same address,
// and the atomic entries make that race well defined.
unsigned int* device_status_ptr()
{
    static std::atomic<unsigned int*> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    unsigned int* hit = cache[dev].load(std::memory_order_acquire);
    if (!hit) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
        hit = static_cast<unsigned int*>(p);
        cache[dev].store(hit, std::memory_order_release);
    }
    return hit;
}

// Scratch of leea_evaluate_shadow_u8_noalloc: the per-tile partial sums of one
// call (2 floats per individual and 128-sample tile), LEEA_NOALLOC_SCRATCH_BYTES
// per device.  Callers of that entry point cannot allocate, so the array is
// static; its contents need no initial value (each call writes every slot it
// reads) and calls that overlap on the device share it.
static __device__ __align__(256) float g_noalloc_scratch[LEEA_NOALLOC_SCRATCH_BYTES / sizeof(float)];

// Device address of g_noalloc_scratch on the current device (looked up once
// per device, with that device current); NULL with the CUDA error in *err.
float* noalloc_scratch_ptr(cudaError_t* err)
{
    static std::atomic<float*> cache[64];  // same-address stores only, as in device_status_ptr
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    float* hit = cache[dev].load(std::memory_order_acquire);
    if (!hit) {
        *err = cudaGetSymbolAddress(reinterpret_cast<void**>(&hit), g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        cache[dev].store(hit, std::memory_order_release);
    }
    return hit;
}

// Synchronises `stream`, reads and clears the status word.
leea_status check_device_status(cudaStream_t stream, uint32_t* flags_out)
{
    cudaError_t err = cudaStreamSynchronize(stream);
    if (err != cudaSuccess) return cuda_fail(err, "stream synchronise");
    unsigned int* p = device_status_ptr();
    if (!p) return fail(LEEA_ECUDA, "device status word unavailable");
    unsigned int v = 0;
    err = cudaMemcpy(&v, p, sizeof(v), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return cuda_fail(err, "status read");
    if (v) {
        const unsigned int zero = 0;
        err = cudaMemcpy(p, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) return cuda_fail(err, "status clear");
    }
    if (flags_out) *flags_out = v;
    if (v & kStatusEvalTimeout)
        return fail(LEEA_ETIMEOUT, "a tensor-core evaluation wait timed out; its fitness values are invalid");
    if (v & kStatusBreedTimeout)
        return fail(LEEA_ETIMEOUT, "a breed kernel wait timed out; the children are invalid");
    if (v & kStatusProbeTimeout)
        return fail(LEEA_ETIMEOUT, "a tensor-core probe wait timed out; the descriptors are invalid");
    if (v & kStatusSelftestTimeout)
        return fail(LEEA_ETIMEOUT, "the self-test's bounded wait gave up (as it is meant to)");
    return LEEA_OK;
}

// Runs the evaluation kernel that `path` selects (LEEA_EVAL_*).
leea_status dispatch_eval(const NetLayout& net, int32_t pop, const float* pop_dev, const float* x,
                          const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                          float* f_adj, int32_t* correct, int32_t path, cudaStream_t stream)
{
    if (net.n_layers > 2) {  // several hidden layers: CUDA-core FP32
        if (path == LEEA_EVAL_TENSOR) return fail(LEEA_EINVAL, "nets with several hidden layers evaluate on CUDA cores");
        LEEA_CUDA_TRY(launch_eval_mlp(net, pop, pop_dev, x, y, batch, alpha, f_inh, f_raw, f_adj, correct, stream),
                      "evaluate kernel");
        return LEEA_OK;
    }
    const bool tc_ok = eval_tc_supported(net, batch, pop_dev, x);
    if (path == LEEA_EVAL_TENSOR && !tc_ok)
        return fail(LEEA_EINVAL, "tensor-core evaluation needs d_0 %% 4 == 0, h %% 16 == 0, h <= 256, "
                                 "d_out <= 16 and 16-byte aligned population and x");
    cudaError_t err;
    if (tc_ok && path != LEEA_EVAL_SIMT) {
        unsigned int* status = device_status_ptr();
        if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
        err = launch_eval_tc(net, pop, pop_dev, x, y, batch, alpha, f_inh, f_raw, f_adj, correct, status, stream);
    } else {
        err = launch_eval_simt(net, pop, pop_dev, x, y, batch, alpha, f_inh, f_raw, f_adj, correct, stream);
    }
    if (err != cudaSuccess) return cuda_fail(err, "evaluate kernel");
    return LEEA_OK;
}

// The same for 8-bit inputs x = k / x_div.
leea_status dispatch_eval_u8(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x, float x_div,
                             const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                             float* f_adj, int32_t* correct, int32_t path, cudaStream_t stream, void* mlp_scratch,
                             void* x16, bool x16_staged)
{
    if (!(x_div > 0.0f) || std::isinf(x_div)) return fail(LEEA_EINVAL, "x_div must be finite and > 0");
    if (net.n_layers > 2) {  // several hidden layers
        const bool tc = eval_mlp_tc_supported(net, pop_dev) && (reinterpret_cast<uintptr_t>(x) & 3u) == 0;
        if (path == LEEA_EVAL_TENSOR && !tc)
            return fail(LEEA_EINVAL, "tensor-core evaluation of deeper nets needs three hidden layers, widths multiples "
                                     "of 16 in [16, 256], d_0 %% 4 == 0, d_0 <= 256, d_out <= 16 "
                                     "and 4-byte aligned inputs");
        if (tc && path != LEEA_EVAL_SIMT) {
            unsigned int* status = device_status_ptr();
            if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
            LEEA_CUDA_TRY(launch_eval_mlp_tc(net, pop, pop_dev, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct,
                                             status, stream, mlp_scratch),
                          "evaluate kernel");
        } else {
            LEEA_CUDA_TRY(launch_eval_mlp_u8(net, pop, pop_dev, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj,
                                             correct, stream),
                          "evaluate kernel");
        }
        return LEEA_OK;
    }
    const bool tc_ok = eval_u8_tc_supported(net, batch, pop_dev);
    if (path == LEEA_EVAL_TENSOR && !tc_ok)
        return fail(LEEA_EINVAL, "tensor-core evaluation of 8-bit inputs needs batch <= 128, d_0 %% 4 == 0, "
                                 "h %% 16 == 0, h <= 128, d_out <= 16 and a 16-byte aligned population");
    cudaError_t err;
    if (tc_ok && path != LEEA_EVAL_SIMT) {
        unsigned int* status = device_status_ptr();
        if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
        void* own = nullptr;  // the call's own FP16 batch, freed in stream order after the evaluation
        if (!x16) {
            LEEA_CUDA_TRY(cudaMallocAsync(&own, eval_u8_x16_bytes(net, batch), stream), "batch staging allocation");
            x16 = own;
            x16_staged = false;
        }
        err = x16_staged ? cudaSuccess : launch_stage_x16(net, x, batch, x16, stream);
        if (err == cudaSuccess)
            err = launch_eval_u8_tc(net, pop, pop_dev, x, x16, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct,
                                    status, stream);
        if (own) {
            const cudaError_t ferr = cudaFreeAsync(own, stream);
            if (err == cudaSuccess) err = ferr;
        }
    } else {
        err = launch_eval_simt_u8(net, pop, pop_dev, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct,
                                  stream);
    }
    if (err != cudaSuccess) return cuda_fail(err, "evaluate kernel");
    return LEEA_OK;
}

leea_status check_pop(int32_t pop)
{
    if (pop <= 0 || pop > kMaxPop) return fail(LEEA_EINVAL, "pop must be in [1, %d]", kMaxPop);
    return LEEA_OK;
}

leea_status check_eval_shape(const NetLayout& net, int32_t batch)
{
    if (net.n_layers < 2) return fail(LEEA_EINVAL, "evaluation needs a hidden layer (n_dims >= 3)");
    if (net.dims[net.n_layers] > 32) return fail(LEEA_EINVAL, "evaluation supports d_out <= 32");
    if (net.n_layers > 2 && !eval_mlp_supported(net))
        return fail(LEEA_EINVAL, "nets with several hidden layers need every layer input and hidden width <= 256");
    if (batch <= 0) return fail(LEEA_EINVAL, "batch must be >= 1");
    return LEEA_OK;
}

int64_t shadow_stride_of(const NetLayout& net, int32_t precision)
{
    return shadow_stride_bytes(net.dims[0], net.dims[1], precision == 1 ? 2 : 1);
}

leea_status check_shadow_shape(const NetLayout& net, int32_t precision)
{
    if (precision != 1 && precision != 2) return fail(LEEA_EINVAL, "precision must be 1 (BF16) or 2 (FP8)");
    if (!eval_shadow_supported(net, precision, 1))
        return fail(LEEA_EINVAL, "the precision form needs n_dims == 3, d_0 %% 16 == 0, h %% 16 == 0, h <= 256, "
                                 "d_out <= 16 and at most 496 TMEM columns for the batch tile");
    return LEEA_OK;
}

leea_status dispatch_eval_shadow(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                                 const uint8_t* shadow, const int32_t* scale_exp, const uint8_t* x, float x_div,
                                 const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                                 float* f_adj, int32_t* correct, float* scratch, cudaStream_t stream)
{
    if (!(x_div > 0.0f) || std::isinf(x_div)) return fail(LEEA_EINVAL, "x_div must be finite and > 0");
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    LEEA_CUDA_TRY(launch_eval_shadow(net, pop, pop_dev, precision, shadow, shadow_stride_of(net, precision),
                                     scale_exp, x, x_div, y, batch, alpha, f_inh, f_raw, f_adj, correct, scratch,
                                     status, stream),
                  "shadow evaluate kernel");
    return LEEA_OK;
}

SelectArgs select_args(int32_t pop, const leea_params* p, uint64_t seed, uint32_t gen)
{
    SelectArgs a{};
    int32_t ne, nc, nm, pl;
    counts_of(pop, p, &ne, &nc, &nm, &pl);
    a.pop = pop;
    a.n_elite = ne;
    a.n_cross = nc;
    a.pool = pl;
    a.sel_op = p->sel_op;
    a.tour_k = p->tour_k;
    a.seed = seed;
    a.gen = gen;
    return a;
}

BreedArgs breed_args(int32_t pop, const NetLayout& net, const leea_params* p, uint64_t seed,
                            uint32_t gen)
{
    BreedArgs a{};
    a.pop = pop;
    a.c = net.c;
    a.c_pad = net.c_pad;
    a.xo_op = p->xo_op;
    a.thr_xo = threshold16(static_cast<double>(p->xo_gene_p));
    a.thr_mut = threshold16(static_cast<double>(p->mut_rate));
    a.sigma = p->sigma;
    a.seed = seed;
    a.gen = gen;
    return a;
}

}  // namespace capi
}  // namespace leea

using namespace leea::capi;

// ------------------------------------------------------------------------
// Plain functions
// ------------------------------------------------------------------------
extern "C" {

const char* leea_last_error(void) { return g_error; }

leea_status leea_default_params(leea_params* out)
{
    if (!out) return fail(LEEA_EINVAL, "out is NULL");
    out->xo_op = 0;
    out->xo_gene_p = 0.5f;
    out->sel_op = 0;
    out->rho = 0.5f;
    out->tour_k = 3;
    out->n_elite = -1;
    out->p_e = 0.05f;
    out->p_c = 0.5f;
    out->sigma = 0.001f;
    out->mut_rate = 1.0f;
    out->alpha = 1.0f;
    out->init = 0;
    out->precision = 0;
    out->eval_path = LEEA_EVAL_AUTO;
    out->sigma_ctl = LEEA_SIGMA_CONST;
    out->sigma_k = 1.0f;
    out->tau = 0.1f;
    return LEEA_OK;
}

int64_t leea_layout_num_params(const int32_t* dims, int32_t n_dims)
{
    NetLayout net;
    return make_layout(dims, n_dims, 0, &net) ? net.c : -1;
}

int64_t leea_padded_params(const int32_t* dims, int32_t n_dims)
{
    NetLayout net;
    return make_layout(dims, n_dims, 0, &net) ? net.c_pad : -1;
}

leea_status leea_counts(int32_t pop, const leea_params* p, int32_t* n_elite, int32_t* n_crossover,
                        int32_t* n_mutation, int32_t* pool)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if ((st = check_params(p))) return st;
    int32_t ne, nc, nm, pl;
    counts_of(pop, p, &ne, &nc, &nm, &pl);
    if (n_elite) *n_elite = ne;
    if (n_crossover) *n_crossover = nc;
    if (n_mutation) *n_mutation = nm;
    if (pool) *pool = pl;
    return LEEA_OK;
}

// ------------------------------------------------------------------------
// Step entry points
// ------------------------------------------------------------------------
leea_status leea_init_population(int32_t pop, const int32_t* dims, int32_t n_dims, int32_t init,
                                 uint64_t seed, float* pop_dev, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if (init != 0 && init != 1) return fail(LEEA_EINVAL, "init must be 0 or 1");
    NetLayout net;
    if (!make_layout(dims, n_dims, init, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if (!pop_dev) return fail(LEEA_EINVAL, "pop_dev is NULL");
    LEEA_CUDA_TRY(launch_init(net, pop, init, seed, pop_dev, static_cast<cudaStream_t>(stream)), "init kernel");
    return LEEA_OK;
}

leea_status leea_rank(int32_t pop, const float* f_adj_dev, int32_t* order_dev, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if (!f_adj_dev || !order_dev) return fail(LEEA_EINVAL, "NULL device pointer");
    LEEA_CUDA_TRY(launch_rank(pop, f_adj_dev, order_dev, static_cast<cudaStream_t>(stream)), "rank kernel");
    return LEEA_OK;
}

leea_status leea_select(int32_t pop, const leea_params* p, const float* f_adj_dev,
                        const int32_t* order_dev, uint64_t seed, uint32_t gen, int32_t* par1_dev,
                        int32_t* par2_dev, int32_t* kind_dev, float* f_inh_dev, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if ((st = check_params(p))) return st;
    if (p->precision != 0) return fail(LEEA_EINVAL, "leea_select takes precision 0; use the state object");
    if ((st = require_const_sigma(p, "leea_select"))) return st;
    if (!f_adj_dev || !order_dev || !par1_dev || !par2_dev || !kind_dev || !f_inh_dev)
        return fail(LEEA_EINVAL, "NULL device pointer");
    const SelectArgs a = select_args(pop, p, seed, gen);
    LEEA_CUDA_TRY(launch_select(a, f_adj_dev, order_dev, par1_dev, par2_dev, kind_dev, f_inh_dev,
                                static_cast<cudaStream_t>(stream)),
                  "select kernel");
    return LEEA_OK;
}

leea_status leea_breed(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_params* p,
                       uint64_t seed, uint32_t gen, const float* parents_dev, const int32_t* par1_dev,
                       const int32_t* par2_dev, const int32_t* kind_dev, float* children_dev,
                       void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if ((st = check_params(p))) return st;
    if (p->precision != 0)
        return fail(LEEA_EINVAL, "leea_breed takes precision 0; use the state object or leea_make_shadow");
    if ((st = require_const_sigma(p, "leea_breed"))) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, p->init, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if (!parents_dev || !par1_dev || !par2_dev || !kind_dev || !children_dev)
        return fail(LEEA_EINVAL, "NULL device pointer");
    const size_t bytes = sizeof(float) * static_cast<size_t>(pop) * static_cast<size_t>(net.c_pad);
    const char* pa = reinterpret_cast<const char*>(parents_dev);
    const char* ch = reinterpret_cast<const char*>(children_dev);
    if (pa < ch + bytes && ch < pa + bytes) return fail(LEEA_EINVAL, "parents and children overlap");
    if ((reinterpret_cast<uintptr_t>(parents_dev) | reinterpret_cast<uintptr_t>(children_dev)) & 15u)
        return fail(LEEA_EINVAL, "population buffers must be 16-byte aligned");
    const BreedArgs a = breed_args(pop, net, p, seed, gen);
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    LEEA_CUDA_TRY(launch_breed(a, parents_dev, par1_dev, par2_dev, kind_dev, children_dev, status,
                               static_cast<cudaStream_t>(stream)),
                  "breed kernel");
    return LEEA_OK;
}

leea_status leea_breed_evaluate_u8(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_params* p,
                                   uint64_t seed, uint32_t gen, const float* parents_dev, const int32_t* par1_dev,
                                   const int32_t* par2_dev, const int32_t* kind_dev, float* children_dev,
                                   const uint8_t* x_u8_dev, float x_div, const int32_t* y_dev, int32_t batch,
                                   float alpha, const float* f_inh_dev, float* f_raw_dev, float* f_adj_dev,
                                   int32_t* correct_dev, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if ((st = check_params(p))) return st;
    if (p->precision != 0) return fail(LEEA_EINVAL, "leea_breed_evaluate_u8 takes precision 0");
    if ((st = require_const_sigma(p, "leea_breed_evaluate_u8"))) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, p->init, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if ((st = check_eval_shape(net, batch))) return st;
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(LEEA_EINVAL, "alpha not in [0,1]");
    if (!(x_div > 0.0f) || std::isinf(x_div)) return fail(LEEA_EINVAL, "x_div must be finite and > 0");
    if (!parents_dev || !par1_dev || !par2_dev || !kind_dev || !children_dev || !x_u8_dev || !y_dev || !f_raw_dev)
        return fail(LEEA_EINVAL, "NULL device pointer");
    const size_t bytes = sizeof(float) * static_cast<size_t>(pop) * static_cast<size_t>(net.c_pad);
    const char* pa = reinterpret_cast<const char*>(parents_dev);
    const char* ch = reinterpret_cast<const char*>(children_dev);
    if (pa < ch + bytes && ch < pa + bytes) return fail(LEEA_EINVAL, "parents and children overlap");
    if (!breed_eval_u8_supported(net, batch, parents_dev, children_dev))
        return fail(LEEA_EINVAL, "the fused breed + evaluate kernel needs n_dims == 3, d_0 %% 16 == 0, h %% 16 == 0, "
                                 "h <= 128, d_out <= 16, batch <= 128 and 16-byte aligned populations");
    const BreedArgs a = breed_args(pop, net, p, seed, gen);
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    LEEA_CUDA_TRY(launch_breed_eval_u8(a, net, parents_dev, par1_dev, par2_dev, kind_dev, children_dev, x_u8_dev,
                                       x_div, y_dev, batch, alpha, f_inh_dev, f_raw_dev, f_adj_dev, correct_dev, status,
                                       static_cast<cudaStream_t>(stream)),
                  "breed + evaluate kernel");
    return LEEA_OK;
}

leea_status leea_evaluate(int32_t pop, const int32_t* dims, int32_t n_dims, const float* pop_dev,
                          const float* x_dev, const int32_t* y_dev, int32_t batch, float alpha,
                          const float* f_inh_dev, float* f_raw_dev, float* f_adj_dev,
                          int32_t* correct_dev, int32_t eval_path, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, 0, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if ((st = check_eval_shape(net, batch))) return st;
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(LEEA_EINVAL, "alpha not in [0,1]");
    if (!pop_dev || !x_dev || !y_dev || !f_raw_dev) return fail(LEEA_EINVAL, "NULL device pointer");
    if (eval_path < LEEA_EVAL_AUTO || eval_path > LEEA_EVAL_TENSOR) return fail(LEEA_EINVAL, "bad eval_path");
    return dispatch_eval(net, pop, pop_dev, x_dev, y_dev, batch, alpha, f_inh_dev, f_raw_dev, f_adj_dev,
                         correct_dev, eval_path, static_cast<cudaStream_t>(stream));
}

leea_status leea_evaluate_u8(int32_t pop, const int32_t* dims, int32_t n_dims, const float* pop_dev,
                             const uint8_t* x_u8_dev, float x_div, const int32_t* y_dev, int32_t batch, float alpha,
                             const float* f_inh_dev, float* f_raw_dev, float* f_adj_dev, int32_t* correct_dev,
                             int32_t eval_path, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, 0, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if ((st = check_eval_shape(net, batch))) return st;
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(LEEA_EINVAL, "alpha not in [0,1]");
    if (!pop_dev || !x_u8_dev || !y_dev || !f_raw_dev) return fail(LEEA_EINVAL, "NULL device pointer");
    if (eval_path < LEEA_EVAL_AUTO || eval_path > LEEA_EVAL_TENSOR) return fail(LEEA_EINVAL, "bad eval_path");
    return dispatch_eval_u8(net, pop, pop_dev, x_u8_dev, x_div, y_dev, batch, alpha, f_inh_dev, f_raw_dev, f_adj_dev,
                            correct_dev, eval_path, static_cast<cudaStream_t>(stream));
}

leea_status leea_maxpool2x2(int32_t batch, int32_t h, int32_t w, const float* x_dev, float* out_dev, void* stream)
{
    if (batch < 0 || h <= 0 || w <= 0 || (h & 1) || (w & 1))
        return fail(LEEA_EINVAL, "max-pooling needs batch >= 0 and even h, w >= 2");
    if (batch > 0 && (!x_dev || !out_dev)) return fail(LEEA_EINVAL, "NULL device pointer");
    LEEA_CUDA_TRY(launch_maxpool2x2(batch, h, w, x_dev, out_dev, static_cast<cudaStream_t>(stream)), "max-pool kernel");
    return LEEA_OK;
}

leea_status leea_maxpool2x2_u8(int32_t batch, int32_t h, int32_t w, const uint8_t* x_dev, uint8_t* out_dev,
                               void* stream)
{
    if (batch < 0 || h <= 0 || w <= 0 || (h & 1) || (w & 1))
        return fail(LEEA_EINVAL, "max-pooling needs batch >= 0 and even h, w >= 2");
    if (batch > 0 && (!x_dev || !out_dev)) return fail(LEEA_EINVAL, "NULL device pointer");
    LEEA_CUDA_TRY(launch_maxpool2x2_u8(batch, h, w, x_dev, out_dev, static_cast<cudaStream_t>(stream)),
                  "max-pool kernel");
    return LEEA_OK;
}

int64_t leea_shadow_stride(const int32_t* dims, int32_t n_dims, int32_t precision)
{
    NetLayout net;
    if (!make_layout(dims, n_dims, 0, &net) || net.n_layers != 2 || (precision != 1 && precision != 2)) return -1;
    return shadow_stride_of(net, precision);
}

leea_status leea_make_shadow(int32_t pop, const int32_t* dims, int32_t n_dims, int32_t precision,
                             const float* pop_dev, uint8_t* shadow_dev, int32_t* scale_exp_dev, float* amax_dev,
                             void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, 0, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if ((st = check_shadow_shape(net, precision))) return st;
    if (!pop_dev || !shadow_dev || !amax_dev || (precision == 2 && !scale_exp_dev))
        return fail(LEEA_EINVAL, "NULL device pointer");
    if ((reinterpret_cast<uintptr_t>(pop_dev) & 15u) || (reinterpret_cast<uintptr_t>(shadow_dev) & 127u))
        return fail(LEEA_EINVAL, "population must be 16-byte and shadow 128-byte aligned");
    LEEA_CUDA_TRY(launch_make_shadow(pop, net.dims[0], net.dims[1], net.c_pad, pop_dev, precision, shadow_dev,
                                     shadow_stride_of(net, precision), scale_exp_dev, amax_dev,
                                     static_cast<cudaStream_t>(stream)),
                  "make shadow kernel");
    return LEEA_OK;
}

int64_t leea_shadow_scratch_bytes(int32_t pop, int32_t batch)
{
    if (pop <= 0 || batch <= 0) return 0;
    return static_cast<int64_t>(eval_shadow_scratch_bytes(pop, batch));
}

leea_status leea_evaluate_shadow_u8(int32_t pop, const int32_t* dims, int32_t n_dims, const float* pop_dev,
                                    int32_t precision, const uint8_t* shadow_dev, const int32_t* scale_exp_dev,
                                    const uint8_t* x_u8_dev, float x_div, const int32_t* y_dev, int32_t batch,
                                    float alpha, const float* f_inh_dev, float* f_raw_dev, float* f_adj_dev,
                                    int32_t* correct_dev, float* scratch_dev, int64_t scratch_bytes, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, 0, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if ((st = check_shadow_shape(net, precision))) return st;
    if (batch <= 0) return fail(LEEA_EINVAL, "batch must be >= 1");
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(LEEA_EINVAL, "alpha not in [0,1]");
    if (!pop_dev || !shadow_dev || !x_u8_dev || !y_dev || !f_raw_dev || (precision == 2 && !scale_exp_dev))
        return fail(LEEA_EINVAL, "NULL device pointer");
    if ((reinterpret_cast<uintptr_t>(pop_dev) & 15u) || (reinterpret_cast<uintptr_t>(shadow_dev) & 127u) ||
        (reinterpret_cast<uintptr_t>(x_u8_dev) & 15u))
        return fail(LEEA_EINVAL, "population, x (16-byte) and shadow (128-byte) must be aligned");
    const int64_t need = static_cast<int64_t>(eval_shadow_scratch_bytes(pop, batch));
    if (need > 0 && (!scratch_dev || scratch_bytes < need))
        return fail(LEEA_EINVAL, "batch %d needs %lld scratch bytes", batch, static_cast<long long>(need));
    return dispatch_eval_shadow(net, pop, pop_dev, precision, shadow_dev, scale_exp_dev, x_u8_dev, x_div, y_dev,
                                batch, alpha, f_inh_dev, f_raw_dev, f_adj_dev, correct_dev, scratch_dev,
                                static_cast<cudaStream_t>(stream));
}

leea_status leea_evaluate_shadow_u8_noalloc(int32_t pop, const int32_t* dims, int32_t n_dims, const float* pop_dev,
                                            int32_t precision, const uint8_t* shadow_dev, const int32_t* scale_exp_dev,
                                            const uint8_t* x_u8_dev, float x_div, const int32_t* y_dev, int32_t batch,
                                            float alpha, const float* f_inh_dev, float* f_raw_dev, float* f_adj_dev,
                                            int32_t* correct_dev, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if (batch <= 0) return fail(LEEA_EINVAL, "batch must be >= 1");
    // The size limit depends on pop and batch alone, so it is checked before
    // anything else about the request.
    const size_t need = eval_shadow_scratch_bytes(pop, batch);
    if (need > static_cast<size_t>(LEEA_NOALLOC_SCRATCH_BYTES))
        return fail(LEEA_EINVAL,
                    "pop %d with batch %d needs %zu scratch bytes, above the %d bytes the allocation-free entry "
                    "point holds; use leea_evaluate_shadow_u8 with caller scratch",
                    pop, batch, need, LEEA_NOALLOC_SCRATCH_BYTES);
    NetLayout net;
    if (!make_layout(dims, n_dims, 0, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if ((st = check_shadow_shape(net, precision))) return st;
    if (!(alpha >= 0.0f && alpha <= 1.0f)) return fail(LEEA_EINVAL, "alpha not in [0,1]");
    if (!pop_dev || !shadow_dev || !x_u8_dev || !y_dev || !f_raw_dev || (precision == 2 && !scale_exp_dev))
        return fail(LEEA_EINVAL, "NULL device pointer");
    if ((reinterpret_cast<uintptr_t>(pop_dev) & 15u) || (reinterpret_cast<uintptr_t>(shadow_dev) & 127u) ||
        (reinterpret_cast<uintptr_t>(x_u8_dev) & 15u))
        return fail(LEEA_EINVAL, "population, x (16-byte) and shadow (128-byte) must be aligned");
    float* scratch = nullptr;
    if (need > 0) {
        cudaError_t err = cudaSuccess;
        scratch = noalloc_scratch_ptr(&err);
        if (!scratch) return cuda_fail(err, "static scratch address lookup");
    }
    return dispatch_eval_shadow(net, pop, pop_dev, precision, shadow_dev, scale_exp_dev, x_u8_dev, x_div, y_dev,
                                batch, alpha, f_inh_dev, f_raw_dev, f_adj_dev, correct_dev, scratch,
                                static_cast<cudaStream_t>(stream));
}

leea_status leea_device_status(void* stream, uint32_t* flags_out)
{
    return check_device_status(static_cast<cudaStream_t>(stream), flags_out);
}

leea_status leea_selftest_wait_timeout(uint32_t limit_us, void* stream)
{
    if (limit_us < 1 || limit_us > 1000000) return fail(LEEA_EINVAL, "limit_us must be in [1, 1000000]");
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    LEEA_CUDA_TRY(launch_wait_timeout_probe(static_cast<uint64_t>(limit_us) * 1000u, status,
                                            static_cast<cudaStream_t>(stream)),
                  "self-test kernel");
    return LEEA_OK;
}

leea_status leea_philox_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t n0,
                             int64_t count, uint32_t* out_dev, void* stream)
{
    if (count < 0 || !out_dev) return fail(LEEA_EINVAL, "bad count or NULL output");
    if (count == 0) return LEEA_OK;
    LEEA_CUDA_TRY(launch_philox_fill(seed, tag, gen, ent, n0, count, out_dev, static_cast<cudaStream_t>(stream)),
                  "philox fill kernel");
    return LEEA_OK;
}

leea_status leea_normal_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t n0,
                             int64_t count, float* out_dev, void* stream)
{
    if (count < 0 || !out_dev) return fail(LEEA_EINVAL, "bad count or NULL output");
    if (count == 0) return LEEA_OK;
    LEEA_CUDA_TRY(launch_normal_fill(seed, tag, gen, ent, n0, count, out_dev, static_cast<cudaStream_t>(stream)),
                  "normal fill kernel");
    return LEEA_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// State object
// ------------------------------------------------------------------------
namespace {

constexpr int kProfRing = 4096;

struct ProfileRing {
    cudaEvent_t ev[LEEA_NUM_STAGES][2][kProfRing];
    int n[LEEA_NUM_STAGES] = {};
    double ms[LEEA_NUM_STAGES] = {};
    int64_t launches[LEEA_NUM_STAGES] = {};
    bool created = false;
};

}  // namespace

struct leea_state {
    int32_t pop;
    NetLayout net;
    leea_params prm;
    uint64_t seed;
    cudaStream_t stream;
    uint32_t gen;
    bool evaluated;
    int cur;
    float* popbuf[2];
    float *f_adj, *f_raw, *f_inh;
    int32_t *correct, *order, *par1, *par2, *kind;
    void* x_stage;      // minibatch staging for the host entry points (float or uint8 rows)
    int32_t* y_stage;
    size_t x_stage_bytes;
    int64_t y_stage_cap;
    bool profiling;
    ProfileRing* prof;
    // precision form (prm.precision > 0)
    uint8_t* shadow[2];  // W1 shadows, paired with popbuf[0] / popbuf[1]
    float* amax[2];      // exact max |W1| per individual, paired likewise
    int32_t* scale_exp;  // FP8 scale exponents of the current population
    int64_t sh_stride;
    float* scratch;      // per-tile partial sums for batch > 128
    size_t scratch_bytes;
    // self-adaptive mutation strength (prm.sigma_ctl == LEEA_SIGMA_SELF)
    float* sigma[2];     // sigma genes, paired with popbuf[0] / popbuf[1]
    // tensor-core evaluation of deeper nets: weight pieces, marks, level tiles
    void* mlp_scratch;
    size_t mlp_scratch_bytes;
    // tensor-core evaluation of d_0-h-d_out nets on 8-bit inputs: the batch as
    // FP16 (at most 128 samples), staged once per generation
    void* x16;
    // precision form: the batch as the pair kernel's operand tiles (grown with the batch)
    void* xop;
    size_t xop_bytes;
    int32_t* sched;  // the group evaluation's two unit counters (zero between launches)
    // single-launch generation of small populations (eval_path SMALL, or AUTO)
    float* f_adj_alt;    // the other fitness buffer: a generation reads one and writes the other
    float* part;         // partial logits [pop][h / 8][batch][d_out] (grown with the batch)
    size_t part_bytes;
    uint32_t* count;     // arrivals per child (zero between launches)
};

namespace {

void free_state(leea_state* s)
{
    if (!s) return;
    cudaFree(s->popbuf[0]);
    cudaFree(s->popbuf[1]);
    cudaFree(s->f_adj);
    cudaFree(s->f_raw);
    cudaFree(s->f_inh);
    cudaFree(s->correct);
    cudaFree(s->order);
    cudaFree(s->par1);
    cudaFree(s->par2);
    cudaFree(s->kind);
    cudaFree(s->x_stage);
    cudaFree(s->y_stage);
    cudaFree(s->shadow[0]);
    cudaFree(s->shadow[1]);
    cudaFree(s->amax[0]);
    cudaFree(s->amax[1]);
    cudaFree(s->scale_exp);
    cudaFree(s->scratch);
    cudaFree(s->sigma[0]);
    cudaFree(s->sigma[1]);
    cudaFree(s->mlp_scratch);
    cudaFree(s->x16);
    cudaFree(s->xop);
    cudaFree(s->sched);
    cudaFree(s->f_adj_alt);
    cudaFree(s->part);
    cudaFree(s->count);
    if (s->prof) {
        if (s->prof->created)
            for (int st = 0; st < LEEA_NUM_STAGES; ++st)
                for (int e = 0; e < 2; ++e)
                    for (int k = 0; k < kProfRing; ++k) cudaEventDestroy(s->prof->ev[st][e][k]);
        delete s->prof;
    }
    delete s;
}

// Folds the recorded event pairs of every stage into the running sums.
leea_status prof_fold(leea_state* s)
{
    ProfileRing* pr = s->prof;
    if (!pr) return LEEA_OK;
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "profile sync");
    for (int st = 0; st < LEEA_NUM_STAGES; ++st) {
        for (int k = 0; k < pr->n[st]; ++k) {
            float ms = 0.0f;
            LEEA_CUDA_TRY(cudaEventElapsedTime(&ms, pr->ev[st][0][k], pr->ev[st][1][k]), "profile elapsed");
            pr->ms[st] += ms;
        }
        pr->launches[st] += pr->n[st];
        pr->n[st] = 0;
    }
    return LEEA_OK;
}

struct StageScope {
    leea_state* s;
    int stage;
    bool on;
    StageScope(leea_state* st, int stage_) : s(st), stage(stage_), on(st->profiling && st->prof)
    {
        if (!on) return;
        if (s->prof->n[stage] == kProfRing) prof_fold(s);
        cudaEventRecord(s->prof->ev[stage][0][s->prof->n[stage]], s->stream);
    }
    void done()
    {
        if (!on) return;
        cudaEventRecord(s->prof->ev[stage][1][s->prof->n[stage]], s->stream);
        s->prof->n[stage]++;
        on = false;
    }
};

// Shadows, exponents and maxima of the current population from its master.
cudaError_t refresh_shadow(leea_state* s)
{
    return launch_make_shadow(s->pop, s->net.dims[0], s->net.dims[1], s->net.c_pad, s->popbuf[s->cur],
                              s->prm.precision, s->shadow[s->cur], s->sh_stride, s->scale_exp, s->amax[s->cur],
                              s->stream);
}

// Mutation strength of the breed with generation counter g >= 1, breed number
// i = g - 1 (Section 3.2): sigma, or sigma 0.99^(i / k) under decay.
float sigma_of_breed(const leea_params& p, uint32_t g)
{
    if (p.sigma_ctl != LEEA_SIGMA_DECAY) return p.sigma;
    const double i = g > 0 ? static_cast<double>(g - 1u) : 0.0;
    return static_cast<float>(static_cast<double>(p.sigma) * std::pow(0.99, i / static_cast<double>(p.sigma_k)));
}

leea_status check_state(leea_state* s)
{
    if (!s) return fail(LEEA_EINVAL, "state is NULL");
    return LEEA_OK;
}

}  // namespace

extern "C" {

leea_status leea_create(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_params* p,
                        uint64_t seed, void* stream, leea_state** out)
{
    if (!out) return fail(LEEA_EINVAL, "out is NULL");
    *out = nullptr;
    leea_status st = check_pop(pop);
    if (st) return st;
    if ((st = check_params(p))) return st;
    leea_state* s = new (std::nothrow) leea_state();
    if (!s) return fail(LEEA_ENOMEM, "host allocation failed");
    if (!make_layout(dims, n_dims, p->init, &s->net)) {
        delete s;
        return fail(LEEA_EINVAL, "invalid dims");
    }
    if (s->net.n_layers < 2 || s->net.dims[s->net.n_layers] > 32 ||
        (s->net.n_layers > 2 && !eval_mlp_supported(s->net))) {
        delete s;
        return fail(LEEA_EINVAL, "the state object evaluates nets with hidden layers (n_dims >= 3), d_out <= 32, and "
                                 "with several hidden layers every layer input and hidden width <= 256");
    }
    if (s->net.n_layers > 2 &&
        (p->precision != 0 || p->eval_path == LEEA_EVAL_FUSED || p->eval_path == LEEA_EVAL_SMALL)) {
        delete s;
        return fail(LEEA_EINVAL, "nets with several hidden layers evaluate FP32 populations, breeding and evaluation "
                                 "as separate kernels");
    }
    if (p->precision != 0 && (st = check_shadow_shape(s->net, p->precision))) {
        delete s;
        return st;
    }
    s->pop = pop;
    s->prm = *p;
    s->seed = seed;
    s->stream = static_cast<cudaStream_t>(stream);
    const size_t np = static_cast<size_t>(pop);
    const size_t pop_bytes = sizeof(float) * np * static_cast<size_t>(s->net.c_pad);
    cudaError_t err = cudaSuccess;
    for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = cudaMalloc(&s->popbuf[b], pop_bytes);
    if (err == cudaSuccess) err = cudaMalloc(&s->f_adj, sizeof(float) * np);
    if (err == cudaSuccess) err = cudaMalloc(&s->f_raw, sizeof(float) * np);
    if (err == cudaSuccess) err = cudaMalloc(&s->f_inh, sizeof(float) * np);
    if (err == cudaSuccess) err = cudaMalloc(&s->correct, sizeof(int32_t) * np);
    if (err == cudaSuccess) err = cudaMalloc(&s->order, sizeof(int32_t) * np);
    if (err == cudaSuccess) err = cudaMalloc(&s->par1, sizeof(int32_t) * np);
    if (err == cudaSuccess) err = cudaMalloc(&s->par2, sizeof(int32_t) * np);
    if (err == cudaSuccess) err = cudaMalloc(&s->kind, sizeof(int32_t) * np);
    if (p->precision != 0) {
        s->sh_stride = shadow_stride_of(s->net, p->precision);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = cudaMalloc(&s->shadow[b], np * s->sh_stride);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = cudaMalloc(&s->amax[b], sizeof(float) * np);
        if (err == cudaSuccess) err = cudaMalloc(&s->scale_exp, sizeof(int32_t) * np);
        if (err == cudaSuccess) err = cudaMemsetAsync(s->scale_exp, 0, sizeof(int32_t) * np, s->stream);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b)  // zero padding of the tiled layout
            err = cudaMemsetAsync(s->shadow[b], 0, np * s->sh_stride, s->stream);
    }
    if (s->net.n_layers > 2 && err == cudaSuccess && eval_mlp_tc_supported(s->net, s->popbuf[0]) &&
        p->eval_path != LEEA_EVAL_SIMT) {
        s->mlp_scratch_bytes = eval_mlp_tc_scratch_bytes(s->net, pop, 0);  // grown with the batch
        err = cudaMalloc(&s->mlp_scratch, s->mlp_scratch_bytes);
    }
    if (s->net.n_layers == 2 && p->precision == 0 && err == cudaSuccess &&
        eval_u8_tc_supported(s->net, 128, s->popbuf[0]))
        err = cudaMalloc(&s->x16, eval_u8_x16_bytes(s->net, 128));
    if (p->sigma_ctl == LEEA_SIGMA_SELF) {
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = cudaMalloc(&s->sigma[b], sizeof(float) * np);
        if (err == cudaSuccess) {  // every individual starts with the sigma gene p->sigma
            std::vector<float> init(np, p->sigma);
            err = cudaMemcpyAsync(s->sigma[0], init.data(), sizeof(float) * np, cudaMemcpyHostToDevice, s->stream);
            if (err == cudaSuccess) err = cudaStreamSynchronize(s->stream);
        }
    }
    if (err != cudaSuccess) {
        free_state(s);
        return cuda_fail(err, "leea_create allocation");
    }
    err = cudaMemsetAsync(s->popbuf[1], 0, pop_bytes, s->stream);
    if (err == cudaSuccess) err = launch_init(s->net, pop, p->init, seed, s->popbuf[0], s->stream);
    if (err == cudaSuccess && p->precision != 0) err = refresh_shadow(s);
    if (err != cudaSuccess) {
        free_state(s);
        return cuda_fail(err, "leea_create init");
    }
    *out = s;
    return LEEA_OK;
}

// One generation of a small population in a single launch (launch_small_gen):
// the first call evaluates the initial population, later calls rank, select,
// breed and evaluate.  The kernel reads the previous fitness from one buffer
// and writes the new one to the other; the buffers then swap.
static leea_status run_small_generation(leea_state* s, const uint8_t* x_dev, const float* xf_dev, float x_div,
                                        const int32_t* y_dev, int32_t batch)
{
    const size_t np = static_cast<size_t>(s->pop);
    if (!s->count) {
        LEEA_CUDA_TRY(cudaMalloc(&s->count, sizeof(uint32_t) * np), "arrival counter allocation");
        LEEA_CUDA_TRY(cudaMemsetAsync(s->count, 0, sizeof(uint32_t) * np, s->stream), "arrival counter clear");
    }
    if (!s->f_adj_alt) LEEA_CUDA_TRY(cudaMalloc(&s->f_adj_alt, sizeof(float) * np), "fitness buffer allocation");
    const size_t need = sizeof(float) * np * static_cast<size_t>(s->net.dims[1] / 8) * static_cast<size_t>(batch) *
                        static_cast<size_t>(s->net.dims[2]);
    if (need > s->part_bytes) {
        LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "scratch sync");
        cudaFree(s->part);
        s->part = nullptr;
        s->part_bytes = 0;
        LEEA_CUDA_TRY(cudaMalloc(&s->part, need), "partial logit scratch allocation");
        s->part_bytes = need;
    }
    const bool first = !s->evaluated;
    SmallGenArgs ga{};
    ga.pop = s->pop;
    ga.d_in = s->net.dims[0];
    ga.h = s->net.dims[1];
    ga.d_out = s->net.dims[2];
    ga.batch = batch;
    ga.c = s->net.c;
    ga.c_pad = s->net.c_pad;
    ga.b1_off = s->net.b_off[0];
    ga.w2_off = s->net.w_off[1];
    ga.b2_off = s->net.b_off[1];
    ga.x_div = x_div;
    ga.alpha = s->prm.alpha;
    ga.order = s->order;
    ga.par1 = s->par1;
    ga.par2 = s->par2;
    ga.kind = s->kind;
    ga.f_inh = s->f_inh;
    ga.f_raw = s->f_raw;
    ga.correct = s->correct;
    ga.part = s->part;
    ga.count = s->count;
    ga.x = x_dev;
    ga.xf = xf_dev;
    ga.y = y_dev;
    if (first) {
        ga.breed = 0;
        ga.popv = s->popbuf[s->cur];
        ga.f_adj = s->f_adj;
        StageScope sc(s, 2);
        LEEA_CUDA_TRY(launch_small_gen(ga, s->stream), "single-launch generation kernel");
        sc.done();
        s->evaluated = true;
        return LEEA_OK;
    }
    const uint32_t g = s->gen + 1;
    const float sigma_g = sigma_of_breed(s->prm, g);
    ga.breed = 1;
    ga.sel = select_args(s->pop, &s->prm, s->seed, g);
    ga.sel.sigma = sigma_g;
    if (s->prm.sigma_ctl == LEEA_SIGMA_SELF) {
        ga.sel.tau = s->prm.tau;
        ga.sel.sigma_in = s->sigma[s->cur];
        ga.sel.sigma_out = s->sigma[s->cur ^ 1];
    }
    ga.br = breed_args(s->pop, s->net, &s->prm, s->seed, g);
    ga.br.sigma = sigma_g;
    ga.parents = s->popbuf[s->cur];
    ga.popv = s->popbuf[s->cur ^ 1];
    ga.f_adj_in = s->f_adj;
    ga.f_adj = s->f_adj_alt;
    {
        StageScope sc(s, 1);
        LEEA_CUDA_TRY(launch_small_gen(ga, s->stream), "single-launch generation kernel");
        sc.done();
    }
    std::swap(s->f_adj, s->f_adj_alt);
    s->cur ^= 1;
    s->gen = g;
    return LEEA_OK;
}

static leea_status run_generation(leea_state* s, const void* x_dev, bool u8, float x_div, const int32_t* y_dev,
                                  int32_t batch)
{
    leea_status st = check_state(s);
    if (st) return st;
    if ((st = check_eval_shape(s->net, batch))) return st;
    if (!x_dev || !y_dev) return fail(LEEA_EINVAL, "NULL minibatch pointer");
    if (u8 && (!(x_div > 0.0f) || std::isinf(x_div))) return fail(LEEA_EINVAL, "x_div must be finite and > 0");
    const int32_t prec = s->prm.precision;
    if (prec != 0) {
        if (!u8) return fail(LEEA_EINVAL, "the precision form evaluates 8-bit inputs (leea_generation_u8*)");
        if (s->prm.eval_path == LEEA_EVAL_SIMT)
            return fail(LEEA_EINVAL, "the precision form runs on the tensor cores (eval_path SIMT not allowed)");
        if (reinterpret_cast<uintptr_t>(x_dev) & 15u) return fail(LEEA_EINVAL, "x must be 16-byte aligned");
        const size_t need = eval_shadow_scratch_bytes(s->pop, batch);
        if (need > s->scratch_bytes) {
            LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "scratch sync");
            cudaFree(s->scratch);
            s->scratch = nullptr;
            s->scratch_bytes = 0;
            LEEA_CUDA_TRY(cudaMalloc(&s->scratch, need), "scratch allocation");
            s->scratch_bytes = need;
        }
    }
    // The precision form's evaluation: two individuals per MMA where the
    // shape allows (h <= 128), else one individual of width up to 256 per MMA
    // (the group evaluation), on the batch staged as operand tiles.
    const bool shadow_pair = prec != 0 && eval_shadow_pair_supported(s->net, prec, batch);
    const bool shadow_group =
        prec != 0 && !shadow_pair && s->net.n_layers == 2 &&
        eval_shadow_group_supported(s->net.dims[0], s->net.dims[2], prec, s->net.dims[1],
                                    eval_shadow_group_size(s->net.dims[1]) * s->net.dims[1]);
    if (shadow_group && !s->sched) {
        LEEA_CUDA_TRY(cudaMalloc(&s->sched, 2 * sizeof(int32_t)), "unit counter allocation");
        LEEA_CUDA_TRY(cudaMemsetAsync(s->sched, 0, 2 * sizeof(int32_t), s->stream), "unit counter clear");
    }
    if (shadow_pair || shadow_group) {
        const size_t need = eval_shadow_pair_xop_bytes(s->net, prec, batch);
        if (need > s->xop_bytes) {
            LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "staging sync");
            cudaFree(s->xop);
            s->xop = nullptr;
            s->xop_bytes = 0;
            LEEA_CUDA_TRY(cudaMalloc(&s->xop, need), "batch staging allocation");
            s->xop_bytes = need;
        }
    }
    if (u8 && s->mlp_scratch) {
        const size_t need = eval_mlp_tc_scratch_bytes(s->net, s->pop, batch);
        if (need > s->mlp_scratch_bytes) {
            LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "scratch sync");
            cudaFree(s->mlp_scratch);
            s->mlp_scratch = nullptr;
            s->mlp_scratch_bytes = 0;
            LEEA_CUDA_TRY(cudaMalloc(&s->mlp_scratch, need), "scratch allocation");
            s->mlp_scratch_bytes = need;
        }
    }
    const bool first = !s->evaluated;
    // Breed and evaluate in one kernel (8-bit inputs of an FP32 object) when
    // asked for.  AUTO keeps the two kernels: at the benchmark's shape both
    // forms are bound by instruction issue, not by memory, and the two
    // kernels measure slightly faster than the fused one.
    const bool fused = s->prm.eval_path == LEEA_EVAL_FUSED;
    if (fused && u8 && !breed_eval_u8_supported(s->net, batch, s->popbuf[0], s->popbuf[1]))
        return fail(LEEA_EINVAL, "the fused breed + evaluate path needs d_0 %% 16 == 0, h %% 16 == 0, h <= 128, "
                                 "d_out <= 16 and batch <= 128");
    if (!u8 && s->prm.eval_path == LEEA_EVAL_FUSED)
        return fail(LEEA_EINVAL, "the fused breed + evaluate path takes 8-bit inputs (leea_generation_u8*)");
    // Small populations: the whole generation in one launch (SMALL, or AUTO
    // when its CTAs, one per child and 8 hidden units, fit twice on the GPU).
    const bool small_ok = prec == 0 && small_gen_supported(s->net, s->pop, batch) &&
                          (reinterpret_cast<uintptr_t>(x_dev) & (u8 ? 3u : 15u)) == 0;
    bool small = false;
    if (s->prm.eval_path == LEEA_EVAL_SMALL) {
        if (!small_ok)
            return fail(LEEA_EINVAL, "the single-launch generation needs a 4-byte aligned 8-bit or 16-byte aligned "
                                     "FP32 batch, one hidden "
                                     "layer with h %% 8 == 0 and h <= 256, d_0 %% 4 == 0 and d_0 <= 2048, "
                                     "d_out <= 32, batch <= 128, pop <= 1024 and the batch in 200 KB of shared memory");
        small = true;
    } else if (s->prm.eval_path == LEEA_EVAL_AUTO && small_ok) {
        int dev = 0, sms = 0;
        LEEA_CUDA_TRY(cudaGetDevice(&dev), "device query");
        LEEA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device query");
        small = small_gen_ctas(s->net, s->pop) <= 2 * sms;
    }
    if (small)
        return run_small_generation(s, u8 ? static_cast<const uint8_t*>(x_dev) : nullptr,
                                    u8 ? nullptr : static_cast<const float*>(x_dev), u8 ? x_div : 1.0f, y_dev, batch);
    // The tensor-core evaluation of 8-bit inputs reads the batch as FP16: a
    // breeding generation stages it beside the selection.
    const bool stage_early = !first && !fused && u8 && prec == 0 && s->x16 && s->prm.eval_path != LEEA_EVAL_SIMT &&
                             s->net.n_layers == 2 && eval_u8_tc_supported(s->net, batch, s->popbuf[0]);
    if (!first) {
        const uint32_t g = s->gen + 1;
        const float sigma_g = sigma_of_breed(s->prm, g);
        const bool self = s->prm.sigma_ctl == LEEA_SIGMA_SELF;
        {
            StageScope sc(s, 0);
            SelectArgs a = select_args(s->pop, &s->prm, s->seed, g);
            a.sigma = sigma_g;
            if (self) {
                a.tau = s->prm.tau;
                a.sigma_in = s->sigma[s->cur];
                a.sigma_out = s->sigma[s->cur ^ 1];
            }
            if (prec != 0) {
                a.precision = prec;
                a.amax_in = s->amax[s->cur];
                a.scale_exp_out = s->scale_exp;
                a.amax_out = s->amax[s->cur ^ 1];
            }
            LEEA_CUDA_TRY(launch_rank_select(a, s->f_adj, s->order, s->par1, s->par2, s->kind, s->f_inh, s->stream),
                          "rank/select kernel");
            if (stage_early)  // runs beside the selection; the breed that follows waits for both
                LEEA_CUDA_TRY(launch_stage_x16(s->net, static_cast<const uint8_t*>(x_dev), batch, s->x16, s->stream),
                              "batch staging kernel");
            if ((shadow_pair || shadow_group) && !fused)
                LEEA_CUDA_TRY(launch_stage_xop(s->net, prec, static_cast<const uint8_t*>(x_dev), batch, s->xop,
                                               s->stream),
                              "batch staging kernel");
            sc.done();
        }
        if (fused) {
            StageScope sc(s, 1);
            BreedArgs a = breed_args(s->pop, s->net, &s->prm, s->seed, g);
            a.sigma = sigma_g;
            if (self) a.sigma_child = s->sigma[s->cur ^ 1];
            unsigned int* status = device_status_ptr();
            if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
            LEEA_CUDA_TRY(launch_breed_eval_u8(a, s->net, s->popbuf[s->cur], s->par1, s->par2, s->kind,
                                               s->popbuf[s->cur ^ 1], static_cast<const uint8_t*>(x_dev), x_div,
                                               y_dev, batch, s->prm.alpha, s->f_inh, s->f_raw, s->f_adj, s->correct,
                                               status, s->stream),
                          "breed + evaluate kernel");
            sc.done();
            s->cur ^= 1;
            s->gen = g;
            return LEEA_OK;
        }
        {
            StageScope sc(s, 1);
            BreedArgs a = breed_args(s->pop, s->net, &s->prm, s->seed, g);
            a.sigma = sigma_g;
            if (self) a.sigma_child = s->sigma[s->cur ^ 1];
            if (prec != 0) {
                a.precision = prec;
                a.n_w1 = static_cast<int64_t>(s->net.dims[0]) * s->net.dims[1];
                a.sh_k = s->net.dims[0];
                a.sh_h = s->net.dims[1];
                a.shadow = s->shadow[s->cur ^ 1];
                a.sh_stride = s->sh_stride;
                a.scale_exp = s->scale_exp;
                a.amax_out = s->amax[s->cur ^ 1];
            }
            unsigned int* status = device_status_ptr();
            if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
            LEEA_CUDA_TRY(launch_breed(a, s->popbuf[s->cur], s->par1, s->par2, s->kind, s->popbuf[s->cur ^ 1],
                                       status, s->stream),
                          "breed kernel");
            sc.done();
        }
        s->cur ^= 1;
        s->gen = g;
    }
    {
        StageScope sc(s, 2);
        if (shadow_pair) {
            unsigned int* status = device_status_ptr();
            if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
            if (first)
                LEEA_CUDA_TRY(launch_stage_xop(s->net, prec, static_cast<const uint8_t*>(x_dev), batch, s->xop,
                                               s->stream),
                              "batch staging kernel");
            LEEA_CUDA_TRY(launch_eval_shadow_pair(s->net, s->pop, s->popbuf[s->cur], prec, s->shadow[s->cur],
                                                  s->sh_stride, s->scale_exp, s->xop, x_div, y_dev, batch,
                                                  s->prm.alpha, first ? nullptr : s->f_inh, s->f_raw, s->f_adj,
                                                  s->correct, s->scratch, status, s->stream),
                          "shadow evaluation kernel");
        } else if (shadow_group) {
            unsigned int* status = device_status_ptr();
            if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
            if (first)
                LEEA_CUDA_TRY(launch_stage_xop(s->net, prec, static_cast<const uint8_t*>(x_dev), batch, s->xop,
                                               s->stream),
                              "batch staging kernel");
            LEEA_CUDA_TRY(launch_eval_shadow_group_run(s->net, s->pop, s->popbuf[s->cur], prec, s->shadow[s->cur],
                                                       s->sh_stride, s->scale_exp, s->xop, x_div, y_dev, batch,
                                                       s->prm.alpha, first ? nullptr : s->f_inh, s->f_raw, s->f_adj,
                                                       s->correct, s->scratch, s->sched, status, s->stream),
                          "shadow group evaluation kernel");
        } else if (prec != 0)
            st = dispatch_eval_shadow(s->net, s->pop, s->popbuf[s->cur], prec, s->shadow[s->cur], s->scale_exp,
                                      static_cast<const uint8_t*>(x_dev), x_div, y_dev, batch, s->prm.alpha,
                                      first ? nullptr : s->f_inh, s->f_raw, s->f_adj, s->correct, s->scratch,
                                      s->stream);
        else if (u8)
            st = dispatch_eval_u8(s->net, s->pop, s->popbuf[s->cur], static_cast<const uint8_t*>(x_dev), x_div, y_dev,
                                  batch, s->prm.alpha, first ? nullptr : s->f_inh, s->f_raw, s->f_adj, s->correct,
                                  s->prm.eval_path, s->stream, s->mlp_scratch, s->x16, stage_early);
        else
            st = dispatch_eval(s->net, s->pop, s->popbuf[s->cur], static_cast<const float*>(x_dev), y_dev, batch,
                               s->prm.alpha, first ? nullptr : s->f_inh, s->f_raw, s->f_adj, s->correct,
                               s->prm.eval_path, s->stream);
        sc.done();
        if (st) return st;
    }
    s->evaluated = true;
    return LEEA_OK;
}

// Copies a host minibatch into the object's staging buffers (grown on demand).
static leea_status stage_batch(leea_state* s, const void* x_host, size_t x_bytes, const int32_t* y_host, int32_t batch)
{
    if (x_bytes > s->x_stage_bytes || batch > s->y_stage_cap) {
        LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "staging sync");
        if (x_bytes > s->x_stage_bytes) {
            cudaFree(s->x_stage);
            s->x_stage = nullptr;
            s->x_stage_bytes = 0;
            LEEA_CUDA_TRY(cudaMalloc(&s->x_stage, x_bytes), "staging allocation");
            s->x_stage_bytes = x_bytes;
        }
        if (batch > s->y_stage_cap) {
            cudaFree(s->y_stage);
            s->y_stage = nullptr;
            s->y_stage_cap = 0;
            LEEA_CUDA_TRY(cudaMalloc(&s->y_stage, sizeof(int32_t) * static_cast<size_t>(batch)), "staging allocation");
            s->y_stage_cap = batch;
        }
    }
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->x_stage, x_host, x_bytes, cudaMemcpyHostToDevice, s->stream), "minibatch copy");
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->y_stage, y_host, sizeof(int32_t) * static_cast<size_t>(batch),
                                  cudaMemcpyHostToDevice, s->stream),
                  "label copy");
    return LEEA_OK;
}

leea_status leea_generation(leea_state* s, const float* x_dev, const int32_t* y_dev, int32_t batch)
{
    return run_generation(s, x_dev, false, 1.0f, y_dev, batch);
}

leea_status leea_generation_u8(leea_state* s, const uint8_t* x_u8_dev, float x_div, const int32_t* y_dev,
                               int32_t batch)
{
    return run_generation(s, x_u8_dev, true, x_div, y_dev, batch);
}

leea_status leea_generation_u8_host(leea_state* s, const uint8_t* x_u8_host, float x_div, const int32_t* y_host,
                                    int32_t batch)
{
    leea_status st = check_state(s);
    if (st) return st;
    if ((st = check_eval_shape(s->net, batch))) return st;
    if (!x_u8_host || !y_host) return fail(LEEA_EINVAL, "NULL minibatch pointer");
    if ((st = stage_batch(s, x_u8_host, static_cast<size_t>(batch) * s->net.dims[0], y_host, batch))) return st;
    return run_generation(s, s->x_stage, true, x_div, s->y_stage, batch);
}

leea_status leea_generation_host(leea_state* s, const float* x_host, const int32_t* y_host, int32_t batch)
{
    leea_status st = check_state(s);
    if (st) return st;
    if ((st = check_eval_shape(s->net, batch))) return st;
    if (!x_host || !y_host) return fail(LEEA_EINVAL, "NULL minibatch pointer");
    if ((st = stage_batch(s, x_host, sizeof(float) * static_cast<size_t>(batch) * s->net.dims[0], y_host, batch)))
        return st;
    return run_generation(s, s->x_stage, false, 1.0f, s->y_stage, batch);
}

static leea_status copy_out(leea_state* s, void* dst, const void* src, size_t bytes, const char* what)
{
    LEEA_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->stream), what);
    return check_device_status(s->stream, nullptr);
}

leea_status leea_fitness(leea_state* s, float* f_adj_host, int32_t* correct_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!s->evaluated) return fail(LEEA_ESTATE, "no generation has been evaluated yet");
    if (!f_adj_host) return fail(LEEA_EINVAL, "f_adj_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpyAsync(f_adj_host, s->f_adj, sizeof(float) * s->pop, cudaMemcpyDeviceToHost, s->stream),
                  "fitness copy");
    if (correct_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(correct_host, s->correct, sizeof(int32_t) * s->pop, cudaMemcpyDeviceToHost,
                                      s->stream),
                      "correct copy");
    return check_device_status(s->stream, nullptr);
}

leea_status leea_raw_fitness(leea_state* s, float* f_raw_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!s->evaluated) return fail(LEEA_ESTATE, "no generation has been evaluated yet");
    if (!f_raw_host) return fail(LEEA_EINVAL, "f_raw_host is NULL");
    return copy_out(s, f_raw_host, s->f_raw, sizeof(float) * s->pop, "raw fitness copy");
}

static bool beats(float a, int32_t ia, float b, int32_t ib)
{
    const float fa = std::isnan(a) ? -INFINITY : a, fb = std::isnan(b) ? -INFINITY : b;
    return fa > fb || (fa == fb && ia < ib);
}

leea_status leea_best_params(leea_state* s, float* out_host, int64_t c)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!s->evaluated) return fail(LEEA_ESTATE, "no generation has been evaluated yet");
    if (!out_host || c != s->net.c) return fail(LEEA_EINVAL, "out_host NULL or c != %lld", (long long)s->net.c);
    std::vector<float> f(static_cast<size_t>(s->pop));
    if ((st = copy_out(s, f.data(), s->f_adj, sizeof(float) * s->pop, "fitness copy"))) return st;
    int32_t best = 0;
    for (int32_t p = 1; p < s->pop; ++p)
        if (beats(f[p], p, f[best], best)) best = p;
    return copy_out(s, out_host, s->popbuf[s->cur] + static_cast<int64_t>(best) * s->net.c_pad,
                    sizeof(float) * static_cast<size_t>(c), "best params copy");
}

leea_status leea_get_population(leea_state* s, float* out_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!out_host) return fail(LEEA_EINVAL, "out_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpy2DAsync(out_host, sizeof(float) * s->net.c, s->popbuf[s->cur],
                                    sizeof(float) * s->net.c_pad, sizeof(float) * s->net.c, s->pop,
                                    cudaMemcpyDeviceToHost, s->stream),
                  "population copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "population sync");
    return LEEA_OK;
}

leea_status leea_set_population(leea_state* s, const float* in_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!in_host) return fail(LEEA_EINVAL, "in_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpy2DAsync(s->popbuf[s->cur], sizeof(float) * s->net.c_pad, in_host,
                                    sizeof(float) * s->net.c, sizeof(float) * s->net.c, s->pop,
                                    cudaMemcpyHostToDevice, s->stream),
                  "population copy");
    if (s->prm.precision != 0) LEEA_CUDA_TRY(refresh_shadow(s), "make shadow kernel");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "population sync");
    return LEEA_OK;
}

leea_status leea_get_shadow(leea_state* s, uint8_t* shadow_host, int32_t* scale_exp_host, float* amax_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (s->prm.precision == 0) return fail(LEEA_ESTATE, "the object computes in FP32 and has no shadows");
    if (shadow_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(shadow_host, s->shadow[s->cur], static_cast<size_t>(s->sh_stride) * s->pop,
                                      cudaMemcpyDeviceToHost, s->stream),
                      "shadow copy");
    if (scale_exp_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(scale_exp_host, s->scale_exp, sizeof(int32_t) * s->pop, cudaMemcpyDeviceToHost,
                                      s->stream),
                      "scale copy");
    if (amax_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(amax_host, s->amax[s->cur], sizeof(float) * s->pop, cudaMemcpyDeviceToHost,
                                      s->stream),
                      "amax copy");
    return check_device_status(s->stream, nullptr);
}

leea_status leea_set_fitness(leea_state* s, const float* f_adj_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!f_adj_host) return fail(LEEA_EINVAL, "f_adj_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->f_adj, f_adj_host, sizeof(float) * s->pop, cudaMemcpyHostToDevice, s->stream),
                  "fitness copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "fitness sync");
    return LEEA_OK;
}

leea_status leea_set_generation(leea_state* s, uint32_t gen, int32_t evaluated)
{
    leea_status st = check_state(s);
    if (st) return st;
    s->gen = gen;
    s->evaluated = evaluated != 0;
    return LEEA_OK;
}

leea_status leea_get_selection(leea_state* s, int32_t* order, int32_t* par1, int32_t* par2, int32_t* kind,
                               float* f_inh)
{
    leea_status st = check_state(s);
    if (st) return st;
    const size_t ni = sizeof(int32_t) * s->pop;
    struct { void* dst; const void* src; size_t n; } copies[] = {
        { order, s->order, ni }, { par1, s->par1, ni }, { par2, s->par2, ni },
        { kind, s->kind, ni }, { f_inh, s->f_inh, sizeof(float) * s->pop } };
    for (auto& c : copies)
        if (c.dst)
            LEEA_CUDA_TRY(cudaMemcpyAsync(c.dst, c.src, c.n, cudaMemcpyDeviceToHost, s->stream), "selection copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "selection sync");
    return LEEA_OK;
}

uint32_t leea_generation_index(const leea_state* s) { return s ? s->gen : 0u; }

leea_status leea_get_sigma(leea_state* s, float* sigma_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!sigma_host) return fail(LEEA_EINVAL, "sigma_host is NULL");
    const size_t np = static_cast<size_t>(s->pop);
    if (s->prm.sigma_ctl == LEEA_SIGMA_SELF) {
        LEEA_CUDA_TRY(cudaMemcpyAsync(sigma_host, s->sigma[s->cur], sizeof(float) * np, cudaMemcpyDeviceToHost,
                                      s->stream),
                      "sigma copy");
        return check_device_status(s->stream, nullptr);
    }
    const float next = sigma_of_breed(s->prm, s->gen + 1u);
    for (size_t p = 0; p < np; ++p) sigma_host[p] = next;
    return LEEA_OK;
}

leea_status leea_set_sigma(leea_state* s, const float* sigma_host)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!sigma_host) return fail(LEEA_EINVAL, "sigma_host is NULL");
    if (s->prm.sigma_ctl != LEEA_SIGMA_SELF) return fail(LEEA_ESTATE, "sigma genes exist under LEEA_SIGMA_SELF only");
    for (int32_t p = 0; p < s->pop; ++p)
        if (!(sigma_host[p] >= 0.0f) || std::isinf(sigma_host[p]))
            return fail(LEEA_EINVAL, "sigma gene %d must be finite and >= 0", p);
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->sigma[s->cur], sigma_host, sizeof(float) * static_cast<size_t>(s->pop),
                                  cudaMemcpyHostToDevice, s->stream),
                  "sigma copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "sigma copy");
    return LEEA_OK;
}

int64_t leea_num_params(const leea_state* s) { return s ? s->net.c : -1; }

leea_status leea_profile_enable(leea_state* s, int32_t enable)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (enable && !s->prof) {
        s->prof = new (std::nothrow) ProfileRing();
        if (!s->prof) return fail(LEEA_ENOMEM, "profile ring allocation");
        for (int stg = 0; stg < LEEA_NUM_STAGES; ++stg)
            for (int e = 0; e < 2; ++e)
                for (int k = 0; k < kProfRing; ++k)
                    LEEA_CUDA_TRY(cudaEventCreate(&s->prof->ev[stg][e][k]), "event create");
        s->prof->created = true;
    }
    s->profiling = enable != 0;
    return LEEA_OK;
}

leea_status leea_profile_read(leea_state* s, double* ms_out, int64_t* launches_out)
{
    leea_status st = check_state(s);
    if (st) return st;
    if (!ms_out || !launches_out) return fail(LEEA_EINVAL, "NULL output");
    if (!s->prof) {
        for (int k = 0; k < LEEA_NUM_STAGES; ++k) { ms_out[k] = 0.0; launches_out[k] = 0; }
        return LEEA_OK;
    }
    if ((st = prof_fold(s))) return st;
    for (int k = 0; k < LEEA_NUM_STAGES; ++k) {
        ms_out[k] = s->prof->ms[k];
        launches_out[k] = s->prof->launches[k];
        s->prof->ms[k] = 0.0;
        s->prof->launches[k] = 0;
    }
    return LEEA_OK;
}

void leea_destroy(leea_state* s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    free_state(s);
}

}  // extern "C"
