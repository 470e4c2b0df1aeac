// leea_surrogate_capi.cu -- C ABI of the surrogate form (include/leea.h):
// the MLP's row-level entry points.
#include "capi_common.h"

#include <cmath>

using namespace leea;
using namespace leea::capi;

namespace {

leea_status check_mlp(int32_t d_in, int32_t h1, int32_t h2)
{
    if (d_in < 1 || d_in > 4096 || h1 < 1 || h1 > 1024 || h2 < 1 || h2 > 1024)
        return fail(LEEA_EINVAL, "surrogate shape must have 1 <= d_in <= 4096 and 1 <= h1, h2 <= 1024");
    if (surrogate_forward_smem(d_in, h1, h2) > 227u * 1024u)
        return fail(LEEA_EINVAL, "surrogate shape too large for the forward kernel's shared memory");
    return LEEA_OK;
}

}  // namespace

extern "C" {

int64_t leea_surrogate_num_params(int32_t d_in, int32_t h1, int32_t h2)
{
    if (d_in < 1 || h1 < 1 || h2 < 1) return -1;
    return surrogate_num_params(d_in, h1, h2);
}

int64_t leea_surrogate_work_floats(int32_t n, int32_t h1, int32_t h2)
{
    if (n < 1 || h1 < 1 || h2 < 1) return -1;
    return static_cast<int64_t>(surrogate_work_floats(n, h1, h2));
}

leea_status leea_surrogate_init(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, float* theta_dev, void* stream)
{
    leea_status st = check_mlp(d_in, h1, h2);
    if (st) return st;
    if (!theta_dev) return fail(LEEA_EINVAL, "NULL device pointer");
    LEEA_CUDA_TRY(launch_surrogate_init(d_in, h1, h2, seed, theta_dev, static_cast<cudaStream_t>(stream)),
                  "surrogate init kernel");
    return LEEA_OK;
}

leea_status leea_surrogate_forward(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta_dev,
                                   const float* x_dev, float* y_dev, void* stream)
{
    leea_status st = check_mlp(d_in, h1, h2);
    if (st) return st;
    if (n < 0) return fail(LEEA_EINVAL, "n must be >= 0");
    if (n == 0) return LEEA_OK;
    if (!theta_dev || !x_dev || !y_dev) return fail(LEEA_EINVAL, "NULL device pointer");
    LEEA_CUDA_TRY(launch_surrogate_forward(n, d_in, h1, h2, theta_dev, x_dev, y_dev, nullptr, nullptr,
                                           static_cast<cudaStream_t>(stream)),
                  "surrogate forward kernel");
    return LEEA_OK;
}

leea_status leea_surrogate_loss_grad(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta_dev,
                                     const float* x_dev, const float* t_dev, float* loss_dev, float* grad_dev,
                                     float* work_dev, int64_t work_floats, void* stream)
{
    leea_status st = check_mlp(d_in, h1, h2);
    if (st) return st;
    if (n < 1) return fail(LEEA_EINVAL, "n must be >= 1");
    if (!theta_dev || !x_dev || !t_dev || !loss_dev || !grad_dev || !work_dev)
        return fail(LEEA_EINVAL, "NULL device pointer");
    if (work_floats < static_cast<int64_t>(surrogate_work_floats(n, h1, h2)))
        return fail(LEEA_EINVAL, "work needs %lld floats", static_cast<long long>(surrogate_work_floats(n, h1, h2)));
    LEEA_CUDA_TRY(launch_surrogate_loss_grad(n, d_in, h1, h2, theta_dev, x_dev, t_dev, loss_dev, grad_dev, work_dev,
                                             static_cast<cudaStream_t>(stream)),
                  "surrogate gradient kernels");
    return LEEA_OK;
}

leea_status leea_surrogate_adam(int64_t n_params, float* theta_dev, const float* grad_dev, float* m_dev, float* v_dev,
                                int64_t step, float lr, float beta1, float beta2, float eps, void* stream)
{
    if (n_params < 1 || step < 1) return fail(LEEA_EINVAL, "n_params and step must be >= 1");
    if (!(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(LEEA_EINVAL, "Adam needs lr > 0, 0 <= beta1, beta2 < 1 and eps > 0");
    if (!theta_dev || !grad_dev || !m_dev || !v_dev) return fail(LEEA_EINVAL, "NULL device pointer");
    LEEA_CUDA_TRY(launch_surrogate_adam(n_params, theta_dev, grad_dev, m_dev, v_dev, step, lr, beta1, beta2, eps,
                                        static_cast<cudaStream_t>(stream)),
                  "surrogate Adam kernel");
    return LEEA_OK;
}

int32_t leea_num_recipes(int32_t pop, const leea_params* p, int32_t mult)
{
    if (pop < 1 || !p || mult < 1 || check_params(p)) return -1;
    int32_t ne, nc, nm, pool;
    counts_of(pop, p, &ne, &nc, &nm, &pool);
    return mult * (nc + nm);
}

leea_status leea_select_recipes(int32_t pop, const leea_params* p, const float* f_adj_dev, const int32_t* order_dev,
                                uint64_t seed, uint32_t gen, int32_t mult, int32_t* par1_dev, int32_t* par2_dev,
                                int32_t* kind_dev, float* f_inh_dev, uint32_t* entity_dev, void* stream)
{
    leea_status st = check_pop(pop);
    if (st) return st;
    if ((st = check_params(p))) return st;
    if ((st = require_const_sigma(p, "leea_select_recipes"))) return st;
    if (mult < 1 || static_cast<int64_t>(mult) * pop > (1 << 26)) return fail(LEEA_EINVAL, "mult must be >= 1");
    if (!f_adj_dev || !order_dev || !par1_dev || !par2_dev || !kind_dev || !f_inh_dev || !entity_dev)
        return fail(LEEA_EINVAL, "NULL device pointer");
    const SelectArgs a = select_args(pop, p, seed, gen);
    LEEA_CUDA_TRY(launch_select_recipes(a, mult, f_adj_dev, order_dev, par1_dev, par2_dev, kind_dev, f_inh_dev,
                                        entity_dev, static_cast<cudaStream_t>(stream)),
                  "recipe selection kernel");
    return LEEA_OK;
}

leea_status leea_breed_entities(int32_t n_parents, const int32_t* dims, int32_t n_dims, const leea_params* p,
                                uint64_t seed, uint32_t gen, const float* parents_dev, const int32_t* par1_dev,
                                const int32_t* par2_dev, const int32_t* kind_dev, const uint32_t* entity_dev,
                                int32_t n_children, float* children_dev, void* stream)
{
    leea_status st = check_pop(n_parents);
    if (st) return st;
    if ((st = check_pop(n_children))) return st;
    if ((st = check_params(p))) return st;
    if (p->precision != 0) return fail(LEEA_EINVAL, "leea_breed_entities takes precision 0");
    if ((st = require_const_sigma(p, "leea_breed_entities"))) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, p->init, &net)) return fail(LEEA_EINVAL, "invalid dims");
    if (!parents_dev || !par1_dev || !par2_dev || !kind_dev || !entity_dev || !children_dev)
        return fail(LEEA_EINVAL, "NULL device pointer");
    if ((reinterpret_cast<uintptr_t>(parents_dev) | reinterpret_cast<uintptr_t>(children_dev)) & 15u)
        return fail(LEEA_EINVAL, "population buffers must be 16-byte aligned");
    BreedArgs a = breed_args(n_children, net, p, seed, gen);
    a.entity = entity_dev;
    a.n_parents = n_parents;
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    LEEA_CUDA_TRY(launch_breed(a, parents_dev, par1_dev, par2_dev, kind_dev, children_dev, status,
                               static_cast<cudaStream_t>(stream)),
                  "breed kernel");
    return LEEA_OK;
}

leea_status leea_descriptors(int32_t n_parents, const int32_t* dims, int32_t n_dims, const leea_params* p,
                             uint64_t seed, uint32_t gen, const float* parents_dev, const float* f_adj_dev,
                             const int32_t* par1_dev, const int32_t* par2_dev, const int32_t* kind_dev,
                             const float* f_inh_dev, const uint32_t* entity_dev, int32_t n,
                             const float* probe_dev, int32_t n_probe, float* desc_dev, void* stream)
{
    leea_status st = check_pop(n_parents);
    if (st) return st;
    if ((st = check_params(p))) return st;
    if ((st = require_const_sigma(p, "leea_descriptors"))) return st;
    NetLayout net;
    if (!make_layout(dims, n_dims, p->init, &net) || net.n_layers != 2)
        return fail(LEEA_EINVAL, "descriptors take d_0-h-d_out nets (n_dims == 3)");
    if (!probe_supported(net.dims[0], net.dims[1], net.dims[2], n_probe, p->precision))
        return fail(LEEA_EINVAL, "descriptors need d_0 %% 16 == 0, h %% 16 == 0, 16 <= h <= 256 (<= 128 with "
                                 "precision >= 1), d_out <= 16 and 1 <= n_probe <= 32");
    if (n < 0) return fail(LEEA_EINVAL, "n must be >= 0");
    if (n == 0) return LEEA_OK;
    if (!parents_dev || !f_adj_dev || !par1_dev || !par2_dev || !kind_dev || !f_inh_dev || !probe_dev || !desc_dev)
        return fail(LEEA_EINVAL, "NULL device pointer");
    if (reinterpret_cast<uintptr_t>(parents_dev) & 15u) return fail(LEEA_EINVAL, "parents must be 16-byte aligned");
    ProbeArgs a{};
    a.k = net.dims[0];
    a.h = net.dims[1];
    a.d_out = net.dims[2];
    a.n_probe = n_probe;
    a.width = 5 + n_probe * net.dims[2];
    a.xo_op = p->xo_op;
    a.c = net.c;
    a.c_pad = net.c_pad;
    a.thr_xo = threshold16(static_cast<double>(p->xo_gene_p));
    a.thr_mut = threshold16(static_cast<double>(p->mut_rate));
    a.gen = gen;
    a.sigma = p->sigma;
    a.seed = seed;
    a.parents = parents_dev;
    a.f_adj = f_adj_dev;
    a.par1 = par1_dev;
    a.par2 = par2_dev;
    a.kind = kind_dev;
    a.f_inh = f_inh_dev;
    a.entity = entity_dev;
    a.probe = probe_dev;
    a.desc = desc_dev;
    a.precision = p->precision;
    a.status = device_status_ptr();
    if (!a.status) return fail(LEEA_ECUDA, "device status word unavailable");
    if (reinterpret_cast<uintptr_t>(probe_dev) & 3u) return fail(LEEA_EINVAL, "probe must be 4-byte aligned");
    LEEA_CUDA_TRY(launch_descriptors(a, n, static_cast<cudaStream_t>(stream)), "probe kernel");
    return LEEA_OK;
}

}  // extern "C"
