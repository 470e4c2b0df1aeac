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

}  // extern "C"
