// leea_surr.cu -- the surrogate form as a state object: every generation
// draws mult x (n_C + n_M) recipes (virtual offspring), describes each with
// the fused breed + probe pass, scores them with the online-trained MLP, makes
// and evaluates only the best (P - n_E) of them plus a stratified audit
// sample of the rest, checks the ranking against the measured fitness
// (Spearman), and trains the MLP on the new (descriptor, fitness) pairs.  The
// choice between the pre-screen and the plain EA's offspring (the first n_C
// crossover and n_M mutation recipes, i.e. ignoring the scores) is a device
// flag that the audit sets for the next generation, so no step waits for the
// host.  The paper has no counterpart: its method evaluates every offspring.
#include "capi_common.h"

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using namespace leea;
using namespace leea::capi;

namespace {

// ---- kernels --------------------------------------------------------------------

// Mean and standard deviation of each descriptor column over `rows` rows
// (one CTA per column, fixed-order sums).
__global__ void feature_stats_kernel(int32_t rows, int32_t width, const float* __restrict__ desc,
                                     float* __restrict__ mu, float* __restrict__ sd)
{
    __shared__ double red[256];
    const int col = blockIdx.x;
    double s = 0.0;
    for (int32_t r = threadIdx.x; r < rows; r += 256) s += desc[static_cast<int64_t>(r) * width + col];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = red[0] / rows;
    __syncthreads();
    double q = 0.0;
    for (int32_t r = threadIdx.x; r < rows; r += 256) {
        const double d = desc[static_cast<int64_t>(r) * width + col] - mean;
        q += d * d;
    }
    red[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mu[col] = static_cast<float>(mean);
        const double v = red[0] / rows;
        sd[col] = static_cast<float>(v > 1e-24 ? sqrt(v) : 1.0);  // a constant column stays as is
    }
}

__global__ void standardize_kernel(int64_t n, int32_t width, const float* __restrict__ desc,
                                   const float* __restrict__ mu, const float* __restrict__ sd, float* __restrict__ out)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n * width;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int col = static_cast<int>(i % width);
        out[i] = (desc[i] - mu[col]) / sd[col];
    }
}

struct ChooseArgs {
    int32_t pop, n_elite, n_cross, n_mut, mult, n_rec, n_audit;
    const int32_t* order;    // ranking of the population's f_adj
    const float* f_adj;
    const int32_t* order_r;  // ranking of the recipes' predicted fitness
    const int32_t* use_screen;
    const int32_t *r_par1, *r_par2, *r_kind;
    const float* r_f_inh;
    const uint32_t* r_entity;
    int32_t *c_par1, *c_par2, *c_kind;
    float* c_f_inh;
    uint32_t* c_entity;
    int32_t *a_par1, *a_par2, *a_kind;
    uint32_t* a_entity;
    int32_t* row_recipe;     // recipe of each training row: children n_elite.., then the audit
    float* amax_c;
    float* amax_a;
};

// Without the pre-screen the offspring are the recipes the plain EA would make:
// crossovers 0 .. n_cross-1 and mutations mult n_cross .. mult n_cross + n_mut - 1.
__device__ __forceinline__ int32_t plain_recipe(const ChooseArgs& a, int32_t s)
{
    return s < a.n_cross ? s : a.mult * a.n_cross + (s - a.n_cross);
}

// Position p of the recipes the plain choice leaves out, in index order.
__device__ __forceinline__ int32_t plain_rest(const ChooseArgs& a, int32_t p)
{
    const int32_t xo_rest = (a.mult - 1) * a.n_cross;
    return p < xo_rest ? a.n_cross + p : a.mult * a.n_cross + a.n_mut + (p - xo_rest);
}

__global__ void choose_kernel(ChooseArgs a)
{
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t k = a.pop - a.n_elite;  // offspring slots
    if (t >= a.pop + a.n_audit) return;
    const bool screen = *a.use_screen != 0;
    if (t < a.n_elite) {
        const int32_t p = a.order[t];
        a.c_kind[t] = 0;
        a.c_par1[t] = p;
        a.c_par2[t] = p;
        a.c_f_inh[t] = a.f_adj[p];
        a.c_entity[t] = static_cast<uint32_t>(t);
        if (a.amax_c) a.amax_c[t] = 0.0f;
        return;
    }
    if (t < a.pop) {
        const int32_t s = t - a.n_elite;
        const int32_t q = screen ? a.order_r[s] : plain_recipe(a, s);
        a.c_kind[t] = a.r_kind[q];
        a.c_par1[t] = a.r_par1[q];
        a.c_par2[t] = a.r_par2[q];
        a.c_f_inh[t] = a.r_f_inh[q];
        a.c_entity[t] = a.r_entity[q];
        a.row_recipe[s] = q;
        if (a.amax_c) a.amax_c[t] = 0.0f;
        return;
    }
    const int32_t i = t - a.pop;  // audit: evenly spaced over the recipes left out
    const int32_t p = static_cast<int32_t>(static_cast<int64_t>(i) * (a.n_rec - k) / a.n_audit);
    const int32_t q = screen ? a.order_r[k + p] : plain_rest(a, p);
    a.a_kind[i] = a.r_kind[q];
    a.a_par1[i] = a.r_par1[q];
    a.a_par2[i] = a.r_par2[q];
    a.a_entity[i] = a.r_entity[q];
    a.row_recipe[k + i] = q;
    if (a.amax_a) a.amax_a[i] = 0.0f;
}

__global__ void gather_rows_kernel(int32_t n_rows, int32_t width, const int32_t* __restrict__ row_recipe,
                                   const float* __restrict__ x_std, float* __restrict__ out)
{
    const int32_t r = blockIdx.x;
    const float* src = x_std + static_cast<int64_t>(row_recipe[r]) * width;
    for (int c = threadIdx.x; c < width; c += blockDim.x) out[static_cast<int64_t>(r) * width + c] = src[c];
}

// Training targets: the rows' measured fitness, z-scored within the
// generation (non-finite values count as the lowest fitness); the rows'
// predictions alongside for the audit.
__global__ void targets_kernel(int32_t n_rows, int32_t k, int32_t n_elite, const float* __restrict__ f_children,
                               const float* __restrict__ f_audit, const float* __restrict__ pred,
                               const int32_t* __restrict__ row_recipe, float* __restrict__ meas,
                               float* __restrict__ pred_rows, float* __restrict__ t_out)
{
    __shared__ double red[256];
    __shared__ double s_mean, s_sd, s_min;
    double s = 0.0, lo = 1e300;
    int n_ok = 0;
    for (int32_t r = threadIdx.x; r < n_rows; r += 256) {
        const float f = r < k ? f_children[n_elite + r] : f_audit[r - k];
        meas[r] = f;
        pred_rows[r] = pred[row_recipe[r]];
        if (isfinite(f)) {
            s += f;
            lo = fmin(lo, static_cast<double>(f));
            ++n_ok;
        }
    }
    // fixed-order reductions: sum, count, minimum
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double sum = red[0];
    __syncthreads();
    red[threadIdx.x] = n_ok;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double cnt = red[0];
    __syncthreads();
    red[threadIdx.x] = lo;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s_mean = cnt > 0 ? sum / cnt : 0.0;
        s_min = cnt > 0 ? red[0] : 0.0;
    }
    __syncthreads();
    double q = 0.0;
    for (int32_t r = threadIdx.x; r < n_rows; r += 256) {
        const double f = isfinite(meas[r]) ? static_cast<double>(meas[r]) : s_min;
        q += (f - s_mean) * (f - s_mean);
    }
    red[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_sd = sqrt(red[0] / (n_rows > 0 ? n_rows : 1));
    __syncthreads();
    const double sd = s_sd > 1e-12 ? s_sd : 1.0;
    for (int32_t r = threadIdx.x; r < n_rows; r += 256) {
        const double f = isfinite(meas[r]) ? static_cast<double>(meas[r]) : s_min;
        t_out[r] = static_cast<float>((f - s_mean) / sd);
    }
}

// Spearman rank correlation of the rows' predictions and measurements from
// their two rankings (rank_kernel: larger first, NaN last, ties to the lower
// index); sets the pre-screen flag for the next generation.
__global__ void __launch_bounds__(1024) audit_kernel(int32_t n, const int32_t* __restrict__ order_p,
                                                     const int32_t* __restrict__ order_m, int32_t* __restrict__ rank_m,
                                                     float* __restrict__ stat, int32_t* __restrict__ use_screen,
                                                     int32_t allow, float min_rho)
{
    __shared__ double red[1024];
    for (int32_t i = threadIdx.x; i < n; i += 1024) rank_m[order_m[i]] = i;
    __syncthreads();
    double d2 = 0.0;
    for (int32_t i = threadIdx.x; i < n; i += 1024) {  // row order_p[i] has score rank i
        const double d = static_cast<double>(i - rank_m[order_p[i]]);
        d2 += d * d;
    }
    red[threadIdx.x] = d2;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nn = static_cast<double>(n);
        const double rho = n > 1 ? 1.0 - 6.0 * red[0] / (nn * (nn * nn - 1.0)) : 0.0;
        stat[0] = static_cast<float>(rho);
        stat[1] = static_cast<float>(*use_screen);
        *use_screen = (allow && rho >= static_cast<double>(min_rho)) ? 1 : 0;
    }
}

constexpr int kSurrStages = 5;

}  // namespace

struct leea_surr {
    int32_t pop = 0;
    NetLayout net{};
    leea_params prm{};
    leea_surrogate_params sp{};
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    int32_t n_elite = 0, n_cross = 0, n_mut = 0, n_rec = 0, n_audit = 0, k = 0, rows = 0, width = 0;
    int64_t n_theta = 0, sh_stride = 0;
    uint32_t gen = 0;
    bool evaluated = false;
    int cur = 0;
    int64_t breeds = 0;  // breeding generations so far (history ring position)
    // population
    float* popbuf[2] = { nullptr, nullptr };
    uint8_t* shadow[2] = { nullptr, nullptr };
    float* amax[2] = { nullptr, nullptr };
    float *f_adj = nullptr, *f_raw = nullptr;
    int32_t *correct = nullptr, *order = nullptr;
    // children of the last breed
    int32_t *c_par1 = nullptr, *c_par2 = nullptr, *c_kind = nullptr;
    float* c_f_inh = nullptr;
    uint32_t* c_entity = nullptr;
    // recipes
    int32_t *r_par1 = nullptr, *r_par2 = nullptr, *r_kind = nullptr, *order_r = nullptr;
    float *r_f_inh = nullptr, *desc = nullptr, *x_std = nullptr, *pred = nullptr;
    uint32_t* r_entity = nullptr;
    // audit offspring
    int32_t *a_par1 = nullptr, *a_par2 = nullptr, *a_kind = nullptr;
    uint32_t* a_entity = nullptr;
    float *a_pop = nullptr, *a_amax = nullptr, *a_f = nullptr;
    uint8_t* a_shadow = nullptr;
    // surrogate and its training data
    float *theta = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr, *work = nullptr, *loss = nullptr;
    float *mu = nullptr, *sd = nullptr, *probe = nullptr;
    float *x_hist = nullptr, *t_hist = nullptr, *meas = nullptr, *pred_rows = nullptr;
    int32_t* row_recipe = nullptr;
    int32_t *rank_p = nullptr, *rank_m = nullptr, *rank_tmp = nullptr;  // audit rankings
    int32_t* use_screen = nullptr;
    float* stats = nullptr;  // per breeding generation: spearman, screened, loss
    int64_t stats_cap = 0, adam_step = 0;
    float* scratch = nullptr;
    size_t scratch_bytes = 0;
    uint8_t* x_stage = nullptr;
    int32_t* y_stage = nullptr;
    size_t x_stage_bytes = 0;
    int64_t y_stage_cap = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    int n_prof = 0;
    double ms[kSurrStages] = {};
    int64_t launches = 0;
};

namespace {

constexpr int kSurrProfRing = 1024;

void free_surr(leea_surr* s)
{
    if (!s) return;
    void* ptrs[] = { s->popbuf[0], s->popbuf[1], s->shadow[0], s->shadow[1], s->amax[0], s->amax[1], s->f_adj,
                     s->f_raw, s->correct, s->order, s->c_par1, s->c_par2, s->c_kind, s->c_f_inh, s->c_entity,
                     s->r_par1, s->r_par2, s->r_kind, s->order_r, s->r_f_inh, s->desc, s->x_std, s->pred,
                     s->r_entity, s->a_par1, s->a_par2, s->a_kind, s->a_entity, s->a_pop, s->a_amax, s->a_f,
                     s->a_shadow, s->theta, s->adam_m, s->adam_v, s->grad, s->work, s->loss, s->mu, s->sd,
                     s->probe, s->x_hist, s->t_hist, s->meas, s->pred_rows, s->row_recipe, s->use_screen,
                     s->stats, s->scratch, s->x_stage, s->y_stage, s->rank_p, s->rank_m, s->rank_tmp };
    for (void* p : ptrs) cudaFree(p);
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    delete s;
}

template <typename T>
cudaError_t alloc(T** p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
}

cudaError_t evaluate(leea_surr* s, const float* popv, const uint8_t* shadow, int32_t n, const uint8_t* x, float x_div,
                     const int32_t* y, int32_t batch, const float* f_inh, float* f_raw, float* f_adj,
                     int32_t* correct, leea_status* st)
{
    if (s->prm.precision == 0)
        *st = dispatch_eval_u8(s->net, n, popv, x, x_div, y, batch, s->prm.alpha, f_inh, f_raw, f_adj, correct,
                               s->prm.eval_path, s->stream);
    else
        *st = dispatch_eval_shadow(s->net, n, popv, s->prm.precision, shadow, nullptr, x, x_div, y, batch,
                                   s->prm.alpha, f_inh, f_raw, f_adj, correct, s->scratch, s->stream);
    return cudaSuccess;
}

BreedArgs surr_breed_args(leea_surr* s, int32_t n, const uint32_t* entity, uint8_t* shadow, float* amax_out)
{
    BreedArgs a = breed_args(n, s->net, &s->prm, s->seed, s->gen + 1);
    a.entity = entity;
    a.n_parents = s->pop;
    if (s->prm.precision == 1) {
        a.precision = 1;
        a.n_w1 = static_cast<int64_t>(s->net.dims[0]) * s->net.dims[1];
        a.sh_k = s->net.dims[0];
        a.sh_h = s->net.dims[1];
        a.shadow = shadow;
        a.sh_stride = s->sh_stride;
        a.amax_out = amax_out;
    }
    return a;
}

void mark(leea_surr* s, int stage, int e)
{
    if (s->profiling) cudaEventRecord(s->ev[(stage * 2 + e) * kSurrProfRing + s->n_prof], s->stream);
}

leea_status fold_profile(leea_surr* s)
{
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "profile sync");
    for (int k = 0; k < s->n_prof; ++k)
        for (int st = 0; st < kSurrStages; ++st) {
            float ms = 0.0f;
            LEEA_CUDA_TRY(cudaEventElapsedTime(&ms, s->ev[(st * 2) * kSurrProfRing + k],
                                               s->ev[(st * 2 + 1) * kSurrProfRing + k]),
                          "profile elapsed");
            s->ms[st] += ms;
        }
    s->launches += s->n_prof;
    s->n_prof = 0;
    return LEEA_OK;
}

leea_status surr_breed_generation(leea_surr* s, const uint8_t* x, float x_div, const int32_t* y, int32_t batch)
{
    const uint32_t g = s->gen + 1;
    const cudaStream_t st = s->stream;
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    if (s->profiling && s->n_prof == kSurrProfRing) {
        leea_status ps = fold_profile(s);
        if (ps) return ps;
    }
    const int32_t d_out = s->net.dims[2];
    // 1. recipes and their descriptors
    mark(s, 0, 0);
    LEEA_CUDA_TRY(launch_rank(s->pop, s->f_adj, s->order, st), "rank kernel");
    SelectArgs sa = select_args(s->pop, &s->prm, s->seed, g);
    LEEA_CUDA_TRY(launch_select_recipes(sa, s->sp.mult, s->f_adj, s->order, s->r_par1, s->r_par2, s->r_kind,
                                        s->r_f_inh, s->r_entity, st),
                  "recipe selection kernel");
    ProbeArgs pa{};
    pa.k = s->net.dims[0];
    pa.h = s->net.dims[1];
    pa.d_out = d_out;
    pa.n_probe = s->sp.n_probe;
    pa.width = s->width;
    pa.xo_op = s->prm.xo_op;
    pa.c = s->net.c;
    pa.c_pad = s->net.c_pad;
    pa.thr_xo = threshold16(static_cast<double>(s->prm.xo_gene_p));
    pa.thr_mut = threshold16(static_cast<double>(s->prm.mut_rate));
    pa.gen = g;
    pa.sigma = s->prm.sigma;
    pa.seed = s->seed;
    pa.parents = s->popbuf[s->cur];
    pa.f_adj = s->f_adj;
    pa.par1 = s->r_par1;
    pa.par2 = s->r_par2;
    pa.kind = s->r_kind;
    pa.f_inh = s->r_f_inh;
    pa.entity = s->r_entity;
    pa.probe = s->probe;
    pa.desc = s->desc;
    pa.precision = s->prm.precision;
    pa.status = device_status_ptr();
    if (!pa.status) return fail(LEEA_ECUDA, "device status word unavailable");
    LEEA_CUDA_TRY(launch_descriptors(pa, s->n_rec, st), "probe kernel");
    mark(s, 0, 1);
    // 2. scores and the choice
    mark(s, 1, 0);
    // Each generation's descriptors are standardised by that generation's column
    // means and deviations: fitness and logits drift as the population learns,
    // and the targets are z-scored within the generation too.
    feature_stats_kernel<<<s->width, 256, 0, st>>>(s->n_rec, s->width, s->desc, s->mu, s->sd);
    LEEA_CUDA_TRY(cudaGetLastError(), "feature statistics kernel");
    standardize_kernel<<<1024, 256, 0, st>>>(s->n_rec, s->width, s->desc, s->mu, s->sd, s->x_std);
    LEEA_CUDA_TRY(cudaGetLastError(), "standardize kernel");
    LEEA_CUDA_TRY(launch_surrogate_forward(s->n_rec, s->width, s->sp.hidden1, s->sp.hidden2, s->theta, s->x_std,
                                           s->pred, nullptr, nullptr, st),
                  "surrogate forward");
    LEEA_CUDA_TRY(launch_rank(s->n_rec, s->pred, s->order_r, st), "rank kernel");
    ChooseArgs ca{};
    ca.pop = s->pop;
    ca.n_elite = s->n_elite;
    ca.n_cross = s->n_cross;
    ca.n_mut = s->n_mut;
    ca.mult = s->sp.mult;
    ca.n_rec = s->n_rec;
    ca.n_audit = s->n_audit;
    ca.order = s->order;
    ca.f_adj = s->f_adj;
    ca.order_r = s->order_r;
    ca.use_screen = s->use_screen;
    ca.r_par1 = s->r_par1;
    ca.r_par2 = s->r_par2;
    ca.r_kind = s->r_kind;
    ca.r_f_inh = s->r_f_inh;
    ca.r_entity = s->r_entity;
    ca.c_par1 = s->c_par1;
    ca.c_par2 = s->c_par2;
    ca.c_kind = s->c_kind;
    ca.c_f_inh = s->c_f_inh;
    ca.c_entity = s->c_entity;
    ca.a_par1 = s->a_par1;
    ca.a_par2 = s->a_par2;
    ca.a_kind = s->a_kind;
    ca.a_entity = s->a_entity;
    ca.row_recipe = s->row_recipe;
    ca.amax_c = s->prm.precision ? s->amax[s->cur ^ 1] : nullptr;
    ca.amax_a = s->prm.precision ? s->a_amax : nullptr;
    choose_kernel<<<(s->pop + s->n_audit + 255) / 256, 256, 0, st>>>(ca);
    LEEA_CUDA_TRY(cudaGetLastError(), "choose kernel");
    mark(s, 1, 1);
    // 3. the chosen offspring and the audit sample are made
    mark(s, 2, 0);
    BreedArgs ba = surr_breed_args(s, s->pop, s->c_entity, s->shadow[s->cur ^ 1], s->amax[s->cur ^ 1]);
    LEEA_CUDA_TRY(launch_breed(ba, s->popbuf[s->cur], s->c_par1, s->c_par2, s->c_kind, s->popbuf[s->cur ^ 1], status,
                               st),
                  "breed kernel");
    if (s->n_audit > 0) {
        BreedArgs aa = surr_breed_args(s, s->n_audit, s->a_entity, s->a_shadow, s->a_amax);
        LEEA_CUDA_TRY(launch_breed(aa, s->popbuf[s->cur], s->a_par1, s->a_par2, s->a_kind, s->a_pop, status, st),
                      "breed kernel (audit)");
    }
    mark(s, 2, 1);
    // 4. evaluation
    mark(s, 3, 0);
    leea_status es = LEEA_OK;
    evaluate(s, s->popbuf[s->cur ^ 1], s->shadow[s->cur ^ 1], s->pop, x, x_div, y, batch, s->c_f_inh, s->f_raw,
             s->f_adj, s->correct, &es);
    if (es) return es;
    if (s->n_audit > 0) {
        evaluate(s, s->a_pop, s->a_shadow, s->n_audit, x, x_div, y, batch, nullptr, s->a_f, nullptr, nullptr, &es);
        if (es) return es;
    }
    mark(s, 3, 1);
    // 5. audit and training
    mark(s, 4, 0);
    const int64_t slot = s->breeds % s->sp.history;
    float* x_slot = s->x_hist + slot * s->rows * s->width;
    float* t_slot = s->t_hist + slot * s->rows;
    targets_kernel<<<1, 256, 0, st>>>(s->rows, s->k, s->n_elite, s->f_raw, s->a_f, s->pred, s->row_recipe, s->meas,
                                      s->pred_rows, t_slot);
    const int64_t stat_i = s->breeds < s->stats_cap ? s->breeds : s->stats_cap - 1;
    LEEA_CUDA_TRY(launch_rank(s->rows, s->pred_rows, s->rank_p, st), "rank kernel");
    LEEA_CUDA_TRY(launch_rank(s->rows, s->meas, s->rank_m, st), "rank kernel");
    audit_kernel<<<1, 1024, 0, st>>>(s->rows, s->rank_p, s->rank_m, s->rank_tmp, s->stats + 3 * stat_i,
                                     s->use_screen, static_cast<int32_t>(g) >= s->sp.warmup ? 1 : 0,
                                     s->sp.min_spearman);
    gather_rows_kernel<<<s->rows, 128, 0, st>>>(s->rows, s->width, s->row_recipe, s->x_std, x_slot);
    LEEA_CUDA_TRY(cudaGetLastError(), "audit kernels");
    const int64_t filled = (s->breeds + 1 < s->sp.history ? s->breeds + 1 : s->sp.history) * s->rows;
    for (int32_t step = 0; step < s->sp.train_steps; ++step) {
        const int64_t off = (static_cast<int64_t>(step) * s->sp.train_batch) % filled;
        const int32_t n = static_cast<int32_t>(filled - off < s->sp.train_batch ? filled - off : s->sp.train_batch);
        const bool last = step + 1 == s->sp.train_steps;  // the recorded loss is the last step's
        LEEA_CUDA_TRY(launch_surrogate_train_step(n, s->width, s->sp.hidden1, s->sp.hidden2, s->theta,
                                                  s->x_hist + off * s->width, s->t_hist + off,
                                                  last ? s->loss : nullptr, s->work, s->adam_m, s->adam_v,
                                                  ++s->adam_step, s->sp.lr, 0.9f, 0.999f, 1e-8f, st),
                      "surrogate training step");
    }
    if (s->sp.train_steps > 0)
        LEEA_CUDA_TRY(cudaMemcpyAsync(s->stats + 3 * stat_i + 2, s->loss, sizeof(float), cudaMemcpyDeviceToDevice, st),
                      "loss copy");
    mark(s, 4, 1);
    if (s->profiling) s->n_prof++;
    s->breeds++;
    s->cur ^= 1;
    s->gen = g;
    return LEEA_OK;
}

leea_status check_surr(leea_surr* s)
{
    if (!s) return fail(LEEA_EINVAL, "surrogate object is NULL");
    return LEEA_OK;
}

}  // namespace

extern "C" {

leea_status leea_surrogate_default_params(leea_surrogate_params* out)
{
    if (!out) return fail(LEEA_EINVAL, "out is NULL");
    out->mult = 4;
    out->n_probe = 32;
    out->hidden1 = 64;
    out->hidden2 = 64;
    out->train_steps = 16;
    out->train_batch = 256;
    out->history = 4;
    out->warmup = 3;
    out->lr = 1e-3f;
    out->audit_frac = 0.05f;
    out->min_spearman = 0.2f;
    out->seed = 0x5EED5EEDull;
    return LEEA_OK;
}

leea_status leea_surr_create(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_params* p,
                             const leea_surrogate_params* sp, uint64_t seed, const float* probe_host, void* stream,
                             leea_surr** out)
{
    if (!out) return fail(LEEA_EINVAL, "out is NULL");
    *out = nullptr;
    leea_status st = check_pop(pop);
    if (st) return st;
    if ((st = check_params(p))) return st;
    if (!sp || !probe_host) return fail(LEEA_EINVAL, "surrogate params and probe inputs are required");
    if (p->precision != 0 && p->precision != 1)
        return fail(LEEA_EINVAL, "the surrogate form evaluates in FP32 (precision 0) or BF16 (precision 1)");
    if ((st = require_const_sigma(p, "the surrogate form"))) return st;
    if (sp->mult < 1 || sp->n_probe < 1 || sp->n_probe > 32 || sp->hidden1 < 1 || sp->hidden1 > 256 ||
        sp->hidden2 < 1 || sp->hidden2 > 256 || sp->train_steps < 0 || sp->train_batch < 1 || sp->history < 1 ||
        sp->warmup < 0 || !(sp->lr > 0.0f) || !(sp->audit_frac >= 0.0f && sp->audit_frac <= 1.0f))
        return fail(LEEA_EINVAL, "invalid surrogate parameters");
    leea_surr* s = new (std::nothrow) leea_surr();
    if (!s) return fail(LEEA_ENOMEM, "host allocation failed");
    if (!make_layout(dims, n_dims, p->init, &s->net) || s->net.n_layers != 2 ||
        !probe_supported(s->net.dims[0], s->net.dims[1], s->net.dims[2], sp->n_probe, p->precision) ||
        (p->precision == 1 && check_shadow_shape(s->net, 1))) {
        delete s;
        return fail(LEEA_EINVAL, "the surrogate form needs d_0-h-d_out nets with d_0 %% 16 == 0, h %% 16 == 0, "
                                 "16 <= h <= 256 (<= 128 in BF16), d_out <= 16");
    }
    s->pop = pop;
    s->prm = *p;
    s->sp = *sp;
    s->seed = seed;
    s->stream = static_cast<cudaStream_t>(stream);
    int32_t pool;
    counts_of(pop, p, &s->n_elite, &s->n_cross, &s->n_mut, &pool);
    s->k = pop - s->n_elite;
    s->n_rec = sp->mult * s->k;
    s->n_audit = sp->mult > 1 ? static_cast<int32_t>(std::lround(sp->audit_frac * (s->n_rec - s->k))) : 0;
    if (s->n_audit > s->n_rec - s->k) s->n_audit = s->n_rec - s->k;
    s->rows = s->k + s->n_audit;
    s->width = 5 + sp->n_probe * s->net.dims[2];
    s->n_theta = surrogate_num_params(s->width, sp->hidden1, sp->hidden2);
    s->stats_cap = 1 << 16;
    if (surrogate_forward_smem(s->width, sp->hidden1, sp->hidden2) > 227u * 1024u || s->rows < 1) {
        free_surr(s);
        return fail(LEEA_EINVAL, "surrogate shape not supported (or no offspring to make)");
    }
    const size_t np = static_cast<size_t>(pop), cp = static_cast<size_t>(s->net.c_pad);
    cudaError_t err = cudaSuccess;
    for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = alloc(&s->popbuf[b], np * cp);
    if (p->precision == 1) {
        s->sh_stride = shadow_stride_of(s->net, 1);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = alloc(&s->shadow[b], np * s->sh_stride);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = alloc(&s->amax[b], np);
        if (err == cudaSuccess) err = alloc(&s->a_shadow, static_cast<size_t>(s->n_audit) * s->sh_stride);
        if (err == cudaSuccess) err = alloc(&s->a_amax, static_cast<size_t>(s->n_audit));
    }
    const size_t nr = static_cast<size_t>(s->n_rec), na = static_cast<size_t>(s->n_audit);
    if (err == cudaSuccess) err = alloc(&s->f_adj, np);
    if (err == cudaSuccess) err = alloc(&s->f_raw, np);
    if (err == cudaSuccess) err = alloc(&s->correct, np);
    if (err == cudaSuccess) err = alloc(&s->order, np);
    if (err == cudaSuccess) err = alloc(&s->c_par1, np);
    if (err == cudaSuccess) err = alloc(&s->c_par2, np);
    if (err == cudaSuccess) err = alloc(&s->c_kind, np);
    if (err == cudaSuccess) err = alloc(&s->c_f_inh, np);
    if (err == cudaSuccess) err = alloc(&s->c_entity, np);
    if (err == cudaSuccess) err = alloc(&s->r_par1, nr);
    if (err == cudaSuccess) err = alloc(&s->r_par2, nr);
    if (err == cudaSuccess) err = alloc(&s->r_kind, nr);
    if (err == cudaSuccess) err = alloc(&s->order_r, nr);
    if (err == cudaSuccess) err = alloc(&s->r_f_inh, nr);
    if (err == cudaSuccess) err = alloc(&s->r_entity, nr);
    if (err == cudaSuccess) err = alloc(&s->pred, nr);
    if (err == cudaSuccess) err = alloc(&s->desc, nr * s->width);
    if (err == cudaSuccess) err = alloc(&s->x_std, nr * s->width);
    if (err == cudaSuccess) err = alloc(&s->a_par1, na);
    if (err == cudaSuccess) err = alloc(&s->a_par2, na);
    if (err == cudaSuccess) err = alloc(&s->a_kind, na);
    if (err == cudaSuccess) err = alloc(&s->a_entity, na);
    if (err == cudaSuccess) err = alloc(&s->a_pop, na * cp);
    if (err == cudaSuccess) err = alloc(&s->a_f, na);
    if (err == cudaSuccess) err = alloc(&s->theta, static_cast<size_t>(s->n_theta));
    if (err == cudaSuccess) err = alloc(&s->adam_m, static_cast<size_t>(s->n_theta));
    if (err == cudaSuccess) err = alloc(&s->adam_v, static_cast<size_t>(s->n_theta));
    if (err == cudaSuccess) err = alloc(&s->grad, static_cast<size_t>(s->n_theta));
    if (err == cudaSuccess) err = alloc(&s->work, surrogate_work_floats(sp->train_batch, sp->hidden1, sp->hidden2));
    if (err == cudaSuccess) err = alloc(&s->loss, 1);
    if (err == cudaSuccess) err = alloc(&s->mu, static_cast<size_t>(s->width));
    if (err == cudaSuccess) err = alloc(&s->sd, static_cast<size_t>(s->width));
    if (err == cudaSuccess) err = alloc(&s->probe, static_cast<size_t>(sp->n_probe) * s->net.dims[0]);
    if (err == cudaSuccess) err = alloc(&s->x_hist, static_cast<size_t>(sp->history) * s->rows * s->width);
    if (err == cudaSuccess) err = alloc(&s->t_hist, static_cast<size_t>(sp->history) * s->rows);
    if (err == cudaSuccess) err = alloc(&s->meas, static_cast<size_t>(s->rows));
    if (err == cudaSuccess) err = alloc(&s->pred_rows, static_cast<size_t>(s->rows));
    if (err == cudaSuccess) err = alloc(&s->row_recipe, static_cast<size_t>(s->rows));
    if (err == cudaSuccess) err = alloc(&s->rank_p, static_cast<size_t>(s->rows));
    if (err == cudaSuccess) err = alloc(&s->rank_m, static_cast<size_t>(s->rows));
    if (err == cudaSuccess) err = alloc(&s->rank_tmp, static_cast<size_t>(s->rows));
    if (err == cudaSuccess) err = alloc(&s->use_screen, 1);
    if (err == cudaSuccess) err = alloc(&s->stats, static_cast<size_t>(3 * s->stats_cap));
    if (err != cudaSuccess) {
        free_surr(s);
        return cuda_fail(err, "leea_surr_create allocation");
    }
    const cudaStream_t cs = s->stream;
    err = cudaMemsetAsync(s->popbuf[1], 0, sizeof(float) * np * cp, cs);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->a_pop, 0, sizeof(float) * (na > 0 ? na : 1) * cp, cs);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->adam_m, 0, sizeof(float) * s->n_theta, cs);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->adam_v, 0, sizeof(float) * s->n_theta, cs);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->use_screen, 0, sizeof(int32_t), cs);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->stats, 0, sizeof(float) * 3 * s->stats_cap, cs);
    if (err == cudaSuccess && p->precision == 1) {
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = cudaMemsetAsync(s->shadow[b], 0, np * s->sh_stride, cs);
        if (err == cudaSuccess) err = cudaMemsetAsync(s->a_shadow, 0, (na > 0 ? na : 1) * s->sh_stride, cs);
    }
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(s->probe, probe_host, sizeof(float) * sp->n_probe * s->net.dims[0],
                              cudaMemcpyHostToDevice, cs);
    if (err == cudaSuccess) err = launch_init(s->net, pop, p->init, seed, s->popbuf[0], cs);
    if (err == cudaSuccess && p->precision == 1)
        err = launch_make_shadow(pop, s->net.dims[0], s->net.dims[1], s->net.c_pad, s->popbuf[0], 1, s->shadow[0],
                                 s->sh_stride, nullptr, s->amax[0], cs);
    if (err == cudaSuccess) err = launch_surrogate_init(s->width, sp->hidden1, sp->hidden2, sp->seed, s->theta, cs);
    if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
    if (err != cudaSuccess) {
        free_surr(s);
        return cuda_fail(err, "leea_surr_create setup");
    }
    *out = s;
    return LEEA_OK;
}

leea_status leea_surr_generation_u8(leea_surr* s, const uint8_t* x_dev, float x_div, const int32_t* y_dev,
                                    int32_t batch)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (!x_dev || !y_dev || batch < 1) return fail(LEEA_EINVAL, "NULL minibatch pointer or batch < 1");
    if (!(x_div > 0.0f) || std::isinf(x_div)) return fail(LEEA_EINVAL, "x_div must be finite and > 0");
    if (s->prm.precision == 1) {
        if (reinterpret_cast<uintptr_t>(x_dev) & 15u) return fail(LEEA_EINVAL, "x must be 16-byte aligned");
        const size_t need = eval_shadow_scratch_bytes(s->pop > s->n_audit ? s->pop : s->n_audit, batch);
        if (need > s->scratch_bytes) {
            LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "scratch sync");
            cudaFree(s->scratch);
            s->scratch = nullptr;
            s->scratch_bytes = 0;
            LEEA_CUDA_TRY(cudaMalloc(&s->scratch, need), "scratch allocation");
            s->scratch_bytes = need;
        }
    }
    if (!s->evaluated) {
        leea_status es = LEEA_OK;
        evaluate(s, s->popbuf[s->cur], s->shadow[s->cur], s->pop, x_dev, x_div, y_dev, batch, nullptr, s->f_raw,
                 s->f_adj, s->correct, &es);
        if (es) return es;
        s->evaluated = true;
        return LEEA_OK;
    }
    return surr_breed_generation(s, x_dev, x_div, y_dev, batch);
}

leea_status leea_surr_generation_u8_host(leea_surr* s, const uint8_t* x_host, float x_div, const int32_t* y_host,
                                         int32_t batch)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (!x_host || !y_host || batch < 1) return fail(LEEA_EINVAL, "NULL minibatch pointer or batch < 1");
    const size_t xb = static_cast<size_t>(batch) * s->net.dims[0];
    if (xb > s->x_stage_bytes || batch > s->y_stage_cap) {
        LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "staging sync");
        cudaFree(s->x_stage);
        cudaFree(s->y_stage);
        s->x_stage = nullptr;
        s->y_stage = nullptr;
        s->x_stage_bytes = 0;
        s->y_stage_cap = 0;
        LEEA_CUDA_TRY(cudaMalloc(&s->x_stage, xb), "staging allocation");
        LEEA_CUDA_TRY(cudaMalloc(&s->y_stage, sizeof(int32_t) * batch), "staging allocation");
        s->x_stage_bytes = xb;
        s->y_stage_cap = batch;
    }
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->x_stage, x_host, xb, cudaMemcpyHostToDevice, s->stream), "minibatch copy");
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->y_stage, y_host, sizeof(int32_t) * batch, cudaMemcpyHostToDevice, s->stream),
                  "label copy");
    return leea_surr_generation_u8(s, s->x_stage, x_div, s->y_stage, batch);
}

leea_status leea_surr_fitness(leea_surr* s, float* f_adj_host, int32_t* correct_host)
{
    leea_status st = check_surr(s);
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

leea_status leea_surr_raw_fitness(leea_surr* s, float* f_raw_host, float* f_audit_host)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (!s->evaluated) return fail(LEEA_ESTATE, "no generation has been evaluated yet");
    if (f_raw_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(f_raw_host, s->f_raw, sizeof(float) * s->pop, cudaMemcpyDeviceToHost, s->stream),
                      "fitness copy");
    if (f_audit_host && s->n_audit > 0)
        LEEA_CUDA_TRY(cudaMemcpyAsync(f_audit_host, s->a_f, sizeof(float) * s->n_audit, cudaMemcpyDeviceToHost,
                                      s->stream),
                      "audit fitness copy");
    return check_device_status(s->stream, nullptr);
}

leea_status leea_surr_get_population(leea_surr* s, float* out_host)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (!out_host) return fail(LEEA_EINVAL, "out_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpy2DAsync(out_host, sizeof(float) * s->net.c, s->popbuf[s->cur], sizeof(float) * s->net.c_pad,
                                    sizeof(float) * s->net.c, s->pop, cudaMemcpyDeviceToHost, s->stream),
                  "population copy");
    return check_device_status(s->stream, nullptr);
}

leea_status leea_surr_set_population(leea_surr* s, const float* in_host)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (!in_host) return fail(LEEA_EINVAL, "in_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpy2DAsync(s->popbuf[s->cur], sizeof(float) * s->net.c_pad, in_host, sizeof(float) * s->net.c,
                                    sizeof(float) * s->net.c, s->pop, cudaMemcpyHostToDevice, s->stream),
                  "population copy");
    if (s->prm.precision == 1)
        LEEA_CUDA_TRY(launch_make_shadow(s->pop, s->net.dims[0], s->net.dims[1], s->net.c_pad, s->popbuf[s->cur], 1,
                                         s->shadow[s->cur], s->sh_stride, nullptr, s->amax[s->cur], s->stream),
                      "make shadow kernel");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "population sync");
    return LEEA_OK;
}

leea_status leea_surr_set_fitness(leea_surr* s, const float* f_adj_host)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (!f_adj_host) return fail(LEEA_EINVAL, "f_adj_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->f_adj, f_adj_host, sizeof(float) * s->pop, cudaMemcpyHostToDevice, s->stream),
                  "fitness copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "fitness sync");
    return LEEA_OK;
}

leea_status leea_surr_set_generation(leea_surr* s, uint32_t gen, int32_t evaluated)
{
    leea_status st = check_surr(s);
    if (st) return st;
    s->gen = gen;
    s->evaluated = evaluated != 0;
    return LEEA_OK;
}

leea_status leea_surr_set_screen(leea_surr* s, int32_t use_screen)
{
    leea_status st = check_surr(s);
    if (st) return st;
    const int32_t v = use_screen ? 1 : 0;
    LEEA_CUDA_TRY(cudaMemcpyAsync(s->use_screen, &v, sizeof(int32_t), cudaMemcpyHostToDevice, s->stream), "flag copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(s->stream), "flag sync");
    return LEEA_OK;
}

leea_status leea_surr_layout(const leea_surr* s, int32_t* n_recipes, int32_t* n_audit, int32_t* width,
                             int64_t* n_theta)
{
    if (!s) return fail(LEEA_EINVAL, "surrogate object is NULL");
    if (n_recipes) *n_recipes = s->n_rec;
    if (n_audit) *n_audit = s->n_audit;
    if (width) *width = s->width;
    if (n_theta) *n_theta = s->n_theta;
    return LEEA_OK;
}

leea_status leea_surr_get_step(leea_surr* s, int32_t* r_par1, int32_t* r_par2, int32_t* r_kind, float* r_f_inh,
                               uint32_t* r_entity, float* desc, float* pred, int32_t* row_recipe, int32_t* c_par1,
                               int32_t* c_par2, int32_t* c_kind, uint32_t* c_entity, float* c_f_inh)
{
    leea_status st = check_surr(s);
    if (st) return st;
    struct Cp { void* dst; const void* src; size_t bytes; } cps[] = {
        { r_par1, s->r_par1, sizeof(int32_t) * s->n_rec },   { r_par2, s->r_par2, sizeof(int32_t) * s->n_rec },
        { r_kind, s->r_kind, sizeof(int32_t) * s->n_rec },   { r_f_inh, s->r_f_inh, sizeof(float) * s->n_rec },
        { r_entity, s->r_entity, sizeof(uint32_t) * s->n_rec },
        { desc, s->desc, sizeof(float) * s->n_rec * s->width }, { pred, s->pred, sizeof(float) * s->n_rec },
        { row_recipe, s->row_recipe, sizeof(int32_t) * s->rows }, { c_par1, s->c_par1, sizeof(int32_t) * s->pop },
        { c_par2, s->c_par2, sizeof(int32_t) * s->pop },     { c_kind, s->c_kind, sizeof(int32_t) * s->pop },
        { c_entity, s->c_entity, sizeof(uint32_t) * s->pop }, { c_f_inh, s->c_f_inh, sizeof(float) * s->pop } };
    for (const Cp& c : cps)
        if (c.dst)
            LEEA_CUDA_TRY(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, s->stream), "step copy");
    return check_device_status(s->stream, nullptr);
}

leea_status leea_surr_get_surrogate(leea_surr* s, float* theta_host, float* mu_host, float* sd_host)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (theta_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(theta_host, s->theta, sizeof(float) * s->n_theta, cudaMemcpyDeviceToHost,
                                      s->stream),
                      "surrogate copy");
    if (mu_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(mu_host, s->mu, sizeof(float) * s->width, cudaMemcpyDeviceToHost, s->stream),
                      "feature mean copy");
    if (sd_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(sd_host, s->sd, sizeof(float) * s->width, cudaMemcpyDeviceToHost, s->stream),
                      "feature sd copy");
    return check_device_status(s->stream, nullptr);
}

leea_status leea_surr_stats(leea_surr* s, int64_t n_max, float* spearman, int32_t* screened, float* loss,
                            int64_t* n_out)
{
    leea_status st = check_surr(s);
    if (st) return st;
    const int64_t n = s->breeds < s->stats_cap ? s->breeds : s->stats_cap;
    const int64_t m = n < n_max ? n : n_max;
    if (n_out) *n_out = m;
    if (m <= 0) return LEEA_OK;
    std::vector<float> buf(static_cast<size_t>(3 * m));
    LEEA_CUDA_TRY(cudaMemcpyAsync(buf.data(), s->stats + 3 * (n - m), sizeof(float) * 3 * m, cudaMemcpyDeviceToHost,
                                  s->stream),
                  "stats copy");
    if ((st = check_device_status(s->stream, nullptr))) return st;
    for (int64_t i = 0; i < m; ++i) {
        if (spearman) spearman[i] = buf[3 * i];
        if (screened) screened[i] = buf[3 * i + 1] != 0.0f ? 1 : 0;
        if (loss) loss[i] = buf[3 * i + 2];
    }
    return LEEA_OK;
}

leea_status leea_surr_best_params(leea_surr* s, float* out_host, int64_t c)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (!s->evaluated) return fail(LEEA_ESTATE, "no generation has been evaluated yet");
    if (!out_host || c != s->net.c) return fail(LEEA_EINVAL, "out_host NULL or c != %lld", (long long)s->net.c);
    std::vector<float> f(static_cast<size_t>(s->pop));
    LEEA_CUDA_TRY(cudaMemcpyAsync(f.data(), s->f_adj, sizeof(float) * s->pop, cudaMemcpyDeviceToHost, s->stream),
                  "fitness copy");
    if ((st = check_device_status(s->stream, nullptr))) return st;
    int32_t best = 0;  // highest f_adj, NaN as -infinity, ties to the lower index
    for (int32_t p = 1; p < s->pop; ++p) {
        const float a = std::isnan(f[p]) ? -INFINITY : f[p], b = std::isnan(f[best]) ? -INFINITY : f[best];
        if (a > b) best = p;
    }
    LEEA_CUDA_TRY(cudaMemcpyAsync(out_host, s->popbuf[s->cur] + static_cast<int64_t>(best) * s->net.c_pad,
                                  sizeof(float) * static_cast<size_t>(c), cudaMemcpyDeviceToHost, s->stream),
                  "best params copy");
    return check_device_status(s->stream, nullptr);
}

uint32_t leea_surr_generation_index(const leea_surr* s) { return s ? s->gen : 0u; }

leea_status leea_surr_profile_enable(leea_surr* s, int32_t enable)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if (enable && s->ev.empty()) {
        s->ev.resize(static_cast<size_t>(kSurrStages) * 2 * kSurrProfRing, nullptr);
        for (cudaEvent_t& e : s->ev) LEEA_CUDA_TRY(cudaEventCreate(&e), "event create");
    }
    if (!enable && s->profiling && (st = fold_profile(s))) return st;
    s->profiling = enable != 0;
    return LEEA_OK;
}

leea_status leea_surr_profile_read(leea_surr* s, double* ms_out, int64_t* generations_out)
{
    leea_status st = check_surr(s);
    if (st) return st;
    if ((st = fold_profile(s))) return st;
    for (int i = 0; i < kSurrStages; ++i) {
        if (ms_out) ms_out[i] = s->ms[i];
        s->ms[i] = 0.0;
    }
    if (generations_out) *generations_out = s->launches;
    s->launches = 0;
    return LEEA_OK;
}

void leea_surr_destroy(leea_surr* s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    free_surr(s);
}

}  // extern "C"
