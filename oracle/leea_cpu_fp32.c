/*
 * leea_cpu_fp32.c -- a multi-core FP32 CPU implementation of one LEEA
 * generation (Algorithm 1; Sections 3.1-3.3): the CPU baseline the GPU
 * throughput is reported beside.
 *
 * TEST INFRASTRUCTURE ONLY, like the oracle it sits beside: only the test
 * suite and the benchmark's CPU-baseline leg may load it.  It shares nothing
 * with the CUDA library.  Ranking and selection are the oracle's own
 * functions (negligible work); breeding and evaluation are restated here in
 * single precision, blocked for the caches and spread over OpenMP threads
 * (children, then individuals), so that the baseline is a reasonable CPU
 * program rather than the deliberately plain oracle.  Random numbers follow
 * the same Philox contract (the oracle's block function, one block per 8
 * mask draws or per two Box-Muller pairs), so the children match the
 * oracle's up to FP32 rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "leea_oracle.h"

/* Threads this library runs with (1 without OpenMP). */
int leea_cpu32_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void block_of(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t blk, uint32_t out[4])
{
    const uint32_t ctr[4] = { blk, ent, gen, tag };
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    leea_cpu_philox(ctr, key, out);
}

/* 16-bit draw k (0..7) of a block: half k & 1 of word k >> 1. */
static uint32_t draw16_of(const uint32_t w[4], int k)
{
    return (k & 1) ? (w[k >> 1] >> 16) : (w[k >> 1] & 0xFFFFu);
}

/* Normals of genes 8u + 2s, 8u + 2s + 1 (pair s of the unit): radius from
 * the first word of the pair, angle from the second. */
static void pair_normals(uint64_t seed, uint32_t gen, uint32_t ent, uint32_t u, int s, float z[2])
{
    uint32_t w[4];
    block_of(seed, LEEA_CPU_TAG_NORMAL, gen, ent, 2u * u + (uint32_t)(s >> 1), w);
    const uint32_t ua = (s & 1) ? w[2] : w[0], ub = (s & 1) ? w[3] : w[1];
    const float r = sqrtf(-2.0f * logf((float)leea_cpu_u01(ua)));
    const float t = 6.283185307179586f * (float)leea_cpu_u01(ub);
    z[0] = r * cosf(t);
    z[1] = r * sinf(t);
}

static void breed_child32(int64_t c, const leea_cpu_params* prm, uint64_t seed, uint32_t gen, uint32_t ent,
                          int32_t kind, const float* a, const float* b, float* out)
{
    const uint32_t thr_xo = leea_cpu_threshold16((double)prm->xo_gene_p);
    const uint32_t thr_mut = leea_cpu_threshold16((double)prm->mut_rate);
    const float sigma = prm->sigma;
    if (kind == LEEA_CPU_ELITE) {
        memcpy(out, a, sizeof(float) * (size_t)c);
        return;
    }
    if (kind == LEEA_CPU_CROSSOVER && prm->xo_op != 0) {
        for (int64_t i = 0; i < c; i++) out[i] = 0.5f * (a[i] + b[i]);
        return;
    }
    for (int64_t i0 = 0; i0 < c; i0 += 8) {
        const uint32_t u = (uint32_t)(i0 >> 3);
        uint32_t w[4];
        const int n = (int)(c - i0 < 8 ? c - i0 : 8);
        if (kind == LEEA_CPU_CROSSOVER) {
            block_of(seed, LEEA_CPU_TAG_XO, gen, ent, u, w);
            for (int k = 0; k < n; k++) out[i0 + k] = draw16_of(w, k) < thr_xo ? b[i0 + k] : a[i0 + k];
        } else {
            block_of(seed, LEEA_CPU_TAG_MUTMASK, gen, ent, u, w);
            float z[4][2];
            int have = 0;
            for (int k = 0; k < n; k++) {
                float v = a[i0 + k];
                if (draw16_of(w, k) < thr_mut) {
                    const int s = k >> 1;
                    if (!(have & (1 << s))) {
                        pair_normals(seed, gen, ent, u, s, z[s]);
                        have |= 1 << s;
                    }
                    v = a[i0 + k] + sigma * z[s][k & 1];
                }
                out[i0 + k] = v;
            }
        }
    }
}

/* Fitness (Eq. 1) of one individual of a dims[0]-h-d_out net, FP32: per four
 * samples, each hidden unit's row of W1 is read once. */
static float evaluate32(const int32_t* dims, const float* theta, const float* x, const int32_t* y, int32_t batch,
                        float* hid, int32_t* correct)
{
    const int32_t k = dims[0], h = dims[1], d_out = dims[2];
    const float* w1 = theta;
    const float* b1 = w1 + (int64_t)h * k;
    const float* w2 = b1 + h;
    const float* b2 = w2 + (int64_t)d_out * h;
    double loss_sum = 0.0;
    int32_t good = 0;
    for (int32_t b0 = 0; b0 < batch; b0 += 4) {
        const int nb = batch - b0 < 4 ? batch - b0 : 4;
        for (int32_t o = 0; o < h; o++) {
            const float* wr = w1 + (int64_t)o * k;
            float acc[4] = { 0.f, 0.f, 0.f, 0.f };
            for (int s = 0; s < nb; s++) {
                const float* xr = x + (int64_t)(b0 + s) * k;
                float t = 0.f;
                for (int32_t i = 0; i < k; i++) t += wr[i] * xr[i];
                acc[s] = t;
            }
            for (int s = 0; s < nb; s++) {
                const float v = acc[s] + b1[o];
                hid[s * h + o] = v > 0.f ? v : 0.f;
            }
        }
        for (int s = 0; s < nb; s++) {
            float z[64];
            for (int32_t j = 0; j < d_out; j++) {
                float t = b2[j];
                for (int32_t o = 0; o < h; o++) t += w2[(int64_t)j * h + o] * hid[s * h + o];
                z[j] = t;
            }
            float zmax = z[0];
            int32_t arg = 0;
            for (int32_t j = 1; j < d_out; j++)
                if (z[j] > zmax) { zmax = z[j]; arg = j; }
            float se = 0.f;
            for (int32_t j = 0; j < d_out; j++) se += expf(z[j] - zmax);
            const int32_t lbl = y[b0 + s];
            loss_sum += (double)(logf(se) + zmax - z[lbl]);
            if (arg == lbl) good++;
        }
    }
    *correct = good;
    return (float)(-loss_sum / (double)batch);
}

/* One generation: rank and select from f_adj (the oracle's functions), breed
 * every child from `parents` into `children`, evaluate them on (x, y) and
 * blend the inherited fitness (Section 3.1).  Nets d_0-h-d_out (n_dims 3,
 * d_out <= 64); populations float[pop][c] in the logical gene order.  Returns
 * LEEA_CPU_OK or an error code; *threads gets the OpenMP threads used. */
int leea_cpu32_generation(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_cpu_params* prm,
                          uint64_t seed, uint32_t gen, const float* parents, const float* f_adj_in, const float* x,
                          const int32_t* y, int32_t batch, float* children, float* f_raw, float* f_adj_out,
                          int32_t* correct, int32_t* threads)
{
    if (n_dims != 3 || dims[2] > 64 || pop <= 0 || batch <= 0 || !parents || !f_adj_in || !x || !y || !children ||
        !f_raw || !f_adj_out || !correct)
        return LEEA_CPU_EINVAL;
    const int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0) return LEEA_CPU_EINVAL;
    double* f64 = (double*)malloc(sizeof(double) * (size_t)pop);
    double* f_inh = (double*)malloc(sizeof(double) * (size_t)pop);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)pop);
    int32_t* p1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)pop);
    int32_t* p2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)pop);
    int32_t* kind = (int32_t*)malloc(sizeof(int32_t) * (size_t)pop);
    int rc = (f64 && f_inh && order && p1 && p2 && kind) ? LEEA_CPU_OK : LEEA_CPU_ENOMEM;
    if (rc == LEEA_CPU_OK) {
        for (int32_t p = 0; p < pop; p++) f64[p] = (double)f_adj_in[p];
        rc = leea_cpu_rank(pop, f64, order);
    }
    if (rc == LEEA_CPU_OK) rc = leea_cpu_select(pop, prm, f64, order, seed, gen, p1, p2, kind, f_inh);
    if (rc == LEEA_CPU_OK) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int32_t j = 0; j < pop; j++)
            breed_child32(c, prm, seed, gen, (uint32_t)j, kind[j], parents + (int64_t)p1[j] * c,
                          parents + (int64_t)p2[j] * c, children + (int64_t)j * c);
        const float alpha = prm->alpha;
#pragma omp parallel
        {
            float* hid = (float*)malloc(sizeof(float) * 4u * (size_t)dims[1]);
#pragma omp for schedule(dynamic, 1)
            for (int32_t j = 0; j < pop; j++) {
                if (!hid) continue;
                const float f = evaluate32(dims, children + (int64_t)j * c, x, y, batch, hid, correct + j);
                f_raw[j] = f;
                f_adj_out[j] = (1.0f - alpha) * (float)f_inh[j] + alpha * f;
            }
            free(hid);
        }
    }
    if (threads) *threads = leea_cpu32_threads();
    free(f64);
    free(f_inh);
    free(order);
    free(p1);
    free(p2);
    free(kind);
    return rc;
}
