/*
 * leea_oracle.c -- FP64 CPU oracle of the LEEA hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see leea_oracle.h).  Plain, slow and written to
 * be checked against the paper by eye: every loop follows the definition it
 * cites, in the order the paper gives, with no blocking or fusion.
 */
#include "leea_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 bit     */
/* multiplies, xor with the other counter words and the round key, and a    */
/* Weyl-sequence bump of the key between rounds.                             */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void leea_cpu_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void stream_block(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                         uint32_t block, uint32_t out[4])
{
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { block, ent, gen, tag };
    leea_cpu_philox(ctr, key, out);
}

/* Scalar draw n of the stream (tag, generation, entity). */
uint32_t leea_cpu_draw(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t n)
{
    uint32_t w[4];
    stream_block(seed, tag, gen, ent, n >> 2, w);
    return w[n & 3u];
}

/* Open-interval uniform from the top 23 bits: (2k + 1) / 2^24, k = u >> 9.
 * Exact in both float and double; never 0, never 1. */
double leea_cpu_u01(uint32_t u)
{
    return (double)((u >> 9) * 2u + 1u) * (1.0 / 16777216.0);
}

/* Standard normal for gene i by the Box-Muller transform: the block i >> 2
 * carries two pairs (words 0,1 and 2,3); the first word of a pair gives the
 * radius, the second the angle; even genes take the cosine, odd the sine. */
double leea_cpu_normal(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t i)
{
    uint32_t w[4];
    stream_block(seed, tag, gen, ent, i >> 2, w);
    uint32_t pair = (i & 3u) >> 1;
    double u1 = leea_cpu_u01(w[2 * pair]);
    double u2 = leea_cpu_u01(w[2 * pair + 1]);
    double r = sqrt(-2.0 * log(u1));
    const double two_pi = 6.283185307179586476925286766559;
    return (i & 1u) ? r * sin(two_pi * u2) : r * cos(two_pi * u2);
}

/* Uniform index in [0, m): floor(u * m / 2^32), multiply-shift without
 * rejection. */
uint32_t leea_cpu_index(uint32_t u, uint32_t m)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)m) >> 32);
}

/* A draw u "hits" with probability q iff u < threshold(q). */
uint64_t leea_cpu_threshold(double q)
{
    if (!(q > 0.0)) return 0;
    if (q >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(q * 4294967296.0);
}

/* 16-bit draw i of a stream, for per-gene masks: block i >> 3 carries eight
 * of them, two per word, the even one in the low half. */
uint32_t leea_cpu_draw16(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t i)
{
    uint32_t w[4];
    stream_block(seed, tag, gen, ent, i >> 3, w);
    uint32_t word = w[(i >> 1) & 3u];
    return (i & 1u) ? (word >> 16) : (word & 0xFFFFu);
}

/* A 16-bit draw hits probability q iff it is below threshold16(q). */
uint32_t leea_cpu_threshold16(double q)
{
    if (!(q > 0.0)) return 0;
    if (q >= 1.0) return 65536u;
    return (uint32_t)floor(q * 65536.0);
}

/* ------------------------------------------------------------------------ */
/* Layout and operator counts                                               */
/* ------------------------------------------------------------------------ */

/* c = sum over layers of (out * in + out)  (Section 3.2, theta in R^c). */
int64_t leea_cpu_num_params(const int32_t* dims, int32_t n_dims)
{
    if (!dims || n_dims < 2) return -1;
    int64_t c = 0;
    for (int l = 0; l + 1 < n_dims; l++) {
        if (dims[l] <= 0 || dims[l + 1] <= 0) return -1;
        c += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    }
    return c;
}

/* Offspring counts of Algorithm 1: p_E*lambda elites, p_C*lambda crossover
 * children, the remaining p_M*lambda mutation children; parents come from the
 * top rho*lambda (Section 3.1).  Rounding: n_E and n_C by round(), n_M takes
 * the rest, the pool is max(1, floor(rho*lambda)). */
int leea_cpu_counts(int32_t pop, const leea_cpu_params* prm, int32_t* n_e,
                    int32_t* n_c, int32_t* n_m, int32_t* pool)
{
    if (pop <= 0 || !prm) return LEEA_CPU_EINVAL;
    int32_t e = prm->n_elite >= 0 ? prm->n_elite
                                  : (int32_t)round((double)prm->p_e * (double)pop);
    if (e > pop) e = pop;
    if (e < 0) e = 0;
    int32_t cc = (int32_t)round((double)prm->p_c * (double)pop);
    if (cc > pop - e) cc = pop - e;
    if (cc < 0) cc = 0;
    int32_t pl = (int32_t)floor((double)prm->rho * (double)pop);
    if (pl < 1) pl = 1;
    if (pl > pop) pl = pop;
    if (n_e) *n_e = e;
    if (n_c) *n_c = cc;
    if (n_m) *n_m = pop - e - cc;
    if (pool) *pool = pl;
    return LEEA_CPU_OK;
}

static int valid_params(const leea_cpu_params* prm)
{
    if (!prm) return 0;
    if (prm->xo_op != 0 && prm->xo_op != 1) return 0;
    if (prm->sel_op != 0 && prm->sel_op != 1) return 0;
    if (!(prm->xo_gene_p >= 0.0f && prm->xo_gene_p <= 1.0f)) return 0;
    if (!(prm->rho > 0.0f && prm->rho <= 1.0f)) return 0;
    if (prm->sel_op == 1 && prm->tour_k < 1) return 0;
    if (!(prm->p_e >= 0.0f && prm->p_e <= 1.0f)) return 0;
    if (!(prm->p_c >= 0.0f && prm->p_c <= 1.0f)) return 0;
    if (!(prm->sigma >= 0.0f) || isinf(prm->sigma)) return 0;
    if (!(prm->mut_rate >= 0.0f && prm->mut_rate <= 1.0f)) return 0;
    if (!(prm->alpha >= 0.0f && prm->alpha <= 1.0f)) return 0;
    if (prm->init != 0 && prm->init != 1) return 0;
    if (prm->precision < 0 || prm->precision > 2) return 0;
    if (prm->sigma_ctl < LEEA_CPU_SIGMA_CONST || prm->sigma_ctl > LEEA_CPU_SIGMA_SELF) return 0;
    if (prm->sigma_ctl == LEEA_CPU_SIGMA_DECAY && !(prm->sigma_k > 0.0f && !isinf(prm->sigma_k))) return 0;
    if (prm->sigma_ctl == LEEA_CPU_SIGMA_SELF && !(prm->tau >= 0.0f && !isinf(prm->tau))) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Initialisation (Section 4.1: Glorot-uniform; the alternative N(0,1/fan_in)) */
/* ------------------------------------------------------------------------ */
int leea_cpu_init(int32_t pop, const int32_t* dims, int32_t n_dims, int32_t init,
                  uint64_t seed, double* pop_out)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || pop <= 0 || !pop_out || (init != 0 && init != 1)) return LEEA_CPU_EINVAL;
    for (int32_t p = 0; p < pop; p++) {
        double* theta = pop_out + (int64_t)p * c;
        int64_t i = 0;
        for (int l = 0; l + 1 < n_dims; l++) {
            int32_t fan_in = dims[l], fan_out = dims[l + 1];
            int64_t nw = (int64_t)fan_out * fan_in;
            for (int64_t k = 0; k < nw; k++, i++) {
                if (init == 0) {
                    double z = leea_cpu_normal(seed, LEEA_CPU_TAG_INIT, 0, (uint32_t)p, (uint32_t)i);
                    theta[i] = z * sqrt(1.0 / (double)fan_in);
                } else {
                    double a = sqrt(6.0 / (double)(fan_in + fan_out));
                    double u = leea_cpu_u01(leea_cpu_draw(seed, LEEA_CPU_TAG_INIT, 0, (uint32_t)p, (uint32_t)i));
                    theta[i] = a * (2.0 * u - 1.0);
                }
            }
            for (int32_t k = 0; k < fan_out; k++, i++) theta[i] = 0.0; /* biases */
        }
    }
    return LEEA_CPU_OK;
}

/* ------------------------------------------------------------------------ */
/* Input stage of the paper's network (Section 4.1): 2x2 max-pooling          */
/* ------------------------------------------------------------------------ */
int leea_cpu_maxpool2x2(int32_t batch, int32_t h, int32_t w, const double* x, double* out)
{
    if (batch < 0 || h <= 0 || w <= 0 || (h & 1) || (w & 1) || (batch > 0 && (!x || !out)))
        return LEEA_CPU_EINVAL;
    int32_t ho = h / 2, wo = w / 2;
    for (int32_t b = 0; b < batch; b++) {
        const double* img = x + (int64_t)b * h * w;
        double* o = out + (int64_t)b * ho * wo;
        for (int32_t i = 0; i < ho; i++) {
            for (int32_t j = 0; j < wo; j++) {
                double m = img[(2 * i) * w + 2 * j];
                double c;
                c = img[(2 * i) * w + 2 * j + 1];
                if (c > m) m = c;
                c = img[(2 * i + 1) * w + 2 * j];
                if (c > m) m = c;
                c = img[(2 * i + 1) * w + 2 * j + 1];
                if (c > m) m = c;
                o[i * wo + j] = m;
            }
        }
    }
    return LEEA_CPU_OK;
}

/* ------------------------------------------------------------------------ */
/* Fitness (Eq. 1): negative mean cross-entropy of the softmax output over   */
/* the batch; hidden layers use ReLU (Section 4.1).  Also counts correct    */
/* argmax predictions, ties to the lowest class.                            */
/* ------------------------------------------------------------------------ */
int leea_cpu_evaluate(int32_t pop, const int32_t* dims, int32_t n_dims,
                      const double* popv, const double* x, const int32_t* y,
                      int32_t batch, double* f_out, int32_t* correct_out,
                      double* logits_out)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || pop <= 0 || batch <= 0 || !popv || !x || !y || !f_out) return LEEA_CPU_EINVAL;
    int32_t d_out = dims[n_dims - 1];
    for (int32_t b = 0; b < batch; b++)
        if (y[b] < 0 || y[b] >= d_out) return LEEA_CPU_EINVAL;
    int32_t widest = 0;
    for (int l = 0; l < n_dims; l++) if (dims[l] > widest) widest = dims[l];
    double* a = (double*)malloc(sizeof(double) * (size_t)widest);
    double* z = (double*)malloc(sizeof(double) * (size_t)widest);
    if (!a || !z) { free(a); free(z); return LEEA_CPU_ENOMEM; }

    for (int32_t p = 0; p < pop; p++) {
        const double* theta = popv + (int64_t)p * c;
        double loss_sum = 0.0;
        int32_t correct = 0;
        for (int32_t b = 0; b < batch; b++) {
            for (int32_t k = 0; k < dims[0]; k++) a[k] = x[(int64_t)b * dims[0] + k];
            const double* w = theta;
            for (int l = 0; l + 1 < n_dims; l++) {
                int32_t n_in = dims[l], n_out = dims[l + 1];
                const double* bias = w + (int64_t)n_out * n_in;
                for (int32_t o = 0; o < n_out; o++) {
                    double acc = 0.0;
                    for (int32_t k = 0; k < n_in; k++) acc += w[(int64_t)o * n_in + k] * a[k];
                    acc += bias[o];
                    int last = (l + 2 == n_dims);
                    z[o] = (!last && acc < 0.0) ? 0.0 : acc; /* ReLU on hidden layers */
                }
                memcpy(a, z, sizeof(double) * (size_t)n_out);
                w = bias + n_out;
            }
            /* a[0..d_out) are the logits.  Cross-entropy against the one-hot
             * label: log(sum_j exp(z_j)) - z_y, with the maximum subtracted. */
            double zmax = a[0];
            int32_t arg = 0;
            for (int32_t j = 1; j < d_out; j++)
                if (a[j] > zmax) { zmax = a[j]; arg = j; }
            double s = 0.0;
            for (int32_t j = 0; j < d_out; j++) s += exp(a[j] - zmax);
            double loss = log(s) + zmax - a[y[b]];
            loss_sum += loss;
            if (arg == y[b]) correct++;
            if (logits_out)
                memcpy(logits_out + ((int64_t)p * batch + b) * d_out, a, sizeof(double) * (size_t)d_out);
        }
        f_out[p] = -loss_sum / (double)batch;
        if (correct_out) correct_out[p] = correct;
    }
    free(a);
    free(z);
    return LEEA_CPU_OK;
}

/* ------------------------------------------------------------------------ */
/* Precision form: BF16 and FP8-e4m3 shadows of W1.                          */
/* ------------------------------------------------------------------------ */

/* Round x to the nearest multiple of the power of two q, ties to even. */
static double round_to_grid(double x, double q)
{
    return nearbyint(x / q) * q;  /* x / q is exact; default rounding is to nearest even */
}

/* BF16: 1 sign, 8 exponent (bias 127), 7 stored mantissa bits. */
double leea_cpu_round_bf16(double x)
{
    if (x == 0.0 || isnan(x) || isinf(x)) return x;
    int e;
    frexp(x, &e);                 /* |x| in [2^(e-1), 2^e) */
    int lead = e - 1;
    if (lead < -126) lead = -126; /* subnormal range: fixed quantum */
    return round_to_grid(x, ldexp(1.0, lead - 7));
}

/* FP8-e4m3 (OCP "FN"): 1 sign, 4 exponent (bias 7), 3 mantissa bits, no
 * infinities; largest finite 448 = 1.75 * 2^8; smallest subnormal 2^-9. */
double leea_cpu_round_e4m3(double x)
{
    if (isnan(x)) return x;
    if (isinf(x)) return x > 0 ? 448.0 : -448.0;
    if (x == 0.0) return x;
    int e;
    frexp(x, &e);
    int lead = e - 1;
    if (lead < -6) lead = -6;     /* subnormals share the quantum 2^-9 */
    double r = round_to_grid(x, ldexp(1.0, lead - 3));
    if (r > 448.0) r = 448.0;     /* saturate to finite */
    if (r < -448.0) r = -448.0;
    return r;
}

int32_t leea_cpu_fp8_scale_exp(double bound)
{
    if (!(bound > 0.0)) return 0;
    int32_t e = -200;
    while (448.0 * ldexp(1.0, e) < bound) e++;
    return e;
}

int leea_cpu_quantize_w1(int32_t pop, const int32_t* dims, int32_t n_dims, const double* popv,
                         int32_t precision, const int32_t* scale_exp, double* out)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || pop <= 0 || !popv || !out || precision < 0 || precision > 2 || (precision == 2 && !scale_exp))
        return LEEA_CPU_EINVAL;
    int64_t n_w1 = (int64_t)dims[0] * dims[1];
    for (int32_t p = 0; p < pop; p++) {
        const double* theta = popv + (int64_t)p * c;
        double* q = out + (int64_t)p * c;
        memmove(q, theta, sizeof(double) * (size_t)c);
        for (int64_t i = 0; i < n_w1; i++) {
            if (precision == 1) {
                q[i] = leea_cpu_round_bf16(q[i]);
            } else if (precision == 2) {
                double s = ldexp(1.0, scale_exp[p]);
                q[i] = leea_cpu_round_e4m3(q[i] / s) * s;
            }
        }
    }
    return LEEA_CPU_OK;
}

int leea_cpu_evaluate_shadow(int32_t pop, const int32_t* dims, int32_t n_dims,
                             const double* popv, int32_t precision, const int32_t* scale_exp,
                             const double* x, const int32_t* y, int32_t batch,
                             double* f_out, int32_t* correct_out)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || pop <= 0 || !popv || precision < 0 || precision > 2 || (precision == 2 && !scale_exp))
        return LEEA_CPU_EINVAL;
    double* q = (double*)malloc(sizeof(double) * (size_t)c);
    if (!q) return LEEA_CPU_ENOMEM;
    int rc = LEEA_CPU_OK;
    for (int32_t p = 0; p < pop && rc == LEEA_CPU_OK; p++) {
        rc = leea_cpu_quantize_w1(1, dims, n_dims, popv + (int64_t)p * c, precision,
                                  scale_exp ? scale_exp + p : NULL, q);
        if (rc == LEEA_CPU_OK)
            rc = leea_cpu_evaluate(1, dims, n_dims, q, x, y, batch, f_out + p,
                                   correct_out ? correct_out + p : NULL, NULL);
    }
    free(q);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sort by fitness, descending (Algorithm 1).  NaN ranks as -infinity; ties  */
/* go to the lower index (a stable sort).                                   */
/* ------------------------------------------------------------------------ */
typedef struct { double f; int32_t idx; } rank_item;

static int rank_cmp(const void* pa, const void* pb)
{
    const rank_item* a = (const rank_item*)pa;
    const rank_item* b = (const rank_item*)pb;
    double fa = isnan(a->f) ? -INFINITY : a->f;
    double fb = isnan(b->f) ? -INFINITY : b->f;
    if (fa > fb) return -1;
    if (fa < fb) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

int leea_cpu_rank(int32_t pop, const double* f_adj, int32_t* order)
{
    if (pop <= 0 || !f_adj || !order) return LEEA_CPU_EINVAL;
    rank_item* items = (rank_item*)malloc(sizeof(rank_item) * (size_t)pop);
    if (!items) return LEEA_CPU_ENOMEM;
    for (int32_t i = 0; i < pop; i++) { items[i].f = f_adj[i]; items[i].idx = i; }
    qsort(items, (size_t)pop, sizeof(rank_item), rank_cmp);
    for (int32_t r = 0; r < pop; r++) order[r] = items[r].idx;
    free(items);
    return LEEA_CPU_OK;
}

/* Does individual a beat individual b? Higher fitness wins, NaN counts as
 * -infinity, equal fitness goes to the lower index. */
static int beats(const double* f_adj, int32_t a, int32_t b)
{
    rank_item ia = { f_adj[a], a }, ib = { f_adj[b], b };
    return rank_cmp(&ia, &ib) < 0;
}

/* One parent for child j, from draws [first, first + k) of its SEL stream.
 * Truncation (Section 3.1): uniform over the top `pool` of the ranking.
 * Tournament: best of k uniform draws (with replacement) over everybody. */
static int32_t pick_parent(int32_t pop, const leea_cpu_params* prm, const double* f_adj,
                           const int32_t* order, int32_t pool, uint64_t seed, uint32_t gen,
                           uint32_t j, uint32_t first)
{
    if (prm->sel_op == 0) {
        uint32_t u = leea_cpu_draw(seed, LEEA_CPU_TAG_SEL, gen, j, first);
        return order[leea_cpu_index(u, (uint32_t)pool)];
    }
    int32_t best = -1;
    for (int32_t t = 0; t < prm->tour_k; t++) {
        uint32_t u = leea_cpu_draw(seed, LEEA_CPU_TAG_SEL, gen, j, first + (uint32_t)t);
        int32_t cand = (int32_t)leea_cpu_index(u, (uint32_t)pop);
        if (best < 0 || beats(f_adj, cand, best)) best = cand;
    }
    return best;
}

/* Elites, crossover pairs and mutation parents of Algorithm 1, in that child
 * order, and the inherited fitness of each child (Section 3.1):
 * f_inh = (f1 + f2) / 2 after crossover, f3 after mutation; an elite keeps
 * its own adjusted fitness. */
int leea_cpu_select(int32_t pop, const leea_cpu_params* prm, const double* f_adj,
                    const int32_t* order, uint64_t seed, uint32_t gen,
                    int32_t* par1, int32_t* par2, int32_t* kind, double* f_inh)
{
    if (pop <= 0 || !valid_params(prm) || !f_adj || !order || !par1 || !par2 || !kind || !f_inh)
        return LEEA_CPU_EINVAL;
    int32_t n_e, n_c, n_m, pool;
    leea_cpu_counts(pop, prm, &n_e, &n_c, &n_m, &pool);
    uint32_t k_draws = (prm->sel_op == 0) ? 1u : (uint32_t)prm->tour_k;
    for (int32_t j = 0; j < pop; j++) {
        if (j < n_e) {
            kind[j] = LEEA_CPU_ELITE;
            par1[j] = par2[j] = order[j];
            f_inh[j] = f_adj[order[j]];
        } else if (j < n_e + n_c) {
            kind[j] = LEEA_CPU_CROSSOVER;
            par1[j] = pick_parent(pop, prm, f_adj, order, pool, seed, gen, (uint32_t)j, 0);
            par2[j] = pick_parent(pop, prm, f_adj, order, pool, seed, gen, (uint32_t)j, k_draws);
            f_inh[j] = 0.5 * (f_adj[par1[j]] + f_adj[par2[j]]);
        } else {
            kind[j] = LEEA_CPU_MUTATION;
            par1[j] = pick_parent(pop, prm, f_adj, order, pool, seed, gen, (uint32_t)j, 0);
            par2[j] = par1[j];
            f_inh[j] = f_adj[par1[j]];
        }
    }
    return LEEA_CPU_OK;
}

/* ------------------------------------------------------------------------ */
/* Crossover and mutation (Section 3.2), children j0 <= j < j1.              */
/*   uniform:     gene i from parent 2 iff its 16-bit XO draw hits xo_gene_p */
/*   arithmetic:  (theta_1 + theta_2) / 2                                    */
/*   mutation:    theta_1 + sigma * N(0,1) on genes whose 16-bit MUTMASK     */
/*                draw hits mut_rate (every gene when mut_rate = 1)          */
/*   elite:       unchanged copy                                             */
/* ------------------------------------------------------------------------ */
/* Child out (c genes) of the given kind from parents a, b, drawing from the
 * streams of Philox entity `ent`. */
static int breed_child(int64_t c, const leea_cpu_params* prm, double sigma, uint64_t seed, uint32_t gen,
                       uint32_t ent, int32_t kind, const double* a, const double* b, double* out)
{
    uint32_t thr_xo = leea_cpu_threshold16((double)prm->xo_gene_p);
    uint32_t thr_mut = leea_cpu_threshold16((double)prm->mut_rate);
    for (int64_t i = 0; i < c; i++) {
        double v;
        if (kind == LEEA_CPU_ELITE) {
            v = a[i];
        } else if (kind == LEEA_CPU_CROSSOVER) {
            if (prm->xo_op == 0) {
                uint32_t u = leea_cpu_draw16(seed, LEEA_CPU_TAG_XO, gen, ent, (uint32_t)i);
                v = (u < thr_xo) ? b[i] : a[i];
            } else {
                v = 0.5 * (a[i] + b[i]);
            }
        } else if (kind == LEEA_CPU_MUTATION) {
            uint32_t u = leea_cpu_draw16(seed, LEEA_CPU_TAG_MUTMASK, gen, ent, (uint32_t)i);
            if (u < thr_mut)
                v = a[i] + sigma * leea_cpu_normal(seed, LEEA_CPU_TAG_NORMAL, gen, ent, (uint32_t)i);
            else
                v = a[i];
        } else {
            return LEEA_CPU_EINVAL;
        }
        out[i] = v;
    }
    return LEEA_CPU_OK;
}

int leea_cpu_breed(int32_t pop, const int32_t* dims, int32_t n_dims,
                   const leea_cpu_params* prm, uint64_t seed, uint32_t gen,
                   const double* parents, const int32_t* par1, const int32_t* par2,
                   const int32_t* kind, int32_t j0, int32_t j1, double* children)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || pop <= 0 || !valid_params(prm) || !parents || !par1 || !par2 || !kind ||
        !children || j0 < 0 || j1 > pop || j0 > j1)
        return LEEA_CPU_EINVAL;
    for (int32_t j = j0; j < j1; j++) {
        if (par1[j] < 0 || par1[j] >= pop || par2[j] < 0 || par2[j] >= pop) return LEEA_CPU_EINVAL;
        int rc = breed_child(c, prm, (double)prm->sigma, seed, gen, (uint32_t)j, kind[j],
                             parents + (int64_t)par1[j] * c, parents + (int64_t)par2[j] * c,
                             children + (int64_t)(j - j0) * c);
        if (rc != LEEA_CPU_OK) return rc;
    }
    return LEEA_CPU_OK;
}

/* ------------------------------------------------------------------------ */
/* Control of the mutation strength (Section 3.2).                          */
/*   constant:       sigma in every breed                                   */
/*   decay:          breed i (i = 0 for the first) uses sigma 0.99^(i/k)    */
/*   self-adaptive:  each individual carries a sigma gene; a mutation child */
/*                   first mutates its parent's gene, sigma' = sigma        */
/*                   exp(tau N(0,1)), then its weights with sigma'; a       */
/*                   crossover child takes the mean of its parents' genes   */
/* ------------------------------------------------------------------------ */
double leea_cpu_sigma_schedule(const leea_cpu_params* prm, uint32_t gen)
{
    double sigma = (double)prm->sigma;
    if (prm->sigma_ctl != LEEA_CPU_SIGMA_DECAY) return sigma;
    double i = gen > 0 ? (double)(gen - 1u) : 0.0;
    return sigma * pow(0.99, i / (double)prm->sigma_k);
}

int leea_cpu_select_sigma(int32_t pop, const leea_cpu_params* prm, uint64_t seed, uint32_t gen,
                          const int32_t* par1, const int32_t* par2, const int32_t* kind,
                          const double* sigma_in, double* sigma_out)
{
    if (pop <= 0 || !valid_params(prm) || !par1 || !par2 || !kind || !sigma_in || !sigma_out)
        return LEEA_CPU_EINVAL;
    for (int32_t j = 0; j < pop; j++) {
        if (par1[j] < 0 || par1[j] >= pop || par2[j] < 0 || par2[j] >= pop) return LEEA_CPU_EINVAL;
        double s1 = sigma_in[par1[j]];
        if (kind[j] == LEEA_CPU_ELITE) {
            sigma_out[j] = s1;
        } else if (kind[j] == LEEA_CPU_CROSSOVER) {
            sigma_out[j] = 0.5 * (s1 + sigma_in[par2[j]]);
        } else if (kind[j] == LEEA_CPU_MUTATION) {
            double z = leea_cpu_normal(seed, LEEA_CPU_TAG_SIGMA, gen, (uint32_t)j, 0u);
            sigma_out[j] = s1 * exp((double)prm->tau * z);
        } else {
            return LEEA_CPU_EINVAL;
        }
    }
    return LEEA_CPU_OK;
}

int leea_cpu_breed_sigma(int32_t pop, const int32_t* dims, int32_t n_dims,
                         const leea_cpu_params* prm, uint64_t seed, uint32_t gen,
                         const double* parents, const int32_t* par1, const int32_t* par2,
                         const int32_t* kind, const double* sigma_child, int32_t j0, int32_t j1,
                         double* children)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || pop <= 0 || !valid_params(prm) || !parents || !par1 || !par2 || !kind ||
        !sigma_child || !children || j0 < 0 || j1 > pop || j0 > j1)
        return LEEA_CPU_EINVAL;
    for (int32_t j = j0; j < j1; j++) {
        if (par1[j] < 0 || par1[j] >= pop || par2[j] < 0 || par2[j] >= pop) return LEEA_CPU_EINVAL;
        int rc = breed_child(c, prm, sigma_child[j], seed, gen, (uint32_t)j, kind[j],
                             parents + (int64_t)par1[j] * c, parents + (int64_t)par2[j] * c,
                             children + (int64_t)(j - j0) * c);
        if (rc != LEEA_CPU_OK) return rc;
    }
    return LEEA_CPU_OK;
}

/* Fitness inheritance (Section 3.1): f_adj = (1 - alpha) f_inh + alpha f.
 * The first evaluation has nothing to inherit: f_adj = f. */
int leea_cpu_inherit(int32_t pop, double alpha, const double* f_inh, const double* f,
                     int32_t first, double* f_adj)
{
    if (pop <= 0 || !f || !f_adj || (!first && !f_inh)) return LEEA_CPU_EINVAL;
    for (int32_t p = 0; p < pop; p++)
        f_adj[p] = first ? f[p] : (1.0 - alpha) * f_inh[p] + alpha * f[p];
    return LEEA_CPU_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 as a state object.  The first generation call evaluates the  */
/* freshly initialised population; every later call sorts, selects, breeds  */
/* with generation counter g = 1, 2, ... and evaluates the new population.  */
/* ------------------------------------------------------------------------ */
struct leea_cpu_state {
    int32_t pop, n_dims;
    int32_t dims[16];
    int64_t c;
    leea_cpu_params prm;
    uint64_t seed;
    uint32_t gen;
    int32_t evaluated;
    double *cur, *next;
    double *f_adj, *f_raw, *f_inh;
    double *sig_cur, *sig_next;  /* sigma genes (self-adaptive) or the breed's strength */
    int32_t *correct, *order, *par1, *par2, *kind;
};

void leea_cpu_destroy(leea_cpu_state* s)
{
    if (!s) return;
    free(s->cur); free(s->next);
    free(s->f_adj); free(s->f_raw); free(s->f_inh);
    free(s->sig_cur); free(s->sig_next);
    free(s->correct); free(s->order); free(s->par1); free(s->par2); free(s->kind);
    free(s);
}

int leea_cpu_create(int32_t pop, const int32_t* dims, int32_t n_dims,
                    const leea_cpu_params* prm, uint64_t seed, leea_cpu_state** out)
{
    if (!out) return LEEA_CPU_EINVAL;
    *out = NULL;
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || n_dims > 16 || pop <= 0 || !valid_params(prm)) return LEEA_CPU_EINVAL;
    leea_cpu_state* s = (leea_cpu_state*)calloc(1, sizeof(*s));
    if (!s) return LEEA_CPU_ENOMEM;
    s->pop = pop; s->n_dims = n_dims; s->c = c; s->prm = *prm; s->seed = seed;
    memcpy(s->dims, dims, sizeof(int32_t) * (size_t)n_dims);
    size_t np = (size_t)pop;
    s->cur = (double*)malloc(sizeof(double) * np * (size_t)c);
    s->next = (double*)malloc(sizeof(double) * np * (size_t)c);
    s->f_adj = (double*)calloc(np, sizeof(double));
    s->f_raw = (double*)calloc(np, sizeof(double));
    s->f_inh = (double*)calloc(np, sizeof(double));
    s->correct = (int32_t*)calloc(np, sizeof(int32_t));
    s->order = (int32_t*)calloc(np, sizeof(int32_t));
    s->par1 = (int32_t*)calloc(np, sizeof(int32_t));
    s->par2 = (int32_t*)calloc(np, sizeof(int32_t));
    s->kind = (int32_t*)calloc(np, sizeof(int32_t));
    s->sig_cur = (double*)calloc(np, sizeof(double));
    s->sig_next = (double*)calloc(np, sizeof(double));
    if (!s->cur || !s->next || !s->f_adj || !s->f_raw || !s->f_inh || !s->correct ||
        !s->order || !s->par1 || !s->par2 || !s->kind || !s->sig_cur || !s->sig_next) {
        leea_cpu_destroy(s);
        return LEEA_CPU_ENOMEM;
    }
    for (size_t p = 0; p < np; p++) s->sig_cur[p] = (double)prm->sigma;  /* initial sigma genes */
    leea_cpu_init(pop, dims, n_dims, prm->init, seed, s->cur);
    *out = s;
    return LEEA_CPU_OK;
}

int leea_cpu_generation(leea_cpu_state* s, const double* x, const int32_t* y, int32_t batch)
{
    if (!s || !x || !y || batch <= 0) return LEEA_CPU_EINVAL;
    int rc;
    int first = !s->evaluated;
    if (!first) {
        uint32_t g = s->gen + 1;
        rc = leea_cpu_rank(s->pop, s->f_adj, s->order);
        if (rc) return rc;
        rc = leea_cpu_select(s->pop, &s->prm, s->f_adj, s->order, s->seed, g,
                             s->par1, s->par2, s->kind, s->f_inh);
        if (rc) return rc;
        if (s->prm.sigma_ctl == LEEA_CPU_SIGMA_SELF) {
            rc = leea_cpu_select_sigma(s->pop, &s->prm, s->seed, g, s->par1, s->par2, s->kind,
                                       s->sig_cur, s->sig_next);
            if (rc) return rc;
        } else {
            double sigma = leea_cpu_sigma_schedule(&s->prm, g);
            for (int32_t j = 0; j < s->pop; j++) s->sig_next[j] = sigma;
        }
        rc = leea_cpu_breed_sigma(s->pop, s->dims, s->n_dims, &s->prm, s->seed, g, s->cur,
                                  s->par1, s->par2, s->kind, s->sig_next, 0, s->pop, s->next);
        if (rc) return rc;
        double* t = s->cur; s->cur = s->next; s->next = t;
        t = s->sig_cur; s->sig_cur = s->sig_next; s->sig_next = t;
        s->gen = g;
    }
    rc = leea_cpu_evaluate(s->pop, s->dims, s->n_dims, s->cur, x, y, batch,
                           s->f_raw, s->correct, NULL);
    if (rc) return rc;
    rc = leea_cpu_inherit(s->pop, (double)s->prm.alpha, s->f_inh, s->f_raw, first, s->f_adj);
    if (rc) return rc;
    s->evaluated = 1;
    return LEEA_CPU_OK;
}

int leea_cpu_fitness(const leea_cpu_state* s, double* f_adj, double* f_raw, int32_t* correct)
{
    if (!s) return LEEA_CPU_EINVAL;
    if (!s->evaluated) return LEEA_CPU_ESTATE;
    size_t np = (size_t)s->pop;
    if (f_adj) memcpy(f_adj, s->f_adj, sizeof(double) * np);
    if (f_raw) memcpy(f_raw, s->f_raw, sizeof(double) * np);
    if (correct) memcpy(correct, s->correct, sizeof(int32_t) * np);
    return LEEA_CPU_OK;
}

int leea_cpu_best_params(const leea_cpu_state* s, double* out, int64_t c)
{
    if (!s || !out || c != s->c) return LEEA_CPU_EINVAL;
    if (!s->evaluated) return LEEA_CPU_ESTATE;
    int32_t best = 0;
    for (int32_t p = 1; p < s->pop; p++)
        if (beats(s->f_adj, p, best)) best = p;
    memcpy(out, s->cur + (int64_t)best * s->c, sizeof(double) * (size_t)s->c);
    return LEEA_CPU_OK;
}

int leea_cpu_get_population(const leea_cpu_state* s, double* out)
{
    if (!s || !out) return LEEA_CPU_EINVAL;
    memcpy(out, s->cur, sizeof(double) * (size_t)s->pop * (size_t)s->c);
    return LEEA_CPU_OK;
}

int leea_cpu_set_population(leea_cpu_state* s, const double* in)
{
    if (!s || !in) return LEEA_CPU_EINVAL;
    memcpy(s->cur, in, sizeof(double) * (size_t)s->pop * (size_t)s->c);
    return LEEA_CPU_OK;
}

int leea_cpu_set_fitness(leea_cpu_state* s, const double* f_adj)
{
    if (!s || !f_adj) return LEEA_CPU_EINVAL;
    memcpy(s->f_adj, f_adj, sizeof(double) * (size_t)s->pop);
    return LEEA_CPU_OK;
}

int leea_cpu_set_generation(leea_cpu_state* s, uint32_t gen, int32_t evaluated)
{
    if (!s) return LEEA_CPU_EINVAL;
    s->gen = gen;
    s->evaluated = evaluated ? 1 : 0;
    return LEEA_CPU_OK;
}

int leea_cpu_get_selection(const leea_cpu_state* s, int32_t* order, int32_t* par1,
                           int32_t* par2, int32_t* kind, double* f_inh)
{
    if (!s) return LEEA_CPU_EINVAL;
    size_t np = (size_t)s->pop;
    if (order) memcpy(order, s->order, sizeof(int32_t) * np);
    if (par1) memcpy(par1, s->par1, sizeof(int32_t) * np);
    if (par2) memcpy(par2, s->par2, sizeof(int32_t) * np);
    if (kind) memcpy(kind, s->kind, sizeof(int32_t) * np);
    if (f_inh) memcpy(f_inh, s->f_inh, sizeof(double) * np);
    return LEEA_CPU_OK;
}

uint32_t leea_cpu_generation_index(const leea_cpu_state* s)
{
    return s ? s->gen : 0;
}

int leea_cpu_get_sigma(const leea_cpu_state* s, double* out)
{
    if (!s || !out) return LEEA_CPU_EINVAL;
    for (int32_t p = 0; p < s->pop; p++)
        out[p] = s->prm.sigma_ctl == LEEA_CPU_SIGMA_SELF ? s->sig_cur[p]
                                                         : leea_cpu_sigma_schedule(&s->prm, s->gen + 1u);
    return LEEA_CPU_OK;
}

int leea_cpu_set_sigma(leea_cpu_state* s, const double* in)
{
    if (!s || !in) return LEEA_CPU_EINVAL;
    if (s->prm.sigma_ctl != LEEA_CPU_SIGMA_SELF) return LEEA_CPU_ESTATE;
    memcpy(s->sig_cur, in, sizeof(double) * (size_t)s->pop);
    return LEEA_CPU_OK;
}

/* ======================================================================== */
/* Surrogate form (a learned pre-screen of offspring; the paper has no       */
/* counterpart).  Offspring are first "recipes" -- a kind, parents and the   */
/* Philox entity whose streams make the child -- described by a feature     */
/* vector, scored by a small MLP, and only the best are made and evaluated. */
/* ======================================================================== */

int64_t leea_cpu_mlp_num_params(int32_t d_in, int32_t h1, int32_t h2)
{
    if (d_in <= 0 || h1 <= 0 || h2 <= 0) return -1;
    return (int64_t)h1 * d_in + h1 + (int64_t)h2 * h1 + h2 + h2 + 1;
}

/* Glorot-uniform weights, U(-a, a) with a = sqrt(6 / (fan_in + fan_out)),
 * from Philox stream (SURR_INIT, generation 0, entity 0, draw = parameter
 * index); zero biases. */
int leea_cpu_mlp_init(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, double* theta)
{
    int64_t np = leea_cpu_mlp_num_params(d_in, h1, h2);
    if (np < 0 || !theta) return LEEA_CPU_EINVAL;
    const int32_t fin[3] = { d_in, h1, h2 }, fout[3] = { h1, h2, 1 };
    int64_t i = 0;
    for (int l = 0; l < 3; l++) {
        double a = sqrt(6.0 / (double)(fin[l] + fout[l]));
        for (int64_t k = 0; k < (int64_t)fin[l] * fout[l]; k++, i++) {
            double u = leea_cpu_u01(leea_cpu_draw(seed, LEEA_CPU_TAG_SURR_INIT, 0, 0, (uint32_t)i));
            theta[i] = a * (2.0 * u - 1.0);
        }
        for (int32_t k = 0; k < fout[l]; k++, i++) theta[i] = 0.0;
    }
    return LEEA_CPU_OK;
}

/* y_r = w3 . relu(W2 relu(W1 x_r + b1) + b2) + b3 for rows r < n of x[n][d_in];
 * hidden activations are also returned when a1 / a2 are not NULL. */
static void mlp_row(int32_t d_in, int32_t h1, int32_t h2, const double* theta, const double* x,
                    double* a1, double* a2, double* y)
{
    const double* W1 = theta;
    const double* b1 = W1 + (int64_t)h1 * d_in;
    const double* W2 = b1 + h1;
    const double* b2 = W2 + (int64_t)h2 * h1;
    const double* w3 = b2 + h2;
    const double b3 = w3[h2];
    for (int32_t u = 0; u < h1; u++) {
        double z = b1[u];
        for (int32_t k = 0; k < d_in; k++) z += W1[(int64_t)u * d_in + k] * x[k];
        a1[u] = z > 0.0 ? z : 0.0;
    }
    for (int32_t u = 0; u < h2; u++) {
        double z = b2[u];
        for (int32_t k = 0; k < h1; k++) z += W2[(int64_t)u * h1 + k] * a1[k];
        a2[u] = z > 0.0 ? z : 0.0;
    }
    double out = b3;
    for (int32_t u = 0; u < h2; u++) out += w3[u] * a2[u];
    *y = out;
}

int leea_cpu_mlp_forward(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const double* theta,
                         const double* x, double* y)
{
    if (n < 0 || leea_cpu_mlp_num_params(d_in, h1, h2) < 0 || !theta || (n > 0 && (!x || !y)))
        return LEEA_CPU_EINVAL;
    double* a1 = (double*)malloc(sizeof(double) * (size_t)h1);
    double* a2 = (double*)malloc(sizeof(double) * (size_t)h2);
    if (!a1 || !a2) {
        free(a1);
        free(a2);
        return LEEA_CPU_ENOMEM;
    }
    for (int32_t r = 0; r < n; r++) mlp_row(d_in, h1, h2, theta, x + (int64_t)r * d_in, a1, a2, y + r);
    free(a1);
    free(a2);
    return LEEA_CPU_OK;
}

/* Mean squared error L = (1/n) sum_r (y_r - t_r)^2 and dL/dtheta by the chain
 * rule (backpropagation through the two ReLU layers). */
int leea_cpu_mlp_loss_grad(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const double* theta,
                           const double* x, const double* t, double* loss, double* grad)
{
    int64_t np = leea_cpu_mlp_num_params(d_in, h1, h2);
    if (n <= 0 || np < 0 || !theta || !x || !t || !loss || !grad) return LEEA_CPU_EINVAL;
    const double* W2 = theta + (int64_t)h1 * d_in + h1;
    const double* w3 = W2 + (int64_t)h2 * h1 + h2;
    double* gW1 = grad;
    double* gb1 = gW1 + (int64_t)h1 * d_in;
    double* gW2 = gb1 + h1;
    double* gb2 = gW2 + (int64_t)h2 * h1;
    double* gw3 = gb2 + h2;
    double* gb3 = gw3 + h2;
    for (int64_t i = 0; i < np; i++) grad[i] = 0.0;
    double* a1 = (double*)malloc(sizeof(double) * (size_t)h1);
    double* a2 = (double*)malloc(sizeof(double) * (size_t)h2);
    double* d1 = (double*)malloc(sizeof(double) * (size_t)h1);
    double* d2 = (double*)malloc(sizeof(double) * (size_t)h2);
    if (!a1 || !a2 || !d1 || !d2) {
        free(a1);
        free(a2);
        free(d1);
        free(d2);
        return LEEA_CPU_ENOMEM;
    }
    double sum = 0.0;
    for (int32_t r = 0; r < n; r++) {
        const double* xr = x + (int64_t)r * d_in;
        double y;
        mlp_row(d_in, h1, h2, theta, xr, a1, a2, &y);
        double e = y - t[r];
        sum += e * e;
        double dy = 2.0 * e / (double)n;            /* dL/dy_r */
        *gb3 += dy;
        for (int32_t u = 0; u < h2; u++) {
            gw3[u] += dy * a2[u];
            d2[u] = a2[u] > 0.0 ? dy * w3[u] : 0.0;  /* dL/dz2_u */
        }
        for (int32_t k = 0; k < h1; k++) d1[k] = 0.0;
        for (int32_t u = 0; u < h2; u++) {
            gb2[u] += d2[u];
            for (int32_t k = 0; k < h1; k++) {
                gW2[(int64_t)u * h1 + k] += d2[u] * a1[k];
                d1[k] += d2[u] * W2[(int64_t)u * h1 + k];
            }
        }
        for (int32_t u = 0; u < h1; u++) {
            double du = a1[u] > 0.0 ? d1[u] : 0.0;  /* dL/dz1_u */
            gb1[u] += du;
            for (int32_t k = 0; k < d_in; k++) gW1[(int64_t)u * d_in + k] += du * xr[k];
        }
    }
    *loss = sum / (double)n;
    free(a1);
    free(a2);
    free(d1);
    free(d2);
    return LEEA_CPU_OK;
}

/* One Adam step (Kingma & Ba, ICLR 2015) at step number `step` (1, 2, ...):
 * m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
 * theta <- theta - lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
int leea_cpu_adam(int64_t n_params, double* theta, const double* grad, double* m, double* v, int64_t step,
                  double lr, double beta1, double beta2, double eps)
{
    if (n_params < 0 || step < 1 || !theta || !grad || !m || !v) return LEEA_CPU_EINVAL;
    double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n_params; i++) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
    return LEEA_CPU_OK;
}

/* The recipes of one generation: mult x (n_C + n_M) virtual offspring.
 * Recipe r < mult n_C is a crossover, the rest mutations; recipe r draws
 * its parents (as a child of that kind in leea_cpu_select) and later its
 * genes from the streams of Philox entity LEEA_CPU_RECIPE_ENTITY0 + r. */
int leea_cpu_select_recipes(int32_t pop, const leea_cpu_params* prm, const double* f_adj,
                            const int32_t* order, uint64_t seed, uint32_t gen, int32_t mult,
                            int32_t* par1, int32_t* par2, int32_t* kind, double* f_inh, uint32_t* entity)
{
    if (pop <= 0 || mult < 1 || !valid_params(prm) || !f_adj || !order || !par1 || !par2 || !kind || !f_inh ||
        !entity)
        return LEEA_CPU_EINVAL;
    int32_t n_e, n_c, n_m, pool;
    leea_cpu_counts(pop, prm, &n_e, &n_c, &n_m, &pool);
    uint32_t k_draws = (prm->sel_op == 0) ? 1u : (uint32_t)prm->tour_k;
    int32_t n_r = mult * (n_c + n_m);
    for (int32_t r = 0; r < n_r; r++) {
        uint32_t ent = LEEA_CPU_RECIPE_ENTITY0 + (uint32_t)r;
        entity[r] = ent;
        if (r < mult * n_c) {
            kind[r] = LEEA_CPU_CROSSOVER;
            par1[r] = pick_parent(pop, prm, f_adj, order, pool, seed, gen, ent, 0);
            par2[r] = pick_parent(pop, prm, f_adj, order, pool, seed, gen, ent, k_draws);
            f_inh[r] = 0.5 * (f_adj[par1[r]] + f_adj[par2[r]]);
        } else {
            kind[r] = LEEA_CPU_MUTATION;
            par1[r] = pick_parent(pop, prm, f_adj, order, pool, seed, gen, ent, 0);
            par2[r] = par1[r];
            f_inh[r] = f_adj[par1[r]];
        }
    }
    return LEEA_CPU_OK;
}

/* n children with explicit Philox entities (leea_cpu_breed uses entity = j). */
int leea_cpu_breed_entities(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_cpu_params* prm,
                            uint64_t seed, uint32_t gen, const double* parents, const int32_t* par1,
                            const int32_t* par2, const int32_t* kind, const uint32_t* entity, int32_t n,
                            double* children)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || pop <= 0 || n < 0 || !valid_params(prm) || !parents || !par1 || !par2 || !kind || !entity ||
        (n > 0 && !children))
        return LEEA_CPU_EINVAL;
    for (int32_t j = 0; j < n; j++) {
        if (par1[j] < 0 || par1[j] >= pop || par2[j] < 0 || par2[j] >= pop) return LEEA_CPU_EINVAL;
        int rc = breed_child(c, prm, (double)prm->sigma, seed, gen, entity[j], kind[j], parents + (int64_t)par1[j] * c,
                             parents + (int64_t)par2[j] * c, children + (int64_t)j * c);
        if (rc != LEEA_CPU_OK) return rc;
    }
    return LEEA_CPU_OK;
}

/* How far a recipe moves from its first parent: the fraction of the c genes
 * a uniform crossover takes from parent 2 (0.5 for arithmetic crossover, 0
 * for a mutation or an elite), and the length sigma ||z (.) m|| of the
 * mutation step over the masked genes (0 unless a mutation). */
int leea_cpu_recipe_stats(const int32_t* dims, int32_t n_dims, const leea_cpu_params* prm, uint64_t seed,
                          uint32_t gen, const int32_t* kind, const uint32_t* entity, int32_t n, double* xo_frac,
                          double* mut_norm)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || n < 0 || !valid_params(prm) || (n > 0 && (!kind || !entity || !xo_frac || !mut_norm)))
        return LEEA_CPU_EINVAL;
    uint32_t thr_xo = leea_cpu_threshold16((double)prm->xo_gene_p);
    uint32_t thr_mut = leea_cpu_threshold16((double)prm->mut_rate);
    for (int32_t j = 0; j < n; j++) {
        xo_frac[j] = 0.0;
        mut_norm[j] = 0.0;
        if (kind[j] == LEEA_CPU_CROSSOVER) {
            if (prm->xo_op == 1) {
                xo_frac[j] = 0.5;
            } else {
                int64_t hits = 0;
                for (int64_t i = 0; i < c; i++)
                    if (leea_cpu_draw16(seed, LEEA_CPU_TAG_XO, gen, entity[j], (uint32_t)i) < thr_xo) hits++;
                xo_frac[j] = (double)hits / (double)c;
            }
        } else if (kind[j] == LEEA_CPU_MUTATION) {
            double ss = 0.0;
            for (int64_t i = 0; i < c; i++)
                if (leea_cpu_draw16(seed, LEEA_CPU_TAG_MUTMASK, gen, entity[j], (uint32_t)i) < thr_mut) {
                    double z = leea_cpu_normal(seed, LEEA_CPU_TAG_NORMAL, gen, entity[j], (uint32_t)i);
                    ss += z * z;
                }
            mut_norm[j] = (double)prm->sigma * sqrt(ss);
        }
    }
    return LEEA_CPU_OK;
}

/* Descriptor of each recipe (row of width 5 + n_probe d_out):
 * [f_adj of parent 1, f_adj of parent 2, f_inh, xo_frac, mut_norm, then the
 *  logits of the child (made by breed_child) on the n_probe probe inputs,
 *  sample-major].  Only two-layer nets (n_dims == 3). */
int leea_cpu_descriptors(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_cpu_params* prm,
                         uint64_t seed, uint32_t gen, const double* parents, const double* f_adj,
                         const int32_t* par1, const int32_t* par2, const int32_t* kind, const double* f_inh,
                         const uint32_t* entity, int32_t n, const double* probe_x, int32_t n_probe, double* desc)
{
    int64_t c = leea_cpu_num_params(dims, n_dims);
    if (c < 0 || n_dims != 3 || pop <= 0 || n < 0 || n_probe <= 0 || !valid_params(prm) || !parents || !f_adj ||
        !probe_x || (n > 0 && (!par1 || !par2 || !kind || !f_inh || !entity || !desc)))
        return LEEA_CPU_EINVAL;
    int32_t d_out = dims[2];
    int64_t width = 5 + (int64_t)n_probe * d_out;
    double* child = (double*)malloc(sizeof(double) * (size_t)c);
    double* logits = (double*)malloc(sizeof(double) * (size_t)n_probe * d_out);
    int32_t* y = (int32_t*)calloc((size_t)n_probe, sizeof(int32_t));
    if (!child || !logits || !y) {
        free(child);
        free(logits);
        free(y);
        return LEEA_CPU_ENOMEM;
    }
    int rc = LEEA_CPU_OK;
    for (int32_t j = 0; j < n && rc == LEEA_CPU_OK; j++) {
        if (par1[j] < 0 || par1[j] >= pop || par2[j] < 0 || par2[j] >= pop) {
            rc = LEEA_CPU_EINVAL;
            break;
        }
        double* row = desc + (int64_t)j * width;
        row[0] = f_adj[par1[j]];
        row[1] = f_adj[par2[j]];
        row[2] = f_inh[j];
        rc = leea_cpu_recipe_stats(dims, n_dims, prm, seed, gen, kind + j, entity + j, 1, row + 3, row + 4);
        if (rc == LEEA_CPU_OK)
            rc = breed_child(c, prm, (double)prm->sigma, seed, gen, entity[j], kind[j], parents + (int64_t)par1[j] * c,
                             parents + (int64_t)par2[j] * c, child);
        /* precision >= 1: the child's W1 as the precision form holds it, the
         * FP32 gene rounded to BF16 (nearest even) */
        if (rc == LEEA_CPU_OK && prm->precision >= 1)
            for (int64_t i = 0; i < (int64_t)dims[0] * dims[1]; i++) child[i] = leea_cpu_round_bf16((double)(float)child[i]);
        double f;
        if (rc == LEEA_CPU_OK) rc = leea_cpu_evaluate(1, dims, n_dims, child, probe_x, y, n_probe, &f, NULL, logits);
        for (int64_t k = 0; rc == LEEA_CPU_OK && k < (int64_t)n_probe * d_out; k++) row[5 + k] = logits[k];
    }
    free(child);
    free(logits);
    free(y);
    return rc;
}
