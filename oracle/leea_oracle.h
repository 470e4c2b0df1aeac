/*
 * leea_oracle.h -- FP64 CPU oracle of the LEEA hot path (Prellberg & Kramer,
 * "Limited Evaluation Evolutionary Optimization of Large Neural Networks").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * seeded inputs and the published definitions they both restate.
 *
 * Everything here is plain, slow, single-threaded C in double precision.
 * Each function names the passage of the paper it follows.
 *
 * Population layout on this side: pop[p * c + i], with the logical gene order
 * of a fully connected net dims[0]-dims[1]-...-dims[n-1]: for each layer l,
 * first W_l (dims[l+1] rows x dims[l] columns, row-major) then b_l.
 * (Section 3.2: the direct encoding theta in R^c.)
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed by
 * the 64-bit seed, with the counter (n >> 2, entity, generation, tag); scalar
 * draw n of a stream is word (n & 3) of that block.  The per-gene crossover
 * and mutation masks use 16-bit draws: draw16 i is half (i & 1) (low half for
 * even i) of word ((i >> 1) & 3) of block (i >> 3), and hits probability q iff
 * it is below floor(q 2^16) (2^16 when q >= 1).
 */
#ifndef LEEA_ORACLE_H
#define LEEA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LEEA_CPU_OK = 0,
    LEEA_CPU_EINVAL = 1,
    LEEA_CPU_ENOMEM = 2,
    LEEA_CPU_ESTATE = 4
};

/* Philox stream tags (counter word 3). */
enum {
    LEEA_CPU_TAG_INIT = 1,    /* entity = individual, n = gene              */
    LEEA_CPU_TAG_SEL = 2,     /* entity = child, n = draw index             */
    LEEA_CPU_TAG_XO = 3,      /* entity = child, n = gene                   */
    LEEA_CPU_TAG_MUTMASK = 4, /* entity = child, n = gene                   */
    LEEA_CPU_TAG_NORMAL = 5,  /* entity = child, n = gene                   */
    LEEA_CPU_TAG_SURR_INIT = 6, /* surrogate weights: entity 0, n = parameter */
    LEEA_CPU_TAG_SIGMA = 7      /* self-adaptive sigma: entity = child, n = 0 */
};

/* Control of the mutation strength (Section 3.2). */
enum { LEEA_CPU_SIGMA_CONST = 0, LEEA_CPU_SIGMA_DECAY = 1, LEEA_CPU_SIGMA_SELF = 2 };

/* Philox entity of recipe r of the surrogate form: LEEA_CPU_RECIPE_ENTITY0 + r. */
#define LEEA_CPU_RECIPE_ENTITY0 0x40000000u

/* How a child of the next generation is made (Algorithm 1). */
enum { LEEA_CPU_ELITE = 0, LEEA_CPU_CROSSOVER = 1, LEEA_CPU_MUTATION = 2 };

/* Operator parameters.  Same meaning as the CUDA library's leea_params, but a
 * separate declaration: the oracle includes nothing from the product. */
typedef struct {
    int32_t xo_op;     /* 0 uniform, 1 arithmetic crossover (Section 3.2)      */
    float xo_gene_p;   /* P(gene taken from parent 2), uniform crossover       */
    int32_t sel_op;    /* 0 truncation (Section 3.1), 1 tournament             */
    float rho;         /* truncation proportion                                */
    int32_t tour_k;    /* tournament size                                      */
    int32_t n_elite;   /* >= 0 explicit count; -1 => round(p_e * pop)          */
    float p_e;         /* elite proportion                                     */
    float p_c;         /* crossover proportion; mutation takes the rest        */
    float sigma;       /* mutation strength (constant control)                 */
    float mut_rate;    /* per-gene mutation probability (1 = every gene)       */
    float alpha;       /* inheritance weight on the fresh evaluation           */
    int32_t init;      /* 0 N(0, 1/fan_in), 1 Glorot-uniform (Section 4.1)     */
    int32_t precision; /* 0 FP32, 1 BF16 shadow, 2 FP8-e4m3 shadow             */
    int32_t sigma_ctl; /* LEEA_CPU_SIGMA_*: constant, decay, self-adaptive     */
    float sigma_k;     /* decay: sigma_i = sigma 0.99^(i / sigma_k)            */
    float tau;         /* self-adaptive: sigma' = sigma exp(tau N(0,1))        */
} leea_cpu_params;

/* ---- random number streams ------------------------------------------- */
void leea_cpu_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t leea_cpu_draw(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t n);
double leea_cpu_u01(uint32_t u);
double leea_cpu_normal(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t i);
uint32_t leea_cpu_index(uint32_t u, uint32_t m);
uint64_t leea_cpu_threshold(double q);
uint32_t leea_cpu_draw16(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent, uint32_t i);
uint32_t leea_cpu_threshold16(double q);

/* ---- layout and operator counts ----------------------------------------- */
int64_t leea_cpu_num_params(const int32_t* dims, int32_t n_dims);
int leea_cpu_counts(int32_t pop, const leea_cpu_params* prm, int32_t* n_e,
                    int32_t* n_c, int32_t* n_m, int32_t* pool);

/* ---- the steps of one generation (Algorithm 1) --------------------------- */
int leea_cpu_init(int32_t pop, const int32_t* dims, int32_t n_dims, int32_t init,
                  uint64_t seed, double* pop_out);
int leea_cpu_evaluate(int32_t pop, const int32_t* dims, int32_t n_dims,
                      const double* popv, const double* x, const int32_t* y,
                      int32_t batch, double* f_out, int32_t* correct_out,
                      double* logits_out);
/* The input stage of the paper's network (Section 4.1): 2x2 max-pooling of
 * each image x[b] (h rows of w pixels, row-major; h and w even) into
 * out[b] ((h/2) x (w/2), row-major): out[i][j] is the largest of the four
 * pixels (2i, 2j), (2i, 2j+1), (2i+1, 2j), (2i+1, 2j+1). */
int leea_cpu_maxpool2x2(int32_t batch, int32_t h, int32_t w, const double* x, double* out);
int leea_cpu_rank(int32_t pop, const double* f_adj, int32_t* order);
int leea_cpu_select(int32_t pop, const leea_cpu_params* prm, const double* f_adj,
                    const int32_t* order, uint64_t seed, uint32_t gen,
                    int32_t* par1, int32_t* par2, int32_t* kind, double* f_inh);
int leea_cpu_breed(int32_t pop, const int32_t* dims, int32_t n_dims,
                   const leea_cpu_params* prm, uint64_t seed, uint32_t gen,
                   const double* parents, const int32_t* par1, const int32_t* par2,
                   const int32_t* kind, int32_t j0, int32_t j1, double* children);
int leea_cpu_inherit(int32_t pop, double alpha, const double* f_inh, const double* f,
                     int32_t first, double* f_adj);

/* ---- control of the mutation strength (Section 3.2) ---------------------- */
/* Mutation strength of the breed with generation counter gen (>= 1), which is
 * breed number i = gen - 1: constant sigma, or sigma 0.99^(i / sigma_k) under
 * decay.  (Self-adaptive control has no schedule; this returns sigma, the
 * initial value of every sigma gene.) */
double leea_cpu_sigma_schedule(const leea_cpu_params* prm, uint32_t gen);
/* Self-adaptive control: the sigma gene of each child from its parents'.
 * Elite: a copy; crossover: the arithmetic mean of the parents' genes;
 * mutation: sigma_parent exp(tau z) with z the normal of draw 0 of the SIGMA
 * stream of (gen, child). */
int leea_cpu_select_sigma(int32_t pop, const leea_cpu_params* prm, uint64_t seed, uint32_t gen,
                          const int32_t* par1, const int32_t* par2, const int32_t* kind,
                          const double* sigma_in, double* sigma_out);
/* leea_cpu_breed with mutation strength sigma_child[j] for child j
 * (j0 <= j < j1; the array is indexed by the absolute child index). */
int leea_cpu_breed_sigma(int32_t pop, const int32_t* dims, int32_t n_dims,
                         const leea_cpu_params* prm, uint64_t seed, uint32_t gen,
                         const double* parents, const int32_t* par1, const int32_t* par2,
                         const int32_t* kind, const double* sigma_child, int32_t j0, int32_t j1,
                         double* children);

/* ---- precision form: reduced-precision shadows of W1 ---------------------- */
/* Round to nearest even into BF16 (8 significant bits, FP32's exponent range). */
double leea_cpu_round_bf16(double x);
/* Round to nearest even into FP8-e4m3 with saturation to +-448 (NaN stays NaN). */
double leea_cpu_round_e4m3(double x);
/* Exponent e of the power-of-two FP8 scale 2^e for an upper bound on |W1|:
 * the smallest e with 448 * 2^e >= bound (0 when bound <= 0). */
int32_t leea_cpu_fp8_scale_exp(double bound);
/* The population with W1 of every individual replaced by the value of its
 * shadow (the rule below); out may equal popv. */
int leea_cpu_quantize_w1(int32_t pop, const int32_t* dims, int32_t n_dims, const double* popv,
                         int32_t precision, const int32_t* scale_exp, double* out);
/* Fitness (Eq. 1) with W1 of every individual replaced by its shadow:
 * precision 1 -> round_bf16(w); precision 2 -> round_e4m3(w / 2^e_p) * 2^e_p
 * with the per-individual exponents scale_exp[p].  The rest of the net and the
 * arithmetic stay FP64. */
int leea_cpu_evaluate_shadow(int32_t pop, const int32_t* dims, int32_t n_dims,
                             const double* popv, int32_t precision, const int32_t* scale_exp,
                             const double* x, const int32_t* y, int32_t batch,
                             double* f_out, int32_t* correct_out);

/* ---- surrogate form (no counterpart in the paper) ------------------------- */
/* MLP d_in -> h1 -> h2 -> 1 with ReLU; parameters theta, flat:
 * W1 [h1][d_in], b1 [h1], W2 [h2][h1], b2 [h2], w3 [h2], b3. */
int64_t leea_cpu_mlp_num_params(int32_t d_in, int32_t h1, int32_t h2);
int leea_cpu_mlp_init(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, double* theta);
int leea_cpu_mlp_forward(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const double* theta,
                         const double* x, double* y);
/* L = mean (y - t)^2 and its gradient. */
int leea_cpu_mlp_loss_grad(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const double* theta,
                           const double* x, const double* t, double* loss, double* grad);
/* One Adam step (Kingma & Ba 2015) with bias correction, step = 1, 2, ... */
int leea_cpu_adam(int64_t n_params, double* theta, const double* grad, double* m, double* v, int64_t step,
                  double lr, double beta1, double beta2, double eps);
/* The mult (n_C + n_M) recipes of a generation: kinds, parents, f_inh, entities. */
int leea_cpu_select_recipes(int32_t pop, const leea_cpu_params* prm, const double* f_adj,
                            const int32_t* order, uint64_t seed, uint32_t gen, int32_t mult,
                            int32_t* par1, int32_t* par2, int32_t* kind, double* f_inh, uint32_t* entity);
/* n children with explicit Philox entities. */
int leea_cpu_breed_entities(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_cpu_params* prm,
                            uint64_t seed, uint32_t gen, const double* parents, const int32_t* par1,
                            const int32_t* par2, const int32_t* kind, const uint32_t* entity, int32_t n,
                            double* children);
/* Crossover fraction and mutation step length of each recipe. */
int leea_cpu_recipe_stats(const int32_t* dims, int32_t n_dims, const leea_cpu_params* prm, uint64_t seed,
                          uint32_t gen, const int32_t* kind, const uint32_t* entity, int32_t n, double* xo_frac,
                          double* mut_norm);
/* Descriptors [f1, f2, f_inh, xo_frac, mut_norm, probe logits (n_probe x d_out)].
 * prm->precision >= 1: the logits use the child's W1 rounded to FP32, then to
 * BF16 (nearest even), as the precision form holds it. */
int leea_cpu_descriptors(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_cpu_params* prm,
                         uint64_t seed, uint32_t gen, const double* parents, const double* f_adj,
                         const int32_t* par1, const int32_t* par2, const int32_t* kind, const double* f_inh,
                         const uint32_t* entity, int32_t n, const double* probe_x, int32_t n_probe, double* desc);

/* ---- the whole algorithm as a state object -------------------------------- */
typedef struct leea_cpu_state leea_cpu_state;
int leea_cpu_create(int32_t pop, const int32_t* dims, int32_t n_dims,
                    const leea_cpu_params* prm, uint64_t seed, leea_cpu_state** out);
int leea_cpu_generation(leea_cpu_state* s, const double* x, const int32_t* y, int32_t batch);
int leea_cpu_fitness(const leea_cpu_state* s, double* f_adj, double* f_raw, int32_t* correct);
int leea_cpu_best_params(const leea_cpu_state* s, double* out, int64_t c);
int leea_cpu_get_population(const leea_cpu_state* s, double* out);
int leea_cpu_set_population(leea_cpu_state* s, const double* in);
int leea_cpu_set_fitness(leea_cpu_state* s, const double* f_adj);
int leea_cpu_set_generation(leea_cpu_state* s, uint32_t gen, int32_t evaluated);
int leea_cpu_get_selection(const leea_cpu_state* s, int32_t* order, int32_t* par1,
                           int32_t* par2, int32_t* kind, double* f_inh);
uint32_t leea_cpu_generation_index(const leea_cpu_state* s);
/* Sigma of each individual of the current population: its sigma gene under
 * self-adaptive control, else the strength the next breed uses. */
int leea_cpu_get_sigma(const leea_cpu_state* s, double* out);
/* Replaces the sigma genes (self-adaptive control only, else ESTATE). */
int leea_cpu_set_sigma(leea_cpu_state* s, const double* in);
void leea_cpu_destroy(leea_cpu_state* s);

#ifdef __cplusplus
}
#endif
#endif /* LEEA_ORACLE_H */
