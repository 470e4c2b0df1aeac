/*
 * leea.h -- C ABI of the GB300 (sm_103a) LEEA library.
 *
 * The limited-evaluation evolutionary algorithm of Prellberg & Kramer,
 * "Limited Evaluation Evolutionary Optimization of Large Neural Networks"
 * (Algorithm 1, Sections 3.1-3.3): a population of `pop` directly encoded
 * fully connected nets is evaluated on one shared minibatch, then ranked,
 * selected, crossed over and mutated into the next generation, all on the GPU.
 *
 * Conventions for every entry point
 *  - Plain C types only.  Pointers named *_dev are CUDA device pointers, *_host
 *    are host pointers.  `stream` is a cudaStream_t passed as void* (NULL means
 *    the legacy default stream).
 *  - Every call returns a leea_status and never aborts; on failure
 *    leea_last_error() returns a message (thread-local, valid until the next
 *    failing call on the same thread).  Argument errors are reported before
 *    any work is enqueued.
 *  - Calls that take a stream only ENQUEUE work on it and return; inputs must
 *    stay valid and outputs untouched until the stream has reached the end of
 *    that work.  Calls that return host data synchronise the stream first.
 *  - Caller-owned buffers stay caller-owned; the library never frees them.
 *
 * Net and population layout (Section 3.2, direct encoding theta in R^c)
 *  - dims = {d_0, d_1, ..., d_L}: layer l maps d_l inputs to d_{l+1} outputs;
 *    every layer but the last is followed by ReLU, the last by softmax
 *    (Section 4.1).  The evaluation kernels take L = 2 (d_0-h-d_out, d_out <=
 *    32); initialisation and breeding take any 1 <= L <= 15.
 *  - Genes of one individual in logical order: for each layer, W_l as d_{l+1}
 *    rows of d_l floats (row-major, out x in), then b_l (d_{l+1} floats).
 *    c = sum_l (d_{l+1} d_l + d_{l+1}).
 *  - On the device an individual occupies c_pad = round_up(c, 32) floats so
 *    that each one starts 128-byte aligned: individual p starts at
 *    pop_dev + p * c_pad; genes c..c_pad-1 are zero.  Host copies made by
 *    leea_get_population / leea_best_params use the unpadded logical layout.
 *  - Minibatch: x is float[batch][d_0] row-major, y is int32[batch] with
 *    labels in [0, d_out).  A label outside that range makes the fitness of
 *    every individual NaN for that batch.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key
 * (seed & 0xffffffff, seed >> 32) and counter (n >> 2, entity, generation, tag);
 * draw n of a stream is word n & 3 of that block.  The per-gene crossover and
 * mutation masks use 16-bit draws instead: draw16 i is half i & 1 (the low
 * half for even i) of word (i >> 1) & 3 of block i >> 3, and it hits
 * probability q iff it is below floor(q 2^16) (always when q >= 1).  Because
 * the generator is counter-based, a run is reproducible from (seed,
 * generation) alone.
 */
#ifndef LEEA_H
#define LEEA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The library is built with hidden visibility; everything declared here is
 * exported. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef enum {
    LEEA_OK = 0,
    LEEA_EINVAL = 1,   /* invalid argument                                   */
    LEEA_ENOMEM = 2,   /* device or host allocation failed                   */
    LEEA_ECUDA = 3,    /* a CUDA call or kernel launch failed                */
    LEEA_ESTATE = 4,   /* call not valid in the object's current state       */
    LEEA_ETIMEOUT = 5  /* a bounded device wait gave up                      */
} leea_status;

/* Philox stream tags (counter word 3). */
enum {
    LEEA_TAG_INIT = 1,     /* entity = individual, n = gene index           */
    LEEA_TAG_SEL = 2,      /* entity = child, n = selection draw            */
    LEEA_TAG_XO = 3,       /* entity = child, n = gene index                */
    LEEA_TAG_MUTMASK = 4,  /* entity = child, n = gene index                */
    LEEA_TAG_NORMAL = 5,   /* entity = child, n = gene index                */
    LEEA_TAG_SIGMA = 7     /* entity = child, n = 0: self-adaptive sigma    */
};

/* How child j of the next generation is made (Algorithm 1). */
enum { LEEA_KIND_ELITE = 0, LEEA_KIND_CROSSOVER = 1, LEEA_KIND_MUTATION = 2 };

/* Operator parameters.  Defaults (leea_default_params) are the paper's
 * hyperparameter block of Section 4. */
typedef struct {
    int32_t xo_op;      /* 0 uniform crossover, 1 arithmetic (Section 3.2)    */
    float xo_gene_p;    /* uniform crossover: P(gene from parent 2); 0.5      */
    int32_t sel_op;     /* 0 truncation (Section 3.1), 1 tournament           */
    float rho;          /* truncation proportion rho in (0, 1]; 0.5           */
    int32_t tour_k;     /* tournament size (>= 1); 3                          */
    int32_t n_elite;    /* elite count; -1 => round(p_e * pop)                */
    float p_e;          /* elite proportion p_E; 0.05                         */
    float p_c;          /* crossover proportion p_C; 0.5; mutation the rest   */
    float sigma;        /* mutation strength sigma (constant); 0.001          */
    float mut_rate;     /* per-gene mutation probability; 1 = every gene      */
    float alpha;        /* inheritance weight alpha on the new fitness; 1     */
    int32_t init;       /* 0 N(0, 1/fan_in), 1 Glorot-uniform (Section 4.1)   */
    int32_t precision;  /* 0 FP32; 1 BF16 / 2 FP8-e4m3 shadow of W1, see below */
    int32_t eval_path;  /* LEEA_EVAL_AUTO / _SIMT / _TENSOR, see below        */
    int32_t sigma_ctl;  /* LEEA_SIGMA_CONST / _DECAY / _SELF, see below        */
    float sigma_k;      /* decay rate k (> 0) of LEEA_SIGMA_DECAY; 1          */
    float tau;          /* learning rate tau (>= 0) of LEEA_SIGMA_SELF; 0.1   */
} leea_params;

/* Control of the mutation strength (Section 3.2).
 *  - CONST: every breed mutates with sigma.
 *  - DECAY: breed number i (i = 0 for the first breed, generation counter
 *    g = i + 1) mutates with sigma 0.99^(i / sigma_k), computed in double on
 *    the host and rounded to FP32.
 *  - SELF: every individual carries a sigma gene, initially sigma.  A mutation
 *    child j first mutates its parent's gene, sigma_j = sigma_parent
 *    exp(tau z) with z the Box-Muller normal of draw 0 of the SIGMA stream of
 *    (g, j), then its weights with sigma_j; a crossover child takes the
 *    arithmetic mean of its parents' genes, an elite copies its own.  The
 *    genes are FP32 (expf on the device).
 * DECAY and SELF are properties of a run: the state object (leea_create)
 * applies them; the step entry points leea_select / leea_breed, the batching
 * form and the surrogate form take CONST only (LEEA_EINVAL otherwise). */
enum { LEEA_SIGMA_CONST = 0, LEEA_SIGMA_DECAY = 1, LEEA_SIGMA_SELF = 2 };

/* Evaluation kernels.  AUTO takes the tensor-core kernel when the shape
 * allows it (d_0 % 4 == 0, h % 16 == 0, h <= 256, d_out <= 16, 16-byte aligned
 * buffers) and the CUDA-core kernel otherwise.  SIMT: exact FP32 FFMA on the
 * CUDA cores.  TENSOR: tcgen05 tensor cores with a three-term TF32 split
 * (X_hi W_hi + X_hi W_lo + X_lo W_hi, FP32 accumulation), which is within
 * ~1e-6 relative of FP32; LEEA_EINVAL if the shape does not allow it.
 * FUSED (state object, 8-bit generation calls, precision 0): every breeding
 * generation makes and evaluates each child in one kernel
 * (leea_breed_evaluate_u8), so the evaluation does not read the new
 * population back from memory; the children are bit-identical to
 * leea_breed's.  It needs d_0 % 16 == 0, h % 16 == 0, h <= 128, d_out <= 16,
 * batch <= 128 (LEEA_EINVAL otherwise); the first evaluation uses the
 * tensor-core kernel.  AUTO keeps breeding and evaluation as two kernels.
 * SMALL (state object, 8-bit or FP32 generation calls, precision 0): the whole
 * generation -- ranking, selection, breeding, evaluation (Algorithm 1) -- in
 * one launch of one CTA per (child, 8 hidden units), each CTA ranking the
 * previous population itself and evaluating the slice it bred (layer 1 on
 * tensor-core tiles, levels exact, weights to 22 bits as in the TENSOR path);
 * the children are bit-identical to leea_breed's, the fitness within the
 * evaluation tolerance of the SIMT kernel's.  It
 * needs one hidden layer, h % 8 == 0, h <= 256, d_0 % 4 == 0, d_0 <= 2048,
 * d_out <= 32, batch <= 128, pop <= 1024, a 4-byte aligned 8-bit or 16-byte
 * aligned FP32 batch and the batch in shared memory (LEEA_EINVAL otherwise);
 * FP32 inputs enter layer 1 as two TF32 pieces as well.  AUTO takes it for such
 * generations when pop * h / 8 is at most twice the number of SMs, where the
 * chain of kernels would be bound by launch and dependency latency. */
enum { LEEA_EVAL_AUTO = 0, LEEA_EVAL_SIMT = 1, LEEA_EVAL_TENSOR = 2, LEEA_EVAL_FUSED = 3, LEEA_EVAL_SMALL = 4 };

/* Precision form (a throughput variant of Eq. 1; the paper itself computes in
 * FP32).  With precision 1 or 2 the population keeps its FP32 master, which
 * breeding updates exactly as in FP32 (small mutation steps are not rounded
 * away), and every individual also carries a shadow of its first-layer weights
 * W1 (genes 0 .. h d_0 - 1):
 *  - precision 1: BF16, round-to-nearest-even of the master;
 *  - precision 2: FP8-e4m3 of w / 2^e_p with saturation to +-448, where e_p is
 *    the individual's scale exponent, the smallest e with 448 2^e >= B_p for
 *    an upper bound B_p on max |W1_p|.  Shadows made from a whole population
 *    (leea_make_shadow, leea_create, leea_set_population) take B_p = the exact
 *    max |W1_p|.  Children take it from their parents' exact maxima: an elite
 *    its parent's, a crossover child the larger of its parents', a mutation
 *    child fmaf(sigma, 5.77, parent's) (5.77 bounds |z| of this library's
 *    normals).  Breeding records each child's exact max |W1| for the next
 *    generation.
 * Evaluation then multiplies 8-bit inputs x = k / x_div by the shadow on the
 * tensor cores with FP32 accumulation (the levels k are exact in BF16, and as
 * the two FP8 pieces 16 floor(k / 16) and k mod 16), scales by 2^e_p / x_div,
 * and computes b1, ReLU, layer 2 and the loss from the FP32 master in FP32.
 * Requirements: n_dims == 3, d_0 % 16 == 0, h % 16 == 0, h <= 256,
 * d_out <= 16 and A <= 496 with A = round_up(8 ceil(d_0 / 16), 16) for BF16
 * and round_up(16 ceil(d_0 / 32), 16) for FP8 (the batch tile's tensor-memory
 * columns; the hidden units are processed in chunks of at most 512 - A).
 * The state object then accepts only the 8-bit generation calls. */
enum { LEEA_PRECISION_FP32 = 0, LEEA_PRECISION_BF16 = 1, LEEA_PRECISION_FP8 = 2 };

/* Fills *out with the paper's defaults (Section 4). */
leea_status leea_default_params(leea_params* out);

/* ---------------------------------------------------------------------- */
/* Layout and operator counts                                              */
/* ---------------------------------------------------------------------- */

/* c, the number of genes of one individual of the layout `dims` (Section
 * 3.2: the direct encoding theta in R^c); -1 if dims is invalid.  The state
 * object's own c is leea_num_params(s). */
int64_t leea_layout_num_params(const int32_t* dims, int32_t n_dims);

/* c_pad = round_up(c, 32), the device stride between individuals; -1 if invalid. */
int64_t leea_padded_params(const int32_t* dims, int32_t n_dims);

/* Offspring counts of Algorithm 1: n_elite = n_elite param or round(p_E pop),
 * n_crossover = round(p_C pop) (clipped to pop - n_elite), n_mutation = the
 * rest; pool = max(1, floor(rho pop)), the truncation pool (Section 3.1).
 * Any output pointer may be NULL. */
leea_status leea_counts(int32_t pop, const leea_params* p, int32_t* n_elite,
                        int32_t* n_crossover, int32_t* n_mutation, int32_t* pool);

/* ---------------------------------------------------------------------- */
/* Step entry points on caller-owned device buffers (stream-ordered)        */
/* ---------------------------------------------------------------------- */

/* Random initial population (Algorithm 1's initial population; Section 4.1).
 * init 0: W ~ N(0, 1/d_l) by Box-Muller on the INIT stream; init 1:
 * Glorot-uniform W ~ U(-a, a), a = sqrt(6 / (d_l + d_{l+1})).  Biases and the
 * padding are zero.  pop_dev: float[pop][c_pad], written. */
leea_status leea_init_population(int32_t pop, const int32_t* dims, int32_t n_dims,
                                 int32_t init, uint64_t seed, float* pop_dev,
                                 void* stream);

/* Sort by fitness, descending (Algorithm 1).  order_dev[r] = index of the
 * r-th best individual; NaN ranks as -infinity, equal fitness goes to the
 * lower index.  f_adj_dev: float[pop] (read); order_dev: int32[pop] (written). */
leea_status leea_rank(int32_t pop, const float* f_adj_dev, int32_t* order_dev,
                      void* stream);

/* Parent selection and inherited fitness (Algorithm 1; Section 3.1).
 * Children 0..n_elite-1 are the elites order[j]; the next n_crossover
 * children get two parents, the rest one.  Truncation: each parent is
 * order[floor(u * pool / 2^32)] with u draw 0 (parent 1) or 1 (parent 2) of
 * the SEL stream of (gen, child).  Tournament: the best of tour_k draws
 * (indices floor(u * pop / 2^32), draws 0..k-1 for parent 1, k..2k-1 for
 * parent 2), ties to the lower index.  f_inh = (f1 + f2)/2 after crossover,
 * f3 after mutation, the elite's own f_adj for an elite.
 * Inputs f_adj_dev float[pop], order_dev int32[pop]; outputs par1_dev,
 * par2_dev, kind_dev int32[pop] and f_inh_dev float[pop].  p->precision must
 * be 0 and p->sigma_ctl LEEA_SIGMA_CONST here: the precision form's scale
 * exponents and the sigma genes come from the state object. */
leea_status leea_select(int32_t pop, const leea_params* p, const float* f_adj_dev,
                        const int32_t* order_dev, uint64_t seed, uint32_t gen,
                        int32_t* par1_dev, int32_t* par2_dev, int32_t* kind_dev,
                        float* f_inh_dev, void* stream);

/* Crossover and mutation (Section 3.2) into a separate children buffer.
 * For child j and gene i: elite -> copy of parent 1; uniform crossover ->
 * parent 2's gene iff XO draw16 i < floor(xo_gene_p 2^16), else parent 1's;
 * arithmetic crossover -> (a + b) / 2; mutation -> a + sigma z_i on genes whose
 * MUTMASK draw16 i < floor(mut_rate 2^16) (all genes when mut_rate = 1), with
 * z_i the Box-Muller normal of the NORMAL stream.  parents_dev and children_dev
 * are float[pop][c_pad] and must not overlap.  p->precision must be 0 here
 * (shadows of a bred population come from the state object or
 * leea_make_shadow), and p->sigma_ctl LEEA_SIGMA_CONST (a decaying strength is
 * passed as p->sigma of each call). */
leea_status leea_breed(int32_t pop, const int32_t* dims, int32_t n_dims,
                       const leea_params* p, uint64_t seed, uint32_t gen,
                       const float* parents_dev, const int32_t* par1_dev,
                       const int32_t* par2_dev, const int32_t* kind_dev,
                       float* children_dev, void* stream);

/* The input stage of the paper's network (Section 4.1): 2x2 max-pooling of
 * each image x[b] (h rows of w values, row-major; h and w even) into
 * out[b] ((h/2) x (w/2), row-major), out[i][j] = the largest of the pixels
 * (2i, 2j), (2i, 2j+1), (2i+1, 2j), (2i+1, 2j+1).  For 8-bit levels the max
 * of levels is a level, so pooling commutes with x = k / x_div.
 * x_dev: [batch][h*w]; out_dev: [batch][(h/2)*(w/2)]. */
leea_status leea_maxpool2x2(int32_t batch, int32_t h, int32_t w, const float* x_dev,
                            float* out_dev, void* stream);
leea_status leea_maxpool2x2_u8(int32_t batch, int32_t h, int32_t w, const uint8_t* x_dev,
                               uint8_t* out_dev, void* stream);

/* leea_breed followed by leea_evaluate_u8 of the children with inheritance
 * (Section 3.2, Eq. 1, Section 3.1), in one kernel: each child is made in
 * shared memory from its parents, written to children_dev and evaluated from
 * there on the tensor cores (8-bit inputs x = k / x_div; the numerics of
 * leea_evaluate_u8's tensor-core path, with layer 2 summed over the two
 * halves of the hidden units).  Children are bit-identical to leea_breed's.
 * n_dims == 3 with d_0 % 16 == 0, h % 16 == 0, h <= 128, d_out <= 16;
 * batch <= 128; parents_dev and children_dev 16-byte aligned and not
 * overlapping; p->precision 0 and p->sigma_ctl LEEA_SIGMA_CONST.  f_inh_dev
 * (float[pop], may be NULL for f_adj = f), f_raw_dev (written), f_adj_dev and
 * correct_dev (may be NULL). */
leea_status leea_breed_evaluate_u8(int32_t pop, const int32_t* dims, int32_t n_dims,
                                   const leea_params* p, uint64_t seed, uint32_t gen,
                                   const float* parents_dev, const int32_t* par1_dev,
                                   const int32_t* par2_dev, const int32_t* kind_dev,
                                   float* children_dev, const uint8_t* x_u8_dev, float x_div,
                                   const int32_t* y_dev, int32_t batch, float alpha,
                                   const float* f_inh_dev, float* f_raw_dev, float* f_adj_dev,
                                   int32_t* correct_dev, void* stream);

/* Fitness of every individual on one minibatch (Eq. 1) and inheritance
 * (Section 3.1).  f = -(1/batch) sum_b CE(softmax(z_b), y_b) computed in FP32
 * with the maximum subtracted; correct = #{b : argmax z_b = y_b} (ties to the
 * lowest class); f_adj = (1 - alpha) f_inh + alpha f, or f_adj = f when
 * f_inh_dev is NULL (the first evaluation).  Reductions have a fixed order,
 * so identical individuals get bitwise identical results.
 * n_dims == 3 (d_0-h-d_out with d_out <= 32), or n_dims > 3 with every layer
 * input and hidden width <= 256 and d_out <= 32 (the paper's 196-256-128-64-10,
 * Section 4.1), layer by layer with ReLU between layers.  Deeper nets take
 * the CUDA cores in exact FP32 (SIMT; AUTO for float inputs), or, for 8-bit
 * inputs and three hidden layers (widths multiples of 16 in [16, 256],
 * d_0 % 4 == 0, d_0 <= 256, d_out <= 16, 4-byte aligned x), the
 * tensor cores (AUTO or TENSOR): FP16 operand pieces of 2^8 w and 2^8 h
 * (hi.hi + hi.lo + lo.hi; the levels are exact), FP32 accumulation, FP32
 * bias, ReLU, last layer and loss; an individual with a weight or activation
 * |v| >= 128 is recomputed in FP32 on the CUDA cores.  That path splits the
 * weights and converts the batch into a library-owned scratch buffer (416 KB
 * per individual for 196-256-128-64-10, plus 64 KB per 128 samples), one per
 * device, shared by these step calls on that device, so such calls must not
 * overlap on one device; growing it frees the old buffer (which synchronises
 * the device).  The state object owns its own.  f_adj_dev and
 * correct_dev may be NULL; f_raw_dev may not.  eval_path: LEEA_EVAL_*. */
leea_status leea_evaluate(int32_t pop, const int32_t* dims, int32_t n_dims,
                          const float* pop_dev, const float* x_dev, const int32_t* y_dev,
                          int32_t batch, float alpha, const float* f_inh_dev,
                          float* f_raw_dev, float* f_adj_dev, int32_t* correct_dev,
                          int32_t eval_path, void* stream);

/* leea_evaluate for minibatches of 8-bit levels: x_u8_dev is uint8[batch][d_0]
 * and the input value is x = k / x_div (x_div = 255 for images stored as
 * bytes, as MNIST's are).  The tensor-core path needs batch <= 128,
 * d_0 % 4 == 0, h % 16 == 0, h <= 128 and d_out <= 16.  It forms layer 1 from
 * exact products: the levels are exact in FP16 and each weight, scaled by
 * 2^8, is split into two FP16 pieces (|2^8 w - w1 - w2| <= max(2^-22 2^8 |w|,
 * 2^-25), a 22-bit significand), so besides that split only the tensor
 * core's FP32 accumulation rounds; an individual with a weight |w| >= 128
 * gets its layer 1 in FP32 FFMA instead.  That path first writes the batch
 * as FP16 into a stream-ordered allocation of batch * round_up(d_0, 8) * 2
 * bytes (cudaMallocAsync on `stream`, freed after the evaluation).
 * Otherwise, or with LEEA_EVAL_SIMT, the CUDA-core kernel computes
 * x = k / x_div in FP32.  x_div must be finite and > 0. */
leea_status leea_evaluate_u8(int32_t pop, const int32_t* dims, int32_t n_dims,
                             const float* pop_dev, const uint8_t* x_u8_dev, float x_div,
                             const int32_t* y_dev, int32_t batch, float alpha,
                             const float* f_inh_dev, float* f_raw_dev, float* f_adj_dev,
                             int32_t* correct_dev, int32_t eval_path, void* stream);

/* Bytes between consecutive individuals' shadows for `precision` (1 or 2):
 * B h 128 with B = ceil(d_0 e / 128) blocks, e = 2 (BF16) or 1 (FP8); -1 if
 * the arguments are invalid.  A shadow is tiled for the tensor cores: block b
 * holds inputs [b w, (b + 1) w) (w = 128 / e) of all h rows of W1, 128 bytes
 * per row, row o at byte 128 (b h + o) of the shadow, and within a row the
 * 16-byte chunk c (inputs b w + c 16 / e ...) is stored at chunk position
 * c XOR (o mod 8).  Inputs past d_0 in the last block are zero. */
int64_t leea_shadow_stride(const int32_t* dims, int32_t n_dims, int32_t precision);

/* Shadows of a whole population (see "Precision form" above): for each p,
 * amax_dev[p] = max |W1_p| (float), scale_exp_dev[p] = e_p (precision 2 only;
 * may be NULL for precision 1) and the shadow at shadow_dev + p * stride
 * (stride = leea_shadow_stride; 128-byte aligned buffer), padding included. */
leea_status leea_make_shadow(int32_t pop, const int32_t* dims, int32_t n_dims, int32_t precision,
                             const float* pop_dev, uint8_t* shadow_dev, int32_t* scale_exp_dev,
                             float* amax_dev, void* stream);

/* Scratch bytes leea_evaluate_shadow_u8 needs for (pop, batch): 0 when
 * batch <= 128, else 8 * ceil(batch / 128) * pop (per-tile partial sums). */
int64_t leea_shadow_scratch_bytes(int32_t pop, int32_t batch);

/* leea_evaluate_u8 with layer 1 on the shadows: x_u8_dev uint8[batch][d_0],
 * pop_dev the FP32 master (b1, W2, b2 are read from it), shadow_dev and
 * scale_exp_dev as leea_make_shadow writes them (scale_exp_dev unused and may be
 * NULL for precision 1; the shadows' padding must be zero, as leea_make_shadow
 * leaves it), x_u8_dev 16-byte aligned.  A batch above 128 samples is split into tiles of 128
 * whose partial sums go to scratch_dev (caller-owned, scratch_bytes >=
 * leea_shadow_scratch_bytes(pop, batch); NULL/0 allowed when that is 0) and
 * are combined in tile order.  Other arguments and outputs as in
 * leea_evaluate_u8. */
leea_status leea_evaluate_shadow_u8(int32_t pop, const int32_t* dims, int32_t n_dims,
                                    const float* pop_dev, int32_t precision,
                                    const uint8_t* shadow_dev, const int32_t* scale_exp_dev,
                                    const uint8_t* x_u8_dev, float x_div, const int32_t* y_dev,
                                    int32_t batch, float alpha, const float* f_inh_dev,
                                    float* f_raw_dev, float* f_adj_dev, int32_t* correct_dev,
                                    float* scratch_dev, int64_t scratch_bytes, void* stream);

/* leea_evaluate_shadow_u8 for callers that cannot allocate or hand over
 * scratch memory -- e.g. a service whose device memory is fully committed to
 * a pool it does not control, or a loop whose latency budget excludes
 * allocator calls.  (The paper has no counterpart: this is a deployment
 * variant of the same evaluation.)  It allocates nothing: the per-tile
 * partial sums go to one static device array of this library, 1 MiB per
 * device (LEEA_NOALLOC_SCRATCH_BYTES), which holds batches and populations
 * with 8 * ceil(batch / 128) * pop <= 1 MiB; larger requests fail with
 * LEEA_EINVAL before any work is enqueued.  Nothing in that array needs to
 * start at zero: every slot the combining step reads is written earlier in
 * the same call.  There is one array per device, so calls whose device work
 * can overlap (other streams, other host threads, without an ordering
 * between them) race on it; order them, e.g. on one stream.  The first call
 * on a device looks up the array's address (with that device current; the
 * lookup is safe from several host threads); make that first call before
 * any stream capture.  Every call sets the kernel's shared-memory size
 * attribute.  No claim is made about use inside CUDA graph capture.  Other
 * arguments, requirements and results as in leea_evaluate_shadow_u8. */
#define LEEA_NOALLOC_SCRATCH_BYTES (1 << 20)
leea_status leea_evaluate_shadow_u8_noalloc(int32_t pop, const int32_t* dims, int32_t n_dims,
                                            const float* pop_dev, int32_t precision,
                                            const uint8_t* shadow_dev, const int32_t* scale_exp_dev,
                                            const uint8_t* x_u8_dev, float x_div, const int32_t* y_dev,
                                            int32_t batch, float alpha, const float* f_inh_dev,
                                            float* f_raw_dev, float* f_adj_dev, int32_t* correct_dev,
                                            void* stream);

/* Synchronises `stream`, then reads and clears this device's status word.
 * Returns LEEA_ETIMEOUT if a kernel's bounded wait gave up since the last
 * check (its outputs are then invalid), LEEA_OK otherwise.  flags_out, if
 * not NULL, receives the raw bits.  The state object's synchronising calls
 * (leea_fitness, leea_best_params, ...) perform the same check. */
leea_status leea_device_status(void* stream, uint32_t* flags_out);

/* Diagnostic of the failure path: enqueues a one-warp kernel whose thread
 * waits on a barrier that nothing completes, with the bounded wait the
 * pipelines use, limited to limit_us microseconds (1 .. 10^6).  When the wait
 * gives up it sets a status bit, so the next leea_device_status on that
 * stream returns LEEA_ETIMEOUT (flag 8) and clears it; the context stays
 * usable.  No fault is involved. */
leea_status leea_selftest_wait_timeout(uint32_t limit_us, void* stream);

/* Diagnostic: words n0 .. n0+count-1 of the Philox stream (tag, gen, ent),
 * written to out_dev (uint32[count]).  Lets a caller check the generator. */
leea_status leea_philox_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                             uint32_t n0, int64_t count, uint32_t* out_dev, void* stream);

/* Diagnostic: the Box-Muller normals z_i, i = n0 .. n0+count-1, of stream
 * (tag, gen, ent) as used by mutation and initialisation (float[count]). */
leea_status leea_normal_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                             uint32_t n0, int64_t count, float* out_dev, void* stream);

/* ---------------------------------------------------------------------- */
/* Algorithm 1 as a library-owned state object                             */
/* ---------------------------------------------------------------------- */

typedef struct leea_state leea_state;

/* Allocates two population buffers of pop x c_pad floats plus per-individual
 * arrays on the current device, and enqueues the initialisation on `stream`,
 * which every later call of this object uses.  *out receives the object.
 * Nets: n_dims == 3 with d_out <= 32, or n_dims > 3 (several hidden layers,
 * every layer input and hidden width <= 256, d_out <= 32; precision 0,
 * breeding and evaluation as separate kernels; evaluation as in
 * leea_evaluate / leea_evaluate_u8). */
leea_status leea_create(int32_t pop, const int32_t* dims, int32_t n_dims,
                        const leea_params* p, uint64_t seed, void* stream,
                        leea_state** out);

/* One generation of Algorithm 1 on the minibatch (x_dev, y_dev).  The first
 * call only evaluates the initial population (f_adj = f).  Every later call
 * increments the generation counter g, sorts by f_adj, selects, breeds into
 * the other buffer with the streams of generation g, swaps the buffers and
 * evaluates the new population with inheritance.  Enqueue only. */
leea_status leea_generation(leea_state* s, const float* x_dev, const int32_t* y_dev,
                            int32_t batch);

/* leea_generation with the minibatch in HOST memory: copies it to a
 * library-owned staging buffer on the object's stream, then runs the
 * generation.  Pageable host buffers are copied before the call returns;
 * pinned (page-locked) ones are read asynchronously and must stay unchanged
 * until the stream has reached the copy. */
leea_status leea_generation_host(leea_state* s, const float* x_host,
                                 const int32_t* y_host, int32_t batch);

/* leea_generation / leea_generation_host for minibatches of 8-bit levels
 * (x = k / x_div, see leea_evaluate_u8). */
leea_status leea_generation_u8(leea_state* s, const uint8_t* x_u8_dev, float x_div,
                               const int32_t* y_dev, int32_t batch);
leea_status leea_generation_u8_host(leea_state* s, const uint8_t* x_u8_host, float x_div,
                                    const int32_t* y_host, int32_t batch);

/* Adjusted fitness f_adj (float[pop]) and, if correct_host is not NULL, the
 * correct-prediction counts of the last evaluation.  f_adj is the fitness
 * Algorithm 1 sorts by: the blend (1 - alpha) f_inh + alpha f of Section 3.1
 * (fitness inheritance), or the raw f of Eq. 1 after the first call.
 * Caller-owned host buffers of pop elements.  Synchronises the object's
 * stream and checks the device status word first (LEEA_ETIMEOUT if a kernel
 * gave up a wait; the values are then invalid). */
leea_status leea_fitness(leea_state* s, float* f_adj_host, int32_t* correct_host);

/* Raw fitness f of the last evaluation, before inheritance.  Synchronises. */
leea_status leea_raw_fitness(leea_state* s, float* f_raw_host);

/* Genes (float[c], logical layout) of the individual with the highest f_adj
 * (ties to the lower index, NaN as -infinity): the head of Algorithm 1's
 * sorted population, the net the algorithm returns.  c must equal
 * leea_num_params(s) (LEEA_EINVAL otherwise), and LEEA_ESTATE before the
 * first generation call; out_host is caller-owned.
 * Synchronises. */
leea_status leea_best_params(leea_state* s, float* out_host, int64_t c);

/* Whole current population, float[pop][c] logical layout.  Synchronises. */
leea_status leea_get_population(leea_state* s, float* out_host);

/* Replaces the current population (float[pop][c] logical layout). */
leea_status leea_set_population(leea_state* s, const float* in_host);

/* Replaces the adjusted fitness vector (float[pop]). */
leea_status leea_set_fitness(leea_state* s, const float* f_adj_host);

/* Sets the generation counter and whether the population counts as evaluated
 * (checkpoint resume and lock-step testing). */
leea_status leea_set_generation(leea_state* s, uint32_t gen, int32_t evaluated);

/* Ranking and selection of the last breed: order, par1, par2, kind int32[pop]
 * and f_inh float[pop]; any pointer may be NULL.  Synchronises. */
leea_status leea_get_selection(leea_state* s, int32_t* order, int32_t* par1,
                               int32_t* par2, int32_t* kind, float* f_inh);

/* Precision form: the current population's shadows (uint8[pop][stride], the
 * tiled layout of leea_shadow_stride), and per individual the FP8 scale
 * exponents and exact max |W1| (any pointer may be NULL).  LEEA_ESTATE for an
 * FP32 object.  Synchronises. */
leea_status leea_get_shadow(leea_state* s, uint8_t* shadow_host, int32_t* scale_exp_host,
                            float* amax_host);

/* Generation counter g (0 before the first breed). */
uint32_t leea_generation_index(const leea_state* s);

/* Mutation strength of each individual of the current population
 * (float[pop]): its sigma gene under LEEA_SIGMA_SELF, otherwise the strength
 * the next breed uses.  Synchronises. */
leea_status leea_get_sigma(leea_state* s, float* sigma_host);

/* Replaces the sigma genes (float[pop], each finite and >= 0); LEEA_ESTATE
 * unless the object runs LEEA_SIGMA_SELF. */
leea_status leea_set_sigma(leea_state* s, const float* sigma_host);

/* c, the length of the genome theta in R^c of the object's nets (Section
 * 3.2's direct encoding: every weight and bias of the net is one gene), or
 * -1 for NULL. */
int64_t leea_num_params(const leea_state* s);

/* Per-stage timing with CUDA events recorded on the object's stream around
 * each kernel of leea_generation.  Stages: 0 ranking + selection (one fused
 * launch for pop <= 4096), 1 breeding (with the evaluation under
 * LEEA_EVAL_FUSED; the whole generation under the single-launch path, which
 * records nothing in stages 0 and 2 after the first evaluation), 2
 * evaluation (no launch after a fused breed). */
#define LEEA_NUM_STAGES 3
leea_status leea_profile_enable(leea_state* s, int32_t enable);

/* Synchronises, then returns per stage the summed kernel time in ms and the
 * number of launches since the last read, and resets both. */
leea_status leea_profile_read(leea_state* s, double* ms_out, int64_t* launches_out);

/* ---------------------------------------------------------------------- */
/* Batching form: many independent runs advanced together                   */
/* ---------------------------------------------------------------------- */

/* One run of the batching form: `pop` nets d_in-hidden-d_out (pop <= 4096),
 * minibatches of `batch` samples, its own seed (streams as in leea_create),
 * and the evaluation's tile, as an autotuner chooses it:
 *   chunk  hidden units per chunk of the layer-2 summation order (and, in the
 *          chunked evaluation, per tensor-core pass): a multiple of 16; 0 =
 *          the widest the tensor memory allows, the order the state object
 *          uses;
 *   group  individuals of the run sharing each MMA in the group evaluation
 *          (the tile's N = group hidden <= 256): 0 = the most that fit. */
typedef struct {
    int32_t pop, hidden, batch, chunk, group;
    uint64_t seed;
} leea_run_spec;

typedef struct leea_multi leea_multi;

/* Creates n_runs runs of Algorithm 1 that share d_in, d_out and the operator
 * parameters p; p->precision must be 1 or 2 (the batching form evaluates on
 * the tensor cores through BF16 or FP8 shadows; see "Precision form").  Each
 * run is initialised from its seed as leea_create would.  All later calls
 * enqueue on `stream`.  Minibatches and per-individual results are PACKED
 * over the runs: run r owns rows [batch_off[r], batch_off[r] + batch_r) of a
 * uint8[total_rows][d_in] minibatch (and of its int32[total_rows] labels),
 * and entries [pop_off[r], pop_off[r] + pop_r) of the float[total_pop]
 * fitness arrays (leea_multi_layout). */
leea_status leea_multi_create(int32_t n_runs, const leea_run_spec* runs, int32_t d_in, int32_t d_out,
                              const leea_params* p, void* stream, leea_multi** out);

/* Packed offsets (int64[n_runs] each, either may be NULL) and totals. */
leea_status leea_multi_layout(const leea_multi* m, int64_t* batch_off, int64_t* pop_off,
                              int64_t* total_rows, int64_t* total_pop);

/* The evaluation shape run `run` uses: hidden units per chunk, chunks per
 * individual, 128-sample tiles per batch and individuals per MMA of the
 * group evaluation (any pointer may be NULL). */
leea_status leea_multi_run_shape(const leea_multi* m, int32_t run, int32_t* chunk, int32_t* n_chunks,
                                 int32_t* m_tiles, int32_t* group);

/* Kernels one evaluation of all runs launches (a stage of
 * leea_multi_profile_read): 2 when every run takes the group evaluation
 * (several individuals per MMA: the batch staging, then the evaluation), 1
 * when the chunked evaluation is used; plus 1 (the combine of per-tile sums)
 * when some run's batch spans several 128-sample tiles. */
leea_status leea_multi_eval_launches(const leea_multi* m, int32_t* launches);

/* The object's own packed minibatch buffers.  A caller that writes the next
 * minibatch there (on the object's stream) saves the copy of
 * leea_multi_generation_u8. */
leea_status leea_multi_batch_buffers(leea_multi* m, uint8_t** x_dev, int32_t** y_dev);

/* One generation of every run on the packed minibatch (levels, x = k / x_div).
 * The first call evaluates every initial population.  Each later call
 * increments the common generation counter g and then, for all runs at once,
 * ranks and selects (one launch), breeds (one persistent launch over the work
 * items of every run) and evaluates (one persistent launch whose CTAs walk
 * precomputed segments of (run, sample tile, individuals)).  These launches
 * are captured into a CUDA graph on the first breeding call of each buffer
 * parity and replayed afterwards; the kernels read g from device memory.  A
 * call with another x_div rebuilds the evaluation tables and the graphs.
 * x_dev / y_dev are copied into the object's buffers unless they are those
 * buffers.  Enqueue only. */
leea_status leea_multi_generation_u8(leea_multi* m, const uint8_t* x_dev, float x_div, const int32_t* y_dev);

/* The same with the packed minibatch in host memory (copied on the stream). */
leea_status leea_multi_generation_u8_host(leea_multi* m, const uint8_t* x_host, float x_div,
                                          const int32_t* y_host);

/* Packed f_adj (and correct counts, if not NULL) of every run.  Synchronises. */
leea_status leea_multi_fitness(leea_multi* m, float* f_adj_host, int32_t* correct_host);

/* Packed raw fitness of the last evaluation.  Synchronises. */
leea_status leea_multi_raw_fitness(leea_multi* m, float* f_raw_host);

/* Run `run`'s current population, float[pop][c] logical layout.  Synchronises. */
leea_status leea_multi_get_population(leea_multi* m, int32_t run, float* out_host);

/* Replaces run `run`'s current population (its shadows are rebuilt). */
leea_status leea_multi_set_population(leea_multi* m, int32_t run, const float* in_host);

/* Replaces the packed f_adj of every run. */
leea_status leea_multi_set_fitness(leea_multi* m, const float* f_adj_host);

/* Sets the generation counter and whether the populations count as evaluated. */
leea_status leea_multi_set_generation(leea_multi* m, uint32_t gen, int32_t evaluated);

/* Run `run`'s ranking and selection of the last breed (any pointer may be
 * NULL; int32 / float arrays of its pop).  Synchronises. */
leea_status leea_multi_get_selection(leea_multi* m, int32_t run, int32_t* order, int32_t* par1,
                                     int32_t* par2, int32_t* kind, float* f_inh);

/* Run `run`'s current shadows (uint8[pop][leea_shadow_stride]), FP8 scale
 * exponents and exact max |W1| (any pointer may be NULL).  Synchronises. */
leea_status leea_multi_get_shadow(leea_multi* m, int32_t run, uint8_t* shadow_host, int32_t* scale_exp_host,
                                  float* amax_host);

/* Generation counter g (0 before the first breed). */
uint32_t leea_multi_generation_index(const leea_multi* m);

/* Per-stage timing: while enabled, generations run as direct launches (not
 * the graph) between CUDA events; stages as LEEA_NUM_STAGES, each stage one
 * launch covering every run. */
leea_status leea_multi_profile_enable(leea_multi* m, int32_t enable);
leea_status leea_multi_profile_read(leea_multi* m, double* ms_out, int64_t* launches_out);

/* Ends the run of Algorithm 1 held by the object: synchronises its stream,
 * then frees the object and all device memory it owns (both population
 * buffers and the per-individual arrays).  NULL is ignored.  Caller-owned
 * buffers (minibatches, the stream) are not touched. */
void leea_multi_destroy(leea_multi* m);

/* Autotuner support: mean time in ms of `reps` shadow evaluations of a
 * population of `pop` random nets d_in-hidden-d_out on a batch of `batch`
 * samples with `chunk` hidden units per pass, on the current device and
 * the legacy default stream.  Allocates and frees its own buffers. */
leea_status leea_tune_shadow_eval(int32_t precision, int32_t d_in, int32_t hidden, int32_t d_out, int32_t batch,
                                  int32_t pop, int32_t chunk, int32_t reps, float* ms_out);

/* Autotuner support: mean time in ms of `reps` group evaluations (batch
 * staging included) of `pop` random nets d_in-hidden-d_out on `batch`
 * samples with `group` individuals per MMA (1 .. min(16, 256 / hidden)), on
 * the current device and the legacy default stream.  LEEA_EINVAL when the
 * group evaluation does not take the shape.  Allocates and frees its own
 * buffers. */
leea_status leea_tune_group_eval(int32_t precision, int32_t d_in, int32_t hidden, int32_t d_out, int32_t batch,
                                 int32_t pop, int32_t group, int32_t reps, float* ms_out);

/* ---------------------------------------------------------------------- */
/* Surrogate form: the learned pre-screen of offspring (no counterpart in   */
/* the paper)                                                               */
/* ---------------------------------------------------------------------- */

/* Recipes: the virtual offspring of one generation, mult x (n_C + n_M) of
 * them (n_C, n_M as leea_counts gives them for pop).  Recipe r < mult n_C is
 * a crossover, the rest mutations.  Recipe r draws its parents like a child
 * of that kind in leea_select, and later its genes, from the Philox streams
 * of entity 2^30 + r.  -1 if the arguments are invalid. */
int32_t leea_num_recipes(int32_t pop, const leea_params* p, int32_t mult);

/* The recipes (int32 / float / uint32 arrays of leea_num_recipes entries) from
 * the population's f_adj_dev and its ranking order_dev (leea_rank); f_inh as
 * for a child of the same kind. */
leea_status leea_select_recipes(int32_t pop, const leea_params* p, const float* f_adj_dev, const int32_t* order_dev,
                                uint64_t seed, uint32_t gen, int32_t mult, int32_t* par1_dev, int32_t* par2_dev,
                                int32_t* kind_dev, float* f_inh_dev, uint32_t* entity_dev, void* stream);

/* leea_breed for n_children children of n_parents parents, child j drawing
 * from the Philox streams of entity entity_dev[j] (materialising recipes). */
leea_status leea_breed_entities(int32_t n_parents, const int32_t* dims, int32_t n_dims, const leea_params* p,
                                uint64_t seed, uint32_t gen, const float* parents_dev, const int32_t* par1_dev,
                                const int32_t* par2_dev, const int32_t* kind_dev, const uint32_t* entity_dev,
                                int32_t n_children, float* children_dev, void* stream);

/* Descriptors of n recipes, float[n][5 + n_probe d_out] (fused breed + probe:
 * the children's genes are made on the fly and never written):
 * [f_adj of parent 1, f_adj of parent 2, f_inh, the fraction of the c genes a
 * uniform crossover takes from parent 2 (0.5 arithmetic, 0 otherwise), the
 * mutation step length sigma ||z (.) m|| over the masked genes (0 otherwise),
 * then the child's logits on the probe inputs probe_dev (float[n_probe][d_0]),
 * sample-major].  entity_dev NULL: entity = recipe index.  Two-layer nets,
 * d_0 % 16 == 0, 16 <= h <= 256 with h % 16 == 0, d_out <= 16, n_probe <= 32.
 * p->precision 0: the logits of the FP32 child (CUDA cores); >= 1: of the
 * child with W1 rounded to BF16 (nearest even) as the precision form holds
 * it, on the tensor cores, the probe inputs carried as two BF16 pieces
 * (needs h <= 128; probe_dev 4-byte aligned). */
leea_status leea_descriptors(int32_t n_parents, const int32_t* dims, int32_t n_dims, const leea_params* p,
                             uint64_t seed, uint32_t gen, const float* parents_dev, const float* f_adj_dev,
                             const int32_t* par1_dev, const int32_t* par2_dev, const int32_t* kind_dev,
                             const float* f_inh_dev, const uint32_t* entity_dev, int32_t n,
                             const float* probe_dev, int32_t n_probe, float* desc_dev, void* stream);

/* The surrogate is an MLP d_in -> h1 -> h2 -> 1 with ReLU after the two
 * hidden layers, FP32.  Parameters theta, flat: W1 [h1][d_in] (row-major),
 * b1 [h1], W2 [h2][h1], b2 [h2], w3 [h2], b3 [1].  Every sum runs in a
 * fixed order, so results do not depend on scheduling. */
int64_t leea_surrogate_num_params(int32_t d_in, int32_t h1, int32_t h2);

/* Glorot-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)), from the
 * Philox stream (tag 6, generation 0, entity 0; draw n = parameter index);
 * zero biases.  theta_dev: float[leea_surrogate_num_params]. */
leea_status leea_surrogate_init(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, float* theta_dev,
                                void* stream);

/* y_dev[r] = MLP(x_dev[r]) for rows r < n of x_dev (float[n][d_in]). */
leea_status leea_surrogate_forward(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta_dev,
                                   const float* x_dev, float* y_dev, void* stream);

/* Floats of workspace leea_surrogate_loss_grad needs for n rows:
 * n (2 + 2 h1 + 2 h2). */
int64_t leea_surrogate_work_floats(int32_t n, int32_t h1, int32_t h2);

/* *loss_dev = (1/n) sum_r (y_r - t_r)^2 and grad_dev = its gradient with
 * respect to theta (backpropagation), for targets t_dev[n]. */
leea_status leea_surrogate_loss_grad(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta_dev,
                                     const float* x_dev, const float* t_dev, float* loss_dev, float* grad_dev,
                                     float* work_dev, int64_t work_floats, void* stream);

/* One Adam step (Kingma & Ba, ICLR 2015) at step number `step` (1, 2, ...):
 * m = beta1 m + (1 - beta1) g; v = beta2 v + (1 - beta2) g^2;
 * theta -= lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps). */
leea_status leea_surrogate_adam(int64_t n_params, float* theta_dev, const float* grad_dev, float* m_dev,
                                float* v_dev, int64_t step, float lr, float beta1, float beta2, float eps,
                                void* stream);

/* The surrogate form as a state object.  Every breeding generation:
 *  1. draws the recipes (leea_select_recipes, mult of them per offspring slot)
 *     and their descriptors (leea_descriptors on the probe inputs);
 *  2. standardises the descriptors (per-column mean and deviation over this
 *     generation's recipes, as fitness and logits drift while the population
 *     learns) and scores them with the MLP;
 *  3. fills the P - n_E offspring slots either with the best-scored recipes
 *     (the pre-screen) or, while the pre-screen is off, with the recipes the
 *     plain EA would make (the first n_C crossover and first n_M mutation
 *     recipes, ignoring the scores), and picks an audit sample of
 *     round(audit_frac (R - P + n_E)) of the other recipes, evenly spaced in
 *     score order (index order while the pre-screen is off);
 *  4. makes and evaluates the offspring and the audit sample;
 *  5. measures the Spearman correlation of scores and measured fitness over
 *     offspring + audit, which switches the pre-screen on for the next
 *     generation iff the generation index has reached `warmup` and the
 *     correlation is at least min_spearman; and
 *  6. appends the rows (standardised descriptor, fitness z-scored within the
 *     generation) to a ring of `history` generations and takes train_steps
 *     Adam steps on consecutive windows of train_batch rows.
 * No step waits for the host.  Elites are copied as in Algorithm 1. */
typedef struct {
    int32_t mult;           /* recipes per offspring slot; 4                         */
    int32_t n_probe;        /* probe inputs (1..32); 32                              */
    int32_t hidden1;        /* MLP hidden widths; 64, 64                             */
    int32_t hidden2;
    int32_t train_steps;    /* Adam steps per generation; 16                         */
    int32_t train_batch;    /* rows per step; 256                                    */
    int32_t history;        /* generations of rows kept; 4                           */
    int32_t warmup;         /* first generation that may use the pre-screen; 3       */
    float lr;               /* Adam learning rate; 1e-3 (betas 0.9, 0.999, eps 1e-8) */
    float audit_frac;       /* audit sample, fraction of the recipes left out; 0.05  */
    float min_spearman;     /* audit correlation needed for the pre-screen; 0.2      */
    uint64_t seed;          /* MLP initialisation                                    */
} leea_surrogate_params;

typedef struct leea_surr leea_surr;

leea_status leea_surrogate_default_params(leea_surrogate_params* out);

/* Creates the object for `pop` nets d_0-h-d_out (p->precision 0: FP32
 * evaluation, 1: BF16 shadows), initialised from `seed` as leea_create does,
 * with probe_host = float[n_probe][d_0] probe inputs (copied). */
leea_status leea_surr_create(int32_t pop, const int32_t* dims, int32_t n_dims, const leea_params* p,
                             const leea_surrogate_params* sp, uint64_t seed, const float* probe_host, void* stream,
                             leea_surr** out);
/* One generation (the first call only evaluates), minibatch of 8-bit levels. */
leea_status leea_surr_generation_u8(leea_surr* s, const uint8_t* x_dev, float x_div, const int32_t* y_dev,
                                    int32_t batch);
leea_status leea_surr_generation_u8_host(leea_surr* s, const uint8_t* x_host, float x_div, const int32_t* y_host,
                                         int32_t batch);
leea_status leea_surr_fitness(leea_surr* s, float* f_adj_host, int32_t* correct_host);
/* Raw fitness of the population and (if not NULL) of the audit sample. */
leea_status leea_surr_raw_fitness(leea_surr* s, float* f_raw_host, float* f_audit_host);
leea_status leea_surr_get_population(leea_surr* s, float* out_host);
leea_status leea_surr_set_population(leea_surr* s, const float* in_host);
leea_status leea_surr_set_fitness(leea_surr* s, const float* f_adj_host);
leea_status leea_surr_set_generation(leea_surr* s, uint32_t gen, int32_t evaluated);
/* Forces the pre-screen flag for the next generation (tests and ablations). */
leea_status leea_surr_set_screen(leea_surr* s, int32_t use_screen);
/* Recipes R, audit size, descriptor width and MLP parameter count. */
leea_status leea_surr_layout(const leea_surr* s, int32_t* n_recipes, int32_t* n_audit, int32_t* width,
                             int64_t* n_theta);
/* The last breeding generation's recipes, descriptors (float[R][width]),
 * scores, the recipe of each training row (offspring, then audit) and the
 * offspring slots' parents, kinds, entities and f_inh.  Any pointer may be
 * NULL.  Synchronises. */
leea_status leea_surr_get_step(leea_surr* s, int32_t* r_par1, int32_t* r_par2, int32_t* r_kind, float* r_f_inh,
                               uint32_t* r_entity, float* desc, float* pred, int32_t* row_recipe, int32_t* c_par1,
                               int32_t* c_par2, int32_t* c_kind, uint32_t* c_entity, float* c_f_inh);
/* The MLP parameters and the descriptor standardisation (any may be NULL). */
leea_status leea_surr_get_surrogate(leea_surr* s, float* theta_host, float* mu_host, float* sd_host);
/* Per breeding generation (the last min(n_max, count)): audit Spearman,
 * whether the pre-screen chose the offspring, and the last training loss. */
leea_status leea_surr_stats(leea_surr* s, int64_t n_max, float* spearman, int32_t* screened, float* loss,
                            int64_t* n_out);
/* Genes (float[c]) of the individual with the highest f_adj (ties to the
 * lower index, NaN as -infinity).  Synchronises. */
leea_status leea_surr_best_params(leea_surr* s, float* out_host, int64_t c);
uint32_t leea_surr_generation_index(const leea_surr* s);
/* Per-stage CUDA-event timing, five stages: recipes + descriptors, scores +
 * choice, breeding, evaluation, audit + training. */
#define LEEA_SURR_STAGES 5
leea_status leea_surr_profile_enable(leea_surr* s, int32_t enable);
leea_status leea_surr_profile_read(leea_surr* s, double* ms_out, int64_t* generations_out);
void leea_surr_destroy(leea_surr* s);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* leea_last_error(void);

/* Ends the run of Algorithm 1 held by the object: synchronises its stream,
 * then frees the object and all device memory it owns (both population
 * buffers and the per-individual arrays).  NULL is ignored.  Caller-owned
 * buffers (minibatches, the stream) are not touched. */
void leea_destroy(leea_state* s);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* LEEA_H */
