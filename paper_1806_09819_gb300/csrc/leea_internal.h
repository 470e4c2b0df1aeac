// leea_internal.h -- launch interface between the C ABI (leea_capi.cu) and the
// kernels.  Host-only declarations; every launcher enqueues on `stream` and
// returns the launch error (cudaSuccess when the launch was accepted).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace leea {

constexpr int kMaxLayers = 15;

// Launches `kernel` with programmatic stream serialisation: its CTAs may be
// scheduled while the previous kernel on the stream finishes, so the kernel
// must wait (griddepcontrol.wait) before it reads that kernel's results.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Bits of the device status word (set by kernels, read and cleared by the host).
constexpr unsigned int kStatusEvalTimeout = 1u;   // a bounded mbarrier wait of the tensor-core eval gave up
constexpr unsigned int kStatusBreedTimeout = 2u;  // a bounded mbarrier wait of the breed kernel gave up
constexpr unsigned int kStatusProbeTimeout = 4u;  // a bounded mbarrier wait of the tensor-core probe gave up
constexpr unsigned int kStatusSelftestTimeout = 8u;  // the self-test's wait gave up, as it is meant to

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

// Bound on |z| for a Box-Muller normal of this library: the radius
// sqrt(-2 ln u1) with u1 >= 2^-24 is at most 5.7683.
constexpr float kNormalBound = 5.77f;

struct SelectArgs {
    int32_t pop, n_elite, n_cross, pool;
    int32_t sel_op, tour_k;
    uint64_t seed;
    uint32_t gen;
    // precision form (precision 0: unused)
    int32_t precision;
    float sigma;
    const float* amax_in;     // exact max |W1| of each parent
    int32_t* scale_exp_out;   // FP8: exponent of each child's power-of-two scale
    float* amax_out;          // zeroed here; breed accumulates each child's max |W1|
    // self-adaptive mutation strength (NULL sigma_out: sigma above for every child)
    float tau;
    const float* sigma_in;    // parents' sigma genes
    float* sigma_out;         // children's sigma genes
};

struct BreedArgs {
    int32_t pop;
    int64_t c, c_pad;
    int32_t xo_op;
    uint32_t thr_xo, thr_mut;  // 16-bit draw thresholds floor(q 2^16), 2^16 when q >= 1
    float sigma;
    uint64_t seed;
    uint32_t gen;
    // precision form (precision 0: unused): shadow of W1 (genes 0 .. n_w1-1)
    int32_t precision;        // 1 BF16, 2 FP8-e4m3 scaled by 2^scale_exp[child]
    int64_t n_w1;             // multiple of 8
    int32_t sh_k, sh_h;       // d_0 and h: W1 is sh_h rows of sh_k
    uint8_t* shadow;          // child j's shadow at shadow + j * sh_stride (tiled, see shadow_offset)
    int64_t sh_stride;        // bytes, multiple of 128
    const int32_t* scale_exp;
    float* amax_out;          // atomic max of |W1| per child
    // surrogate form: child j draws from the streams of Philox entity entity[j]
    // (NULL: entity j); parents are indices below n_parents (0: pop)
    const uint32_t* entity;
    int32_t n_parents;
    // self-adaptive mutation strength: child j mutates with sigma_child[j] (NULL: sigma)
    const float* sigma_child;
};

// Tiled shadow layout.  An individual's W1 shadow is a sequence of blocks, one
// per 128 bytes of a row (64 BF16 or 128 FP8 inputs): block b holds K-elements
// [b kw, (b+1) kw) of all h rows, 128 bytes per row, with 16-byte chunk c of
// row o stored at chunk position c ^ (o & 7) -- the 128-byte swizzle the
// tensor core reads K-major operands in.  A block is thus copied to shared
// memory verbatim; elements past d_0 in the last block are zero.
__host__ __device__ inline int32_t shadow_blocks(int32_t k, int32_t elem) { return (k * elem + 127) / 128; }
__host__ __device__ inline int64_t shadow_stride_bytes(int32_t k, int32_t h, int32_t elem)
{
    return static_cast<int64_t>(shadow_blocks(k, elem)) * h * 128;
}
__host__ __device__ inline int64_t shadow_offset(int32_t h, int32_t elem, int32_t o, int32_t k)
{
    const int32_t byte = k * elem;  // within the row
    const int32_t b = byte >> 7, c = (byte >> 4) & 7, w = byte & 15;
    return (static_cast<int64_t>(b) * h + o) * 128 + (((c ^ (o & 7)) << 4) | w);
}

// Device exponent of the FP8 scale: smallest e with 448 * 2^e >= bound.
__host__ __device__ inline int32_t fp8_scale_exp(float bound)
{
    if (!(bound > 0.0f)) return 0;
    int ex = 0;
    frexpf(bound, &ex);            // bound in [2^(ex-1), 2^ex)
    const int32_t lead = ex - 1;
    return bound <= ldexpf(1.75f, lead) ? lead - 8 : lead - 7;
}

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

// Many runs at once (the batching form).  Each kernel reads the generation g
// from gen_dev, so that a captured CUDA graph replays with the next g.
struct SelectRun {
    SelectArgs a;  // a.gen unused
    const float* f_adj;
    int32_t *order, *par1, *par2, *kind;
    float* f_inh;
};
// CTA r: rank + select of run r (pop <= 4096).
cudaError_t launch_rank_select_runs(const SelectRun* runs_dev, int32_t n_runs, const uint32_t* gen_dev,
                                    cudaStream_t stream);
struct BreedRun {
    BreedArgs a;         // a.gen unused
    const float* parents;
    const int32_t *par1, *par2, *kind;
    float* children;
    int32_t chunks;      // work items per child
    int64_t item0;       // first of the run's pop * chunks items in the global list
};
cudaError_t launch_breed_runs(const BreedRun* runs_dev, int32_t n_runs, int64_t n_items, const uint32_t* gen_dev,
                              unsigned int* status, cudaStream_t stream);
// Items (chunks of genes) per child of a net with c_pad padded genes.
int32_t breed_chunks(int64_t c_pad);
// Precision form: shadows of W1 for a whole population from its FP32 master
// (exact max |W1| per individual, FP8 exponents from it).
cudaError_t launch_make_shadow(int32_t pop, int32_t k, int32_t h, int64_t c_pad, const float* pop_dev,
                               int32_t precision, uint8_t* shadow, int64_t sh_stride, int32_t* scale_exp, float* amax,
                               cudaStream_t stream);
// Evaluation of 8-bit inputs against BF16 / FP8 shadows of W1 (tcgen05).
// One run's evaluation problem; hidden units in n_chunks chunks of cw (the
// last one possibly narrower), batch in m_tiles tiles of 128 samples.
struct ShadowRun {
    int32_t pop, h, batch, m_tiles, cw, n_chunks;
    int64_t c_pad, sh_stride;
    float inv_div, alpha;
    const float* popv;
    const uint8_t* shadow;
    const uint8_t* x;
    const int32_t* y;
    const float* f_inh;
    const int32_t* scale_exp;
    float* f_raw;
    float* f_adj;
    int32_t* correct;
    float* scratch;  // m_tiles > 1: 2 m_tiles pop floats of per-tile partial sums
    // The group evaluation (batching form): the batch staged as operand tiles,
    // [m_tiles][k_blocks][pieces][128 rows][128 B], and individuals per MMA.
    const uint8_t* xop;
    int32_t group;
};
// Individuals [p0, p1) of run `run` on its 128-sample tile mt.
struct ShadowSeg {
    int32_t run, mt, p0, p1;
};
bool eval_shadow_supported(const NetLayout& net, int32_t precision, int32_t batch);
// The state object's shadow evaluation, two individuals per MMA (h <= 128,
// d_0 % 16 == 0, d_out <= 16): the batch staged by launch_stage_xop into
// xop (eval_shadow_pair_xop_bytes, 16-byte aligned) earlier on the stream;
// scratch as eval_shadow_scratch_bytes when the batch spans several
// 128-sample tiles.
bool eval_shadow_pair_supported(const NetLayout& net, int32_t precision, int32_t batch);
size_t eval_shadow_pair_xop_bytes(const NetLayout& net, int32_t precision, int32_t batch);
cudaError_t launch_stage_xop(const NetLayout& net, int32_t precision, const uint8_t* x, int32_t batch, void* xop,
                             cudaStream_t stream);
cudaError_t launch_eval_shadow_pair(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                                    const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp,
                                    const void* xop, float x_div, const int32_t* y, int32_t batch, float alpha,
                                    const float* f_inh, float* f_raw, float* f_adj, int32_t* correct, float* scratch,
                                    unsigned int* status, cudaStream_t stream);
size_t eval_shadow_scratch_bytes(int32_t pop, int32_t batch);
// Sums each run's per-tile partial losses (runs with m_tiles > 1) in tile order.
cudaError_t launch_combine_shadow_tiles(const ShadowRun* runs_dev, int32_t n_runs, int32_t pop_max,
                                        cudaStream_t stream);
cudaError_t launch_combine_shadow_run_tiles(const ShadowRun& run, cudaStream_t stream);
// The batching form's evaluation over a table of runs (h <= 256, h % 16 == 0,
// d_0 % 16 == 0, d_out <= 16): group = eval_shadow_group_size(h) individuals
// share every MMA (N = group h <= 256); each run's batch staged into its xop
// by launch_stage_xop_tiles earlier on the stream.
struct XopTile {
    const uint8_t* x;  // the tile's first sample (8-bit levels, d_0 per sample)
    int32_t rows;      // samples of the tile (1 .. 128); the rest are zero
    uint8_t* dst;      // [k_blocks][pieces][128 rows][128 B]
};
// One unit of the group evaluation: individuals [p, p + n) of run `run` on
// its 128-sample tile mt.  CTAs take units from the table in order through
// a device counter pair sched[2] (zero before the first launch; each launch
// leaves it at zero).
struct GroupUnit {
    int32_t run, mt, p, n;
};
int32_t eval_shadow_group_size(int32_t h);
// The group evaluation of one run (the state object, h > 128): the batch
// staged by launch_stage_xop into xop; sched: two int32 counters, zero before
// the first launch (each launch leaves them at zero); scratch as
// eval_shadow_scratch_bytes when the batch spans several 128-sample tiles.
cudaError_t launch_eval_shadow_group_run(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                                         const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp,
                                         const void* xop, float x_div, const int32_t* y, int32_t batch, float alpha,
                                         const float* f_inh, float* f_raw, float* f_adj, int32_t* correct,
                                         float* scratch, int32_t* sched, unsigned int* status, cudaStream_t stream);
bool eval_shadow_group_supported(int32_t k, int32_t d_out, int32_t precision, int32_t h, int32_t n_max);
size_t eval_shadow_group_xop_bytes(int32_t k, int32_t precision, int32_t batch);
cudaError_t launch_stage_xop_tiles(const XopTile* tiles_dev, int32_t n_tiles, int32_t k, int32_t precision,
                                   cudaStream_t stream);
cudaError_t launch_eval_shadow_group(int32_t k, int32_t d_out, int32_t precision, int32_t n_max,
                                     const ShadowRun* runs_dev, int32_t n_runs, int32_t pop_max, bool any_tiles,
                                     const GroupUnit* units_dev, int32_t n_units, int32_t* sched_dev, int32_t grid,
                                     unsigned int* status, cudaStream_t stream);
// Widest hidden chunk the tensor memory leaves room for next to the batch tile.
int32_t eval_shadow_max_chunk(int32_t precision, int32_t k);
// chunk: hidden units per chunk (multiple of 16), 0 for the widest.
ShadowRun shadow_run(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                     const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp, const uint8_t* x,
                     float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                     float* f_adj, int32_t* correct, float* scratch, int32_t chunk);
cudaError_t launch_eval_shadow(const NetLayout& net, int32_t pop, const float* pop_dev, int32_t precision,
                               const uint8_t* shadow, int64_t sh_stride, const int32_t* scale_exp,
                               const uint8_t* x, float x_div, const int32_t* y, int32_t batch, float alpha,
                               const float* f_inh, float* f_raw, float* f_adj, int32_t* correct, float* scratch,
                               unsigned int* status, cudaStream_t stream, int32_t chunk = 0);
// Many runs of d_0-h_r-d_out nets in one launch: runs_dev[n_runs], CTA b walks
// segs_dev[seg_off_dev[b] .. seg_off_dev[b+1]); h_max and cw_max bound every run's.
cudaError_t launch_eval_shadow_runs(int32_t k, int32_t d_out, int32_t precision, int32_t h_max, int32_t cw_max,
                                    int32_t n_runs, int32_t pop_max, bool any_tiles, const ShadowRun* runs_dev,
                                    const ShadowSeg* segs_dev, const int32_t* seg_off_dev, int32_t grid,
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
// tensor-core evaluation (two individuals per MMA, exact FP16 pieces) for
// batch <= 128, d_0 % 4 == 0, h % 16 == 0, h <= 128, d_out <= 16.  The
// tensor-core path reads the batch as FP16 from x16 (eval_u8_x16_bytes(net,
// batch) bytes, 16-byte aligned), which launch_stage_x16 fills from the levels
// earlier on the same stream; the staging kernel lets its successor start at
// once and waits for its own predecessor before it ends.
cudaError_t launch_eval_simt_u8(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                                float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                float* f_raw, float* f_adj, int32_t* correct, cudaStream_t stream);
bool eval_u8_tc_supported(const NetLayout& net, int32_t batch, const float* pop_dev);
size_t eval_u8_x16_bytes(const NetLayout& net, int32_t batch);
cudaError_t launch_stage_x16(const NetLayout& net, const uint8_t* x, int32_t batch, void* x16, cudaStream_t stream);
cudaError_t launch_eval_u8_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                              const void* x16, float x_div, const int32_t* y, int32_t batch, float alpha,
                              const float* f_inh, float* f_raw, float* f_adj, int32_t* correct, unsigned int* status,
                              cudaStream_t stream);
// Evaluation of nets with several hidden layers (n_dims >= 3; every layer
// input and hidden width <= 256, d_out <= 32), FP32 on the CUDA cores; and the
// 2x2 max-pooling input stage of the paper's network (h, w even).
bool eval_mlp_supported(const NetLayout& net);
cudaError_t launch_eval_mlp(const NetLayout& net, int32_t pop, const float* pop_dev, const float* x, const int32_t* y,
                            int32_t batch, float alpha, const float* f_inh, float* f_raw, float* f_adj,
                            int32_t* correct, cudaStream_t stream);
cudaError_t launch_eval_mlp_u8(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x, float x_div,
                               const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                               float* f_adj, int32_t* correct, cudaStream_t stream);
// The same, only for the individuals p with only[p] != 0.
cudaError_t launch_eval_mlp_u8_only(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x,
                                    float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                    float* f_raw, float* f_adj, int32_t* correct, const int32_t* only,
                                    cudaStream_t stream);
// Nets with three hidden layers (the paper's 196-256-128-64-10) on the tensor
// cores for 8-bit inputs: d0 % 4 == 0, d0 <= 256, hidden widths multiples of 16
// in [16, 256], d_out <= 16; FP32-class accuracy (FP16
// operand pieces), individuals with a weight or activation |v| >= 128
// recomputed in FP32 on the CUDA cores.
bool eval_mlp_tc_supported(const NetLayout& net, const float* pop_dev);
// Scratch of one evaluation: the weights as FP16 pieces, the marks and the
// batch's levels as FP16 operand tiles.
size_t eval_mlp_tc_scratch_bytes(const NetLayout& net, int32_t pop, int32_t batch);
// scratch: eval_mlp_tc_scratch_bytes(net, pop, batch) bytes of device memory owned by
// the caller, or NULL for a library-owned buffer shared by every such call
// (which must then not overlap on the device).
cudaError_t launch_eval_mlp_tc(const NetLayout& net, int32_t pop, const float* pop_dev, const uint8_t* x, float x_div,
                               const int32_t* y, int32_t batch, float alpha, const float* f_inh, float* f_raw,
                               float* f_adj, int32_t* correct, unsigned int* status, cudaStream_t stream,
                               void* scratch = nullptr);
cudaError_t launch_maxpool2x2(int32_t batch, int32_t h, int32_t w, const float* x, float* out, cudaStream_t stream);
cudaError_t launch_maxpool2x2_u8(int32_t batch, int32_t h, int32_t w, const uint8_t* x, uint8_t* out,
                                 cudaStream_t stream);
// Crossover, mutation and evaluation of every child in one kernel (8-bit
// inputs; d_0 % 16 == 0, h % 16 == 0, h <= 128, d_out <= 16, batch <= 128,
// 16-byte aligned populations).  Operators and streams from b (b.pop children
// of b.pop parents); results as launch_eval_u8_tc with the children.
bool breed_eval_u8_supported(const NetLayout& net, int32_t batch, const float* parents, const float* children);
cudaError_t launch_breed_eval_u8(const BreedArgs& b, const NetLayout& net, const float* parents, const int32_t* par1,
                                 const int32_t* par2, const int32_t* kind, float* children, const uint8_t* x,
                                 float x_div, const int32_t* y, int32_t batch, float alpha, const float* f_inh,
                                 float* f_raw, float* f_adj, int32_t* correct, unsigned int* status,
                                 cudaStream_t stream);
// One generation (ranking, selection, breeding, evaluation of 8-bit or FP32
// inputs) in a single launch for small FP32 populations of d_0-h-d_out nets: one CTA
// per (child, 8 hidden units).  Children bit-identical to breed_kernel's,
// fitness within FP32 rounding of eval_simt_kernel's.  f_adj_in and f_adj
// must not alias (every CTA ranks the whole previous population); count
// holds pop zeros between launches; part has room for pop x (h / 8) x batch
// x d_out floats.
struct SmallGenArgs {
    SelectArgs sel;          // breed: the selection (sigma as the breed's)
    BreedArgs br;            // breed: the operators and streams
    int32_t breed;           // 0: evaluate the population in popv (the first evaluation)
    int32_t pop, d_in, h, d_out, batch;
    int32_t n_slices, n_pow2, b2_units;  // set by the launcher
    int64_t region_floats;     // set by the launcher
    int64_t c, c_pad, b1_off, w2_off, b2_off;
    float x_div, alpha;
    const float* parents;    // breed: the previous population
    float* popv;             // the children (breed) or the population evaluated
    const float* f_adj_in;   // breed: the previous adjusted fitness
    int32_t *order, *par1, *par2, *kind;
    float* f_inh;
    float *f_raw, *f_adj;
    int32_t* correct;        // nullable
    float* part;             // [pop][h / 8][batch][d_out] partial logits of the slices
    uint32_t* count;         // [pop] arrivals per child
    const uint8_t* x;        // [batch][d_0] levels, 4-byte aligned (when xf is NULL)
    const float* xf;         // [batch][d_0] FP32 inputs, 16-byte aligned, or NULL
    const int32_t* y;
};
bool small_gen_supported(const NetLayout& net, int32_t pop, int32_t batch);
int32_t small_gen_ctas(const NetLayout& net, int32_t pop);
size_t small_gen_smem_bytes(int32_t d_in, int32_t h, int32_t d_out, int32_t batch, int32_t pop);
cudaError_t launch_small_gen(SmallGenArgs a, cudaStream_t stream);
// Surrogate form: recipes (virtual offspring) and their descriptors.
constexpr uint32_t kRecipeEntity0 = 0x40000000u;  // Philox entity of recipe r: kRecipeEntity0 + r
// Recipes r < mult n_cross are crossovers, the rest mutations; parents as
// select_child picks them, from the streams of entity kRecipeEntity0 + r.
cudaError_t launch_select_recipes(const SelectArgs& a, int32_t mult, const float* f_adj, const int32_t* order,
                                  int32_t* par1, int32_t* par2, int32_t* kind, float* f_inh, uint32_t* entity,
                                  cudaStream_t stream);
struct ProbeArgs {
    int32_t k, h, d_out, n_probe, width, xo_op;
    int32_t precision;       // 0: FP32 child (CUDA cores); >= 1: the child's W1 in BF16 (tensor cores)
    int64_t c, c_pad;
    uint32_t thr_xo, thr_mut, gen;
    float sigma;
    uint64_t seed;
    const float* parents;
    const float* f_adj;
    const int32_t *par1, *par2, *kind;
    const float* f_inh;
    const uint32_t* entity;  // NULL: entity = recipe index
    const float* probe;      // float[n_probe][k]
    float* desc;             // float[n][width], width = 5 + n_probe d_out
    unsigned int* status;    // device status word (bounded waits of the tensor-core probe)
};
bool probe_supported(int32_t k, int32_t h, int32_t d_out, int32_t n_probe, int32_t precision);
// precision 0: probe_kernel (leea_probe.cu); >= 1: probe_tc_kernel (leea_probe_tc.cu).
cudaError_t launch_descriptors(const ProbeArgs& a, int32_t n_recipes, cudaStream_t stream);
bool probe_tc_supported(int32_t k, int32_t h, int32_t d_out, int32_t n_probe);
cudaError_t launch_descriptors_tc(const ProbeArgs& a, int32_t n_recipes, cudaStream_t stream);

// Surrogate form: the MLP d_in -> h1 -> h2 -> 1 (leea_surrogate.cu).
int64_t surrogate_num_params(int32_t d_in, int32_t h1, int32_t h2);
size_t surrogate_forward_smem(int32_t d_in, int32_t h1, int32_t h2);
// Workspace of launch_surrogate_loss_grad, in floats.
size_t surrogate_work_floats(int32_t n, int32_t h1, int32_t h2);
cudaError_t launch_surrogate_init(int32_t d_in, int32_t h1, int32_t h2, uint64_t seed, float* theta,
                                  cudaStream_t stream);
// y[n] = MLP(x[n][d_in]); a1 [n][h1] and a2 [n][h2] (ReLU outputs) kept when not NULL.
cudaError_t launch_surrogate_forward(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta,
                                     const float* x, float* y, float* a1, float* a2, cudaStream_t stream);
// loss = mean (y - t)^2 and its gradient (all in-order sums).
cudaError_t launch_surrogate_loss_grad(int32_t n, int32_t d_in, int32_t h1, int32_t h2, const float* theta,
                                       const float* x, const float* t, float* loss, float* grad, float* work,
                                       cudaStream_t stream);
cudaError_t launch_surrogate_adam(int64_t n_params, float* theta, const float* grad, float* m, float* v, int64_t step,
                                  float lr, float beta1, float beta2, float eps, cudaStream_t stream);
// One training step of the state object: forward with the per-row deltas,
// the gradient with the Adam update (step number `step`) fused, and the loss
// only when `loss` is not NULL.  work: surrogate_work_floats(n, h1, h2).
cudaError_t launch_surrogate_train_step(int32_t n, int32_t d_in, int32_t h1, int32_t h2, float* theta, const float* x,
                                        const float* t, float* loss, float* work, float* m, float* v, int64_t step,
                                        float lr, float beta1, float beta2, float eps, cudaStream_t stream);

// The failure path of the bounded waits, exercised without a fault: one
// thread waits on an mbarrier that nothing completes, gives up after limit_ns
// and sets kStatusSelftestTimeout.
cudaError_t launch_wait_timeout_probe(uint64_t limit_ns, unsigned int* status, cudaStream_t stream);

cudaError_t launch_philox_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                               uint32_t n0, int64_t count, uint32_t* out, cudaStream_t stream);
cudaError_t launch_normal_fill(uint64_t seed, uint32_t tag, uint32_t gen, uint32_t ent,
                               uint32_t n0, int64_t count, float* out, cudaStream_t stream);

}  // namespace leea
