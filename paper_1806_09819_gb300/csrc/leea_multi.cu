// leea_multi.cu -- the batching form: many independent runs of Algorithm 1
// (each its own population size, hidden width, batch size and seed) advanced
// in lockstep generations.  Per generation, three persistent launches cover
// every run at once -- rank + selection (one CTA per run), breeding (work
// items of all runs in one list) and the shadow evaluation (each CTA walks
// its segments of (run, sample tile, individuals)) -- and they are captured
// once into a CUDA graph per buffer parity and replayed.  The kernels read
// the generation counter from device memory, which the graph itself
// advances, so a replay needs no new arguments.
#include "capi_common.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using namespace leea;
using namespace leea::capi;

namespace {

struct RunBuf {
    int32_t pop = 0, h = 0, batch = 0, chunk = 0;
    uint64_t seed = 0;
    NetLayout net{};
    int32_t m_tiles = 1, cw = 0, n_chunks = 1;
    int32_t group = 1;      // individuals per MMA in the group evaluation
    int64_t xop_off = 0;    // its staged batch tiles within leea_multi::xop
    int64_t batch_off = 0, pop_off = 0, sh_stride = 0;
    float* popbuf[2] = { nullptr, nullptr };
    uint8_t* shadow[2] = { nullptr, nullptr };
    float* amax[2] = { nullptr, nullptr };
    int32_t* scale_exp = nullptr;
    int32_t *order = nullptr, *par1 = nullptr, *par2 = nullptr, *kind = nullptr;
    float* scratch = nullptr;
};

__global__ void bump_generation_kernel(uint32_t* gen) { *gen += 1u; }

constexpr int kMultiProfRing = 4096;

}  // namespace

struct leea_multi {
    int32_t n_runs = 0, d_in = 0, d_out = 0;
    leea_params prm{};
    cudaStream_t stream = nullptr;
    std::vector<RunBuf> runs;
    int64_t total_rows = 0, total_pop = 0, breed_items = 0;
    int32_t h_max = 0, cw_max = 0, pop_max = 0, eval_grid = 0;
    bool any_tiles = false;
    // The group evaluation (several individuals per MMA) when every run fits
    // it, else the chunked kernel; its batch tiles, restaged every evaluation.
    bool grouped = false;
    int32_t n_max = 0;  // widest unit: max over runs of group h
    uint8_t* xop = nullptr;
    XopTile* xtiles = nullptr;
    int32_t n_xtiles = 0;
    GroupUnit* units = nullptr;  // the group evaluation's work, taken by CTAs in order
    int32_t n_units = 0;
    int32_t* sched = nullptr;    // its counters
    float *f_adj = nullptr, *f_raw = nullptr, *f_inh = nullptr;  // packed over the runs
    int32_t* correct = nullptr;
    uint8_t* x = nullptr;  // packed minibatch: the graph's fixed inputs
    int32_t* y = nullptr;
    uint32_t* gen_dev = nullptr;
    uint32_t gen = 0, gen_stage = 0;
    bool evaluated = false;
    int cur = 0;
    float x_div = 0.0f;  // of the current evaluation tables; 0 before the first call
    SelectRun* sel_tab[2] = { nullptr, nullptr };
    BreedRun* breed_tab[2] = { nullptr, nullptr };
    ShadowRun* eval_tab[3] = { nullptr, nullptr, nullptr };  // initial, after breeding from buffer 0, from 1
    ShadowSeg* segs = nullptr;
    int32_t* seg_off = nullptr;
    cudaGraphExec_t graph[2] = { nullptr, nullptr };
    cudaStream_t capture = nullptr;  // graphs are recorded here (the caller's stream may be the legacy one)
    // profiling: per stage (select, breed, evaluate) CUDA event pairs
    bool profiling = false;
    std::vector<cudaEvent_t> ev;  // [stage][2][ring]
    int n_prof[LEEA_NUM_STAGES] = {};
    double ms[LEEA_NUM_STAGES] = {};
    int64_t launches[LEEA_NUM_STAGES] = {};
};

namespace {

void free_multi(leea_multi* m)
{
    if (!m) return;
    for (RunBuf& r : m->runs) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(r.popbuf[b]);
            cudaFree(r.shadow[b]);
            cudaFree(r.amax[b]);
        }
        cudaFree(r.scale_exp);
        cudaFree(r.order);
        cudaFree(r.par1);
        cudaFree(r.par2);
        cudaFree(r.kind);
        cudaFree(r.scratch);
    }
    cudaFree(m->f_adj);
    cudaFree(m->f_raw);
    cudaFree(m->f_inh);
    cudaFree(m->correct);
    cudaFree(m->x);
    cudaFree(m->y);
    cudaFree(m->xop);
    cudaFree(m->xtiles);
    cudaFree(m->units);
    cudaFree(m->sched);
    cudaFree(m->gen_dev);
    for (int c = 0; c < 2; ++c) {
        cudaFree(m->sel_tab[c]);
        cudaFree(m->breed_tab[c]);
        if (m->graph[c]) cudaGraphExecDestroy(m->graph[c]);
    }
    for (int t = 0; t < 3; ++t) cudaFree(m->eval_tab[t]);
    cudaFree(m->segs);
    cudaFree(m->seg_off);
    if (m->capture) cudaStreamDestroy(m->capture);
    for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
    delete m;
}

template <typename T>
cudaError_t alloc(T** p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
}

template <typename T>
cudaError_t upload(T** dev, const std::vector<T>& host)
{
    if (!*dev) {
        cudaError_t err = alloc(dev, host.size());
        if (err != cudaSuccess) return err;
    }
    return cudaMemcpy(*dev, host.data(), sizeof(T) * host.size(), cudaMemcpyHostToDevice);
}

// Evaluation table `which`: 0 = the initial populations (buffer 0, no
// inheritance); 1 + c = after breeding from buffer c into buffer c ^ 1.
cudaError_t build_eval_table(leea_multi* m, int which, float x_div)
{
    std::vector<ShadowRun> tab(m->n_runs);
    const int buf = which == 0 ? 0 : ((which - 1) ^ 1);
    for (int32_t i = 0; i < m->n_runs; ++i) {
        RunBuf& r = m->runs[i];
        tab[i] = shadow_run(r.net, r.pop, r.popbuf[buf], m->prm.precision, r.shadow[buf], r.sh_stride, r.scale_exp,
                            m->x + r.batch_off * m->d_in, x_div, m->y + r.batch_off, r.batch, m->prm.alpha,
                            which == 0 ? nullptr : m->f_inh + r.pop_off, m->f_raw + r.pop_off,
                            m->f_adj + r.pop_off, m->correct + r.pop_off, r.scratch, r.cw);
        tab[i].xop = m->grouped ? m->xop + r.xop_off : nullptr;
        tab[i].group = r.group;
    }
    return upload(&m->eval_tab[which], tab);
}

cudaError_t build_step_tables(leea_multi* m, int c)
{
    std::vector<SelectRun> sel(m->n_runs);
    std::vector<BreedRun> br(m->n_runs);
    for (int32_t i = 0; i < m->n_runs; ++i) {
        RunBuf& r = m->runs[i];
        SelectRun& s = sel[i];
        s.a = select_args(r.pop, &m->prm, r.seed, 0);
        s.a.precision = m->prm.precision;
        s.a.sigma = m->prm.sigma;
        s.a.amax_in = r.amax[c];
        s.a.scale_exp_out = r.scale_exp;
        s.a.amax_out = r.amax[c ^ 1];
        s.f_adj = m->f_adj + r.pop_off;
        s.order = r.order;
        s.par1 = r.par1;
        s.par2 = r.par2;
        s.kind = r.kind;
        s.f_inh = m->f_inh + r.pop_off;
        BreedRun& b = br[i];
        b.a = breed_args(r.pop, r.net, &m->prm, r.seed, 0);
        b.a.precision = m->prm.precision;
        b.a.n_w1 = static_cast<int64_t>(r.net.dims[0]) * r.net.dims[1];
        b.a.sh_k = r.net.dims[0];
        b.a.sh_h = r.net.dims[1];
        b.a.shadow = r.shadow[c ^ 1];
        b.a.sh_stride = r.sh_stride;
        b.a.scale_exp = r.scale_exp;
        b.a.amax_out = r.amax[c ^ 1];
        b.parents = r.popbuf[c];
        b.par1 = r.par1;
        b.par2 = r.par2;
        b.kind = r.kind;
        b.children = r.popbuf[c ^ 1];
        b.chunks = breed_chunks(r.net.c_pad);
        b.item0 = 0;
    }
    int64_t item = 0;
    for (int32_t i = 0; i < m->n_runs; ++i) {
        br[i].item0 = item;
        item += static_cast<int64_t>(br[i].a.pop) * br[i].chunks;
    }
    m->breed_items = item;
    cudaError_t err = upload(&m->sel_tab[c], sel);
    if (err == cudaSuccess) err = upload(&m->breed_tab[c], br);
    return err;
}

// Splits the evaluation work -- (run, tile, individual) units in that order,
// each costing about its number of hidden chunks (chunked kernel) or 1/group
// of a pass over K (group kernel) -- into `grid` contiguous ranges of equal
// cost, one per CTA, cut into segments at run and tile edges.
cudaError_t build_segments(leea_multi* m, int grid)
{
    struct Block { int32_t run, mt, pop; double cost; };
    std::vector<Block> blocks;
    double total = 0.0;
    for (int32_t i = 0; i < m->n_runs; ++i) {
        const RunBuf& r = m->runs[i];
        for (int32_t mt = 0; mt < r.m_tiles; ++mt) {
            const double cost = m->grouped ? 1.0 / r.group : r.n_chunks + 0.25;
            blocks.push_back(Block{ i, mt, r.pop, cost });
            total += r.pop * cost;
        }
    }
    std::vector<ShadowSeg> segs;
    std::vector<int32_t> off(grid + 1, 0);
    size_t bi = 0;
    int32_t p = 0;  // next individual of blocks[bi]
    double done = 0.0;
    for (int g = 0; g < grid; ++g) {
        off[g] = static_cast<int32_t>(segs.size());
        const double target = total * (g + 1) / grid;
        while (bi < blocks.size() && (done < target - 1e-9 || g == grid - 1)) {
            const Block& b = blocks[bi];
            // individuals of this block that fit below the target (at least one)
            int32_t n = static_cast<int32_t>(std::ceil((target - done) / b.cost - 1e-9));
            if (g == grid - 1 || n > b.pop - p) n = b.pop - p;
            if (n < 1) n = 1;
            segs.push_back(ShadowSeg{ b.run, b.mt, p, p + n });
            done += n * b.cost;
            p += n;
            if (p == b.pop) {
                ++bi;
                p = 0;
            }
        }
    }
    off[grid] = static_cast<int32_t>(segs.size());
    if (segs.empty()) segs.push_back(ShadowSeg{ 0, 0, 0, 0 });
    cudaError_t err = upload(&m->segs, segs);
    if (err == cudaSuccess) err = upload(&m->seg_off, off);
    return err;
}

leea_status set_x_div(leea_multi* m, float x_div)
{
    if (m->x_div == x_div) return LEEA_OK;
    LEEA_CUDA_TRY(cudaStreamSynchronize(m->stream), "multi sync");
    for (int t = 0; t < 3; ++t) LEEA_CUDA_TRY(build_eval_table(m, t, x_div), "evaluation tables");
    for (int c = 0; c < 2; ++c)
        if (m->graph[c]) {
            cudaGraphExecDestroy(m->graph[c]);
            m->graph[c] = nullptr;
        }
    m->x_div = x_div;
    return LEEA_OK;
}

cudaError_t launch_eval(leea_multi* m, int which, unsigned int* status, cudaStream_t stream)
{
    if (m->grouped) {
        cudaError_t err = launch_stage_xop_tiles(m->xtiles, m->n_xtiles, m->d_in, m->prm.precision, stream);
        if (err != cudaSuccess) return err;
        return launch_eval_shadow_group(m->d_in, m->d_out, m->prm.precision, m->n_max, m->eval_tab[which], m->n_runs,
                                        m->pop_max, m->any_tiles, m->units, m->n_units, m->sched, m->eval_grid, status,
                                        stream);
    }
    return launch_eval_shadow_runs(m->d_in, m->d_out, m->prm.precision, m->h_max, m->cw_max, m->n_runs, m->pop_max,
                                   m->any_tiles, m->eval_tab[which], m->segs, m->seg_off, m->eval_grid, status,
                                   stream);
}

// One breeding generation from buffer c: the generation counter, then the
// three multi-run launches.  Enqueued directly, or recorded into a graph.
cudaError_t enqueue_step(leea_multi* m, int c, unsigned int* status, bool events, cudaStream_t stream)
{
    auto mark = [&](int stage, int e) {
        if (events) cudaEventRecord(m->ev[(stage * 2 + e) * kMultiProfRing + m->n_prof[stage]], stream);
    };
    bump_generation_kernel<<<1, 1, 0, stream>>>(m->gen_dev);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    mark(0, 0);
    err = launch_rank_select_runs(m->sel_tab[c], m->n_runs, m->gen_dev, stream);
    if (err != cudaSuccess) return err;
    mark(0, 1);
    mark(1, 0);
    err = launch_breed_runs(m->breed_tab[c], m->n_runs, m->breed_items, m->gen_dev, status, stream);
    if (err != cudaSuccess) return err;
    mark(1, 1);
    mark(2, 0);
    err = launch_eval(m, 1 + c, status, stream);
    if (err != cudaSuccess) return err;
    mark(2, 1);
    if (events)
        for (int st = 0; st < LEEA_NUM_STAGES; ++st) m->n_prof[st]++;
    return cudaSuccess;
}

leea_status prof_fold(leea_multi* m)
{
    LEEA_CUDA_TRY(cudaStreamSynchronize(m->stream), "profile sync");
    for (int st = 0; st < LEEA_NUM_STAGES; ++st) {
        for (int k = 0; k < m->n_prof[st]; ++k) {
            float ms = 0.0f;
            LEEA_CUDA_TRY(cudaEventElapsedTime(&ms, m->ev[(st * 2) * kMultiProfRing + k],
                                               m->ev[(st * 2 + 1) * kMultiProfRing + k]),
                          "profile elapsed");
            m->ms[st] += ms;
        }
        m->launches[st] += m->n_prof[st];
        m->n_prof[st] = 0;
    }
    return LEEA_OK;
}

leea_status run_multi_generation(leea_multi* m)
{
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    if (!m->evaluated) {
        LEEA_CUDA_TRY(launch_eval(m, 0, status, m->stream), "multi-run evaluate");
        m->evaluated = true;
        return LEEA_OK;
    }
    const int c = m->cur;
    if (m->profiling) {
        if (m->n_prof[0] == kMultiProfRing) {
            leea_status st = prof_fold(m);
            if (st) return st;
        }
        LEEA_CUDA_TRY(enqueue_step(m, c, status, true, m->stream), "multi-run generation");
    } else {
        if (!m->graph[c]) {
            LEEA_CUDA_TRY(cudaStreamBeginCapture(m->capture, cudaStreamCaptureModeRelaxed), "graph capture");
            const cudaError_t err = enqueue_step(m, c, status, false, m->capture);
            cudaGraph_t g = nullptr;
            const cudaError_t end = cudaStreamEndCapture(m->capture, &g);
            if (err != cudaSuccess || end != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(err != cudaSuccess ? err : end, "graph capture of a generation");
            }
            const cudaError_t inst = cudaGraphInstantiate(&m->graph[c], g, 0);
            cudaGraphDestroy(g);
            if (inst != cudaSuccess) {
                m->graph[c] = nullptr;
                return cuda_fail(inst, "graph instantiation");
            }
        }
        LEEA_CUDA_TRY(cudaGraphLaunch(m->graph[c], m->stream), "graph launch");
    }
    m->cur ^= 1;
    m->gen += 1;
    return LEEA_OK;
}

leea_status check_multi(const leea_multi* m)
{
    if (!m) return fail(LEEA_EINVAL, "multi-run object is NULL");
    return LEEA_OK;
}

leea_status check_run(const leea_multi* m, int32_t run)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (run < 0 || run >= m->n_runs) return fail(LEEA_EINVAL, "run %d not in [0, %d)", run, m->n_runs);
    return LEEA_OK;
}

cudaError_t refresh_run_shadow(leea_multi* m, RunBuf& r, int buf)
{
    return launch_make_shadow(r.pop, r.net.dims[0], r.net.dims[1], r.net.c_pad, r.popbuf[buf], m->prm.precision,
                              r.shadow[buf], r.sh_stride, r.scale_exp, r.amax[buf], m->stream);
}

}  // namespace

extern "C" {

leea_status leea_multi_create(int32_t n_runs, const leea_run_spec* specs, int32_t d_in, int32_t d_out,
                              const leea_params* p, void* stream, leea_multi** out)
{
    if (!out) return fail(LEEA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_runs < 1 || n_runs > 4096 || !specs) return fail(LEEA_EINVAL, "n_runs must be in [1, 4096] with specs");
    leea_status st = check_params(p);
    if (st) return st;
    if (p->precision != 1 && p->precision != 2)
        return fail(LEEA_EINVAL, "the batching form evaluates through BF16 or FP8 shadows: precision 1 or 2");
    if ((st = require_const_sigma(p, "the batching form"))) return st;
    leea_multi* m = new (std::nothrow) leea_multi();
    if (!m) return fail(LEEA_ENOMEM, "host allocation failed");
    m->n_runs = n_runs;
    m->d_in = d_in;
    m->d_out = d_out;
    m->prm = *p;
    m->stream = static_cast<cudaStream_t>(stream);
    m->runs.resize(n_runs);
    for (int32_t i = 0; i < n_runs; ++i) {
        RunBuf& r = m->runs[i];
        const leea_run_spec& sp = specs[i];
        const int32_t dims[3] = { d_in, sp.hidden, d_out };
        if (sp.pop < 1 || sp.pop > 4096 || sp.batch < 1 || !make_layout(dims, 3, p->init, &r.net)) {
            free_multi(m);
            return fail(LEEA_EINVAL, "run %d: pop must be in [1, 4096], batch >= 1 and the dims valid", i);
        }
        if ((st = check_shadow_shape(r.net, p->precision))) {
            free_multi(m);
            return st;
        }
        const int32_t cw_max = eval_shadow_max_chunk(p->precision, d_in);
        if (sp.chunk < 0 || sp.chunk % 16 != 0 || sp.chunk > cw_max) {
            free_multi(m);
            return fail(LEEA_EINVAL, "run %d: chunk must be 0 or a multiple of 16 up to %d", i, cw_max);
        }
        if (sp.group < 0 || sp.group > eval_shadow_group_size(sp.hidden)) {
            free_multi(m);
            return fail(LEEA_EINVAL, "run %d: group must be 0 or in [1, %d]", i, eval_shadow_group_size(sp.hidden));
        }
        r.pop = sp.pop;
        r.h = sp.hidden;
        r.batch = sp.batch;
        r.chunk = sp.chunk;
        r.seed = sp.seed;
        // chunk width and tiles as the evaluation kernel will use them
        const ShadowRun proto = shadow_run(r.net, r.pop, nullptr, p->precision, nullptr, 0, nullptr, nullptr, 1.0f,
                                           nullptr, r.batch, p->alpha, nullptr, nullptr, nullptr, nullptr, nullptr,
                                           r.chunk);
        r.cw = proto.cw;
        r.n_chunks = proto.n_chunks;
        r.m_tiles = proto.m_tiles;
        r.sh_stride = shadow_stride_of(r.net, p->precision);
        r.batch_off = m->total_rows;
        r.pop_off = m->total_pop;
        m->total_rows += r.batch;
        m->total_pop += r.pop;
        m->h_max = r.h > m->h_max ? r.h : m->h_max;
        m->cw_max = r.cw > m->cw_max ? r.cw : m->cw_max;
        m->pop_max = r.pop > m->pop_max ? r.pop : m->pop_max;
        m->any_tiles = m->any_tiles || r.m_tiles > 1;
        r.group = sp.group > 0 ? sp.group : eval_shadow_group_size(r.h);
        m->n_max = r.group * r.h > m->n_max ? r.group * r.h : m->n_max;
    }
    m->grouped = true;
    for (int32_t i = 0; i < n_runs; ++i)
        m->grouped = m->grouped && eval_shadow_group_supported(d_in, d_out, p->precision, m->runs[i].h, m->n_max);
    int64_t xop_bytes = 0;
    if (m->grouped) {
        for (int32_t i = 0; i < n_runs; ++i) {
            RunBuf& r = m->runs[i];
            r.xop_off = xop_bytes;
            xop_bytes += static_cast<int64_t>(eval_shadow_group_xop_bytes(d_in, p->precision, r.batch));
        }
    }
    cudaError_t err = cudaSuccess;
    for (int32_t i = 0; i < n_runs && err == cudaSuccess; ++i) {
        RunBuf& r = m->runs[i];
        const size_t np = static_cast<size_t>(r.pop);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = alloc(&r.popbuf[b], np * r.net.c_pad);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = alloc(&r.shadow[b], np * r.sh_stride);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) err = alloc(&r.amax[b], np);
        if (err == cudaSuccess) err = alloc(&r.scale_exp, np);
        if (err == cudaSuccess) err = alloc(&r.order, np);
        if (err == cudaSuccess) err = alloc(&r.par1, np);
        if (err == cudaSuccess) err = alloc(&r.par2, np);
        if (err == cudaSuccess) err = alloc(&r.kind, np);
        if (err == cudaSuccess && r.m_tiles > 1)
            err = alloc(&r.scratch, eval_shadow_scratch_bytes(r.pop, r.batch) / sizeof(float));
    }
    if (err == cudaSuccess) err = alloc(&m->f_adj, m->total_pop);
    if (err == cudaSuccess) err = alloc(&m->f_raw, m->total_pop);
    if (err == cudaSuccess) err = alloc(&m->f_inh, m->total_pop);
    if (err == cudaSuccess) err = alloc(&m->correct, m->total_pop);
    if (err == cudaSuccess) err = alloc(&m->x, static_cast<size_t>(m->total_rows) * d_in);
    if (err == cudaSuccess) err = alloc(&m->y, m->total_rows);
    if (err == cudaSuccess) err = alloc(&m->gen_dev, 1);
    if (err == cudaSuccess && m->grouped) {
        err = alloc(&m->xop, static_cast<size_t>(xop_bytes));
        // one staging tile per (run, 128-sample tile)
        const int64_t tile_bytes = static_cast<int64_t>(eval_shadow_group_xop_bytes(d_in, p->precision, 1));
        std::vector<XopTile> xt;
        for (int32_t i = 0; i < n_runs; ++i) {
            const RunBuf& r = m->runs[i];
            for (int32_t mt = 0; mt < r.m_tiles; ++mt)
                xt.push_back(XopTile{ m->x + (r.batch_off + 128 * mt) * d_in, std::min(128, r.batch - 128 * mt),
                                      m->xop + r.xop_off + mt * tile_bytes });
        }
        m->n_xtiles = static_cast<int32_t>(xt.size());
        if (err == cudaSuccess) err = upload(&m->xtiles, xt);
        // units: each group of individuals on all its sample tiles in turn
        std::vector<GroupUnit> units;
        for (int32_t i = 0; i < n_runs; ++i) {
            const RunBuf& r = m->runs[i];
            for (int32_t p0 = 0; p0 < r.pop; p0 += r.group)
                for (int32_t mt = 0; mt < r.m_tiles; ++mt)
                    units.push_back(GroupUnit{ i, mt, p0, std::min(r.group, r.pop - p0) });
        }
        m->n_units = static_cast<int32_t>(units.size());
        if (err == cudaSuccess) err = upload(&m->units, units);
        if (err == cudaSuccess) err = alloc(&m->sched, 2);
        if (err == cudaSuccess) err = cudaMemset(m->sched, 0, 2 * sizeof(int32_t));
    }
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&m->capture, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
        free_multi(m);
        return cuda_fail(err, "leea_multi_create allocation");
    }
    // initial populations (as leea_create), their shadows, zeroed padding
    err = cudaMemsetAsync(m->gen_dev, 0, sizeof(uint32_t), m->stream);
    for (int32_t i = 0; i < n_runs && err == cudaSuccess; ++i) {
        RunBuf& r = m->runs[i];
        const size_t np = static_cast<size_t>(r.pop);
        err = cudaMemsetAsync(r.popbuf[1], 0, sizeof(float) * np * r.net.c_pad, m->stream);
        for (int b = 0; b < 2 && err == cudaSuccess; ++b)
            err = cudaMemsetAsync(r.shadow[b], 0, np * r.sh_stride, m->stream);
        if (err == cudaSuccess) err = cudaMemsetAsync(r.scale_exp, 0, sizeof(int32_t) * np, m->stream);
        if (err == cudaSuccess) err = launch_init(r.net, r.pop, p->init, r.seed, r.popbuf[0], m->stream);
        if (err == cudaSuccess) err = refresh_run_shadow(m, r, 0);
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(m->stream);
    for (int c = 0; c < 2 && err == cudaSuccess; ++c) err = build_step_tables(m, c);
    if (err == cudaSuccess) {
        int dev = 0, sms = 0;
        err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        m->eval_grid = sms;
        if (err == cudaSuccess) err = build_segments(m, sms);
    }
    if (err != cudaSuccess) {
        free_multi(m);
        return cuda_fail(err, "leea_multi_create setup");
    }
    *out = m;
    return LEEA_OK;
}

leea_status leea_multi_layout(const leea_multi* m, int64_t* batch_off, int64_t* pop_off, int64_t* total_rows,
                              int64_t* total_pop)
{
    leea_status st = check_multi(m);
    if (st) return st;
    for (int32_t i = 0; i < m->n_runs; ++i) {
        if (batch_off) batch_off[i] = m->runs[i].batch_off;
        if (pop_off) pop_off[i] = m->runs[i].pop_off;
    }
    if (total_rows) *total_rows = m->total_rows;
    if (total_pop) *total_pop = m->total_pop;
    return LEEA_OK;
}

leea_status leea_multi_run_shape(const leea_multi* m, int32_t run, int32_t* chunk, int32_t* n_chunks,
                                 int32_t* m_tiles, int32_t* group)
{
    leea_status st = check_run(m, run);
    if (st) return st;
    if (chunk) *chunk = m->runs[run].cw;
    if (n_chunks) *n_chunks = m->runs[run].n_chunks;
    if (m_tiles) *m_tiles = m->runs[run].m_tiles;
    if (group) *group = m->runs[run].group;
    return LEEA_OK;
}

leea_status leea_multi_eval_launches(const leea_multi* m, int32_t* launches)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (!launches) return fail(LEEA_EINVAL, "launches is NULL");
    *launches = (m->grouped ? 2 : 1) + (m->any_tiles ? 1 : 0);
    return LEEA_OK;
}

leea_status leea_multi_batch_buffers(leea_multi* m, uint8_t** x_dev, int32_t** y_dev)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (x_dev) *x_dev = m->x;
    if (y_dev) *y_dev = m->y;
    return LEEA_OK;
}

leea_status leea_multi_generation_u8(leea_multi* m, const uint8_t* x_dev, float x_div, const int32_t* y_dev)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (!x_dev || !y_dev) return fail(LEEA_EINVAL, "NULL minibatch pointer");
    if (!(x_div > 0.0f) || std::isinf(x_div)) return fail(LEEA_EINVAL, "x_div must be finite and > 0");
    if ((st = set_x_div(m, x_div))) return st;
    if (x_dev != m->x)
        LEEA_CUDA_TRY(cudaMemcpyAsync(m->x, x_dev, static_cast<size_t>(m->total_rows) * m->d_in,
                                      cudaMemcpyDeviceToDevice, m->stream),
                      "minibatch copy");
    if (y_dev != m->y)
        LEEA_CUDA_TRY(cudaMemcpyAsync(m->y, y_dev, sizeof(int32_t) * m->total_rows, cudaMemcpyDeviceToDevice,
                                      m->stream),
                      "label copy");
    return run_multi_generation(m);
}

leea_status leea_multi_generation_u8_host(leea_multi* m, const uint8_t* x_host, float x_div, const int32_t* y_host)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (!x_host || !y_host) return fail(LEEA_EINVAL, "NULL minibatch pointer");
    if (!(x_div > 0.0f) || std::isinf(x_div)) return fail(LEEA_EINVAL, "x_div must be finite and > 0");
    if ((st = set_x_div(m, x_div))) return st;
    LEEA_CUDA_TRY(cudaMemcpyAsync(m->x, x_host, static_cast<size_t>(m->total_rows) * m->d_in, cudaMemcpyHostToDevice,
                                  m->stream),
                  "minibatch copy");
    LEEA_CUDA_TRY(cudaMemcpyAsync(m->y, y_host, sizeof(int32_t) * m->total_rows, cudaMemcpyHostToDevice, m->stream),
                  "label copy");
    return run_multi_generation(m);
}

leea_status leea_multi_fitness(leea_multi* m, float* f_adj_host, int32_t* correct_host)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (!m->evaluated) return fail(LEEA_ESTATE, "no generation has been evaluated yet");
    if (!f_adj_host) return fail(LEEA_EINVAL, "f_adj_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpyAsync(f_adj_host, m->f_adj, sizeof(float) * m->total_pop, cudaMemcpyDeviceToHost,
                                  m->stream),
                  "fitness copy");
    if (correct_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(correct_host, m->correct, sizeof(int32_t) * m->total_pop,
                                      cudaMemcpyDeviceToHost, m->stream),
                      "correct copy");
    return check_device_status(m->stream, nullptr);
}

leea_status leea_multi_raw_fitness(leea_multi* m, float* f_raw_host)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (!m->evaluated) return fail(LEEA_ESTATE, "no generation has been evaluated yet");
    if (!f_raw_host) return fail(LEEA_EINVAL, "f_raw_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpyAsync(f_raw_host, m->f_raw, sizeof(float) * m->total_pop, cudaMemcpyDeviceToHost,
                                  m->stream),
                  "raw fitness copy");
    return check_device_status(m->stream, nullptr);
}

leea_status leea_multi_get_population(leea_multi* m, int32_t run, float* out_host)
{
    leea_status st = check_run(m, run);
    if (st) return st;
    if (!out_host) return fail(LEEA_EINVAL, "out_host is NULL");
    RunBuf& r = m->runs[run];
    LEEA_CUDA_TRY(cudaMemcpy2DAsync(out_host, sizeof(float) * r.net.c, r.popbuf[m->cur], sizeof(float) * r.net.c_pad,
                                    sizeof(float) * r.net.c, r.pop, cudaMemcpyDeviceToHost, m->stream),
                  "population copy");
    return check_device_status(m->stream, nullptr);
}

leea_status leea_multi_set_population(leea_multi* m, int32_t run, const float* in_host)
{
    leea_status st = check_run(m, run);
    if (st) return st;
    if (!in_host) return fail(LEEA_EINVAL, "in_host is NULL");
    RunBuf& r = m->runs[run];
    LEEA_CUDA_TRY(cudaMemcpy2DAsync(r.popbuf[m->cur], sizeof(float) * r.net.c_pad, in_host, sizeof(float) * r.net.c,
                                    sizeof(float) * r.net.c, r.pop, cudaMemcpyHostToDevice, m->stream),
                  "population copy");
    LEEA_CUDA_TRY(refresh_run_shadow(m, r, m->cur), "make shadow kernel");
    LEEA_CUDA_TRY(cudaStreamSynchronize(m->stream), "population sync");
    return LEEA_OK;
}

leea_status leea_multi_set_fitness(leea_multi* m, const float* f_adj_host)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (!f_adj_host) return fail(LEEA_EINVAL, "f_adj_host is NULL");
    LEEA_CUDA_TRY(cudaMemcpyAsync(m->f_adj, f_adj_host, sizeof(float) * m->total_pop, cudaMemcpyHostToDevice,
                                  m->stream),
                  "fitness copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(m->stream), "fitness sync");
    return LEEA_OK;
}

leea_status leea_multi_set_generation(leea_multi* m, uint32_t gen, int32_t evaluated)
{
    leea_status st = check_multi(m);
    if (st) return st;
    m->gen = gen;
    m->gen_stage = gen;
    m->evaluated = evaluated != 0;
    LEEA_CUDA_TRY(cudaMemcpyAsync(m->gen_dev, &m->gen_stage, sizeof(uint32_t), cudaMemcpyHostToDevice, m->stream),
                  "generation copy");
    LEEA_CUDA_TRY(cudaStreamSynchronize(m->stream), "generation sync");
    return LEEA_OK;
}

leea_status leea_multi_get_selection(leea_multi* m, int32_t run, int32_t* order, int32_t* par1, int32_t* par2,
                                     int32_t* kind, float* f_inh)
{
    leea_status st = check_run(m, run);
    if (st) return st;
    RunBuf& r = m->runs[run];
    const size_t n = static_cast<size_t>(r.pop);
    const int32_t* src[4] = { r.order, r.par1, r.par2, r.kind };
    int32_t* dst[4] = { order, par1, par2, kind };
    for (int k = 0; k < 4; ++k)
        if (dst[k])
            LEEA_CUDA_TRY(cudaMemcpyAsync(dst[k], src[k], sizeof(int32_t) * n, cudaMemcpyDeviceToHost, m->stream),
                          "selection copy");
    if (f_inh)
        LEEA_CUDA_TRY(cudaMemcpyAsync(f_inh, m->f_inh + r.pop_off, sizeof(float) * n, cudaMemcpyDeviceToHost,
                                      m->stream),
                      "f_inh copy");
    return check_device_status(m->stream, nullptr);
}

leea_status leea_multi_get_shadow(leea_multi* m, int32_t run, uint8_t* shadow_host, int32_t* scale_exp_host,
                                  float* amax_host)
{
    leea_status st = check_run(m, run);
    if (st) return st;
    RunBuf& r = m->runs[run];
    if (shadow_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(shadow_host, r.shadow[m->cur], static_cast<size_t>(r.sh_stride) * r.pop,
                                      cudaMemcpyDeviceToHost, m->stream),
                      "shadow copy");
    if (scale_exp_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(scale_exp_host, r.scale_exp, sizeof(int32_t) * r.pop, cudaMemcpyDeviceToHost,
                                      m->stream),
                      "scale copy");
    if (amax_host)
        LEEA_CUDA_TRY(cudaMemcpyAsync(amax_host, r.amax[m->cur], sizeof(float) * r.pop, cudaMemcpyDeviceToHost,
                                      m->stream),
                      "amax copy");
    return check_device_status(m->stream, nullptr);
}

uint32_t leea_multi_generation_index(const leea_multi* m) { return m ? m->gen : 0u; }

leea_status leea_multi_profile_enable(leea_multi* m, int32_t enable)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if (enable && m->ev.empty()) {
        m->ev.resize(static_cast<size_t>(LEEA_NUM_STAGES) * 2 * kMultiProfRing, nullptr);
        for (cudaEvent_t& e : m->ev) LEEA_CUDA_TRY(cudaEventCreate(&e), "event create");
    }
    if (!enable && m->profiling && (st = prof_fold(m))) return st;
    m->profiling = enable != 0;
    return LEEA_OK;
}

leea_status leea_multi_profile_read(leea_multi* m, double* ms_out, int64_t* launches_out)
{
    leea_status st = check_multi(m);
    if (st) return st;
    if ((st = prof_fold(m))) return st;
    for (int s = 0; s < LEEA_NUM_STAGES; ++s) {
        if (ms_out) ms_out[s] = m->ms[s];
        if (launches_out) launches_out[s] = m->launches[s];
        m->ms[s] = 0.0;
        m->launches[s] = 0;
    }
    return LEEA_OK;
}

void leea_multi_destroy(leea_multi* m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    free_multi(m);
}

leea_status leea_tune_shadow_eval(int32_t precision, int32_t d_in, int32_t hidden, int32_t d_out, int32_t batch,
                                  int32_t pop, int32_t chunk, int32_t reps, float* ms_out)
{
    if (!ms_out || reps < 1 || pop < 1 || batch < 1) return fail(LEEA_EINVAL, "bad tuning arguments");
    const int32_t dims[3] = { d_in, hidden, d_out };
    NetLayout net;
    if (!make_layout(dims, 3, 0, &net)) return fail(LEEA_EINVAL, "invalid dims");
    leea_status st = check_shadow_shape(net, precision);
    if (st) return st;
    const int32_t cw_max = eval_shadow_max_chunk(precision, d_in);
    if (chunk < 0 || chunk % 16 != 0 || chunk > cw_max)
        return fail(LEEA_EINVAL, "chunk must be 0 or a multiple of 16 up to %d", cw_max);
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    const int64_t stride = shadow_stride_of(net, precision);
    float *popv = nullptr, *f = nullptr, *amax = nullptr, *scratch = nullptr;
    uint8_t *shadow = nullptr, *x = nullptr;
    int32_t *y = nullptr, *se = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = alloc(&popv, static_cast<size_t>(pop) * net.c_pad);
    if (err == cudaSuccess) err = alloc(&shadow, static_cast<size_t>(pop) * stride);
    if (err == cudaSuccess) err = alloc(&f, static_cast<size_t>(pop));
    if (err == cudaSuccess) err = alloc(&amax, static_cast<size_t>(pop));
    if (err == cudaSuccess) err = alloc(&se, static_cast<size_t>(pop));
    if (err == cudaSuccess) err = alloc(&x, static_cast<size_t>(batch) * d_in);
    if (err == cudaSuccess) err = alloc(&y, static_cast<size_t>(batch));
    if (err == cudaSuccess && eval_shadow_scratch_bytes(pop, batch) > 0)
        err = alloc(&scratch, eval_shadow_scratch_bytes(pop, batch) / sizeof(float));
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaMemset(x, 0x5A, static_cast<size_t>(batch) * d_in);
    if (err == cudaSuccess) err = cudaMemset(y, 0, sizeof(int32_t) * batch);
    if (err == cudaSuccess) err = cudaMemset(shadow, 0, static_cast<size_t>(pop) * stride);
    if (err == cudaSuccess) err = launch_init(net, pop, 0, 12345u, popv, nullptr);
    if (err == cudaSuccess)
        err = launch_make_shadow(pop, d_in, hidden, net.c_pad, popv, precision, shadow, stride, se, amax, nullptr);
    auto once = [&]() {
        return launch_eval_shadow(net, pop, popv, precision, shadow, stride, se, x, 255.0f, y, batch, 1.0f, nullptr,
                                  f, nullptr, nullptr, scratch, status, nullptr, chunk);
    };
    if (err == cudaSuccess) err = once();  // warm-up
    if (err == cudaSuccess) err = cudaEventRecord(e0, nullptr);
    for (int32_t i = 0; i < reps && err == cudaSuccess; ++i) err = once();
    if (err == cudaSuccess) err = cudaEventRecord(e1, nullptr);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(popv);
    cudaFree(shadow);
    cudaFree(f);
    cudaFree(amax);
    cudaFree(se);
    cudaFree(x);
    cudaFree(y);
    cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "tuning run");
    *ms_out = ms / static_cast<float>(reps);
    return check_device_status(nullptr, nullptr);
}

leea_status leea_tune_group_eval(int32_t precision, int32_t d_in, int32_t hidden, int32_t d_out, int32_t batch,
                                 int32_t pop, int32_t group, int32_t reps, float* ms_out)
{
    if (!ms_out || reps < 1 || pop < 1 || batch < 1) return fail(LEEA_EINVAL, "bad tuning arguments");
    const int32_t dims[3] = { d_in, hidden, d_out };
    NetLayout net;
    if (!make_layout(dims, 3, 0, &net)) return fail(LEEA_EINVAL, "invalid dims");
    leea_status st = check_shadow_shape(net, precision);
    if (st) return st;
    const int32_t g_max = eval_shadow_group_size(hidden);
    if (group < 1 || group > g_max) return fail(LEEA_EINVAL, "group must be in [1, %d]", g_max);
    if (!eval_shadow_group_supported(d_in, d_out, precision, hidden, group * hidden))
        return fail(LEEA_EINVAL, "the group evaluation does not take %d-%d-%d", d_in, hidden, d_out);
    unsigned int* status = device_status_ptr();
    if (!status) return fail(LEEA_ECUDA, "device status word unavailable");
    const int64_t stride = shadow_stride_of(net, precision);
    const int32_t m_tiles = (batch + 127) / 128;
    const int64_t tile_bytes = static_cast<int64_t>(eval_shadow_group_xop_bytes(d_in, precision, 1));
    float *popv = nullptr, *f = nullptr, *amax = nullptr, *scratch = nullptr;
    uint8_t *shadow = nullptr, *x = nullptr, *xop = nullptr;
    int32_t *y = nullptr, *se = nullptr, *sched = nullptr;
    ShadowRun* run_dev = nullptr;
    XopTile* tiles_dev = nullptr;
    GroupUnit* units_dev = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, sms = 0;
    cudaError_t err = alloc(&popv, static_cast<size_t>(pop) * net.c_pad);
    if (err == cudaSuccess) err = alloc(&shadow, static_cast<size_t>(pop) * stride);
    if (err == cudaSuccess) err = alloc(&f, static_cast<size_t>(pop));
    if (err == cudaSuccess) err = alloc(&amax, static_cast<size_t>(pop));
    if (err == cudaSuccess) err = alloc(&se, static_cast<size_t>(pop));
    if (err == cudaSuccess) err = alloc(&x, static_cast<size_t>(batch) * d_in);
    if (err == cudaSuccess) err = alloc(&y, static_cast<size_t>(batch));
    if (err == cudaSuccess) err = alloc(&xop, static_cast<size_t>(m_tiles * tile_bytes));
    if (err == cudaSuccess) err = alloc(&sched, 2);
    if (err == cudaSuccess && eval_shadow_scratch_bytes(pop, batch) > 0)
        err = alloc(&scratch, eval_shadow_scratch_bytes(pop, batch) / sizeof(float));
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaMemset(x, 0x5A, static_cast<size_t>(batch) * d_in);
    if (err == cudaSuccess) err = cudaMemset(y, 0, sizeof(int32_t) * batch);
    if (err == cudaSuccess) err = cudaMemset(sched, 0, 2 * sizeof(int32_t));
    if (err == cudaSuccess) err = cudaMemset(shadow, 0, static_cast<size_t>(pop) * stride);
    if (err == cudaSuccess) err = launch_init(net, pop, 0, 12345u, popv, nullptr);
    if (err == cudaSuccess)
        err = launch_make_shadow(pop, d_in, hidden, net.c_pad, popv, precision, shadow, stride, se, amax, nullptr);
    if (err == cudaSuccess) {
        ShadowRun r = shadow_run(net, pop, popv, precision, shadow, stride, se, x, 255.0f, y, batch, 1.0f, nullptr,
                                 f, nullptr, nullptr, scratch, 0);
        r.xop = xop;
        r.group = group;
        std::vector<ShadowRun> runs(1, r);
        std::vector<XopTile> tiles;
        for (int32_t mt = 0; mt < m_tiles; ++mt)
            tiles.push_back(XopTile{ x + static_cast<int64_t>(128) * mt * d_in, std::min(128, batch - 128 * mt),
                                     xop + mt * tile_bytes });
        std::vector<GroupUnit> units;
        for (int32_t p0 = 0; p0 < pop; p0 += group)
            for (int32_t mt = 0; mt < m_tiles; ++mt) units.push_back(GroupUnit{ 0, mt, p0, std::min(group, pop - p0) });
        err = upload(&run_dev, runs);
        if (err == cudaSuccess) err = upload(&tiles_dev, tiles);
        if (err == cudaSuccess) err = upload(&units_dev, units);
        if (err == cudaSuccess) err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        auto once = [&]() {
            cudaError_t e = launch_stage_xop_tiles(tiles_dev, m_tiles, d_in, precision, nullptr);
            if (e != cudaSuccess) return e;
            return launch_eval_shadow_group(d_in, d_out, precision, group * hidden, run_dev, 1, pop, m_tiles > 1,
                                            units_dev, static_cast<int32_t>(units.size()), sched, sms, status,
                                            nullptr);
        };
        if (err == cudaSuccess) err = once();  // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(e0, nullptr);
        for (int32_t i = 0; i < reps && err == cudaSuccess; ++i) err = once();
        if (err == cudaSuccess) err = cudaEventRecord(e1, nullptr);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    }
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(popv);
    cudaFree(shadow);
    cudaFree(f);
    cudaFree(amax);
    cudaFree(se);
    cudaFree(x);
    cudaFree(y);
    cudaFree(xop);
    cudaFree(sched);
    cudaFree(scratch);
    cudaFree(run_dev);
    cudaFree(tiles_dev);
    cudaFree(units_dev);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "tuning run");
    *ms_out = ms / static_cast<float>(reps);
    return LEEA_OK;
}

}  // extern "C"
