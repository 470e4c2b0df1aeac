"""Control of the mutation strength (Section 3.2) through the state object, in
lock step with the oracle: exponential decay sigma 0.99^(i/k) and the
self-adaptive sigma gene (sigma' = sigma exp(tau z) before the child's own
mutation, the parents' mean after crossover).  Both sides start from the same
population, fitness, sigma genes and generation counter and run one
generation; selection must agree bit-exactly, sigma genes within FP32
rounding of exp, children within the breed tolerance at each child's own
strength, fitness within the evaluation tolerance."""
import numpy as np
import pytest

from helpers import assert_correct_close, assert_fitness_close, assert_genes_close, decode_bf16, decode_e4m3, untile_shadow
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu

NORMAL_BOUND = np.float32(5.77)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _lockstep(gpu, oracle_mod, dims, pop, batch, prm, seed=21, gen0=40, sample=None, precision=0):
    c = gpu.leea_layout_num_params(dims)
    st = gpu.LeeaState(pop, dims, gpu.Params(**prm, precision=precision), seed)
    try:
        rng = np.random.default_rng(seed)
        pop0 = synthetic.random_population(pop, c, seed=seed + 1, scale=0.1)
        f0 = rng.normal(-2.3, 0.05, size=pop).astype(np.float32)
        f0[::5] = f0[0]  # ties
        st.leea_set_population(pop0)
        st.leea_set_fitness(f0)
        st.leea_set_generation(gen0, True)
        self_adaptive = prm.get("sigma_ctl", 0) == gpu.SIGMA_SELF
        if self_adaptive:
            sig0 = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), size=pop)).astype(np.float32)
            st.leea_set_sigma(sig0)
            np.testing.assert_array_equal(st.leea_get_sigma(), sig0)
        levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
        y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
        st.leea_generation_u8(_dev(levels), _dev(y), 255.0)
        x64 = levels.astype(np.float64) / 255.0
        assert st.gen == gen0 + 1
        order, par1, par2, kind, f_inh = st.leea_get_selection()
        kids = st.leea_get_population()
        sig_gpu = st.leea_get_sigma()
        f_raw = st.leea_raw_fitness()
        f_adj, cor = st.leea_fitness(with_correct=True)

        o_prm = oracle_mod.Params(**{k: v for k, v in prm.items() if k != "eval_path"})
        f0d = f0.astype(np.float64)
        o_order = oracle_mod.rank(f0d)
        np.testing.assert_array_equal(order, o_order)
        o1, o2, ok, ofi = oracle_mod.select(o_prm, f0d, o_order, seed, gen0 + 1)
        np.testing.assert_array_equal(par1, o1)
        np.testing.assert_array_equal(par2, o2)
        np.testing.assert_array_equal(kind, ok)
        if self_adaptive:
            sig_ref = oracle_mod.select_sigma(o_prm, seed, gen0 + 1, o1, o2, ok, sig0.astype(np.float64))
            # elites and crossover children: one FP32 rounding; mutation children: expf in FP32
            np.testing.assert_allclose(sig_gpu, sig_ref, rtol=1e-6, atol=0)
            moved = ok == oracle_mod.MUTATION
            if prm["tau"] > 0:
                assert (sig_gpu[moved] != sig0[o1[moved]]).mean() > 0.99
            else:  # exp(0 z) = 1: the parent's gene
                np.testing.assert_array_equal(sig_gpu[moved], sig0[o1[moved]])
        else:
            sig_ref = np.full(pop, oracle_mod.sigma_schedule(o_prm, gen0 + 1))
            np.testing.assert_allclose(sig_gpu, oracle_mod.sigma_schedule(o_prm, gen0 + 2), rtol=2 ** -23)

        rows = np.arange(pop) if sample is None else np.asarray(sample)
        pop0d = pop0.astype(np.float64)
        for j in rows:
            ref = oracle_mod.breed_sigma(o_prm, dims, seed, gen0 + 1, pop0d, o1, o2, ok, sig_ref, j0=int(j),
                                         j1=int(j) + 1)
            assert_genes_close(kids[j][None], ref, float(sig_ref[j]), what=f"child {j}")

        evald = kids[rows].astype(np.float64)
        if precision:
            n = dims[0] * dims[1]
            am_par = np.abs(pop0[:, :n]).max(axis=1)
            sh, se, am = st.leea_get_shadow(precision)
            np.testing.assert_array_equal(am, np.abs(kids[:, :n]).max(axis=1))
            if precision == 2:
                # each child's exponent bounds its own max |W1| with its own strength
                for j in range(pop):
                    b = np.float32(am_par[par1[j]])
                    if kind[j] == 1:
                        b = max(b, np.float32(am_par[par2[j]]))
                    elif kind[j] == 2:
                        b = np.float32(np.float64(sig_gpu[j]) * np.float64(NORMAL_BOUND) + np.float64(b))
                    assert se[j] == oracle_mod.fp8_scale_exp(float(b)), j
            elem = 2 if precision == 1 else 1
            raw = untile_shadow(sh[rows], dims[0], dims[1], elem).reshape(len(rows), n * elem)
            if precision == 1:
                vals = decode_bf16(raw.view(np.uint16))
            else:
                vals = decode_e4m3(raw) * np.ldexp(1.0, se[rows].astype(np.int64))[:, None]
            q = oracle_mod.quantize_w1(evald, dims, precision, se[rows])
            np.testing.assert_array_equal(vals, q[:, :n])
            evald = q
        f_ref, cor_ref, logits = oracle_mod.evaluate(evald, dims, x64, y, want_logits=True)
        assert_fitness_close(f_raw[rows], f_ref)
        if not precision:
            assert_correct_close(cor[rows], cor_ref, logits)
        adj = oracle_mod.inherit(float(np.float32(o_prm.alpha)), ofi[rows], f_ref, first=False)
        assert_fitness_close(f_adj[rows], adj, "f_adj")
    finally:
        st.close()


SMALL = dict(dims=[784, 32, 10], pop=32, batch=16)
FULL = dict(dims=[784, 112, 10], pop=1000, batch=100)
SAMPLE = [0, 1, 2, 49, 50, 51, 300, 549, 550, 551, 777, 998, 999]


@pytest.mark.parametrize("k,gen0", [(1.0, 40), (4.0, 250), (0.5, 0)])
def test_decay_lockstep_small(gpu, oracle_mod, k, gen0):
    prm = dict(sel_op=1, tour_k=3, sigma=0.05, mut_rate=0.5, alpha=0.2, sigma_ctl=gpu.SIGMA_DECAY, sigma_k=k)
    _lockstep(gpu, oracle_mod, **SMALL, prm=prm, gen0=gen0)


@pytest.mark.parametrize("xo_op,tau", [(0, 0.3), (1, 1.0), (1, 0.0)])
def test_self_adaptive_lockstep_small(gpu, oracle_mod, xo_op, tau):
    prm = dict(xo_op=xo_op, n_elite=2, sigma=0.01, alpha=0.5, sigma_ctl=gpu.SIGMA_SELF, tau=tau)
    _lockstep(gpu, oracle_mod, **SMALL, prm=prm)


def test_self_adaptive_lockstep_full_size_sampled(gpu, oracle_mod):
    # The benchmark's workload (P = 1000, 784-112-10, B = 100) with sigma genes,
    # the tensor-core evaluation; a sample of children recomputed one by one.
    prm = dict(n_elite=50, xo_op=1, p_c=0.5, sigma=0.005, sigma_ctl=gpu.SIGMA_SELF, tau=0.2)
    _lockstep(gpu, oracle_mod, **FULL, prm=prm, sample=SAMPLE)


def test_decay_lockstep_full_size_sampled(gpu, oracle_mod):
    prm = dict(n_elite=1, p_c=0.5, sigma=0.01, mut_rate=0.1, sigma_ctl=gpu.SIGMA_DECAY, sigma_k=3.0)
    _lockstep(gpu, oracle_mod, **FULL, prm=prm, sample=SAMPLE, gen0=123)


def test_self_adaptive_paper_network(gpu, oracle_mod):
    # The paper's 196-256-128-64-10 (tensor-core evaluation of three hidden
    # layers) with sigma genes and its Section 4.5 operators.
    prm = dict(p_c=0.75, sigma=0.001, alpha=1.0, init=1, sigma_ctl=gpu.SIGMA_SELF, tau=0.3)
    _lockstep(gpu, oracle_mod, dims=[196, 256, 128, 64, 10], pop=40, batch=64, prm=prm)


@pytest.mark.parametrize("ctl", ["self", "decay"])
def test_sigma_control_fused_breed_evaluate(gpu, oracle_mod, ctl):
    # The fused breed + evaluate kernel reads each child's own strength too.
    extra = dict(sigma_ctl=gpu.SIGMA_SELF, tau=0.5) if ctl == "self" else dict(sigma_ctl=gpu.SIGMA_DECAY, sigma_k=2.0)
    prm = dict(n_elite=2, sigma=0.01, alpha=0.5, eval_path=gpu.EVAL_FUSED, **extra)
    _lockstep(gpu, oracle_mod, **SMALL, prm=prm)
    _lockstep(gpu, oracle_mod, **FULL, prm=dict(prm, mut_rate=0.1), sample=SAMPLE)


@pytest.mark.parametrize("precision", [1, 2])
def test_self_adaptive_precision_form(gpu, oracle_mod, precision):
    # FP8: a mutation child's scale exponent must use its own mutated sigma.
    prm = dict(n_elite=2, sigma=0.02, mut_rate=0.1, sigma_ctl=gpu.SIGMA_SELF, tau=1.0, alpha=0.5)
    _lockstep(gpu, oracle_mod, dims=[784, 32, 10], pop=64, batch=100, prm=prm, precision=precision)


def test_sigma_genes_persist_and_drift(gpu):
    # Over many generations the genes stay positive and finite, elites keep
    # theirs, and with tau > 0 the population's strengths spread out.
    dims, pop = [784, 32, 10], 64
    st = gpu.LeeaState(pop, dims, gpu.Params(sigma=0.01, n_elite=4, sigma_ctl=gpu.SIGMA_SELF, tau=0.3), 3)
    try:
        x, y = synthetic.make_split(32, seed=4)
        xd, yd = _dev(synthetic.to_levels(x)), _dev(y)
        for _ in range(12):
            st.leea_generation_u8(xd, yd, 255.0)
        before = st.leea_get_sigma()
        st.leea_generation_u8(xd, yd, 255.0)
        order, par1, _, kind, _ = st.leea_get_selection()
        after = st.leea_get_sigma()
        assert np.isfinite(after).all() and (after > 0).all()
        np.testing.assert_array_equal(after[kind == 0], before[par1[kind == 0]])
        assert np.std(np.log(after)) > 0.1
    finally:
        st.close()


def test_sigma_state_errors(gpu):
    dims = [784, 32, 10]
    st = gpu.LeeaState(8, dims, gpu.Params(), 1)
    try:
        np.testing.assert_array_equal(st.leea_get_sigma(), np.full(8, np.float32(0.001)))
        with pytest.raises(gpu.LeeaError) as e:
            st.leea_set_sigma(np.ones(8, dtype=np.float32))
        assert e.value.status == gpu.ESTATE
    finally:
        st.close()
    st = gpu.LeeaState(8, dims, gpu.Params(sigma_ctl=gpu.SIGMA_SELF), 1)
    try:
        bad = np.ones(8, dtype=np.float32)
        bad[3] = -1.0
        with pytest.raises(gpu.LeeaError) as e:
            st.leea_set_sigma(bad)
        assert e.value.status == gpu.EINVAL
    finally:
        st.close()
    with pytest.raises(gpu.LeeaError):
        gpu.MultiRun([gpu.RunSpec(16, 32, 16)], 784, 10, gpu.Params(precision=1, sigma_ctl=gpu.SIGMA_DECAY))
