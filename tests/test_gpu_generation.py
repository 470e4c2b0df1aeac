"""Whole generations of Algorithm 1 through the state object, in lock step with
the oracle: both sides start from the same state (population, f_adj,
generation counter, seed), run one generation, and must agree -- selection
bit-exactly, children and fitness within the stated tolerances.  Also the
run-level invariants, the host-buffer entry point, and sampled parity at the
full P = 1000, 784-112-10, B = 100 workload in the benchmark's launch shape."""
import numpy as np
import pytest

from helpers import assert_correct_close, assert_fitness_close, assert_genes_close
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu

CONFIG_SMALL = dict(dims=[784, 32, 10], pop=32, batch=16,
                    prm=dict(sel_op=1, tour_k=3, xo_op=0, sigma=0.01, alpha=0.2))
CONFIG_FULL = dict(dims=[784, 112, 10], pop=1000, batch=100,
                   prm=dict(n_elite=1, xo_op=0, p_c=0.5, sigma=0.005, mut_rate=0.1))


def _dev_batch(x, y):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda(), torch.from_numpy(np.ascontiguousarray(y)).cuda()


def _lockstep(gpu, oracle_mod, dims, pop, batch, prm, seed=11, gen0=3, sample=None, u8=False):
    """One generation from a common state; returns nothing, asserts parity.
    With u8=True the minibatch goes in as 8-bit levels k (x = k / 255).  With
    a sample, the oracle breeds only the sampled children, but evaluates every
    child the GPU made (the fitness of the whole population is compared)."""
    c = gpu.leea_layout_num_params(dims)
    st = gpu.LeeaState(pop, dims, gpu.Params(**prm), seed)
    pop0 = synthetic.random_population(pop, c, seed=seed + 1, scale=0.1)
    f0 = np.random.default_rng(seed).normal(-2.3, 0.05, size=pop).astype(np.float32)
    f0[::7] = f0[0]  # ties
    st.leea_set_population(pop0)
    st.leea_set_fitness(f0)
    st.leea_set_generation(gen0, True)
    if dims[0] == 784:
        x, y = synthetic.make_split(batch, seed=seed + 2)
    else:
        x, y = synthetic.tiny_problem(dims[0], dims[-1], batch, seed=seed + 2)
    if u8:
        xl, yd = _dev_batch(synthetic.to_levels(x), y)
        st.leea_generation_u8(xl, yd, 255.0)
        x = synthetic.to_levels(x).astype(np.float64) / 255.0
    else:
        st.leea_generation(*_dev_batch(x, y))
    assert st.gen == gen0 + 1
    order, par1, par2, kind, f_inh = st.leea_get_selection()
    kids = st.leea_get_population()
    f_adj, cor = st.leea_fitness(with_correct=True)
    f_raw = st.leea_raw_fitness()

    o_prm = oracle_mod.Params(**{k: v for k, v in prm.items() if k != "eval_path"})
    f0d = f0.astype(np.float64)
    o_order = oracle_mod.rank(f0d)
    np.testing.assert_array_equal(order, o_order)
    o1, o2, ok, ofi = oracle_mod.select(o_prm, f0d, o_order, seed, gen0 + 1)
    np.testing.assert_array_equal(par1, o1)
    np.testing.assert_array_equal(par2, o2)
    np.testing.assert_array_equal(kind, ok)
    np.testing.assert_allclose(f_inh, ofi, rtol=2 ** -23, atol=0)

    rows = np.arange(pop) if sample is None else sample
    pop0d = pop0.astype(np.float64)
    for j in rows:
        ref = oracle_mod.breed(o_prm, dims, seed, gen0 + 1, pop0d, o1, o2, ok, j0=int(j), j1=int(j) + 1)
        assert_genes_close(kids[j][None], ref, o_prm.sigma, what=f"child {j}")
    f_ref, cor_ref, logits = oracle_mod.evaluate(kids.astype(np.float64), dims, x.astype(np.float64), y,
                                                 want_logits=True)
    assert_fitness_close(f_raw, f_ref)
    assert_correct_close(cor, cor_ref, logits)
    adj = oracle_mod.inherit(float(np.float32(o_prm.alpha)), ofi, f_ref, first=False)
    assert_fitness_close(f_adj, adj, "f_adj")
    st.close()


@pytest.mark.parametrize("path", [1, 2])
def test_lockstep_small_config(gpu, oracle_mod, path):
    prm = dict(CONFIG_SMALL["prm"], eval_path=path)
    _lockstep(gpu, oracle_mod, CONFIG_SMALL["dims"], CONFIG_SMALL["pop"], CONFIG_SMALL["batch"], prm)


@pytest.mark.parametrize("prm", [dict(sigma=0.5), dict(sel_op=1, tour_k=2, xo_op=1, alpha=0.5),
                                 dict(n_elite=4, p_c=0.0, sigma=0.1)])
def test_lockstep_2_2_2(gpu, oracle_mod, prm):
    _lockstep(gpu, oracle_mod, [2, 2, 2], 4, 8, prm)


@pytest.mark.parametrize("path", [1, 2, 3])
def test_lockstep_full_size_sampled_u8(gpu, oracle_mod, path):
    sample = np.array([0, 1, 2, 250, 499, 500, 501, 502, 777, 998, 999])
    prm = dict(CONFIG_FULL["prm"], eval_path=path)
    _lockstep(gpu, oracle_mod, CONFIG_FULL["dims"], CONFIG_FULL["pop"], CONFIG_FULL["batch"], prm, sample=sample,
              u8=True)


@pytest.mark.parametrize("path", [1, 2, 3])
def test_lockstep_small_config_u8(gpu, oracle_mod, path):
    prm = dict(CONFIG_SMALL["prm"], eval_path=path)
    _lockstep(gpu, oracle_mod, CONFIG_SMALL["dims"], CONFIG_SMALL["pop"], CONFIG_SMALL["batch"], prm, u8=True)


@pytest.mark.parametrize("path", [1, 2])
def test_lockstep_full_size_sampled(gpu, oracle_mod, path):
    # Full workload; the oracle recomputes a sample of children (the elite,
    # crossover and mutation children, first and last) one by one.
    sample = np.array([0, 1, 2, 250, 499, 500, 501, 502, 777, 998, 999])
    prm = dict(CONFIG_FULL["prm"], eval_path=path)
    _lockstep(gpu, oracle_mod, CONFIG_FULL["dims"], CONFIG_FULL["pop"], CONFIG_FULL["batch"], prm, sample=sample)


@pytest.mark.parametrize("pop,batch,path,u8", [(1, 1, 2, True), (2, 3, 3, True), (1, 2, 1, False), (2, 1, 2, False),
                                               (3, 128, 3, True)])
def test_lockstep_degenerate_sizes(gpu, oracle_mod, pop, batch, path, u8):
    # A population of one or two (the lone individual is elite, crossover
    # partner or mutation parent of itself) and batches of one sample; the
    # largest batch the 8-bit tensor-core and fused paths take.
    prm = dict(sigma=0.05, n_elite=-1, eval_path=path)
    _lockstep(gpu, oracle_mod, [784, 32, 10], pop, batch, prm, u8=u8)


def test_first_generation_evaluates_the_initial_population(gpu, oracle_mod):
    dims, pop, batch = [784, 32, 10], 8, 16
    prm = dict(init=1)
    st = gpu.LeeaState(pop, dims, gpu.Params(**prm), 5)
    x, y = synthetic.make_split(batch, seed=1)
    st.leea_generation(*_dev_batch(x, y))
    assert st.gen == 0
    init = oracle_mod.init(pop, dims, 1, 5)
    np.testing.assert_allclose(st.leea_get_population(), init, rtol=1e-6, atol=1e-9)
    f_ref, _ = oracle_mod.evaluate(st.leea_get_population().astype(np.float64), dims, x, y)
    f_adj = st.leea_fitness()
    assert_fitness_close(f_adj, f_ref)
    np.testing.assert_array_equal(f_adj, st.leea_raw_fitness())


def test_run_matches_oracle_run_statistically(gpu, oracle_mod):
    # 20 generations of the small configuration from the same seed on both
    # sides.  Trajectories diverge once FP32 and FP64 order two near-equal
    # fitnesses differently, so compare the outcome, not the path.
    dims, pop, batch, prm = CONFIG_SMALL["dims"], CONFIG_SMALL["pop"], CONFIG_SMALL["batch"], CONFIG_SMALL["prm"]
    (xtr, ytr), _ = synthetic.dataset(n_train=2000, n_test=1)
    idx = synthetic.batch_indices(2000, batch, 21)
    st = gpu.LeeaState(pop, dims, gpu.Params(**prm), 1)
    ost = oracle_mod.State(pop, dims, oracle_mod.Params(**prm), 1)
    for g in range(21):
        x, y = xtr[idx[g]], ytr[idx[g]]
        st.leea_generation(*_dev_batch(x, y))
        ost.generation(x, y)
        if g == 0:
            assert_fitness_close(st.leea_fitness(), ost.fitness()[0])
    fg, fo = st.leea_fitness(), ost.fitness()[0]
    assert abs(np.median(fg) - np.median(fo)) < 0.3


def test_best_persists_without_variation(gpu):
    dims, pop, batch = [784, 32, 10], 16, 32
    st = gpu.LeeaState(pop, dims, gpu.Params(n_elite=1, p_c=0.0, sigma=0.0), 3)
    x, y = _dev_batch(*synthetic.make_split(batch, seed=9))
    st.leea_generation(x, y)
    best = st.leea_best_params()
    fmax = st.leea_fitness().max()
    for _ in range(8):
        st.leea_generation(x, y)
        np.testing.assert_array_equal(st.leea_best_params(), best)
        f = st.leea_fitness()
        assert f.max() >= fmax
        fmax = f.max()


def test_host_entry_point_matches_device_entry_point(gpu):
    import torch
    dims, pop, batch = [784, 32, 10], 32, 16
    prm = gpu.Params(**CONFIG_SMALL["prm"])
    a = gpu.LeeaState(pop, dims, prm, 21)
    b = gpu.LeeaState(pop, dims, prm, 21)
    for g in range(4):
        x, y = synthetic.make_split(batch, seed=100 + g)
        a.leea_generation(*_dev_batch(x, y))
        b.leea_generation_host(torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory())
    np.testing.assert_array_equal(a.leea_fitness(), b.leea_fitness())
    np.testing.assert_array_equal(a.leea_get_population(), b.leea_get_population())


def test_u8_host_entry_point_matches_device_entry_point(gpu):
    import torch
    dims, pop, batch = [784, 112, 10], 64, 100
    prm = gpu.Params(n_elite=1, sigma=0.005, mut_rate=0.1)
    a = gpu.LeeaState(pop, dims, prm, 5)
    b = gpu.LeeaState(pop, dims, prm, 5)
    for g in range(3):
        x, y = synthetic.make_split(batch, seed=200 + g)
        k = synthetic.to_levels(x)
        a.leea_generation_u8(*_dev_batch(k, y))
        b.leea_generation_u8_host(torch.from_numpy(k).pin_memory(), torch.from_numpy(y).pin_memory())
    np.testing.assert_array_equal(a.leea_fitness(), b.leea_fitness())
    np.testing.assert_array_equal(a.leea_get_population(), b.leea_get_population())


def test_profiling_counts_launches(gpu):
    # The chain of kernels (here with the tensor-core evaluation): a selection,
    # a breed and an evaluation stage per generation after the first, which
    # evaluates only.  AUTO at this size: one launch per generation, counted
    # as the breed stage (the first, evaluating, launch as the evaluation).
    dims, pop, batch = [784, 32, 10], 32, 16
    x, y = _dev_batch(*synthetic.make_split(batch, seed=3))
    for path, expect in ((gpu.EVAL_TENSOR, (4, 4, 5)), (gpu.EVAL_AUTO, (0, 4, 1))):
        st = gpu.LeeaState(pop, dims, gpu.Params(eval_path=path), 2)
        try:
            st.leea_profile_enable(True)
            for _ in range(5):
                st.leea_generation(x, y)
            prof = st.leea_profile_read()
            assert (prof["select"][1], prof["breed"][1], prof["evaluate"][1]) == expect, (path, prof)
            assert all(ms >= 0 for ms, _ in prof.values())
            assert st.leea_profile_read()["evaluate"] == (0.0, 0)
        finally:
            st.close()


def test_state_errors(gpu):
    dims = [784, 32, 10]
    st = gpu.LeeaState(4, dims, gpu.Params(), 2)
    with pytest.raises(gpu.LeeaError) as e:
        st.leea_fitness()
    assert e.value.status == gpu.ESTATE
    x, y = _dev_batch(*synthetic.make_split(3, seed=3))
    assert st.lib.leea_generation(st._h, x.data_ptr(), y.data_ptr(), 0) == gpu.EINVAL
    assert st.lib.leea_generation(st._h, None, y.data_ptr(), 3) == gpu.EINVAL
