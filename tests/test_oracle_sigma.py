"""Pins of the oracle's control of the mutation strength (Section 3.2):
constant, exponential decay sigma_i = sigma 0.99^(i/k), and self-adaptation
(sigma as a gene, mutated by exp(tau N(0,1)) before it scales the child's
own mutation; the arithmetic mean of the parents' genes after crossover)."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1806_09819_gb300 import synthetic


def _run(oracle_mod, prm, dims, pop, seed, gens, x, y):
    st = oracle_mod.State(pop, dims, prm, seed=seed)
    for _ in range(gens):
        st.generation(x, y)
    return st


def test_decay_starts_at_sigma_and_a_huge_k_is_constant(oracle_mod):
    dims, pop = [40, 6, 5], 12
    x, y = synthetic.tiny_problem(40, 5, 16, seed=3)
    const = _run(oracle_mod, oracle_mod.Params(sigma=0.05), dims, pop, 4, 2, x, y)
    # The first breed is breed i = 0: sigma 0.99^0 = sigma, bitwise the constant run.
    decay = _run(oracle_mod, oracle_mod.Params(sigma=0.05, sigma_ctl=oracle_mod.SIGMA_DECAY, sigma_k=1.0),
                 dims, pop, 4, 2, x, y)
    np.testing.assert_array_equal(decay.population(), const.population())
    # Later breeds differ ...
    const.generation(x, y)
    decay.generation(x, y)
    assert not np.array_equal(decay.population(), const.population())
    # ... unless k is so large that 0.99^(i/k) rounds to 1.
    flat = _run(oracle_mod, oracle_mod.Params(sigma=0.05, sigma_ctl=oracle_mod.SIGMA_DECAY, sigma_k=1e30),
                dims, pop, 4, 3, x, y)
    np.testing.assert_array_equal(flat.population(), const.population())


@pytest.mark.parametrize("k,breeds_before", [(1.0, 100), (4.0, 100), (2.5, 7)])
def test_decay_step_length_follows_the_schedule(oracle_mod, k, breeds_before):
    # Only mutation children, every gene mutated: child - parent = sigma_i z
    # with z ~ N(0,1), so the sample deviation over all genes estimates sigma_i
    # (about 50k genes: relative standard error ~0.3 %).
    dims, pop, sigma = [200, 40, 10], 6, 0.02
    prm = oracle_mod.Params(sigma=sigma, sigma_ctl=oracle_mod.SIGMA_DECAY, sigma_k=k, n_elite=0, p_c=0.0)
    x, y = synthetic.tiny_problem(200, 10, 8, seed=5)
    st = oracle_mod.State(pop, dims, prm, seed=6)
    st.generation(x, y)
    st.set_generation(breeds_before, True)  # the next breed is breed number i = breeds_before
    parents = st.population()
    st.generation(x, y)
    _, par1, _, kind, _ = st.selection()
    assert (kind == oracle_mod.MUTATION).all()
    step = st.population() - parents[par1]
    expect = sigma * 0.99 ** (breeds_before / k)
    assert abs(step.std() / expect - 1.0) < 0.02
    # The state reports the strength of the breed after this one.
    sigma32 = float(np.float32(sigma))  # the parameter block holds FP32
    np.testing.assert_allclose(st.sigma(), sigma32 * 0.99 ** ((breeds_before + 1) / k), rtol=1e-12)


def test_constant_and_schedule_helpers(oracle_mod):
    prm = oracle_mod.Params(sigma=0.3)
    assert oracle_mod.sigma_schedule(prm, 1) == pytest.approx(0.3, rel=1e-7)
    assert oracle_mod.sigma_schedule(prm, 500) == oracle_mod.sigma_schedule(prm, 1)
    d = oracle_mod.Params(sigma=0.3, sigma_ctl=oracle_mod.SIGMA_DECAY, sigma_k=10.0)
    # 0.99^(i/k) halves sigma after i = k ln 2 / -ln 0.99 breeds.
    i_half = 10.0 * math.log(2.0) / -math.log(0.99)
    lo, hi = int(math.floor(i_half)), int(math.ceil(i_half))
    s = float(np.float32(0.3))
    assert oracle_mod.sigma_schedule(d, lo + 1) > s / 2 > oracle_mod.sigma_schedule(d, hi + 1)


def test_self_adaptive_with_tau_zero_is_constant_sigma(oracle_mod):
    dims, pop = [40, 6, 5], 14
    x, y = synthetic.tiny_problem(40, 5, 16, seed=7)
    for xo_op in (0, 1):
        const = _run(oracle_mod, oracle_mod.Params(sigma=0.05, xo_op=xo_op), dims, pop, 9, 4, x, y)
        sa = _run(oracle_mod, oracle_mod.Params(sigma=0.05, xo_op=xo_op, sigma_ctl=oracle_mod.SIGMA_SELF, tau=0.0),
                  dims, pop, 9, 4, x, y)
        np.testing.assert_array_equal(sa.population(), const.population())
        np.testing.assert_array_equal(sa.sigma(), np.full(pop, float(np.float32(0.05))))


def test_self_adaptive_genes_follow_the_operators(oracle_mod):
    dims, pop, tau = [4, 3, 2], 400, 0.3
    prm = oracle_mod.Params(sigma=0.01, sigma_ctl=oracle_mod.SIGMA_SELF, tau=tau)
    x, y = synthetic.tiny_problem(4, 2, 8, seed=1)
    st = oracle_mod.State(pop, dims, prm, seed=2)
    st.generation(x, y)
    sig0 = 0.001 * (1.0 + np.arange(pop)) ** 0.5  # distinct genes
    st.set_sigma(sig0)
    np.testing.assert_array_equal(st.sigma(), sig0)
    st.generation(x, y)
    _, par1, par2, kind, _ = st.selection()
    sig1 = st.sigma()
    el, xo, mu = (kind == oracle_mod.ELITE), (kind == oracle_mod.CROSSOVER), (kind == oracle_mod.MUTATION)
    n_e, n_c, n_m, _ = oracle_mod.counts(pop, prm)
    assert (el.sum(), xo.sum(), mu.sum()) == (n_e, n_c, n_m)
    np.testing.assert_array_equal(sig1[el], sig0[par1[el]])                          # copied
    np.testing.assert_array_equal(sig1[xo], 0.5 * (sig0[par1[xo]] + sig0[par2[xo]]))  # arithmetic mean
    z = np.log(sig1[mu] / sig0[par1[mu]]) / float(np.float32(tau))                    # log-normal step
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # The step of child j is draw 0 of the SIGMA stream of (generation, child j).
    js = np.flatnonzero(mu)[:5]
    for j, zj in zip(js, z[:5]):
        assert zj == pytest.approx(oracle_mod.normal(2, oracle_mod.TAG_SIGMA, 1, int(j), 0), abs=1e-12)


def test_self_adaptive_mutation_uses_the_mutated_sigma(oracle_mod):
    # sigma' is drawn first and then scales the child's weight mutation
    # (sigma' = sigma e^{tau z}, theta' = theta + sigma' N(0,1)): with tau = 1 the
    # children's step lengths follow sigma', not the parent's gene.
    dims, pop = [200, 40, 10], 8
    prm = oracle_mod.Params(sigma=0.01, sigma_ctl=oracle_mod.SIGMA_SELF, tau=1.0, n_elite=0, p_c=0.0)
    x, y = synthetic.tiny_problem(200, 10, 8, seed=5)
    st = oracle_mod.State(pop, dims, prm, seed=12)
    st.generation(x, y)
    parents = st.population()
    st.generation(x, y)
    _, par1, _, kind, _ = st.selection()
    assert (kind == oracle_mod.MUTATION).all()
    sig = st.sigma()
    step_sd = (st.population() - parents[par1]).std(axis=1)
    np.testing.assert_allclose(step_sd / sig, 1.0, atol=0.03)
    moved = np.abs(np.log(sig / 0.01)) > 0.2
    assert moved.any()
    assert (np.abs(step_sd[moved] / 0.01 - 1.0) > 0.1).all()


def test_breed_sigma_with_a_constant_array_is_breed(oracle_mod):
    dims = [30, 7, 5]
    c = oracle_mod.num_params(dims)
    rng = np.random.default_rng(0)
    parents = rng.normal(size=(10, c))
    par1 = rng.integers(0, 10, 10).astype(np.int32)
    par2 = rng.integers(0, 10, 10).astype(np.int32)
    kind = np.array([0, 1, 1, 2, 2, 2, 1, 2, 0, 2], dtype=np.int32)
    prm = oracle_mod.Params(sigma=0.2, mut_rate=0.7)
    a = oracle_mod.breed(prm, dims, 5, 3, parents, par1, par2, kind)
    b = oracle_mod.breed_sigma(prm, dims, 5, 3, parents, par1, par2, kind, np.full(10, float(np.float32(0.2))))
    np.testing.assert_array_equal(a, b)
    # Per-child strengths: a mutation child's step scales with its own sigma.
    s = np.linspace(0.1, 1.0, 10)
    d = oracle_mod.breed_sigma(prm, dims, 5, 3, parents, par1, par2, kind, s)
    for j in np.flatnonzero(kind == oracle_mod.MUTATION):
        np.testing.assert_allclose((d[j] - parents[par1[j]]) / s[j], (a[j] - parents[par1[j]]) / np.float32(0.2),
                                   rtol=1e-9, atol=1e-12)


def test_invalid_sigma_control_is_rejected(oracle_mod):
    dims = [4, 3, 2]
    for bad in (oracle_mod.Params(sigma_ctl=3), oracle_mod.Params(sigma_ctl=oracle_mod.SIGMA_DECAY, sigma_k=0.0),
                oracle_mod.Params(sigma_ctl=oracle_mod.SIGMA_SELF, tau=-1.0)):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.State(4, dims, bad, seed=0)
    st = oracle_mod.State(4, dims, oracle_mod.Params(), seed=0)
    with pytest.raises(oracle_mod.OracleError):
        st.set_sigma(np.ones(4))
