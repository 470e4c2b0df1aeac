"""Pins of fitness inheritance (Section 3.1), the whole-run invariants of
Algorithm 1, and initialisation (Section 4.1)."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1806_09819_gb300 import synthetic


def test_alpha_one_disables_inheritance(oracle_mod):
    f = np.array([-1.0, -2.0, np.nan])
    f_inh = np.array([-5.0, -6.0, -7.0])
    np.testing.assert_array_equal(oracle_mod.inherit(1.0, f_inh, f, first=False), f)
    np.testing.assert_array_equal(oracle_mod.inherit(0.3, None, f, first=True), f)


@pytest.mark.parametrize("alpha", [0.2, 0.5])
def test_inheritance_closed_form_for_reevaluated_elites(oracle_mod, alpha):
    # All individuals are elites: each one is re-evaluated every generation on
    # a new batch and keeps its own f_adj as f_inh, so after t generations
    # f_adj = (1-a)^t f_0 + a sum_{s=1..t} (1-a)^(t-s) f_s.
    dims, pop, gens = [784, 8, 10], 6, 7
    prm = oracle_mod.Params(n_elite=pop, alpha=alpha)
    st = oracle_mod.State(pop, dims, prm, seed=3)
    (xtr, ytr), _ = synthetic.dataset(n_train=gens * 16 + 16, n_test=1)
    ids = np.arange(pop)
    history = {i: [] for i in range(pop)}
    for g in range(gens + 1):
        st.generation(xtr[16 * g:16 * g + 16], ytr[16 * g:16 * g + 16])
        if g > 0:
            order = st.selection()[0]
            ids = ids[order]  # child j is a copy of parent order[j]
        f_adj, f_raw, _ = st.fitness()
        for j in range(pop):
            history[ids[j]].append(f_raw[j])
    f_adj, _, _ = st.fitness()
    alpha = float(np.float32(alpha))  # the parameter block carries alpha as float32
    for j in range(pop):
        fs = history[ids[j]]
        t = len(fs) - 1
        closed = (1 - alpha) ** t * fs[0] + alpha * sum((1 - alpha) ** (t - s) * fs[s] for s in range(1, t + 1))
        assert abs(f_adj[j] - closed) < 1e-12


def test_best_individual_persists_without_variation(oracle_mod):
    # sigma = 0, no crossover, elitism: the best stays bitwise; on a fixed batch
    # (alpha = 1) the best fitness never decreases.
    dims, pop = [784, 6, 10], 10
    prm = oracle_mod.Params(n_elite=1, p_c=0.0, sigma=0.0)
    st = oracle_mod.State(pop, dims, prm, seed=8)
    x, y = synthetic.make_split(24, 5)
    st.generation(x, y)
    best = st.best_params()
    fmax = st.fitness()[0].max()
    for _ in range(6):
        st.generation(x, y)
        np.testing.assert_array_equal(st.best_params(), best)
        assert st.fitness()[0].max() >= fmax
        fmax = st.fitness()[0].max()


def test_variation_eventually_improves_on_a_fixed_batch(oracle_mod):
    dims, pop = [784, 6, 10], 16
    prm = oracle_mod.Params(n_elite=1, sigma=0.05)
    st = oracle_mod.State(pop, dims, prm, seed=2)
    x, y = synthetic.make_split(32, 6)
    st.generation(x, y)
    f0 = st.fitness()[0].max()
    for _ in range(15):
        st.generation(x, y)
    assert st.fitness()[0].max() > f0


def test_normal_init_has_fan_in_variance(oracle_mod):
    dims = [784, 32, 10]
    popv = oracle_mod.init(4, dims, 0, seed=1)
    w1 = popv[:, :784 * 32].ravel() * math.sqrt(784)
    w2 = popv[:, 784 * 32 + 32:784 * 32 + 32 + 320].ravel() * math.sqrt(32)
    assert stats.kstest(w1, "norm").pvalue > 1e-4
    assert stats.kstest(w2, "norm").pvalue > 1e-4
    assert (popv[:, 784 * 32:784 * 32 + 32] == 0).all() and (popv[:, -10:] == 0).all()


def test_glorot_uniform_init(oracle_mod):
    dims = [784, 32, 10]
    popv = oracle_mod.init(3, dims, 1, seed=2)
    a1 = math.sqrt(6.0 / (784 + 32))
    w1 = popv[:, :784 * 32].ravel()
    assert np.abs(w1).max() < a1
    assert stats.kstest((w1 + a1) / (2 * a1), "uniform").pvalue > 1e-4
    a2 = math.sqrt(6.0 / (32 + 10))
    w2 = popv[:, 784 * 32 + 32:784 * 32 + 32 + 320].ravel()
    assert np.abs(w2).max() < a2


def test_init_is_deterministic_and_individuals_differ(oracle_mod):
    a = oracle_mod.init(3, [5, 4, 3], 0, seed=9)
    b = oracle_mod.init(3, [5, 4, 3], 0, seed=9)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a[0], a[1])
