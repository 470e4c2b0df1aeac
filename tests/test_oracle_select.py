"""Pins of the oracle's ranking and selection (Algorithm 1; Section 3.1)."""
import numpy as np
import pytest
from scipy import stats


def test_counts_follow_the_proportions(oracle_mod):
    P = oracle_mod.Params
    # Paper defaults p_E .05, p_C .5, p_M .45 at lambda = 1000 (Section 4).
    assert oracle_mod.counts(1000, P()) == (50, 500, 450, 500)
    # "elitism 1", uniform crossover 0.5, truncation rho .5.
    assert oracle_mod.counts(1000, P(n_elite=1)) == (1, 500, 499, 500)
    # lambda = 2000, p_C .75, p_M .2 (Section 4.5).
    assert oracle_mod.counts(2000, P(p_c=0.75)) == (100, 1500, 400, 1000)
    # Rounding: round(0.05 * 32) = 2; pool never empty.
    assert oracle_mod.counts(32, P(rho=0.01)) == (2, 16, 14, 1)
    assert oracle_mod.counts(1, P()) == (0, 1, 0, 1)  # round(0.5) = 1, half away from zero


def _ref_order(f):
    key = np.where(np.isnan(f), -np.inf, f)
    return np.lexsort((np.arange(len(f)), -key)).astype(np.int32)


@pytest.mark.parametrize("seed", range(4))
def test_rank_matches_library_sort_with_ties_and_nan(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    f = rng.choice([-2.0, -1.5, -1.0, 0.0, -0.0, np.nan, -np.inf], size=257)
    f[:50] = rng.normal(size=50)
    np.testing.assert_array_equal(oracle_mod.rank(f), _ref_order(f))


def test_elites_and_inherited_fitness(oracle_mod):
    rng = np.random.default_rng(3)
    pop = 40
    f = rng.normal(size=pop)
    order = oracle_mod.rank(f)
    prm = oracle_mod.Params(n_elite=3, p_c=0.5)
    p1, p2, kind, f_inh = oracle_mod.select(prm, f, order, seed=9, gen=4)
    n_e, n_c, n_m, pool = oracle_mod.counts(pop, prm)
    assert (kind[:n_e] == oracle_mod.ELITE).all()
    assert (kind[n_e:n_e + n_c] == oracle_mod.CROSSOVER).all()
    assert (kind[n_e + n_c:] == oracle_mod.MUTATION).all()
    np.testing.assert_array_equal(p1[:n_e], order[:n_e])
    np.testing.assert_array_equal(f_inh[:n_e], f[order[:n_e]])
    xo = slice(n_e, n_e + n_c)
    np.testing.assert_allclose(f_inh[xo], 0.5 * (f[p1[xo]] + f[p2[xo]]), rtol=0, atol=0)
    mu = slice(n_e + n_c, pop)
    np.testing.assert_array_equal(f_inh[mu], f[p1[mu]])
    np.testing.assert_array_equal(p1[mu], p2[mu])
    # Truncation: every parent comes from the top `pool` of the ranking.
    top = set(order[:pool].tolist())
    assert set(p1[n_e:].tolist()) <= top and set(p2[xo].tolist()) <= top


def test_truncation_draws_are_uniform_over_the_pool(oracle_mod):
    pop = 50
    f = -np.arange(pop, dtype=np.float64)  # rank r is individual r
    order = oracle_mod.rank(f)
    prm = oracle_mod.Params(n_elite=0, p_c=1.0, rho=0.4)
    pool = oracle_mod.counts(pop, prm)[3]
    counts = np.zeros(pop)
    for g in range(1, 401):
        p1, p2, _, _ = oracle_mod.select(prm, f, order, seed=1, gen=g)
        np.add.at(counts, p1, 1)
        np.add.at(counts, p2, 1)
    assert counts[pool:].sum() == 0
    assert stats.chisquare(counts[:pool]).pvalue > 1e-4


def test_tournament_winner_distribution_closed_form(oracle_mod):
    # With k draws with replacement from P, the winner has rank r (1 = best)
    # with probability ((P - r + 1)^k - (P - r)^k) / P^k.
    pop, k, gens = 20, 3, 50000
    f = np.linspace(0.0, -1.0, pop)  # distinct, rank r-1 is individual r-1
    order = oracle_mod.rank(f)
    prm = oracle_mod.Params(sel_op=1, tour_k=k, n_elite=0, p_c=0.0)
    counts = np.zeros(pop)
    for g in range(1, gens + 1):
        p1, _, _, _ = oracle_mod.select(prm, f, order, seed=123, gen=g)
        np.add.at(counts, p1, 1)
    r = np.arange(1, pop + 1)
    expected = ((pop - r + 1.0) ** k - (pop - r) ** k) / pop ** k * counts.sum()
    assert stats.chisquare(counts, expected).pvalue > 1e-4


def test_tournament_ties_go_to_lower_index(oracle_mod):
    pop = 6
    f = np.zeros(pop)  # everybody ties: the lowest drawn index wins
    order = oracle_mod.rank(f)
    prm = oracle_mod.Params(sel_op=1, tour_k=4, n_elite=0, p_c=0.0)
    for g in range(1, 50):
        p1, _, _, _ = oracle_mod.select(prm, f, order, seed=5, gen=g)
        for j in range(pop):
            draws = [oracle_mod.index(oracle_mod.draw(5, oracle_mod.TAG_SEL, g, j, t), pop) for t in range(4)]
            assert p1[j] == min(draws)
