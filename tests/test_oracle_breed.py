"""Pins of the oracle's crossover and mutation (Section 3.2)."""
import numpy as np
import pytest
from scipy import stats

DIMS = [30, 7, 5]


def _setup(oracle_mod, kinds, seed=0):
    c = oracle_mod.num_params(DIMS)
    rng = np.random.default_rng(seed)
    pop = len(kinds)
    parents = rng.normal(0.0, 1.0, size=(pop, c))
    par1 = rng.integers(0, pop, size=pop).astype(np.int32)
    par2 = rng.integers(0, pop, size=pop).astype(np.int32)
    return parents, par1, par2, np.asarray(kinds, dtype=np.int32)


def test_crossover_of_identical_parents_returns_the_parent(oracle_mod):
    parents, par1, _, kind = _setup(oracle_mod, [oracle_mod.CROSSOVER] * 8)
    for xo_op in (0, 1):
        prm = oracle_mod.Params(xo_op=xo_op)
        kids = oracle_mod.breed(prm, DIMS, 3, 1, parents, par1, par1, kind)
        np.testing.assert_array_equal(kids, parents[par1])  # bitwise, (a + a)/2 == a


def test_zero_sigma_or_zero_rate_mutation_returns_the_parent(oracle_mod):
    parents, par1, _, kind = _setup(oracle_mod, [oracle_mod.MUTATION] * 8)
    for prm in (oracle_mod.Params(sigma=0.0), oracle_mod.Params(sigma=0.5, mut_rate=0.0)):
        kids = oracle_mod.breed(prm, DIMS, 3, 1, parents, par1, par1, kind)
        np.testing.assert_array_equal(kids, parents[par1])


def test_elite_is_an_exact_copy(oracle_mod):
    parents, par1, par2, kind = _setup(oracle_mod, [oracle_mod.ELITE] * 5)
    kids = oracle_mod.breed(oracle_mod.Params(sigma=1.0), DIMS, 3, 1, parents, par1, par2, kind)
    np.testing.assert_array_equal(kids, parents[par1])


@pytest.mark.parametrize("q", [0.0, 0.3, 0.5, 1.0])
def test_uniform_crossover_takes_each_gene_from_one_parent(oracle_mod, q):
    parents, par1, par2, kind = _setup(oracle_mod, [oracle_mod.CROSSOVER] * 40, seed=1)
    par2 = (par1 + 1) % 40  # distinct parents: every gene is decidable
    kids = oracle_mod.breed(oracle_mod.Params(xo_gene_p=q), DIMS, 7, 2, parents, par1, par2, kind)
    from_a = kids == parents[par1]
    from_b = kids == parents[par2]
    assert (from_a | from_b).all()
    frac = from_b.mean()
    n = kids.size
    assert abs(frac - q) <= 5 * np.sqrt(q * (1 - q) / n) + 1e-12
    # The choice is the 16-bit XO draw of (gen, child, gene) against floor(q 2^16).
    thr = oracle_mod.threshold16(q)
    for j in (0, 17):
        for i in (0, 1, 2, 3, 7, 8, 100, len(kids[j]) - 1):
            u = oracle_mod.draw16(7, oracle_mod.TAG_XO, 2, j, i)
            assert from_b[j, i] == (u < thr) or parents[par1[j], i] == parents[par2[j], i]


def test_arithmetic_crossover_is_the_mean(oracle_mod):
    parents, par1, par2, kind = _setup(oracle_mod, [oracle_mod.CROSSOVER] * 10, seed=2)
    kids = oracle_mod.breed(oracle_mod.Params(xo_op=1), DIMS, 1, 1, parents, par1, par2, kind)
    np.testing.assert_array_equal(kids, 0.5 * (parents[par1] + parents[par2]))


def test_mutation_mask_rate_and_normal_steps(oracle_mod):
    parents, par1, _, kind = _setup(oracle_mod, [oracle_mod.MUTATION] * 60, seed=4)
    sigma, rate = 0.01, 0.1
    kids = oracle_mod.breed(oracle_mod.Params(sigma=sigma, mut_rate=rate), DIMS, 11, 3, parents, par1, par1, kind)
    diff = kids - parents[par1]
    mask = diff != 0.0
    n = mask.size
    assert abs(mask.mean() - rate) <= 5 * np.sqrt(rate * (1 - rate) / n)
    steps = diff[mask] / sigma
    assert stats.kstest(steps, "norm").pvalue > 1e-4
    # Every gene mutates when mut_rate = 1 (the paper's operator).
    kids1 = oracle_mod.breed(oracle_mod.Params(sigma=sigma, mut_rate=1.0), DIMS, 11, 3, parents, par1, par1, kind)
    assert ((kids1 - parents[par1]) != 0).mean() > 0.999


def test_children_subrange_matches_full_breed(oracle_mod):
    parents, par1, par2, _ = _setup(oracle_mod, [0] * 12, seed=5)
    kind = np.array([0, 1, 1, 2, 2, 1, 2, 0, 1, 2, 2, 1], dtype=np.int32)
    prm = oracle_mod.Params(sigma=0.1, mut_rate=0.5)
    full = oracle_mod.breed(prm, DIMS, 2, 9, parents, par1, par2, kind)
    part = oracle_mod.breed(prm, DIMS, 2, 9, parents, par1, par2, kind, j0=4, j1=9)
    np.testing.assert_array_equal(part, full[4:9])
