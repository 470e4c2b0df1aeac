"""Host logic of the experiment harness (Section 4's protocol): the settings
grids carry the paper's stated values, scaling keeps the sample budget's
shape, and significance is the one-sided Mann-Whitney U test."""
import itertools

import numpy as np
import pytest

from paper_1806_09819_gb300 import experiments as E


def test_grids_follow_the_paper():
    d = E.settings("large")[0]
    assert (d["pop"], d["batch"], d["params"]["p_c"], d["params"]["p_e"], d["params"]["sigma"]) == (
        2000, 1024, 0.75, 0.05, 0.001)
    assert d["params"]["alpha"] == 1.0 and d["params"]["rho"] == 0.5 and d["params"]["xo_op"] == 0
    sp = E.settings("selective-pressure")
    assert sorted({s["params"]["rho"] for s in sp}) == [0.1, 0.2, 0.5, 1.0]
    ba = E.settings("batch-alpha")
    assert len(ba) == 18 and {s["params"]["alpha"] for s in ba} == {0.0, 0.5, 1.0}
    cs = E.settings("crossover-sigma")
    assert len(cs) == 24 and {s["params"].get("sigma_ctl", 0) for s in cs} == {0, 1, 2}
    with pytest.raises(ValueError):
        E.settings("nope")


def test_scaling_keeps_the_sample_budget_shape():
    small, large = E._setting(batch=32), E._setting(batch=512)
    a, b = E.scaled(small, 0.1), E.scaled(large, 0.1)
    # the same number of training samples: smaller batches run longer
    assert a["generations"] == int(E.SAMPLE_BUDGET * 0.1) // 32 and b["generations"] == int(E.SAMPLE_BUDGET * 0.1) // 512
    assert a["pop"] == 100 and E.scaled(E._setting(pop=50), 0.1)["pop"] == 20


def test_mann_whitney_is_one_sided():
    rng = np.random.default_rng(0)
    hi, lo = rng.normal(1.0, 0.1, 15), rng.normal(0.0, 0.1, 15)
    assert E.mann_whitney_greater(hi, lo) < 1e-4
    assert E.mann_whitney_greater(lo, hi) > 0.99


def test_mann_whitney_exact_against_enumeration():
    # no ties, small samples: the exact p-value equals the share of all
    # C(m + n, m) equally likely rank sets whose U is at least the observed one
    rng = np.random.default_rng(3)
    for m, n in ((3, 4), (5, 2), (4, 6), (1, 7)):
        v = rng.permutation(m + n).astype(float)
        a, b = v[:m], v[m:]
        u_obs = sum(float(x > y) for x in a for y in b)
        us = []
        for pos in itertools.combinations(range(m + n), m):
            xs = [float(i) for i in pos]
            ys = [float(i) for i in range(m + n) if i not in pos]
            us.append(sum(float(x > y) for x in xs for y in ys))
        want = np.mean(np.asarray(us) >= u_obs)
        assert abs(E.mann_whitney_greater(a, b) - want) < 1e-12


def test_mann_whitney_null_counts_are_binomial_totals():
    for m, n in ((1, 1), (3, 5), (8, 8), (15, 15)):
        c = E._u_null_counts(m, n)
        assert len(c) == m * n + 1 and c.sum() == float(np.round(np.exp(
            np.sum(np.log(np.arange(1, m + n + 1))) - np.sum(np.log(np.arange(1, m + 1)))
            - np.sum(np.log(np.arange(1, n + 1))))))
        np.testing.assert_array_equal(c, c[::-1])  # U and m n - U are equally likely


def test_mann_whitney_matches_scipy_where_available():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(11)
    for m, n, ties in ((15, 15, False), (15, 15, True), (6, 9, False), (20, 7, True)):
        a, b = rng.normal(0.2, 1.0, m), rng.normal(0.0, 1.0, n)
        if ties:
            a, b = np.round(a * 2) / 2, np.round(b * 2) / 2
        want = stats.mannwhitneyu(a, b, alternative="greater").pvalue
        assert abs(E.mann_whitney_greater(a, b) - want) < 1e-9, (m, n, ties)
