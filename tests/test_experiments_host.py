"""Host logic of the experiment harness (Section 4's protocol): the settings
grids carry the paper's stated values, scaling keeps the sample budget's
shape, and significance is the one-sided Mann-Whitney U test."""
import numpy as np
import pytest

pytest.importorskip("scipy")
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
