"""Values the paper states (tests/golden/paper_facts.json, each with its
section) checked against the oracle's layout and operator counts."""
import json
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")


@pytest.fixture(scope="module")
def facts():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_paper_net_has_92k_params(oracle_mod, facts):
    net = facts["paper_net"]
    d0 = (net["input_side"] // net["pool"]) ** 2
    dims = [d0] + net["hidden_and_output_units"]
    c = oracle_mod.num_params(dims)
    assert c == 92234
    assert round(c / 1000) == net["params_stated_thousands"]


@pytest.mark.parametrize("block", ["default_hyperparameters", "sgd_comparison_hyperparameters"])
def test_offspring_proportions_add_up(oracle_mod, facts, block):
    h = facts[block]
    assert abs(h["p_e"] + h["p_c"] + h["p_m"] - 1.0) < 1e-12
    prm = oracle_mod.Params(p_e=h["p_e"], p_c=h["p_c"], rho=h["rho"], alpha=h["alpha"], sigma=h["sigma"])
    n_e, n_c, n_m, pool = oracle_mod.counts(h["lambda"], prm)
    lam = h["lambda"]
    assert (n_e, n_c, n_m) == (round(h["p_e"] * lam), round(h["p_c"] * lam), round(h["p_m"] * lam))
    assert pool == int(h["rho"] * lam)


def test_oracle_defaults_are_the_paper_block(oracle_mod, facts):
    h = facts["default_hyperparameters"]
    p = oracle_mod.Params()
    assert (p.xo_op, p.p_e, p.p_c, p.alpha, p.sigma, p.rho) == (0, h["p_e"], h["p_c"], h["alpha"], h["sigma"], h["rho"])


def test_capacity_claim_is_consistent(facts):
    # 8k nets x 92k FP32 params plus the largest activations at batch 64 fit in 16 GB.
    cap = facts["capacity_claim"]
    params_bytes = cap["networks"] * 92234 * 4
    act_bytes = cap["networks"] * cap["batch"] * (196 + 256 + 128 + 64 + 10) * 4
    assert params_bytes + act_bytes < cap["gpu_memory_gb"] * 1e9
