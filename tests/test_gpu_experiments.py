"""The experiment harness end to end on the GPU at a tiny scale: runs finish,
report accuracies in [0, 1], are reproducible from their seed, and training
beats the untrained population."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_harness_runs_and_is_reproducible(gpu):
    import torch
    from paper_1806_09819_gb300 import experiments as E
    data = E.Data(torch.device("cuda", 0), n_train=4000, n_val=1000)
    s = E.scaled(E._setting(pop=400, batch=128, sigma=0.01), 0.1)
    a = E.run_one(s, 7, data, generations=60)
    b = E.run_one(s, 7, data, generations=60)
    assert a["val_accuracy"] == b["val_accuracy"] and a["val_fitness"] == b["val_fitness"]
    assert 0.0 <= a["val_accuracy"] <= 1.0
    untrained = E.run_one(s, 7, data, generations=0)
    assert a["val_fitness"] > untrained["val_fitness"]
    assert a["val_accuracy"] > untrained["val_accuracy"]
