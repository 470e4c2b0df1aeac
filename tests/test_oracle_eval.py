"""Pins of the oracle's fitness (Eq. 1: negative mean cross-entropy of the
softmax output; ReLU hidden layers, Section 4.1) against closed forms, brute
force, and torch's float64 library routines."""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_1806_09819_gb300 import synthetic


def _split(theta, dims):
    """Unpack one individual (W row-major out x in, then b, per layer)."""
    out, i = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = theta[i:i + a * b].reshape(b, a)
        i += a * b
        bias = theta[i:i + b]
        i += b
        out.append((W, bias))
    assert i == len(theta)
    return out


def _torch_fitness(popv, dims, x, y):
    """Independent float64 forward with torch library ops."""
    f = []
    for theta in popv:
        a = torch.tensor(x, dtype=torch.float64)
        layers = _split(np.asarray(theta), dims)
        for l, (W, b) in enumerate(layers):
            a = a @ torch.tensor(W).T + torch.tensor(b)
            if l + 1 < len(layers):
                a = torch.relu(a)
        f.append(-F.cross_entropy(a, torch.tensor(y, dtype=torch.long)).item())
    return np.array(f)


def test_zero_weights_give_minus_log_classes(oracle_mod):
    dims = [784, 32, 10]
    c = oracle_mod.num_params(dims)
    popv = np.zeros((3, c))
    x, y = synthetic.make_split(50, 3)
    f, cor = oracle_mod.evaluate(popv, dims, x, y)
    np.testing.assert_allclose(f, -math.log(10.0), rtol=0, atol=1e-13)
    # All logits tie: argmax goes to class 0.
    assert (cor == int((y == 0).sum())).all()


def test_identity_net_reduces_to_library_cross_entropy(oracle_mod):
    # W1 = I, b1 = +s (ReLU inactive for x > -s), W2 = I, b2 = -s => logits = x.
    d, s = 10, 50.0
    dims = [d, d, d]
    theta = np.concatenate([np.eye(d).ravel(), np.full(d, s), np.eye(d).ravel(), np.full(d, -s)])
    rng = np.random.default_rng(0)
    x = rng.normal(0.0, 3.0, size=(40, d))
    y = rng.integers(0, d, size=40).astype(np.int32)
    f, _ = oracle_mod.evaluate(theta[None, :], dims, x, y)
    ref = -F.cross_entropy(torch.tensor(x), torch.tensor(y, dtype=torch.long)).item()
    assert abs(f[0] - ref) < 1e-12


@pytest.mark.parametrize("dims,batch", [([784, 32, 10], 16), ([784, 112, 10], 7), ([5, 3, 4], 9),
                                        ([196, 256, 128, 64, 10], 5), ([6, 4], 3)])
def test_random_nets_match_torch_float64(oracle_mod, dims, batch):
    c = oracle_mod.num_params(dims)
    rng = np.random.default_rng(len(dims) * 100 + batch)
    popv = rng.normal(0.0, 0.2, size=(4, c))
    x = rng.uniform(0.0, 1.0, size=(batch, dims[0]))
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    f, _ = oracle_mod.evaluate(popv, dims, x, y)
    np.testing.assert_allclose(f, _torch_fitness(popv, dims, x, y), rtol=1e-12, atol=1e-12)


def test_brute_force_2_2_2(oracle_mod):
    # Hand-written scalar formula of a 2-2-2 net for P = 4 individuals.
    dims = [2, 2, 2]
    rng = np.random.default_rng(11)
    popv = rng.normal(0.0, 1.0, size=(4, 12))
    x = rng.uniform(-1, 1, size=(6, 2))
    y = rng.integers(0, 2, size=6).astype(np.int32)
    f, cor = oracle_mod.evaluate(popv, dims, x, y)
    for p in range(4):
        w11, w12, w21, w22, c1, c2, v11, v12, v21, v22, d1, d2 = popv[p]
        tot, ok = 0.0, 0
        for b in range(6):
            x1, x2 = x[b]
            h1 = max(0.0, w11 * x1 + w12 * x2 + c1)
            h2 = max(0.0, w21 * x1 + w22 * x2 + c2)
            z1 = v11 * h1 + v12 * h2 + d1
            z2 = v21 * h1 + v22 * h2 + d2
            q = [math.exp(z1) / (math.exp(z1) + math.exp(z2)), math.exp(z2) / (math.exp(z1) + math.exp(z2))]
            tot += -math.log(q[y[b]])
            ok += int((0 if z1 >= z2 else 1) == y[b])
        assert abs(f[p] - (-tot / 6)) < 1e-12
        assert cor[p] == ok


def test_logits_output_and_argmax_ties(oracle_mod):
    dims = [3, 2, 3]
    theta = np.zeros(oracle_mod.num_params(dims))
    theta[-3:] = [1.0, 1.0, 0.0]  # b2: classes 0 and 1 tie on top
    x = np.zeros((4, 3))
    y = np.array([0, 1, 2, 0], dtype=np.int32)
    f, cor, logits = oracle_mod.evaluate(theta[None], dims, x, y, want_logits=True)
    np.testing.assert_array_equal(logits[0], np.tile([1.0, 1.0, 0.0], (4, 1)))
    assert cor[0] == 2  # ties go to class 0


def test_nan_weights_give_nan_fitness(oracle_mod):
    dims = [4, 3, 2]
    popv = np.zeros((2, oracle_mod.num_params(dims)))
    popv[1, 0] = np.nan
    x = np.ones((3, 4))
    y = np.zeros(3, dtype=np.int32)
    f, _ = oracle_mod.evaluate(popv, dims, x, y)
    assert np.isfinite(f[0]) and np.isnan(f[1])


def test_bad_labels_are_rejected(oracle_mod):
    dims = [4, 3, 2]
    popv = np.zeros((1, oracle_mod.num_params(dims)))
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.evaluate(popv, dims, np.ones((2, 4)), np.array([0, 2], dtype=np.int32))


def test_maxpool_matches_library_reduction(oracle_mod):
    # Section 4.1's input stage against numpy's reshape-and-max on 28x28 images
    # (and a non-square shape); ties and the block layout decide every value.
    rng = np.random.default_rng(8)
    for h, w, n in ((28, 28, 17), (6, 10, 3)):
        x = rng.integers(0, 256, size=(n, h, w)).astype(np.float64)
        x[0, :2, :2] = 7.0  # a block of equal pixels
        ref = x.reshape(n, h // 2, 2, w // 2, 2).max(axis=(2, 4)).reshape(n, -1)
        np.testing.assert_array_equal(oracle_mod.maxpool2x2(x, h, w), ref)
    # The pixel positions matter: a single bright pixel lands in its block.
    x = np.zeros((1, 4, 4))
    x[0, 3, 0] = 5.0
    np.testing.assert_array_equal(oracle_mod.maxpool2x2(x, 4, 4), [[0.0, 0.0, 5.0, 0.0]])
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.maxpool2x2(np.zeros((1, 3 * 4)), 3, 4)
