"""Pins of the oracle's surrogate-form functions: the MLP against PyTorch's
float64 layers and autograd and against central finite differences, Adam
against torch.optim.Adam and its closed-form first step, and the recipe
descriptors against the children they describe."""
import numpy as np
import pytest
import torch
from scipy import stats

D_IN, H1, H2 = 13, 7, 5


def _torch_mlp(theta, d_in, h1, h2):
    th = torch.tensor(theta, dtype=torch.float64)
    i = 0
    W1 = th[i:i + h1 * d_in].reshape(h1, d_in); i += h1 * d_in
    b1 = th[i:i + h1]; i += h1
    W2 = th[i:i + h2 * h1].reshape(h2, h1); i += h2 * h1
    b2 = th[i:i + h2]; i += h2
    w3 = th[i:i + h2]; i += h2
    b3 = th[i]
    return W1, b1, W2, b2, w3, b3


def _random_theta(oracle_mod, seed=0, d_in=D_IN, h1=H1, h2=H2):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.5, size=oracle_mod.mlp_num_params(d_in, h1, h2))


def test_num_params(oracle_mod):
    assert oracle_mod.mlp_num_params(325, 64, 64) == 325 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def test_forward_matches_torch(oracle_mod):
    theta = _random_theta(oracle_mod)
    x = np.random.default_rng(1).normal(size=(20, D_IN))
    W1, b1, W2, b2, w3, b3 = _torch_mlp(theta, D_IN, H1, H2)
    xt = torch.tensor(x)
    ref = torch.relu(torch.relu(xt @ W1.T + b1) @ W2.T + b2) @ w3 + b3
    np.testing.assert_allclose(oracle_mod.mlp_forward(theta, x, D_IN, H1, H2), ref.numpy(), rtol=1e-13, atol=1e-13)


def test_loss_and_gradient_match_torch_autograd(oracle_mod):
    theta = _random_theta(oracle_mod, seed=2)
    rng = np.random.default_rng(3)
    x, t = rng.normal(size=(31, D_IN)), rng.normal(size=31)
    loss, grad = oracle_mod.mlp_loss_grad(theta, x, t, D_IN, H1, H2)
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    i = 0
    parts = []
    for n in (H1 * D_IN, H1, H2 * H1, H2, H2, 1):
        parts.append(th[i:i + n]); i += n
    W1, b1, W2, b2, w3, b3 = (parts[0].reshape(H1, D_IN), parts[1], parts[2].reshape(H2, H1), parts[3], parts[4],
                              parts[5][0])
    y = torch.relu(torch.relu(torch.tensor(x) @ W1.T + b1) @ W2.T + b2) @ w3 + b3
    lt = torch.mean((y - torch.tensor(t)) ** 2)
    lt.backward()
    assert abs(loss - lt.item()) <= 1e-13 * abs(loss)
    np.testing.assert_allclose(grad, th.grad.numpy(), rtol=1e-11, atol=1e-13)


def test_gradient_matches_central_differences(oracle_mod):
    theta = _random_theta(oracle_mod, seed=4)
    rng = np.random.default_rng(5)
    x, t = rng.normal(size=(9, D_IN)), rng.normal(size=9)
    _, grad = oracle_mod.mlp_loss_grad(theta, x, t, D_IN, H1, H2)
    h = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (oracle_mod.mlp_loss_grad(tp, x, t, D_IN, H1, H2)[0] -
                 oracle_mod.mlp_loss_grad(tm, x, t, D_IN, H1, H2)[0]) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-5, atol=1e-8)


def test_adam_matches_torch_and_first_step_closed_form(oracle_mod):
    rng = np.random.default_rng(6)
    theta = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(4)]
    m, v = np.zeros(50), np.zeros(50)
    th = theta.copy()
    p = torch.tensor(theta.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for k, g in enumerate(grads, start=1):
        th_new, m, v = oracle_mod.adam(th, g, m, v, k, lr=1e-2)
        if k == 1:  # m_hat = g, v_hat = g^2: the step is lr * g / (|g| + eps)
            np.testing.assert_allclose(th - th_new, 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
        th = th_new
        opt.zero_grad()
        p.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_init_is_glorot_uniform(oracle_mod):
    d_in, h1, h2 = 325, 64, 64
    theta = oracle_mod.mlp_init(d_in, h1, h2, seed=9)
    W1 = theta[:h1 * d_in]
    b1 = theta[h1 * d_in:h1 * d_in + h1]
    a = np.sqrt(6.0 / (d_in + h1))
    assert np.abs(W1).max() <= a and (b1 == 0).all() and theta[-1] == 0.0
    assert stats.kstest((W1 + a) / (2 * a), "uniform").pvalue > 1e-4
    assert not np.array_equal(theta, oracle_mod.mlp_init(d_in, h1, h2, seed=10))


DIMS = [24, 8, 3]
PRM = dict(sigma=0.1, mut_rate=0.3, n_elite=2, p_c=0.5, xo_gene_p=0.4)


def _population(oracle_mod, pop=10, seed=0):
    rng = np.random.default_rng(seed)
    c = oracle_mod.num_params(DIMS)
    return rng.normal(size=(pop, c)), rng.normal(-2.0, 0.3, size=pop)


def test_recipes_follow_the_selection_rules(oracle_mod):
    popv, f = _population(oracle_mod, pop=40)
    prm = oracle_mod.Params(**PRM)
    order = oracle_mod.rank(f)
    n_e, n_c, n_m, pool = oracle_mod.counts(40, prm)
    p1, p2, kind, f_inh, ent = oracle_mod.select_recipes(prm, f, order, 5, 3, 4)
    assert kind.size == 4 * (n_c + n_m)
    assert (kind[:4 * n_c] == oracle_mod.CROSSOVER).all() and (kind[4 * n_c:] == oracle_mod.MUTATION).all()
    np.testing.assert_array_equal(ent, oracle_mod.RECIPE_ENTITY0 + np.arange(kind.size))
    top = set(order[:pool].tolist())
    assert set(p1.tolist()) <= top and set(p2.tolist()) <= top
    np.testing.assert_array_equal(p1[4 * n_c:], p2[4 * n_c:])
    np.testing.assert_allclose(f_inh[:4 * n_c], 0.5 * (f[p1[:4 * n_c]] + f[p2[:4 * n_c]]), rtol=0, atol=0)
    np.testing.assert_array_equal(f_inh[4 * n_c:], f[p1[4 * n_c:]])
    # draws over the truncation pool are uniform
    p1b, _, _, _, _ = oracle_mod.select_recipes(prm, f, order, 6, 1, 400)
    counts = np.bincount(np.searchsorted(np.sort(order[:pool]), p1b), minlength=pool)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_breed_entities_equals_breed_with_entity_j(oracle_mod):
    popv, _ = _population(oracle_mod, pop=12)
    prm = oracle_mod.Params(**PRM)
    kind = np.array([0, 1, 1, 2, 2, 1, 2, 0, 1, 2, 2, 1], dtype=np.int32)
    p1 = np.arange(12, dtype=np.int32)[::-1].copy()
    p2 = (p1 + 3) % 12
    full = oracle_mod.breed(prm, DIMS, 7, 2, popv, p1, p2, kind)
    np.testing.assert_array_equal(oracle_mod.breed_entities(prm, DIMS, 7, 2, popv, p1, p2, kind, np.arange(12)), full)


def test_recipe_stats_describe_the_child(oracle_mod):
    popv, f = _population(oracle_mod, pop=30, seed=1)
    prm = oracle_mod.Params(**PRM)
    order = oracle_mod.rank(f)
    p1, p2, kind, f_inh, ent = oracle_mod.select_recipes(prm, f, order, 11, 4, 3)
    p2 = np.where(kind == oracle_mod.CROSSOVER, np.where(p2 == p1, (p1 + 1) % 30, p2), p2).astype(np.int32)
    kids = oracle_mod.breed_entities(prm, DIMS, 11, 4, popv, p1, p2, kind, ent)
    xf, mn = oracle_mod.recipe_stats(prm, DIMS, 11, 4, kind, ent)
    c = oracle_mod.num_params(DIMS)
    xo = kind == oracle_mod.CROSSOVER
    from_b = (kids[xo] == popv[p2[xo]]) & (popv[p1[xo]] != popv[p2[xo]])
    np.testing.assert_allclose(xf[xo], from_b.sum(axis=1) / c, rtol=0, atol=1e-15)
    mu = kind == oracle_mod.MUTATION
    np.testing.assert_allclose(mn[mu], np.linalg.norm(kids[mu] - popv[p1[mu]], axis=1), rtol=1e-12)
    assert (xf[mu] == 0).all() and (mn[xo] == 0).all()
    arith = oracle_mod.Params(**{**PRM, "xo_op": 1})
    assert (oracle_mod.recipe_stats(arith, DIMS, 11, 4, kind, ent)[0][xo] == 0.5).all()


def test_descriptors_hold_parent_fitness_stats_and_probe_logits(oracle_mod):
    popv, f = _population(oracle_mod, pop=16, seed=2)
    prm = oracle_mod.Params(**PRM)
    order = oracle_mod.rank(f)
    p1, p2, kind, f_inh, ent = oracle_mod.select_recipes(prm, f, order, 3, 9, 2)
    probe = np.random.default_rng(4).uniform(0, 1, size=(5, DIMS[0]))
    desc = oracle_mod.descriptors(prm, DIMS, 3, 9, popv, f, p1, p2, kind, f_inh, ent, probe)
    assert desc.shape == (kind.size, 5 + 5 * DIMS[-1])
    np.testing.assert_array_equal(desc[:, 0], f[p1])
    np.testing.assert_array_equal(desc[:, 1], f[p2])
    np.testing.assert_array_equal(desc[:, 2], f_inh)
    xf, mn = oracle_mod.recipe_stats(prm, DIMS, 3, 9, kind, ent)
    np.testing.assert_array_equal(desc[:, 3], xf)
    np.testing.assert_array_equal(desc[:, 4], mn)
    kids = oracle_mod.breed_entities(prm, DIMS, 3, 9, popv, p1, p2, kind, ent)
    _, _, logits = oracle_mod.evaluate(kids, DIMS, probe, np.zeros(5, dtype=np.int32), want_logits=True)
    np.testing.assert_array_equal(desc[:, 5:], logits.reshape(kind.size, -1))


def test_bf16_descriptors_use_the_bf16_child(oracle_mod):
    # precision 1: the logits are those of the child whose W1 is its FP32 value
    # rounded to BF16 (quantize_w1 is pinned to torch's bfloat16 rounding);
    # the other columns do not change.
    popv, f = _population(oracle_mod, pop=16, seed=6)
    prm = oracle_mod.Params(**PRM)
    prm_b = oracle_mod.Params(**PRM, precision=1)
    order = oracle_mod.rank(f)
    p1, p2, kind, f_inh, ent = oracle_mod.select_recipes(prm, f, order, 3, 9, 2)
    probe = np.random.default_rng(8).uniform(0, 1, size=(4, DIMS[0]))
    d32 = oracle_mod.descriptors(prm, DIMS, 3, 9, popv, f, p1, p2, kind, f_inh, ent, probe)
    d16 = oracle_mod.descriptors(prm_b, DIMS, 3, 9, popv, f, p1, p2, kind, f_inh, ent, probe)
    np.testing.assert_array_equal(d16[:, :5], d32[:, :5])
    kids = oracle_mod.breed_entities(prm, DIMS, 3, 9, popv, p1, p2, kind, ent)
    n_w1 = DIMS[0] * DIMS[1]
    q = kids.copy()
    q[:, :n_w1] = oracle_mod.quantize_w1(kids.astype(np.float32).astype(np.float64), DIMS, 1, None)[:, :n_w1]
    _, _, logits = oracle_mod.evaluate(q, DIMS, probe, np.zeros(4, dtype=np.int32), want_logits=True)
    np.testing.assert_array_equal(d16[:, 5:], logits.reshape(kind.size, -1))
    assert np.abs(d16[:, 5:] - d32[:, 5:]).max() > 0  # the rounding is visible
