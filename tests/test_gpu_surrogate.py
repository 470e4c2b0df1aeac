"""Parity of the surrogate form's hand-written MLP kernels (forward, mean
squared error gradient, Adam) with the FP64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(325, 64, 64, 256), (325, 64, 64, 37), (13, 7, 5, 9), (40, 33, 17, 100)]


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float32))).cuda()


@pytest.mark.parametrize("d_in,h1,h2,n", SHAPES[:1] + SHAPES[2:3])
def test_init_matches_oracle(gpu, oracle_mod, d_in, h1, h2, n):
    import torch
    theta = torch.empty(gpu.leea_surrogate_num_params(d_in, h1, h2), dtype=torch.float32, device="cuda")
    gpu.leea_surrogate_init(d_in, h1, h2, 77, theta)
    ref = oracle_mod.mlp_init(d_in, h1, h2, 77)
    np.testing.assert_allclose(theta.cpu().numpy(), ref, rtol=3e-7, atol=0)


@pytest.mark.parametrize("d_in,h1,h2,n", SHAPES)
def test_forward_and_gradient_match_oracle(gpu, oracle_mod, d_in, h1, h2, n):
    import torch
    rng = np.random.default_rng(d_in + n)
    theta = oracle_mod.mlp_init(d_in, h1, h2, 5) + rng.normal(0, 0.01, size=oracle_mod.mlp_num_params(d_in, h1, h2))
    theta = theta.astype(np.float32).astype(np.float64)  # the same values on both sides
    x = rng.normal(size=(n, d_in)).astype(np.float32).astype(np.float64)
    t = rng.normal(size=n).astype(np.float32).astype(np.float64)
    th_d, x_d, t_d = _t(theta), _t(x), _t(t)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    gpu.leea_surrogate_forward(n, d_in, h1, h2, th_d, x_d, y)
    y_ref = oracle_mod.mlp_forward(theta, x, d_in, h1, h2)
    np.testing.assert_allclose(y.cpu().numpy(), y_ref, rtol=1e-5, atol=1e-5)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    grad = torch.empty_like(th_d)
    work = torch.empty(gpu.leea_surrogate_work_floats(n, h1, h2), dtype=torch.float32, device="cuda")
    gpu.leea_surrogate_loss_grad(n, d_in, h1, h2, th_d, x_d, t_d, loss, grad, work)
    assert gpu.leea_device_status() == 0
    l_ref, g_ref = oracle_mod.mlp_loss_grad(theta, x, t, d_in, h1, h2)
    assert abs(loss.item() - l_ref) <= 1e-5 * abs(l_ref)
    g = grad.cpu().numpy()
    np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=1e-4 * np.abs(g_ref).max())


def test_adam_matches_oracle(gpu, oracle_mod):
    import torch
    rng = np.random.default_rng(3)
    n = 1000
    theta = rng.normal(size=n).astype(np.float32).astype(np.float64)
    m, v = np.zeros(n), np.zeros(n)
    th_d, m_d, v_d = _t(theta), _t(m), _t(v)
    for step in range(1, 4):
        g = rng.normal(size=n).astype(np.float32).astype(np.float64)
        gpu.leea_surrogate_adam(n, th_d, _t(g), m_d, v_d, step, lr=1e-2)
        # the hyperparameters as the FP32 values the kernel receives
        f32 = lambda q: float(np.float32(q))
        theta, m, v = oracle_mod.adam(theta, g, m, v, step, lr=f32(1e-2), beta1=f32(0.9), beta2=f32(0.999),
                                      eps=f32(1e-8))
        np.testing.assert_allclose(th_d.cpu().numpy(), theta, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(m_d.cpu().numpy(), m, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(v_d.cpu().numpy(), v, rtol=1e-5, atol=1e-9)


def test_training_fits_a_smooth_target(gpu):
    """The kernels train: 300 Adam steps on y = sin(x0) + x1 x2 cut the loss tenfold."""
    import torch
    d_in, h1, h2, n = 8, 32, 32, 512
    rng = np.random.default_rng(0)
    x = rng.normal(size=(n, d_in)).astype(np.float32)
    t = (np.sin(x[:, 0]) + x[:, 1] * x[:, 2]).astype(np.float32)
    npar = gpu.leea_surrogate_num_params(d_in, h1, h2)
    th = torch.empty(npar, dtype=torch.float32, device="cuda")
    gpu.leea_surrogate_init(d_in, h1, h2, 1, th)
    m, v = torch.zeros_like(th), torch.zeros_like(th)
    grad, loss = torch.empty_like(th), torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(gpu.leea_surrogate_work_floats(n, h1, h2), dtype=torch.float32, device="cuda")
    x_d, t_d = _t(x), _t(t)
    losses = []
    for step in range(1, 301):
        gpu.leea_surrogate_loss_grad(n, d_in, h1, h2, th, x_d, t_d, loss, grad, work)
        if step in (1, 300):
            losses.append(loss.item())
        gpu.leea_surrogate_adam(npar, th, grad, m, v, step, lr=1e-2)
    assert losses[1] < 0.1 * losses[0], losses


def test_surrogate_argument_errors(gpu):
    import torch
    th = torch.empty(10, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.LeeaError):
        gpu.leea_surrogate_init(0, 4, 4, 1, th)
    with pytest.raises(gpu.LeeaError, match="work"):
        x = torch.empty((5, 3), dtype=torch.float32, device="cuda")
        gpu.leea_surrogate_loss_grad(5, 3, 4, 4, th, x, th, th, th, torch.empty(3, device="cuda"))
    with pytest.raises(gpu.LeeaError):
        gpu.leea_surrogate_adam(10, th, th, th, th, 0)


# ---- recipes, their materialisation and descriptors ------------------------------------
PRM_S = dict(sigma=0.05, mut_rate=0.2, n_elite=2, p_c=0.5, xo_gene_p=0.5)


def _recipes(gpu, oracle_mod, pop=40, mult=4, seed=7, gen=3, **extra):
    import torch
    rng = np.random.default_rng(pop)
    f = rng.normal(-2.3, 0.2, size=pop).astype(np.float32)
    prm = gpu.Params(**PRM_S, **extra)
    n = gpu.leea_num_recipes(pop, prm, mult)
    fd = _t(f)
    order = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_rank(pop, fd, order)
    p1, p2, kind, ent = (torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4))
    f_inh = torch.empty(n, dtype=torch.float32, device="cuda")
    gpu.leea_select_recipes(pop, prm, fd, order, seed, gen, mult, p1, p2, kind, f_inh, ent)
    return f, order, (p1, p2, kind, f_inh, ent)


@pytest.mark.parametrize("sel_op", [0, 1])
def test_recipes_bit_exact(gpu, oracle_mod, sel_op):
    pop, mult = 40, 4
    f, order, (p1, p2, kind, f_inh, ent) = _recipes(gpu, oracle_mod, pop, mult, sel_op=sel_op, tour_k=3)
    oprm = oracle_mod.Params(**PRM_S, sel_op=sel_op, tour_k=3)
    o_order = oracle_mod.rank(f.astype(np.float64))
    np.testing.assert_array_equal(order.cpu().numpy(), o_order)
    r1, r2, rk, rinh, rent = oracle_mod.select_recipes(oprm, f.astype(np.float64), o_order, 7, 3, mult)
    np.testing.assert_array_equal(p1.cpu().numpy(), r1)
    np.testing.assert_array_equal(p2.cpu().numpy(), r2)
    np.testing.assert_array_equal(kind.cpu().numpy(), rk)
    np.testing.assert_array_equal(ent.cpu().numpy().view(np.uint32), rent)
    np.testing.assert_allclose(f_inh.cpu().numpy(), rinh, rtol=2 ** -23, atol=0)


def test_breed_entities_matches_oracle(gpu, oracle_mod):
    import torch
    from helpers import assert_genes_close, to_device_pop
    dims = [64, 32, 10]
    pop, mult = 24, 2
    f, order, (p1, p2, kind, f_inh, ent) = _recipes(gpu, oracle_mod, pop, mult)
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    parents = np.random.default_rng(4).normal(0, 0.3, size=(pop, c)).astype(np.float32)
    n = kind.numel()
    kids = torch.zeros((n, cp), dtype=torch.float32, device="cuda")
    gpu.leea_breed_entities(pop, dims, gpu.Params(**PRM_S), 7, 3, to_device_pop(parents, cp), p1, p2, kind, ent, n,
                            kids)
    assert gpu.leea_device_status() == 0
    ref = oracle_mod.breed_entities(oracle_mod.Params(**PRM_S), dims, 7, 3, parents.astype(np.float64),
                                    p1.cpu().numpy(), p2.cpu().numpy(), kind.cpu().numpy(),
                                    ent.cpu().numpy().view(np.uint32))
    assert_genes_close(kids[:, :c].cpu().numpy(), ref, PRM_S["sigma"])


@pytest.mark.parametrize("dims,n_probe", [([784, 112, 10], 32), ([64, 32, 10], 32), ([128, 256, 16], 7),
                                          ([96, 16, 3], 1), ([784, 128, 10], 20)])
@pytest.mark.parametrize("xo_op", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_descriptors_match_oracle(gpu, oracle_mod, dims, n_probe, xo_op, precision):
    # precision 0: the FP32 child on the CUDA cores; 1: the child's W1 in BF16
    # on the tensor cores (h <= 128), against the oracle's BF16 rounding of it
    import torch
    from helpers import to_device_pop
    if precision == 1 and dims[1] > 128:
        pytest.skip("the tensor-core probe takes h <= 128")
    pop, mult = 20, 2
    prm = gpu.Params(**PRM_S, xo_op=xo_op, precision=precision)
    oprm = oracle_mod.Params(**PRM_S, xo_op=xo_op, precision=precision)
    f, order, (p1, p2, kind, f_inh, ent) = _recipes(gpu, oracle_mod, pop, mult)
    # add two elite-kind rows (plain copies) at the end
    kind_h = np.concatenate([kind.cpu().numpy(), [0, 0]]).astype(np.int32)
    p1_h = np.concatenate([p1.cpu().numpy(), [3, 5]]).astype(np.int32)
    p2_h = np.concatenate([p2.cpu().numpy(), [3, 5]]).astype(np.int32)
    inh_h = np.concatenate([f_inh.cpu().numpy(), f[[3, 5]]]).astype(np.float32)
    ent_h = np.concatenate([ent.cpu().numpy().view(np.uint32), [11, 12]]).astype(np.uint32)
    n = kind_h.size
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    parents = np.random.default_rng(dims[1]).normal(0, 0.1, size=(pop, c)).astype(np.float32)
    probe = (np.random.default_rng(5).integers(0, 256, size=(n_probe, dims[0])) / 255.0).astype(np.float32)
    desc = torch.empty((n, 5 + n_probe * dims[-1]), dtype=torch.float32, device="cuda")
    gpu.leea_descriptors(pop, dims, prm, 7, 3, to_device_pop(parents, cp), _t(f), _t(p1_h).int(), _t(p2_h).int(),
                         _t(kind_h).int(), _t(inh_h), torch.from_numpy(ent_h.view(np.int32)).cuda(), n, _t(probe),
                         n_probe, desc)
    got = desc.cpu().numpy().astype(np.float64)
    ref = oracle_mod.descriptors(oprm, dims, 7, 3, parents.astype(np.float64), f.astype(np.float64), p1_h, p2_h,
                                 kind_h, inh_h.astype(np.float64), ent_h, probe.astype(np.float64))
    np.testing.assert_array_equal(got[:, :3], ref[:, :3].astype(np.float32))
    np.testing.assert_allclose(got[:, 3], ref[:, 3], rtol=1e-6, atol=0)
    np.testing.assert_allclose(got[:, 4], ref[:, 4], rtol=1e-5, atol=0)
    scale = np.abs(ref[:, 5:]).max()
    if precision == 0:
        np.testing.assert_allclose(got[:, 5:], ref[:, 5:], rtol=1e-4, atol=1e-5 * scale)
        return
    # BF16: against the oracle's evaluation of the same FP32 children (made by
    # leea_breed_entities, itself checked against the oracle) rounded to BF16
    kids = torch.zeros((n, cp), dtype=torch.float32, device="cuda")
    gpu.leea_breed_entities(pop, dims, gpu.Params(**PRM_S, xo_op=xo_op), 7, 3, to_device_pop(parents, cp),
                            _t(p1_h).int(), _t(p2_h).int(), _t(kind_h).int(),
                            torch.from_numpy(ent_h.view(np.int32)).cuda(), n, kids)
    q = oracle_mod.quantize_w1(kids[:, :c].cpu().numpy().astype(np.float64), dims, 1, None)
    _, _, same = oracle_mod.evaluate(q, dims, probe.astype(np.float64), np.zeros(n_probe, dtype=np.int32),
                                     want_logits=True)
    np.testing.assert_allclose(got[:, 5:], same.reshape(n, -1), rtol=1e-4, atol=1e-5 * scale)
    # and against the oracle's own children: an FP32 child gene one ulp off the
    # oracle's may round to the neighbouring BF16 value, which moves a logit by
    # up to ulp_bf16(w) max|x| max|W2| per such gene
    err = np.abs(got[:, 5:] - ref[:, 5:])
    tight = err <= 1e-4 * np.abs(ref[:, 5:]) + 1e-5 * scale
    flip = 2.0 ** -7 * np.abs(parents).max() * 1.5 * np.abs(probe).max() * np.abs(parents).max() * 1.5
    assert tight.mean() >= 0.999 and (err <= 2 * flip + 1e-5 * scale).all(), (tight.mean(), err.max(), flip)
