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
