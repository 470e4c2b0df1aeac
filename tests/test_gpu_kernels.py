"""Parity of each step entry point (CUDA, through the C ABI) with the FP64
oracle on the same seeded inputs: random streams, initialisation, ranking,
selection, breeding and evaluation."""
import numpy as np
import pytest

from helpers import (assert_correct_close, assert_fitness_close, assert_genes_close, from_device_pop,
                     to_device_pop)
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


# ---- random streams (bit-exact words, normals within 1e-6 relative) ---------------
@pytest.mark.parametrize("tag,gen,ent,n0,count", [(1, 0, 0, 0, 1000), (2, 7, 31, 3, 257), (3, 123, 999, 89000, 50),
                                                  (4, 2**31 + 5, 2**24, 0, 64), (5, 1, 1, 1, 4099)])
def test_philox_words_bit_exact(gpu, oracle_mod, tag, gen, ent, n0, count):
    torch = _torch()
    seed = 0x0123456789ABCDEF
    out = torch.zeros(count, dtype=torch.int64, device="cuda")  # room for uint32
    buf = torch.zeros(count, dtype=torch.int32, device="cuda")
    gpu.leea_philox_fill(seed, tag, gen, ent, n0, count, buf)
    got = buf.cpu().numpy().view(np.uint32)
    ref = np.array([oracle_mod.draw(seed, tag, gen, ent, n0 + t) for t in range(count)], dtype=np.uint32)
    np.testing.assert_array_equal(got, ref)
    del out


def test_normals_match(gpu, oracle_mod):
    torch = _torch()
    seed, count = 99, 6000
    buf = torch.zeros(count, dtype=torch.float32, device="cuda")
    gpu.leea_normal_fill(seed, 5, 3, 17, 0, count, buf)
    got = buf.cpu().numpy().astype(np.float64)
    ref = np.array([oracle_mod.normal(seed, 5, 3, 17, i) for i in range(count)])
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-9)


# ---- initialisation --------------------------------------------------------------
@pytest.mark.parametrize("dims", [[784, 32, 10], [2, 2, 2], [5, 3, 4], [196, 256, 128, 64, 10]])
@pytest.mark.parametrize("init", [0, 1])
def test_init_matches_oracle(gpu, oracle_mod, dims, init):
    torch = _torch()
    pop = 3
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    t = torch.full((pop, cp), 7.0, dtype=torch.float32, device="cuda")
    gpu.leea_init_population(pop, dims, init, 2024, t)
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    ref = oracle_mod.init(pop, dims, init, 2024)
    np.testing.assert_allclose(got[:, :c], ref, rtol=1e-6, atol=1e-9)
    assert (got[:, c:] == 0).all()


# ---- ranking (bit-exact) ------------------------------------------------------------
@pytest.mark.parametrize("pop", [1, 7, 256, 257, 1000, 2049, 5000])
def test_rank_bit_exact(gpu, oracle_mod, pop):
    torch = _torch()
    rng = np.random.default_rng(pop)
    f = rng.normal(-2.0, 0.3, size=pop).astype(np.float32)
    if pop > 10:
        f[rng.integers(0, pop, size=pop // 5)] = -2.0          # ties
        f[rng.integers(0, pop, size=max(1, pop // 50))] = np.nan
        f[rng.integers(0, pop, size=max(1, pop // 50))] = -np.inf
        f[rng.integers(0, pop, size=2)] = -0.0
        f[rng.integers(0, pop, size=2)] = 0.0
    fd = torch.from_numpy(f).cuda()
    order = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_rank(pop, fd, order)
    np.testing.assert_array_equal(order.cpu().numpy(), oracle_mod.rank(f.astype(np.float64)))


# ---- selection (bit-exact indices) ---------------------------------------------------------
SEL_CASES = [
    dict(pop=4, prm=dict()),
    dict(pop=32, prm=dict(sel_op=1, tour_k=3)),
    dict(pop=1000, prm=dict(n_elite=1)),
    dict(pop=1000, prm=dict(sel_op=1, tour_k=5, p_c=0.75)),
    dict(pop=4097, prm=dict(rho=0.1, p_e=0.01)),
    dict(pop=1, prm=dict()),
    dict(pop=33, prm=dict(sel_op=1, tour_k=1, n_elite=0, p_c=1.0)),
]


@pytest.mark.parametrize("case", SEL_CASES, ids=lambda c: f"pop{c['pop']}-{c['prm']}")
def test_select_bit_exact(gpu, oracle_mod, case):
    torch = _torch()
    pop = case["pop"]
    rng = np.random.default_rng(pop)
    f = rng.normal(-2.0, 0.2, size=pop).astype(np.float32)
    f[rng.integers(0, pop, size=pop // 4)] = -2.0
    fd = torch.from_numpy(f).cuda()
    order = torch.empty(pop, dtype=torch.int32, device="cuda")
    outs = [torch.empty(pop, dtype=torch.int32, device="cuda") for _ in range(3)]
    f_inh = torch.empty(pop, dtype=torch.float32, device="cuda")
    seed, gen = 31337, 12
    gpu.leea_rank(pop, fd, order)
    gpu.leea_select(pop, gpu.Params(**case["prm"]), fd, order, seed, gen, *outs, f_inh)
    torch.cuda.synchronize()
    f64 = f.astype(np.float64)
    o_order = oracle_mod.rank(f64)
    p1, p2, kind, fi = oracle_mod.select(oracle_mod.Params(**case["prm"]), f64, o_order, seed, gen)
    np.testing.assert_array_equal(outs[0].cpu().numpy(), p1)
    np.testing.assert_array_equal(outs[1].cpu().numpy(), p2)
    np.testing.assert_array_equal(outs[2].cpu().numpy(), kind)
    np.testing.assert_allclose(f_inh.cpu().numpy(), fi, rtol=2 ** -23, atol=0)


# ---- breeding -------------------------------------------------------------------------
BREED_CASES = [
    dict(dims=[784, 32, 10], pop=32, prm=dict(sel_op=1, sigma=0.01)),
    dict(dims=[784, 112, 10], pop=24, prm=dict(n_elite=1, sigma=0.005, mut_rate=0.1)),
    dict(dims=[784, 112, 10], pop=16, prm=dict(xo_op=1, sigma=0.02, p_c=0.75)),
    dict(dims=[2, 2, 2], pop=4, prm=dict(sigma=0.3)),
    dict(dims=[5, 3, 4], pop=9, prm=dict(xo_gene_p=0.2, mut_rate=0.5, sigma=0.1)),
    dict(dims=[196, 256, 128, 64, 10], pop=8, prm=dict(sigma=0.001)),
]


@pytest.mark.parametrize("case", BREED_CASES, ids=lambda c: f"{c['dims']}-{c['pop']}-{c['prm']}")
def test_breed_matches_oracle(gpu, oracle_mod, case):
    torch = _torch()
    dims, pop = case["dims"], case["pop"]
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    parents = synthetic.random_population(pop, c, seed=pop + c, scale=0.2)
    f = np.random.default_rng(1).normal(-2.0, 0.2, size=pop)
    o_prm = oracle_mod.Params(**case["prm"])
    order = oracle_mod.rank(f)
    seed, gen = 77, 5
    p1, p2, kind, _ = oracle_mod.select(o_prm, f, order, seed, gen)
    par_d = to_device_pop(parents, cp)
    kid_d = torch.full_like(par_d, 3.0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    gpu.leea_breed(pop, dims, gpu.Params(**case["prm"]), seed, gen, par_d, t(p1), t(p2), t(kind), kid_d)
    torch.cuda.synchronize()
    got = kid_d.cpu().numpy()
    assert (got[:, c:] == 0).all(), "padding must stay zero"
    ref = oracle_mod.breed(o_prm, dims, seed, gen, parents.astype(np.float64), p1, p2, kind)
    assert_genes_close(got[:, :c], ref, o_prm.sigma)
    # Masks are decided on integers: compare them exactly where they are visible.
    par1v, par2v = parents[p1].astype(np.float64), parents[p2].astype(np.float64)
    for j in range(pop):
        g, r = got[j, :c].astype(np.float64), ref[j]
        if kind[j] == oracle_mod.CROSSOVER and o_prm.xo_op == 0:
            decid = par1v[j] != par2v[j]
            np.testing.assert_array_equal((g == par2v[j])[decid], (r == par2v[j])[decid])
        elif kind[j] == oracle_mod.MUTATION:
            step = np.abs(r - par1v[j])
            vis = (step == 0) | (step > 8 * 2.0 ** -23 * np.abs(par1v[j]))
            np.testing.assert_array_equal((g != par1v[j])[vis], (r != par1v[j])[vis])
        elif kind[j] == oracle_mod.ELITE:
            np.testing.assert_array_equal(g, par1v[j])


def test_breed_rejects_overlap(gpu):
    torch = _torch()
    dims = [4, 3, 2]
    cp = gpu.leea_padded_params(dims)
    buf = torch.zeros((2, cp), dtype=torch.float32, device="cuda")
    idx = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu.LeeaError):
        gpu.leea_breed(2, dims, gpu.Params(), 1, 1, buf, idx, idx, idx, buf)


# ---- evaluation -------------------------------------------------------------------------
EVAL_CASES = [
    ([2, 2, 2], 4, 8), ([784, 32, 10], 32, 16), ([784, 112, 10], 64, 100), ([784, 37, 10], 5, 19),
    ([5, 3, 4], 6, 1), ([784, 200, 10], 3, 129), ([784, 112, 10], 4, 512), ([784, 16, 10], 7, 33),
    ([100, 300, 32], 3, 70), ([784, 256, 10], 2, 256),
    # shapes for the tensor-core kernel: ragged sample tiles, K < 32, P > SM count, d_out = 16
    ([784, 48, 10], 3, 128), ([784, 112, 10], 2, 129), ([16, 16, 2], 5, 7), ([784, 128, 16], 4, 77),
    ([784, 112, 10], 400, 100), ([784, 112, 10], 1, 1), ([36, 64, 10], 9, 300),
]


def _tc_shape(dims):
    return len(dims) == 3 and dims[0] % 4 == 0 and dims[1] % 16 == 0 and dims[1] <= 256 and dims[2] <= 16


def _eval_params():
    out = []
    for dims, pop, batch in EVAL_CASES:
        out.append(pytest.param(dims, pop, batch, 1, id=f"simt-{dims}-{pop}-{batch}"))
        if _tc_shape(dims):
            out.append(pytest.param(dims, pop, batch, 2, id=f"tensor-{dims}-{pop}-{batch}"))
    return out


@pytest.mark.parametrize("dims,pop,batch,path", _eval_params())
def test_evaluate_matches_oracle(gpu, oracle_mod, dims, pop, batch, path):
    torch = _torch()
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    popv = synthetic.random_population(pop, c, seed=c + batch, scale=0.15)
    if dims[0] == 784:
        x, y = synthetic.make_split(batch, seed=batch)
    else:
        x, y = synthetic.tiny_problem(dims[0], dims[-1], batch, seed=batch)
        y = y % dims[-1]
    f_inh = np.random.default_rng(3).normal(-2.3, 0.1, size=pop).astype(np.float32)
    alpha = 0.2
    pd = to_device_pop(popv, cp)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    fi_d = torch.from_numpy(f_inh).cuda()
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    f_adj = torch.empty_like(f_raw)
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_evaluate(pop, dims, pd, xd, yd, batch, alpha, fi_d, f_raw, f_adj, cor, eval_path=path)
    assert gpu.leea_device_status() == 0
    f_ref, cor_ref, logits = oracle_mod.evaluate(popv.astype(np.float64), dims, x.astype(np.float64), y,
                                                 want_logits=True)
    assert_fitness_close(f_raw.cpu().numpy(), f_ref)
    assert_correct_close(cor.cpu().numpy(), cor_ref, logits)
    adj_ref = oracle_mod.inherit(float(np.float32(alpha)), f_inh.astype(np.float64), f_ref, first=False)
    assert_fitness_close(f_adj.cpu().numpy(), adj_ref, "f_adj")
    # First evaluation (no f_inh): f_adj = f exactly.
    gpu.leea_evaluate(pop, dims, pd, xd, yd, batch, alpha, None, f_raw, f_adj, cor, eval_path=path)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(f_adj.cpu().numpy(), f_raw.cpu().numpy())


def test_tensor_path_rejects_unsupported_shapes(gpu):
    torch = _torch()
    dims = [784, 37, 10]
    cp = gpu.leea_padded_params(dims)
    pd = torch.zeros((2, cp), dtype=torch.float32, device="cuda")
    x = torch.zeros((4, 784), dtype=torch.float32, device="cuda")
    y = torch.zeros(4, dtype=torch.int32, device="cuda")
    f = torch.empty(2, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.LeeaError) as e:
        gpu.leea_evaluate(2, dims, pd, x, y, 4, 1.0, None, f, eval_path=gpu.EVAL_TENSOR)
    assert e.value.status == gpu.EINVAL


@pytest.mark.parametrize("path", [1, 2])
def test_evaluate_zero_weights_and_clones(gpu, oracle_mod, path):
    torch = _torch()
    dims, pop, batch = [784, 112, 10], 6, 100
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    x, y = synthetic.make_split(batch, seed=4)
    popv = np.zeros((pop, c), dtype=np.float32)
    popv[3:] = synthetic.random_population(1, c, seed=5)  # three identical clones
    pd = to_device_pop(popv, cp)
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_evaluate(pop, dims, pd, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), batch, 1.0, None,
                      f_raw, None, cor, eval_path=path)
    torch.cuda.synchronize()
    f = f_raw.cpu().numpy()
    assert np.all(np.abs(f[:3] + np.log(10.0)) < 1e-6)
    assert (cor.cpu().numpy()[:3] == (y == 0).sum()).all()
    assert f[3] == f[4] == f[5]  # bitwise: fixed reduction order


def test_tensor_and_simt_paths_agree_at_full_size(gpu):
    torch = _torch()
    dims, pop, batch = [784, 112, 10], 1000, 100
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    pd = torch.empty((pop, cp), dtype=torch.float32, device="cuda")
    gpu.leea_init_population(pop, dims, 0, 99, pd)
    x, y = synthetic.make_split(batch, seed=8)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = {}
    for path in (1, 2):
        f = torch.empty(pop, dtype=torch.float32, device="cuda")
        gpu.leea_evaluate(pop, dims, pd, xd, yd, batch, 1.0, None, f, eval_path=path)
        out[path] = f.cpu().numpy()
    assert gpu.leea_device_status() == 0
    assert_fitness_close(out[2], out[1].astype(np.float64), "tensor vs simt")


def test_evaluate_bad_label_gives_nan_and_errors(gpu):
    torch = _torch()
    dims = [4, 3, 2]
    cp = gpu.leea_padded_params(dims)
    pd = torch.zeros((2, cp), dtype=torch.float32, device="cuda")
    x = torch.ones((3, 4), dtype=torch.float32, device="cuda")
    y = torch.tensor([0, 5, 1], dtype=torch.int32, device="cuda")
    f_raw = torch.empty(2, dtype=torch.float32, device="cuda")
    gpu.leea_evaluate(2, dims, pd, x, y, 3, 1.0, None, f_raw)
    torch.cuda.synchronize()
    assert np.isnan(f_raw.cpu().numpy()).all()
    with pytest.raises(gpu.LeeaError):
        gpu.leea_evaluate(2, dims, pd, x, y, 0, 1.0, None, f_raw)
    with pytest.raises(gpu.LeeaError):  # d_out > 32: rejected before any launch
        gpu.leea_evaluate(2, [4, 3, 3, 40], pd, x, y, 3, 1.0, None, f_raw)


# ---- evaluation of 8-bit inputs (x = k / 255) ------------------------------------------------
U8_CASES = [
    ([784, 112, 10], 64, 100), ([784, 32, 10], 32, 16), ([784, 112, 10], 3, 128), ([784, 16, 10], 5, 1),
    ([36, 64, 10], 9, 33), ([784, 48, 16], 4, 77), ([784, 112, 10], 400, 100), ([784, 112, 10], 3, 129),
    ([784, 37, 10], 3, 20), ([12, 256, 10], 3, 50),
    # pairs and single individuals mixed on the CTAs (152 < pop < 304), the widest
    # pair (N = 256) with 16 outputs, inputs beyond a 512-column batch tile
    ([784, 112, 10], 200, 100), ([784, 128, 16], 5, 128), ([1600, 64, 10], 5, 40), ([20, 16, 3], 309, 7),
]


def _u8_tc_shape(dims, batch):
    k, h, d_out = dims
    return k % 4 == 0 and h % 16 == 0 and h <= 128 and d_out <= 16 and batch <= 128


def _u8_params():
    out = []
    for dims, pop, batch in U8_CASES:
        out.append(pytest.param(dims, pop, batch, 1, id=f"simt-{dims}-{pop}-{batch}"))
        if _u8_tc_shape(dims, batch):
            out.append(pytest.param(dims, pop, batch, 2, id=f"tensor-{dims}-{pop}-{batch}"))
    return out


@pytest.mark.parametrize("dims,pop,batch,path", _u8_params())
def test_evaluate_u8_matches_oracle(gpu, oracle_mod, dims, pop, batch, path):
    torch = _torch()
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    popv = synthetic.random_population(pop, c, seed=c + 7 * batch, scale=0.15)
    rng = np.random.default_rng(batch)
    levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    f_inh = rng.normal(-2.3, 0.1, size=pop).astype(np.float32)
    pd = to_device_pop(popv, cp)
    xd, yd = torch.from_numpy(levels).cuda(), torch.from_numpy(y).cuda()
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    f_adj = torch.empty_like(f_raw)
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_evaluate_u8(pop, dims, pd, xd, 255.0, yd, batch, 0.3, torch.from_numpy(f_inh).cuda(), f_raw, f_adj, cor,
                         eval_path=path)
    assert gpu.leea_device_status() == 0
    x64 = levels.astype(np.float64) / 255.0
    f_ref, cor_ref, logits = oracle_mod.evaluate(popv.astype(np.float64), dims, x64, y, want_logits=True)
    assert_fitness_close(f_raw.cpu().numpy(), f_ref)
    assert_correct_close(cor.cpu().numpy(), cor_ref, logits)
    adj_ref = oracle_mod.inherit(float(np.float32(0.3)), f_inh.astype(np.float64), f_ref, first=False)
    assert_fitness_close(f_adj.cpu().numpy(), adj_ref, "f_adj")


def test_evaluate_u8_tensor_rejects_large_batches(gpu):
    torch = _torch()
    dims = [784, 112, 10]
    cp = gpu.leea_padded_params(dims)
    pd = torch.zeros((2, cp), dtype=torch.float32, device="cuda")
    x = torch.zeros((129, 784), dtype=torch.uint8, device="cuda")
    y = torch.zeros(129, dtype=torch.int32, device="cuda")
    f = torch.empty(2, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.LeeaError):
        gpu.leea_evaluate_u8(2, dims, pd, x, 255.0, y, 129, 1.0, None, f, eval_path=gpu.EVAL_TENSOR)
    with pytest.raises(gpu.LeeaError):
        gpu.leea_evaluate_u8(2, dims, pd, x, 0.0, y, 129, 1.0, None, f)


def test_evaluate_u8_clones_and_zero_weights(gpu):
    torch = _torch()
    dims, pop, batch = [784, 112, 10], 7, 100
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    x, y = synthetic.make_split(batch, seed=4)
    popv = np.zeros((pop, c), dtype=np.float32)
    popv[3:] = synthetic.random_population(1, c, seed=5)
    pd = to_device_pop(popv, cp)
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_evaluate_u8(pop, dims, pd, torch.from_numpy(synthetic.to_levels(x)).cuda(), 255.0,
                         torch.from_numpy(y).cuda(), batch, 1.0, None, f_raw, None, cor, eval_path=gpu.EVAL_TENSOR)
    assert gpu.leea_device_status() == 0
    f = f_raw.cpu().numpy()
    assert np.all(np.abs(f[:3] + np.log(10.0)) < 1e-6)
    assert (cor.cpu().numpy()[:3] == (y == 0).sum()).all()
    assert f[3] == f[4] == f[5] == f[6]


def test_evaluate_u8_tensor_weights_outside_the_piece_range(gpu, oracle_mod):
    # Weights with |w| >= 128 do not fit the tensor path's FP16 pieces; those
    # individuals take the FP32 fallback. 400 individuals put several of them
    # on one CTA in consecutive and non-consecutive turns; the others, and
    # 127.5 (just inside the range), stay on the tensor path.
    torch = _torch()
    dims, pop, batch = [784, 112, 10], 400, 100
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    popv = synthetic.random_population(pop, c, seed=21, scale=0.05)
    for p_, w_ in ((3, 300.0), (155, -128.0), (307, 1.0e6), (160, 200.0), (9, 127.5), (161, -127.5)):
        popv[p_, (p_ * 37) % (dims[0] * dims[1])] = w_
    x, y = synthetic.make_split(batch, seed=6)
    levels = synthetic.to_levels(x)
    pd = to_device_pop(popv, cp)
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_evaluate_u8(pop, dims, pd, torch.from_numpy(levels).cuda(), 255.0, torch.from_numpy(y).cuda(), batch,
                         1.0, None, f_raw, None, cor, eval_path=gpu.EVAL_TENSOR)
    assert gpu.leea_device_status() == 0
    f_ref, cor_ref, logits = oracle_mod.evaluate(popv.astype(np.float64), dims, levels.astype(np.float64) / 255.0, y,
                                                 want_logits=True)
    assert_fitness_close(f_raw.cpu().numpy(), f_ref)
    assert_correct_close(cor.cpu().numpy(), cor_ref, logits)


def test_u8_and_float_inputs_agree(gpu):
    # The same images as float x = k/255 and as levels k: both paths within
    # the fitness tolerance of each other at the full workload size.
    torch = _torch()
    dims, pop, batch = [784, 112, 10], 1000, 100
    cp = gpu.leea_padded_params(dims)
    pd = torch.empty((pop, cp), dtype=torch.float32, device="cuda")
    gpu.leea_init_population(pop, dims, 0, 17, pd)
    x, y = synthetic.make_split(batch, seed=9)
    yd = torch.from_numpy(y).cuda()
    f_float = torch.empty(pop, dtype=torch.float32, device="cuda")
    f_u8 = torch.empty(pop, dtype=torch.float32, device="cuda")
    gpu.leea_evaluate(pop, dims, pd, torch.from_numpy(x).cuda(), yd, batch, 1.0, None, f_float, eval_path=1)
    gpu.leea_evaluate_u8(pop, dims, pd, torch.from_numpy(synthetic.to_levels(x)).cuda(), 255.0, yd, batch, 1.0, None,
                         f_u8, eval_path=2)
    assert gpu.leea_device_status() == 0
    assert_fitness_close(f_u8.cpu().numpy(), f_float.cpu().numpy().astype(np.float64), "u8 vs float")


def test_bounded_wait_gives_up_and_the_context_stays_usable(gpu):
    # The failure path of every pipeline wait, without a fault: a wait that
    # nothing completes runs to its limit, the kernel reports it through the
    # status word, the host reads LEEA_ETIMEOUT, and the context keeps working.
    import time
    torch = _torch()
    gpu.leea_device_status()  # start from a clear status word
    t0 = time.perf_counter()
    gpu.leea_selftest_wait_timeout(20000)  # 20 ms
    with pytest.raises(gpu.LeeaError) as e:
        gpu.leea_device_status()
    assert e.value.status == gpu.ETIMEOUT
    assert time.perf_counter() - t0 >= 0.02
    assert gpu.leea_device_status() == 0  # read and cleared
    dims, pop = [784, 32, 10], 3
    pd = torch.zeros((pop, gpu.leea_padded_params(dims)), dtype=torch.float32, device="cuda")
    x = torch.zeros((16, 784), dtype=torch.uint8, device="cuda")
    y = torch.arange(16, dtype=torch.int32, device="cuda") % 10
    f = torch.empty(pop, dtype=torch.float32, device="cuda")
    gpu.leea_evaluate_u8(pop, dims, pd, x, 255.0, y, 16, 1.0, None, f)
    np.testing.assert_allclose(f.cpu().numpy(), -np.log(10.0), rtol=1e-6)  # zero nets
    assert gpu.leea_device_status() == 0
    with pytest.raises(gpu.LeeaError):
        gpu.leea_selftest_wait_timeout(0)
