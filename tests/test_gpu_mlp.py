"""The paper's own network (Section 4.1): 2x2 max-pooling of the 28x28 input,
then fully connected layers 196-256-128-64-10 with ReLU.  Parity of the CUDA
max-pool (bit-exact) and of the multi-layer FP32 evaluation (within the
evaluation tolerance, correct counts exact up to argmax near-ties) with the
FP64 oracle, and whole generations of the state object on this net in lock
step with the oracle, at small sizes and sampled at lambda = 2000, B = 1024."""
import numpy as np
import pytest

from helpers import assert_correct_close, assert_fitness_close, assert_genes_close, to_device_pop
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu

PAPER_DIMS = [196, 256, 128, 64, 10]
PAPER_PRM = dict(xo_op=0, p_e=0.05, p_c=0.75, sigma=0.001, rho=0.5, alpha=1.0)  # Section 4.5


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("h,w,batch", [(28, 28, 37), (6, 10, 5), (2, 2, 1)])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_maxpool_bit_exact(gpu, oracle_mod, h, w, batch, dtype):
    torch = _torch()
    rng = np.random.default_rng(h * w + batch)
    if dtype == "u8":
        x = rng.integers(0, 256, size=(batch, h * w)).astype(np.uint8)
    else:
        x = rng.normal(size=(batch, h * w)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty((batch, (h // 2) * (w // 2)), dtype=xd.dtype, device="cuda")
    gpu.leea_maxpool2x2(batch, h, w, xd, out)
    torch.cuda.synchronize()
    ref = oracle_mod.maxpool2x2(x.astype(np.float64), h, w)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), ref)


def test_maxpool_rejects_odd_sizes(gpu):
    torch = _torch()
    x = torch.zeros((2, 27 * 28), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.LeeaError):
        gpu.leea_maxpool2x2(2, 27, 28, x, x)


MLP_CASES = [
    (PAPER_DIMS, 8, 1024, "u8"),
    (PAPER_DIMS, 5, 37, "f32"),
    ([20, 7, 5, 3], 6, 3, "f32"),
    ([64, 33, 17, 9, 5, 2], 4, 65, "u8"),
    ([100, 50, 40, 32], 3, 32, "f32"),
    ([256, 256, 256, 16], 3, 31, "u8"),
]


@pytest.mark.parametrize("dims,pop,batch,inp", MLP_CASES, ids=lambda v: str(v))
def test_mlp_evaluate_matches_oracle(gpu, oracle_mod, dims, pop, batch, inp):
    torch = _torch()
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    popv = synthetic.random_population(pop, c, seed=c + batch, scale=0.15)
    popv[pop - 1] = popv[0]  # identical individuals: identical results
    rng = np.random.default_rng(batch)
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    pd = to_device_pop(popv, cp)
    f_inh = rng.normal(-2.0, 0.1, size=pop).astype(np.float32)
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    f_adj = torch.empty(pop, dtype=torch.float32, device="cuda")
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    yd = torch.from_numpy(y).cuda()
    if inp == "u8":
        levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
        gpu.leea_evaluate_u8(pop, dims, pd, torch.from_numpy(levels).cuda(), 255.0, yd, batch, 0.3,
                             torch.from_numpy(f_inh).cuda(), f_raw, f_adj, cor)
        x64 = levels.astype(np.float64) / 255.0
    else:
        x = rng.uniform(-1.0, 1.0, size=(batch, dims[0])).astype(np.float32)
        gpu.leea_evaluate(pop, dims, pd, torch.from_numpy(x).cuda(), yd, batch, 0.3,
                          torch.from_numpy(f_inh).cuda(), f_raw, f_adj, cor)
        x64 = x.astype(np.float64)
    torch.cuda.synchronize()
    f_ref, cor_ref, logits = oracle_mod.evaluate(popv.astype(np.float64), dims, x64, y, want_logits=True)
    fr = f_raw.cpu().numpy()
    assert_fitness_close(fr, f_ref)
    assert_correct_close(cor.cpu().numpy(), cor_ref, logits)
    assert_fitness_close(f_adj.cpu().numpy(), oracle_mod.inherit(float(np.float32(0.3)), f_inh, f_ref, first=False),
                         "f_adj")
    assert fr[0].view(np.uint32) == fr[pop - 1].view(np.uint32)


def _eval_u8(gpu, dims, popv, levels, y, path, f_inh=None, alpha=1.0):
    torch = _torch()
    pop, batch = popv.shape[0], levels.shape[0]
    pd = to_device_pop(popv, gpu.leea_padded_params(dims))
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    f_adj = torch.empty(pop, dtype=torch.float32, device="cuda")
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    fi = None if f_inh is None else torch.from_numpy(f_inh).cuda()
    gpu.leea_evaluate_u8(pop, dims, pd, torch.from_numpy(levels).cuda(), 255.0, torch.from_numpy(y).cuda(), batch,
                         alpha, fi, f_raw, f_adj, cor, eval_path=path)
    torch.cuda.synchronize()
    return f_raw.cpu().numpy(), f_adj.cpu().numpy(), cor.cpu().numpy()


TC_CASES = [(PAPER_DIMS, 6, 1024), (PAPER_DIMS, 5, 129), (PAPER_DIMS, 3, 1), (PAPER_DIMS, 160, 100),
            ([64, 48, 32, 16, 4], 7, 200), ([256, 256, 128, 128, 16], 3, 77),
            # layers 2 and 3 wider than 128: three MMAs per 16 inputs, not the merged pair
            ([128, 64, 256, 256, 10], 4, 150),
            # d0 not a multiple of 64 (a partial last level block), a 48-wide merged layer
            ([100, 32, 48, 16, 7], 5, 140),
            # the smallest shape: one 16-input block, 16-wide layers
            ([4, 16, 16, 16, 2], 3, 5)]


@pytest.mark.parametrize("dims,pop,batch", TC_CASES, ids=lambda v: str(v))
def test_mlp_tensor_cores_match_oracle(gpu, oracle_mod, dims, pop, batch):
    # Three hidden layers on tcgen05 (FP16 operand pieces, FP32 accumulation):
    # within the evaluation tolerance of the FP64 oracle, like the FP32 kernel.
    c = gpu.leea_layout_num_params(dims)
    popv = synthetic.random_population(pop, c, seed=c + batch + 1, scale=0.12)
    rng = np.random.default_rng(batch + 5)
    levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    f_inh = rng.normal(-2.0, 0.1, size=pop).astype(np.float32)
    f_tc, a_tc, c_tc = _eval_u8(gpu, dims, popv, levels, y, gpu.EVAL_TENSOR, f_inh, 0.3)
    f_ref, cor_ref, logits = oracle_mod.evaluate(popv.astype(np.float64), dims, levels.astype(np.float64) / 255.0, y,
                                                 want_logits=True)
    assert_fitness_close(f_tc, f_ref, "tensor-core fitness")
    assert_correct_close(c_tc, cor_ref, logits)
    assert_fitness_close(a_tc, oracle_mod.inherit(float(np.float32(0.3)), f_inh, f_ref, first=False), "f_adj")
    f_simt, _, _ = _eval_u8(gpu, dims, popv, levels, y, gpu.EVAL_SIMT)
    assert_fitness_close(f_tc, f_simt.astype(np.float64), "tensor cores vs CUDA cores")


def test_mlp_tensor_cores_fall_back_outside_the_piece_range(gpu, oracle_mod):
    # A weight of 200 in W2, and an individual whose layer-1 activations exceed
    # 128: both are recomputed in FP32; the others stay on the tensor cores.
    dims = PAPER_DIMS
    c = gpu.leea_layout_num_params(dims)
    popv = synthetic.random_population(6, c, seed=3, scale=0.1)
    w2 = 196 * 256 + 256
    popv[1, w2 + 77] = 200.0
    popv[3, :196 * 256] *= 40.0
    rng = np.random.default_rng(2)
    levels = rng.integers(0, 256, size=(300, 196)).astype(np.uint8)
    y = rng.integers(0, 10, size=300).astype(np.int32)
    f_tc, _, c_tc = _eval_u8(gpu, dims, popv, levels, y, gpu.EVAL_AUTO)
    f_ref, cor_ref, logits = oracle_mod.evaluate(popv.astype(np.float64), dims, levels.astype(np.float64) / 255.0, y,
                                                 want_logits=True)
    assert_fitness_close(f_tc, f_ref)
    assert_correct_close(c_tc, cor_ref, logits)


def test_mlp_rejects_tensor_path_and_wide_layers(gpu):
    torch = _torch()
    y = torch.zeros(4, dtype=torch.int32, device="cuda")
    f = torch.empty(2, dtype=torch.float32, device="cuda")
    deep = [64, 32, 32, 32, 16, 4]  # four hidden layers: CUDA cores only
    pdd = torch.zeros((2, gpu.leea_padded_params(deep)), dtype=torch.float32, device="cuda")
    xd = torch.zeros((4, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.LeeaError):
        gpu.leea_evaluate_u8(2, deep, pdd, xd, 255.0, y, 4, 1.0, None, f, eval_path=gpu.EVAL_TENSOR)
    wide = [300, 16, 8, 4]
    pw = torch.zeros((2, gpu.leea_padded_params(wide)), dtype=torch.float32, device="cuda")
    xw = torch.zeros((4, 300), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.LeeaError):
        gpu.leea_evaluate_u8(2, wide, pw, xw, 255.0, y, 4, 1.0, None, f)


def test_paper_net_state_object_limits(gpu):
    # Deeper nets: FP32 populations, breeding and evaluation as separate kernels.
    for prm in (dict(eval_path=gpu.EVAL_FUSED), dict(precision=1)):
        with pytest.raises(gpu.LeeaError) as e:
            gpu.LeeaState(8, PAPER_DIMS, gpu.Params(**prm), 1)
        assert e.value.status == gpu.EINVAL


def _paper_lockstep(gpu, oracle_mod, pop, batch, seed=13, gen0=5, sample=None):
    """One generation of the paper's net from a common state: raw 28x28 levels
    pooled on the GPU, selection bit-exact, children and fitness within
    tolerance."""
    torch = _torch()
    dims = PAPER_DIMS
    c = gpu.leea_layout_num_params(dims)
    st = gpu.LeeaState(pop, dims, gpu.Params(**PAPER_PRM), seed)
    try:
        pop0 = synthetic.random_population(pop, c, seed=seed + 1, scale=0.08)
        f0 = np.random.default_rng(seed).normal(-2.3, 0.05, size=pop).astype(np.float32)
        st.leea_set_population(pop0)
        st.leea_set_fitness(f0)
        st.leea_set_generation(gen0, True)
        x, y = synthetic.make_split(batch, seed=seed + 2)
        raw = synthetic.to_levels(x)                      # [batch, 784] levels of 28x28 images
        raw_d = torch.from_numpy(raw).cuda()
        pooled_d = torch.empty((batch, 196), dtype=torch.uint8, device="cuda")
        gpu.leea_maxpool2x2(batch, 28, 28, raw_d, pooled_d)
        st.leea_generation_u8(pooled_d, torch.from_numpy(y).cuda(), 255.0)
        order, par1, par2, kind, f_inh = st.leea_get_selection()
        kids = st.leea_get_population()
        f_adj, cor = st.leea_fitness(with_correct=True)
        f_raw = st.leea_raw_fitness()
    finally:
        st.close()
    o_prm = oracle_mod.Params(**PAPER_PRM)
    f0d = f0.astype(np.float64)
    o_order = oracle_mod.rank(f0d)
    np.testing.assert_array_equal(order, o_order)
    o1, o2, ok, ofi = oracle_mod.select(o_prm, f0d, o_order, seed, gen0 + 1)
    np.testing.assert_array_equal(par1, o1)
    np.testing.assert_array_equal(par2, o2)
    np.testing.assert_array_equal(kind, ok)
    rows = np.arange(pop) if sample is None else np.asarray(sample)
    for j in rows:
        ref = oracle_mod.breed(o_prm, dims, seed, gen0 + 1, pop0.astype(np.float64), o1, o2, ok, j0=int(j),
                               j1=int(j) + 1)
        assert_genes_close(kids[j][None], ref, o_prm.sigma, what=f"child {j}")
    x64 = oracle_mod.maxpool2x2(raw.astype(np.float64), 28, 28) / 255.0
    f_ref, cor_ref, logits = oracle_mod.evaluate(kids[rows].astype(np.float64), dims, x64, y, want_logits=True)
    assert_fitness_close(f_raw[rows], f_ref)
    assert_correct_close(cor[rows], cor_ref, logits)
    assert_fitness_close(f_adj[rows], f_ref, "f_adj (alpha = 1)")


def test_paper_net_lockstep_small(gpu, oracle_mod):
    _paper_lockstep(gpu, oracle_mod, pop=40, batch=96)


def test_paper_net_lockstep_full_size_sampled(gpu, oracle_mod):
    # lambda = 2000, B = 1024 (Section 4.5): elites, crossover and mutation
    # children, first and last, recomputed one by one.
    _paper_lockstep(gpu, oracle_mod, pop=2000, batch=1024, sample=[0, 1, 99, 100, 101, 1599, 1600, 1601, 1999])


def test_paper_net_learns(gpu):
    # A few hundred generations on a fixed pooled batch improve the best fitness.
    torch = _torch()
    x, y = synthetic.make_split(256, seed=3)
    raw_d = torch.from_numpy(synthetic.to_levels(x)).cuda()
    pooled = torch.empty((256, 196), dtype=torch.uint8, device="cuda")
    gpu.leea_maxpool2x2(256, 28, 28, raw_d, pooled)
    yd = torch.from_numpy(y).cuda()
    st = gpu.LeeaState(200, PAPER_DIMS, gpu.Params(**dict(PAPER_PRM, sigma=0.01)), 4)
    try:
        st.leea_generation_u8(pooled, yd)
        f0 = st.leea_fitness().max()
        for _ in range(150):
            st.leea_generation_u8(pooled, yd)
        assert st.leea_fitness().max() > f0 + 0.1
    finally:
        st.close()


def test_paper_net_state_object_across_batch_sizes(gpu, oracle_mod):
    # One state object, batches growing and shrinking (its tensor-core scratch
    # holds the batch's level tiles and grows with it): each generation's raw
    # fitness matches the oracle's evaluation of that generation's children.
    torch = _torch()
    dims = PAPER_DIMS
    pop = 24
    st = gpu.LeeaState(pop, dims, gpu.Params(**PAPER_PRM), 21)
    try:
        for g, batch in enumerate((50, 300, 129, 1, 1024)):
            rng = np.random.default_rng(100 + g)
            levels = rng.integers(0, 256, size=(batch, 196)).astype(np.uint8)
            y = rng.integers(0, 10, size=batch).astype(np.int32)
            st.leea_generation_u8(torch.from_numpy(levels).cuda(), torch.from_numpy(y).cuda())
            kids = st.leea_get_population()
            f_raw = st.leea_raw_fitness()
            _, cor = st.leea_fitness(with_correct=True)
            f_ref, cor_ref, logits = oracle_mod.evaluate(kids.astype(np.float64), dims,
                                                         levels.astype(np.float64) / 255.0, y, want_logits=True)
            assert_fitness_close(f_raw, f_ref, f"batch {batch}")
            assert_correct_close(cor, cor_ref, logits)
    finally:
        st.close()
