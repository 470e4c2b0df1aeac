"""The fused breed + evaluate kernel (Section 3.2 and Eq. 1 in one pass), through
the C ABI: its children must be bit-identical to the breeding kernel's on the
same selection, and its fitness must match the FP64 oracle's evaluation of
those children within the evaluation tolerance; both against the oracle's own
breed as well.  Also the state object's fused path, the FP32 fallback for
weights outside the FP16 piece range, invalid parents, and the shape limits."""
import numpy as np
import pytest

from helpers import assert_correct_close, assert_fitness_close, assert_genes_close, to_device_pop
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _i32(a):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _fused_vs_separate(gpu, oracle_mod, dims, pop, batch, prm, seed=7, gen=9, scale=0.2, plant=None):
    torch = _torch()
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    parents = synthetic.random_population(pop, c, seed=pop + c + batch, scale=scale)
    if plant is not None:
        plant(parents)
    rng = np.random.default_rng(seed)
    f = rng.normal(-2.0, 0.2, size=pop).astype(np.float32)
    o_prm = oracle_mod.Params(**prm)
    order = oracle_mod.rank(f.astype(np.float64))
    p1, p2, kind, f_inh = oracle_mod.select(o_prm, f.astype(np.float64), order, seed, gen)
    levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    par_d = to_device_pop(parents, cp)
    sep_d = torch.full_like(par_d, 3.0)
    fus_d = torch.full_like(par_d, 5.0)
    xd, yd = torch.from_numpy(levels).cuda(), _i32(y)
    fi = torch.from_numpy(f_inh.astype(np.float32)).cuda()
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    f_adj = torch.empty(pop, dtype=torch.float32, device="cuda")
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    g_prm = gpu.Params(**prm)
    gpu.leea_breed(pop, dims, g_prm, seed, gen, par_d, _i32(p1), _i32(p2), _i32(kind), sep_d)
    gpu.leea_breed_evaluate_u8(pop, dims, g_prm, seed, gen, par_d, _i32(p1), _i32(p2), _i32(kind), fus_d, xd, 255.0,
                               yd, batch, 0.25, fi, f_raw, f_adj, cor)
    torch.cuda.synchronize()
    fused = fus_d.cpu().numpy()
    # Children: bit-identical to the breeding kernel's, padding zero.
    np.testing.assert_array_equal(fused.view(np.uint32), sep_d.cpu().numpy().view(np.uint32))
    assert (fused[:, c:] == 0).all()
    # ... and within the breed tolerance of the oracle's children.
    ref = oracle_mod.breed(o_prm, dims, seed, gen, parents.astype(np.float64), p1, p2, kind)
    assert_genes_close(fused[:, :c], ref, o_prm.sigma)
    # Fitness of the children as made, against the FP64 oracle.
    x64 = levels.astype(np.float64) / 255.0
    f_ref, cor_ref, logits = oracle_mod.evaluate(fused[:, :c].astype(np.float64), dims, x64, y, want_logits=True)
    assert_fitness_close(f_raw.cpu().numpy(), f_ref)
    assert_correct_close(cor.cpu().numpy(), cor_ref, logits)
    adj = oracle_mod.inherit(0.25, f_inh, f_ref, first=False)
    assert_fitness_close(f_adj.cpu().numpy(), adj, "f_adj")
    # The same arithmetic in the same order as the separate tensor-core
    # evaluation of the same children: bit-identical results.
    s_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    s_adj = torch.empty(pop, dtype=torch.float32, device="cuda")
    s_cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_evaluate_u8(pop, dims, sep_d, xd, 255.0, yd, batch, 0.25, fi, s_raw, s_adj, s_cor,
                         eval_path=gpu.EVAL_TENSOR)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(f_raw.cpu().numpy().view(np.uint32), s_raw.cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(f_adj.cpu().numpy().view(np.uint32), s_adj.cpu().numpy().view(np.uint32))
    np.testing.assert_array_equal(cor.cpu().numpy(), s_cor.cpu().numpy())
    return f_raw.cpu().numpy()


FUSED_CASES = [
    dict(dims=[784, 112, 10], pop=24, batch=100, prm=dict(n_elite=1, sigma=0.005, mut_rate=0.1)),
    dict(dims=[784, 112, 10], pop=200, batch=100, prm=dict(n_elite=3, p_c=0.5, sigma=0.01)),
    dict(dims=[784, 32, 10], pop=32, batch=16, prm=dict(sel_op=1, sigma=0.01)),
    dict(dims=[784, 96, 10], pop=40, batch=128, prm=dict(xo_op=1, p_c=0.75, sigma=0.02)),
    dict(dims=[784, 16, 10], pop=17, batch=1, prm=dict(xo_gene_p=0.2, mut_rate=0.5, sigma=0.1)),
    dict(dims=[64, 48, 3], pop=9, batch=57, prm=dict(sigma=0.3, p_e=0.2)),
    dict(dims=[784, 112, 16], pop=5, batch=100, prm=dict(p_c=0.0, n_elite=0, sigma=0.05)),
]


@pytest.mark.parametrize("case", FUSED_CASES, ids=lambda c: f"{c['dims']}-{c['pop']}-B{c['batch']}")
def test_fused_matches_separate_and_oracle(gpu, oracle_mod, case):
    _fused_vs_separate(gpu, oracle_mod, case["dims"], case["pop"], case["batch"], case["prm"])


def test_fused_full_population_size(gpu, oracle_mod):
    # The benchmark's shape (1000 children of 784-112-10, B = 100): more
    # children than SMs, every CTA walks several; all children compared.
    _fused_vs_separate(gpu, oracle_mod, [784, 112, 10], 1000, 100,
                       dict(n_elite=1, p_c=0.5, sigma=0.005, mut_rate=0.1), seed=3, gen=77)


def test_fused_weights_outside_the_piece_range(gpu, oracle_mod):
    # A parent with |w| >= 128 in W1: its elite child takes the FP32 FFMA fallback.
    def plant(p):
        p[0, 5] = 300.0
        p[0, 784 * 7 + 3] = -1000.0

    _fused_vs_separate(gpu, oracle_mod, [784, 32, 10], 12, 64, dict(n_elite=12, p_c=0.0), scale=0.05, plant=plant)


def test_fused_invalid_parent_gives_nan(gpu):
    torch = _torch()
    dims, pop, batch = [784, 32, 10], 4, 8
    cp = gpu.leea_padded_params(dims)
    par_d = torch.zeros((pop, cp), dtype=torch.float32, device="cuda")
    kid_d = torch.zeros_like(par_d)
    p1 = _i32([0, 1, 7, 2])  # child 2 names a parent outside the population
    kind = _i32([0, 2, 2, 2])
    x = torch.zeros((batch, 784), dtype=torch.uint8, device="cuda")
    y = torch.zeros(batch, dtype=torch.int32, device="cuda")
    f = torch.empty(pop, dtype=torch.float32, device="cuda")
    gpu.leea_breed_evaluate_u8(pop, dims, gpu.Params(sigma=0.0), 1, 1, par_d, p1, p1, kind, kid_d, x, 255.0, y, batch,
                               1.0, None, f)
    torch.cuda.synchronize()
    kids = kid_d.cpu().numpy()
    c = gpu.leea_layout_num_params(dims)
    assert np.isnan(kids[2, :c]).all() and (kids[2, c:] == 0).all()
    fv = f.cpu().numpy()
    assert np.isnan(fv[2]) and np.isfinite(fv[[0, 1, 3]]).all()
    np.testing.assert_allclose(fv[[0, 1, 3]], -np.log(10.0), rtol=1e-6)  # zero nets


def test_fused_shape_limits(gpu):
    torch = _torch()
    x = torch.zeros((8, 784), dtype=torch.uint8, device="cuda")
    y = torch.zeros(8, dtype=torch.int32, device="cuda")
    f = torch.empty(4, dtype=torch.float32, device="cuda")
    idx = _i32([0, 0, 0, 0])
    for dims, batch in (([784, 144, 10], 8), ([784, 24, 10], 8), ([780, 32, 10], 8), ([784, 32, 10], 129)):
        cp = gpu.leea_padded_params(dims)
        a = torch.zeros((4, cp), dtype=torch.float32, device="cuda")
        b = torch.zeros_like(a)
        xb = torch.zeros((batch, dims[0]), dtype=torch.uint8, device="cuda")
        yb = torch.zeros(batch, dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.LeeaError) as e:
            gpu.leea_breed_evaluate_u8(4, dims, gpu.Params(), 1, 1, a, idx, idx, idx, b, xb, 255.0, yb, batch, 1.0,
                                       None, f)
        assert e.value.status == gpu.EINVAL
    cp = gpu.leea_padded_params([784, 32, 10])
    a = torch.zeros((4, cp), dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.LeeaError):  # parents and children overlap
        gpu.leea_breed_evaluate_u8(4, [784, 32, 10], gpu.Params(), 1, 1, a, idx, idx, idx, a, x, 255.0, y, 8, 1.0,
                                   None, f)
    with pytest.raises(gpu.LeeaError):  # self-adaptive sigma lives in the state object
        gpu.leea_breed_evaluate_u8(4, [784, 32, 10], gpu.Params(sigma_ctl=gpu.SIGMA_SELF), 1, 1, a, idx, idx, idx,
                                   torch.zeros_like(a), x, 255.0, y, 8, 1.0, None, f)


def test_state_object_fused_path(gpu, oracle_mod):
    # FUSED: one launch per breeding generation for breed + evaluate, none for
    # stage 2; AUTO and TENSOR: two.  Population and fitness are identical.
    torch = _torch()
    dims, pop, batch = [784, 112, 10], 300, 100
    x, y = synthetic.make_split(batch, seed=2)
    xd, yd = torch.from_numpy(synthetic.to_levels(x)).cuda(), _i32(y)
    runs = {}
    for path in (gpu.EVAL_AUTO, gpu.EVAL_FUSED, gpu.EVAL_TENSOR):
        st = gpu.LeeaState(pop, dims, gpu.Params(n_elite=2, sigma=0.01, mut_rate=0.1, alpha=0.5, eval_path=path), 5)
        try:
            st.leea_generation_u8(xd, yd)
            st.leea_profile_enable(True)
            for _ in range(3):
                st.leea_generation_u8(xd, yd)
            prof = st.leea_profile_read()
            runs[path] = (st.leea_get_population(), st.leea_fitness(), prof)
        finally:
            st.close()
    assert runs[gpu.EVAL_FUSED][2]["breed"][1] == 3 and runs[gpu.EVAL_FUSED][2]["evaluate"][1] == 0
    for path in (gpu.EVAL_AUTO, gpu.EVAL_TENSOR):
        assert runs[path][2]["breed"][1] == 3 and runs[path][2]["evaluate"][1] == 3
    # Same children, same evaluation arithmetic: the three runs are identical.
    for path in (gpu.EVAL_AUTO, gpu.EVAL_FUSED):
        np.testing.assert_array_equal(runs[path][0], runs[gpu.EVAL_TENSOR][0])
        np.testing.assert_array_equal(runs[path][1], runs[gpu.EVAL_TENSOR][1])


def test_state_object_fused_errors(gpu):
    torch = _torch()
    with pytest.raises(gpu.LeeaError):  # the fused path evaluates FP32 populations
        gpu.LeeaState(8, [784, 32, 10], gpu.Params(precision=1, eval_path=gpu.EVAL_FUSED), 1)
    st = gpu.LeeaState(8, [784, 24, 10], gpu.Params(eval_path=gpu.EVAL_FUSED), 1)
    try:
        x = torch.zeros((8, 784), dtype=torch.uint8, device="cuda")
        y = torch.zeros(8, dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.LeeaError) as e:  # h % 16 != 0
            st.leea_generation_u8(x, y)
        assert e.value.status == gpu.EINVAL
    finally:
        st.close()
    st = gpu.LeeaState(8, [784, 32, 10], gpu.Params(eval_path=gpu.EVAL_FUSED), 1)
    try:
        xf = torch.zeros((8, 784), dtype=torch.float32, device="cuda")
        y = torch.zeros(8, dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.LeeaError):  # 8-bit inputs only
            st.leea_generation(xf, y)
    finally:
        st.close()
