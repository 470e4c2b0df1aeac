"""Parity of the precision form (BF16 / FP8-e4m3 shadows of W1 with FP32
accumulation) with the oracle: the shadows bit-exact against the oracle's
rounding of the same FP32 master, the FP8 scale exponents bit-exact against
the bound rule, the fitness within the FP32 tolerance of the oracle's
evaluation with the quantized W1, and within 2e-2 of the FP64 evaluation of
the unquantized master."""
import numpy as np
import pytest
from scipy import stats

from helpers import (assert_correct_close, assert_fitness_close, decode_bf16, decode_e4m3, to_device_pop,
                     untile_shadow)
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu

NORMAL_BOUND = np.float32(5.77)  # bound on |z| of the library's Box-Muller normals


def _torch():
    import torch
    return torch


def _n_w1(dims):
    return int(dims[0]) * int(dims[1])


def _shadow_values(gpu, raw, dims, precision, scale_exp):
    """Decoded shadow values (float64[pop, n_w1], W1 row-major) of tiled shadows."""
    k, h = int(dims[0]), int(dims[1])
    elem = 2 if precision == 1 else 1
    rows = untile_shadow(raw, k, h, elem).reshape(raw.shape[0], h * k * elem)
    if precision == 1:
        return decode_bf16(rows.view(np.uint16))
    return decode_e4m3(rows) * np.ldexp(1.0, np.asarray(scale_exp, dtype=np.int64))[:, None]


def _padding_is_zero(raw, dims, precision):
    k, h = int(dims[0]), int(dims[1])
    elem = 2 if precision == 1 else 1
    k_full = (k * elem + 127) // 128 * 128 // elem
    return not untile_shadow(raw, k_full, h, elem)[:, :, k * elem:].any()


def _make_shadow(gpu, popv, dims, precision):
    torch = _torch()
    pop = popv.shape[0]
    cp = gpu.leea_padded_params(dims)
    stride = gpu.leea_shadow_stride(dims, precision)
    pd = to_device_pop(popv, cp)
    sh = torch.full((pop, stride), 0xA5, dtype=torch.uint8, device="cuda")  # padding must be overwritten
    se = torch.full((pop,), -999, dtype=torch.int32, device="cuda")
    am = torch.full((pop,), -1.0, dtype=torch.float32, device="cuda")
    gpu.leea_make_shadow(pop, dims, precision, pd, sh, se, am)
    torch.cuda.synchronize()
    return pd, sh, se, am


def _oracle_scale_exp(oracle_mod, amax):
    return np.array([oracle_mod.fp8_scale_exp(float(a)) for a in amax], dtype=np.int32)


def _special_population(dims, pop=6, seed=11):
    """Rows of very different magnitude, an all-zero W1, and values on rounding ties."""
    c = int(dims[0]) * int(dims[1]) + int(dims[1]) + int(dims[2]) * int(dims[1]) + int(dims[2])
    popv = synthetic.random_population(pop, c, seed=seed, scale=1.0)
    scales = [0.05, 0.003, 1.0, 37.0, 0.2, 0.0][:pop]
    n = _n_w1(dims)
    for p, s in enumerate(scales):
        popv[p, :n] *= np.float32(s)
    special = np.array([0.0, -0.0, 1e-30, -1e-30, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 2 ** -9, 3 * 2 ** -11,
                        2 ** -10, -0.0713, 0.1, 240.0 / 256, 1.75, 1.875, 2.0], dtype=np.float32)
    popv[2, :special.size] = special
    return popv


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("dims", [[784, 112, 10], [64, 16, 4]])
def test_make_shadow_bit_exact(gpu, oracle_mod, dims, precision):
    popv = _special_population(dims)
    n = _n_w1(dims)
    _, sh, se, am = _make_shadow(gpu, popv, dims, precision)
    amax_ref = np.abs(popv[:, :n]).max(axis=1)
    np.testing.assert_array_equal(am.cpu().numpy(), amax_ref)
    se_ref = _oracle_scale_exp(oracle_mod, amax_ref.astype(np.float64))
    if precision == 2:
        np.testing.assert_array_equal(se.cpu().numpy(), se_ref)
    got = _shadow_values(gpu, sh.cpu().numpy(), dims, precision, se_ref)
    ref = oracle_mod.quantize_w1(popv.astype(np.float64), dims, precision, se_ref)[:, :n]
    np.testing.assert_array_equal(got, ref)
    assert _padding_is_zero(sh.cpu().numpy(), dims, precision)
    if precision == 2:  # the scale keeps every value inside the FP8 range: no saturation
        assert (np.abs(got) <= 448.0 * np.ldexp(1.0, se_ref.astype(np.int64))[:, None]).all()


# (dims, pop, batch): ragged populations, one and several 128-sample tiles, ragged last tile
SHADOW_CASES = [
    ([784, 112, 10], 37, 100),
    ([784, 112, 10], 9, 256),
    ([784, 112, 10], 5, 300),
    ([784, 32, 10], 200, 129),
    ([784, 32, 10], 3, 1),
    ([64, 16, 4], 160, 128),
    ([128, 256, 10], 7, 77),
    ([96, 48, 16], 11, 513),
    ([784, 256, 10], 13, 100),   # hidden units in 3 chunks (96, 96, 64)
    ([784, 160, 10], 6, 200),    # 2 chunks of 80, 2 sample tiles
]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("dims,pop,batch", SHADOW_CASES)
def test_evaluate_shadow_matches_oracle(gpu, oracle_mod, dims, pop, batch, precision):
    torch = _torch()
    c = gpu.leea_layout_num_params(dims)
    popv = synthetic.random_population(pop, c, seed=c + batch, scale=0.15)
    rng = np.random.default_rng(batch + 1000 * precision)
    levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    f_inh = rng.normal(-2.3, 0.1, size=pop).astype(np.float32)
    pd, sh, se, _ = _make_shadow(gpu, popv, dims, precision)
    xd, yd = torch.from_numpy(levels).cuda(), torch.from_numpy(y).cuda()
    f_raw = torch.empty(pop, dtype=torch.float32, device="cuda")
    f_adj = torch.empty_like(f_raw)
    cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    nbytes = gpu.leea_shadow_scratch_bytes(pop, batch)
    assert nbytes == (0 if batch <= 128 else 8 * ((batch + 127) // 128) * pop)
    scratch = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device="cuda") if nbytes else None
    gpu.leea_evaluate_shadow_u8(pop, dims, pd, precision, sh, se, xd, 255.0, yd, batch, 0.3,
                                torch.from_numpy(f_inh).cuda(), f_raw, f_adj, cor, scratch)
    assert gpu.leea_device_status() == 0
    amax = np.abs(popv[:, :_n_w1(dims)]).max(axis=1).astype(np.float64)
    se_ref = _oracle_scale_exp(oracle_mod, amax)
    x64 = levels.astype(np.float64) / 255.0
    q = oracle_mod.quantize_w1(popv.astype(np.float64), dims, precision, se_ref)
    f_ref, cor_ref, logits = oracle_mod.evaluate(q, dims, x64, y, want_logits=True)
    got = f_raw.cpu().numpy()
    assert_fitness_close(got, f_ref, "shadow fitness")
    assert_correct_close(cor.cpu().numpy(), cor_ref, logits)
    adj_ref = oracle_mod.inherit(float(np.float32(0.3)), f_inh.astype(np.float64), f_ref, first=False)
    assert_fitness_close(f_adj.cpu().numpy(), adj_ref, "f_adj")
    # Against the FP64 evaluation of the unquantized master: within 2e-2 relative.
    f64, _ = oracle_mod.evaluate(popv.astype(np.float64), dims, x64, y)
    rel = np.abs(got - f64) / np.abs(f64)
    assert rel.max() <= 2e-2, rel.max()


def test_evaluate_shadow_argument_errors(gpu):
    torch = _torch()
    dims = [784, 32, 10]
    pop, batch = 4, 200
    popv = synthetic.random_population(pop, gpu.leea_layout_num_params(dims), seed=1)
    pd, sh, se, _ = _make_shadow(gpu, popv, dims, 1)
    x = torch.zeros((batch, 784), dtype=torch.uint8, device="cuda")
    y = torch.zeros(batch, dtype=torch.int32, device="cuda")
    f = torch.empty(pop, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.LeeaError, match="scratch"):  # two tiles need scratch
        gpu.leea_evaluate_shadow_u8(pop, dims, pd, 1, sh, se, x, 255.0, y, batch, 1.0, None, f)
    small = torch.empty(3, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.LeeaError, match="scratch"):
        gpu.leea_evaluate_shadow_u8(pop, dims, pd, 1, sh, se, x, 255.0, y, batch, 1.0, None, f, scratch_dev=small)
    with pytest.raises(gpu.LeeaError):  # h above 256
        gpu.leea_make_shadow(pop, [784, 272, 10], 1, pd, sh, se, f)
    with pytest.raises(gpu.LeeaError):  # d_0 not a multiple of 16
        gpu.leea_make_shadow(pop, [780, 32, 10], 1, pd, sh, se, f)
    with pytest.raises(gpu.LeeaError):
        gpu.leea_evaluate_shadow_u8(pop, dims, pd, 3, sh, se, x, 255.0, y, 100, 1.0, None, f)
    # 13 blocks of 64 BF16 inputs, 7 blocks of 128 FP8 inputs, 32 rows of 128 bytes each
    assert gpu.leea_shadow_stride(dims, 1) == 13 * 32 * 128 and gpu.leea_shadow_stride(dims, 2) == 7 * 32 * 128
    assert gpu.leea_shadow_stride([96, 16, 2], 2) == 16 * 128
    assert gpu.leea_shadow_stride(dims, 0) == -1


def _bound_exp(oracle_mod, kind, par1, par2, amax_par, sigma):
    """Children's FP8 exponents from their parents' exact maxima (FP32 arithmetic)."""
    out = np.empty(kind.size, dtype=np.int32)
    s32 = np.float32(sigma)
    for j in range(kind.size):
        b = np.float32(amax_par[par1[j]])
        if kind[j] == 1:
            b = max(b, np.float32(amax_par[par2[j]]))
        elif kind[j] == 2:
            b = np.float32(np.float64(s32) * np.float64(NORMAL_BOUND) + np.float64(b))
        out[j] = oracle_mod.fp8_scale_exp(float(b))
    return out


def _state_generation(gpu, oracle_mod, precision, dims, pop, batch, sigma, gens=2, sample=None):
    torch = _torch()
    prm = gpu.Params(sigma=sigma, mut_rate=0.1, n_elite=2, p_c=0.5, precision=precision, alpha=0.5)
    c = gpu.leea_layout_num_params(dims)
    n = _n_w1(dims)
    st = gpu.LeeaState(pop, dims, prm, seed=77)
    try:
        popv = synthetic.random_population(pop, c, seed=5, scale=0.1)
        popv[3, :n] *= np.float32(10.0)  # one individual of another magnitude
        st.leea_set_population(popv)
        rng = np.random.default_rng(3)
        levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
        y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
        xd, yd = torch.from_numpy(levels).cuda(), torch.from_numpy(y).cuda()
        st.leea_generation_u8(xd, yd)
        x64 = levels.astype(np.float64) / 255.0
        parents = popv
        for _ in range(gens):
            _, _, am_par = st.leea_get_shadow(precision)
            np.testing.assert_array_equal(am_par, np.abs(parents[:, :n]).max(axis=1))
            st.leea_generation_u8(xd, yd)
            _, par1, par2, kind, _ = st.leea_get_selection()
            kids = st.leea_get_population()
            sh, se, am = st.leea_get_shadow(precision)
            np.testing.assert_array_equal(am, np.abs(kids[:, :n]).max(axis=1))
            assert _padding_is_zero(sh[:8], dims, precision)
            se_ref = _bound_exp(oracle_mod, kind, par1, par2, am_par, sigma)
            if precision == 2:
                np.testing.assert_array_equal(se, se_ref)
            rows = np.arange(pop) if sample is None else np.asarray(sample)
            got = _shadow_values(gpu, sh[rows], dims, precision, se_ref[rows])
            q = oracle_mod.quantize_w1(kids[rows].astype(np.float64), dims, precision, se_ref[rows])
            np.testing.assert_array_equal(got, q[:, :n])
            f_raw = st.leea_raw_fitness()
            f_ref, _ = oracle_mod.evaluate(q, dims, x64, y)
            assert_fitness_close(f_raw[rows], f_ref, "state shadow fitness")
            parents = kids
        return st.leea_raw_fitness()
    finally:
        st.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_state_breeds_shadows_and_scales(gpu, oracle_mod, precision):
    # sigma large enough that the mutation term of the bound decides some exponents.
    _state_generation(gpu, oracle_mod, precision, [784, 32, 10], 64, 100, sigma=0.05, gens=3)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("dims,pop,batch", [([784, 160, 10], 40, 200), ([784, 256, 10], 19, 100),
                                            ([96, 48, 16], 33, 130), ([64, 160, 4], 20, 50)])
def test_state_wide_hidden_generations(gpu, oracle_mod, precision, dims, pop, batch):
    # h above 128: the state object evaluates one individual per MMA of N = h
    # (one pass over K); h = 48 with 16 outputs: two individuals per MMA and
    # the layer-2 code for outputs other than 10.  Fitness against the
    # oracle's evaluation of the same shadows, generation by generation.
    _state_generation(gpu, oracle_mod, precision, dims, pop, batch, sigma=0.02, gens=2)


@pytest.mark.parametrize("precision", [1, 2])
def test_state_full_size_sampled(gpu, oracle_mod, precision):
    # 4096 MLPs 784-112-10 on batches of 256: every shadow exponent checked, 10 individuals in full.
    sample = [0, 1, 2, 3, 1000, 2047, 2048, 3001, 4094, 4095]
    _state_generation(gpu, oracle_mod, precision, [784, 112, 10], 4096, 256, sigma=0.005, gens=1, sample=sample)


def test_precision_state_errors(gpu):
    torch = _torch()
    with pytest.raises(gpu.LeeaError):  # d_0 not a multiple of 16
        gpu.LeeaState(8, [780, 128, 10], gpu.Params(precision=1), seed=1)
    st = gpu.LeeaState(8, [784, 32, 10], gpu.Params(precision=2), seed=1)
    try:
        x = torch.zeros((16, 784), dtype=torch.float32, device="cuda")
        y = torch.zeros(16, dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.LeeaError, match="8-bit"):
            st.leea_generation(x, y)
    finally:
        st.close()
    st = gpu.LeeaState(8, [784, 32, 10], gpu.Params(precision=1, eval_path=gpu.EVAL_SIMT), seed=1)
    try:
        x = torch.zeros((16, 784), dtype=torch.uint8, device="cuda")
        y = torch.zeros(16, dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.LeeaError, match="tensor cores"):
            st.leea_generation_u8(x, y)
    finally:
        st.close()
    st = gpu.LeeaState(8, [784, 32, 10], gpu.Params(), seed=1)
    try:
        with pytest.raises(gpu.LeeaError):
            st.leea_get_shadow(1)
    finally:
        st.close()
    pd = torch.zeros((4, 32), dtype=torch.float32, device="cuda")
    i = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu.LeeaError, match="precision"):
        gpu.leea_breed(4, [2, 2, 2], gpu.Params(precision=1), 1, 1, pd, i, i, i, pd.clone())


@pytest.mark.parametrize("precision", [1, 2])
def test_rank_agreement_reported(gpu, oracle_mod, precision, capsys):
    # Reported, not pinned: how the shadow fitness ranks a population against the
    # FP64 evaluation of the master (Spearman and top-10% overlap).
    torch = _torch()
    dims, pop, batch = [784, 112, 10], 128, 256
    c = gpu.leea_layout_num_params(dims)
    popv = synthetic.random_population(pop, c, seed=21, scale=0.05)
    x, y = synthetic.make_split(batch, seed=4)
    levels = synthetic.to_levels(x)
    pd, sh, se, _ = _make_shadow(gpu, popv, dims, precision)
    f = torch.empty(pop, dtype=torch.float32, device="cuda")
    scratch = torch.empty(gpu.leea_shadow_scratch_bytes(pop, batch) // 4, dtype=torch.float32, device="cuda")
    gpu.leea_evaluate_shadow_u8(pop, dims, pd, precision, sh, se, torch.from_numpy(levels).cuda(), 255.0,
                                torch.from_numpy(y).cuda(), batch, 1.0, None, f, scratch_dev=scratch)
    got = f.cpu().numpy()
    f64, _ = oracle_mod.evaluate(popv.astype(np.float64), dims, x.astype(np.float64), y)
    rho = stats.spearmanr(got, f64).statistic
    k = pop // 10
    top = len(set(np.argsort(-got)[:k]) & set(np.argsort(-f64)[:k])) / k
    rel = np.abs(got - f64) / np.abs(f64)
    with capsys.disabled():
        print(f"\n[precision {precision}] spearman {rho:.4f} top-10% overlap {top:.2f} "
              f"max rel loss error {rel.max():.2e} (P={pop}, B={batch})")
    assert rel.max() <= 2e-2
