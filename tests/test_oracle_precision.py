"""Pins of the oracle's precision-form rounding (BF16 and FP8-e4m3 with
saturation) and of the evaluation with quantized W1."""
import numpy as np
import pytest
import torch

from paper_1806_09819_gb300 import synthetic


def _vals():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(0, 1, 2000), rng.normal(0, 0.05, 2000), rng.uniform(-400, 400, 500),
                        [0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 2 ** -9, 2 ** -10, 3 * 2 ** -11, 447.0, 448.0,
                         -0.0713, 1e-30, 2 ** -126, 2 ** -130]])
    return v.astype(np.float32).astype(np.float64)  # values exactly representable in FP32


def test_bf16_rounding_matches_library(oracle_mod):
    v = _vals()
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle_mod.round_bf16(x) for x in v])
    np.testing.assert_array_equal(got, ref)


def test_e4m3_rounding_matches_library_in_range(oracle_mod):
    v = _vals()
    v = v[np.abs(v) < 464.0]  # the library conversion does not saturate; stay in range
    ref = torch.tensor(v, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([oracle_mod.round_e4m3(x) for x in v])
    np.testing.assert_array_equal(got, ref)


def test_e4m3_saturates_to_finite(oracle_mod):
    for x, want in [(464.0, 448.0), (470.0, 448.0), (1e6, 448.0), (-1e6, -448.0), (float("inf"), 448.0),
                    (2 ** -10, 0.0), (3 * 2 ** -11, 2 ** -9), (240.0, 240.0), (15.0, 15.0)]:
        assert oracle_mod.round_e4m3(x) == want, x
    assert np.isnan(oracle_mod.round_e4m3(float("nan")))
    # integers 0..16 and 16*a (a <= 15) are exact: the two-piece encoding of 8-bit levels
    for k in range(0, 17):
        assert oracle_mod.round_e4m3(float(k)) == k
    for a in range(0, 16):
        assert oracle_mod.round_e4m3(16.0 * a) == 16.0 * a


def test_fp8_scale_exponent(oracle_mod):
    assert oracle_mod.fp8_scale_exp(0.0) == 0
    for bound in [1e-3, 0.17, 0.5, 1.0, 448.0, 449.0, 3.5]:
        e = oracle_mod.fp8_scale_exp(bound)
        assert 448.0 * 2.0 ** e >= bound > 448.0 * 2.0 ** (e - 1)


@pytest.mark.parametrize("precision", [1, 2])
def test_shadow_evaluation(oracle_mod, precision):
    dims = [784, 32, 10]
    c = oracle_mod.num_params(dims)
    popv = synthetic.random_population(5, c, seed=3, scale=0.05).astype(np.float64)
    x, y = synthetic.make_split(40, seed=2)
    amax = np.abs(popv[:, :784 * 32]).max(axis=1)
    se = np.array([oracle_mod.fp8_scale_exp(a) for a in amax], dtype=np.int32)
    f, _ = oracle_mod.evaluate_shadow(popv, dims, precision, se, x, y)
    # Same as evaluating the explicitly quantized population in full precision.
    q = popv.copy()
    for p in range(5):
        for i in range(784 * 32):
            if precision == 1:
                q[p, i] = oracle_mod.round_bf16(popv[p, i])
            else:
                s = 2.0 ** se[p]
                q[p, i] = oracle_mod.round_e4m3(popv[p, i] / s) * s
    f_ref, _ = oracle_mod.evaluate(q, dims, x, y)
    np.testing.assert_array_equal(f, f_ref)
    np.testing.assert_array_equal(oracle_mod.quantize_w1(popv, dims, precision, se), q)
    # The shadow's loss error against the FP64 master is small but not zero.
    f64, _ = oracle_mod.evaluate(popv, dims, x, y)
    err = np.abs(f - f64) / np.abs(f64)
    assert err.max() < (2e-3 if precision == 1 else 2e-2)
    assert err.max() > 0


def test_precision_zero_is_plain_evaluation(oracle_mod):
    dims = [784, 16, 10]
    c = oracle_mod.num_params(dims)
    popv = synthetic.random_population(3, c, seed=4).astype(np.float64)
    x, y = synthetic.make_split(8, seed=5)
    f0, _ = oracle_mod.evaluate_shadow(popv, dims, 0, None, x, y)
    np.testing.assert_array_equal(f0, oracle_mod.evaluate(popv, dims, x, y)[0])


def test_test_decoders_match_library():
    # The tests' BF16 and FP8 decoders against PyTorch's CPU conversions.
    from helpers import decode_bf16, decode_e4m3
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = decode_e4m3(codes)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(got[ok], ref[ok])
    bits = np.random.default_rng(1).integers(0, 2 ** 16, size=5000).astype(np.uint16)
    bits = bits[(bits & 0x7F80) != 0x7F80]  # finite patterns
    ref = torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(decode_bf16(bits), ref)
