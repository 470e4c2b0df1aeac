"""Helpers shared by the GPU parity tests: moving populations between the
oracle's unpadded float64 layout and the library's padded device layout, and
the comparison rules (tolerances) the parity tests use."""
from __future__ import annotations

import numpy as np

# Fitness: |f_gpu - f_oracle| <= 1e-5 * max(|f|, 1e-2)  (FP32 vs FP64 oracle).
FIT_RTOL = 1e-5
FIT_FLOOR = 1e-2


def to_device_pop(popv, c_pad: int):
    import torch
    popv = np.asarray(popv, dtype=np.float32)
    P, c = popv.shape
    t = torch.zeros((P, c_pad), dtype=torch.float32)
    t[:, :c] = torch.from_numpy(popv)
    return t.cuda()


def from_device_pop(t, c: int) -> np.ndarray:
    return t[:, :c].cpu().numpy()


def assert_fitness_close(f_gpu, f_ref, what="fitness"):
    f_gpu = np.asarray(f_gpu, dtype=np.float64)
    f_ref = np.asarray(f_ref, dtype=np.float64)
    assert f_gpu.shape == f_ref.shape
    nan_g, nan_r = np.isnan(f_gpu), np.isnan(f_ref)
    np.testing.assert_array_equal(nan_g, nan_r, err_msg=f"{what}: NaN pattern")
    ok = ~nan_r
    err = np.abs(f_gpu[ok] - f_ref[ok])
    tol = FIT_RTOL * np.maximum(np.abs(f_ref[ok]), FIT_FLOOR)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, f"{what}: {bad.size} outside tolerance, worst {(err / tol).max():.3g}x tol"


def ambiguous_samples(logits: np.ndarray, rel: float = 1e-4) -> np.ndarray:
    """Per individual, how many samples have a top-2 logit gap small enough
    that FP32 and FP64 may disagree on the argmax."""
    s = np.sort(logits, axis=-1)
    gap = s[..., -1] - s[..., -2]
    scale = np.maximum(np.abs(s[..., -1]), 1.0)
    return (gap <= rel * scale).sum(axis=-1)


def assert_correct_close(cor_gpu, cor_ref, logits_ref):
    amb = ambiguous_samples(logits_ref)
    diff = np.abs(np.asarray(cor_gpu, dtype=np.int64) - np.asarray(cor_ref, dtype=np.int64))
    assert (diff <= amb).all(), f"correct counts differ beyond near-ties: {diff[diff > amb]}"


def assert_genes_close(gpu, ref, sigma: float, what="genes"):
    """Children: FP32 result of the FP64 oracle's arithmetic: one FP32 rounding
    plus 1e-6 relative on the mutation step (Box-Muller in FP32)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    tol = 2.0 ** -23 * np.abs(ref) + 1e-6 * sigma * 8.0 + 1e-30
    bad = np.abs(gpu - ref) > tol
    assert not bad.any(), f"{what}: {bad.sum()} genes outside tolerance, first {np.argwhere(bad)[:3].tolist()}"


def decode_bf16(bits) -> np.ndarray:
    """Values (float64) of BF16 bit patterns (uint16): the upper half of an FP32."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def _e4m3_table() -> np.ndarray:
    """Value of each of the 256 FP8-e4m3 codes (OCP 8-bit floating point: 1 sign,
    4 exponent bits with bias 7, 3 mantissa bits; exponent 0 subnormal; S.1111.111
    NaN; no infinities)."""
    t = np.empty(256, dtype=np.float64)
    for b in range(256):
        s, e, m = b >> 7, (b >> 3) & 15, b & 7
        if e == 15 and m == 7:
            v = np.nan
        elif e == 0:
            v = m * 2.0 ** -9
        else:
            v = (1.0 + m / 8.0) * 2.0 ** (e - 7)
        t[b] = -v if s else v
    return t


E4M3_TABLE = _e4m3_table()


def decode_e4m3(codes) -> np.ndarray:
    return E4M3_TABLE[np.asarray(codes, dtype=np.uint8)]


def untile_shadow(raw, k: int, h: int, elem: int) -> np.ndarray:
    """Row-major bytes (uint8[pop][h][k elem]) of shadows in the tiled layout:
    block b holds bytes [128 b, 128 b + 128) of every row, row o at 128 (b h + o),
    its 16-byte chunk c at chunk position c ^ (o % 8)."""
    raw = np.asarray(raw, dtype=np.uint8)
    pop = raw.shape[0]
    nb = (k * elem + 127) // 128
    t = raw[:, :nb * h * 128].reshape(pop, nb, h, 8, 16)
    o = np.arange(h)[:, None]
    pos = np.arange(8)[None, :] ^ (o % 8)                    # position of chunk c in row o
    rows = t[:, :, np.arange(h)[:, None], pos, :]            # [pop, nb, h, 8 (c), 16]
    rows = rows.transpose(0, 2, 1, 3, 4).reshape(pop, h, nb * 128)
    return np.ascontiguousarray(rows[:, :, :k * elem])
