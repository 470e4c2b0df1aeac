"""Pins of the oracle's random streams (Philox4x32-10, uniforms, normals).

The generator is pinned against cuRAND's host-side Philox4_32_10 generator, a
library implementation of the same published algorithm (Salmon et al., SC'11)
that shares nothing with the oracle: cuRAND's host output block j is Philox
of the counter (j >> 16, 0, j & 0xffff, 0) under key (seed lo, seed hi).
"""
import ctypes
import ctypes.util
import math

import numpy as np
import pytest
from scipy import stats


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand_words(seed: int, n: int) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not loadable")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = (ctypes.c_uint32 * n)()
        assert lib.curandGenerate(gen, out, ctypes.c_size_t(n)) == 0
        return np.frombuffer(out, dtype=np.uint32).copy()
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 0x123456789ABCDEF0, 0xFEEDBEEF01234567, 42])
def test_philox_matches_curand_host_generator(oracle_mod, seed):
    blocks = 65536 + 4
    words = _curand_words(seed, 4 * blocks)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for j in list(range(0, 8)) + [1000, 65535, 65536, 65537, 65539]:
        ctr = (j >> 16, 0, j & 0xFFFF, 0)
        np.testing.assert_array_equal(oracle_mod.philox(ctr, key), words[4 * j:4 * j + 4], err_msg=f"block {j}")


def test_stream_counter_layout(oracle_mod):
    # Draw n of stream (tag, gen, ent) is word n&3 of Philox((n>>2, ent, gen, tag)).
    seed = 0xDEADBEEFCAFEF00D
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for tag, gen, ent, n in [(1, 0, 5, 0), (2, 7, 3, 5), (3, 11, 999, 89049), (5, 2**31, 2**20, 13)]:
        blk = oracle_mod.philox((n >> 2, ent, gen, tag), key)
        assert oracle_mod.draw(seed, tag, gen, ent, n) == int(blk[n & 3])


def test_u01_open_interval_and_exact():
    import oracle
    lo = oracle.u01(0)
    hi = oracle.u01(0xFFFFFFFF)
    assert lo == 2.0 ** -24 and hi == 1.0 - 2.0 ** -24
    for u in [0, 1, 511, 512, 0x80000000, 0xFFFFFFFF, 123456789]:
        v = oracle.u01(u)
        assert 0.0 < v < 1.0
        assert float(np.float32(v)) == v  # exact in FP32, so the GPU can match it bitwise


def test_index_and_threshold_edges(oracle_mod):
    assert oracle_mod.index(0, 7) == 0
    assert oracle_mod.index(0xFFFFFFFF, 7) == 6
    assert oracle_mod.index(0x80000000, 2) == 1
    assert oracle_mod.threshold(0.0) == 0
    assert oracle_mod.threshold(1.0) == 2 ** 32
    assert oracle_mod.threshold(0.5) == 2 ** 31
    assert oracle_mod.threshold(0.1) == math.floor(0.1 * 2 ** 32)


def test_index_is_uniform(oracle_mod):
    m, n = 37, 74000
    counts = np.zeros(m)
    for k in range(n):
        counts[oracle_mod.index(oracle_mod.draw(9, 2, 1, k // 64, k % 64), m)] += 1
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4, (chi2, p)


def test_normals_are_standard_normal(oracle_mod):
    z = np.array([oracle_mod.normal(77, 5, 3, e, i) for e in range(10) for i in range(2000)])
    assert abs(z.mean()) < 0.05 and abs(z.std() - 1.0) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # The cosine and sine partners of one Box-Muller pair are uncorrelated.
    pairs = z.reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 0.05


def test_normal_uses_box_muller_pairs(oracle_mod):
    # Genes 4b+0/4b+1 share words (0,1) of block b; 4b+2/4b+3 share (2,3):
    # partners have the same radius.
    seed, tag, gen, ent = 5, 5, 9, 4
    for b in range(5):
        for pair in range(2):
            i = 4 * b + 2 * pair
            r0 = math.hypot(oracle_mod.normal(seed, tag, gen, ent, i), oracle_mod.normal(seed, tag, gen, ent, i + 1))
            u1 = oracle_mod.u01(oracle_mod.draw(seed, tag, gen, ent, i))
            assert abs(r0 - math.sqrt(-2.0 * math.log(u1))) < 1e-12


def test_draw16_layout_and_threshold(oracle_mod):
    # 16-bit draw i: half (i & 1) of word ((i >> 1) & 3) of block (i >> 3).
    seed = 0x5EED5EED12345678
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for tag, gen, ent in [(3, 4, 9), (4, 1, 0)]:
        for i in range(0, 40):
            blk = oracle_mod.philox((i >> 3, ent, gen, tag), key)
            word = int(blk[(i >> 1) & 3])
            expect = (word >> 16) if (i & 1) else (word & 0xFFFF)
            assert oracle_mod.draw16(seed, tag, gen, ent, i) == expect
    assert oracle_mod.threshold16(0.0) == 0
    assert oracle_mod.threshold16(0.5) == 32768
    assert oracle_mod.threshold16(1.0) == 65536
    assert oracle_mod.threshold16(0.1) == 6553


def test_draw16_is_uniform(oracle_mod):
    u = np.array([oracle_mod.draw16(3, 4, 5, e, i) for e in range(4) for i in range(8192)])
    counts = np.bincount(u >> 10, minlength=64)  # 64 equal bins
    assert stats.chisquare(counts).pvalue > 1e-4
