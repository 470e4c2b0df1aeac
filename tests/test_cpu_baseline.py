"""The FP32 multi-core CPU baseline (oracle/leea_cpu_fp32.c) makes the same
generation as the FP64 oracle: selection from the oracle itself, children
within FP32 rounding of the oracle's (masks and parents identical), fitness
within the FP32 evaluation tolerance.  It is a baseline to time, so this
only checks that it computes the method."""
import numpy as np

from helpers import assert_correct_close, assert_fitness_close
from paper_1806_09819_gb300 import synthetic


def test_fp32_baseline_generation_matches_oracle(oracle_mod):
    dims, pop, batch = [64, 16, 10], 24, 20
    prm = oracle_mod.Params(n_elite=2, p_c=0.5, sigma=0.05, mut_rate=0.3, alpha=0.5, rho=0.5)
    c = oracle_mod.num_params(dims)
    parents = synthetic.random_population(pop, c, seed=3, scale=0.2).astype(np.float32)
    f_adj = np.random.default_rng(4).normal(-2.3, 0.1, size=pop).astype(np.float32)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, size=(batch, dims[0])).astype(np.float32)
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    seed, gen = 77, 9
    kids, f_raw, f_out, cor, threads = oracle_mod.cpu32_generation(prm, dims, seed, gen, parents, f_adj, x, y)
    assert threads >= 1
    f64 = f_adj.astype(np.float64)
    order = oracle_mod.rank(f64)
    p1, p2, kind, f_inh = oracle_mod.select(prm, f64, order, seed, gen)
    ref = oracle_mod.breed(prm, dims, seed, gen, parents.astype(np.float64), p1, p2, kind)
    # identical masks and parents: differences are FP32 rounding of sigma z only
    np.testing.assert_allclose(kids, ref, rtol=0, atol=1e-6 + 1e-5 * float(prm.sigma))
    f_ref, cor_ref, logits = oracle_mod.evaluate(kids.astype(np.float64), dims, x.astype(np.float64), y,
                                                 want_logits=True)
    assert_fitness_close(f_raw, f_ref)
    assert_correct_close(cor, cor_ref, logits)
    adj = oracle_mod.inherit(float(np.float32(prm.alpha)), f_inh, f_ref, first=False)
    assert_fitness_close(f_out, adj, "f_adj")
