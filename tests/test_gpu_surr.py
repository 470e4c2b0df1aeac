"""The surrogate form's state object: one generation in lock-step with the
oracle (recipes, descriptors, scores, the choice with and without the
pre-screen, the made children and their fitness), and what the trained
network gains over ranking offspring by their inherited fitness, the only
estimate the method without it has before evaluating them."""
import numpy as np
import pytest
from scipy import stats

from helpers import assert_fitness_close, assert_genes_close
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu

PRM = dict(sigma=0.05, mut_rate=0.2, n_elite=2, p_c=0.5)
DIMS = [64, 32, 10]


def _state(gpu, precision=0, pop=48, **sp):
    base = dict(mult=3, n_probe=8, hidden1=16, hidden2=8, train_steps=2, train_batch=64, history=2, warmup=0,
                audit_frac=0.2)
    base.update(sp)
    probe = (np.random.default_rng(11).integers(0, 256, size=(base["n_probe"], DIMS[0])) / 255.0).astype(np.float32)
    st = gpu.SurrState(pop, DIMS, gpu.Params(**PRM, precision=precision), gpu.SurrogateParams(**base), seed=9,
                       probe=probe)
    return st, probe


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("screen", [True, False])
def test_surrogate_generation_matches_oracle(gpu, oracle_mod, precision, screen):
    import torch
    st, probe = _state(gpu, precision)
    try:
        pop, c = st.pop, st.c
        rng = np.random.default_rng(3)
        parents = synthetic.random_population(pop, c, seed=4, scale=0.2)
        f_adj = rng.normal(-2.3, 0.2, size=pop).astype(np.float32)
        st.set_population(parents)
        st.set_fitness(f_adj)
        st.set_generation(5, True)
        st.set_screen(screen)
        theta0, _, _ = st.get_surrogate()
        batch = 40
        levels = rng.integers(0, 256, size=(batch, DIMS[0])).astype(np.uint8)
        y = rng.integers(0, DIMS[-1], size=batch).astype(np.int32)
        st.generation_u8(torch.from_numpy(levels).cuda(), torch.from_numpy(y).cuda())
        assert st.gen == 6
        step = st.get_step()
        oprm = oracle_mod.Params(**PRM, precision=precision)
        f64 = f_adj.astype(np.float64)
        order = oracle_mod.rank(f64)
        r1, r2, rk, rinh, rent = oracle_mod.select_recipes(oprm, f64, order, 9, 6, 3)
        np.testing.assert_array_equal(step["r_par1"], r1)
        np.testing.assert_array_equal(step["r_par2"], r2)
        np.testing.assert_array_equal(step["r_kind"], rk)
        np.testing.assert_array_equal(step["r_entity"], rent)
        desc_ref = oracle_mod.descriptors(oprm, DIMS, 9, 6, parents.astype(np.float64), f64, r1, r2, rk,
                                          step["r_f_inh"].astype(np.float64), rent, probe.astype(np.float64))
        d = step["desc"].astype(np.float64)
        np.testing.assert_allclose(d[:, 5:], desc_ref[:, 5:], rtol=1e-4, atol=1e-5 * np.abs(desc_ref[:, 5:]).max())
        np.testing.assert_allclose(d[:, :5], desc_ref[:, :5], rtol=1e-5, atol=1e-7)
        # scores: the oracle MLP on the descriptors standardised as the object did
        _, mu, sd = st.get_surrogate()
        xs = (d - mu.astype(np.float64)) / sd.astype(np.float64)
        np.testing.assert_allclose(mu, d.mean(axis=0), rtol=1e-5, atol=1e-6)
        pred_ref = oracle_mod.mlp_forward(theta0.astype(np.float64), xs, st.width, 16, 8)
        np.testing.assert_allclose(step["pred"], pred_ref, rtol=1e-4, atol=1e-4 * np.abs(pred_ref).max())
        # the choice: elites, then the best-scored recipes (or the plain EA's)
        n_e, n_c, n_m, _ = oracle_mod.counts(pop, oprm)
        k, R = pop - n_e, st.n_recipes
        order_r = np.lexsort((np.arange(R), -step["pred"].astype(np.float64)))
        chosen = order_r[:k] if screen else np.concatenate([np.arange(n_c), 3 * n_c + np.arange(n_m)])
        np.testing.assert_array_equal(step["row_recipe"][:k], chosen)
        rest = order_r[k:] if screen else np.setdiff1d(np.arange(R), chosen)
        audit = rest[(np.arange(st.n_audit) * (R - k)) // st.n_audit]
        np.testing.assert_array_equal(step["row_recipe"][k:], audit)
        np.testing.assert_array_equal(step["c_par1"][:n_e], order[:n_e])
        np.testing.assert_array_equal(step["c_kind"][:n_e], 0)
        np.testing.assert_array_equal(step["c_entity"][n_e:], rent[chosen])
        # the made children and their fitness
        kids = st.get_population()
        ref = oracle_mod.breed_entities(oprm, DIMS, 9, 6, parents.astype(np.float64), step["c_par1"], step["c_par2"],
                                        step["c_kind"], step["c_entity"])
        assert_genes_close(kids, ref, PRM["sigma"])
        f_raw, f_audit = st.raw_fitness()
        x64 = levels.astype(np.float64) / 255.0
        q = ref if precision == 0 else oracle_mod.quantize_w1(kids.astype(np.float64), DIMS, 1, None)
        f_ref, _ = oracle_mod.evaluate(q, DIMS, x64, y)
        assert_fitness_close(f_raw, f_ref, "children")
        a_kids = oracle_mod.breed_entities(oprm, DIMS, 9, 6, parents.astype(np.float64), r1[audit], r2[audit],
                                           rk[audit], rent[audit])
        if precision == 1:
            a_kids = oracle_mod.quantize_w1(a_kids, DIMS, 1, None)
        fa_ref, _ = oracle_mod.evaluate(a_kids, DIMS, x64, y)
        assert_fitness_close(f_audit, fa_ref, "audit")
        rho, screened, loss = st.stats()
        assert len(rho) == 1 and -1.0 <= rho[0] <= 1.0 and screened[0] == int(screen) and np.isfinite(loss[0])
        theta1, _, _ = st.get_surrogate()
        assert not np.array_equal(theta0, theta1)  # the generation trained the network
    finally:
        st.close()


def test_surrogate_full_size_sampled(gpu, oracle_mod):
    """One pre-screened generation at the benchmark's size and launch shape
    (population 2048, 784-112-10, 4 recipes per slot = 8,188 recipes, 32
    probe images, BF16): every recipe bit-exact; sampled descriptors, scores,
    made children and their fitness against the oracle."""
    import torch
    pop, dims, batch = 2048, [784, 112, 10], 100
    prm_d = dict(sigma=0.005, mut_rate=0.1, n_elite=1, p_c=0.5)
    (xtr, ytr), (xte, _) = synthetic.dataset(n_train=2000, n_test=64)
    probe = xte[:32]
    sp = gpu.SurrogateParams(mult=4, n_probe=32, warmup=0)
    st = gpu.SurrState(pop, dims, gpu.Params(**prm_d, precision=1), sp, seed=13, probe=probe)
    try:
        c = st.c
        parents = synthetic.random_population(pop, c, seed=8, scale=0.05)
        f_adj = np.random.default_rng(2).normal(-2.3, 0.3, size=pop).astype(np.float32)
        st.set_population(parents)
        st.set_fitness(f_adj)
        st.set_generation(11, True)
        st.set_screen(True)
        theta0, _, _ = st.get_surrogate()
        levels = synthetic.to_levels(xtr[:batch])
        y = ytr[:batch]
        st.generation_u8(torch.from_numpy(levels).cuda(), torch.from_numpy(y).cuda())
        step = st.get_step()
        oprm = oracle_mod.Params(**prm_d, precision=1)
        f64 = f_adj.astype(np.float64)
        order = oracle_mod.rank(f64)
        r1, r2, rk, rinh, rent = oracle_mod.select_recipes(oprm, f64, order, 13, 12, 4)
        assert st.n_recipes == r1.size == 8188
        np.testing.assert_array_equal(step["r_par1"], r1)
        np.testing.assert_array_equal(step["r_par2"], r2)
        np.testing.assert_array_equal(step["r_kind"], rk)
        np.testing.assert_array_equal(step["r_entity"], rent)
        sample = np.array([0, 1, 2047, 4093, 4094, 4095, 6000, 8187])
        p64 = parents.astype(np.float64)
        ref = oracle_mod.descriptors(oprm, dims, 13, 12, p64, f64, r1[sample], r2[sample], rk[sample],
                                     step["r_f_inh"][sample].astype(np.float64), rent[sample], probe.astype(np.float64))
        got = step["desc"][sample].astype(np.float64)
        np.testing.assert_array_equal(got[:, :3], ref[:, :3].astype(np.float32))
        np.testing.assert_allclose(got[:, 3:5], ref[:, 3:5], rtol=1e-5, atol=0)
        scale = np.abs(ref[:, 5:]).max()
        err = np.abs(got[:, 5:] - ref[:, 5:])
        # (an FP32 child gene one ulp off the oracle's may round to the other
        # BF16 neighbour: a few logits move by up to a BF16 ulp of a weight)
        assert (err <= 1e-4 * np.abs(ref[:, 5:]) + 1e-4 * scale).mean() >= 0.999, err.max()
        assert err.max() <= 1e-2 * scale
        # scores of the sampled recipes: the oracle MLP on the standardised descriptors
        _, mu, sd = st.get_surrogate()
        xs = (step["desc"][sample].astype(np.float64) - mu.astype(np.float64)) / sd.astype(np.float64)
        pred_ref = oracle_mod.mlp_forward(theta0.astype(np.float64), xs, st.width, 64, 64)
        np.testing.assert_allclose(step["pred"][sample], pred_ref, rtol=1e-4, atol=1e-4 * np.abs(pred_ref).max())
        # sampled made children and their fitness on the batch
        kids = st.get_population()
        slots = np.array([1, 2, 1000, 2046, 2047])
        ref_kids = oracle_mod.breed_entities(oprm, dims, 13, 12, p64, step["c_par1"][slots], step["c_par2"][slots],
                                             step["c_kind"][slots], step["c_entity"][slots])
        assert_genes_close(kids[slots], ref_kids, prm_d["sigma"])
        f_raw, _ = st.raw_fitness()
        q = oracle_mod.quantize_w1(kids[slots].astype(np.float64), dims, 1, None)
        f_ref, _ = oracle_mod.evaluate(q, dims, levels.astype(np.float64) / 255.0, y)
        assert_fitness_close(f_raw[slots], f_ref, "children")
    finally:
        st.close()


def test_trained_surrogate_ranks_offspring_better_than_inherited_fitness(gpu):
    """On the synthetic task: after a few generations of online training the
    network's scores rank the audited offspring (made and evaluated whatever
    their score) by their measured fitness better than f_inh does."""
    import torch
    pop, dims, batch = 256, [784, 32, 10], 100
    (xtr, ytr), (xte, _) = synthetic.dataset(n_train=20000, n_test=64)
    probe = xte[:32]
    sp = gpu.SurrogateParams(mult=4, n_probe=32, train_steps=32, history=4, warmup=3, audit_frac=0.25)
    st = gpu.SurrState(pop, dims, gpu.Params(sigma=0.01, mut_rate=0.1, n_elite=2, p_c=0.5), sp, seed=5, probe=probe)
    try:
        levels = synthetic.to_levels(xtr)
        idx = synthetic.batch_indices(len(ytr), batch, 40, seed=77)
        rho_model, rho_inh = [], []
        for g in range(40):
            st.generation_u8(torch.from_numpy(levels[idx[g]]).cuda(), torch.from_numpy(ytr[idx[g]]).cuda())
            if g >= 25:
                step = st.get_step()
                f_raw, f_audit = st.raw_fitness()
                k = pop - 2
                rows = step["row_recipe"][k:]  # the audit: spread over all scores
                rho_model.append(stats.spearmanr(step["pred"][rows], f_audit).statistic)
                rho_inh.append(stats.spearmanr(step["r_f_inh"][rows], f_audit).statistic)
        rho_s, scr, _ = st.stats()
        print(f"\n[surrogate] audit Spearman: trained network {np.mean(rho_model):.3f}, "
              f"f_inh {np.mean(rho_inh):.3f}; pre-screen used in {int(scr.sum())} of {len(scr)} generations")
        assert np.mean(rho_model) > np.mean(rho_inh) + 0.05
    finally:
        st.close()


def test_surrogate_argument_errors(gpu):
    probe = np.zeros((8, DIMS[0]), dtype=np.float32)
    with pytest.raises(gpu.LeeaError):
        gpu.SurrState(16, DIMS, gpu.Params(precision=2), gpu.SurrogateParams(n_probe=8), seed=1, probe=probe)
    with pytest.raises(gpu.LeeaError):
        gpu.SurrState(16, DIMS, gpu.Params(), gpu.SurrogateParams(n_probe=33), seed=1, probe=probe)
    with pytest.raises(gpu.LeeaError):
        gpu.SurrState(16, [60, 32, 10], gpu.Params(), gpu.SurrogateParams(n_probe=8), seed=1, probe=probe)
