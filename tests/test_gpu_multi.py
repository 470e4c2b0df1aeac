"""The batching form (many runs in one multi-run object): each run's trajectory
equals that of a single-run state object with the same seed and minibatches
(bit for bit), one generation checked against the oracle in lock-step, the
captured graph replaying exactly what direct launches compute, and the
autotuner's choices."""
import numpy as np
import pytest

from helpers import assert_fitness_close, assert_genes_close, decode_bf16, decode_e4m3, untile_shadow
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu

D_IN, D_OUT = 784, 10
SPECS = [(50, 16, 8, 11), (300, 112, 200, 12), (37, 256, 129, 13), (129, 48, 64, 14)]  # pop, h, batch, seed
PRM = dict(sigma=0.02, mut_rate=0.1, n_elite=2, p_c=0.5, alpha=0.5)


def _specs(gpu, chunk=0):
    return [gpu.RunSpec(pop=p, hidden=h, batch=b, chunk=chunk, seed=s) for p, h, b, s in SPECS]


def _batches(m, n_gens, seed=7):
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, 256, size=(n_gens, m.total_rows, D_IN)).astype(np.uint8)
    ys = rng.integers(0, D_OUT, size=(n_gens, m.total_rows)).astype(np.int32)
    return xs, ys


@pytest.mark.parametrize("precision", [1, 2])
def test_multi_matches_single_run_objects(gpu, precision):
    import torch
    prm = gpu.Params(**PRM, precision=precision)
    m = gpu.MultiRun(_specs(gpu), D_IN, D_OUT, prm)
    singles = [gpu.LeeaState(p, [D_IN, h, D_OUT], prm, seed=s) for p, h, b, s in SPECS]
    try:
        n_gens = 4
        xs, ys = _batches(m, n_gens)
        for g in range(n_gens):
            m.generation_u8(torch.from_numpy(xs[g]).cuda(), torch.from_numpy(ys[g]).cuda())
            for r, st in enumerate(singles):
                rows = m.rows_slice(r)
                st.leea_generation_u8(torch.from_numpy(np.ascontiguousarray(xs[g][rows])).cuda(),
                                      torch.from_numpy(np.ascontiguousarray(ys[g][rows])).cuda())
            f_multi = m.raw_fitness()
            assert m.gen == g
            for r, st in enumerate(singles):
                np.testing.assert_array_equal(f_multi[m.run_slice(r)], st.leea_raw_fitness(), err_msg=f"run {r}")
        for r, st in enumerate(singles):
            np.testing.assert_array_equal(m.get_population(r), st.leea_get_population(), err_msg=f"run {r}")
            sel_m, sel_s = m.get_selection(r), st.leea_get_selection()
            for a, b in zip(sel_m, sel_s):
                np.testing.assert_array_equal(a, b)
    finally:
        m.close()
        for st in singles:
            st.close()


def test_multi_other_outputs_matches_single_run_objects(gpu):
    # 16 and 3 outputs (not the usual 10): the group evaluation's general
    # layer-2 code, one-, two- and many-individual units, one and several tiles.
    import torch
    for d_out, specs in ((16, [(40, 144, 150, 21), (70, 32, 40, 22), (25, 96, 260, 23)]),
                         (3, [(30, 16, 20, 24), (17, 208, 129, 25)])):
        prm = gpu.Params(**PRM, precision=1)
        m = gpu.MultiRun([gpu.RunSpec(pop=p, hidden=h, batch=b, seed=s) for p, h, b, s in specs], D_IN, d_out, prm)
        singles = [gpu.LeeaState(p, [D_IN, h, d_out], prm, seed=s) for p, h, b, s in specs]
        try:
            rng = np.random.default_rng(d_out)
            for g in range(3):
                xs = rng.integers(0, 256, size=(m.total_rows, D_IN)).astype(np.uint8)
                ys = rng.integers(0, d_out, size=m.total_rows).astype(np.int32)
                m.generation_u8(torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda())
                for r, st in enumerate(singles):
                    rows = m.rows_slice(r)
                    st.leea_generation_u8(torch.from_numpy(np.ascontiguousarray(xs[rows])).cuda(),
                                          torch.from_numpy(np.ascontiguousarray(ys[rows])).cuda())
                f_multi = m.raw_fitness()
                for r, st in enumerate(singles):
                    np.testing.assert_array_equal(f_multi[m.run_slice(r)], st.leea_raw_fitness(),
                                                  err_msg=f"d_out {d_out} run {r} generation {g}")
        finally:
            m.close()
            for st in singles:
                st.close()


def test_graph_replay_equals_direct_launches(gpu):
    import torch
    prm = gpu.Params(**PRM, precision=1)
    a = gpu.MultiRun(_specs(gpu), D_IN, D_OUT, prm)
    b = gpu.MultiRun(_specs(gpu), D_IN, D_OUT, prm)
    try:
        b.profile_enable(True)  # direct launches between events
        xs, ys = _batches(a, 5, seed=3)
        for g in range(5):
            x, y = torch.from_numpy(xs[g]).cuda(), torch.from_numpy(ys[g]).cuda()
            a.generation_u8(x, y)
            b.generation_u8(x, y)
        np.testing.assert_array_equal(a.fitness(), b.fitness())
        prof = b.profile_read()
        assert all(prof[k][1] == 4 for k in ("select", "breed", "evaluate")), prof
        for r in range(len(SPECS)):
            np.testing.assert_array_equal(a.get_population(r), b.get_population(r))
    finally:
        a.close()
        b.close()


def _bound_exp(oracle_mod, kind, par1, par2, amax_par, sigma):
    out = np.empty(kind.size, dtype=np.int32)
    s32 = np.float32(sigma)
    for j in range(kind.size):
        bnd = np.float32(amax_par[par1[j]])
        if kind[j] == 1:
            bnd = max(bnd, np.float32(amax_par[par2[j]]))
        elif kind[j] == 2:
            bnd = np.float32(np.float64(s32) * np.float64(np.float32(5.77)) + np.float64(bnd))
        out[j] = oracle_mod.fp8_scale_exp(float(bnd))
    return out


@pytest.mark.parametrize("precision", [1, 2])
def test_multi_generation_matches_oracle(gpu, oracle_mod, precision):
    import torch
    prm = gpu.Params(**PRM, precision=precision)
    oprm = oracle_mod.Params(**PRM)
    specs = [gpu.RunSpec(pop=24, hidden=16, batch=40, seed=21), gpu.RunSpec(pop=17, hidden=160, batch=150, seed=22)]
    m = gpu.MultiRun(specs, D_IN, D_OUT, prm)
    try:
        rng = np.random.default_rng(5)
        parents, n_w1 = [], []
        for r, sp in enumerate(specs):
            dims = [D_IN, sp.hidden, D_OUT]
            popv = synthetic.random_population(sp.pop, gpu.leea_layout_num_params(dims), seed=30 + r, scale=0.1)
            m.set_population(r, popv)
            parents.append(popv)
            n_w1.append(D_IN * sp.hidden)
        f_adj = rng.normal(-2.3, 0.1, size=m.total_pop).astype(np.float32)
        m.set_fitness(f_adj)
        m.set_generation(4, True)
        xs, ys = _batches(m, 1, seed=9)
        m.generation_u8(torch.from_numpy(xs[0]).cuda(), torch.from_numpy(ys[0]).cuda())
        f_raw = m.raw_fitness()
        assert m.gen == 5
        for r, sp in enumerate(specs):
            dims = [D_IN, sp.hidden, D_OUT]
            fa = f_adj[m.run_slice(r)].astype(np.float64)
            order, par1, par2, kind, f_inh = m.get_selection(r)
            o_order = oracle_mod.rank(fa)
            o_p1, o_p2, o_kind, o_inh = oracle_mod.select(oprm, fa, o_order, sp.seed, 5)
            np.testing.assert_array_equal(order, o_order)
            np.testing.assert_array_equal(par1, o_p1)
            np.testing.assert_array_equal(par2, o_p2)
            np.testing.assert_array_equal(kind, o_kind)
            kids = m.get_population(r)
            ref = oracle_mod.breed(oprm, dims, sp.seed, 5, parents[r].astype(np.float64), par1, par2, kind)
            assert_genes_close(kids, ref, PRM["sigma"], f"run {r} children")
            sh, se, am = m.get_shadow(r, precision)
            np.testing.assert_array_equal(am, np.abs(kids[:, :n_w1[r]]).max(axis=1))
            amax_par = np.abs(parents[r][:, :n_w1[r]]).max(axis=1)
            se_ref = _bound_exp(oracle_mod, kind, par1, par2, amax_par, PRM["sigma"])
            if precision == 2:
                np.testing.assert_array_equal(se, se_ref)
            elem = 2 if precision == 1 else 1
            rows = untile_shadow(sh, D_IN, sp.hidden, elem).reshape(sp.pop, -1)
            got = decode_bf16(rows.view(np.uint16)) if precision == 1 else \
                decode_e4m3(rows) * np.ldexp(1.0, se_ref.astype(np.int64))[:, None]
            q = oracle_mod.quantize_w1(kids.astype(np.float64), dims, precision, se_ref)
            np.testing.assert_array_equal(got, q[:, :n_w1[r]])
            x64 = xs[0][m.rows_slice(r)].astype(np.float64) / 255.0
            f_ref, _ = oracle_mod.evaluate(q, dims, x64, ys[0][m.rows_slice(r)])
            assert_fitness_close(f_raw[m.run_slice(r)], f_ref, f"run {r} fitness")
    finally:
        m.close()


def test_multi_argument_errors(gpu):
    prm = gpu.Params(**PRM, precision=1)
    with pytest.raises(gpu.LeeaError, match="precision"):
        gpu.MultiRun(_specs(gpu), D_IN, D_OUT, gpu.Params(**PRM))
    with pytest.raises(gpu.LeeaError):
        gpu.MultiRun([gpu.RunSpec(pop=5000, hidden=16, batch=8)], D_IN, D_OUT, prm)
    with pytest.raises(gpu.LeeaError, match="chunk"):
        gpu.MultiRun([gpu.RunSpec(pop=5, hidden=64, batch=8, chunk=24)], D_IN, D_OUT, prm)
    with pytest.raises(gpu.LeeaError):
        gpu.MultiRun([gpu.RunSpec(pop=5, hidden=40, batch=8)], D_IN, D_OUT, prm)  # h % 16 != 0


def test_autotune_picks_a_candidate_and_caches(gpu, tmp_path):
    from paper_1806_09819_gb300 import autotune
    specs = [gpu.RunSpec(pop=100, hidden=256, batch=64), gpu.RunSpec(pop=100, hidden=48, batch=300)]
    cache = str(tmp_path / "tune.json")
    tuned, timings = autotune.tune(specs, D_IN, D_OUT, 1, cache_path=cache, pop=160, reps=2)
    assert len(timings) == 2
    for sp in tuned:  # both classes take the group evaluation: the tuner picks the group
        assert sp.chunk == 0 and sp.group in autotune.group_candidates(sp.hidden)
    assert all(len(t) == len(autotune.group_candidates(h)) for t, h in zip(timings.values(), (256, 48)))
    tuned2, timings2 = autotune.tune(specs, D_IN, D_OUT, 1, cache_path=cache)
    assert timings2 == {} and [s.group for s in tuned2] == [s.group for s in tuned]
    # a tuned multi-run object uses the chosen groups
    m = gpu.MultiRun(tuned, D_IN, D_OUT, gpu.Params(**PRM, precision=1))
    try:
        for r, sp in enumerate(tuned):
            assert m.run_shape(r)[3] == sp.group
    finally:
        m.close()
    # a group wider than N = 256 allows is refused
    with pytest.raises(gpu.LeeaError, match="group"):
        gpu.MultiRun([gpu.RunSpec(pop=5, hidden=128, batch=8, group=3)], D_IN, D_OUT, gpu.Params(**PRM, precision=1))
