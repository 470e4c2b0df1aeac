"""The single-launch generation of small populations (eval_path SMALL; AUTO at
the small configuration): one kernel ranks, selects, breeds and evaluates
(Algorithm 1; Sections 3.1-3.3).  Against two independent checks:

* the two-kernel path with the CUDA-core evaluation (eval_path SIMT) from the
  same state, generation after generation: selection, children and sigma
  genes bit-identical (the same operators and streams); fitness within the
  evaluation tolerance (the same FP32 products, summed in another fixed
  order), correct counts equal up to near-ties of the FP64 logits; the SIMT
  fitness is handed to the single-launch state before the next generation so
  that both select from the same values;
* the FP64 oracle in lock step: selection exact, children and fitness within
  the stated tolerances (tests/test_gpu_generation.py's _lockstep).
Also AUTO's choice of the path, the batch scratch growing between calls, the
determinism of the fitness and the shape limits."""
import numpy as np
import pytest

from helpers import assert_correct_close, assert_fitness_close
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _batch(dims, batch, seed):
    torch = _torch()
    if dims[0] == 784:
        x, y = synthetic.make_split(batch, seed=seed)
        lv = synthetic.to_levels(x)
    else:
        rng = np.random.default_rng(seed)
        lv = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
        y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    return torch.from_numpy(np.ascontiguousarray(lv)).cuda(), torch.from_numpy(np.ascontiguousarray(y)).cuda()


def _bits(a):
    a = np.asarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a


SMALL_CASES = [
    # the small benchmark configuration: P 32, 784-32-10, batch 16
    dict(dims=[784, 32, 10], pop=32, batches=[16] * 4, prm=dict(n_elite=1, p_c=0.5, sigma=0.005, mut_rate=0.1)),
    # tournament, arithmetic crossover, inheritance blend, every gene mutated
    dict(dims=[784, 16, 10], pop=20, batches=[1, 7, 16],
         prm=dict(sel_op=1, tour_k=3, xo_op=1, alpha=0.3, sigma=0.02, mut_rate=1.0)),
    # odd shapes: d_0 = 100 (quarters of 28 inputs, the last 16), h = 24 (three slices), d_out = 3;
    # batches up to the limit (tiles of 32, 64, 128)
    dict(dims=[100, 24, 3], pop=9, batches=[33, 128, 64, 5], prm=dict(n_elite=2, xo_gene_p=0.2, sigma=0.1)),
    # one slice per child, 16 outputs, decaying sigma; a population of one; d_0 = 8 (empty quarters)
    dict(dims=[64, 8, 16], pop=1, batches=[3, 3], prm=dict(n_elite=0, sigma=0.05, sigma_ctl=1, sigma_k=2.0)),
    dict(dims=[8, 16, 4], pop=5, batches=[12, 1], prm=dict(sigma=0.2)),
    # self-adaptive sigma genes; populations of two and 64
    dict(dims=[784, 32, 10], pop=2, batches=[16, 2], prm=dict(sigma=0.01, sigma_ctl=2, tau=0.3, n_elite=0)),
    dict(dims=[196, 48, 10], pop=64, batches=[24, 24, 100],
         prm=dict(sigma=0.01, sigma_ctl=2, tau=0.1, p_c=0.75, n_elite=-1, p_e=0.05)),
    # the largest cluster: 8 slices per child (h = 64), tournament selection, 40 individuals (bitonic ranking)
    dict(dims=[256, 64, 10], pop=40, batches=[30, 12], prm=dict(sel_op=1, tour_k=2, sigma=0.03, p_c=0.6)),
    # a large population: 1024 rank keys sorted in shared memory, 600 clusters of one slice
    dict(dims=[16, 8, 4], pop=600, batches=[4, 9, 4], prm=dict(sigma=0.05, p_c=0.3, n_elite=-1, p_e=0.1)),
    # more than 8 slices per child (h = 72 and 128): the hand-over through L2 and an arrival counter
    dict(dims=[64, 72, 10], pop=5, batches=[8, 8, 20], prm=dict(sigma=0.05, n_elite=1)),
    dict(dims=[784, 128, 10], pop=3, batches=[16, 16], prm=dict(sigma=0.01, mut_rate=0.3)),
]


@pytest.mark.parametrize("case", SMALL_CASES, ids=lambda c: f"{c['dims']}-P{c['pop']}-B{c['batches']}")
def test_small_generation_matches_two_kernel_simt_path(gpu, oracle_mod, case):
    from paper_1806_09819_gb300 import leea
    dims, pop, prm = case["dims"], case["pop"], case["prm"]
    sigma = prm.get("sigma_ctl", 0) == 2
    ref = gpu.LeeaState(pop, dims, gpu.Params(**prm, eval_path=leea.EVAL_SIMT), seed=123)
    sgl = gpu.LeeaState(pop, dims, gpu.Params(**prm, eval_path=leea.EVAL_SMALL), seed=123)
    try:
        for g, b in enumerate(case["batches"]):
            xd, yd = _batch(dims, b, seed=1000 + g)
            for st in (ref, sgl):
                st.leea_generation_u8(xd, yd, 255.0)
            kids = ref.leea_get_population()
            np.testing.assert_array_equal(_bits(sgl.leea_get_population()), _bits(kids),
                                          err_msg=f"generation {g}: children")
            if g > 0:
                for x, y in zip(sgl.leea_get_selection(), ref.leea_get_selection()):
                    np.testing.assert_array_equal(_bits(x), _bits(y), err_msg=f"generation {g}: selection")
            if sigma:
                np.testing.assert_array_equal(_bits(sgl.leea_get_sigma()), _bits(ref.leea_get_sigma()))
            f_ref, cor_ref = ref.leea_fitness(with_correct=True)
            f_sgl, cor_sgl = sgl.leea_fitness(with_correct=True)
            assert_fitness_close(sgl.leea_raw_fitness(), ref.leea_raw_fitness(), f"generation {g}: f_raw")
            assert_fitness_close(f_sgl, f_ref, f"generation {g}: f_adj")
            x64 = xd.cpu().numpy().astype(np.float64) / 255.0
            _, _, logits = oracle_mod.evaluate(kids.astype(np.float64), dims, x64, yd.cpu().numpy(),
                                               want_logits=True)
            assert_correct_close(cor_sgl, cor_ref, logits)
            sgl.leea_set_fitness(f_ref)  # both select from the same values next
    finally:
        ref.close()
        sgl.close()


def test_small_generation_is_deterministic(gpu):
    from paper_1806_09819_gb300 import leea
    runs = []
    for _ in range(2):
        st = gpu.LeeaState(32, [784, 32, 10], gpu.Params(sigma=0.005, mut_rate=0.1, eval_path=leea.EVAL_SMALL), 4)
        try:
            for g in range(4):
                st.leea_generation_u8(*_batch([784, 32, 10], 16, seed=g), 255.0)
            runs.append((st.leea_get_population(), st.leea_fitness(with_correct=True)))
        finally:
            st.close()
    np.testing.assert_array_equal(_bits(runs[0][0]), _bits(runs[1][0]))
    np.testing.assert_array_equal(_bits(runs[0][1][0]), _bits(runs[1][1][0]))
    np.testing.assert_array_equal(runs[0][1][1], runs[1][1][1])


def test_small_generation_lockstep_with_oracle(gpu, oracle_mod):
    from test_gpu_generation import CONFIG_SMALL, _lockstep
    from paper_1806_09819_gb300 import leea
    prm = dict(CONFIG_SMALL["prm"], eval_path=leea.EVAL_SMALL)
    _lockstep(gpu, oracle_mod, CONFIG_SMALL["dims"], CONFIG_SMALL["pop"], CONFIG_SMALL["batch"], prm, u8=True)
    # the benchmark's operators; odd shapes; the degenerate population of one
    _lockstep(gpu, oracle_mod, [784, 32, 10], 32, 16,
              dict(n_elite=1, p_c=0.5, sigma=0.005, mut_rate=0.1, eval_path=leea.EVAL_SMALL), u8=True)
    _lockstep(gpu, oracle_mod, [784, 24, 10], 7, 40, dict(sigma=0.05, xo_op=1, eval_path=leea.EVAL_SMALL), u8=True)
    _lockstep(gpu, oracle_mod, [784, 8, 10], 1, 1, dict(sigma=0.05, n_elite=-1, eval_path=leea.EVAL_SMALL), u8=True)


def test_auto_takes_the_single_launch_generation_when_small(gpu):
    from paper_1806_09819_gb300 import leea
    xd, yd = _batch([784, 32, 10], 16, seed=3)
    st = gpu.LeeaState(32, [784, 32, 10], gpu.Params(sigma=0.005, mut_rate=0.1), seed=9)
    try:
        st.leea_generation_u8(xd, yd, 255.0)
        st.leea_profile_enable(True)
        for _ in range(5):
            st.leea_generation_u8(xd, yd, 255.0)
        prof = st.leea_profile_read()
        launches = [prof[s][1] for s in leea.STAGES]
        assert launches == [0, 5, 0], prof
        # the same children and fitness as the explicit path
        ref = gpu.LeeaState(32, [784, 32, 10], gpu.Params(sigma=0.005, mut_rate=0.1, eval_path=leea.EVAL_SMALL),
                            seed=9)
        try:
            for _ in range(6):
                ref.leea_generation_u8(xd, yd, 255.0)
            np.testing.assert_array_equal(_bits(st.leea_get_population()), _bits(ref.leea_get_population()))
            np.testing.assert_array_equal(_bits(st.leea_fitness()), _bits(ref.leea_fitness()))
        finally:
            ref.close()
    finally:
        st.close()
    # a population too large for it: AUTO keeps the chain of kernels
    big = gpu.LeeaState(1000, [784, 32, 10], gpu.Params(), seed=9)
    try:
        big.leea_generation_u8(xd, yd, 255.0)
        big.leea_profile_enable(True)
        big.leea_generation_u8(xd, yd, 255.0)
        prof = big.leea_profile_read()
        assert prof[leea.STAGES[0]][1] == 1 and prof[leea.STAGES[2]][1] == 1, prof
    finally:
        big.close()


def test_small_generation_limits(gpu):
    from paper_1806_09819_gb300 import leea
    torch = _torch()
    with pytest.raises(gpu.LeeaError):  # FP32 populations only
        gpu.LeeaState(8, [784, 32, 10], gpu.Params(precision=1, eval_path=leea.EVAL_SMALL), 1)
    with pytest.raises(gpu.LeeaError):  # one hidden layer
        gpu.LeeaState(8, [196, 32, 16, 10], gpu.Params(eval_path=leea.EVAL_SMALL), 1)
    for dims, batch in (([784, 12, 10], 8), ([784, 32, 10], 129), ([30, 16, 10], 8)):  # h % 8, batch, d_0 % 4
        st = gpu.LeeaState(8, dims, gpu.Params(eval_path=leea.EVAL_SMALL), 1)
        try:
            x = torch.zeros((batch, dims[0]), dtype=torch.uint8, device="cuda")
            y = torch.zeros(batch, dtype=torch.int32, device="cuda")
            with pytest.raises(gpu.LeeaError) as e:
                st.leea_generation_u8(x, y, 255.0)
            assert e.value.status == gpu.EINVAL
        finally:
            st.close()
    st = gpu.LeeaState(8, [784, 32, 10], gpu.Params(eval_path=leea.EVAL_SMALL), 1)
    try:  # FP32 batches 16-byte aligned (this one is 4 bytes off)
        xf = torch.zeros(8 * 784 + 1, dtype=torch.float32, device="cuda")[1:].view(8, 784)
        y = torch.zeros(8, dtype=torch.int32, device="cuda")
        with pytest.raises(gpu.LeeaError) as e:
            st.leea_generation(xf, y)
        assert e.value.status == gpu.EINVAL
    finally:
        st.close()


def test_auto_switches_between_the_paths_with_the_batch(gpu, oracle_mod):
    # Batches inside the single-launch limits take it, a batch past them the
    # chain of kernels; the object's fitness buffers stay consistent across the
    # switches (children bit-identical to the two-kernel CUDA-core path's,
    # fitness within tolerance, the oracle's near-ties allowed).
    from paper_1806_09819_gb300 import leea
    dims, pop = [784, 32, 10], 32
    prm = dict(sigma=0.01, mut_rate=0.1, n_elite=1)
    ref = gpu.LeeaState(pop, dims, gpu.Params(**prm, eval_path=leea.EVAL_SIMT), seed=77)
    auto = gpu.LeeaState(pop, dims, gpu.Params(**prm), seed=77)
    try:
        for g, b in enumerate([16, 200, 16, 16, 150, 8]):
            xd, yd = _batch(dims, b, seed=500 + g)
            auto.leea_profile_enable(True)
            for st in (ref, auto):
                st.leea_generation_u8(xd, yd, 255.0)
            prof = auto.leea_profile_read()
            single = b <= 128
            if g > 0:
                assert (prof[leea.STAGES[0]][1] == 0) == single, (b, prof)
            kids = ref.leea_get_population()
            np.testing.assert_array_equal(_bits(auto.leea_get_population()), _bits(kids), err_msg=f"batch {b}")
            f_ref, cor_ref = ref.leea_fitness(with_correct=True)
            f_auto, cor_auto = auto.leea_fitness(with_correct=True)
            assert_fitness_close(f_auto, f_ref, f"batch {b}: f_adj")
            x64 = xd.cpu().numpy().astype(np.float64) / 255.0
            _, _, logits = oracle_mod.evaluate(kids.astype(np.float64), dims, x64, yd.cpu().numpy(), want_logits=True)
            assert_correct_close(cor_auto, cor_ref, logits)
            auto.leea_set_fitness(f_ref)
    finally:
        ref.close()
        auto.close()


def _batch_f32(dims, batch, seed):
    torch = _torch()
    if dims[0] == 784:
        x, y = synthetic.make_split(batch, seed=seed)
    else:
        x, y = synthetic.tiny_problem(dims[0], dims[-1], batch, seed=seed)
    return torch.from_numpy(np.ascontiguousarray(x)).cuda(), torch.from_numpy(np.ascontiguousarray(y)).cuda()


@pytest.mark.parametrize("case", [
    dict(dims=[784, 32, 10], pop=32, batches=[16, 16, 5], prm=dict(sel_op=1, tour_k=3, sigma=0.01, alpha=0.2)),
    dict(dims=[100, 24, 3], pop=9, batches=[33, 100], prm=dict(n_elite=2, xo_op=1, sigma=0.1)),
    dict(dims=[64, 72, 10], pop=5, batches=[8, 20], prm=dict(sigma=0.05)),
], ids=lambda c: f"{c['dims']}-P{c['pop']}")
def test_small_generation_fp32_inputs_match_the_cuda_core_path(gpu, oracle_mod, case):
    # FP32 batches (x_hi w_hi + x_hi w_lo + x_lo w_hi on the tensor cores):
    # children bit-identical, fitness within the evaluation tolerance of the
    # two-kernel CUDA-core path and of the FP64 oracle's evaluation of the same children.
    from paper_1806_09819_gb300 import leea
    dims, pop, prm = case["dims"], case["pop"], case["prm"]
    ref = gpu.LeeaState(pop, dims, gpu.Params(**prm, eval_path=leea.EVAL_SIMT), seed=31)
    sgl = gpu.LeeaState(pop, dims, gpu.Params(**prm, eval_path=leea.EVAL_SMALL), seed=31)
    try:
        for g, b in enumerate(case["batches"]):
            xd, yd = _batch_f32(dims, b, seed=700 + g)
            for st in (ref, sgl):
                st.leea_generation(xd, yd)
            kids = ref.leea_get_population()
            np.testing.assert_array_equal(_bits(sgl.leea_get_population()), _bits(kids))
            f_ref, cor_ref = ref.leea_fitness(with_correct=True)
            f_sgl, cor_sgl = sgl.leea_fitness(with_correct=True)
            assert_fitness_close(f_sgl, f_ref, f"generation {g}: f_adj")
            o_f, _, logits = oracle_mod.evaluate(kids.astype(np.float64), dims, xd.cpu().numpy().astype(np.float64),
                                                 yd.cpu().numpy(), want_logits=True)
            assert_fitness_close(sgl.leea_raw_fitness(), o_f, f"generation {g}: f_raw vs the oracle")
            assert_correct_close(cor_sgl, cor_ref, logits)
            sgl.leea_set_fitness(f_ref)
    finally:
        ref.close()
        sgl.close()


def test_small_generation_fp32_lockstep_with_oracle(gpu, oracle_mod):
    from test_gpu_generation import CONFIG_SMALL, _lockstep
    from paper_1806_09819_gb300 import leea
    prm = dict(CONFIG_SMALL["prm"], eval_path=leea.EVAL_SMALL)
    _lockstep(gpu, oracle_mod, CONFIG_SMALL["dims"], CONFIG_SMALL["pop"], CONFIG_SMALL["batch"], prm, u8=False)
    _lockstep(gpu, oracle_mod, [784, 16, 10], 5, 3, dict(sigma=0.05, xo_op=1, eval_path=leea.EVAL_SMALL), u8=False)
