"""The reference arm of bench.py (the oracle on the host cores) follows the
native arm's configuration: its JSON line carries the same metric and the
contract's keys, and configurations it does not cover say so."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra) -> dict:
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *extra],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_reference_arm_small_configuration():
    sys.path.insert(0, ROOT)
    import bench
    line = _run("--config", "small", "--steps", "3", "--warmup", "3")
    assert line["impl"] == "reference" and line["metric"] == bench.SMALL_METRIC
    assert line["unit"] == "generations/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "generations/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "all 32 children" in line["cpu_baseline"]["sample"] or "32 of 32" in line["cpu_baseline"]["sample"]


def test_reference_arm_names_what_it_does_not_cover():
    line = _run("--config", "batching", "--steps", "3", "--warmup", "3")
    assert line["impl"] == "reference" and "batching" in line["unavailable"]


def test_oracle_pool_generation_equals_the_serial_oracle(oracle_mod):
    # The oracle spread over worker processes computes exactly what one
    # process computes: the same FP64 code on the same children.
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_1806_09819_gb300 import synthetic
    dims, pop, batch = [40, 16, 10], 30, 12
    params = dict(bench.PARAMS, alpha=0.5)
    c = oracle_mod.num_params(dims)
    parents = synthetic.random_population(pop, c, seed=8, scale=0.2).astype(np.float64)
    f_adj = np.random.default_rng(9).normal(-2.3, 0.1, size=pop)
    rng = np.random.default_rng(10)
    x = rng.uniform(0, 1, size=(batch, dims[0]))
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    pool = bench.OraclePool(parents, dims, params, x, y, workers=2)
    try:
        secs = pool.generation(f_adj, gen=5, seed=3, chunk=4)
    finally:
        pool.close()
    assert secs > 0
    prm = oracle_mod.Params(**params)
    order = oracle_mod.rank(f_adj)
    p1, p2, kind, f_inh = oracle_mod.select(prm, f_adj, order, 3, 5)
    kids = oracle_mod.breed(prm, dims, 3, 5, parents, p1, p2, kind)
    f, _ = oracle_mod.evaluate(kids, dims, x, y)
    want = oracle_mod.inherit(float(prm.alpha), f_inh, f, first=False)
    np.testing.assert_array_equal(pool.last_f_adj, want)
