"""Experiment harness of the paper's Section 4 on synthetic data.

The paper studies its method on MNIST with the network of Section 4.1 (2x2
max-pooling, 196-256-128-64-10) and repeats every setting with 15 seeds,
comparing settings by one-sided Mann-Whitney U tests.  This module runs the
same protocol through the library on the synthetic 28x28 stand-in
(``synthetic.py``): 45k training / 5k validation images, a fresh training
batch per generation, the validation accuracy of the individual with the
highest adjusted fitness at the end.

Experiments (settings as in Section 4; ``scale`` < 1 shrinks populations and
generation counts for quick runs):

* ``batch-alpha``        Section 4.2: population size x inheritance alpha x batch size
* ``selective-pressure`` Section 4.3: truncation proportion rho at two batch and population sizes
* ``crossover-sigma``    Section 4.4: uniform / arithmetic crossover x p_C x constant,
                         decaying or self-adaptive mutation strength
* ``large``              Section 4.5: lambda = 2000, batch 1024, p_C = 0.75

    python -m paper_1806_09819_gb300.experiments --exp selective-pressure --seeds 15 --out results.json
"""
from __future__ import annotations

import argparse
import itertools
import json
import time

import numpy as np

PAPER_DIMS = [196, 256, 128, 64, 10]
# Section 4's defaults (p_M = 1 - p_E - p_C; every gene mutated; Glorot-uniform init).
DEFAULTS = dict(xo_op=0, p_e=0.05, p_c=0.5, sigma=0.001, rho=0.5, alpha=1.0, mut_rate=1.0, init=1, n_elite=-1)
DEFAULT_POP, DEFAULT_BATCH = 1000, 512
SAMPLE_BUDGET = 2_000_000  # training samples seen per run: generations = budget / batch (small batches run longer)
MIN_GENERATIONS = 200


def _setting(pop=DEFAULT_POP, batch=DEFAULT_BATCH, **prm) -> dict:
    p = dict(DEFAULTS)
    p.update(prm)
    return {"pop": int(pop), "batch": int(batch), "params": p}


def settings(name: str) -> list[dict]:
    """The grid of one experiment (the paper's values where it states them)."""
    if name == "batch-alpha":
        return [_setting(pop=lam, batch=b, alpha=a)
                for lam, a, b in itertools.product((250, 1000), (0.0, 0.5, 1.0), (32, 128, 512))]
    if name == "selective-pressure":
        return [_setting(pop=lam, batch=b, rho=r)
                for (lam, b), r in itertools.product(((250, 32), (1000, 512)), (0.1, 0.2, 0.5, 1.0))]
    if name == "crossover-sigma":
        out = []
        for xo, pc, ctl in itertools.product((0, 1), (0.0, 0.25, 0.5, 0.75), (0, 1, 2)):
            extra = {1: dict(sigma_ctl=1, sigma_k=10.0), 2: dict(sigma_ctl=2, tau=0.1)}.get(ctl, {})
            out.append(_setting(xo_op=xo, p_c=pc, **extra))
        return out
    if name == "large":
        return [_setting(pop=2000, batch=1024, p_c=0.75)]
    raise ValueError(f"unknown experiment {name!r}")


def scaled(s: dict, scale: float) -> dict:
    """A smaller copy of a setting (population and sample budget times scale)."""
    out = json.loads(json.dumps(s))
    out["pop"] = max(20, int(round(s["pop"] * scale)))
    out["generations"] = max(int(MIN_GENERATIONS * scale), int(SAMPLE_BUDGET * scale / s["batch"]))
    return out


def _average_ranks(v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Ranks 1..n of v with ties given their average rank, and the sizes of the tie groups."""
    order = np.argsort(v, kind="stable")
    s = v[order]
    ranks = np.empty(len(v), dtype=np.float64)
    ties = []
    i = 0
    while i < len(s):
        j = i
        while j + 1 < len(s) and s[j + 1] == s[i]:
            j += 1
        ranks[order[i:j + 1]] = 0.5 * (i + j) + 1.0
        ties.append(j - i + 1)
        i = j + 1
    return ranks, np.asarray(ties, dtype=np.float64)


def _u_null_counts(m: int, n: int) -> np.ndarray:
    """Number of arrangements of m x's among n y's with each value of U = #(x > y), u = 0..m n
    (no ties): N(m, n, u) = N(m - 1, n, u - n) + N(m, n - 1, u)."""
    prev = [np.ones(1, dtype=np.float64) for _ in range(n + 1)]  # m = 0: U = 0 for every n
    for i in range(1, m + 1):
        cur = [np.ones(1, dtype=np.float64)]  # n = 0: U = 0
        for j in range(1, n + 1):
            c = np.zeros(i * j + 1)
            a = prev[j]             # the largest value is an x: it beats all j y's
            c[j:j + len(a)] += a
            b = cur[j - 1]          # the largest value is a y
            c[:len(b)] += b
            cur.append(c)
        prev = cur
    return prev[n]


def mann_whitney_greater(a, b) -> float:
    """One-sided Mann-Whitney U test (Section 4 reports significance this way):
    p-value of 'a tends to be larger than b'.  U = R_a - n_a (n_a + 1) / 2 from
    average ranks; the exact null distribution when there are no ties and a
    sample has at most 8 values, else the normal approximation with the tie
    correction of the variance and a continuity correction of 1/2."""
    import math
    a, b = np.asarray(a, float), np.asarray(b, float)
    m, n = len(a), len(b)
    if m == 0 or n == 0:
        return float("nan")
    ranks, ties = _average_ranks(np.concatenate([a, b]))
    u = float(ranks[:m].sum() - m * (m + 1) / 2.0)
    if min(m, n) <= 8 and np.all(ties == 1):
        counts = _u_null_counts(m, n)
        return float(counts[int(round(u)):].sum() / counts.sum())
    tot = m + n
    var = m * n / 12.0 * ((tot + 1) - float(np.sum(ties ** 3 - ties)) / (tot * (tot - 1)))
    if var <= 0.0:
        return 1.0
    z = (u - m * n / 2.0 - 0.5) / math.sqrt(var)
    return float(0.5 * math.erfc(z / math.sqrt(2.0)))


class Data:
    """Synthetic training and validation images as pooled 8-bit levels on the device."""

    def __init__(self, device, n_train: int = 45000, n_val: int = 5000):
        import torch
        from . import leea, synthetic
        (x, y), _ = synthetic.dataset(n_train=n_train + n_val, n_test=1)
        lv = synthetic.to_levels(x)  # [n, 784]
        raw = torch.from_numpy(lv).to(device)
        pooled = torch.empty((raw.shape[0], 196), dtype=torch.uint8, device=device)
        leea.leea_maxpool2x2(raw.shape[0], 28, 28, raw, pooled)
        yt = torch.from_numpy(y).to(device)
        self.x_train, self.y_train = pooled[:n_train], yt[:n_train]
        self.x_val, self.y_val = pooled[n_train:], yt[n_train:]
        self.n_train = n_train


def run_one(s: dict, seed: int, data: Data, generations: int | None = None) -> dict:
    """One EA run of a setting; returns the final validation accuracy and fitness."""
    import torch
    from . import leea, synthetic
    pop, batch = s["pop"], s["batch"]
    gens = generations if generations is not None else s.get("generations", MIN_GENERATIONS)
    idx = synthetic.batch_indices(data.n_train, batch, gens + 1, seed=synthetic.BATCH_SEED + seed)
    idx_d = torch.from_numpy(idx.astype(np.int64)).to(data.x_train.device)
    st = leea.LeeaState(pop, PAPER_DIMS, leea.Params(**s["params"]), seed=seed)
    try:
        t0 = time.perf_counter()
        for g in range(gens + 1):  # the first call evaluates the initial population
            st.leea_generation_u8(data.x_train[idx_d[g]].contiguous(), data.y_train[idx_d[g]].contiguous())
        f_adj = st.leea_fitness()
        best = st.leea_best_params()
        secs = time.perf_counter() - t0
    finally:
        st.close()
    cp = leea.leea_padded_params(PAPER_DIMS)
    pd = torch.zeros((1, cp), dtype=torch.float32, device=data.x_val.device)
    pd[0, :best.size] = torch.from_numpy(best)
    n_val = data.y_val.shape[0]
    f = torch.empty(1, dtype=torch.float32, device=pd.device)
    cor = torch.empty(1, dtype=torch.int32, device=pd.device)
    leea.leea_evaluate_u8(1, PAPER_DIMS, pd, data.x_val, 255.0, data.y_val, n_val, 1.0, None, f, None, cor)
    torch.cuda.synchronize()
    return {"seed": seed, "val_accuracy": int(cor.item()) / n_val, "val_fitness": float(f.item()),
            "best_train_fitness": float(np.max(f_adj)), "generations": gens, "seconds": secs}


def run_experiment(name: str, seeds: int, scale: float = 1.0, device=None, log=print) -> dict:
    import torch
    device = device or torch.device("cuda", 0)
    data = Data(device)
    rows = []
    for s in settings(name):
        sc = scaled(s, scale)
        runs = [run_one(sc, 1000 + k, data) for k in range(seeds)]
        acc = [r["val_accuracy"] for r in runs]
        rows.append({"setting": sc, "runs": runs, "median_val_accuracy": float(np.median(acc))})
        log(f"{name}: pop {sc['pop']} batch {sc['batch']} {sc['params']} -> median val acc {np.median(acc):.4f}")
    # The best setting against every other (one-sided Mann-Whitney U, as the paper reports significance).
    best = max(range(len(rows)), key=lambda i: rows[i]["median_val_accuracy"])
    a = [r["val_accuracy"] for r in rows[best]["runs"]]
    for i, row in enumerate(rows):
        row["p_best_greater"] = None if i == best or seeds < 2 else mann_whitney_greater(
            a, [r["val_accuracy"] for r in row["runs"]])
    return {"experiment": name, "seeds": seeds, "scale": scale, "data": "synthetic 28x28 (45k train / 5k val)",
            "best_setting": best, "rows": rows}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--exp", required=True, choices=["batch-alpha", "selective-pressure", "crossover-sigma", "large"])
    ap.add_argument("--seeds", type=int, default=15)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    from . import build as B
    B.build()
    res = run_experiment(args.exp, args.seeds, args.scale)
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text)
    else:
        print(text)


if __name__ == "__main__":
    main()
