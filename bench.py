#!/usr/bin/env python3
"""Throughput of the LEEA hot path on GB300: generations/s (and network-samples/s)
of P = 1000 nets 784-112-10 (89,050 parameters) on batches of 100 synthetic
MNIST-shaped images, FP32, with the roofline fraction of the dominant kernel.

One step = one generation of Algorithm 1 through the C ABI (rank, select,
breed, evaluate).  The population (2 x 356 MB) is larger than L2, so no flush
is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--config plain|small|precision-bf16|precision-fp8|batching|surrogate|paper-net]

--config small measures the small configuration (P = 32 nets 784-32-10,
batch 16), which launch latency bounds: each generation is timed between CUDA
events with L2 flushed in between, and the line adds microseconds per
generation.  --config paper-net measures the paper's own network (Section
4.1: 2x2 max-pooling, 196-256-128-64-10) at its Section 4.5 setting (lambda =
2000, batch 1024) on the tensor cores.

--config precision-* measures the precision form instead (P = 4096 nets
784-112-10, batch 256, BF16 or FP8-e4m3 shadows of W1 with FP32 accumulation
and FP32 masters) and reports the shadow fitness against the FP64 evaluation
of the masters on a sample of the final population.  --config batching
measures the batching form: 64 independent runs (P in [50, 2000], h in
[16, 256], batch in [8, 512], log-uniform from a fixed seed; BF16 shadows)
advanced together, one CUDA graph per generation, tile shapes from the
autotuner; the value counts every run's generations.  --config surrogate
runs the surrogate form (population 2048 nets 784-112-10, 4 x 2047 recipes
per generation of which the best-scored 2047 are made, BF16 evaluation, MLP
pre-screen trained online) and the plain FP32 path on the same batches, and
reports both generation rates and synthetic-test accuracy curves, and the
time each needs to reach the accuracy both attain.

N > 1 (under torch.distributed.run) runs N independent replicas, one per GPU
(the generation's selection needs every parent, so a run does not shard);
the value is all replicas' generations over the slowest replica's time.
--impl reference times the FP64 oracle on the host cores for the plain, small
and paper-net configurations (a bounded sample of each generation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "generations/sec and network·samples/sec at P=1000, 89k MLP; % of roofline"
PAPER_METRIC = ("generations/sec and network·samples/sec, the paper's 92k-parameter network at lambda=2000, "
                "batch 1024; % of roofline")
SMALL_METRIC = "generations/sec and microseconds per generation at P=32, 784-32-10, batch 16; % of roofline"
POP, DIMS, BATCH = 1000, [784, 112, 10], 100
PARAMS = dict(xo_op=0, xo_gene_p=0.5, sel_op=0, rho=0.5, n_elite=1, p_c=0.5, sigma=0.005, mut_rate=0.1,
              alpha=1.0, init=0)
WORKLOAD = ("P=1000 MLPs 784-112-10 (89,050 params, FP32), batch 100 synthetic 28x28 images; uniform crossover "
            "p_C=0.5, truncation rho=0.5, elitism 1, mutation sigma=0.005 on 10% of genes, alpha=1")
PRECISION_WORKLOAD = ("P=4096 MLPs 784-112-10, batch 256 synthetic 28x28 images, {name} shadows of W1 (FP32 "
                      "accumulation, FP32 masters); operators as the plain workload")
PAPER_POP, PAPER_DIMS, PAPER_BATCH = 2000, [196, 256, 128, 64, 10], 1024
PAPER_PARAMS = dict(xo_op=0, xo_gene_p=0.5, sel_op=0, rho=0.5, n_elite=-1, p_e=0.05, p_c=0.75, sigma=0.001,
                    mut_rate=1.0, alpha=1.0, init=1)
PAPER_WORKLOAD = ("the paper's network (Section 4.1): 2x2 max-pool of 28x28 synthetic images, then 196-256-128-64-10 "
                  "(92,042 params, FP32); lambda=2000, batch 1024, uniform crossover p_C=0.75, p_E=0.05, "
                  "rho=0.5, sigma=0.001 on every gene, alpha=1 (Section 4.5); the max-pool runs in every step")
SMALL_POP, SMALL_DIMS, SMALL_BATCH = 32, [784, 32, 10], 16
SMALL_WORKLOAD = ("P=32 MLPs 784-32-10 (25,450 params, FP32), batch 16 synthetic 28x28 images as 8-bit levels; "
                  "operators as the plain workload")
CONFIGS = {"plain": dict(pop=1000, batch=100, precision=0),
           "small": dict(pop=SMALL_POP, batch=SMALL_BATCH, precision=0),
           "paper-net": dict(pop=PAPER_POP, batch=PAPER_BATCH, precision=0),
           "precision-bf16": dict(pop=4096, batch=256, precision=1),
           "precision-fp8": dict(pop=4096, batch=256, precision=2),
           "batching": dict(runs=64, pop=(50, 2000), hidden=(16, 256), batch=(8, 512), precision=1, seed=4242),
           "surrogate": dict(pop=2048, batch=100, precision=1, mult=4, n_probe=32)}
SURROGATE_WORKLOAD = ("surrogate form: population 2048 MLPs 784-112-10, 4 recipes per offspring slot (8,188 per "
                      "generation), the best-scored 2,047 made and evaluated (BF16 shadows) plus a 5% audit sample; "
                      "MLP 325-64-64-1 trained online; batch 100 synthetic images; plain EA: the same population, "
                      "operators and batches in FP32")
BATCHING_WORKLOAD = ("64 independent LEEA runs of 784-h-10 MLPs, P in [50,2000], h in [16,256] (multiple of 16), "
                     "batch in [8,512], log-uniform (seed 4242); BF16 shadows of W1, FP32 masters; operators as the "
                     "plain workload; one CUDA graph per generation, individuals per MMA from the autotuner")


def batching_specs(cfg: dict):
    """The batching workload's runs: (pop, hidden, batch, seed), log-uniform from a fixed seed."""
    import numpy as np
    rng = np.random.default_rng(cfg["seed"])

    def logu(lo, hi):
        return float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    out = []
    for r in range(cfg["runs"]):
        pop = int(round(logu(*cfg["pop"])))
        hidden = int(min(cfg["hidden"][1], max(cfg["hidden"][0], 16 * round(logu(*cfg["hidden"]) / 16))))
        batch = int(round(logu(*cfg["batch"])))
        out.append((pop, hidden, batch, 5000 + r))
    return out
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ_NOMINAL = 152, 128, 2070.0
STAGES = ("select", "breed", "evaluate")

# DRAM traffic per launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), valid only while the kernel source is unchanged.
TRAFFIC = {
    "breed": {"bytes_per_launch": 472.53e6, "src_sha": "3ba6876d0f989830", "capture": "P=1000 plain workload"},
    "evaluate": {"bytes_per_launch": 368.68e6, "src_sha": "921b0e7934e40403", "capture": "P=1000 plain workload"},
    "breed_evaluate": {"bytes_per_launch": 738.19e6, "src_sha": "23e25d83744d9797", "capture": "P=1000 plain workload"},
    # eval_mlp_tc_kernel alone (each individual's weight pieces read once from
    # DRAM, the other tiles from L2); the stage also splits the weights
    "evaluate_paper_net": {"bytes_per_launch": 869.79e6, "src_sha": "407558790a9f32f1",
                           "capture": "paper-net workload, eval_mlp_tc_kernel"},
}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), float(m.get("sm_max_mhz", SM_MAX_MHZ_NOMINAL)), "measured"
    except Exception:
        return 6800.0, SM_MAX_MHZ_NOMINAL, "fallback"


def _tensor_peak() -> tuple[float, str]:
    """Dense FP16/BF16 tensor peak (TFLOP/s) for a kernel timed inside a long step."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["bf16_tflops_sustained"]), "measured (cuBLAS BF16, sustained; FP16 runs at the BF16 rate)"
    except Exception:
        return 1700.0, "fallback (BF16 sustained; FP16 runs at the BF16 rate)"


def _src_sha(name: str) -> str:
    p = os.path.join(ROOT, "paper_1806_09819_gb300", "csrc", name)
    with open(p, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


# --------------------------------------------------------------------------------
# distributed plumbing (replicas only)
# --------------------------------------------------------------------------------
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(world: int, use_cuda: bool):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def max_over_ranks(value: float, dist, device=None) -> float:
    """Max of a host float over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


PROFILE_EVERY = 8  # generations per profiled one inside the timed region


def kernels_per_generation(pop: int, batch: int, precision: int, fused: bool = False, x16: bool = False) -> dict:
    """Kernel launches per stage of one state-object generation: ranking and
    selection run as one kernel below 512 nets and as two above (plus the
    kernel that stages the batch as operand tiles for the tensor-core
    evaluations of 8-bit inputs, x16); breeding and evaluation are one fused kernel on the
    8-bit FP32 path, else two; the shadow evaluation adds a combining kernel
    when the batch spans several 128-sample tiles."""
    sel = (2 if pop >= 512 else 1) + (1 if x16 else 0)
    if fused:
        return {"select": sel, "breed_evaluate": 1}
    return {"select": sel, "breed": 1, "evaluate": 1 + (1 if precision > 0 and batch > 128 else 0)}


def job_rate(world: int, units_per_rank: float, ms_local: float, dist, device=None):
    """(slowest rank's ms, whole-job units per second): every rank processed
    units_per_rank units; the job took as long as its slowest rank."""
    ms_max = max_over_ranks(ms_local, dist, device)
    return ms_max, world * units_per_rank / (ms_max / 1000.0)


def barrier(dist, device=None):
    if dist is None:
        return
    import torch
    t = torch.zeros(1, device=device)
    dist.all_reduce(t)


# --------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self):
        return len(self.lines)

    def stop(self, since: int = 0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l.split(",") for l in self.lines[max(0, since - 1):] if l.count(",") >= 6]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except ValueError:
                continue
            for name, v in zip(names, r[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_id_for(dev: int) -> str | None:
    try:
        import torch
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        return None


# --------------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# --------------------------------------------------------------------------------
def oracle_step_sample(parents64, f_adj64, x64, y, n_children: int, gen: int, seed: int = 0) -> float:
    """Rank + select all P children, then breed and evaluate `n_children` of
    them (strided over elite, crossover and mutation children) in this
    process; returns the CPU seconds taken."""
    import numpy as np
    import oracle
    prm = oracle.Params(**PARAMS)
    t0 = time.perf_counter()
    order = oracle.rank(f_adj64)
    p1, p2, kind, f_inh = oracle.select(prm, f_adj64, order, seed, gen)
    rows = np.linspace(0, POP - 1, n_children).round().astype(int)
    kids = np.concatenate([oracle.breed(prm, DIMS, seed, gen, parents64, p1, p2, kind, j0=int(j), j1=int(j) + 1)
                           for j in rows])
    f, _ = oracle.evaluate(kids, DIMS, x64, y)
    oracle.inherit(float(prm.alpha), f_inh[rows], f, first=False)
    return time.perf_counter() - t0


# The oracle on every host core: worker processes (started with spawn) each
# breed and evaluate ranges of children with the unchanged oracle; the parents
# sit in one shared-memory block, the minibatch and the operators are sent once.
_ORACLE_POOL_STATE: dict = {}


def _oracle_worker_init(shm_name, shape, dims, params, x64, y):
    import numpy as np
    from multiprocessing import shared_memory
    import oracle
    oracle.build()
    # The creating process owns the block (and unlinks it); workers share its
    # resource tracker, so mapping the block here registers nothing new.
    shm = shared_memory.SharedMemory(name=shm_name)
    _ORACLE_POOL_STATE.update(shm=shm, parents=np.ndarray(shape, dtype=np.float64, buffer=shm.buf), dims=dims,
                              prm=oracle.Params(**params), x=x64, y=y)


def _oracle_worker_task(task):
    import oracle
    j0, j1, seed, gen, p1, p2, kind = task
    st = _ORACLE_POOL_STATE
    kids = oracle.breed(st["prm"], st["dims"], seed, gen, st["parents"], p1, p2, kind, j0=j0, j1=j1)
    f, _ = oracle.evaluate(kids, st["dims"], st["x"], st["y"])
    return j0, f


class OraclePool:
    """Whole generations of the oracle spread over `workers` processes."""

    def __init__(self, parents64, dims, params: dict, x64, y, workers: int | None = None):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import numpy as np
        self.workers = workers or (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
        self.dims, self.params = list(dims), dict(params)
        self.shm = shared_memory.SharedMemory(create=True, size=parents64.nbytes)
        self.parents = np.ndarray(parents64.shape, dtype=np.float64, buffer=self.shm.buf)
        self.parents[:] = parents64
        self.pool = mp.get_context("spawn").Pool(
            self.workers, initializer=_oracle_worker_init,
            initargs=(self.shm.name, parents64.shape, self.dims, self.params, x64, y))

    def generation(self, f_adj64, gen: int, seed: int = 0, chunk: int = 4, stride: int = 1) -> float:
        """Rank + select in this process, then breed + evaluate every child
        (every `stride`-th child when stride > 1: a bounded sample) on the
        workers (tasks of `chunk` children, handed out as workers free up);
        returns the wall-clock seconds of the generation."""
        import numpy as np
        import oracle
        prm = oracle.Params(**self.params)
        pop = len(f_adj64)
        t0 = time.perf_counter()
        order = oracle.rank(f_adj64)
        p1, p2, kind, f_inh = oracle.select(prm, f_adj64, order, seed, gen)
        if stride > 1:  # the sample: single-child tasks of every stride-th child
            tasks = [(j, j + 1, seed, gen, p1, p2, kind) for j in range(0, pop, stride)]
        else:
            tasks = [(j, min(pop, j + chunk), seed, gen, p1, p2, kind) for j in range(0, pop, chunk)]
        f = np.full(pop, np.nan)
        for j0, fj in self.pool.imap_unordered(_oracle_worker_task, tasks):
            f[j0:j0 + len(fj)] = fj
        if stride == 1:
            self.last_f_adj = oracle.inherit(float(prm.alpha), f_inh, f, first=False)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


def oracle_inputs(parents=None, f_adj=None):
    import numpy as np
    import oracle
    from paper_1806_09819_gb300 import synthetic
    oracle.build()
    c = oracle.num_params(DIMS)
    if parents is None:
        parents = synthetic.random_population(POP, c, seed=1, scale=0.05)
    if f_adj is None:
        f_adj = np.random.default_rng(2).normal(-2.3, 0.05, size=POP).astype(np.float32)
    x, y = synthetic.make_split(BATCH, seed=4)
    return parents.astype(np.float64), f_adj.astype(np.float64), x.astype(np.float64), y


def cpu_baseline(parents=None, f_adj=None, generations: int = 2) -> dict:
    """The oracle (unchanged, FP64) on every host core: whole generations of
    the benchmark workload, the workers started outside the timing."""
    parents64, f_adj64, x64, y = oracle_inputs(parents, f_adj)
    pool = OraclePool(parents64, DIMS, PARAMS, x64, y)
    try:
        pool.generation(f_adj64, gen=1)  # workers load the oracle
        secs = [pool.generation(f_adj64, gen=2 + g) for g in range(generations)]
    finally:
        pool.close()
    s = min(secs)
    return {"value": 1.0 / s, "unit": "generations/s", "cores": pool.workers, "kind": "oracle",
            "sample": f"whole generations ({POP} children bred and evaluated, batch {BATCH}) of the unchanged FP64 "
                      f"oracle, children spread over {pool.workers} worker processes; best of {generations}",
            "seconds": s, "network_samples_per_sec": POP * BATCH / s}


def cpu_baseline_fp32(parents=None, f_adj=None, generations: int = 3) -> dict:
    """The FP32 multi-core variant of the oracle (oracle/leea_cpu_fp32.c,
    OpenMP over children and individuals): whole generations."""
    import oracle
    parents64, f_adj64, x64, y = oracle_inputs(parents, f_adj)
    prm = oracle.Params(**PARAMS)
    p32, f32, x32 = parents64.astype("float32"), f_adj64.astype("float32"), x64.astype("float32")
    oracle.cpu32_generation(prm, DIMS, 0, 1, p32, f32, x32, y)  # warm-up (pages, threads)
    secs, threads = [], 1
    for g in range(generations):
        t0 = time.perf_counter()
        _, _, _, _, threads = oracle.cpu32_generation(prm, DIMS, 0, 2 + g, p32, f32, x32, y)
        secs.append(time.perf_counter() - t0)
    s = min(secs)
    return {"value": 1.0 / s, "unit": "generations/s", "cores": threads, "kind": "fp32 OpenMP variant of the oracle",
            "sample": f"whole generations ({POP} children, batch {BATCH}) in FP32 on {threads} threads; "
                      f"best of {generations}", "seconds": s, "network_samples_per_sec": POP * BATCH / s}


def precision_report(st, levels, y, precision: int, n: int = 64) -> dict:
    """Shadow fitness of the last generation vs the oracle's FP64 evaluation of the
    FP32 masters on the same batch, for n individuals spread over the population:
    loss error relative to max(|f|, 1e-2), Spearman rank correlation and top-10%
    overlap (reported, not pinned: a converged population's losses differ by less
    than FP32 resolves), and the error against the oracle's evaluation of the
    same shadows' values."""
    import numpy as np
    import oracle
    from scipy import stats
    oracle.build()
    f_gpu = st.leea_raw_fitness()
    popv = st.leea_get_population()
    rows = np.linspace(0, len(f_gpu) - 1, n).round().astype(int)
    x64 = levels.astype(np.float64) / 255.0
    f64, _ = oracle.evaluate(popv[rows].astype(np.float64), DIMS, x64, y)
    # the same individuals with their shadows' values (the library's own scale exponents)
    _, scale_exp, _ = st.leea_get_shadow(precision)
    fq, _ = oracle.evaluate_shadow(popv[rows].astype(np.float64), DIMS, precision, scale_exp[rows], x64, y)
    g = f_gpu[rows].astype(np.float64)
    err = np.abs(g - f64)
    rel = err / np.maximum(np.abs(f64), 1e-2)  # relative, with the FP32 rule's floor for losses near 0
    k = max(1, n // 10)
    top = len(set(np.argsort(-g)[:k].tolist()) & set(np.argsort(-f64)[:k].tolist())) / k
    return {"individuals": int(n), "max_rel_loss_error": float(rel.max()), "mean_rel_loss_error": float(rel.mean()),
            "max_abs_loss_error": float(err.max()), "mean_loss_fp64": float(-f64.mean()),
            "loss_spread_fp64": float(f64.std()), "spearman": float(stats.spearmanr(g, f64).statistic),
            "max_rel_error_vs_quantized_oracle": float((np.abs(g - fq) / np.maximum(np.abs(fq), 1e-2)).max()),
            "top10_overlap": float(top)}


# --------------------------------------------------------------------------------
# arms
# --------------------------------------------------------------------------------
def run_reference(args, rank: int, world: int):
    """The oracle as the reference arm, on the native arm's configuration: each
    step a bounded sample of one generation (the whole generation for the
    small configuration)."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1806_09819_gb300 import synthetic
    oracle.build()
    if args.config == "plain":
        parents64, f_adj64, x64, y = oracle_inputs()
        pool = OraclePool(parents64, DIMS, PARAMS, x64, y)
        pool.generation(f_adj64, gen=1)  # the workers load the oracle outside the timing
        try:
            # Whole generations while the K + W steps fit about two minutes;
            # else each step a bounded sample (every stride-th child) sized so
            # that they do.
            t_full = pool.generation(f_adj64, gen=2)
            budget = 120.0
            stride = max(1, math.ceil((args.steps + args.warmup) * t_full / budget))
            n_children = len(range(0, POP, stride))
            for w in range(args.warmup):
                pool.generation(f_adj64, gen=3 + w, stride=stride)
            secs = [pool.generation(f_adj64, gen=100 + k, stride=stride) for k in range(args.steps)]
        finally:
            pool.close()
        total = sum(secs)
        gen_per_s = args.steps * (n_children / POP) / total
        sample = (f"whole generations: rank+select of {POP} nets, breed+evaluate of all {POP} children (batch "
                  f"{BATCH}) with the unchanged FP64 oracle over {pool.workers} worker processes" if stride == 1 else
                  f"per step rank+select of {POP} nets and breed+evaluate of {n_children} of the {POP} children "
                  f"(every {stride}th; batch {BATCH}) with the unchanged FP64 oracle over {pool.workers} worker "
                  f"processes; value = ({n_children}/{POP}) generations per measured step (a whole generation "
                  f"took {t_full:.2f} s, too long for {args.steps + args.warmup} steps in a few minutes)")
        line = {"impl": "reference", "metric": METRIC, "value": gen_per_s, "unit": "generations/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "host CPU run"},
                "cpu_baseline": {"value": gen_per_s, "unit": "generations/s", "cores": pool.workers, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": gen_per_s, "unit": "generations/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0},
                "network_samples_per_sec": gen_per_s * POP * BATCH}
        print(json.dumps(line), flush=True)
        return
    elif args.config == "small":
        pop, batch, workload, metric = SMALL_POP, SMALL_BATCH, SMALL_WORKLOAD, SMALL_METRIC
        parents = synthetic.random_population(pop, oracle.num_params(SMALL_DIMS), seed=1, scale=0.05)
        f_adj = np.random.default_rng(2).normal(-2.3, 0.05, size=pop).astype(np.float32)
        x, y = synthetic.make_split(batch, seed=4)
        x64 = synthetic.to_levels(x).astype(np.float64) / 255.0

        def step(n, gen):
            return small_cpu_baseline(parents, f_adj, x64, y)["seconds"]
    elif args.config == "paper-net":
        pop, batch, workload, metric = PAPER_POP, PAPER_BATCH, PAPER_WORKLOAD, PAPER_METRIC
        par64 = synthetic.random_population(pop, oracle.num_params(PAPER_DIMS), seed=1, scale=0.05).astype(np.float64)
        f64 = np.random.default_rng(2).normal(-2.3, 0.05, size=pop)
        x, y = synthetic.make_split(batch, seed=4)
        pooled64 = oracle.maxpool2x2(synthetic.to_levels(x).astype(np.float64), 28, 28) / 255.0

        def step(n, gen):
            return paper_step_sample(par64, f64, pooled64, y, n, gen)
    else:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the plain, small and paper-net "
                                                              f"configurations, not {args.config}"}), flush=True)
        return
    per_step_budget = 60.0 / max(1, args.steps + args.warmup)
    if args.config == "small":
        n_children = pop  # a whole generation per step
    else:
        probe = step(2, 1) / 2.0
        n_children = int(max(1, min(pop, round(per_step_budget / max(probe, 1e-6)))))
    for w in range(args.warmup):
        step(n_children, 2 + w)
    total = 0.0
    for k in range(args.steps):
        total += step(n_children, 100 + k)
    gen_per_s = args.steps * (n_children / pop) / total
    sample = (f"per step: rank+select of {pop} nets, breed+evaluate of {n_children} of {pop} children, "
              f"batch {batch}; value = steps*({n_children}/{pop}) / seconds")
    line = {"impl": "reference", "metric": metric, "value": gen_per_s, "unit": "generations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * pop / n_children * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "l2": "host CPU run"},
            "cpu_baseline": {"value": gen_per_s, "unit": "generations/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gen_per_s, "unit": "generations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "network_samples_per_sec": gen_per_s * pop * batch}
    print(json.dumps(line), flush=True)


def paper_step_sample(par64, f64, pooled64, y, n_children: int, gen: int) -> float:
    """The oracle on one generation of the paper's network: rank + select all
    lambda children, breed and evaluate n_children of them (strided); returns
    the CPU seconds taken."""
    import numpy as np
    import oracle
    prm = oracle.Params(**PAPER_PARAMS)
    t0 = time.perf_counter()
    order = oracle.rank(f64)
    p1, p2, kind, f_inh = oracle.select(prm, f64, order, 0, gen)
    rows = np.linspace(0, PAPER_POP - 1, n_children).round().astype(int)
    kids = np.concatenate([oracle.breed(prm, PAPER_DIMS, 0, gen, par64, p1, p2, kind, j0=int(j), j1=int(j) + 1)
                           for j in rows])
    f, _ = oracle.evaluate(kids, PAPER_DIMS, pooled64, y)
    oracle.inherit(float(prm.alpha), f_inh[rows], f, first=False)
    return time.perf_counter() - t0


def paper_cpu_baseline(parents, f_adj, pooled64, y, n_children: int) -> dict:
    """The oracle on one generation of the paper's network (paper_step_sample)."""
    import numpy as np
    import oracle
    oracle.build()
    secs = paper_step_sample(parents.astype(np.float64), f_adj.astype(np.float64), pooled64, y, n_children, 1)
    gen_per_s = (n_children / PAPER_POP) / secs
    return {"value": gen_per_s, "unit": "generations/s", "cores": 1, "kind": "oracle",
            "sample": f"one generation's rank+select over all {PAPER_POP} nets, breed+evaluate of {n_children} of "
                      f"the {PAPER_POP} children (strided), batch {PAPER_BATCH}; value = ({n_children}/{PAPER_POP}) "
                      "/ seconds", "seconds": secs, "network_samples_per_sec": gen_per_s * PAPER_POP * PAPER_BATCH}


def run_paper_net(args, rank: int, world: int, local_rank: int):
    """The paper's own network and its large-population setting (Sections 4.1, 4.5)."""
    import numpy as np
    import torch
    from paper_1806_09819_gb300 import build as B
    from paper_1806_09819_gb300 import leea, synthetic

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = dist_init(world, True)
    if rank == 0 or world == 1:
        B.build()
    barrier(dist, dev)
    B.build()
    leea.load_library()
    steps, warmup = args.steps, args.warmup
    pop, batch, dims = PAPER_POP, PAPER_BATCH, PAPER_DIMS
    (xtr, ytr), _ = synthetic.dataset(n_train=60000, n_test=1)
    xtr = synthetic.to_levels(xtr)  # [60000, 784] 8-bit levels of 28x28 images
    n_batches = warmup + 1 + steps
    idx = synthetic.batch_indices(len(ytr), batch, n_batches, seed=synthetic.BATCH_SEED + rank)
    xs = torch.from_numpy(xtr[idx]).to(dev)  # raw images, resident in HBM
    ys = torch.from_numpy(ytr[idx]).to(dev)
    pooled = torch.empty((batch, 196), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(st, xk, yk):
        leea.leea_maxpool2x2(batch, 28, 28, xk, pooled, stream=stream)
        st.leea_generation_u8(pooled, yk, 255.0)

    st = leea.LeeaState(pop, dims, leea.Params(**PAPER_PARAMS, eval_path=args.eval_path), seed=1000 + rank,
                        stream=stream)
    for k in range(warmup + 1):  # the first call evaluates the initial population
        step(st, xs[k], ys[k])
    torch.cuda.synchronize(dev)
    st.leea_profile_enable(True)
    st.leea_profile_read()
    clocks = ClockSampler(_gpu_id_for(local_rank))
    clocks.start()
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    mark = clocks.mark()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(steps):
        st.leea_profile_enable(k % PROFILE_EVERY == 0)
        step(st, xs[warmup + 1 + k], ys[warmup + 1 + k])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    clk = clocks.stop(mark)
    ms = ev0.elapsed_time(ev1)
    prof = st.leea_profile_read()
    st.leea_profile_enable(False)
    ms_max, gen_per_s = job_rate(world, steps, ms, dist, dev)

    # end to end: the raw batch from pinned host memory, pooled, a generation, the fitness read back
    e2e_steps = max(10, min(steps, 200))
    sel = idx[np.arange(e2e_steps) % n_batches]
    xh = torch.from_numpy(xtr[sel]).pin_memory()
    yh = torch.from_numpy(ytr[sel]).pin_memory()
    xd = torch.empty((batch, 784), dtype=torch.uint8, device=dev)
    yd = torch.empty(batch, dtype=torch.int32, device=dev)
    f_host = None
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        xd.copy_(xh[k], non_blocking=True)
        yd.copy_(yh[k], non_blocking=True)
        step(st, xd, yd)
        f_host = st.leea_fitness()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e = {"value": world * e2e_steps / t_e2e, "unit": "generations/s",
           "h2d_bytes_per_step": int(xh[0].numel() + yh[0].numel() * 4), "d2h_bytes_per_step": int(f_host.nbytes),
           "steps": e2e_steps}

    hbm_peak, sm_max_mhz, peak_src = _peaks()
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    n_e, n_c, n_m, _ = leea.leea_counts(pop, leea.Params(**PAPER_PARAMS))
    c = leea.leea_layout_num_params(dims)
    macs = sum(dims[l] * dims[l + 1] for l in range(len(dims) - 1))
    tensor = args.eval_path != leea.EVAL_SIMT  # 8-bit inputs, three hidden layers: tcgen05 FP16 pieces
    t_peak, t_src = _tensor_peak()
    work = {"breed": ("hbm", 4.0 * c * (2 * n_e + 3 * n_c + 2 * n_m) / 1e9, "GB/s", hbm_peak),
            "evaluate": ("tensor" if tensor else "alu", 2.0 * pop * batch * macs / 1e12, "TFLOP/s",
                         t_peak if tensor else fp32_peak),
            "select": ("latency", None, None, None)}
    kernels = {}
    for name in STAGES:
        tot_ms, launches = prof[name]
        per = tot_ms / max(1, launches)
        bound, units, unit, peak = work[name]
        entry = {"launches": launches, "ms_per_launch": per,
                 "share": tot_ms / max(1e-12, sum(v[0] for v in prof.values()))}
        if units is not None:
            ach = units / (per / 1000.0)
            entry.update({"bound": bound, "achieved": ach, "unit": unit, "peak": peak, "frac": ach / peak})
        kernels[name] = entry
    kd = kernels["evaluate"]
    if tensor:  # MMA work issued: 128-sample tiles, K padded to 16, 2 pieces (layer 1) or 3 products (layers 2-3)
        tiles = (batch + 127) // 128
        k16 = [(d + 15) // 16 * 16 for d in dims]
        issued = sum((2 if l == 0 else 3) * 2.0 * 128 * k16[l] * dims[l + 1] for l in range(3))
        kd["tensor_tflops_issued"] = pop * tiles * issued / 1e12 / (kd["ms_per_launch"] / 1000.0)
    tr = TRAFFIC["evaluate_paper_net"]
    traffic = (tr["bytes_per_launch"] if tensor and (pop, batch) == (PAPER_POP, PAPER_BATCH)
               and tr["src_sha"] == _src_sha("leea_eval_mlp_tc.cu") else None)
    roofline = {"kernel": "evaluate", "bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
                "unit": "TFLOP/s", "frac": kd["frac"], "traffic": traffic,
                "traffic_kernel": "eval_mlp_tc_kernel (DRAM bytes of the main kernel; not the weight split)",
                "peak_source": t_src if tensor else
                "derived: FP32 FFMA, 152 SM x 128 lanes x 2 x max SM clock (no measured FP32 peak)"}
    line = {"metric": PAPER_METRIC, "value": gen_per_s, "unit": "generations/s", "n_gpus": world, "steps": steps, "warmup": warmup,
            "ms_per_step": ms_max / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": PAPER_WORKLOAD, "parallelism": "replicas" if world > 1 else "single GPU",
                       "kernel_timing": f"CUDA events around each kernel of every {PROFILE_EVERY}th generation "
                                        "inside the timed region",
                       "input": "uint8 levels k of 28x28 images, x = k/255, pooled on the GPU each step",
                       "eval_kernel": ("tcgen05, FP16 operand pieces (FP32-class), FP32 accumulation in TMEM; layer 4 "
                                       "and the loss in FP32" if tensor else
                                       "CUDA-core FP32, layers chained in shared memory (64-sample tiles)"),
                       "l2": f"inputs larger than L2 (2 population buffers of "
                             f"{pop * leea.leea_padded_params(dims) * 4 / 1e6:.0f} MB), no flush"},
            "network_samples_per_sec": gen_per_s * pop * batch, "e2e": e2e,
            # + the max-pool; the tensor-core evaluation is four launches: the weight split, the level
            # tiles, the kernel and the FP32 recomputation of marked individuals
            "gpu_launches": int(steps * (1 + (3 if tensor else 0) + sum(kernels_per_generation(pop, batch, 0).values()))),
            "roofline": roofline, "kernels": kernels, "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        x_last = xtr[idx[warmup + steps]].astype(np.float64)
        import oracle
        oracle.build()
        pooled_h = oracle.maxpool2x2(x_last, 28, 28) / 255.0
        line["cpu_baseline"] = paper_cpu_baseline(st.leea_get_population(), st.leea_fitness(), pooled_h,
                                                  ytr[idx[warmup + steps]], n_children=40)
    st.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def small_cpu_baseline(parents, f_adj, x64, y) -> dict:
    """The oracle on one host core: one whole generation of the small workload
    (rank, select, breed and evaluate all P children, inheritance)."""
    import numpy as np
    import oracle
    oracle.build()
    prm = oracle.Params(**PARAMS)
    p64, f64 = parents.astype(np.float64), f_adj.astype(np.float64)
    t0 = time.perf_counter()
    order = oracle.rank(f64)
    p1, p2, kind, f_inh = oracle.select(prm, f64, order, 0, 1)
    kids = oracle.breed(prm, SMALL_DIMS, 0, 1, p64, p1, p2, kind)
    f, _ = oracle.evaluate(kids, SMALL_DIMS, x64, y)
    oracle.inherit(float(prm.alpha), f_inh, f, first=False)
    secs = time.perf_counter() - t0
    return {"value": 1.0 / secs, "unit": "generations/s", "cores": 1, "kind": "oracle",
            "sample": f"one whole generation: rank+select, breed and evaluate all {SMALL_POP} children, "
                      f"batch {SMALL_BATCH}", "seconds": secs}


def run_small(args, rank: int, world: int, local_rank: int):
    """The small configuration (P=32, 784-32-10, batch 16): launch latency, not
    bytes, bounds a generation, so each generation is timed on its own between
    CUDA events with L2 flushed in between (the population is 3 MB)."""
    import numpy as np
    import torch
    from paper_1806_09819_gb300 import build as B
    from paper_1806_09819_gb300 import leea, synthetic
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = dist_init(world, True)
    if rank == 0 or world == 1:
        B.build()
    barrier(dist, dev)
    B.build()
    leea.load_library()
    steps, warmup = args.steps, args.warmup
    pop, batch, dims = SMALL_POP, SMALL_BATCH, SMALL_DIMS
    (xtr, ytr), _ = synthetic.dataset(n_train=60000, n_test=1)
    xtr = synthetic.to_levels(xtr)
    n_batches = warmup + 1 + steps
    idx = synthetic.batch_indices(len(ytr), batch, n_batches, seed=synthetic.BATCH_SEED + rank)
    xs = torch.from_numpy(xtr[idx]).to(dev)
    ys = torch.from_numpy(ytr[idx]).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # larger than the 126 MB L2
    st = leea.LeeaState(pop, dims, leea.Params(**PARAMS, eval_path=args.eval_path), seed=1000 + rank, stream=stream)
    for k in range(warmup + 1):  # the first call evaluates the initial population
        if k == warmup:  # which kernels a breeding generation launches
            st.leea_profile_enable(True)
        st.leea_generation_u8(xs[k], ys[k], 255.0)
    stage_launches = {s: n for s, (_, n) in st.leea_profile_read().items()}
    st.leea_profile_enable(False)
    single_launch = stage_launches == {"select": 0, "breed": 1, "evaluate": 0}
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(_gpu_id_for(local_rank))
    clocks.start()
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    mark = clocks.mark()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 255)  # outside the timed pair: the next generation starts from DRAM
        evs[k][0].record(stream)
        st.leea_generation_u8(xs[warmup + 1 + k], ys[warmup + 1 + k], 255.0)
        evs[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    clk = clocks.stop(mark)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_max, gen_per_s = job_rate(world, steps, ms, dist, dev)
    # back to back, no flush: the steady state with the population in L2
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        st.leea_generation_u8(xs[warmup + 1 + k], ys[warmup + 1 + k], 255.0)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    us_b2b = e0.elapsed_time(e1) * 1000.0 / steps

    # end to end through the host-batch call: H2D of the batch, a generation, the fitness read back
    e2e_steps = max(10, min(steps, 500))
    sel = idx[np.arange(e2e_steps) % n_batches]
    xh = torch.from_numpy(xtr[sel]).pin_memory()  # the batches in pinned host memory
    yh = torch.from_numpy(ytr[sel]).pin_memory()
    f_host = None
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        st.leea_generation_u8_host(xh[k], yh[k], 255.0)
        f_host = st.leea_fitness()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e = {"value": world * e2e_steps / t_e2e, "unit": "generations/s",
           "h2d_bytes_per_step": int(xh[0].numel() + yh[0].numel() * 4), "d2h_bytes_per_step": int(f_host.nbytes),
           "steps": e2e_steps}

    hbm_peak, _, peak_src = _peaks()
    n_e, n_c, n_m, _ = leea.leea_counts(pop, leea.Params(**PARAMS))
    c = leea.leea_layout_num_params(dims)
    gen_bytes = 8.0 * c * (n_e + n_c + n_m) + 4.0 * c * pop  # breed (one read, one write per gene), evaluation
    us = ms_max * 1000.0 / steps
    roofline = {"kernel": "generation", "bound": "hbm", "achieved": gen_bytes / (us * 1e-6) / 1e9,
                "peak": hbm_peak, "unit": "GB/s", "frac": gen_bytes / (us * 1e-6) / 1e9 / hbm_peak,
                "traffic": None, "peak_source": f"{peak_src} (HBM copy)",
                "note": "launch-latency bound: a generation's algorithmic bytes over its whole time"}
    line = {"metric": SMALL_METRIC, "value": gen_per_s, "unit": "generations/s", "n_gpus": world, "steps": steps, "warmup": warmup,
            "ms_per_step": ms_max / steps, "us_per_generation": us, "us_per_generation_back_to_back": us_b2b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SMALL_WORKLOAD, "parallelism": "replicas" if world > 1 else "single GPU",
                       "timing": "CUDA events around each generation, L2 flushed (256 MB write) between "
                                 "generations outside the events; back to back: one event pair, no flush",
                       "input": "uint8 levels k, x = k/255",
                       "l2": "flushed between timed generations"},
            "network_samples_per_sec": gen_per_s * pop * batch, "e2e": e2e,
            "gpu_launches": int(steps * (1 if single_launch else sum(kernels_per_generation(
                pop, batch, 0, x16=args.eval_path in (0, 2)).values()))),
            "roofline": roofline, "clocks": clk}
    line["config"]["generation"] = ("one kernel: ranking, selection, breeding and evaluation (one CTA per child "
                                    "and 8 hidden units; layer 1 on m16n8k8 TF32 tiles, the levels exact, each "
                                    "weight as two TF32 pieces: 22-bit significands, exact products, FP32 "
                                    "accumulation)" if single_launch else "a chain of kernels")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        x64 = xtr[idx[warmup + steps]].astype(np.float64) / 255.0
        line["cpu_baseline"] = small_cpu_baseline(st.leea_get_population(), st.leea_fitness(), x64,
                                                  ytr[idx[warmup + steps]])
    st.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batching(args, rank: int, world: int, local_rank: int):
    """The batching form: every run's generations per second, one graph per generation."""
    import numpy as np
    import torch
    from paper_1806_09819_gb300 import autotune
    from paper_1806_09819_gb300 import build as B
    from paper_1806_09819_gb300 import leea, synthetic

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = dist_init(world, True)
    if rank == 0 or world == 1:
        B.build()
    barrier(dist, dev)
    B.build()
    leea.load_library()
    cfg = CONFIGS["batching"]
    steps, warmup = args.steps, args.warmup
    runs = batching_specs(cfg)
    if args.runs:  # profiling override: the first runs only
        runs = runs[:args.runs]
    specs = [leea.RunSpec(pop=p, hidden=h, batch=b, seed=s + 100 * rank) for p, h, b, s in runs]
    specs, _ = autotune.tune(specs, DIMS[0], DIMS[2], cfg["precision"])
    prm = leea.Params(**PARAMS, precision=cfg["precision"])
    stream = torch.cuda.current_stream(dev)
    m = leea.MultiRun(specs, DIMS[0], DIMS[2], prm, stream=stream)
    # a pool of packed minibatches (each run's batch drawn from the synthetic training set)
    (xtr, ytr), _ = synthetic.dataset(n_train=60000, n_test=1)
    lv = synthetic.to_levels(xtr)
    n_pool = 16
    rng = np.random.default_rng(synthetic.BATCH_SEED + rank)
    xs = np.empty((n_pool, m.total_rows, DIMS[0]), dtype=np.uint8)
    ys = np.empty((n_pool, m.total_rows), dtype=np.int32)
    for k in range(n_pool):
        for r, sp in enumerate(specs):
            idx = rng.choice(len(ytr), size=sp.batch, replace=False)
            xs[k, m.rows_slice(r)] = lv[idx]
            ys[k, m.rows_slice(r)] = ytr[idx]
    xd, yd = torch.from_numpy(xs).to(dev), torch.from_numpy(ys).to(dev)
    for k in range(warmup + 1):
        m.generation_u8(xd[k % n_pool], yd[k % n_pool])
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(_gpu_id_for(local_rank))
    clocks.start()
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    mark = clocks.mark()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(steps):
        m.generation_u8(xd[k % n_pool], yd[k % n_pool])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    clk = clocks.stop(mark)
    n_runs = len(specs)
    ms_max, gen_per_s = job_rate(world, n_runs * steps, ev0.elapsed_time(ev1), dist, dev)
    samples_per_gen = sum(sp.pop * sp.batch for sp in specs)

    # per-stage times: direct launches between events (same kernels as the graph)
    prof_steps = min(steps, 200)
    m.profile_enable(True)
    for k in range(prof_steps):
        m.generation_u8(xd[k % n_pool], yd[k % n_pool])
    prof = m.profile_read()
    m.profile_enable(False)
    eval_launches = m.eval_launches()

    # end to end: packed host minibatch in, packed fitness out
    e2e_steps = max(10, min(steps, 500))
    xh = torch.from_numpy(xs).pin_memory()
    yh = torch.from_numpy(ys).pin_memory()
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    f_host = None
    for k in range(e2e_steps):
        m.generation_u8_host(xh[k % n_pool], yh[k % n_pool])
        f_host = m.fitness()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e = {"value": world * n_runs * e2e_steps / t_e2e, "unit": "run-generations/s",
           "h2d_bytes_per_step": int(xs[0].nbytes + ys[0].nbytes), "d2h_bytes_per_step": int(f_host.nbytes),
           "steps": e2e_steps}

    hbm_peak, _, peak_src = _peaks()
    breed_b = evaluate_b = 0.0
    for sp in specs:
        dims = [DIMS[0], sp.hidden, DIMS[2]]
        c = leea.leea_layout_num_params(dims)
        n_e, n_c, n_m, _ = leea.leea_counts(sp.pop, leea.Params(**PARAMS))
        shadow = DIMS[0] * sp.hidden * 2
        breed_b += (8.0 * c + shadow) * (n_e + n_c + n_m)  # one read and one write per gene, the shadow written
        evaluate_b += (shadow + 4.0 * (c - DIMS[0] * sp.hidden)) * sp.pop
    work = {"breed": breed_b / 1e9, "evaluate": evaluate_b / 1e9}
    kernels = {}
    tot = sum(v[0] for v in prof.values())
    for name in STAGES:
        ms, launches = prof[name]
        per = ms / max(1, launches)
        entry = {"launches": launches, "ms_per_launch": per, "share": ms / max(1e-12, tot)}
        if name in work:
            ach = work[name] / (per / 1000.0)
            entry.update({"bound": "hbm", "achieved": ach, "unit": "GB/s", "peak": hbm_peak, "frac": ach / hbm_peak})
        kernels[name] = entry
    dom = max(("breed", "evaluate"), key=lambda n: prof[n][0])
    kd = kernels[dom]
    line = {"metric": "run-generations/sec of 64 uneven LEEA runs advanced together (batching form)",
            "value": gen_per_s, "unit": "run-generations/s", "n_gpus": world, "steps": steps, "warmup": warmup,
            "ms_per_step": ms_max / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (f32 accumulate)", "data": "synthetic",
            "config": {"workload": BATCHING_WORKLOAD, "parallelism": "replicas" if world > 1 else "single GPU",
                       "runs": [{"pop": sp.pop, "hidden": sp.hidden, "batch": sp.batch, "chunk": sp.chunk,
                                 "group": sp.group}
                                for sp in specs],
                       "l2": "inputs larger than L2 (populations of all runs, 2 buffers), no flush"},
            "network_samples_per_sec": gen_per_s / n_runs * samples_per_gen,
            "e2e": e2e, "gpu_launches": int(steps * (3 + eval_launches)),  # generation bump, select, breed, evaluation
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": kd["achieved"], "peak": kd["peak"],
                         "unit": "GB/s", "frac": kd["frac"], "traffic": None,
                         "peak_source": f"{peak_src} (HBM copy)"},
            "kernels": kernels, "clocks": clk}
    m.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_surrogate(args, rank: int, world: int, local_rank: int):
    """The surrogate form against the plain FP32 path: generations/s and test accuracy."""
    import numpy as np
    import torch
    from paper_1806_09819_gb300 import build as B
    from paper_1806_09819_gb300 import leea, synthetic

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = dist_init(world, True)
    if rank == 0 or world == 1:
        B.build()
    barrier(dist, dev)
    B.build()
    leea.load_library()
    cfg = CONFIGS["surrogate"]
    pop, batch = cfg["pop"], cfg["batch"]
    gens = args.steps
    every = max(1, gens // 12)
    (xtr, ytr), (xte, yte) = synthetic.dataset(n_train=60000, n_test=10000)
    lv_tr, lv_te = synthetic.to_levels(xtr), synthetic.to_levels(xte)
    idx = synthetic.batch_indices(len(ytr), batch, gens + 1, seed=synthetic.BATCH_SEED + rank)
    xs = torch.from_numpy(lv_tr[idx]).to(dev)
    ys = torch.from_numpy(ytr[idx]).to(dev)
    xt, yt = torch.from_numpy(lv_te).to(dev), torch.from_numpy(yte).to(dev)
    stream = torch.cuda.current_stream(dev)
    cp = leea.leea_padded_params(DIMS)

    def test_acc(params):
        pd = torch.zeros((1, cp), dtype=torch.float32, device=dev)
        pd[0, :params.size] = torch.from_numpy(params)
        f = torch.empty(1, dtype=torch.float32, device=dev)
        cor = torch.empty(1, dtype=torch.int32, device=dev)
        leea.leea_evaluate_u8(1, DIMS, pd, xt, 255.0, yt, len(yte), 1.0, None, f, None, cor, stream=stream)
        return float(cor.item()) / len(yte)

    def run(make, step, best):
        obj = make()
        ms, curve = 0.0, []
        step(obj, 0)  # evaluates the initial population
        for g in range(1, gens + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(obj, g)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            if g % every == 0 or g == gens:
                curve.append((g, ms, test_acc(best(obj))))
        return obj, curve

    prm_plain = leea.Params(**PARAMS)
    plain, curve_p = run(lambda: leea.LeeaState(pop, DIMS, prm_plain, seed=31 + rank, stream=stream),
                         lambda st, g: st.leea_generation_u8(xs[g], ys[g], 255.0), lambda st: st.leea_best_params())
    plain.close()
    sp = leea.SurrogateParams(mult=cfg["mult"], n_probe=cfg["n_probe"])
    probe = xte[:cfg["n_probe"]].astype(np.float32)
    prm_s = leea.Params(**PARAMS, precision=cfg["precision"])
    surr, curve_s = run(lambda: leea.SurrState(pop, DIMS, prm_s, sp, seed=31 + rank, probe=probe, stream=stream),
                        lambda st, g: st.generation_u8(xs[g], ys[g], 255.0), lambda st: st.best_params())
    rho, screened, loss = surr.stats()
    surr.profile_enable(True)
    for g in range(min(gens, 50)):
        surr.generation_u8(xs[g % (gens + 1)], ys[g % (gens + 1)], 255.0)
    prof, n_prof = surr.profile_read()
    surr.close()

    def time_to(curve, acc):
        for g, ms, a in curve:
            if a >= acc:
                return g, ms
        return None, None
    target = min(curve_p[-1][2], curve_s[-1][2])
    gp, tp = time_to(curve_p, target)
    gs, ts = time_to(curve_s, target)
    gen_s = gens / (curve_s[-1][1] / 1000.0)
    gen_p = gens / (curve_p[-1][1] / 1000.0)
    line = {"metric": "generations/sec of the surrogate form (population 2048, 8,188 offspring recipes per "
                      "generation, 784-112-10, batch 100, BF16) and its time-to-accuracy against plain FP32",
            "value": world * gen_s, "unit": "generations/s", "n_gpus": world, "steps": gens, "warmup": 0,
            "ms_per_step": curve_s[-1][1] / gens, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 eval, f32 surrogate", "data": "synthetic",
            "config": {"workload": SURROGATE_WORKLOAD, "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "populations larger than L2, no flush"},
            "plain_fp32": {"generations_per_sec": gen_p, "accuracy_curve": curve_p},
            "surrogate_bf16": {"generations_per_sec": gen_s, "accuracy_curve": curve_s,
                               "audit_spearman_mean_last_half": float(np.mean(rho[len(rho) // 2:])) if len(rho) else None,
                               "prescreen_generations": int(screened.sum()), "generations": int(len(screened)),
                               "stage_ms_per_generation": {k: v / max(1, n_prof) for k, v in prof.items()}},
            "time_to_accuracy": {"accuracy": target, "plain_generations": gp, "plain_ms": tp,
                                 "surrogate_generations": gs, "surrogate_ms": ts,
                                 "speedup": (tp / ts) if tp and ts else None},
            "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_native(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch
    from paper_1806_09819_gb300 import build as B
    from paper_1806_09819_gb300 import leea, synthetic

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = dist_init(world, True)
    if rank == 0 or world == 1:
        B.build()
    barrier(dist, dev)
    B.build()
    leea.load_library()

    steps, warmup = args.steps, args.warmup
    cfg = CONFIGS[args.config]
    pop, batch, precision = cfg["pop"], cfg["batch"], cfg["precision"]
    if args.pop or args.batch:  # a smaller case of the same kernels, for profiling; not a bench value
        pop, batch = args.pop or pop, args.batch or batch
    (xtr, ytr), _ = synthetic.dataset(n_train=60000, n_test=1)
    u8 = args.input == "u8" or precision > 0
    if u8:  # the images as their 8-bit levels k (x = k / 255), as MNIST stores them
        xtr = synthetic.to_levels(xtr)
    n_batches = warmup + 1 + steps
    idx = synthetic.batch_indices(len(ytr), batch, n_batches, seed=synthetic.BATCH_SEED + rank)
    xs = torch.from_numpy(xtr[idx]).to(dev)       # [n_batches, B, 784], resident in HBM
    ys = torch.from_numpy(ytr[idx]).to(dev)
    stream = torch.cuda.current_stream(dev)

    def gen(st, k):
        if u8:
            st.leea_generation_u8(xs[k], ys[k], 255.0)
        else:
            st.leea_generation(xs[k], ys[k])

    prm = leea.Params(**PARAMS, eval_path=args.eval_path, precision=precision)
    st = leea.LeeaState(pop, DIMS, prm, seed=1000 + rank, stream=stream)
    for k in range(warmup + 1):  # the first call evaluates the initial population
        gen(st, k)
        if k == 0 and precision and rank == 0:
            report_initial = precision_report(st, xs[0].cpu().numpy(), ys[0].cpu().numpy(), precision)
    torch.cuda.synchronize(dev)
    st.leea_profile_enable(True)
    st.leea_profile_read()

    clocks = ClockSampler(_gpu_id_for(local_rank))
    clocks.start()
    # ---- timed region: K generations, inputs resident in HBM ----
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    mark = clocks.mark()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for k in range(steps):
        # per-kernel CUDA events on every PROFILE_EVERY-th generation only: events
        # between kernels cost time and stop a kernel from starting early
        st.leea_profile_enable(k % PROFILE_EVERY == 0)
        gen(st, warmup + 1 + k)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist, dev)
    clk = clocks.stop(mark)
    ms = ev0.elapsed_time(ev1)
    prof = st.leea_profile_read()
    st.leea_profile_enable(False)
    ms_max, gen_per_s = job_rate(world, steps, ms, dist, dev)
    # Breeding and evaluation ran as one kernel (stage 1) when stage 2 has no launch.
    fused = prof["evaluate"][1] == 0 and prof["breed"][1] > 0
    if fused:
        prof = {"select": prof["select"], "breed_evaluate": prof["breed"]}

    # ---- end to end through the host-buffer entry point ----
    e2e_steps = max(10, min(steps, 1000))
    sel = idx[np.arange(e2e_steps) % n_batches]
    xh = torch.from_numpy(xtr[sel]).pin_memory()
    yh = torch.from_numpy(ytr[sel]).pin_memory()
    f_host = None
    barrier(dist, dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        if u8:
            st.leea_generation_u8_host(xh[k], yh[k], 255.0)
        else:
            st.leea_generation_host(xh[k], yh[k])
        f_host = st.leea_fitness()                    # device->host read of the step's result
    t_e2e = time.perf_counter() - t0
    barrier(dist, dev)
    t_e2e = max_over_ranks(t_e2e, dist, dev)
    e2e = {"value": world * e2e_steps / t_e2e, "unit": "generations/s",
           "h2d_bytes_per_step": int(xh[0].numel() * xh.element_size() + yh[0].numel() * 4),
           "d2h_bytes_per_step": int(f_host.nbytes), "steps": e2e_steps}

    # ---- roofline of the dominant kernel ----
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    n_e, n_c, n_m, _ = leea.leea_counts(pop, leea.Params(**PARAMS))
    c = leea.leea_layout_num_params(DIMS)
    d0, h, d_out = DIMS
    tensor_eval = args.eval_path != leea.EVAL_SIMT
    elem = {0: 4, 1: 2, 2: 1}[precision]
    shadow_bytes = d0 * h * elem if precision else 0  # per child written by breed, read by evaluate
    work = {
        # one read and one write per child gene (8c bytes per child in FP32; a
        # crossover child's second parent is not counted: repeats hit L2), plus
        # the shadow of W1 written in the precision form
        "breed": ("hbm", (8.0 * c + shadow_bytes) * (n_e + n_c + n_m) / 1e9, "GB/s", hbm_peak),
        # tensor-core path: the per-individual weight stream (X stays in L2);
        # precision form: the shadow of W1 plus b1, W2, b2 from the master;
        # CUDA-core path: FP32 FFMA work
        "evaluate": (("hbm", (shadow_bytes + 4.0 * (c - d0 * h) if precision else 4.0 * c) * pop / 1e9, "GB/s",
                      hbm_peak) if tensor_eval else
                     ("alu", 2.0 * pop * batch * (d0 * h + h * d_out) / 1e12, "TFLOP/s",
                      SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12)),
        "select": ("latency", None, None, None),
    }
    # fused: the breed's bytes (parents in, children out); the evaluation's
    # weight stream is gone (the minibatch stays in L2)
    work["breed_evaluate"] = work["breed"]
    names = ("select", "breed_evaluate") if fused else STAGES
    kernels = {}
    for name in names:
        tot_ms, launches = prof[name]
        per = tot_ms / max(1, launches)
        bound, units, unit, peak = work[name]
        entry = {"launches": launches, "ms_per_launch": per, "share": tot_ms / max(1e-12, sum(v[0] for v in prof.values()))}
        if units is not None:
            ach = units / (per / 1000.0)
            entry.update({"bound": bound, "achieved": ach, "unit": unit, "peak": peak, "frac": ach / peak})
        kernels[name] = entry
    dom = "breed_evaluate" if fused else max(("breed", "evaluate"), key=lambda n: prof[n][0])
    kd = kernels[dom]
    src = {"breed": "leea_breed.cu", "breed_evaluate": "leea_breed_eval.cu",
           "evaluate": (("leea_eval_shadow.cu" if precision else "leea_eval_u8.cu") if u8 else "leea_eval_tc.cu")
           if tensor_eval else "leea_eval_simt.cu"}[dom]
    tr = TRAFFIC.get(dom) if (args.config, pop, batch, u8) == ("plain", POP, BATCH, True) else None
    traffic = tr["bytes_per_launch"] if tr and tr.get("src_sha") == _src_sha(src) else None
    roofline = {"kernel": dom, "bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
                "unit": kd["unit"], "frac": kd["frac"], "traffic": traffic,
                "peak_source": f"{peak_src} ({'HBM copy' if kd['unit'] == 'GB/s' else 'FP32 FFMA: 152 SM x 128 lanes x 2 x max SM clock'})"}
    if traffic is not None and kd["unit"] == "GB/s":  # DRAM bytes the kernel really moved, at its measured time
        roofline["dram_frac"] = traffic / (kd["ms_per_launch"] / 1000.0) / 1e9 / kd["peak"]
    # the whole generation: breed and evaluation algorithmic bytes over the
    # step time (the evaluation's weight stream is gone when the two are fused)
    if fused or tensor_eval:
        gen_alg = work["breed"][1] + (0.0 if fused else work["evaluate"][1])
        roofline["generation"] = {"algorithmic_gb": gen_alg, "ms": ms_max / steps,
                                  "achieved": gen_alg / (ms_max / steps / 1000.0),
                                  "frac": gen_alg / (ms_max / steps / 1000.0) / hbm_peak,
                                  "floor_ms": gen_alg / hbm_peak * 1000.0}
    if tensor_eval:  # tensor-core work issued (passes, M padded to 128-sample tiles, K to the MMA step)
        k_pad = {0: 784 if u8 else 800, 1: 784, 2: 800}[precision]
        passes = {0: 2 if u8 else 3, 1: 1, 2: 2}[precision]  # u8: two FP16 weight pieces; float: 3xTF32
        tiles = (batch + 127) // 128
        ev = "breed_evaluate" if fused else "evaluate"
        kernels[ev]["tensor_tflops_issued"] = (passes * 2.0 * pop * tiles * 128 * k_pad * h / 1e12) / (
            prof[ev][0] / max(1, prof[ev][1]) / 1000.0)

    pname = {1: "BF16", 2: "FP8-e4m3 (per-individual power-of-two scale)"}.get(precision)
    workload = PRECISION_WORKLOAD.format(name=pname) if precision else WORKLOAD
    if (pop, batch) != (cfg["pop"], cfg["batch"]):
        workload = f"PROFILING OVERRIDE P={pop}, batch {batch} (not the benchmark workload): " + workload
    eval_kernel = ("tcgen05 " + {1: "kind::f16 on BF16 shadows", 2: "kind::f8f6f4 on FP8 shadows, 2 input pieces"}[
        precision] + ", two individuals per MMA (N = 2h), batch tile from shared memory" if precision else
                   (("tcgen05 kind::f16, two individuals per MMA (N = 2h), W1 as two FP16 pieces of 2^8 w "
                     "(22-bit significands, exact products, FP32 accumulation)" if u8 else "tcgen05 3xTF32")
                    if tensor_eval else "CUDA-core FP32 FFMA"))
    if fused:
        eval_kernel = "fused breed + evaluate (children made in shared memory, written once, fed to " + eval_kernel + ")"
    pop_mb = pop * leea.leea_padded_params(DIMS) * 4 / 1e6
    line = {"metric": METRIC, "value": gen_per_s, "unit": "generations/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_max / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {0: "f32", 1: "bf16 (f32 accumulate)", 2: "fp8-e4m3 (f32 accumulate)"}[
                precision], "data": "synthetic",
            "config": {"workload": workload, "parallelism": "replicas" if world > 1 else "single GPU",
                       "kernel_timing": f"CUDA events around each kernel of every {PROFILE_EVERY}th generation "
                                        "inside the timed region",
                       "input": "uint8 levels k, x = k/255" if u8 else "float32 x",
                       "eval_kernel": eval_kernel,
                       "l2": f"inputs larger than L2 (2 population buffers of {pop_mb:.0f} MB), no flush"},
            "network_samples_per_sec": gen_per_s * pop * batch,
            "e2e": e2e,
            "gpu_launches": int(steps * sum(kernels_per_generation(
                pop, batch, precision, fused, x16=(u8 and tensor_eval and not fused) or precision > 0).values())),
            "roofline": roofline,
            "kernels": kernels, "clocks": clk}
    if precision and rank == 0:
        # the last generation evaluated the last end-to-end batch
        line["precision_vs_fp64"] = {
            "initial_population": report_initial,
            "final_population": precision_report(st, xh[e2e_steps - 1].numpy(), yh[e2e_steps - 1].numpy(),
                                                   precision)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not precision:
        pop_now = st.leea_get_population()
        f_now = st.leea_fitness()
        line["cpu_baseline"] = cpu_baseline(pop_now, f_now)
        line["cpu_baseline_fp32"] = cpu_baseline_fp32(pop_now, f_now)
    st.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eval-path", type=int, default=0,
                    help="0 auto (fused breed + evaluate where it applies), 1 CUDA-core FP32, 2 tensor cores as a "
                         "separate kernel, 3 fused")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="plain",
                    help="plain: the headline FP32 workload; small: P=32, 784-32-10, batch 16 (launch latency); "
                         "precision-*: P=4096, batch 256, BF16/FP8 shadows; "
                         "batching: 64 uneven runs together; paper-net: the paper's 196-256-128-64-10 behind 2x2 "
                         "max-pooling at lambda=2000, batch 1024")
    ap.add_argument("--pop", type=int, default=0, help="override the population size (small profiling cases)")
    ap.add_argument("--batch", type=int, default=0, help="override the batch size (small profiling cases)")
    ap.add_argument("--runs", type=int, default=0,
                    help="batching form: only the first N runs (small profiling cases, not the workload)")
    ap.add_argument("--input", choices=["u8", "f32"], default="u8",
                    help="minibatch as 8-bit levels (x = k/255, the images' own encoding) or as float32")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == "small":
        run_small(args, rank, world, local_rank)
    elif args.config == "paper-net":
        run_paper_net(args, rank, world, local_rank)
    elif args.config == "batching":
        run_batching(args, rank, world, local_rank)
    elif args.config == "surrogate":
        run_surrogate(args, rank, world, local_rank)
    else:
        run_native(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
