"""FP64 CPU oracle of the LEEA hot path -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``leea_oracle.c`` (plain C, double
precision, single-threaded) through ctypes and numpy; it never imports the
CUDA package, and the CUDA package never imports it.

Every function takes and returns numpy arrays in the oracle's own layout:
populations are ``float64[pop, c]`` in the logical gene order of Section 3.2
(per layer: W row-major out x in, then b).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "leea_oracle.c")
_HDR = os.path.join(_HERE, "leea_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libleea_oracle.so")

TAG_INIT, TAG_SEL, TAG_XO, TAG_MUTMASK, TAG_NORMAL = 1, 2, 3, 4, 5
TAG_SIGMA = 7
ELITE, CROSSOVER, MUTATION = 0, 1, 2
SIGMA_CONST, SIGMA_DECAY, SIGMA_SELF = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: same results on x86 and Arm)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    stamp_path = os.path.join(os.path.dirname(_OUT), "STAMP")
    try:
        with open(stamp_path) as fh:
            same_host = fh.read() == platform.machine()
    except OSError:
        same_host = False
    if force or not same_host or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
            "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
        with open(stamp_path, "w") as fh:
            fh.write(platform.machine())
    return _OUT


@dataclass
class Params:
    """Operator parameters; defaults are the paper's (Section 4, hyperparameter block)."""
    xo_op: int = 0          # 0 uniform, 1 arithmetic crossover
    xo_gene_p: float = 0.5  # P(gene from parent 2) in uniform crossover
    sel_op: int = 0         # 0 truncation, 1 tournament
    rho: float = 0.5        # truncation proportion
    tour_k: int = 3         # tournament size
    n_elite: int = -1       # -1 => round(p_e * pop)
    p_e: float = 0.05
    p_c: float = 0.5
    sigma: float = 0.001
    mut_rate: float = 1.0   # 1.0 mutates every gene, as in the paper
    alpha: float = 1.0      # 1.0 disables inheritance
    init: int = 0           # 0 N(0, 1/fan_in), 1 Glorot-uniform
    precision: int = 0      # 0 FP32, 1 BF16 shadow, 2 FP8 shadow
    sigma_ctl: int = 0      # SIGMA_CONST, SIGMA_DECAY or SIGMA_SELF (Section 3.2)
    sigma_k: float = 1.0    # decay: breed i uses sigma * 0.99 ** (i / sigma_k)
    tau: float = 0.1        # self-adaptive: sigma' = sigma * exp(tau * N(0, 1))


class _CParams(ctypes.Structure):
    _fields_ = [
        ("xo_op", ctypes.c_int32), ("xo_gene_p", ctypes.c_float),
        ("sel_op", ctypes.c_int32), ("rho", ctypes.c_float),
        ("tour_k", ctypes.c_int32), ("n_elite", ctypes.c_int32),
        ("p_e", ctypes.c_float), ("p_c", ctypes.c_float),
        ("sigma", ctypes.c_float), ("mut_rate", ctypes.c_float),
        ("alpha", ctypes.c_float), ("init", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("sigma_ctl", ctypes.c_int32),
        ("sigma_k", ctypes.c_float), ("tau", ctypes.c_float),
    ]


def _cparams(p: Params) -> _CParams:
    return _CParams(**{f.name: getattr(p, f.name) for f in fields(Params)})


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        i32, u32, u64, i64, dbl = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
        vp = ctypes.c_void_p
        L.leea_cpu_philox.argtypes = [P(u32), P(u32), P(u32)]
        L.leea_cpu_philox.restype = None
        L.leea_cpu_draw.argtypes = [u64, u32, u32, u32, u32]
        L.leea_cpu_draw.restype = u32
        L.leea_cpu_u01.argtypes = [u32]
        L.leea_cpu_u01.restype = dbl
        L.leea_cpu_normal.argtypes = [u64, u32, u32, u32, u32]
        L.leea_cpu_normal.restype = dbl
        L.leea_cpu_index.argtypes = [u32, u32]
        L.leea_cpu_index.restype = u32
        L.leea_cpu_threshold.argtypes = [dbl]
        L.leea_cpu_threshold.restype = u64
        L.leea_cpu_round_bf16.argtypes = [dbl]
        L.leea_cpu_round_bf16.restype = dbl
        L.leea_cpu_round_e4m3.argtypes = [dbl]
        L.leea_cpu_round_e4m3.restype = dbl
        L.leea_cpu_fp8_scale_exp.argtypes = [dbl]
        L.leea_cpu_fp8_scale_exp.restype = i32
        L.leea_cpu_quantize_w1.argtypes = [i32, vp, i32, vp, i32, vp, vp]
        L.leea_cpu_evaluate_shadow.argtypes = [i32, vp, i32, vp, i32, vp, vp, vp, i32, vp, vp]
        L.leea_cpu_evaluate_shadow.restype = ctypes.c_int
        L.leea_cpu_draw16.argtypes = [u64, u32, u32, u32, u32]
        L.leea_cpu_draw16.restype = u32
        L.leea_cpu_threshold16.argtypes = [dbl]
        L.leea_cpu_threshold16.restype = u32
        L.leea_cpu_num_params.argtypes = [vp, i32]
        L.leea_cpu_num_params.restype = i64
        L.leea_cpu_counts.argtypes = [i32, P(_CParams), P(i32), P(i32), P(i32), P(i32)]
        L.leea_cpu_init.argtypes = [i32, vp, i32, i32, u64, vp]
        L.leea_cpu_evaluate.argtypes = [i32, vp, i32, vp, vp, vp, i32, vp, vp, vp]
        L.leea_cpu_rank.argtypes = [i32, vp, vp]
        L.leea_cpu_maxpool2x2.argtypes = [i32, i32, i32, vp, vp]
        L.leea_cpu_select.argtypes = [i32, P(_CParams), vp, vp, u64, u32, vp, vp, vp, vp]
        L.leea_cpu_breed.argtypes = [i32, vp, i32, P(_CParams), u64, u32, vp, vp, vp, vp, i32, i32, vp]
        L.leea_cpu_inherit.argtypes = [i32, dbl, vp, vp, i32, vp]
        L.leea_cpu_sigma_schedule.argtypes = [P(_CParams), u32]
        L.leea_cpu_sigma_schedule.restype = dbl
        L.leea_cpu_select_sigma.argtypes = [i32, P(_CParams), u64, u32, vp, vp, vp, vp, vp]
        L.leea_cpu_breed_sigma.argtypes = [i32, vp, i32, P(_CParams), u64, u32, vp, vp, vp, vp, vp, i32, i32, vp]
        L.leea_cpu_get_sigma.argtypes = [vp, vp]
        L.leea_cpu_set_sigma.argtypes = [vp, vp]
        L.leea_cpu_create.argtypes = [i32, vp, i32, P(_CParams), u64, P(vp)]
        L.leea_cpu_generation.argtypes = [vp, vp, vp, i32]
        L.leea_cpu_fitness.argtypes = [vp, vp, vp, vp]
        L.leea_cpu_best_params.argtypes = [vp, vp, i64]
        L.leea_cpu_get_population.argtypes = [vp, vp]
        L.leea_cpu_set_population.argtypes = [vp, vp]
        L.leea_cpu_set_fitness.argtypes = [vp, vp]
        L.leea_cpu_set_generation.argtypes = [vp, u32, i32]
        L.leea_cpu_get_selection.argtypes = [vp, vp, vp, vp, vp, vp]
        L.leea_cpu_generation_index.argtypes = [vp]
        L.leea_cpu_generation_index.restype = u32
        L.leea_cpu_destroy.argtypes = [vp]
        L.leea_cpu_destroy.restype = None
        L.leea_cpu_mlp_num_params.argtypes = [i32, i32, i32]
        L.leea_cpu_mlp_num_params.restype = i64
        L.leea_cpu_mlp_init.argtypes = [i32, i32, i32, u64, vp]
        L.leea_cpu_mlp_forward.argtypes = [i32, i32, i32, i32, vp, vp, vp]
        L.leea_cpu_mlp_loss_grad.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, vp]
        L.leea_cpu_adam.argtypes = [i64, vp, vp, vp, vp, i64, dbl, dbl, dbl, dbl]
        L.leea_cpu_select_recipes.argtypes = [i32, P(_CParams), vp, vp, u64, u32, i32, vp, vp, vp, vp, vp]
        L.leea_cpu_breed_entities.argtypes = [i32, vp, i32, P(_CParams), u64, u32, vp, vp, vp, vp, vp, i32, vp]
        L.leea_cpu_recipe_stats.argtypes = [vp, i32, P(_CParams), u64, u32, vp, vp, i32, vp, vp]
        L.leea_cpu_descriptors.argtypes = [i32, vp, i32, P(_CParams), u64, u32, vp, vp, vp, vp, vp, vp, vp, i32,
                                           vp, i32, vp]
        for name in ("leea_cpu_mlp_init", "leea_cpu_mlp_forward", "leea_cpu_mlp_loss_grad", "leea_cpu_adam",
                     "leea_cpu_select_recipes", "leea_cpu_breed_entities", "leea_cpu_recipe_stats",
                     "leea_cpu_descriptors"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("leea_cpu_counts", "leea_cpu_init", "leea_cpu_evaluate", "leea_cpu_rank",
                     "leea_cpu_select", "leea_cpu_breed", "leea_cpu_inherit", "leea_cpu_create",
                     "leea_cpu_generation", "leea_cpu_fitness", "leea_cpu_best_params",
                     "leea_cpu_get_population", "leea_cpu_set_population", "leea_cpu_set_fitness",
                     "leea_cpu_set_generation", "leea_cpu_get_selection"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# ---- random streams -------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().leea_cpu_philox(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def draw(seed: int, tag: int, gen: int, ent: int, n: int) -> int:
    return int(lib().leea_cpu_draw(seed, tag, gen, ent, n))


def u01(u: int) -> float:
    return float(lib().leea_cpu_u01(u))


def normal(seed: int, tag: int, gen: int, ent: int, i: int) -> float:
    return float(lib().leea_cpu_normal(seed, tag, gen, ent, i))


def index(u: int, m: int) -> int:
    return int(lib().leea_cpu_index(u, m))


def threshold(q: float) -> int:
    return int(lib().leea_cpu_threshold(float(q)))


def draw16(seed: int, tag: int, gen: int, ent: int, i: int) -> int:
    return int(lib().leea_cpu_draw16(seed, tag, gen, ent, i))


def threshold16(q: float) -> int:
    return int(lib().leea_cpu_threshold16(float(q)))


# ---- precision form -------------------------------------------------------
def round_bf16(x: float) -> float:
    return float(lib().leea_cpu_round_bf16(float(x)))


def round_e4m3(x: float) -> float:
    return float(lib().leea_cpu_round_e4m3(float(x)))


def fp8_scale_exp(bound: float) -> int:
    return int(lib().leea_cpu_fp8_scale_exp(float(bound)))


def quantize_w1(popv, dims, precision: int, scale_exp) -> np.ndarray:
    """The population with W1 replaced by its BF16 (1) or scaled FP8-e4m3 (2) shadow's value."""
    d = _dims(dims)
    pv = _f64(popv)
    out = np.empty_like(pv)
    se = None if scale_exp is None else _i32(scale_exp)
    _check(lib().leea_cpu_quantize_w1(pv.shape[0], _ptr(d), len(d), _ptr(pv), int(precision), _ptr(se), _ptr(out)),
           "quantize_w1")
    return out


def evaluate_shadow(popv, dims, precision: int, scale_exp, x, y):
    """Fitness with W1 replaced by its BF16 (1) or scaled FP8-e4m3 (2) shadow."""
    d = _dims(dims)
    pv = _f64(popv)
    pop = pv.shape[0]
    xv = _f64(x).reshape(-1, int(d[0]))
    yv = _i32(y)
    se = None if scale_exp is None else _i32(scale_exp)
    f = np.empty(pop, dtype=np.float64)
    cor = np.empty(pop, dtype=np.int32)
    _check(lib().leea_cpu_evaluate_shadow(pop, _ptr(d), len(d), _ptr(pv), int(precision), _ptr(se), _ptr(xv),
                                          _ptr(yv), xv.shape[0], _ptr(f), _ptr(cor)), "evaluate_shadow")
    return f, cor


# ---- layout ---------------------------------------------------------------
def num_params(dims) -> int:
    d = _dims(dims)
    return int(lib().leea_cpu_num_params(_ptr(d), len(d)))


def counts(pop: int, prm: Params) -> tuple[int, int, int, int]:
    e, c, m, pl = (ctypes.c_int32() for _ in range(4))
    cp = _cparams(prm)
    _check(lib().leea_cpu_counts(pop, ctypes.byref(cp), ctypes.byref(e), ctypes.byref(c),
                                 ctypes.byref(m), ctypes.byref(pl)), "counts")
    return e.value, c.value, m.value, pl.value


# ---- steps ----------------------------------------------------------------
def init(pop: int, dims, init_kind: int, seed: int) -> np.ndarray:
    d = _dims(dims)
    out = np.empty((pop, num_params(d)), dtype=np.float64)
    _check(lib().leea_cpu_init(pop, _ptr(d), len(d), init_kind, seed, _ptr(out)), "init")
    return out


def evaluate(popv, dims, x, y, want_logits: bool = False):
    """Returns (f[pop], correct[pop]) or (f, correct, logits[pop, batch, d_out])."""
    d = _dims(dims)
    pv = _f64(popv)
    pop = pv.shape[0]
    xv = _f64(x).reshape(-1, int(d[0]))
    yv = _i32(y)
    batch = xv.shape[0]
    f = np.empty(pop, dtype=np.float64)
    cor = np.empty(pop, dtype=np.int32)
    logits = np.empty((pop, batch, int(d[-1])), dtype=np.float64) if want_logits else None
    _check(lib().leea_cpu_evaluate(pop, _ptr(d), len(d), _ptr(pv), _ptr(xv), _ptr(yv), batch,
                                   _ptr(f), _ptr(cor), _ptr(logits)), "evaluate")
    return (f, cor, logits) if want_logits else (f, cor)


def maxpool2x2(x, h: int, w: int) -> np.ndarray:
    """Section 4.1's input stage: 2x2 max-pooling of images x[b] (h x w, row-major)."""
    xv = _f64(x).reshape(-1, h * w)
    out = np.empty((xv.shape[0], (h // 2) * (w // 2)), dtype=np.float64)
    _check(lib().leea_cpu_maxpool2x2(xv.shape[0], h, w, _ptr(xv), _ptr(out)), "maxpool2x2")
    return out


def rank(f_adj) -> np.ndarray:
    f = _f64(f_adj)
    order = np.empty(f.shape[0], dtype=np.int32)
    _check(lib().leea_cpu_rank(f.shape[0], _ptr(f), _ptr(order)), "rank")
    return order


def select(prm: Params, f_adj, order, seed: int, gen: int):
    """Returns (par1, par2, kind, f_inh)."""
    f = _f64(f_adj)
    o = _i32(order)
    pop = f.shape[0]
    par1, par2, kind = (np.empty(pop, dtype=np.int32) for _ in range(3))
    f_inh = np.empty(pop, dtype=np.float64)
    cp = _cparams(prm)
    _check(lib().leea_cpu_select(pop, ctypes.byref(cp), _ptr(f), _ptr(o), seed, gen,
                                 _ptr(par1), _ptr(par2), _ptr(kind), _ptr(f_inh)), "select")
    return par1, par2, kind, f_inh


def breed(prm: Params, dims, seed: int, gen: int, parents, par1, par2, kind,
          j0: int = 0, j1: int | None = None) -> np.ndarray:
    d = _dims(dims)
    pv = _f64(parents)
    pop = pv.shape[0]
    j1 = pop if j1 is None else j1
    out = np.empty((j1 - j0, pv.shape[1]), dtype=np.float64)
    cp = _cparams(prm)
    _check(lib().leea_cpu_breed(pop, _ptr(d), len(d), ctypes.byref(cp), seed, gen, _ptr(pv),
                                _ptr(_i32(par1)), _ptr(_i32(par2)), _ptr(_i32(kind)),
                                j0, j1, _ptr(out)), "breed")
    return out


def sigma_schedule(prm: Params, gen: int) -> float:
    """Mutation strength of the breed with generation counter gen (Section 3.2)."""
    cp = _cparams(prm)
    return float(lib().leea_cpu_sigma_schedule(ctypes.byref(cp), gen))


def select_sigma(prm: Params, seed: int, gen: int, par1, par2, kind, sigma_in) -> np.ndarray:
    """Self-adaptive control: the children's sigma genes from their parents'."""
    si = _f64(sigma_in)
    out = np.empty_like(si)
    cp = _cparams(prm)
    _check(lib().leea_cpu_select_sigma(si.shape[0], ctypes.byref(cp), seed, gen, _ptr(_i32(par1)),
                                       _ptr(_i32(par2)), _ptr(_i32(kind)), _ptr(si), _ptr(out)),
           "select_sigma")
    return out


def breed_sigma(prm: Params, dims, seed: int, gen: int, parents, par1, par2, kind, sigma_child,
                j0: int = 0, j1: int | None = None) -> np.ndarray:
    """breed() with mutation strength sigma_child[j] for child j."""
    d = _dims(dims)
    pv = _f64(parents)
    pop = pv.shape[0]
    j1 = pop if j1 is None else j1
    out = np.empty((j1 - j0, pv.shape[1]), dtype=np.float64)
    cp = _cparams(prm)
    _check(lib().leea_cpu_breed_sigma(pop, _ptr(d), len(d), ctypes.byref(cp), seed, gen, _ptr(pv),
                                      _ptr(_i32(par1)), _ptr(_i32(par2)), _ptr(_i32(kind)),
                                      _ptr(_f64(sigma_child)), j0, j1, _ptr(out)), "breed_sigma")
    return out


def inherit(alpha: float, f_inh, f, first: bool) -> np.ndarray:
    fv = _f64(f)
    fi = None if f_inh is None else _f64(f_inh)
    out = np.empty_like(fv)
    _check(lib().leea_cpu_inherit(fv.shape[0], float(alpha), _ptr(fi), _ptr(fv), int(first),
                                  _ptr(out)), "inherit")
    return out


# ---- Algorithm 1 as a state object ---------------------------------------------
class State:
    """The oracle's LEEA run (the leea_cpu_* state ABI)."""

    def __init__(self, pop: int, dims, prm: Params, seed: int):
        self.pop = pop
        self.dims = _dims(dims)
        self.c = num_params(self.dims)
        self._cp = _cparams(prm)
        h = ctypes.c_void_p()
        _check(lib().leea_cpu_create(pop, _ptr(self.dims), len(self.dims), ctypes.byref(self._cp),
                                     seed, ctypes.byref(h)), "create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.leea_cpu_destroy(h)
            self._h = None

    def generation(self, x, y) -> None:
        xv = _f64(x).reshape(-1, int(self.dims[0]))
        yv = _i32(y)
        _check(lib().leea_cpu_generation(self._h, _ptr(xv), _ptr(yv), xv.shape[0]), "generation")

    def fitness(self):
        f_adj = np.empty(self.pop, dtype=np.float64)
        f_raw = np.empty(self.pop, dtype=np.float64)
        cor = np.empty(self.pop, dtype=np.int32)
        _check(lib().leea_cpu_fitness(self._h, _ptr(f_adj), _ptr(f_raw), _ptr(cor)), "fitness")
        return f_adj, f_raw, cor

    def best_params(self) -> np.ndarray:
        out = np.empty(self.c, dtype=np.float64)
        _check(lib().leea_cpu_best_params(self._h, _ptr(out), self.c), "best_params")
        return out

    def population(self) -> np.ndarray:
        out = np.empty((self.pop, self.c), dtype=np.float64)
        _check(lib().leea_cpu_get_population(self._h, _ptr(out)), "get_population")
        return out

    def set_population(self, popv) -> None:
        pv = _f64(popv)
        assert pv.shape == (self.pop, self.c)
        _check(lib().leea_cpu_set_population(self._h, _ptr(pv)), "set_population")

    def set_fitness(self, f_adj) -> None:
        _check(lib().leea_cpu_set_fitness(self._h, _ptr(_f64(f_adj))), "set_fitness")

    def set_generation(self, gen: int, evaluated: bool) -> None:
        _check(lib().leea_cpu_set_generation(self._h, gen, int(evaluated)), "set_generation")

    @property
    def gen(self) -> int:
        return int(lib().leea_cpu_generation_index(self._h))

    def sigma(self) -> np.ndarray:
        """Sigma genes (self-adaptive control) or the next breed's strength, per individual."""
        out = np.empty(self.pop, dtype=np.float64)
        _check(lib().leea_cpu_get_sigma(self._h, _ptr(out)), "get_sigma")
        return out

    def set_sigma(self, sigma) -> None:
        _check(lib().leea_cpu_set_sigma(self._h, _ptr(_f64(sigma))), "set_sigma")

    def selection(self):
        """Returns (order, par1, par2, kind, f_inh) of the last breed."""
        arrs = [np.empty(self.pop, dtype=np.int32) for _ in range(4)]
        f_inh = np.empty(self.pop, dtype=np.float64)
        _check(lib().leea_cpu_get_selection(self._h, *[_ptr(a) for a in arrs], _ptr(f_inh)),
               "get_selection")
        return (*arrs, f_inh)


# ---- surrogate form (no counterpart in the paper) --------------------------------
RECIPE_ENTITY0 = 0x40000000
TAG_SURR_INIT = 6


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def mlp_num_params(d_in: int, h1: int, h2: int) -> int:
    return int(lib().leea_cpu_mlp_num_params(d_in, h1, h2))


def mlp_init(d_in: int, h1: int, h2: int, seed: int) -> np.ndarray:
    theta = np.empty(mlp_num_params(d_in, h1, h2), dtype=np.float64)
    _check(lib().leea_cpu_mlp_init(d_in, h1, h2, seed, _ptr(theta)), "mlp_init")
    return theta


def mlp_forward(theta, x, d_in: int, h1: int, h2: int) -> np.ndarray:
    xv = _f64(x).reshape(-1, d_in)
    y = np.empty(xv.shape[0], dtype=np.float64)
    _check(lib().leea_cpu_mlp_forward(xv.shape[0], d_in, h1, h2, _ptr(_f64(theta)), _ptr(xv), _ptr(y)),
           "mlp_forward")
    return y


def mlp_loss_grad(theta, x, t, d_in: int, h1: int, h2: int):
    """(mean squared error, gradient) of the MLP's predictions against t."""
    xv = _f64(x).reshape(-1, d_in)
    tv = _f64(t)
    th = _f64(theta)
    grad = np.empty_like(th)
    loss = ctypes.c_double()
    _check(lib().leea_cpu_mlp_loss_grad(xv.shape[0], d_in, h1, h2, _ptr(th), _ptr(xv), _ptr(tv),
                                        ctypes.byref(loss), _ptr(grad)), "mlp_loss_grad")
    return float(loss.value), grad


def adam(theta, grad, m, v, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8):
    """One Adam step; returns new (theta, m, v)."""
    th, mm, vv = _f64(theta).copy(), _f64(m).copy(), _f64(v).copy()
    _check(lib().leea_cpu_adam(th.shape[0], _ptr(th), _ptr(_f64(grad)), _ptr(mm), _ptr(vv), step, lr, beta1, beta2,
                               eps), "adam")
    return th, mm, vv


def select_recipes(prm: Params, f_adj, order, seed: int, gen: int, mult: int):
    """(par1, par2, kind, f_inh, entity) of the mult (n_C + n_M) recipes."""
    f = _f64(f_adj)
    pop = f.shape[0]
    _, n_c, n_m, _ = counts(pop, prm)
    n = mult * (n_c + n_m)
    par1, par2, kind = (np.empty(n, dtype=np.int32) for _ in range(3))
    f_inh = np.empty(n, dtype=np.float64)
    ent = np.empty(n, dtype=np.uint32)
    cp = _cparams(prm)
    _check(lib().leea_cpu_select_recipes(pop, ctypes.byref(cp), _ptr(f), _ptr(_i32(order)), seed, gen, mult,
                                         _ptr(par1), _ptr(par2), _ptr(kind), _ptr(f_inh), _ptr(ent)),
           "select_recipes")
    return par1, par2, kind, f_inh, ent


def breed_entities(prm: Params, dims, seed: int, gen: int, parents, par1, par2, kind, entity) -> np.ndarray:
    d = _dims(dims)
    pv = _f64(parents)
    n = len(kind)
    out = np.empty((n, pv.shape[1]), dtype=np.float64)
    cp = _cparams(prm)
    _check(lib().leea_cpu_breed_entities(pv.shape[0], _ptr(d), len(d), ctypes.byref(cp), seed, gen, _ptr(pv),
                                         _ptr(_i32(par1)), _ptr(_i32(par2)), _ptr(_i32(kind)), _ptr(_u32(entity)),
                                         n, _ptr(out)), "breed_entities")
    return out


def recipe_stats(prm: Params, dims, seed: int, gen: int, kind, entity):
    """(xo_frac, mut_norm) per recipe."""
    d = _dims(dims)
    n = len(kind)
    xf, mn = np.empty(n, dtype=np.float64), np.empty(n, dtype=np.float64)
    cp = _cparams(prm)
    _check(lib().leea_cpu_recipe_stats(_ptr(d), len(d), ctypes.byref(cp), seed, gen, _ptr(_i32(kind)),
                                       _ptr(_u32(entity)), n, _ptr(xf), _ptr(mn)), "recipe_stats")
    return xf, mn


def descriptors(prm: Params, dims, seed: int, gen: int, parents, f_adj, par1, par2, kind, f_inh, entity, probe_x):
    """float64[n][5 + n_probe d_out] descriptors of the recipes."""
    d = _dims(dims)
    pv = _f64(parents)
    px = _f64(probe_x).reshape(-1, int(d[0]))
    n = len(kind)
    out = np.empty((n, 5 + px.shape[0] * int(d[-1])), dtype=np.float64)
    cp = _cparams(prm)
    _check(lib().leea_cpu_descriptors(pv.shape[0], _ptr(d), len(d), ctypes.byref(cp), seed, gen, _ptr(pv),
                                      _ptr(_f64(f_adj)), _ptr(_i32(par1)), _ptr(_i32(par2)), _ptr(_i32(kind)),
                                      _ptr(_f64(f_inh)), _ptr(_u32(entity)), n, _ptr(px), px.shape[0], _ptr(out)),
           "descriptors")
    return out


# ---- the FP32 multi-core CPU baseline (leea_cpu_fp32.c) ----------------------
_SRC32 = os.path.join(_HERE, "leea_cpu_fp32.c")
_OUT32 = os.path.join(_HERE, "_build", "libleea_cpu32.so")
_lib32 = None


def build32(force: bool = False) -> str:
    """Compile the FP32 baseline (OpenMP where gcc has it) with the oracle
    linked in (its ranking, selection and Philox block).  The baseline's file
    alone is compiled for speed; the oracle's keeps its own flags."""
    os.makedirs(os.path.dirname(_OUT32), exist_ok=True)
    newest = max(os.path.getmtime(_SRC32), os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    stamp_path = os.path.join(os.path.dirname(_OUT32), "STAMP32")
    try:
        with open(stamp_path) as fh:
            same_host = fh.read() == platform.machine()
    except OSError:
        same_host = False
    if force or not same_host or not os.path.exists(_OUT32) or os.path.getmtime(_OUT32) < newest:
        bdir = os.path.dirname(_OUT32)
        o_oracle = os.path.join(bdir, f"oracle32_{os.getpid()}.o")
        o_fp32 = os.path.join(bdir, f"fp32_{os.getpid()}.o")
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-c", "-o", o_oracle, _SRC])
        fast = ["-O3", "-fno-math-errno", "-fno-trapping-math", "-fno-signed-zeros", "-fassociative-math"]
        omp = ["-fopenmp"]
        try:
            subprocess.check_call(["gcc", "-std=gnu99", *fast, *omp, "-fPIC", "-c", "-o", o_fp32, _SRC32])
        except subprocess.CalledProcessError:
            omp = []
            subprocess.check_call(["gcc", "-std=gnu99", *fast, "-fPIC", "-c", "-o", o_fp32, _SRC32])
        tmp = _OUT32 + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-shared", *omp, "-o", tmp, o_oracle, o_fp32, "-lm"])
        os.replace(tmp, _OUT32)
        for f in (o_oracle, o_fp32):
            os.remove(f)
        with open(stamp_path, "w") as fh:
            fh.write(platform.machine())
    return _OUT32


def lib32() -> ctypes.CDLL:
    global _lib32
    if _lib32 is None:
        L = ctypes.CDLL(build32())
        vp, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        L.leea_cpu32_threads.argtypes = []
        L.leea_cpu32_threads.restype = ctypes.c_int
        L.leea_cpu32_generation.argtypes = [i32, vp, i32, ctypes.POINTER(_CParams), u64, u32, vp, vp, vp, vp, i32,
                                            vp, vp, vp, vp, vp]
        L.leea_cpu32_generation.restype = ctypes.c_int
        _lib32 = L
    return _lib32


def cpu32_generation(prm: Params, dims, seed: int, gen: int, parents, f_adj, x, y):
    """One generation on every host core in FP32 (the CPU baseline): returns
    (children float32[pop, c], f_raw, f_adj, correct, threads used)."""
    d = _dims(dims)
    pv = np.ascontiguousarray(np.asarray(parents, dtype=np.float32))
    pop = pv.shape[0]
    fa = np.ascontiguousarray(np.asarray(f_adj, dtype=np.float32))
    xv = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).reshape(-1, int(d[0]))
    yv = _i32(y)
    kids = np.empty_like(pv)
    f_raw = np.empty(pop, dtype=np.float32)
    f_out = np.empty(pop, dtype=np.float32)
    cor = np.empty(pop, dtype=np.int32)
    thr = ctypes.c_int32(0)
    cp = _cparams(prm)
    _check(lib32().leea_cpu32_generation(pop, _ptr(d), len(d), ctypes.byref(cp), seed, gen, _ptr(pv), _ptr(fa),
                                         _ptr(xv), _ptr(yv), xv.shape[0], _ptr(kids), _ptr(f_raw), _ptr(f_out),
                                         _ptr(cor), ctypes.byref(thr)), "cpu32_generation")
    return kids, f_raw, f_out, cor, int(thr.value)
