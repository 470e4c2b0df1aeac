"""Thin ctypes binding of the C ABI in ``include/leea.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libleea.so``.  Device buffers are torch CUDA tensors (torch is used
for device memory and streams); each function passes their data pointers and
the current torch stream straight through.  If the library cannot be loaded
the functions raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, fields

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libleea.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT = range(6)
TAG_INIT, TAG_SEL, TAG_XO, TAG_MUTMASK, TAG_NORMAL = 1, 2, 3, 4, 5
TAG_SIGMA = 7
SIGMA_CONST, SIGMA_DECAY, SIGMA_SELF = 0, 1, 2
KIND_ELITE, KIND_CROSSOVER, KIND_MUTATION = 0, 1, 2
EVAL_AUTO, EVAL_SIMT, EVAL_TENSOR, EVAL_FUSED, EVAL_SMALL = 0, 1, 2, 3, 4
PRECISION_FP32, PRECISION_BF16, PRECISION_FP8 = 0, 1, 2
NUM_STAGES = 3
STAGES = ("select", "breed", "evaluate")  # select = ranking + selection


class LeeaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"LEEA status {status}: {msg}")
        self.status = status


class leea_run_spec(ctypes.Structure):
    _fields_ = [("pop", ctypes.c_int32), ("hidden", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("group", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class leea_surrogate_params(ctypes.Structure):
    _fields_ = [("mult", ctypes.c_int32), ("n_probe", ctypes.c_int32), ("hidden1", ctypes.c_int32),
                ("hidden2", ctypes.c_int32), ("train_steps", ctypes.c_int32), ("train_batch", ctypes.c_int32),
                ("history", ctypes.c_int32), ("warmup", ctypes.c_int32), ("lr", ctypes.c_float),
                ("audit_frac", ctypes.c_float), ("min_spearman", ctypes.c_float), ("seed", ctypes.c_uint64)]


class leea_params(ctypes.Structure):
    _fields_ = [
        ("xo_op", ctypes.c_int32), ("xo_gene_p", ctypes.c_float),
        ("sel_op", ctypes.c_int32), ("rho", ctypes.c_float),
        ("tour_k", ctypes.c_int32), ("n_elite", ctypes.c_int32),
        ("p_e", ctypes.c_float), ("p_c", ctypes.c_float),
        ("sigma", ctypes.c_float), ("mut_rate", ctypes.c_float),
        ("alpha", ctypes.c_float), ("init", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("eval_path", ctypes.c_int32),
        ("sigma_ctl", ctypes.c_int32), ("sigma_k", ctypes.c_float), ("tau", ctypes.c_float),
    ]


@dataclass
class Params:
    """Operator parameters (fields of ``leea_params``); defaults are the paper's."""
    xo_op: int = 0
    xo_gene_p: float = 0.5
    sel_op: int = 0
    rho: float = 0.5
    tour_k: int = 3
    n_elite: int = -1
    p_e: float = 0.05
    p_c: float = 0.5
    sigma: float = 0.001
    mut_rate: float = 1.0
    alpha: float = 1.0
    init: int = 0
    precision: int = 0  # PRECISION_FP32, PRECISION_BF16 or PRECISION_FP8
    eval_path: int = 0  # EVAL_AUTO, EVAL_SIMT, EVAL_TENSOR, EVAL_FUSED or EVAL_SMALL
    sigma_ctl: int = 0  # SIGMA_CONST, SIGMA_DECAY or SIGMA_SELF (Section 3.2)
    sigma_k: float = 1.0
    tau: float = 0.1

    def c_struct(self) -> leea_params:
        return leea_params(**{f.name: getattr(self, f.name) for f in fields(Params)})


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Loads ``libleea.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"LEEA CUDA library not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    i32, u32, u64, i64, f32 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_float
    vp = ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "leea_default_params": [P(leea_params)],
        "leea_layout_num_params": ([vp, i32], i64),
        "leea_padded_params": ([vp, i32], i64),
        "leea_counts": [i32, P(leea_params), P(i32), P(i32), P(i32), P(i32)],
        "leea_init_population": [i32, vp, i32, i32, u64, vp, vp],
        "leea_rank": [i32, vp, vp, vp],
        "leea_select": [i32, P(leea_params), vp, vp, u64, u32, vp, vp, vp, vp, vp],
        "leea_breed": [i32, vp, i32, P(leea_params), u64, u32, vp, vp, vp, vp, vp, vp],
        "leea_maxpool2x2": [i32, i32, i32, vp, vp, vp],
        "leea_maxpool2x2_u8": [i32, i32, i32, vp, vp, vp],
        "leea_breed_evaluate_u8": [i32, vp, i32, P(leea_params), u64, u32, vp, vp, vp, vp, vp, vp, f32, vp, i32, f32,
                                   vp, vp, vp, vp, vp],
        "leea_evaluate": [i32, vp, i32, vp, vp, vp, i32, f32, vp, vp, vp, vp, i32, vp],
        "leea_device_status": [vp, P(u32)],
        "leea_selftest_wait_timeout": [u32, vp],
        "leea_shadow_stride": ([vp, i32, i32], i64),
        "leea_make_shadow": [i32, vp, i32, i32, vp, vp, vp, vp, vp],
        "leea_shadow_scratch_bytes": ([i32, i32], i64),
        "leea_evaluate_shadow_u8": [i32, vp, i32, vp, i32, vp, vp, vp, f32, vp, i32, f32, vp, vp, vp, vp, vp, i64,
                                    vp],
        "leea_get_shadow": [vp, vp, vp, vp],
        "leea_evaluate_shadow_u8_noalloc": [i32, vp, i32, vp, i32, vp, vp, vp, f32, vp, i32, f32, vp, vp, vp, vp,
                                            vp],
        "leea_evaluate_u8": [i32, vp, i32, vp, vp, f32, vp, i32, f32, vp, vp, vp, vp, i32, vp],
        "leea_generation_u8": [vp, vp, f32, vp, i32],
        "leea_generation_u8_host": [vp, vp, f32, vp, i32],
        "leea_philox_fill": [u64, u32, u32, u32, u32, i64, vp, vp],
        "leea_normal_fill": [u64, u32, u32, u32, u32, i64, vp, vp],
        "leea_create": [i32, vp, i32, P(leea_params), u64, vp, P(vp)],
        "leea_generation": [vp, vp, vp, i32],
        "leea_generation_host": [vp, vp, vp, i32],
        "leea_fitness": [vp, vp, vp],
        "leea_raw_fitness": [vp, vp],
        "leea_best_params": [vp, vp, i64],
        "leea_get_population": [vp, vp],
        "leea_set_population": [vp, vp],
        "leea_set_fitness": [vp, vp],
        "leea_set_generation": [vp, u32, i32],
        "leea_get_selection": [vp, vp, vp, vp, vp, vp],
        "leea_generation_index": ([vp], u32),
        "leea_get_sigma": [vp, vp],
        "leea_set_sigma": [vp, vp],
        "leea_num_params": ([vp], i64),
        "leea_profile_enable": [vp, i32],
        "leea_profile_read": [vp, vp, vp],
        "leea_multi_create": [i32, vp, i32, i32, P(leea_params), vp, P(vp)],
        "leea_multi_layout": [vp, vp, vp, vp, vp],
        "leea_multi_run_shape": [vp, i32, vp, vp, vp, vp],
        "leea_multi_eval_launches": [vp, vp],
        "leea_multi_batch_buffers": [vp, P(vp), P(vp)],
        "leea_multi_generation_u8": [vp, vp, f32, vp],
        "leea_multi_generation_u8_host": [vp, vp, f32, vp],
        "leea_multi_fitness": [vp, vp, vp],
        "leea_multi_raw_fitness": [vp, vp],
        "leea_multi_get_population": [vp, i32, vp],
        "leea_multi_set_population": [vp, i32, vp],
        "leea_multi_set_fitness": [vp, vp],
        "leea_multi_set_generation": [vp, u32, i32],
        "leea_multi_get_selection": [vp, i32, vp, vp, vp, vp, vp],
        "leea_multi_get_shadow": [vp, i32, vp, vp, vp],
        "leea_multi_generation_index": ([vp], u32),
        "leea_multi_profile_enable": [vp, i32],
        "leea_multi_profile_read": [vp, vp, vp],
        "leea_multi_destroy": ([vp], None),
        "leea_tune_shadow_eval": [i32, i32, i32, i32, i32, i32, i32, i32, P(f32)],
        "leea_tune_group_eval": [i32, i32, i32, i32, i32, i32, i32, i32, P(f32)],
        "leea_num_recipes": ([i32, P(leea_params), i32], i32),
        "leea_select_recipes": [i32, P(leea_params), vp, vp, u64, u32, i32, vp, vp, vp, vp, vp, vp],
        "leea_breed_entities": [i32, vp, i32, P(leea_params), u64, u32, vp, vp, vp, vp, vp, i32, vp, vp],
        "leea_descriptors": [i32, vp, i32, P(leea_params), u64, u32, vp, vp, vp, vp, vp, vp, vp, i32, vp, i32,
                             vp, vp],
        "leea_surrogate_num_params": ([i32, i32, i32], i64),
        "leea_surrogate_init": [i32, i32, i32, u64, vp, vp],
        "leea_surrogate_forward": [i32, i32, i32, i32, vp, vp, vp, vp],
        "leea_surrogate_work_floats": ([i32, i32, i32], i64),
        "leea_surrogate_loss_grad": [i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, i64, vp],
        "leea_surrogate_adam": [i64, vp, vp, vp, vp, i64, f32, f32, f32, f32, vp],
        "leea_surrogate_default_params": [P(leea_surrogate_params)],
        "leea_surr_create": [i32, vp, i32, P(leea_params), P(leea_surrogate_params), u64, vp, vp, P(vp)],
        "leea_surr_generation_u8": [vp, vp, f32, vp, i32],
        "leea_surr_generation_u8_host": [vp, vp, f32, vp, i32],
        "leea_surr_fitness": [vp, vp, vp],
        "leea_surr_raw_fitness": [vp, vp, vp],
        "leea_surr_get_population": [vp, vp],
        "leea_surr_set_population": [vp, vp],
        "leea_surr_set_fitness": [vp, vp],
        "leea_surr_set_generation": [vp, u32, i32],
        "leea_surr_set_screen": [vp, i32],
        "leea_surr_layout": [vp, vp, vp, vp, vp],
        "leea_surr_get_step": [vp] + [vp] * 13,
        "leea_surr_get_surrogate": [vp, vp, vp, vp],
        "leea_surr_stats": [vp, i64, vp, vp, vp, vp],
        "leea_surr_best_params": [vp, vp, i64],
        "leea_surr_generation_index": ([vp], u32),
        "leea_surr_profile_enable": [vp, i32],
        "leea_surr_profile_read": [vp, vp, vp],
        "leea_surr_destroy": ([vp], None),
        "leea_last_error": ([], ctypes.c_char_p),
        "leea_destroy": ([vp], None),
    }
    for name, spec in sig.items():
        fn = getattr(L, name)
        if isinstance(spec, tuple):
            fn.argtypes, fn.restype = spec
        else:
            fn.argtypes, fn.restype = spec, ctypes.c_int
    _lib = L
    return L


def exported_symbols() -> list[str]:
    """Names of the entry points the binding expects the library to export."""
    return ["leea_default_params", "leea_layout_num_params", "leea_padded_params", "leea_counts",
            "leea_init_population", "leea_rank", "leea_select", "leea_breed", "leea_breed_evaluate_u8",
            "leea_maxpool2x2", "leea_maxpool2x2_u8",
            "leea_evaluate",
            "leea_device_status", "leea_selftest_wait_timeout", "leea_evaluate_u8", "leea_generation_u8", "leea_generation_u8_host",
            "leea_philox_fill", "leea_normal_fill", "leea_create", "leea_generation",
            "leea_generation_host", "leea_fitness", "leea_raw_fitness", "leea_best_params",
            "leea_get_population", "leea_set_population", "leea_set_fitness", "leea_set_generation",
            "leea_get_selection", "leea_generation_index", "leea_num_params", "leea_get_sigma",
            "leea_set_sigma",
            "leea_profile_enable", "leea_profile_read", "leea_last_error", "leea_destroy",
            "leea_shadow_stride", "leea_make_shadow", "leea_shadow_scratch_bytes", "leea_evaluate_shadow_u8",
            "leea_get_shadow", "leea_evaluate_shadow_u8_noalloc",
            "leea_multi_create", "leea_multi_layout", "leea_multi_run_shape", "leea_multi_eval_launches",
            "leea_multi_batch_buffers",
            "leea_multi_generation_u8", "leea_multi_generation_u8_host", "leea_multi_fitness",
            "leea_multi_raw_fitness", "leea_multi_get_population", "leea_multi_set_population",
            "leea_multi_set_fitness", "leea_multi_set_generation", "leea_multi_get_selection",
            "leea_multi_get_shadow", "leea_multi_generation_index", "leea_multi_profile_enable",
            "leea_multi_profile_read", "leea_multi_destroy", "leea_tune_shadow_eval", "leea_tune_group_eval",
            "leea_surrogate_num_params", "leea_surrogate_init", "leea_surrogate_forward",
            "leea_surrogate_work_floats", "leea_surrogate_loss_grad", "leea_surrogate_adam",
            "leea_num_recipes", "leea_select_recipes", "leea_breed_entities", "leea_descriptors",
            "leea_surrogate_default_params", "leea_surr_create", "leea_surr_generation_u8",
            "leea_surr_generation_u8_host", "leea_surr_fitness", "leea_surr_raw_fitness", "leea_surr_get_population",
            "leea_surr_set_population", "leea_surr_set_fitness", "leea_surr_set_generation", "leea_surr_set_screen",
            "leea_surr_layout", "leea_surr_get_step", "leea_surr_get_surrogate", "leea_surr_stats",
            "leea_surr_generation_index", "leea_surr_profile_enable", "leea_surr_profile_read", "leea_surr_destroy",
            "leea_surr_best_params"]


def _check(rc: int) -> None:
    if rc != OK:
        msg = load_library().leea_last_error()
        raise LeeaError(rc, msg.decode() if msg else "")


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _dptr(t) -> int | None:
    """Device pointer of a torch CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _hp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- plain functions ------------------------------------------------------------
def leea_default_params() -> Params:
    s = leea_params()
    _check(load_library().leea_default_params(ctypes.byref(s)))
    return Params(**{f.name: getattr(s, f.name) for f in fields(Params)})


def leea_layout_num_params(dims) -> int:
    d = _dims(dims)
    return int(load_library().leea_layout_num_params(_hp(d), len(d)))


def leea_padded_params(dims) -> int:
    d = _dims(dims)
    return int(load_library().leea_padded_params(_hp(d), len(d)))


def leea_counts(pop: int, prm: Params) -> tuple[int, int, int, int]:
    vals = [ctypes.c_int32() for _ in range(4)]
    cp = prm.c_struct()
    _check(load_library().leea_counts(pop, ctypes.byref(cp), *[ctypes.byref(v) for v in vals]))
    return tuple(v.value for v in vals)


# ---- step entry points (torch CUDA tensors) ------------------------------------------
def leea_init_population(pop: int, dims, init: int, seed: int, pop_dev, stream=None) -> None:
    d = _dims(dims)
    _check(load_library().leea_init_population(pop, _hp(d), len(d), init, seed, _dptr(pop_dev), _stream(stream)))


def leea_rank(pop: int, f_adj_dev, order_dev, stream=None) -> None:
    _check(load_library().leea_rank(pop, _dptr(f_adj_dev), _dptr(order_dev), _stream(stream)))


def leea_select(pop: int, prm: Params, f_adj_dev, order_dev, seed: int, gen: int,
                par1_dev, par2_dev, kind_dev, f_inh_dev, stream=None) -> None:
    cp = prm.c_struct()
    _check(load_library().leea_select(pop, ctypes.byref(cp), _dptr(f_adj_dev), _dptr(order_dev), seed, gen,
                                      _dptr(par1_dev), _dptr(par2_dev), _dptr(kind_dev), _dptr(f_inh_dev),
                                      _stream(stream)))


def leea_breed(pop: int, dims, prm: Params, seed: int, gen: int, parents_dev, par1_dev, par2_dev,
               kind_dev, children_dev, stream=None) -> None:
    d = _dims(dims)
    cp = prm.c_struct()
    _check(load_library().leea_breed(pop, _hp(d), len(d), ctypes.byref(cp), seed, gen, _dptr(parents_dev),
                                     _dptr(par1_dev), _dptr(par2_dev), _dptr(kind_dev), _dptr(children_dev),
                                     _stream(stream)))


def leea_maxpool2x2(batch: int, h: int, w: int, x_dev, out_dev, stream=None) -> None:
    """2x2 max-pooling of [batch][h*w] images (float32 or uint8 tensors) into [batch][(h/2)*(w/2)]."""
    fn = load_library().leea_maxpool2x2_u8 if x_dev.dtype.itemsize == 1 else load_library().leea_maxpool2x2
    _check(fn(int(batch), int(h), int(w), _dptr(x_dev), _dptr(out_dev), _stream(stream)))


def leea_breed_evaluate_u8(pop: int, dims, prm: Params, seed: int, gen: int, parents_dev, par1_dev, par2_dev,
                           kind_dev, children_dev, x_u8_dev, x_div: float, y_dev, batch: int, alpha: float, f_inh_dev,
                           f_raw_dev, f_adj_dev=None, correct_dev=None, stream=None) -> None:
    d = _dims(dims)
    cp = prm.c_struct()
    _check(load_library().leea_breed_evaluate_u8(pop, _hp(d), len(d), ctypes.byref(cp), seed, gen, _dptr(parents_dev),
                                                 _dptr(par1_dev), _dptr(par2_dev), _dptr(kind_dev),
                                                 _dptr(children_dev), _dptr(x_u8_dev), float(x_div), _dptr(y_dev),
                                                 batch, float(alpha), _dptr(f_inh_dev), _dptr(f_raw_dev),
                                                 _dptr(f_adj_dev), _dptr(correct_dev), _stream(stream)))


def leea_evaluate(pop: int, dims, pop_dev, x_dev, y_dev, batch: int, alpha: float, f_inh_dev,
                  f_raw_dev, f_adj_dev=None, correct_dev=None, eval_path: int = EVAL_AUTO, stream=None) -> None:
    d = _dims(dims)
    _check(load_library().leea_evaluate(pop, _hp(d), len(d), _dptr(pop_dev), _dptr(x_dev), _dptr(y_dev), batch,
                                        float(alpha), _dptr(f_inh_dev), _dptr(f_raw_dev), _dptr(f_adj_dev),
                                        _dptr(correct_dev), int(eval_path), _stream(stream)))


def leea_evaluate_u8(pop: int, dims, pop_dev, x_u8_dev, x_div: float, y_dev, batch: int, alpha: float, f_inh_dev,
                     f_raw_dev, f_adj_dev=None, correct_dev=None, eval_path: int = EVAL_AUTO, stream=None) -> None:
    d = _dims(dims)
    _check(load_library().leea_evaluate_u8(pop, _hp(d), len(d), _dptr(pop_dev), _dptr(x_u8_dev), float(x_div),
                                           _dptr(y_dev), batch, float(alpha), _dptr(f_inh_dev), _dptr(f_raw_dev),
                                           _dptr(f_adj_dev), _dptr(correct_dev), int(eval_path), _stream(stream)))


def leea_shadow_stride(dims, precision: int) -> int:
    d = _dims(dims)
    return int(load_library().leea_shadow_stride(_hp(d), len(d), int(precision)))


def leea_make_shadow(pop: int, dims, precision: int, pop_dev, shadow_dev, scale_exp_dev, amax_dev,
                     stream=None) -> None:
    d = _dims(dims)
    _check(load_library().leea_make_shadow(pop, _hp(d), len(d), int(precision), _dptr(pop_dev), _dptr(shadow_dev),
                                           _dptr(scale_exp_dev), _dptr(amax_dev), _stream(stream)))


def leea_shadow_scratch_bytes(pop: int, batch: int) -> int:
    return int(load_library().leea_shadow_scratch_bytes(pop, batch))


def leea_evaluate_shadow_u8(pop: int, dims, pop_dev, precision: int, shadow_dev, scale_exp_dev, x_u8_dev,
                            x_div: float, y_dev, batch: int, alpha: float, f_inh_dev, f_raw_dev, f_adj_dev=None,
                            correct_dev=None, scratch_dev=None, stream=None) -> None:
    d = _dims(dims)
    nbytes = 0 if scratch_dev is None else scratch_dev.numel() * scratch_dev.element_size()
    _check(load_library().leea_evaluate_shadow_u8(
        pop, _hp(d), len(d), _dptr(pop_dev), int(precision), _dptr(shadow_dev), _dptr(scale_exp_dev),
        _dptr(x_u8_dev), float(x_div), _dptr(y_dev), batch, float(alpha), _dptr(f_inh_dev), _dptr(f_raw_dev),
        _dptr(f_adj_dev), _dptr(correct_dev), _dptr(scratch_dev), nbytes, _stream(stream)))


NOALLOC_SCRATCH_BYTES = 1 << 20


def leea_evaluate_shadow_u8_noalloc(pop: int, dims, pop_dev, precision: int, shadow_dev, scale_exp_dev, x_u8_dev,
                                    x_div: float, y_dev, batch: int, alpha: float, f_inh_dev, f_raw_dev,
                                    f_adj_dev=None, correct_dev=None, stream=None) -> None:
    """leea_evaluate_shadow_u8 with the library's static scratch (allocates nothing)."""
    d = _dims(dims)
    _check(load_library().leea_evaluate_shadow_u8_noalloc(
        pop, _hp(d), len(d), _dptr(pop_dev), int(precision), _dptr(shadow_dev), _dptr(scale_exp_dev),
        _dptr(x_u8_dev), float(x_div), _dptr(y_dev), batch, float(alpha), _dptr(f_inh_dev), _dptr(f_raw_dev),
        _dptr(f_adj_dev), _dptr(correct_dev), _stream(stream)))


def leea_device_status(stream=None) -> int:
    """Synchronises, reads and clears the device status word; raises on a timeout flag."""
    flags = ctypes.c_uint32()
    _check(load_library().leea_device_status(_stream(stream), ctypes.byref(flags)))
    return flags.value


def leea_selftest_wait_timeout(limit_us: int, stream=None) -> None:
    """Enqueues a bounded wait that runs out after limit_us (the failure path, no fault)."""
    _check(load_library().leea_selftest_wait_timeout(int(limit_us), _stream(stream)))


def leea_philox_fill(seed: int, tag: int, gen: int, ent: int, n0: int, count: int, out_dev, stream=None) -> None:
    _check(load_library().leea_philox_fill(seed, tag, gen, ent, n0, count, _dptr(out_dev), _stream(stream)))


def leea_normal_fill(seed: int, tag: int, gen: int, ent: int, n0: int, count: int, out_dev, stream=None) -> None:
    _check(load_library().leea_normal_fill(seed, tag, gen, ent, n0, count, _dptr(out_dev), _stream(stream)))


# ---- the state object --------------------------------------------------------------
class LeeaState:
    """Algorithm 1 as a library-owned object (``leea_create`` ... ``leea_destroy``)."""

    def __init__(self, pop: int, dims, prm: Params, seed: int, stream=None):
        self.lib = load_library()
        self.pop = pop
        self.dims = _dims(dims)
        self._cp = prm.c_struct()
        h = ctypes.c_void_p()
        _check(self.lib.leea_create(pop, _hp(self.dims), len(self.dims), ctypes.byref(self._cp), seed,
                                    _stream(stream), ctypes.byref(h)))
        self._h = h
        self.c = int(self.lib.leea_num_params(h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            self.lib.leea_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def leea_generation(self, x_dev, y_dev) -> None:
        _check(self.lib.leea_generation(self._h, _dptr(x_dev), _dptr(y_dev), int(y_dev.shape[0])))

    def leea_generation_u8(self, x_u8_dev, y_dev, x_div: float = 255.0) -> None:
        _check(self.lib.leea_generation_u8(self._h, _dptr(x_u8_dev), float(x_div), _dptr(y_dev), int(y_dev.shape[0])))

    def _host_batch(self, x_host, y_host, x_dtype: str):
        """Host pointers and batch size of a host minibatch, after the checks the C call cannot make:
        C-contiguous CPU buffers of the right dtypes, x holding batch * d_0 elements."""
        bufs = []
        for name, arr, want in (("x", x_host, x_dtype), ("y", y_host, "int32")):
            if hasattr(arr, "data_ptr"):  # torch tensor
                if arr.is_cuda:
                    raise ValueError(f"{name} must be a host (CPU) tensor")
                if str(arr.dtype).replace("torch.", "") != want:
                    raise ValueError(f"{name} must be {want}, got {arr.dtype}")
                if not arr.is_contiguous():
                    raise ValueError(f"{name} must be contiguous")
                bufs.append((arr.data_ptr(), int(arr.numel()), tuple(arr.shape)))
            else:
                a = np.asarray(arr)
                if a.dtype != np.dtype(want):
                    raise ValueError(f"{name} must be {want}, got {a.dtype}")
                if not a.flags["C_CONTIGUOUS"]:
                    raise ValueError(f"{name} must be C-contiguous")
                bufs.append((a.ctypes.data, int(a.size), a.shape))
        (xp, xn, _), (yp, yn, yshape) = bufs
        if len(yshape) != 1:
            raise ValueError("y must be one-dimensional (one label per sample)")
        if xn != yn * self.dims[0]:
            raise ValueError(f"x holds {xn} elements; batch {yn} x d_0 {self.dims[0]} = {yn * self.dims[0]} expected")
        return xp, yp, yn

    def leea_generation_u8_host(self, x_u8_host, y_host, x_div: float = 255.0) -> None:
        """x_u8_host uint8[batch][d_0], y_host int32[batch]: CPU torch tensors (ideally pinned) or numpy arrays."""
        xp, yp, batch = self._host_batch(x_u8_host, y_host, "uint8")
        _check(self.lib.leea_generation_u8_host(self._h, xp, float(x_div), yp, batch))

    def leea_generation_host(self, x_host, y_host) -> None:
        """x_host float32[batch][d_0], y_host int32[batch]: CPU torch tensors (ideally pinned) or numpy arrays."""
        xp, yp, batch = self._host_batch(x_host, y_host, "float32")
        _check(self.lib.leea_generation_host(self._h, xp, yp, batch))

    def leea_fitness(self, with_correct: bool = False):
        f = np.empty(self.pop, dtype=np.float32)
        cor = np.empty(self.pop, dtype=np.int32) if with_correct else None
        _check(self.lib.leea_fitness(self._h, _hp(f), None if cor is None else _hp(cor)))
        return (f, cor) if with_correct else f

    def leea_raw_fitness(self) -> np.ndarray:
        f = np.empty(self.pop, dtype=np.float32)
        _check(self.lib.leea_raw_fitness(self._h, _hp(f)))
        return f

    def leea_best_params(self) -> np.ndarray:
        out = np.empty(self.c, dtype=np.float32)
        _check(self.lib.leea_best_params(self._h, _hp(out), self.c))
        return out

    def leea_get_population(self) -> np.ndarray:
        out = np.empty((self.pop, self.c), dtype=np.float32)
        _check(self.lib.leea_get_population(self._h, _hp(out)))
        return out

    def leea_set_population(self, popv) -> None:
        a = np.ascontiguousarray(np.asarray(popv, dtype=np.float32))
        assert a.shape == (self.pop, self.c)
        _check(self.lib.leea_set_population(self._h, _hp(a)))

    def leea_set_fitness(self, f_adj) -> None:
        a = np.ascontiguousarray(np.asarray(f_adj, dtype=np.float32))
        _check(self.lib.leea_set_fitness(self._h, _hp(a)))

    def leea_set_generation(self, gen: int, evaluated: bool) -> None:
        _check(self.lib.leea_set_generation(self._h, gen, int(evaluated)))

    def leea_get_selection(self):
        """(order, par1, par2, kind, f_inh) of the last breed."""
        ints = [np.empty(self.pop, dtype=np.int32) for _ in range(4)]
        f_inh = np.empty(self.pop, dtype=np.float32)
        _check(self.lib.leea_get_selection(self._h, *[_hp(a) for a in ints], _hp(f_inh)))
        return (*ints, f_inh)

    def leea_get_shadow(self, precision: int):
        """(shadow uint8[pop][stride] in the tiled layout, scale_exp int32[pop], amax float32[pop])."""
        sh = np.empty((self.pop, leea_shadow_stride(self.dims, precision)), dtype=np.uint8)
        se = np.empty(self.pop, dtype=np.int32)
        am = np.empty(self.pop, dtype=np.float32)
        _check(self.lib.leea_get_shadow(self._h, _hp(sh), _hp(se), _hp(am)))
        return sh, se, am

    def leea_get_sigma(self) -> np.ndarray:
        """Sigma genes (SIGMA_SELF) or the next breed's strength, float32[pop]."""
        out = np.empty(self.pop, dtype=np.float32)
        _check(self.lib.leea_get_sigma(self._h, _hp(out)))
        return out

    def leea_set_sigma(self, sigma) -> None:
        a = np.ascontiguousarray(np.asarray(sigma, dtype=np.float32))
        assert a.shape == (self.pop,)
        _check(self.lib.leea_set_sigma(self._h, _hp(a)))

    @property
    def gen(self) -> int:
        return int(self.lib.leea_generation_index(self._h))

    def leea_profile_enable(self, on: bool = True) -> None:
        _check(self.lib.leea_profile_enable(self._h, int(on)))

    def leea_profile_read(self):
        """{stage: (ms_total, launches)} since the last read."""
        ms = np.zeros(NUM_STAGES, dtype=np.float64)
        n = np.zeros(NUM_STAGES, dtype=np.int64)
        _check(self.lib.leea_profile_read(self._h, _hp(ms), _hp(n)))
        return {STAGES[k]: (float(ms[k]), int(n[k])) for k in range(NUM_STAGES)}


# ---- the batching form -------------------------------------------------------------
@dataclass
class RunSpec:
    """One run of the batching form (fields of ``leea_run_spec``)."""
    pop: int
    hidden: int
    batch: int
    chunk: int = 0
    seed: int = 0
    group: int = 0


class MultiRun:
    """Many independent runs advanced together (``leea_multi_create`` ... ``leea_multi_destroy``).
    Minibatches and per-individual results are packed over the runs (see ``layout``)."""

    def __init__(self, specs, d_in: int, d_out: int, prm: Params, stream=None):
        self.lib = load_library()
        self.specs = list(specs)
        self.n_runs = len(self.specs)
        self.d_in, self.d_out = d_in, d_out
        arr = (leea_run_spec * self.n_runs)(*[leea_run_spec(sp.pop, sp.hidden, sp.batch, sp.chunk, sp.group, sp.seed)
                                               for sp in self.specs])
        self._cp = prm.c_struct()
        h = ctypes.c_void_p()
        _check(self.lib.leea_multi_create(self.n_runs, ctypes.cast(arr, ctypes.c_void_p), d_in, d_out,
                                          ctypes.byref(self._cp), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.batch_off = np.zeros(self.n_runs, dtype=np.int64)
        self.pop_off = np.zeros(self.n_runs, dtype=np.int64)
        tr, tp = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.leea_multi_layout(h, _hp(self.batch_off), _hp(self.pop_off), ctypes.byref(tr),
                                          ctypes.byref(tp)))
        self.total_rows, self.total_pop = tr.value, tp.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            self.lib.leea_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run_shape(self, run: int):
        """(chunk, n_chunks, m_tiles, group) of run `run`'s evaluation."""
        v = [ctypes.c_int32() for _ in range(4)]
        _check(self.lib.leea_multi_run_shape(self._h, run, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def eval_launches(self) -> int:
        """Kernels one evaluation of all runs launches."""
        v = ctypes.c_int32()
        _check(self.lib.leea_multi_eval_launches(self._h, ctypes.byref(v)))
        return int(v.value)

    def batch_buffers(self):
        x, y = ctypes.c_void_p(), ctypes.c_void_p()
        _check(self.lib.leea_multi_batch_buffers(self._h, ctypes.byref(x), ctypes.byref(y)))
        return x.value, y.value

    def generation_u8(self, x_dev, y_dev, x_div: float = 255.0) -> None:
        _check(self.lib.leea_multi_generation_u8(self._h, _dptr(x_dev), float(x_div), _dptr(y_dev)))

    def generation_u8_host(self, x_host, y_host, x_div: float = 255.0) -> None:
        xh = x_host if not isinstance(x_host, np.ndarray) else np.ascontiguousarray(x_host, dtype=np.uint8)
        yh = y_host if not isinstance(y_host, np.ndarray) else np.ascontiguousarray(y_host, dtype=np.int32)
        xp = _hp(xh) if isinstance(xh, np.ndarray) else xh.data_ptr()
        yp = _hp(yh) if isinstance(yh, np.ndarray) else yh.data_ptr()
        _check(self.lib.leea_multi_generation_u8_host(self._h, xp, float(x_div), yp))

    def fitness(self, with_correct: bool = False):
        f = np.empty(self.total_pop, dtype=np.float32)
        cor = np.empty(self.total_pop, dtype=np.int32) if with_correct else None
        _check(self.lib.leea_multi_fitness(self._h, _hp(f), None if cor is None else _hp(cor)))
        return (f, cor) if with_correct else f

    def raw_fitness(self) -> np.ndarray:
        f = np.empty(self.total_pop, dtype=np.float32)
        _check(self.lib.leea_multi_raw_fitness(self._h, _hp(f)))
        return f

    def run_slice(self, run: int) -> slice:
        return slice(int(self.pop_off[run]), int(self.pop_off[run]) + self.specs[run].pop)

    def rows_slice(self, run: int) -> slice:
        return slice(int(self.batch_off[run]), int(self.batch_off[run]) + self.specs[run].batch)

    def num_params(self, run: int) -> int:
        return leea_layout_num_params([self.d_in, self.specs[run].hidden, self.d_out])

    def get_population(self, run: int) -> np.ndarray:
        out = np.empty((self.specs[run].pop, self.num_params(run)), dtype=np.float32)
        _check(self.lib.leea_multi_get_population(self._h, run, _hp(out)))
        return out

    def set_population(self, run: int, popv) -> None:
        a = np.ascontiguousarray(np.asarray(popv, dtype=np.float32))
        assert a.shape == (self.specs[run].pop, self.num_params(run))
        _check(self.lib.leea_multi_set_population(self._h, run, _hp(a)))

    def set_fitness(self, f_adj) -> None:
        a = np.ascontiguousarray(np.asarray(f_adj, dtype=np.float32))
        assert a.shape == (self.total_pop,)
        _check(self.lib.leea_multi_set_fitness(self._h, _hp(a)))

    def set_generation(self, gen: int, evaluated: bool) -> None:
        _check(self.lib.leea_multi_set_generation(self._h, gen, int(evaluated)))

    def get_selection(self, run: int):
        n = self.specs[run].pop
        ints = [np.empty(n, dtype=np.int32) for _ in range(4)]
        f_inh = np.empty(n, dtype=np.float32)
        _check(self.lib.leea_multi_get_selection(self._h, run, *[_hp(a) for a in ints], _hp(f_inh)))
        return (*ints, f_inh)

    def get_shadow(self, run: int, precision: int):
        sp = self.specs[run]
        sh = np.empty((sp.pop, leea_shadow_stride([self.d_in, sp.hidden, self.d_out], precision)), dtype=np.uint8)
        se = np.empty(sp.pop, dtype=np.int32)
        am = np.empty(sp.pop, dtype=np.float32)
        _check(self.lib.leea_multi_get_shadow(self._h, run, _hp(sh), _hp(se), _hp(am)))
        return sh, se, am

    @property
    def gen(self) -> int:
        return int(self.lib.leea_multi_generation_index(self._h))

    def profile_enable(self, on: bool = True) -> None:
        _check(self.lib.leea_multi_profile_enable(self._h, int(on)))

    def profile_read(self):
        ms = np.zeros(NUM_STAGES, dtype=np.float64)
        n = np.zeros(NUM_STAGES, dtype=np.int64)
        _check(self.lib.leea_multi_profile_read(self._h, _hp(ms), _hp(n)))
        return {STAGES[k]: (float(ms[k]), int(n[k])) for k in range(NUM_STAGES)}


def leea_tune_shadow_eval(precision: int, d_in: int, hidden: int, d_out: int, batch: int, pop: int, chunk: int,
                          reps: int = 5) -> float:
    ms = ctypes.c_float()
    _check(load_library().leea_tune_shadow_eval(precision, d_in, hidden, d_out, batch, pop, chunk, reps,
                                                ctypes.byref(ms)))
    return float(ms.value)


def leea_tune_group_eval(precision: int, d_in: int, hidden: int, d_out: int, batch: int, pop: int, group: int,
                         reps: int = 5) -> float:
    ms = ctypes.c_float()
    _check(load_library().leea_tune_group_eval(precision, d_in, hidden, d_out, batch, pop, group, reps,
                                               ctypes.byref(ms)))
    return float(ms.value)


# ---- surrogate MLP (row level) ------------------------------------------------------
def leea_surrogate_num_params(d_in: int, h1: int, h2: int) -> int:
    return int(load_library().leea_surrogate_num_params(d_in, h1, h2))


def leea_surrogate_init(d_in: int, h1: int, h2: int, seed: int, theta_dev, stream=None) -> None:
    _check(load_library().leea_surrogate_init(d_in, h1, h2, seed, _dptr(theta_dev), _stream(stream)))


def leea_surrogate_forward(n: int, d_in: int, h1: int, h2: int, theta_dev, x_dev, y_dev, stream=None) -> None:
    _check(load_library().leea_surrogate_forward(n, d_in, h1, h2, _dptr(theta_dev), _dptr(x_dev), _dptr(y_dev),
                                                 _stream(stream)))


def leea_surrogate_work_floats(n: int, h1: int, h2: int) -> int:
    return int(load_library().leea_surrogate_work_floats(n, h1, h2))


def leea_surrogate_loss_grad(n: int, d_in: int, h1: int, h2: int, theta_dev, x_dev, t_dev, loss_dev, grad_dev,
                             work_dev, stream=None) -> None:
    _check(load_library().leea_surrogate_loss_grad(n, d_in, h1, h2, _dptr(theta_dev), _dptr(x_dev), _dptr(t_dev),
                                                   _dptr(loss_dev), _dptr(grad_dev), _dptr(work_dev),
                                                   work_dev.numel(), _stream(stream)))


def leea_surrogate_adam(n_params: int, theta_dev, grad_dev, m_dev, v_dev, step: int, lr: float = 1e-3,
                        beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    _check(load_library().leea_surrogate_adam(n_params, _dptr(theta_dev), _dptr(grad_dev), _dptr(m_dev),
                                              _dptr(v_dev), step, float(lr), float(beta1), float(beta2), float(eps),
                                              _stream(stream)))


# ---- recipes and descriptors (surrogate form) ---------------------------------------
def leea_num_recipes(pop: int, prm: Params, mult: int) -> int:
    cp = prm.c_struct()
    return int(load_library().leea_num_recipes(pop, ctypes.byref(cp), mult))


def leea_select_recipes(pop: int, prm: Params, f_adj_dev, order_dev, seed: int, gen: int, mult: int, par1_dev,
                        par2_dev, kind_dev, f_inh_dev, entity_dev, stream=None) -> None:
    cp = prm.c_struct()
    _check(load_library().leea_select_recipes(pop, ctypes.byref(cp), _dptr(f_adj_dev), _dptr(order_dev), seed, gen,
                                              mult, _dptr(par1_dev), _dptr(par2_dev), _dptr(kind_dev),
                                              _dptr(f_inh_dev), _dptr(entity_dev), _stream(stream)))


def leea_breed_entities(n_parents: int, dims, prm: Params, seed: int, gen: int, parents_dev, par1_dev, par2_dev,
                        kind_dev, entity_dev, n_children: int, children_dev, stream=None) -> None:
    d = _dims(dims)
    cp = prm.c_struct()
    _check(load_library().leea_breed_entities(n_parents, _hp(d), len(d), ctypes.byref(cp), seed, gen,
                                              _dptr(parents_dev), _dptr(par1_dev), _dptr(par2_dev), _dptr(kind_dev),
                                              _dptr(entity_dev), n_children, _dptr(children_dev), _stream(stream)))


def leea_descriptors(n_parents: int, dims, prm: Params, seed: int, gen: int, parents_dev, f_adj_dev, par1_dev,
                     par2_dev, kind_dev, f_inh_dev, entity_dev, n: int, probe_dev, n_probe: int, desc_dev,
                     stream=None) -> None:
    d = _dims(dims)
    cp = prm.c_struct()
    _check(load_library().leea_descriptors(n_parents, _hp(d), len(d), ctypes.byref(cp), seed, gen, _dptr(parents_dev),
                                           _dptr(f_adj_dev), _dptr(par1_dev), _dptr(par2_dev), _dptr(kind_dev),
                                           _dptr(f_inh_dev), _dptr(entity_dev), n, _dptr(probe_dev), n_probe,
                                           _dptr(desc_dev), _stream(stream)))


# ---- the surrogate form as a state object ---------------------------------------------
SURR_STAGES = ("recipes", "scores", "breed", "evaluate", "training")


@dataclass
class SurrogateParams:
    """Fields of ``leea_surrogate_params``; defaults as ``leea_surrogate_default_params``."""
    mult: int = 4
    n_probe: int = 32
    hidden1: int = 64
    hidden2: int = 64
    train_steps: int = 16
    train_batch: int = 256
    history: int = 4
    warmup: int = 3
    lr: float = 1e-3
    audit_frac: float = 0.05
    min_spearman: float = 0.2
    seed: int = 0x5EED5EED

    def c_struct(self) -> leea_surrogate_params:
        return leea_surrogate_params(**{f.name: getattr(self, f.name) for f in fields(SurrogateParams)})


class SurrState:
    """The surrogate form (``leea_surr_create`` ... ``leea_surr_destroy``)."""

    def __init__(self, pop: int, dims, prm: Params, sp: SurrogateParams, seed: int, probe, stream=None):
        self.lib = load_library()
        self.pop = pop
        self.dims = _dims(dims)
        self._cp, self._sp = prm.c_struct(), sp.c_struct()
        self.probe = np.ascontiguousarray(np.asarray(probe, dtype=np.float32))
        h = ctypes.c_void_p()
        _check(self.lib.leea_surr_create(pop, _hp(self.dims), len(self.dims), ctypes.byref(self._cp),
                                         ctypes.byref(self._sp), seed, _hp(self.probe), _stream(stream),
                                         ctypes.byref(h)))
        self._h = h
        self.c = leea_layout_num_params(self.dims)
        v = [ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()]
        _check(self.lib.leea_surr_layout(h, *[ctypes.byref(x) for x in v]))
        self.n_recipes, self.n_audit, self.width, self.n_theta = (x.value for x in v)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            self.lib.leea_surr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def generation_u8(self, x_dev, y_dev, x_div: float = 255.0) -> None:
        _check(self.lib.leea_surr_generation_u8(self._h, _dptr(x_dev), float(x_div), _dptr(y_dev), int(y_dev.numel())))

    def generation_u8_host(self, x_host, y_host, x_div: float = 255.0) -> None:
        _check(self.lib.leea_surr_generation_u8_host(self._h, x_host.data_ptr(), float(x_div), y_host.data_ptr(),
                                                     int(y_host.numel())))

    def fitness(self, with_correct: bool = False):
        f = np.empty(self.pop, dtype=np.float32)
        cor = np.empty(self.pop, dtype=np.int32) if with_correct else None
        _check(self.lib.leea_surr_fitness(self._h, _hp(f), None if cor is None else _hp(cor)))
        return (f, cor) if with_correct else f

    def raw_fitness(self):
        f = np.empty(self.pop, dtype=np.float32)
        fa = np.empty(max(self.n_audit, 1), dtype=np.float32)
        _check(self.lib.leea_surr_raw_fitness(self._h, _hp(f), _hp(fa)))
        return f, fa[:self.n_audit]

    def get_population(self) -> np.ndarray:
        out = np.empty((self.pop, self.c), dtype=np.float32)
        _check(self.lib.leea_surr_get_population(self._h, _hp(out)))
        return out

    def set_population(self, popv) -> None:
        a = np.ascontiguousarray(np.asarray(popv, dtype=np.float32))
        _check(self.lib.leea_surr_set_population(self._h, _hp(a)))

    def set_fitness(self, f_adj) -> None:
        a = np.ascontiguousarray(np.asarray(f_adj, dtype=np.float32))
        _check(self.lib.leea_surr_set_fitness(self._h, _hp(a)))

    def set_generation(self, gen: int, evaluated: bool) -> None:
        _check(self.lib.leea_surr_set_generation(self._h, gen, int(evaluated)))

    def set_screen(self, on: bool) -> None:
        _check(self.lib.leea_surr_set_screen(self._h, int(on)))

    def get_step(self) -> dict:
        R, P = self.n_recipes, self.pop
        out = dict(r_par1=np.empty(R, np.int32), r_par2=np.empty(R, np.int32), r_kind=np.empty(R, np.int32),
                   r_f_inh=np.empty(R, np.float32), r_entity=np.empty(R, np.uint32),
                   desc=np.empty((R, self.width), np.float32), pred=np.empty(R, np.float32),
                   row_recipe=np.empty(self.n_rows(), np.int32),
                   c_par1=np.empty(P, np.int32), c_par2=np.empty(P, np.int32), c_kind=np.empty(P, np.int32),
                   c_entity=np.empty(P, np.uint32), c_f_inh=np.empty(P, np.float32))
        keys = ["r_par1", "r_par2", "r_kind", "r_f_inh", "r_entity", "desc", "pred", "row_recipe", "c_par1", "c_par2",
                "c_kind", "c_entity", "c_f_inh"]
        _check(self.lib.leea_surr_get_step(self._h, *[_hp(out[k]) for k in keys]))
        return out

    def n_rows(self) -> int:
        return self.n_recipes // max(1, self._sp.mult) + self.n_audit

    def best_params(self) -> np.ndarray:
        out = np.empty(self.c, dtype=np.float32)
        _check(self.lib.leea_surr_best_params(self._h, _hp(out), self.c))
        return out

    def get_surrogate(self):
        th = np.empty(self.n_theta, np.float32)
        mu, sd = np.empty(self.width, np.float32), np.empty(self.width, np.float32)
        _check(self.lib.leea_surr_get_surrogate(self._h, _hp(th), _hp(mu), _hp(sd)))
        return th, mu, sd

    def stats(self, n_max: int = 1 << 16):
        rho = np.empty(n_max, np.float32)
        scr = np.empty(n_max, np.int32)
        loss = np.empty(n_max, np.float32)
        n = ctypes.c_int64()
        _check(self.lib.leea_surr_stats(self._h, n_max, _hp(rho), _hp(scr), _hp(loss), ctypes.byref(n)))
        k = n.value
        return rho[:k], scr[:k], loss[:k]

    @property
    def gen(self) -> int:
        return int(self.lib.leea_surr_generation_index(self._h))

    def profile_enable(self, on: bool = True) -> None:
        _check(self.lib.leea_surr_profile_enable(self._h, int(on)))

    def profile_read(self):
        ms = np.zeros(len(SURR_STAGES), dtype=np.float64)
        n = ctypes.c_int64()
        _check(self.lib.leea_surr_profile_read(self._h, _hp(ms), ctypes.byref(n)))
        return {SURR_STAGES[k]: float(ms[k]) for k in range(len(SURR_STAGES))}, int(n.value)
