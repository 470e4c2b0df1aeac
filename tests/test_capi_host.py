"""The CUDA library builds for sm_103a, loads, exports every entry point that
include/leea.h declares, and its host-only logic (layout, operator counts,
argument checking) agrees with the oracle.  No compute call is made."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1806_09819_gb300 import build as B
from paper_1806_09819_gb300 import leea

HEADER = os.path.join(B.INCLUDE, "leea.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return leea.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(leea_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_what_the_binding_binds():
    assert declared_functions() == sorted(leea.exported_symbols())


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    # and nothing else under the leea_ prefix is required by the binding
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (leea_\w+)", out))
    assert set(declared_functions()) <= exported


def test_default_params_are_the_papers(lib, oracle_mod):
    d = leea.leea_default_params()
    o = oracle_mod.Params()
    for f in ("xo_op", "sel_op", "tour_k", "n_elite", "init", "precision"):
        assert getattr(d, f) == getattr(o, f)
    for f in ("xo_gene_p", "rho", "p_e", "p_c", "sigma", "mut_rate", "alpha"):
        assert np.float32(getattr(d, f)) == np.float32(getattr(o, f))
    # Constant mutation strength by default; the decay rate and tau (which the
    # paper does not state) are the same readings on both sides.
    assert d.sigma_ctl == o.sigma_ctl == leea.SIGMA_CONST
    assert np.float32(d.sigma_k) == np.float32(o.sigma_k) and np.float32(d.tau) == np.float32(o.tau)


@pytest.mark.parametrize("dims", [[784, 112, 10], [784, 32, 10], [2, 2, 2], [196, 256, 128, 64, 10], [3, 1]])
def test_layout_matches_oracle(lib, oracle_mod, dims):
    c = leea.leea_layout_num_params(dims)
    assert c == oracle_mod.num_params(dims)
    cp = leea.leea_padded_params(dims)
    assert cp % 32 == 0 and c <= cp < c + 32


def test_invalid_dims(lib):
    assert leea.leea_layout_num_params([784]) == -1
    assert leea.leea_layout_num_params([784, 0, 10]) == -1


def test_counts_match_oracle(lib, oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(300):
        pop = int(rng.integers(1, 5000))
        kw = dict(p_e=float(rng.uniform(0, 0.3)), p_c=float(rng.uniform(0, 1)), rho=float(rng.uniform(0.01, 1)),
                  n_elite=int(rng.choice([-1, 0, 1, 3])))
        assert leea.leea_counts(pop, leea.Params(**kw)) == oracle_mod.counts(pop, oracle_mod.Params(**kw))


def test_argument_errors_are_reported_before_any_work(lib):
    with pytest.raises(leea.LeeaError) as e:
        leea.leea_counts(0, leea.Params())
    assert e.value.status == leea.EINVAL and "pop" in str(e.value)
    with pytest.raises(leea.LeeaError) as e:
        leea.leea_counts(10, leea.Params(rho=0.0))
    assert "rho" in str(e.value)
    # leea_create validates before touching the device.
    d = np.array([784, 112, 10], dtype=np.int32)
    h = ctypes.c_void_p()
    bad = leea.Params(sigma=-1.0).c_struct()
    rc = lib.leea_create(10, d.ctypes.data_as(ctypes.c_void_p), 3, ctypes.byref(bad), 1, None, ctypes.byref(h))
    assert rc == leea.EINVAL and h.value is None
    assert b"sigma" in lib.leea_last_error()
    for kw, word in ((dict(sigma_ctl=3), b"sigma_ctl"), (dict(sigma_ctl=leea.SIGMA_DECAY, sigma_k=0.0), b"sigma_k"),
                     (dict(sigma_ctl=leea.SIGMA_SELF, tau=-0.5), b"tau")):
        bad = leea.Params(**kw).c_struct()
        rc = lib.leea_create(10, d.ctypes.data_as(ctypes.c_void_p), 3, ctypes.byref(bad), 1, None, ctypes.byref(h))
        assert rc == leea.EINVAL and h.value is None
        assert word in lib.leea_last_error()
    # Outside the state object the mutation strength is a constant argument.
    self_p = leea.Params(sigma_ctl=leea.SIGMA_SELF).c_struct()
    n = ctypes.c_void_p(16)  # never dereferenced: the check comes first
    rc = lib.leea_select(10, ctypes.byref(self_p), n, n, 1, 1, n, n, n, n, None)
    assert rc == leea.EINVAL and b"sigma_ctl" in lib.leea_last_error()
    # Several hidden layers: every layer input and hidden width <= 256, FP32 only.
    good = leea.Params().c_struct()
    d4 = np.array([784, 256, 128, 64, 10], dtype=np.int32)
    rc = lib.leea_create(10, d4.ctypes.data_as(ctypes.c_void_p), 5, ctypes.byref(good), 1, None, ctypes.byref(h))
    assert rc == leea.EINVAL and b"256" in lib.leea_last_error()
    d4 = np.array([196, 256, 128, 64, 10], dtype=np.int32)
    bf16 = leea.Params(precision=1).c_struct()
    rc = lib.leea_create(10, d4.ctypes.data_as(ctypes.c_void_p), 5, ctypes.byref(bf16), 1, None, ctypes.byref(h))
    assert rc == leea.EINVAL
    # The evaluation paths: SMALL (the single-launch generation) is the last one; it takes FP32
    # populations of nets with one hidden layer.
    assert leea.leea_counts(10, leea.Params(eval_path=leea.EVAL_SMALL))[0] >= 0
    with pytest.raises(leea.LeeaError) as e:
        leea.leea_counts(10, leea.Params(eval_path=leea.EVAL_SMALL + 1))
    assert "eval_path" in str(e.value)
    with pytest.raises(leea.LeeaError) as e:
        leea.leea_counts(10, leea.Params(eval_path=leea.EVAL_SMALL, precision=1))
    assert "single-launch" in str(e.value)
    small_deep = leea.Params(eval_path=leea.EVAL_SMALL).c_struct()
    rc = lib.leea_create(10, d4.ctypes.data_as(ctypes.c_void_p), 5, ctypes.byref(small_deep), 1, None, ctypes.byref(h))
    assert rc == leea.EINVAL and h.value is None


def test_oracle_and_library_share_no_code():
    # The two sides are separate translation units with separate headers.
    csrc = B.CSRC
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "leea_oracle" not in text and "oracle/" not in text
    here = os.path.dirname(os.path.abspath(__file__))
    otext = open(os.path.join(here, "..", "oracle", "leea_oracle.c")).read()
    assert "philox.cuh" not in otext and "leea.h\"" not in otext


def test_autotune_candidates():
    from paper_1806_09819_gb300 import autotune
    # 784 inputs: the batch tile takes 400 TMEM columns in either precision, leaving 112
    assert autotune.max_chunk(1, 784) == 112 and autotune.max_chunk(2, 784) == 112
    assert autotune.max_chunk(1, 64) == 128
    assert autotune.effective_chunk(256, 112) == 96      # 3 equal chunks
    assert autotune.effective_chunk(112, 112) == 112
    assert autotune.effective_chunk(48, 112) == 48
    c = autotune.candidates(1, 784, 256)
    assert c[0] == 96 and all(16 <= x <= 112 and x % 16 == 0 for x in c) and len(set(c)) == len(c)
    # group evaluation: N = group * hidden <= 256, at most 16 individuals per MMA
    assert autotune.max_group(16) == 16 and autotune.max_group(112) == 2 and autotune.max_group(256) == 1
    assert autotune.group_candidates(16) == [16, 8, 4] and autotune.group_candidates(112) == [2, 1]
    assert autotune.group_candidates(256) == [1] and autotune.group_candidates(80) == [3, 1]


def test_header_is_plain_c(tmp_path):
    # The boundary is a C ABI: the header compiles as strict C99 and as C++.
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "leea.h"\nint main(void) { leea_params p; leea_status s = leea_default_params(&p);\n'
                   '  return (int)s + (int)p.sigma_ctl; }\n')
    inc = os.path.dirname(HEADER)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, "-c", str(src), "-o",
                    str(tmp_path / "c.o")], check=True)
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-I", inc, "-x", "c++", "-c", str(src), "-o",
                    str(tmp_path / "cc.o")], check=True)


def test_noalloc_rejects_oversize_before_touching_the_device(lib):
    # pop x ceil(batch / 128) x 8 bytes above LEEA_NOALLOC_SCRATCH_BYTES: refused
    # from pop and batch alone, with NULL for every buffer (no CUDA call is made).
    dims = np.array([784, 32, 10], dtype=np.int32)
    assert leea.leea_shadow_scratch_bytes(20000, 1024) > leea.NOALLOC_SCRATCH_BYTES
    rc = lib.leea_evaluate_shadow_u8_noalloc(20000, dims.ctypes.data_as(ctypes.c_void_p), 3, None, 1, None, None,
                                             None, ctypes.c_float(255.0), None, 1024, ctypes.c_float(1.0), None, None,
                                             None, None, None)
    assert rc == leea.EINVAL and b"scratch bytes" in lib.leea_last_error()


def test_host_minibatch_checks():
    # The host-buffer generation calls check what the C call cannot see: dtype,
    # contiguity and x holding batch * d_0 elements (no object or device needed).
    st = leea.LeeaState.__new__(leea.LeeaState)
    st.dims = [784, 32, 10]
    x = np.zeros((16, 784), dtype=np.uint8)
    y = np.zeros(16, dtype=np.int32)
    _, _, batch = st._host_batch(x, y, "uint8")
    assert batch == 16
    with pytest.raises(ValueError, match="uint8"):
        st._host_batch(x.astype(np.float32), y, "uint8")
    with pytest.raises(ValueError, match="int32"):
        st._host_batch(x, y.astype(np.int64), "uint8")
    with pytest.raises(ValueError, match="contiguous"):
        st._host_batch(np.zeros((16, 1568), dtype=np.uint8)[:, ::2], y, "uint8")
    with pytest.raises(ValueError, match="expected"):
        st._host_batch(x[:15], y, "uint8")
    import torch
    _, _, batch = st._host_batch(torch.zeros((16, 784), dtype=torch.float32), torch.zeros(16, dtype=torch.int32),
                                 "float32")
    assert batch == 16
    with pytest.raises(ValueError, match="float32"):
        st._host_batch(torch.zeros((16, 784), dtype=torch.float64), torch.zeros(16, dtype=torch.int32), "float32")
