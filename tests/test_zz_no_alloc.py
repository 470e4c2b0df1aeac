"""The allocation-free shadow evaluation (leea_evaluate_shadow_u8_noalloc,
static scratch) against the entry point with caller scratch
(leea_evaluate_shadow_u8): the same fitness on two calls in a row, and a clear
error for requests beyond its fixed scratch size.  Kept in its own file,
collected last, so that it also runs after every other GPU test."""
import numpy as np
import pytest

from helpers import assert_fitness_close, to_device_pop
from paper_1806_09819_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("dims,pop,batch", [([784, 112, 10], 37, 300), ([784, 32, 10], 200, 129),
                                            ([64, 16, 4], 5, 100)])
def test_noalloc_matches_caller_scratch_entry(gpu, dims, pop, batch, precision):
    import torch
    c, cp = gpu.leea_layout_num_params(dims), gpu.leea_padded_params(dims)
    popv = synthetic.random_population(pop, c, seed=pop + batch, scale=0.1)
    rng = np.random.default_rng(batch)
    levels = rng.integers(0, 256, size=(batch, dims[0])).astype(np.uint8)
    y = rng.integers(0, dims[-1], size=batch).astype(np.int32)
    f_inh = torch.from_numpy(rng.normal(-2.3, 0.1, size=pop).astype(np.float32)).cuda()
    pd = to_device_pop(popv, cp)
    sh = torch.zeros((pop, gpu.leea_shadow_stride(dims, precision)), dtype=torch.uint8, device="cuda")
    se = torch.zeros(pop, dtype=torch.int32, device="cuda")
    am = torch.zeros(pop, dtype=torch.float32, device="cuda")
    gpu.leea_make_shadow(pop, dims, precision, pd, sh, se, am)
    xd, yd = torch.from_numpy(levels).cuda(), torch.from_numpy(y).cuda()

    nbytes = gpu.leea_shadow_scratch_bytes(pop, batch)
    scratch = torch.empty(max(nbytes // 4, 1), dtype=torch.float32, device="cuda") if nbytes else None
    ref = [torch.empty(pop, dtype=torch.float32, device="cuda") for _ in range(2)]
    ref_cor = torch.empty(pop, dtype=torch.int32, device="cuda")
    gpu.leea_evaluate_shadow_u8(pop, dims, pd, precision, sh, se, xd, 255.0, yd, batch, 0.25, f_inh, ref[0], ref[1],
                                ref_cor, scratch)
    assert gpu.leea_device_status() == 0
    want_raw, want_adj, want_cor = (t.cpu().numpy() for t in (*ref, ref_cor))

    for _ in range(2):  # two calls in a row on the same static scratch
        f_raw = torch.full((pop,), float("nan"), dtype=torch.float32, device="cuda")
        f_adj = torch.full_like(f_raw, float("nan"))
        cor = torch.full((pop,), -1, dtype=torch.int32, device="cuda")
        gpu.leea_evaluate_shadow_u8_noalloc(pop, dims, pd, precision, sh, se, xd, 255.0, yd, batch, 0.25, f_inh,
                                            f_raw, f_adj, cor)
        assert gpu.leea_device_status() == 0
        # the same kernels on the same inputs, only the scratch differs: bit-identical
        np.testing.assert_array_equal(f_raw.cpu().numpy().view(np.uint32), want_raw.view(np.uint32))
        np.testing.assert_array_equal(f_adj.cpu().numpy().view(np.uint32), want_adj.view(np.uint32))
        np.testing.assert_array_equal(cor.cpu().numpy(), want_cor)
        # and within the evaluation tolerance of the caller-scratch entry (the same bar as every evaluation test)
        assert_fitness_close(f_raw.cpu().numpy(), want_raw.astype(np.float64), "noalloc f_raw")


def test_noalloc_rejects_requests_beyond_its_scratch(gpu):
    import torch
    dims = [784, 32, 10]
    pop, batch = 20000, 1024  # 8 tiles x 20000 individuals x 8 bytes > 1 MiB
    assert gpu.leea_shadow_scratch_bytes(pop, batch) > gpu.NOALLOC_SCRATCH_BYTES
    # NULL device pointers throughout: the size check comes first, and with no
    # buffers no kernel could be launched whatever the later checks did
    with pytest.raises(gpu.LeeaError, match="scratch bytes"):
        gpu.leea_evaluate_shadow_u8_noalloc(pop, dims, None, 1, None, None, None, 255.0, None, batch, 1.0, None,
                                            None)
    # the largest population that fits at this batch is accepted by the size check
    assert gpu.leea_shadow_scratch_bytes(16384, batch) <= gpu.NOALLOC_SCRATCH_BYTES
