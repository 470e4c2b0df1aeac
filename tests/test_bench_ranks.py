"""The replicas-only multi-GPU path of bench.py on CPU: two gloo ranks, the
barrier, the max over ranks and the whole-job rate (every rank runs its own
independent replica; the job lasts as long as the slowest one)."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init(world, use_cuda=False)
    bench.barrier(dist)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
    ms_max, rate = bench.job_rate(world, 40, ms_local, dist)
    top = bench.max_over_ranks(float(rank) + 0.5, dist)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"ms_max": ms_max, "rate": rate, "top": top}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    res = [json.loads((tmp_path / f"rank{r}.json").read_text()) for r in range(2)]
    for r in res:
        assert r["ms_max"] == 150.0
        assert r["rate"] == pytest.approx(2 * 40 / 0.150)  # 80 units in 150 ms
        assert r["top"] == 1.5


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1, use_cuda=False) is None
    ms_max, rate = bench.job_rate(1, 10, 200.0, None)
    assert ms_max == 200.0 and rate == pytest.approx(50.0)
