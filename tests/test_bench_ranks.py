"""Host logic of bench.py's multi-rank launch (replicas, one process per GPU),
exercised with world-size-2 gloo process groups on the CPU: the timing every
rank reports is the slowest rank's, and the reference arm runs on rank 0 only."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = (bench._env_rank(), bench.max_over_ranks(10.0 + 5.0 * rank))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        (r, w, local), value = out[rank]
        assert (r, w, local) == (rank, world, rank)
        assert value == 15.0


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_reference_arm_skips_nonzero_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, ref_iters, ref_prox = 1, 0, 1, 1

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""


def test_ct_f_star_prefers_the_oracle_value(tmp_path):
    """The CT record takes the committed oracle F* when it exists and reports the
    GPU's long-run minimum beside it; without the file it falls back to the GPU's."""
    import json
    import bench
    path = tmp_path / "fstar.json"
    fs, src, chk = bench.ct_f_star(352.9143, path=str(path))
    assert fs == 352.9143 and "GPU" in src and chk is None
    path.write_text(json.dumps({"f_star": 352.9142}))
    fs, src, chk = bench.ct_f_star(352.9143, path=str(path))
    assert fs == 352.9142 and "oracle" in src
    assert chk["gpu_pdhg_min"] == 352.9143 and abs(chk["rel_diff"] - 0.0001 / 352.9142) < 1e-12
