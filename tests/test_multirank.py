"""The bench's N > 1 path on the host (CPU, gloo, world size 2): independent replicas
with their own Philox keys, whole-job figures from the slowest rank's time and every
rank's segments, and the reference arm running on rank 0 only.  The path shards without
a data-path collective; the only exchange is this final reduction of the figures."""
import json
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # rank r: 10 + r ms timed, 100 (r + 1) segments; e2e 5 (r + 1) s, 7 (r + 1) segments
        got = bench.combine_ranks(dist, "cpu", 10.0 + rank, 5.0 * (rank + 1), 100 * (rank + 1),
                                  7 * (rank + 1))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"combined": got, "seed": bench.replica_seed(rank)}, f)
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:  # every rank sees the same whole-job figures
        ms, e2e_s, segs, e2e_segs = r["combined"]
        assert ms == 11.0 and e2e_s == 10.0  # the slowest rank's times
        assert segs == 300 and e2e_segs == 21  # all ranks' units
    assert res[0]["seed"] != res[1]["seed"]  # replicas draw other random numbers


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        steps, warmup = 1, 1

    assert bench.run_reference(Args(), 1, 2) is None
    assert capsys.readouterr().out == ""
