"""The multi-GPU path of bench.py (replicas, one process per GPU) on the host: two
gloo ranks check the max over ranks, the barrier, the whole-job throughput and
end-to-end figures of replicas and that the oracle's reference arm prints only on
rank 0."""
import json
import os
import socket
import sys
from datetime import timedelta

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": "2",
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", timeout=timedelta(seconds=60))
    ws = 2
    got = {}
    # the slowest rank sets the job's time
    got["max"] = bench.max_over_ranks(10.0 + rank * 5.0, ws)
    bench.barrier(ws)
    # replicas: each rank processes 1,000 units per step; rank 1 is slower
    step_ms = [2.0, 2.0, 2.0] if rank == 0 else [3.0, 3.0, 3.0]
    got["rate"], got["ms_per_step"] = bench.job_rate(step_ms, 1000, 3, ws)
    # end to end: each rank's median step, the job's is the slower rank's
    got["e2e"] = bench.e2e_job_summary([10.0, 12.0, 11.0] if rank == 0 else [20.0, 24.0, 21.0], 1000, 100, 200, ws)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump(got, f)


def test_two_gloo_ranks_aggregate_like_the_benchmark(tmp_path):
    port = _free_port()
    torch.multiprocessing.spawn(_rank_main, args=(port, str(tmp_path)), nprocs=2, join=True)
    for rank in (0, 1):
        got = json.load(open(tmp_path / ("rank%d.json" % rank)))
        assert got["max"] == 15.0
        # 2 ranks x 1,000 units x 3 steps in the slower rank's 9 ms
        assert got["ms_per_step"] == pytest.approx(3.0)
        assert got["rate"] == pytest.approx(2 * 1000 * 3 / 9e-3)
        e2e = got["e2e"]
        assert e2e["ms_per_step"] == 21.0 and e2e["max_ms"] == 24.0
        assert e2e["mean_ms"] == pytest.approx(65.0 / 3)
        assert e2e["value"] == pytest.approx(2 * 1000 / 21e-3)
        assert (e2e["h2d_bytes_per_step"], e2e["d2h_bytes_per_step"]) == (200, 400)


def test_reference_arm_prints_on_rank_0_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        n, steps, warmup, gpus = 2, 1, 0, 2
    bench.run_reference(Args, 2, 1)  # rank 1: no work, no line
    assert capsys.readouterr().out == ""
    bench.run_reference(Args, 2, 0)  # rank 0: the oracle's line
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
