"""The N > 1 host path of bench.py on CPU: two gloo ranks (world size 2) on 127.0.0.1.

In its replica mode (`--parallel replicas`: one independent system per GPU, weak scaling, no
data-path collective) bench.py's only cross-rank steps are the barrier around the timed region
and the maximum of the step times over the ranks; the whole-job value is the systems all ranks
processed over that maximum. The q-sharded default mode (one system, one sum of Sigma_c over the
ranks) is covered by test_shard_gloo.py. Here the same
helpers run under gloo with planted per-rank times, and the reference arm's rank handling (rank 0
alone prints) is checked in-process."""
import io
import json
import os
import socket
import sys
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench                                # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, ms_e2e = bench.max_over_ranks(times[rank], world, "cpu")
        dist.barrier()
        res = dict(rank=rank, ms=ms, ms_e2e=ms_e2e, value=bench.seconds_per_system(ms, world),
                   seed=bench.replica_seed("cfg1", rank))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_step_time(tmp_path):
    world = 2
    times = [[8200.0, 8400.0], [8300.0, 8350.0]]      # (device-resident, end-to-end) ms per rank
    mp.spawn(_worker, args=(world, _free_port(), times, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms"] == 8300.0 and r["ms_e2e"] == 8400.0      # every rank sees the maxima
        assert abs(r["value"] - 8.3 / 2) < 1e-12                  # 2 systems in the slowest step
    assert res[0]["seed"] != res[1]["seed"]                         # replicas process different systems


def test_single_process_needs_no_group():
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.seconds_per_system(8300.0, 1) == 8.3


def test_reference_arm_prints_on_rank_zero_only():
    from paper_2011_01400_gb300.synth import make_system

    class A:
        steps, warmup, gpus, config = 1, 0, 2, "tiny"

    s = make_system("tiny", seed=1)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A, s, world=2, rank=1)
    assert buf.getvalue() == ""
