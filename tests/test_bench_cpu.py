"""Host-side logic of bench.py without a GPU: the max-over-ranks reduction of two gloo ranks
(the replicas path at N > 1), the aggregate throughput, the clock-sample summary and the
reference arm's JSON line on a small grid."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    m = bench._max_over_ranks(ms, world, torch.device("cpu"))
    out.put((rank, m, bench.aggregate_value(10, world, m)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == 150.0
    assert res[0][2] == pytest.approx(2 * 10 / 0.150)


def test_aggregate_value_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_value(10, 1, 2000.0) == pytest.approx(5.0)


def test_clock_summary():
    sys.path.insert(0, ROOT)
    import bench
    lines = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2000, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = bench.ClockSampler.summarise(lines)
    assert s["sm_mhz"] == 2000 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]


@pytest.mark.parametrize("args", [["--n3", "32"], ["--workload", "c2", "--nx", "64"]], ids=["c3", "c2"])
def test_reference_arm_line_on_a_small_grid(args):
    """The reference arm's line: the oracle timed on K Arnoldi iterations; its bookkeeping
    (steps x ms_per_step) is the timed work actually run, and value is the implied
    implicit-step rate, which the sample's description states."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                        "--warmup", "1"] + args, capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["unit"] == "implicit steps/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["steps"] == 3 and line["step_unit"] == "oracle Arnoldi iteration"
    # the implied step is longer than one sampled iteration
    assert line["implied_ms_per_implicit_step"] > line["ms_per_step"]
    assert line["value"] == pytest.approx(1000.0 / line["implied_ms_per_implicit_step"])
