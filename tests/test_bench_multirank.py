"""The N > 1 host logic of bench.py, run as two gloo ranks on the CPU: the
shards are disjoint (each rank its own seeded sequence), the time is the
slowest rank's (all-reduce MAX), the value counts every rank's work, and the
reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        ms = bench.max_over_ranks(my_ms, dist, "cpu")
        value, ms_step = bench.job_value(1000, world, ms, steps=5)

        class A:
            gpus, steps, warmup = world, 5, 3
        import io
        import contextlib
        buf = io.StringIO()
        if rank != 0:  # the reference arm prints nothing and does no work off rank 0
            with contextlib.redirect_stdout(buf):
                ref = bench.run_reference(A, rank, world)
        else:
            ref = "rank0"
        out[rank] = (ms, value, ms_step, bench.rank_seed(rank), ref, buf.getvalue() if rank else "")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    (ms0, v0, st0, seed0, _, _), (ms1, v1, st1, seed1, ref1, printed1) = out[0], out[1]
    assert ms0 == ms1 == 15.0  # the slowest rank's time everywhere
    assert v0 == v1 == pytest.approx(1000 * 2 / (3.0 * 1e-3))  # both ranks' units over 3 ms per step
    assert st0 == 3.0
    assert seed0 != seed1  # disjoint shards
    assert ref1 is None and printed1 == ""


def test_reference_arm_line():
    """--impl reference times the oracle in bounded steps and prints the
    contract's line with our arm's metric, unit and direction."""
    import json
    import subprocess
    sys.path.insert(0, ROOT)
    import bench
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "macroblocks/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "macroblocks/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
