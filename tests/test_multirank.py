"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks.

Every rank runs the whole step on its own GPU; the step time is the slowest
rank's (an all-reduce MAX) and the value counts every rank's work-items.  The
reference arm prints from rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = [12.5, 20.0][rank]  # rank 1 is the slow one
        got = bench.max_over_ranks(step_ms, world, device="cpu")
        rate = bench.job_rate(1000.0, world, got * 1e-3)
        q.put((rank, got, rate))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_step_and_all_ranks_count():
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
    assert [r[1] for r in res] == [20.0, 20.0]
    assert all(r[2] == pytest.approx(2 * 1000.0 / 0.020) for r in res)


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_rate(10.0, 1, 2.0) == 5.0


@pytest.mark.parametrize("rank,prints", [(0, True), (1, False)])
def test_reference_arm_prints_on_rank_zero_only(rank, prints):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--only",
                        "mandelbrot", "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    if prints:
        assert len(lines) == 1
        d = json.loads(lines[0])
        assert d["impl"] == "reference" and d["value"] > 0
        # the line the driver reads: the same keys as the kernel arm's, the
        # oracle described, and no host-device copies
        for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                  "vs_baseline", "dtype", "data", "config"):
            assert k in d, k
        assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True  # warm-up raised to 3
        assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
        assert d["cpu_baseline"]["value"] == d["value"]
        assert d["e2e"] == dict(value=d["value"], unit=d["unit"], h2d_bytes_per_step=0, d2h_bytes_per_step=0)
        # the same configuration description as the kernel arm's line, and the
        # sample each step times
        import bench
        w = bench.Mandelbrot(None, None, 0)
        w.host_setup()
        assert d["config"] == json.loads(json.dumps(bench.step_config([w])))
        assert d["sampled_fraction"] == {"mandelbrot": bench.CPU_SAMPLE}  # one row of 1024
    else:
        assert lines == []
