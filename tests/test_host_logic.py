"""Host-side logic that needs no GPU: batch table layout and batch splitting,
the Chrome trace, and the bench's balance, efficiency and rate helpers."""
import numpy as np


def test_instance_table_layout_matches_the_header():
    from paper_1805_02755_gb300.batching import INSTANCE_DTYPE
    # ecl_binomial_instance: 7 pointers, int64 first, int64 n, float r, int32 pad
    assert INSTANCE_DTYPE.itemsize == 80
    assert INSTANCE_DTYPE.fields["first"][1] == 56 and INSTANCE_DTYPE.fields["r"][1] == 72


def test_view_and_image_tables_match_the_header():
    # the offsets a C compiler gives ecl_mandelbrot_view and ecl_gaussian_image
    # on a 64-bit target (checked against the header's own declarations)
    import os
    import subprocess
    import tempfile
    from paper_1805_02755_gb300.batching import IMAGE_DTYPE, VIEW_DTYPE
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = (
        '#include <stddef.h>\n#include <stdio.h>\n#include "ecl.h"\nint main(void) {\n'
        'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ecl_mandelbrot_view), '
        'offsetof(ecl_mandelbrot_view, max_iter), offsetof(ecl_mandelbrot_view, first), '
        'offsetof(ecl_mandelbrot_view, wgs), sizeof(ecl_gaussian_image), offsetof(ecl_gaussian_image, W), '
        'offsetof(ecl_gaussian_image, first), offsetof(ecl_gaussian_image, tiles));\nreturn 0;\n}\n')
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "t.c"), os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(root, "include"), c, "-o", exe], check=True)
        got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    v, i = VIEW_DTYPE.fields, IMAGE_DTYPE.fields
    assert got == [VIEW_DTYPE.itemsize, v["max_iter"][1], v["first"][1], v["wgs"][1],
                   IMAGE_DTYPE.itemsize, i["W"][1], i["first"][1], i["tiles"][1]]


def test_batch_sizes_in_work_groups_and_tiles():
    from paper_1805_02755_gb300.batching import GaussianBatch, MandelbrotBatch
    assert MandelbrotBatch.workgroups(1024, 1024) == 1024 and MandelbrotBatch.workgroups(1, 1) == 1
    assert MandelbrotBatch.workgroups(33, 31) == 1 and MandelbrotBatch.workgroups(1025, 1) == 2
    assert GaussianBatch.tiles(224, 32) == 1 and GaussianBatch.tiles(225, 33) == 4 and GaussianBatch.tiles(1, 1) == 1
    assert GaussianBatch.tiles(8192, 8192) == 256 * 37


def test_split_uneven_sums_and_skews():
    from paper_1805_02755_gb300.batching import split_uneven
    for n, parts in [(1 << 20, 64), (1000, 7), (64, 64)]:
        s = split_uneven(n, parts, seed=1)
        assert sum(s) == n and len(s) == parts and min(s) >= 1
    s = np.array(split_uneven(1 << 20, 64, seed=1))
    assert s.max() > 8 * np.median(s)


def test_chrome_trace_of_package_records(tmp_path):
    import json
    import numpy as np
    import paper_1805_02755_gb300 as E
    st = np.zeros(3, dtype=E.PKG_STAT_DTYPE)
    st["t0_ns"] = [1000, 1500, 4000]
    st["t1_ns"] = [3000, 5000, 4000]
    st["pkg"] = [0, 1, 2]
    st["device"] = [0, 1, 0]
    st["cta"] = [3, 7, 3]
    st["off_wg"] = [0, 4, 8]
    st["len_wg"] = [4, 4, 2]
    path = str(tmp_path / "t.json")
    tr = E.chrome_trace(st, path)
    ev = tr["traceEvents"]
    assert [e["ph"] for e in ev] == ["X"] * 3
    assert [e["ts"] for e in ev] == [0.0, 0.5, 3.0]  # microseconds from the first fetch
    assert [e["dur"] for e in ev] == [2.0, 3.5, 0.0]
    assert [(e["pid"], e["tid"]) for e in ev] == [(0, 3), (1, 7), (0, 3)]
    assert ev[1]["args"] == {"off_wg": 4, "len_wg": 4, "smid": 0}
    assert json.load(open(path)) == tr
    assert E.chrome_trace(st[:0])["traceEvents"] == []


def _pkg_stats(rows):
    import paper_1805_02755_gb300 as E
    a = np.zeros(len(rows), dtype=E.PKG_STAT_DTYPE)
    for i, (dev, t0, t1) in enumerate(rows):
        a[i]["device"], a[i]["t0_ns"], a[i]["t1_ns"] = dev, t0, t1
    return a


def _worker_stats(rows):
    import paper_1805_02755_gb300 as E
    a = np.zeros(len(rows), dtype=E.WORKER_STAT_DTYPE)
    for i, (busy, chunks) in enumerate(rows):
        a[i]["busy_ns"], a[i]["chunks"], a[i]["cta"] = busy, chunks, i
    return a


def test_balance_is_first_over_last_device_finish():
    """Sec. 7.3 balance T_FD / T_LD: each device's last package end, from the
    first package start; one device balances trivially."""
    import bench
    st = _pkg_stats([(0, 100, 300), (1, 100, 500), (0, 300, 400), (1, 120, 200)])
    assert bench.balance_of(st) == (400 - 100) / (500 - 100)
    assert bench.balance_of(_pkg_stats([(0, 10, 50), (0, 50, 90)])) == 1.0
    assert bench.balance_of(_pkg_stats([])) is None


def test_worker_efficiency_and_the_grid_form():
    """Mean over max busy time of the persistent CTAs; none for Static over one
    device, which runs as a grid of one-chunk CTAs."""
    import bench
    ws = _worker_stats([(100, 3), (50, 2), (150, 4)])
    assert bench.worker_efficiency(ws, dict(devices=2, ctas_per_device=2, ctas=4)) == 100 / 150
    grid = _worker_stats([(30, 1), (90, 1)])
    assert bench.worker_efficiency(grid, dict(devices=1, ctas_per_device=2, ctas=2)) is None
    # one device of persistent CTAs with several chunks each is not the grid form
    assert bench.worker_efficiency(ws, dict(devices=1, ctas_per_device=3, ctas=3)) == 100 / 150


def test_job_rate_counts_every_rank():
    import bench
    assert bench.job_rate(1000, 4, 2.0) == 2000.0
    assert bench.max_over_ranks(1.5, 1) == 1.5


def test_engines_default_to_torchs_current_device(monkeypatch):
    # Under torchrun each rank sets its own CUDA device; an engine (and the
    # batching helpers built on it) created without a device ordinal must
    # take that device, not device 0.  Checked on the host with the C call
    # and torch's device query replaced.
    import torch
    import paper_1805_02755_gb300 as E
    seen = []
    monkeypatch.setattr(E, "ecl_engine_create", lambda device, stream=None: seen.append(device) or 0)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)
    assert E.current_device() == 3
    assert E.current_device(1) == 1
    E.Engine()
    E.Engine(2)
    assert seen == [3, 2]
