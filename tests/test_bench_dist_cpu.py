"""Host logic of the benchmark's multi-process path, on the CPU.

Leaves are independent, so under torchrun every rank condenses its own
leaves with no data-path collective; the only cross-rank steps are the
barriers around the timed region and the max over ranks of the elapsed
time.  Those run here as two `gloo` ranks (world size 2, 127.0.0.1).
"""

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


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    r, ws = bench.dist_setup()
    assert (r, ws) == (rank, world)
    assert dist.get_backend() == "gloo"
    bench.barrier(ws)
    t = bench.max_over_ranks(10.0 * (rank + 1), ws)   # each rank's "elapsed ms"
    bench.barrier(ws)
    q.put((rank, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 20.0), (1, 20.0)]   # both ranks see the slowest rank's time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    assert bench.dist_setup() == (0, 1)
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_clock_sampler_parses_nvidia_smi_lines():
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(uuid="GPU-abc")
    cs.lines = [
        "0, GPU-abc, 1900, 2032, 700.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, GPU-abc, 1800, 2032, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, GPU-other, 300, 2032, 90.0, 0x0, Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 1850 and s["sm_max_mhz"] == 2032 and s["samples"] == 2
    assert s["reasons"] == ["sw_power_cap"]


def test_algorithmic_flops_per_leaf():
    sys.path.insert(0, ROOT)
    import bench
    assert abs(bench.leaf_flops(20) / 1e6 - 37.98) < 0.01   # LU 22.67 + TRSM 15.12 + DtN 0.19 Mflop
    assert bench.leaf_flops(20, 1) > bench.leaf_flops(20)
    assert abs(bench.leaf_flops(30) / 1e6 - 459.65) < 0.01
