"""The benchmark's multi-rank host logic on CPU: two gloo ranks (127.0.0.1)
reduce their timings to the maximum, the whole-job throughput counts the
cells of every rank, and the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    e2e = bench.max_over_ranks(2.0 - rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, e2e))


def test_two_gloo_ranks_reduce_to_the_slowest():
    mp = pytest.importorskip("torch.multiprocessing")
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
    assert res == [(0, 15.0, 2.0), (1, 15.0, 2.0)]


def test_whole_job_throughput_counts_every_rank():
    # 2 ranks x 3 runs of 1024^2 cells x 300 steps in 0.6 s
    v = bench.whole_job_mlups(2, 3 * 1024 * 1024, 300, 0.6)
    assert v == pytest.approx(2 * 3 * 1024 * 1024 * 300 / 0.6 / 1e6)
    assert bench.max_over_ranks(3.5) == 3.5  # single process: no reduction


def test_reference_arm_runs_on_rank_zero_only():
    class Args:
        steps, warmup, gpus = 1, 0, 2
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(Args(), 2, 1)
    assert buf.getvalue() == ""


def test_issue_ceiling_counts_schedulers_and_lanes():
    """152 SMs x 4 schedulers x 2070 MHz, 32 cells per warp instruction: at
    3322 warp instructions per cell the full-issue rate is 12,123 MLUPS; the
    committed profile's count is used only while the kernel sources match."""
    import bench

    assert bench.issue_ceiling(3322, 152, 2070.0) == pytest.approx(152 * 4 * 2070e6 * 32 / 3322 / 1e6)
    assert bench.issue_ceiling(None, 152, 2070.0) is None and bench.issue_ceiling(3322, 0, 2070.0) is None
    ipc = bench.profiled_instructions("fp32")
    assert ipc is None or ipc > 1000


def test_kernel_hash_ignores_comments():
    """The code identity that ties an ncu summary to the kernel sources does
    not move when only a comment or a blank line changes, and does when code
    does."""
    import bench

    a = "int f(int x) {\n    return x + 1;  // one more\n}\n"
    b = "/* a note */\nint f(int x) {\n\n    return x + 1;\n}  // end\n"
    c = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench.code_only(a) == bench.code_only(b) != bench.code_only(c)
