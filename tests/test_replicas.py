"""The bench's multi-GPU path is replicas only (independent problems, no data-path
collective): its whole-job numbers are the slowest rank's time and the sum of every
rank's iterations.  Checked with two gloo ranks on the CPU.  Also: the roofline line's captured
DRAM traffic is reported only for the kernel source it was measured on."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, it = bench.job_totals([1.5, 2.5][rank], [30.0, 31.0][rank], world, "cpu")
    q.put((rank, t, it))
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2.5, 61.0), (1, 2.5, 61.0)]


def test_job_totals_single_rank():
    import bench
    assert bench.job_totals(1.25, 7.0, 1, "cpu") == (1.25, 7.0)


def test_roofline_traffic_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    # the factor's DRAM traffic is reported only while its kernel source is the one the
    # capture measured (sha256 of kernels_warp.cuh), only at the captured size and element
    # size; an edited source makes it null
    import shutil
    import bench
    val = bench.captured_traffic("factor", 4, 5000)
    assert val is not None and val > 0
    assert bench.captured_traffic("factor", 4, 4999) is None
    assert bench.captured_traffic("factor", 8, 5000) is None
    assert bench.captured_traffic("solve", 4, 5000) is None
    root = tmp_path / "repo"
    csrc = root / "paper_2607_15420_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_2607_15420_gb300", "csrc", "kernels_warp.cuh")
    shutil.copy(src, csrc / "kernels_warp.cuh")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.captured_traffic("factor", 4, 5000) == val
    with open(csrc / "kernels_warp.cuh", "a") as f:
        f.write("\n// edited\n")
    assert bench.captured_traffic("factor", 4, 5000) is None
