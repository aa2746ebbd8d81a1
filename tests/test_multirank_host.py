"""The multi-rank host logic of bench.py on CPU: world size 2 over gloo (127.0.0.1).  Every
rank runs its own independent controller (replicas, no collective on the data path); the
timed region is the slowest rank's and the value counts every rank's units."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = 1.5 + rank                                 # rank 1 is the slower one
        slowest = bench.reduce_max(mine, dist, "cpu")
        q.put((rank, slowest, bench.whole_job_rate(1000.0, world, slowest)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_the_slowest_and_count_every_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, slowest, rate in got:
        assert slowest == pytest.approx(2.5)              # max over the ranks
        assert rate == pytest.approx(2 * 1000.0 / 2.5)    # units of both ranks over the slowest time


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.25) == 3.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_clock_sampler_keeps_only_samples_inside_the_timed_windows(tmp_path, monkeypatch):
    """The NVML sampler runs as a process of its own and timestamps its samples; stop() keeps
    those inside the mark_start/mark_end windows.  Here a stand-in process writes samples at
    known times (no GPU or NVML on this host)."""
    import subprocess
    import time
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.nvml_path = str(tmp_path / "samples.nvml")
    now = time.time()
    s.windows = [(now + 10.0, now + 20.0)]
    s.t0, s.t1 = now + 10.0, now + 20.0
    with open(s.nvml_path, "w") as f:
        f.write("%.6f,2032,2032,0\n" % (now + 5.0))     # before the window: dropped
        f.write("%.6f,1900,2032,4\n" % (now + 12.0))    # inside, with reason bit 4
        f.write("%.6f,2032,2032,0\n" % (now + 25.0))    # after: dropped (and ends the wait)
        f.write("not a sample\n")
    s.nvml_p = subprocess.Popen([sys.executable, "-c", "import time; time.sleep(30)"])
    rows = s._stop_nvml()
    assert s.nvml_p.poll() is not None                  # the sampler process was stopped
    assert len(rows) == 1 and rows[0]["sm"] == 1900.0 and rows[0]["smax"] == 2032.0
    assert [r for r, on in rows[0]["reasons"].items() if on] == [r for r, b in bench._REASON_BITS.items() if b == 4]
