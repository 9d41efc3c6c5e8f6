"""The multi-rank path of bench.py on CPU with the gloo backend (2 ranks).

Frames are independent, so ranks are replicas: each rank decodes its own
frames and only the timing is combined.  Checked here without a GPU: the
frame shards are disjoint and their seeded inputs differ, the maximum over
ranks reaches every rank, the whole-job rate counts every rank's bits over
the slowest rank's time, and the reference arm's non-zero ranks leave
without work.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    from paper_1204_5882_gb300 import synth as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = S.WORKLOADS["bsc_p02_n16"]
    F = 3
    first = bench.rank_first_frame(rank, F)
    x, _ = S.frames(w, first, F)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
    dist.barrier()
    q.put((rank, first, x.tobytes(), ms, bench.job_rate(world, F, w.N, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, f0, x0, ms0, v0), (r1, f1, x1, ms1, v1) = out
    assert (r0, r1) == (0, 1) and (f0, f1) == (0, 3)      # disjoint shards of 3 frames
    assert x0 != x1                                        # different seeded inputs
    assert ms0 == ms1 == 15.0                              # max over ranks, on every rank
    assert v0 == v1 == pytest.approx(2 * 3 * (1 << 16) / 15e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, None, torch.device("cpu")) == 7.5
    assert bench.job_rate(1, 64, 1 << 20, 9.4) == pytest.approx(64 * 2 ** 20 / 9.4e-3 / 1e6)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
