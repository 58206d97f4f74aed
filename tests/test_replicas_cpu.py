"""Replica path of bench.py, on CPU with a world-size-2 gloo process group.

`bench.py --gpus N` runs one independent chain per rank on its own data
(replicas only: the top tree levels of one chain couple all its rows, so a
chain does not shard) and reports the whole-job rate from the slowest rank.
Here two gloo ranks with different per-step times agree on the slowest time
and on the job rate, and the reference arm prints nothing off rank 0.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PER_MS = (10.0, 12.5)    # device time per step of rank 0, rank 1
E2E_S = (0.011, 0.013)   # end-to-end time per step


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sys.path.insert(0, ROOT)
        import bench

        per, e2e = bench.max_over_ranks([PER_MS[rank], E2E_S[rank]], world, "cpu")
        value, e2e_value = bench.job_rates(per, e2e, world)
        q.put((rank, per, e2e, value, e2e_value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for _, per, e2e, value, e2e_value in out:
        assert per == max(PER_MS) and e2e == max(E2E_S)
        assert value == pytest.approx(2 * 1e3 / max(PER_MS), rel=1e-15)
        assert e2e_value == pytest.approx(2 / max(E2E_S), rel=1e-15)


def test_single_rank_keeps_its_own_times():
    sys.path.insert(0, ROOT)
    import bench

    per, e2e = bench.max_over_ranks([PER_MS[1], E2E_S[1]], 1, "cpu")
    assert (per, e2e) == (PER_MS[1], E2E_S[1])
    assert bench.job_rates(per, e2e, 1) == pytest.approx((1e3 / PER_MS[1], 1 / E2E_S[1]))


def test_reference_arm_is_silent_off_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
