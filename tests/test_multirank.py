"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
job's time is the largest rank time, the job's rate counts every replica's
markers, and the reference arm runs on rank 0 alone."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    b = _bench()
    ms = [1.5, 4.0][rank]                      # this rank's own time
    job_ms = b.max_over_ranks(ms, world, device="cpu")
    rate = b.job_rate(1000, world, 10, job_ms / 1e3)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"job_ms": job_ms, "rate": rate}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["job_ms"] == 4.0                        # the slower rank's time
        assert r["rate"] == pytest.approx(1000 * 2 * 10 / 4.0e-3)


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(2.5, 1) == 2.5
    assert b.job_rate(10, 1, 4, 2.0) == 20.0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
