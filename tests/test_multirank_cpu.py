"""The N > 1 path of the benchmark on CPU: two `gloo` ranks on 127.0.0.1.

Under torchrun each rank runs an independent replica (no collective on the data path);
the only collectives are the timing barrier and the MAX over ranks of the timed region,
and rank 0 alone prints. These tests run those host-side pieces with the gloo backend
(the GPU run uses NCCL with the same calls), and check that the reference arm's other
ranks leave without work.
"""
import importlib.util
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    b = load_bench()
    w, r, local = b.dist_setup()
    dist.init_process_group("gloo")
    dist.barrier()
    secs = b.max_over_ranks(1.0 + 0.5 * r, w)      # rank 1 is the slow replica
    value = b.job_mlups(w, 4_000_000, secs)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, secs, value))


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == 1.5 for o in out)                 # MAX over ranks, seen by both
    assert all(abs(o[4] - 2 * 4.0 / 1.5) < 1e-12 for o in out)   # whole-job MLUPS


def test_single_rank_needs_no_process_group():
    b = load_bench()
    assert b.max_over_ranks(2.5, 1) == 2.5
    assert b.job_mlups(1, 2_000_000, 2.0) == 1.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    b = load_bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert b.main() == 0
    assert capsys.readouterr().out == ""
