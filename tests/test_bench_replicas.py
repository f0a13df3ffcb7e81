"""bench.py's multi-GPU path is N independent replicas (the evaluation is not sharded): the step
time is the slowest rank's, the value the whole job's, and only rank 0 reports. Checked here with
two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = _bench()
    step_ms = bench.max_over_ranks(1.0 + rank)  # rank 1 is the slower replica
    out[rank] = (step_ms, bench.replica_value(1e9, world, step_ms), bench._dist_env()[:2])
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for rank in (0, 1):
        step_ms, value, (r, w) = res[rank]
        assert (r, w) == (rank, 2)
        assert step_ms == 2.0                  # max over ranks
        assert value == 2 * 1e9 / 2.0e-3       # both replicas' pairs over the slowest step


def test_single_process_is_its_own_max():
    bench = _bench()
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_value(7.0e9, 1, 0.5) == 7.0e9 / 0.5e-3


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    bench = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
