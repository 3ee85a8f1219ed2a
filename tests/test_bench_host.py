"""CPU checks of bench.py's host logic: the replica timing reduction over a
2-rank gloo process group, the algorithmic byte/flop model, and the workload
descriptions."""
import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_local = 1.0 + rank                     # rank 1 is the slow one
    t, value = bench.replica_value(100.0, t_local, world)
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_value_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        t, value = out[r]
        assert t == 2.0                      # max over ranks
        assert value == 2 * 100.0 / 2.0      # all ranks' work / slowest time


def test_single_rank_value():
    assert bench.replica_value(30.0, 1.5, 1) == (1.5, 20.0)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_algorithmic_model(p):
    nb = {1: 4, 2: 10, 3: 20}[p]
    b1, f1 = bench.algorithmic_model(p, 1000, "roe", 8, 1)
    b2, _ = bench.algorithmic_model(p, 1000, "roe", 8, 2)
    assert b1 == 1000 * (5 * nb * 8 * 2 + 32)       # read U, write U1
    assert b2 == 1000 * (5 * nb * 8 * 3 + 32)       # and the RK base state
    _, fr = bench.algorithmic_model(p, 1000, "rusanov", 8, 1)
    assert f1 > fr > 0


def test_workload_configs():
    class A:
        workload = "c3"
    c = bench.config_of(A())
    assert c["tets"] == 6 * 64 ** 3 and c["order"] == 3 and c["dofs"] == 6 * 64 ** 3 * 100
    A.workload = "c5"
    assert bench.config_of(A())["tets"] == 96 * 48 * 48 * 6


def test_measured_traffic_scales_with_elements_and_checks_sources(monkeypatch):
    import bench
    key = ("mixed", 3, "roe")
    per_elem, files, _ = bench.MEASURED_TRAFFIC[key]
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, key, (per_elem, files, bench.kernel_source_hash(files)))
    assert bench.measured_traffic("f16x2-tc/f32/ff32", 3, "roe", 1000) == pytest.approx(per_elem * 1000)
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, key, (per_elem, files, "0" * 16))
    assert bench.measured_traffic("f16x2-tc/f32/ff32", 3, "roe", 1000) is None
    assert bench.measured_traffic("f32", 2, "rusanov", 1000) is None
