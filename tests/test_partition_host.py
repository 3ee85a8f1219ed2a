"""CPU checks of the partitioned layout (the multi-process form of the paper's
per-process grid, Sec. III-B): the host-only plan covers the element order
with contiguous slabs on 96-element boundaries and its halos are exactly the
other slabs' face neighbours (recomputed from the oracle's face matching); and
a world-size-2 gloo run exchanges the halo blocks and reduces the time-step
minimum and the conserved totals over the ranks."""
import math
import os
import socket

import numpy as np
import pytest

from oracle.mesh import jacobians, match_faces
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I


def _internal_neighbours(m, renumber):
    """[ne][4] neighbours in internal ids (boundary -1) and perm (caller -> internal)."""
    perm, _, _ = dg.dg_element_order(m.tet_vid, m.tet_xyz, None if all(m.periodic) else m.bc_tag, renumber)
    nbr, _, _ = match_faces(m.tet_vid, None if all(m.periodic) else m.bc_tag)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    out = np.full((m.ne, 4), -1, dtype=np.int64)
    for f in range(4):
        n = nbr[inv, f]
        out[:, f] = np.where(n >= 0, perm[np.maximum(n, 0)], -1)
    return out, perm


@pytest.mark.parametrize("renumber", [dg.DG_ORDER_RCM, dg.DG_ORDER_MORTON])
@pytest.mark.parametrize("kind", ["periodic", "box"])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_plan_slabs_and_halos(renumber, kind, k):
    m = I.make_periodic_cube(5, jitter=0.15) if kind == "periodic" else I.make_box_channel(6, 4, 4, jitter=0.15)
    tag = None if kind == "periodic" else m.bc_tag
    nbr, _ = _internal_neighbours(m, renumber)
    end = 0
    for r in range(k):
        first, count, ids, part = dg.dg_partition_plan(m.tet_vid, m.tet_xyz, tag, renumber, k, r)
        assert first == end and count > 0
        assert first % 96 == 0
        end = first + count
        own = np.zeros(m.ne, dtype=bool)
        own[first:end] = True
        n = nbr[first:end].ravel()
        expect = np.unique(n[(n >= 0) & ~own[np.maximum(n, 0)]])
        np.testing.assert_array_equal(ids, expect)
        assert np.all(np.diff(ids) > 0)
        # each halo element's owner is the slab that holds it
        for g, q in zip(ids, part):
            fq, cq, _, _ = dg.dg_partition_plan(m.tet_vid, m.tet_xyz, tag, renumber, k, int(q))
            assert fq <= g < fq + cq
    assert end == m.ne


def test_plan_rejects_too_many_partitions():
    m = I.make_periodic_cube(4, jitter=0.1)                       # 384 elements: 4 slabs of 96
    dg.dg_partition_plan(m.tet_vid, m.tet_xyz, None, dg.DG_ORDER_RCM, 4, 0)
    with pytest.raises(dg.DGError) as e:
        dg.dg_partition_plan(m.tet_vid, m.tet_xyz, None, dg.DG_ORDER_RCM, 5, 0)
    assert e.value.status == 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, result_file):
    import torch
    import torch.distributed as dist
    from paper_2209_01877_gb300.partition import HaloExchange, allreduce_min, allreduce_sum, make_plan
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = I.make_box_channel(4, 3, 3, jitter=0.15)
        nbr, perm = _internal_neighbours(m, dg.DG_ORDER_MORTON)
        plan = make_plan(m.tet_vid, m.tet_xyz, m.bc_tag, dg.DG_ORDER_MORTON, world, rank)
        # a seeded global state in internal order; every rank holds only its own slab of it
        U = I.uniform(21, m.ne * 5 * 4, 0.5, 1.5).reshape(m.ne, 5, 4)
        Uint = np.empty_like(U)
        Uint[perm] = U
        own = torch.from_numpy(Uint[plan.first:plan.first + plan.count].copy())
        ex = HaloExchange(plan)
        halo = torch.zeros((len(plan.halo_ids), 5, 4), dtype=torch.float64)
        ex.exchange(own, halo)
        ok_halo = bool(np.array_equal(halo.numpy(), Uint[plan.halo_ids]))
        # reductions: local totals of the own elements and a local minimum, over the ranks
        _, det, _ = jacobians(m.tet_xyz)
        detI = np.empty_like(det)
        detI[perm] = det
        sl = slice(plan.first, plan.first + plan.count)
        tot = torch.from_numpy(np.einsum("e,ev->v", detI[sl], Uint[sl, :, 0]) / math.sqrt(6.0))
        allreduce_sum(tot)
        ref_tot = np.einsum("e,ev->v", detI, Uint[:, :, 0]) / math.sqrt(6.0)
        ok_tot = bool(np.all(np.abs(tot.numpy() - ref_tot) <= 1e-13 * np.abs(ref_tot)))
        mn = torch.tensor([float(detI[sl].min())], dtype=torch.float64)
        allreduce_min(mn)
        ok_min = float(mn.item()) == float(detI.min())
        with open(f"{result_file}.{rank}", "w") as fh:
            fh.write(f"{int(ok_halo)} {int(ok_tot)} {int(ok_min)} {len(plan.halo_ids)}\n")
    finally:
        dist.destroy_process_group()


def test_halo_exchange_and_reductions_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "res")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ok_halo, ok_tot, ok_min, nh = open(f"{out}.{r}").read().split()
        assert int(nh) > 0
        assert ok_halo == "1" and ok_tot == "1" and ok_min == "1", (r, ok_halo, ok_tot, ok_min)
