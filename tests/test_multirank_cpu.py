"""Multi-process paths on CPU (gloo, world size 2): frequency sharding of one
migration with a rank-ordered image reduction, and independent lines per rank
(the benchmark's weak-scaling layout).  The per-rank computation is the FP64
oracle; what is under test is the sharding and the exchange."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    import sys
    sys.path.insert(0, ROOT)
    import oracle as O
    import workloads as W
    w = W.Workload("shard", nx=96, dx=12.5, nt=256, dt=0.004, nz=24, dz=5.0, f_lo=5.0, f_hi=60.0, L=8, seed=4)
    v, refl = W.layered_lens_model(w)
    vm = (0.5 * v).astype(np.float32)
    sec = W.normal_incidence_section(w, v, refl)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    kmax = float(om[-1] / vm.min())
    table = O.design_operators(w.nk, kmax, w.dx, w.dz, w.L)
    _, dk = O.k_grid(w.nk, kmax)
    return w, vm, table, O.q_values(om, dk), O.band_dft(sec, w.i0, w.nw)


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle as O
    from paper_1912_05529_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, vm, table, qv, P0 = _problem()
        j0, n = D.frequency_block(w.nw, world, rank)
        if n:
            _, img = O.migrate(P0[j0:j0 + n], vm, table, qv[j0:j0 + n])
        else:
            img = np.zeros((w.nz, w.nx))
        total = D.reduce_images_rank_order(torch.from_numpy(img))
        # weak-scaling layout: an independent line per rank, no exchange
        own = float(np.abs(O.migrate(P0[: 3] * (rank + 1), vm, table, qv[:3])[1]).sum())
        q.put((rank, total.numpy(), own))
    finally:
        dist.destroy_process_group()


def test_frequency_blocks_cover_band_exactly():
    from paper_1912_05529_gb300.distributed import frequency_block
    for nw in (1, 5, 56, 221):
        for world in (1, 2, 3, 8):
            blocks = [frequency_block(nw, world, r) for r in range(world)]
            assert sum(n for _, n in blocks) == nw
            pos = 0
            for j0, n in blocks:
                assert j0 == pos
                pos += n
            assert max(n for _, n in blocks) - min(n for _, n in blocks) <= 1


def test_shard_desc_keeps_table_range():
    import paper_1912_05529_gb300 as fx
    from paper_1912_05529_gb300.distributed import shard_desc
    d = fx.desc_for(nx=64, nz=10, nt=2000, dx=12.5, dz=5.0, dt=0.002, f_lo=5, f_hi=60, L=12, v_min=750.0)
    parts = [shard_desc(d, 3, r) for r in range(3)]
    assert sum(p.nw for p in parts) == d.nw
    assert [p.i0 for p in parts] == [d.i0, d.i0 + parts[0].nw, d.i0 + parts[0].nw + parts[1].nw]
    assert all(p.k_max == d.k_max and p.nk == d.nk for p in parts)
    assert shard_desc(fx.Desc(nx=8, nz=1, nt=64, nw=1, i0=1, L=4, nk=2, dx=1, dz=1, dt=1,
                              theta_max_deg=65, k_max=1.0), 2, 1) is None


def test_two_rank_frequency_shard_equals_single_process():
    import oracle as O
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w, vm, table, qv, P0 = _problem()
    _, full = O.migrate(P0, vm, table, qv)
    res.sort()
    for _, total, _ in res:
        assert np.max(np.abs(total - full)) <= 1e-12 * np.max(np.abs(full))
    assert np.array_equal(res[0][1], res[1][1])       # every rank holds the same sum
    assert res[0][2] > 0 and math.isclose(res[1][2], 2 * res[0][2], rel_tol=1e-12)  # linear in the data


def _shard_worker(rank, world, port, q):
    # the library's shard helper with the oracle as the per-rank depth loop:
    # the helper's bookkeeping (i0, nw, k_max of each block) and rank-order
    # reduction against the full-band oracle
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle as O
    import paper_1912_05529_gb300 as fx
    from paper_1912_05529_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, vm, table, qv, P0 = _problem()
        d = fx.Desc(nx=w.nx, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz, dt=w.dt,
                    theta_max_deg=w.theta_deg, k_max=float(O.omegas(w.i0, w.nw, w.nt, w.dt)[-1] / vm.min()))
        j0, n = D.frequency_block(w.nw, world, rank)

        def oracle_block(sd, slab, vel, tab, launch, stream):
            om = O.omegas(sd.i0, sd.nw, sd.nt, sd.dt)
            _, dk = O.k_grid(sd.nk, sd.k_max)
            _, img = O.migrate(slab, vel, tab, O.q_values(om, dk))
            return torch.from_numpy(img)

        total = D.migrate_frequency_shard(d, P0[j0:j0 + n], vm, table, migrate_fn=oracle_block)
        q.put((rank, total.numpy(), j0, n))
    finally:
        dist.destroy_process_group()


def test_shard_helper_matches_full_band_oracle():
    import oracle as O
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w, vm, table, qv, P0 = _problem()
    _, full = O.migrate(P0, vm, table, qv)
    assert [r[2] for r in res] == [0, res[0][3]] and sum(r[3] for r in res) == w.nw
    for _, total, _, _ in res:
        assert np.max(np.abs(total - full)) <= 1e-12 * np.max(np.abs(full))
    assert np.array_equal(res[0][1], res[1][1])


def _problem3d():
    import sys
    sys.path.insert(0, ROOT)
    import oracle as O
    import oracle.fx3d as F
    import workloads as W
    w = W.Workload3d("shard3d", nx=20, ny=14, dx=20.0, nt=64, dt=0.004, nz=8, dz=10.0, f_lo=5.0, f_hi=40.0,
                     L=4, nk=48, seed=6)
    v, refl = W.layered_lens_model_3d(w)
    vm = (0.5 * v).astype(np.float32)
    sec = W.normal_incidence_section_3d(w, v, refl)
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    kmax = float(om[-1] / vm.min())
    table = F.design2d_operators(w.nk, kmax, w.dx, w.dz, w.L)
    P0 = O.band_dft(sec.reshape(w.ny * w.nx, w.nt), w.i0, w.nw).reshape(w.nw, w.ny, w.nx)
    return w, vm, table, kmax, P0


def _shard3d_worker(rank, world, port, q):
    # the shard helper on a 3-D description, the 3-D oracle as the per-rank
    # depth loop: each rank's block (i0, nw) and the rank-order image sum
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle as O
    import oracle.fx3d as F
    import paper_1912_05529_gb300 as fx
    from paper_1912_05529_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, vm, table, kmax, P0 = _problem3d()
        d = fx.Desc3d(nx=w.nx, ny=w.ny, nz=w.nz, nt=w.nt, nw=w.nw, i0=w.i0, L=w.L, nk=w.nk, dx=w.dx, dz=w.dz,
                      dt=w.dt, theta_max_deg=w.theta_deg, k_max=kmax)
        j0, n = D.frequency_block(w.nw, world, rank)

        def oracle_block(sd, slab, vel, tab, launch, stream):
            assert (sd.ny, sd.nx) == (w.ny, w.nx) and sd.k_max == kmax
            om = O.omegas(sd.i0, sd.nw, sd.nt, sd.dt)
            _, dk = O.k_grid(sd.nk, sd.k_max)
            _, img = F.migrate3d(slab, vel, tab, O.q_values(om, dk))
            return torch.from_numpy(img)

        total = D.migrate_frequency_shard(d, P0[j0:j0 + n], vm, table, migrate_fn=oracle_block)
        q.put((rank, total.numpy(), j0, n))
    finally:
        dist.destroy_process_group()


def test_shard_helper_3d_matches_full_band_oracle():
    import oracle as O
    import oracle.fx3d as F
    O.build()
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard3d_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w, vm, table, kmax, P0 = _problem3d()
    om = O.omegas(w.i0, w.nw, w.nt, w.dt)
    _, dk = O.k_grid(w.nk, kmax)
    _, full = F.migrate3d(P0, vm, table, O.q_values(om, dk))
    assert [r[2] for r in res] == [0, res[0][3]] and sum(r[3] for r in res) == w.nw
    for _, total, _, _ in res:
        assert total.shape == (w.nz, w.ny, w.nx)
        assert np.max(np.abs(total - full)) <= 1e-12 * np.max(np.abs(full))
    assert np.array_equal(res[0][1], res[1][1])
