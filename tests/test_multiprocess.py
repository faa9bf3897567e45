"""The N > 1 paths without GPUs (gloo, world size 2, on CPU): bench.py's ranks are
independent replicas and the job's step time is the maximum over ranks; the sector
partition of the multi-GPU design evolves contiguous N-ranges apart and rebuilds
the moments from per-rank sums with a two-layer halo."""
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
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, "cpu")  # rank 1 is the slow one
        dist.barrier()
        q.put((rank, ms, bench.job_throughput(world, 4.0e9, ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_with_two_gloo_ranks():
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
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 15.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 4.0e9 / 15e-3)


# ------------------------------------------------ sector partition with a halo

def _partition_case():
    import numpy as np

    import workloads as wl

    M = 5
    w = wl.dispersion_quadratic(M)
    L = wl.long_range_coupling(M, 0.15)
    z = np.array([0.5, 0.9j, 1.1, -0.6 + 0.4j, 0.3])
    return M, w, L, z, 0, 9


def _partition_rank(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle as orc
    from paper_2111_00050_gb300 import partition

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        M, w, L, z, n_lo, n_hi = _partition_case()
        full = orc.Space(M, orc.all_sectors(M, n_lo, n_hi))
        psi0, _ = orc.coherent_state(full, z)
        plans = partition.plan(full.sectors, [float(d) for d in full.dims], world)
        me = plans[rank]
        # this rank's sectors evolve alone: no data from other ranks
        own = orc.Space(M, [full.sectors[s] for s in me.sectors])
        x = np.concatenate([psi0[full.sector_slice(s)] for s in me.sectors])
        x = orc.rk4(own, w, L, x, 2e-3, 25)
        # observation step: the two layers below this rank's range arrive from the
        # rank that holds them (each rank sends its top two layers up)
        top = [i for i, s in enumerate(me.sectors) if full.sectors[s][0] > me.n_hi - 2]
        send = np.concatenate([x[own.sector_slice(i)] for i in top]) if top else np.zeros(0, complex)
        if rank + 1 < world:
            dist.send(torch.from_numpy(send.view(np.float64).copy()), dst=rank + 1)
        halo = np.zeros(0, complex)
        if rank > 0 and me.halo:
            prev = plans[rank - 1]  # holds both halo layers here (it has more than two layers)
            n_sent = int(sum(full.dims[s] for s in prev.sectors if full.sectors[s][0] > prev.n_hi - 2))
            whole = torch.zeros(2 * n_sent, dtype=torch.float64)
            dist.recv(whole, src=rank - 1)
            got = whole.numpy().view(np.complex128)
            # keep the sectors of the two layers below n_lo (the sender's top layers)
            sent_secs = [s for s in prev.sectors if full.sectors[s][0] > prev.n_hi - 2]
            offs = np.cumsum([0] + [int(full.dims[s]) for s in sent_secs])
            halo = np.concatenate([got[offs[i]:offs[i + 1]] for i, s in enumerate(sent_secs) if s in me.halo])
        # partial moments: sources are this rank's kets, targets its kets and the halo
        ext = orc.Space(M, [full.sectors[s] for s in me.halo] + [full.sectors[s] for s in me.sectors])
        phi = np.concatenate([halo, x])
        src = np.concatenate([np.zeros_like(halo), x])
        raw = [np.vdot(src, src).real, 0.0]
        N_of = ext.basis.sum(axis=1)
        raw[1] = float(np.sum(np.abs(src) ** 2 * N_of))
        a = [np.vdot(phi, orc.apply_mode_op(ext, src, "a", i)) for i in range(M)]
        Mij = [np.vdot(phi, orc.apply_mode_op(ext, orc.apply_mode_op(ext, src, "a", j), "adag", i))
               for i in range(M) for j in range(M)]
        aa = [np.vdot(phi, orc.apply_mode_op(ext, orc.apply_mode_op(ext, src, "a", j), "a", i))
              for i in range(M) for j in range(M)]
        vec = np.concatenate([raw, np.array(a + Mij + aa, dtype=np.complex128).view(np.float64)])
        t = torch.from_numpy(vec.copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        q.put((rank, me.n_lo, me.n_hi, t.numpy()))
    finally:
        dist.destroy_process_group()


def test_sector_partition_with_halo_reproduces_the_moments():
    """The multi-GPU design on two gloo ranks with the CPU oracle: contiguous
    N-ranges of a coherent state (M = 5, N <= 9) evolve on separate ranks without
    communication; at the observation step each rank receives the two layers below
    its range, sums the moments over its own kets, and the sum over ranks equals
    the single-process moments of the whole evolved state."""
    import numpy as np
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    import oracle as orc
    from paper_2111_00050_gb300 import partition

    M, w, L, z, n_lo, n_hi = _partition_case()
    full = orc.Space(M, orc.all_sectors(M, n_lo, n_hi))
    plans = partition.plan(full.sectors, [float(d) for d in full.dims], 2)
    assert plans[0].n_lo == n_lo and plans[1].n_hi == n_hi and plans[0].n_hi + 1 == plans[1].n_lo
    assert abs(plans[0].work - plans[1].work) < 0.35 * (plans[0].work + plans[1].work)
    psi0, _ = orc.coherent_state(full, z)
    ref_state = orc.rk4(full, w, L, psi0, 2e-3, 25)
    m = orc.moments(full, ref_state)
    ref = np.concatenate([[m["norm"], m["N"]],
                          np.concatenate([m["a"], m["Mij"].reshape(-1), m["aa"].reshape(-1)]).view(np.float64)])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, lo, hi, got in res:
        np.testing.assert_allclose(got, ref, atol=1e-12)


def test_partition_plan_balances_layers():
    """Contiguous layers, every sector on exactly one rank, halos of two layers, and
    more ranks than layers give empty ranges."""
    sys.path.insert(0, ROOT)
    from paper_2111_00050_gb300 import partition

    sectors = [(N, P) for N in range(0, 12) for P in range(3)]
    weights = [float((N + 1) ** 3) for N, _ in sectors]
    for nr in (1, 2, 3, 5):
        plans = partition.plan(sectors, weights, nr)
        owned = sorted(s for p in plans for s in p.sectors)
        assert owned == list(range(len(sectors)))
        for p in plans[1:]:
            if p.sectors:
                assert all(sectors[s][0] in (p.n_lo - 1, p.n_lo - 2) for s in p.halo)
                assert partition.owner_of_layer(plans, p.n_lo - 1) == p.rank - 1
        works = [p.work for p in plans if p.sectors]
        assert max(works) <= 2.2 * sum(weights) / nr
    plans = partition.plan(sectors[:6], weights[:6], 4)  # 2 layers, 4 ranks
    assert sum(1 for p in plans if not p.sectors) == 2
