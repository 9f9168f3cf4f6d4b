"""The halo plan of a channel split along y, on CPU with two gloo ranks.

Each rank owns one slab (its interior rows plus a ghost row on each side) and
advances it with the oracle's routines, exchanging ghost rows with the other
rank over torch.distributed (gloo) exactly as the library's plan
(nh_slab_plan, read from the C library on the host) prescribes: populations
after every LB step, u / n^P / n / sigma between the stages of an FD update.
The interior rows must equal the single-domain oracle run bit for bit, which
shows that the plan names every row and component the stencils read.  The
oracle is the compute engine here; the library is used for its plan only.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2503_06610_gb300 import inputs as I

NX, NY, NZ = 10, 9, 6
SPLIT = [4, 5]
STEPS = 7
DT_FD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _params():
    return dict(I.LESLIE_ALIGN_09, nx=NX, ny=NY, nz=NZ, walls_z=True, anchoring="none", shifted=True, tau=0.8,
                g=(1e-5, -3e-6, 0.0), K=0.03, q0=0.6, W0=0.01, dt_fd=DT_FD, alpha1=0.1, alpha4p=0.2)


def _rows(k):
    y0 = sum(SPLIT[:k])
    return (y0 - 1 + np.arange(SPLIT[k] + 2)) % NY


def _split(a, comps, k):
    return np.ascontiguousarray(np.asarray(a).reshape(comps, NZ, NY, NX)[:, :, _rows(k), :].reshape(comps, -1))


def _exchange(rank, plan, field, comps, ny_slab):
    """Apply the plan's row copies to this rank's field [comps][N_slab] over gloo."""
    f = field.reshape(comps, NZ, ny_slab, NX)
    reqs, recvs = [], []
    for j, (src, srow, dst, drow, cs) in enumerate(plan):
        if src == rank:
            buf = torch.from_numpy(np.ascontiguousarray(f[cs, :, srow, :]))
            reqs.append(dist.isend(buf, dst=dst, tag=j))
        if dst == rank:
            buf = torch.empty((len(cs), NZ, NX), dtype=torch.float64)
            reqs.append(dist.irecv(buf, src=src, tag=j))
            recvs.append((buf, drow, cs))
    for r in reqs:
        r.wait()
    for buf, drow, cs in recvs:
        f[cs, :, drow, :] = buf.numpy()
    return f.reshape(comps, -1)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2503_06610_gb300 import nh
    plans = {kind: nh.nh_slab_plan(SPLIT, kind) for kind in (0, 1, 2)}
    ny = SPLIT[rank] + 2
    p = O.OracleParams.from_dict(dict(_params(), ny=ny))
    n0 = I.skyrmion_tubes(NX, NY, NZ, [(5.0, 4.0)], 3.5)
    n = _split(n0, 3, rank)
    u = np.zeros((3, p.N))
    f = O.init_populations(p)
    sig = _exchange(rank, plans[2], O.stress(p, n, u), 9, ny)
    F = O.force(p, sig)
    for s in range(1, STEPS + 1):
        f, rho, u = O.lb_step(p, f, F)
        f = _exchange(rank, plans[0], f, 19, ny)
        if s % DT_FD == 0:
            u = _exchange(rank, plans[1], u, 3, ny)
            rate_old = O.director_rate(p, n, u)
            nP = _exchange(rank, plans[1], n + DT_FD * rate_old, 3, ny)
            rate_P = O.director_rate(p, nP, u)
            n = n + DT_FD * (0.5 * (rate_old + rate_P))
            n = n / np.sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2])
            n = _exchange(rank, plans[1], n, 3, ny)
            sig = _exchange(rank, plans[2], O.stress(p, n, u), 9, ny)
            F = O.force(p, sig)
    inner = lambda a, c: a.reshape(c, NZ, ny, NX)[:, :, 1:-1, :].copy()
    out[rank] = (inner(n, 3), inner(u, 3), inner(f, 19))
    dist.barrier()
    dist.destroy_process_group()


def test_two_slab_halo_plan_gloo(oracle_mod):
    O = oracle_mod
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    p = O.OracleParams.from_dict(_params())
    n0 = I.skyrmion_tubes(NX, NY, NZ, [(5.0, 4.0)], 3.5)
    ref = O.OracleSim(p, n0).step(STEPS)
    for k in range(world):
        y = slice(sum(SPLIT[:k]), sum(SPLIT[:k + 1]))
        n, u, f = out[k]
        assert np.array_equal(n, ref.n.reshape(3, NZ, NY, NX)[:, :, y, :])
        assert np.array_equal(u, ref.u.reshape(3, NZ, NY, NX)[:, :, y, :])
        assert np.array_equal(f, ref.f.reshape(19, NZ, NY, NX)[:, :, y, :])
    assert np.max(np.abs(ref.u)) > 1e-7


def test_slab_plan_rows_and_components():
    from paper_2503_06610_gb300 import nh
    nh.load_library()
    plan = nh.nh_slab_plan([3, 4, 2], nh.NH_HALO_POPULATIONS)
    assert len(plan) == 6
    # slab 1: lower ghost from slab 0's last interior row, upper ghost from slab 2's first
    assert plan[2] == (0, 3, 1, 0, [3, 7, 10, 15, 17])
    assert plan[3] == (2, 1, 1, 5, [4, 8, 9, 16, 18])
    # periodic: slab 0's lower ghost comes from the last slab
    assert plan[0] == (2, 2, 0, 0, [3, 7, 10, 15, 17])
    # one slab is its own neighbour: the periodic channel
    assert nh.nh_slab_plan([5], nh.NH_HALO_VECTOR) == [(0, 5, 0, 0, [0, 1, 2]), (0, 1, 0, 6, [0, 1, 2])]
    assert nh.nh_slab_plan([2, 2], nh.NH_HALO_STRESS)[0][4] == list(range(9))
    for bad in (([], 0), ([0, 3], 0), ([3], 7)):
        with pytest.raises(nh.NHError) as e:
            nh.nh_slab_plan(*bad)
        assert e.value.code == nh.NH_EINVAL
