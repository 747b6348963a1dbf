"""The slab decomposition's host logic, on the CPU: the partition of the rows
(klb_slab_partition) and the neighbours whose rows fill each slab's ghost rows
(klb_slab_neighbors), exercised by two gloo ranks that each own one slab of a
grid, exchange the three rows next to each cut every step and step their slab
with the FP64 oracle: the gathered result equals the oracle's whole-grid run
bit for bit (a node's update reads only its stencil, Eq. 47).  No GPU: the two
C functions are host-only and the steps are the oracle's."""
import os
import socket

import numpy as np
import pytest

from oracle import core
from paper_1010_4124_gb300 import inputs, klb

NX, NY, STEPS = 24, 23, 4


def _problem(bcy):
    return inputs.Problem("slabs", NX, NY, 0.01, 0.012, 2e-5, 4e-5, STEPS, bc_x=("periodic", "periodic"),
                          bc_y=(bcy, bcy))


def _params(pb):
    return core.Params(nx=pb.nx, ny=pb.ny, dx=pb.dx, dy=pb.dy, dt=pb.dt, tau=pb.tau, bc_x=pb.bc_x, bc_y=pb.bc_y)


def test_partition_and_neighbors():
    r0, r = klb.slab_partition(23, 3)
    assert r == [8, 8, 7] and r0 == [0, 8, 16]
    with pytest.raises(klb.KlbError):
        klb.slab_partition(8, 3)  # a slab of 2 rows: shallower than the ghost layer
    for bcy, expect in (("periodic", [(2, 1), (0, 2), (1, 0)]), ("outflow", [(-1, 1), (0, 2), (1, -1)])):
        p = klb.make_params(NX, 23, 0.01, 0.01, 1e-5, 1e-5, bc_y=(bcy, bcy))
        assert [klb.slab_neighbors(p, 3, k) for k in range(3)] == expect


def _slab_step(p_full, f_slab, lo_rows, hi_rows):
    """One oracle step of a slab whose ghost rows (3 below, 3 above) are given:
    the slab with its ghost rows as a window, stepped with a periodic y (the
    window's rim is wrong after the step and is cut off)."""
    win = np.concatenate([lo_rows, f_slab, hi_rows], axis=1)
    pw = core.Params(nx=p_full.nx, ny=win.shape[1], dx=p_full.dx, dy=p_full.dy, dt=p_full.dt, tau=p_full.tau,
                     bc_x=p_full.bc_x, bc_y=("periodic", "periodic"))
    return core.step(pw, win)[:, 3:-3, :]


def _rank(rank, world, port, bcy, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb = _problem(bcy)
    p = _params(pb)
    f = core.init_feq(p, *inputs.smooth_random_fields(NX, NY, seed=5, amp=0.08))
    r0, r = klb.slab_partition(NY, world)
    kp = klb.make_params(NX, NY, pb.dx, pb.dy, pb.dt, pb.tau, bc_y=pb.bc_y)
    below, above = klb.slab_neighbors(kp, world, rank)
    mine = f[:, r0[rank]:r0[rank] + r[rank], :].copy()
    for _ in range(STEPS):
        # my edge rows to the neighbours, theirs into my ghost rows; a side
        # without a neighbour is the domain's own (outflow: the edge row copied)
        lo = np.repeat(mine[:, :1, :], 3, axis=1)
        hi = np.repeat(mine[:, -1:, :], 3, axis=1)
        reqs = []
        recv = {}
        for nb, rows, key in ((below, mine[:, :3, :], "lo"), (above, mine[:, -3:, :], "hi")):
            if nb < 0:
                continue
            if nb == rank:  # one slab, periodic: its own rows
                recv[key] = (mine[:, -3:, :] if key == "lo" else mine[:, :3, :]).copy()
                continue
            buf = torch.empty(rows.shape, dtype=torch.float64)
            recv[key] = buf
            tag_send = 0 if key == "lo" else 1  # a lower side's rows are the neighbour's upper ghosts
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(rows)), nb, tag=tag_send))
            reqs.append(dist.irecv(buf, nb, tag=1 - tag_send))
        for q in reqs:
            q.wait()
        if "lo" in recv:
            lo = np.asarray(recv["lo"])
        if "hi" in recv:
            hi = np.asarray(recv["hi"])
        mine = _slab_step(p, mine, lo, hi)
    gathered = [torch.empty((19, r[k], NX), dtype=torch.float64) for k in range(world)] if rank == 0 else None
    if rank == 0:
        gathered[0].copy_(torch.from_numpy(mine))
        for k in range(1, world):
            dist.recv(gathered[k], k)
        np.save(out, np.concatenate([g.numpy() for g in gathered], axis=1))
    else:
        dist.send(torch.from_numpy(np.ascontiguousarray(mine)), 0)
    dist.destroy_process_group()


@pytest.mark.parametrize("bcy", ["periodic", "outflow"])
def test_two_gloo_ranks_reproduce_the_whole_grid(bcy, tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "slabs.npy")
    mp.start_processes(_rank, args=(2, port, bcy, out), nprocs=2, start_method="spawn")
    pb = _problem(bcy)
    p = _params(pb)
    f = core.init_feq(p, *inputs.smooth_random_fields(NX, NY, seed=5, amp=0.08))
    ref, _ = core.run(p, f, STEPS)
    got = np.load(out)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)
