"""One shot split into two z slabs over two gloo ranks on the CPU.

Each rank steps its slab with the FP64 oracle and, before every step,
exchanges the four u^n planes next to the cut with its neighbour: the halo
exchange of the paper's distributed runs (Sec. 6.4, a Cartesian split; here
along z only).  The radius-4 stencil of an owned plane then sees exactly the
neighbours it has in one domain, and every point update is computed by the
same operations, so the decomposed run must equal the monolithic oracle bit
for bit: final wavefield and traces, with a source and receivers on and next
to the cut.  The layers are off: the oracle derives its damping profile from
its own grid, which is the global profile only without layers.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import workloads as W

R = 4   # stencil radius: halo planes per side


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    p = W.tiny_problem(shape=(30, 20, 24), nt=25, nbl=0, nsrc=2, nrec=12, seed=17)
    p.src_ijk[0] = [10, 9, 14]          # one plane above the cut (k = 15)
    p.src_ijk[1] = [5, 5, 15]           # on the first plane below it
    p.rec_ijk[:4] = [[3, 3, 15], [4, 4, 14], [20, 10, 0], [20, 10, 29]]
    return p


def _slab_run(rank, dist):
    import torch

    import oracle
    p = _problem()
    nz, ny, nx = p.vel.shape
    cut = nz // 2
    own = (0, cut) if rank == 0 else (cut, nz)
    lo, hi = (0, cut + R) if rank == 0 else (cut - R, nz)     # the slab with its halo
    vel = np.ascontiguousarray(p.vel[lo:hi])
    src_sel = [s for s in range(len(p.src_ijk)) if own[0] <= p.src_ijk[s][2] < own[1]]
    rec_sel = [r for r in range(len(p.rec_ijk)) if own[0] <= p.rec_ijk[r][2] < own[1]]
    src = p.src_ijk[src_sel] - np.array([0, 0, lo], np.int32)
    rec = p.rec_ijk[rec_sel] - np.array([0, 0, lo], np.int32)
    up = np.zeros(vel.shape)
    uc = np.zeros(vel.shape)
    traces = np.zeros((p.nt, len(p.rec_ijk)))
    send_lo = cut - R - lo if rank == 0 else cut - lo         # my owned planes next to the cut
    recv_lo = cut - lo if rank == 0 else 0                    # my halo planes
    for n in range(p.nt):
        mine = torch.from_numpy(np.ascontiguousarray(uc[send_lo:send_lo + R]))
        theirs = torch.empty_like(mine)
        if rank == 0:
            dist.send(mine, 1)
            dist.recv(theirs, 1)
        else:
            dist.recv(theirs, 0)
            dist.send(mine, 0)
        uc[recv_lo:recv_lo + R] = theirs.numpy()
        tr, up, uc = oracle.forward(vel, p.h, p.dt, 1, nbl=0, src_ijk=src, wavelet=p.wavelet[src_sel, n:n + 1],
                                    rec_ijk=rec, u_prev0=up, u_cur0=uc, want_state=True, nthreads=1)
        traces[n, rec_sel] = tr[0]
    return uc[own[0] - lo:own[1] - lo], traces


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u, tr = _slab_run(rank, dist)
    out[rank] = (u, tr)
    dist.barrier()
    dist.destroy_process_group()


def test_two_z_slabs_equal_one_domain_bit_for_bit(orc):
    mgr = mp.get_context("spawn").Manager()   # the oracle fixture has started OpenMP threads
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    p = _problem()
    tr_o, _, u_o = orc.forward(p.vel, p.h, p.dt, p.nt, nbl=0, src_ijk=p.src_ijk, wavelet=p.wavelet,
                               rec_ijk=p.rec_ijk, want_state=True, nthreads=1)
    u = np.concatenate([out[0][0], out[1][0]], axis=0)
    tr = out[0][1] + out[1][1]           # each receiver is recorded by the rank that owns its plane
    assert np.abs(u_o).max() > 0 and np.abs(tr_o[:, :2]).max() > 0
    assert np.array_equal(u, u_o)
    assert np.array_equal(tr, tr_o)
