"""The N > 1 host path of bench.py on CPU: world_size 2 over gloo.

Each rank runs an independent replica; the job time is the slowest rank's
time (max over ranks) and the whole-job rate counts every rank's units.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    bench._barrier(ws)
    ms_local = [1.5, 4.0][rank]
    ms, rate = bench.aggregate(ws, ms_local, 1000)
    out[rank] = (ms, rate)
    tdist.destroy_process_group()


def test_two_ranks_gloo_max_time_and_total_rate():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True,
                       start_method="spawn")
    for rank in range(2):
        ms, rate = out[rank]
        assert ms == pytest.approx(4.0)
        assert rate == pytest.approx(2 * 1000 / 4.0e-3)


# ---------------------------------------------------------------------------
# The multi-rank data plane's host logic (paper_2112_01852_gb300.dist) on two
# gloo ranks: the t-ring exchange delivers each face to the right neighbour,
# the all-reduce sums over ranks, and the distributed CG, run over a stand-in
# vector space whose operator needs the same face exchange (a massive
# Laplacian on a periodic 1D lattice split into slabs, CPU tensors), reaches
# the dense solution.


def _ring_ops(comm, n_loc, nrhs, m2, dtype=None):
    import torch
    dtype = torch.float64 if dtype is None else dtype

    class RingOps:
        def new(self):
            return torch.zeros(nrhs, n_loc, dtype=dtype)

        def apply(self, out, inp):
            # faces: the first site goes to the rank below, the last to the rank above
            send_dn = inp[:, :1].contiguous()
            send_up = inp[:, -1:].contiguous()
            recv_up, recv_dn = torch.empty_like(send_dn), torch.empty_like(send_up)
            comm.exchange(send_dn, send_up, recv_up, recv_dn)
            right = torch.cat([inp[:, 1:], recv_up], dim=1)
            left = torch.cat([recv_dn, inp[:, :-1]], dim=1)
            out.copy_((m2 + 2.0) * inp - left - right)

        def dot(self, a, b):
            return comm.allreduce((a * b).sum(dim=1).tolist())

        def axpby(self, y, a, x, b):
            y.copy_(torch.tensor(a, dtype=dtype)[:, None] * x +
                    torch.tensor(b, dtype=dtype)[:, None] * y)

    return RingOps()


def _dist_worker(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as tdist
    from paper_2112_01852_gb300 import dist
    tdist.init_process_group("gloo", rank=rank, world_size=world,
                             init_method="tcp://127.0.0.1:%d" % port)
    comm = dist.TComm()
    assert (comm.rank, comm.size, comm.up, comm.dn) == (rank, world, (rank + 1) % world,
                                                         (rank - 1) % world)
    send_dn = torch.full((3,), 10.0 * rank + 1.0)
    send_up = torch.full((3,), 10.0 * rank + 2.0)
    recv_up, recv_dn = torch.empty(3), torch.empty(3)
    comm.exchange(send_dn, send_up, recv_up, recv_dn)
    exch = (float(recv_up[0]), float(recv_dn[0]))
    red = comm.allreduce([rank + 1.0, 2.0 ** rank])
    # distributed CG on the slab-decomposed ring
    n_loc, nrhs, m2 = 8, 2, 0.3
    N = n_loc * world
    rng = np.random.default_rng(7)
    bglob = rng.standard_normal((nrhs, N))
    ops = _ring_ops(comm, n_loc, nrhs, m2)
    b = torch.from_numpy(bglob[:, rank * n_loc:(rank + 1) * n_loc].copy())
    x = ops.new()
    conv, iters, res = dist.cg(ops, x, b, nrhs, 1e-12, 500)
    xs = comm.allgather_numpy(x.numpy())
    # mixed precision by defect correction: float64 residuals and solution,
    # float32 inner CG
    lo = _ring_ops(comm, n_loc, nrhs, m2, torch.float32)
    xm = ops.new()
    mconv, miters, mouter, mres = dist.mixed_cg(ops, lo, lambda o, i: o.copy_(i),
                                                lambda o, i: o.copy_(i), xm, b, nrhs, 1e-12,
                                                2000, inner_tol=1e-4)
    xms = comm.allgather_numpy(xm.numpy())
    out[rank] = (exch, red, conv, iters, res, np.concatenate(xs, axis=1) if world > 1 else xs,
                 (mconv, miters, mouter, mres,
                  np.concatenate(xms, axis=1) if world > 1 else xms))
    tdist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_data_plane_and_distributed_cg(world):
    import numpy as np
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_dist_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    n_loc, nrhs, m2 = 8, 2, 0.3
    N = n_loc * world
    A = (m2 + 2.0) * np.eye(N) - np.roll(np.eye(N), 1, axis=1) - np.roll(np.eye(N), -1, axis=1)
    bglob = np.random.default_rng(7).standard_normal((nrhs, N))
    want = np.linalg.solve(A, bglob.T).T
    for rank in range(world):
        exch, red, conv, iters, res, x, mixed = out[rank]
        mconv, miters, mouter, mres, xm = mixed
        assert all(mconv) and max(mres) <= 1e-12 and 2 <= mouter <= 8, (mouter, mres)
        assert np.allclose(xm, want, rtol=0, atol=1e-10)
        up, dn = (rank + 1) % world, (rank - 1) % world
        # recv_up is the rank above's send_dn, recv_dn the rank below's send_up
        assert exch == (10.0 * up + 1.0, 10.0 * dn + 2.0)
        assert red == [sum(range(1, world + 1)) * 1.0, float(2 ** world - 1)]
        assert all(conv) and max(res) <= 1e-12 and 0 < iters <= 500
        assert np.allclose(x, want, rtol=0, atol=1e-10)


def test_mixed_cg_single_process_edge_cases():
    # defect correction on one process (no torch.distributed): an RHS that is
    # already solved gets a zero correction and stays converged, an iteration
    # budget too small to converge reports not converged, and a zero RHS is
    # solved by x = 0
    import numpy as np
    import torch
    from paper_2112_01852_gb300 import dist

    class LocalComm:
        def exchange(self, send_dn, send_up, recv_up, recv_dn):
            recv_up.copy_(send_dn)  # one rank: both neighbours are itself
            recv_dn.copy_(send_up)

        def allreduce(self, values):
            return list(values)

    n, nrhs, m2 = 16, 3, 0.3
    hi = _ring_ops(LocalComm(), n, nrhs, m2)
    lo = _ring_ops(LocalComm(), n, nrhs, m2, torch.float32)
    A = (m2 + 2.0) * np.eye(n) - np.roll(np.eye(n), 1, axis=1) - np.roll(np.eye(n), -1, axis=1)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((nrhs, n))
    b[2] = 0.0                                   # a zero right-hand side
    x = hi.new()
    x[1] = torch.from_numpy(np.linalg.solve(A, b[1]))  # RHS 1 starts solved
    bt = torch.from_numpy(b)
    conv, iters, outer, res = dist.mixed_cg(hi, lo, lambda o, i: o.copy_(i),
                                            lambda o, i: o.copy_(i), x, bt, nrhs, 1e-12, 500,
                                            inner_tol=1e-4)
    assert all(conv) and max(res) <= 1e-12, res
    assert np.allclose(x.numpy()[:2], np.linalg.solve(A, b[:2].T).T, rtol=0, atol=1e-10)
    assert np.all(x.numpy()[2] == 0.0)
    x2 = hi.new()
    conv2, iters2, _, res2 = dist.mixed_cg(hi, lo, lambda o, i: o.copy_(i),
                                           lambda o, i: o.copy_(i), x2, bt, nrhs, 1e-12, 2,
                                           inner_tol=1e-4)
    assert iters2 <= 4 and not conv2[0] and res2[0] > 1e-12
