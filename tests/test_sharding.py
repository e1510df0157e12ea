"""Band sharding on CPU ranks (gloo, world size 2): the partition and the
reduction that ShardedSolver puts around the GPU solve, with the FP64 oracle
as each rank's local solve. The reduced J, F, Q_rad must equal the oracle's
single-rank solve of all bands (to FP64 rounding of the band sums)."""
import os
import socket

import numpy as np
import pytest

from paper_2107_08145_b300.sharded import band_partition


def test_partition_covers_every_band_once():
    for nb in range(0, 13):
        for world in range(1, 9):
            parts = [band_partition(nb, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == nb
            for (a0, a1), (c0, c1) in zip(parts, parts[1:]):
                assert a1 == c0 and a0 <= a1
            sizes = [b1 - b0 for b0, b1 in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        band_partition(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, shape, nbands, q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2107_08145_b300.sharded import band_partition, reduce_band_sums
    from tests.gpu_common import random_case

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx, ny, nz = shape
        chi, S = random_case(nx, ny, nz, nbands, seed=5)
        b0, b1 = band_partition(nbands, world, rank)
        if b1 > b0:
            P = oracle.Problem(nx, ny, nz, b1 - b0, max_wrap_iters=100000)
            loc = P.solve(chi[b0:b1], S[b0:b1], nthreads=1)
            J, F, Q = (torch.from_numpy(np.ascontiguousarray(loc[k])) for k in ("J", "F", "Q"))
            itop = loc["I_top"]
        else:
            J = torch.zeros((nz, ny, nx), dtype=torch.float64)
            F = torch.zeros((3, nz, ny, nx), dtype=torch.float64)
            Q = torch.zeros((nz, ny, nx), dtype=torch.float64)
            itop = None
        reduce_band_sums(J, F, Q)
        q.put((rank, b0, b1, J.numpy(), F.numpy(), Q.numpy(), itop))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nbands,world", [(4, 2), (3, 2), (1, 2)])
def test_two_gloo_ranks_equal_one(nbands, world):
    import multiprocessing as mp

    import oracle
    from tests.gpu_common import random_case

    shape = (10, 8, 7)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, shape, nbands, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nx, ny, nz = shape
    chi, S = random_case(nx, ny, nz, nbands, seed=5)
    ref = oracle.Problem(nx, ny, nz, nbands, max_wrap_iters=100000).solve(chi, S, nthreads=1)
    itop = np.zeros_like(ref["I_top"])
    for rank, b0, b1, J, F, Q, it in res:
        for got, k in ((J, "J"), (F, "F"), (Q, "Q")):
            scale = np.abs(ref[k]).max()
            assert np.abs(got - ref[k]).max() <= 1e-13 * scale, (rank, k)
        if it is not None:
            itop[b0:b1] = it
    assert np.array_equal(itop, ref["I_top"])  # each band's I_top from the rank that solved it
