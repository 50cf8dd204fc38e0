"""The sharded J/K design on CPU: gloo ranks (world size 2) split the auxiliary
index into contiguous 128-function blocks, build their partial J and K with the
oracle and sum them with one all-reduce each; the bench's max-over-ranks
timing.  No GPU: every machine here has one."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2601_08077_gb300 import shard


def test_aux_block_ranges_partition():
    for naux in (1, 127, 128, 129, 300, 900, 3600):
        for world in (1, 2, 3, 4, 8):
            rs = shard.aux_block_ranges(naux, world)
            assert len(rs) == world
            assert rs[0][0] == 0 and rs[-1][1] == naux
            for (a0, a1), (b0, b1) in zip(rs, rs[1:]):
                assert a1 == b0
            nb = [-(-(p1 - p0) // 128) for p0, p1 in rs]
            assert max(nb) - min(nb) <= 1
            assert all(p0 % 128 == 0 for p0, p1 in rs if p1 > p0)   # empty runs sit at naux
    with pytest.raises(ValueError):
        shard.aux_block_ranges(10, 0)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    from oracle import df_oracle as O
    from paper_2601_08077_gb300 import inputs, shard as sh
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, B, C, D = inputs.make_inputs(inputs.SMALL)
        p0, p1 = sh.aux_block_ranges(B.shape[0], world)[rank]
        Bs = B[p0:p1]
        J = torch.from_numpy(O.coulomb(Bs, O.rho(Bs, D)))   # rho_P needs only B_P
        K = torch.from_numpy(O.exchange(Bs, C))
        sh.allreduce_sum_(J)
        sh.allreduce_sum_(K)
        t = sh.max_over_ranks(10.0 * (rank + 1))
        if rank == 0:
            np.save(os.path.join(outdir, "J.npy"), J.numpy())
            np.save(os.path.join(outdir, "K.npy"), K.numpy())
            np.save(os.path.join(outdir, "t.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_sharded_build_sums_to_the_full_build(tmp_path):
    from oracle import df_oracle as O
    from paper_2601_08077_gb300 import inputs
    world = 2
    mp.get_context("spawn")
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    _, B, C, D = inputs.make_inputs(inputs.SMALL)
    J_ref = O.coulomb(B, O.rho(B, D))
    K_ref = O.exchange(B, C)
    J = np.load(tmp_path / "J.npy")
    K = np.load(tmp_path / "K.npy")
    # the same sums in another order: FP64 rounding only
    assert np.max(np.abs(J - J_ref)) <= 1e-13 * np.max(np.abs(J_ref))
    assert np.max(np.abs(K - K_ref)) <= 1e-13 * np.max(np.abs(K_ref))
    assert float(np.load(tmp_path / "t.npy")[0]) == 20.0
