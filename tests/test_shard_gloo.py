"""World-size-2 test of the mode sharding on CPU (gloo): each rank advances its shard of
sine modes (with the oracle as the CPU stand-in for the per-mode solve), the shards are
all-gathered, and the result equals the unsharded solve."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1901_05128_gb300.shard import mode_shards


def test_mode_shards_cover_exactly():
    for n in (1, 7, 64, 65025):
        for w in (1, 2, 3, 8):
            sh = mode_shards(n, w)
            assert sh[0][0] == 0 and sh[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
            sizes = [hi - lo for lo, hi in sh]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import cq_inputs as ci
    from oracle import scheme as OS
    from oracle import spatial as OSP
    from paper_1901_05128_gb300.shard import gather_modal

    p = ci.Problem(0.35, 0.65, 0.4, 1.0, 120, 2, 9, ci.BDF2, ci.FAST, 8, 16, 9)
    G0 = ci.g0_uniform(p.M, p.dim, 5)
    nm = p.M ** p.dim
    lo, hi = mode_shards(nm, world)[rank]
    lam = OSP.mode_eigenvalues(p.M, p.dim)[lo:hi]
    g0 = OSP.to_modal(G0, p.M, p.dim)[:, lo:hi]
    local = OS.solve_modal(p, lam, g0)[p.N]
    full = gather_modal(torch.tensor(local), nm).numpy()
    if rank == 0:
        np.save(out_path, OSP.to_physical(full, p.M, p.dim))
    dist.destroy_process_group()


def test_sharded_solve_equals_unsharded(tmp_path):
    import cq_inputs as ci
    from oracle import scheme as OS
    out = str(tmp_path / "gn.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    p = ci.Problem(0.35, 0.65, 0.4, 1.0, 120, 2, 9, ci.BDF2, ci.FAST, 8, 16, 9)
    ref = OS.solve(p, ci.g0_uniform(p.M, p.dim, 5))
    got = np.load(out)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
