"""World-size-2 tests of the mode sharding on CPU (gloo). ``solve_sharded`` (the product's
sharded solve) runs with a CPU stand-in for the binding whose ``fp2s_solve_modes`` is the
oracle's per-mode scheme (the CUDA entry point itself is tested on the GPU, shard by shard,
in test_gpu_modes.py); the shards are all-gathered and the result equals the unsharded
solve."""
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

    from paper_1901_05128_gb300.shard import solve_sharded

    p = ci.Problem(0.35, 0.65, 0.4, 1.0, 120, 2, 9, ci.BDF2, ci.FAST, 8, 16, 9)
    G0 = ci.g0_uniform(p.M, p.dim, 5)
    nm = p.M ** p.dim
    g0m = torch.tensor(OSP.to_modal(G0, p.M, p.dim))
    full = solve_sharded(_OracleBinding(p, rank), "problem", g0m).numpy()
    if rank == 0:
        np.save(out_path, OSP.to_physical(full, p.M, p.dim))
    # more ranks than modes: the empty shards contribute nothing
    tiny = ci.Problem(0.35, 0.65, 0.4, 1.0, 20, 1, 1, ci.BE, ci.FAST, 8, 0, 2)
    one = solve_sharded(_OracleBinding(tiny, rank), "problem",
                        torch.tensor([[1.0], [0.5]], dtype=torch.float64)).numpy()
    if rank == 0:
        np.save(out_path + ".tiny.npy", one)
    dist.destroy_process_group()


class _OracleBinding:
    """CPU stand-in for the binding module: fp2s_solve_modes runs the oracle's per-mode
    scheme on the requested range; the size query returns a dummy size. Records the ranges
    it was asked for."""

    def __init__(self, p, rank):
        self.p, self.rank, self.calls = p, rank, []

    def workspace(self, nbytes, device):
        return torch.empty(nbytes, dtype=torch.uint8, device=device)

    def fp2s_solve_modes(self, problem, lo, hi, g0, gN, ws, stream=None):
        from oracle import scheme as OS
        from oracle import spatial as OSP
        if ws is None:
            return 256
        assert g0.shape == (2, hi - lo)
        self.calls.append((lo, hi))
        lam = OSP.mode_eigenvalues(self.p.M, self.p.dim)[lo:hi]
        gN.copy_(torch.tensor(OS.solve_modal(self.p, lam, g0.numpy())[self.p.N]))
        return 0


def test_sharded_solve_equals_unsharded(tmp_path):
    import cq_inputs as ci
    from oracle import scheme as OS
    out = str(tmp_path / "gn.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    p = ci.Problem(0.35, 0.65, 0.4, 1.0, 120, 2, 9, ci.BDF2, ci.FAST, 8, 16, 9)
    ref = OS.solve(p, ci.g0_uniform(p.M, p.dim, 5))
    got = np.load(out)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
    tiny = ci.Problem(0.35, 0.65, 0.4, 1.0, 20, 1, 1, ci.BE, ci.FAST, 8, 0, 2)
    from oracle import spatial as OSP
    ref1 = OS.solve_modal(tiny, OSP.mode_eigenvalues(1, 1), np.array([[1.0], [0.5]]))[tiny.N]
    assert np.array_equal(np.load(out + ".tiny.npy"), ref1)
