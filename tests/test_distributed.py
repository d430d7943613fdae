"""Multi-rank combination of independent shift sets (world size 2, gloo, CPU):
every rank gets the Eq. (3) estimate of the union of all ranks' shifts, equal
to the oracle's estimate of the concatenated per-shift values."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1811_11722_gb300.distributed import combine_across_ranks
    rng = np.random.default_rng(100 + rank)
    m = 5 + 3 * rank  # uneven shift counts per rank
    ps = np.stack([1.0 + 1e-3 * rng.normal(size=m), 1e-4 * rng.normal(size=m)], axis=1)
    np.save(os.path.join(outdir, f"ps{rank}.npy"), ps)
    r = combine_across_ranks(ps).as_dict()
    np.save(os.path.join(outdir, f"res{rank}.npy"), np.concatenate([r["mean"], r["var"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_two_ranks_gloo(tmp_path, oracle_lib):
    torch = pytest.importorskip("torch")
    from paper_1811_11722_gb300 import build
    build.build_library()
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    rows = np.concatenate([np.load(tmp_path / "ps0.npy"), np.load(tmp_path / "ps1.npy")], axis=0)
    _, mean, var = oracle_lib.estimate(rows, 1)
    for rank in range(2):
        res = np.load(tmp_path / f"res{rank}.npy")
        assert np.allclose(res[:2], mean, rtol=1e-15, atol=1e-300)
        assert np.allclose(res[2:], var, rtol=1e-12, atol=1e-300)
