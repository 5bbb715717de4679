"""Multi-rank path on CPU (gloo, world size 2): disjoint history ranges per
rank, transported independently, then combined by one sum-reduction, give the
same tally as a single process over the whole range.  The per-rank transport
here is the oracle (the GPU library needs a GPU); the sharding and the
combine step are the ones the GPU path uses."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_0910_0329_gb300 import sharding, workloads as W


def test_history_ranges_are_disjoint_and_cover():
    seen = set()
    for step in range(3):
        for rank in range(4):
            f, n = sharding.history_range(rank, 4, step, 10)
            ids = set(range(f, f + n))
            assert not (ids & seen)
            seen |= ids
    assert seen == set(range(120))
    parts = sharding.split(1001, 3)
    assert [n for _, n in parts] == [334, 334, 333]
    assert parts[1][0] == 334 and sum(n for _, n in parts) == 1001
    with pytest.raises(ValueError):
        sharding.history_range(4, 4, 0, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out_dir):
    import torch.distributed as dist

    from oracle import oracle as O

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.c1_photon_wbw()
    first, cnt = sharding.split(n, world)[rank]
    r = O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, cnt, 11, h0=first, workers=1)
    s1 = torch.from_numpy(r.S1.copy())
    s2 = torch.from_numpy(r.S2.copy())
    sharding.combine_tallies([s1, s2])
    if rank == 0:
        np.save(os.path.join(out_dir, "s1.npy"), s1.numpy())
        np.save(os.path.join(out_dir, "s2.npy"), s2.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_combine_equals_single_process(tmp_path):
    n = 600
    mp.start_processes(_worker, args=(2, _free_port(), n, str(tmp_path)), nprocs=2, start_method="spawn")
    from oracle import oracle as O

    wl = W.c1_photon_wbw()
    ref = O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, n, 11, workers=1)
    np.testing.assert_allclose(np.load(tmp_path / "s1.npy"), ref.S1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.load(tmp_path / "s2.npy"), ref.S2, rtol=1e-12, atol=1e-12)
