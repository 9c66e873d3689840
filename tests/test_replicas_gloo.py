"""The multi-GPU path on CPU: two gloo ranks each run their own chains (the
oracle stands in for each rank's device), merge with the replica all-reduce,
and the result equals Resolve over the union of both ranks' chains."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run_rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2605_08916_gb300 import scenes as S
        from paper_2605_08916_gb300.replicas import merge_and_resolve, replica_seed
        mix = S.gaussian_mixture(seed=2, d=4, K=2, sig_range=(0.1, 0.12), width=8, height=8)
        tgt = O.target(mix)
        k0 = 1.0 / (64 * 1e-5)
        prm = O.make_params(L=1, drift="exact", k0=k0)
        r = O.restore_run(tgt, prm, seed=replica_seed(77, rank), chain_ids=np.arange(256), n_steps=32,
                          record=False)
        acc = torch.from_numpy(r["accum"].copy())
        img, total = merge_and_resolve(acc, r["tour_count"], k0)
        np.save(os.path.join(out_dir, f"img{rank}.npy"), img.numpy())
        np.save(os.path.join(out_dir, f"tc{rank}.npy"), np.array([total]))
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_equals_union(tmp_path):
    port = _free_port()
    mp.start_processes(_run_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    from oracle import oracle as O
    from paper_2605_08916_gb300 import scenes as S
    from paper_2605_08916_gb300.replicas import replica_seed
    mix = S.gaussian_mixture(seed=2, d=4, K=2, sig_range=(0.1, 0.12), width=8, height=8)
    tgt = O.target(mix)
    k0 = 1.0 / (64 * 1e-5)
    prm = O.make_params(L=1, drift="exact", k0=k0)
    acc = 0
    tc = 0
    for rank in range(2):
        r = O.restore_run(tgt, prm, seed=replica_seed(77, rank), chain_ids=np.arange(256), n_steps=32, record=False)
        acc = acc + r["accum"]
        tc += r["tour_count"]
    union = acc * (k0 / tc)
    for rank in range(2):
        img = np.load(tmp_path / f"img{rank}.npy")
        assert int(np.load(tmp_path / f"tc{rank}.npy")[0]) == tc
        assert np.array_equal(img, union)
    assert replica_seed(77, 0) == 77 and replica_seed(77, 1) != 77
