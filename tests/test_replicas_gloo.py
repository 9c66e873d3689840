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


def _oracle_resolve(accum, tour_count, k0):
    """Stands in for the library's Resolve on a rank without a GPU."""
    from oracle import oracle as O
    return torch.from_numpy(O.resolve(accum.numpy(), k0, tour_count))


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
        img, total = merge_and_resolve(acc, r["tour_count"], k0, resolve=_oracle_resolve)
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


class _OracleRank:
    """Stands in for one rank's renderer: Alg. 1 and the following steps run
    by the oracle on this rank's chains."""

    def __init__(self, tgt):
        self.tgt = tgt

    def init_chains(self, n, seed, params, frame=0):
        from oracle import oracle as O
        r = O.restore_run(self.tgt, params, seed, np.arange(n), n_steps=0, record=False)
        self.n, self.seed, self.params = n, seed, params
        self.p_init_sum = r["p_init_sum"]
        self.p_lambda = r["p_init_sum"] / n

    def p_sum(self):
        return self.p_init_sum, self.n

    @staticmethod
    def k0_from_p_sum(p_sum, n, params):
        return p_sum / n / (params.m * params.dt)

    def run(self, n_steps):
        from oracle import oracle as O
        return O.restore_run(self.tgt, self.params, self.seed, np.arange(self.n), n_steps=n_steps, record=False)


def _mixture():
    from oracle import oracle as O
    from paper_2605_08916_gb300 import scenes as S
    return O.target(S.gaussian_mixture(seed=4, d=4, K=3, sig_range=(0.05, 0.08), width=8, height=8))


def _run_rank_agreed(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2605_08916_gb300.replicas import init_chains_agreed, merge_and_resolve, replica_seed
        r = _OracleRank(_mixture())
        k0 = init_chains_agreed(r, 200 + 56 * rank, replica_seed(91, rank), O.make_params(L=1, drift="exact", k0=0.0))
        out = r.run(24)
        img, total = merge_and_resolve(torch.from_numpy(out["accum"].copy()), out["tour_count"], k0,
                                       resolve=_oracle_resolve)
        np.save(os.path.join(out_dir, f"agreed{rank}.npy"), np.concatenate([[k0, total], img.numpy().ravel()]))
    finally:
        dist.destroy_process_group()


def test_ranks_agree_on_k0_and_merge_to_the_union(tmp_path):
    """Alg. 1 with p_lambda estimated from the union of both ranks' initial
    samples (chain counts differ per rank), then 24 steps and the merge:
    equals one run over the union with that k0, and both ranks use it."""
    port = _free_port()
    mp.start_processes(_run_rank_agreed, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    from oracle import oracle as O
    from paper_2605_08916_gb300.replicas import replica_seed
    tgt = _mixture()
    ns = [200, 256]
    est = O.make_params(L=1, drift="exact", k0=0.0)
    sums = [O.restore_run(tgt, est, replica_seed(91, k), np.arange(ns[k]), 0, record=False)["p_init_sum"]
            for k in range(2)]
    local_k0 = [s / n / (est.m * est.dt) for s, n in zip(sums, ns)]
    k0 = sum(sums) / sum(ns) / (est.m * est.dt)
    assert abs(local_k0[0] / local_k0[1] - 1.0) > 1e-3      # the ranks' own estimates differ
    prm = O.make_params(L=1, drift="exact", k0=k0)
    acc, tc = 0, 0
    for k in range(2):
        r = O.restore_run(tgt, prm, replica_seed(91, k), np.arange(ns[k]), 24, record=False)
        acc = acc + r["accum"]
        tc += r["tour_count"]
    union = (acc * (k0 / tc)).ravel()
    for k in range(2):
        got = np.load(tmp_path / f"agreed{k}.npy")
        assert got[0] == pytest.approx(k0, rel=1e-15)
        assert int(got[1]) == tc
        np.testing.assert_allclose(got[2:], union, rtol=1e-13, atol=0)


def test_init_agreement_without_a_process_group_is_local():
    from oracle import oracle as O
    from paper_2605_08916_gb300.replicas import agree_p_sum, init_chains_agreed
    assert agree_p_sum(2.5, 10) == (2.5, 10)
    big = (1 << 62) + 3   # counts travel as 64-bit integers, exactly
    assert agree_p_sum(1.0, big) == (1.0, big)
    r = _OracleRank(_mixture())
    k0 = init_chains_agreed(r, 64, 5, O.make_params(L=1, drift="exact", k0=0.0))
    assert k0 == pytest.approx(r.p_lambda / (64 * 1e-5), rel=1e-12)
    assert r.params.k0 == k0
    given = O.make_params(L=1, drift="exact", k0=123.0)
    assert init_chains_agreed(r, 64, 5, given) == 123.0 and r.params is given


def test_merge_hands_the_summed_buffers_to_resolve():
    """Without a process group the merge is the identity on (accum, tour
    count), and Resolve receives them with k0 unchanged; the tour count
    stays an exact 64-bit integer."""
    from paper_2605_08916_gb300.replicas import merge_and_resolve
    seen = []

    def resolve(acc, tc, k0):
        seen.append((acc.clone(), tc, k0))
        return acc * 0 + 1

    big = (1 << 62) + 1
    img, total = merge_and_resolve(torch.full((12,), 3.0, dtype=torch.float64), big, 5.0, resolve=resolve)
    assert total == big and seen[0][1] == big and seen[0][2] == 5.0
    assert torch.equal(seen[0][0], torch.full((12,), 3.0, dtype=torch.float64)) and torch.equal(img, torch.ones(12,
                                                                                                         dtype=torch.float64))
