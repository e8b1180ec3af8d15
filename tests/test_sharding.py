"""Batch sharding of a GWAS job across ranks: the partitioner, the merge of
per-rank results and the torch.distributed transport, on CPU with gloo ranks
(world size 2 and 3).  Per-rank results are the FP64 reference statistics of
the rank's own SNP columns: the semi-parallel statistics of a SNP depend only
on its column and the covariate phase, so shards must merge into exactly the
full computation."""
import os
import socket

import numpy as np
import pytest

from oracle import gwas_fp64
from paper_1902_04303_gb300.datagen import make_gwas
from paper_1902_04303_gb300.sharding import merge_shards, shard_batches, snp_range


@pytest.mark.parametrize("n_batches", [0, 1, 2, 5, 42, 1563])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_cover_every_batch_once_and_balance(n_batches, world):
    ranges = [shard_batches(n_batches, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n_batches
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0  # contiguous, no gap, no overlap
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n_batches
    assert sizes == sorted(sizes, reverse=True)


def test_bad_shard_requests_raise():
    for args in ((4, 0, 0), (4, 2, 2), (4, 2, -1), (-1, 2, 0)):
        with pytest.raises(ValueError):
            shard_batches(*args)


def test_merge_rejects_overlap_and_reports_gaps():
    k = 10
    a = np.arange(k, dtype=float)
    num, den, ok = merge_shards([(0, 4, a, a), (4, 10, a, a)], k)
    assert ok and np.array_equal(num, a)
    _, _, ok = merge_shards([(0, 4, a, a), (5, 10, a, a)], k)
    assert not ok
    with pytest.raises(RuntimeError):
        merge_shards([(0, 5, a, a), (4, 10, a, a)], k)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, d, k, tau, kappa, out_dir):
    import torch.distributed as dist

    from paper_1902_04303_gb300.sharding import gather_results, max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data = make_gwas(n, d, k, seed=3)
        A = gwas_fp64.xtx_inv(data.X)
        n_batches = -(-k // tau)
        b0, b1 = shard_batches(n_batches, world, rank)
        s0, s1 = snp_range(b0, b1, tau, k)
        num = np.full(k, np.nan)
        den = np.full(k, np.nan)
        if s1 > s0:
            ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S[:, s0:s1], kappa=kappa, A=A)
            num[s0:s1] = ref["num"]
            den[s0:s1] = ref["den"]
        gnum, gden, complete = gather_results(num, den, b0, b1, tau)
        slowest = max_over_ranks(10.0 + rank)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), num=gnum, den=gden,
                 complete=complete, slowest=slowest)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,k,tau", [(2, 300, 64), (3, 100, 64)])
def test_gloo_ranks_merge_into_the_full_computation(tmp_path, world, k, tau):
    """world 3 with two batches leaves one rank without work."""
    import torch.multiprocessing as mp

    n, d, kappa = 40, 3, 1
    mp.start_processes(_rank_main, args=(world, _free_port(), n, d, k, tau, kappa, str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    data = make_gwas(n, d, k, seed=3)
    full = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=kappa,
                                        A=gwas_fp64.xtx_inv(data.X))
    for r in range(world):
        got = np.load(tmp_path / ("rank%d.npz" % r))
        assert bool(got["complete"])
        # the same statistics up to BLAS blocking of the column subsets
        assert np.allclose(got["num"], full["num"], rtol=1e-12, atol=1e-12)
        assert np.allclose(got["den"], full["den"], rtol=1e-12, atol=1e-12)
        assert float(got["slowest"]) == 10.0 + world - 1


class _PlainJob:
    """Stand-in for gwhe.Job with the same call sequence, computing the FP64
    reference statistics of the batches it is asked for."""

    def __init__(self, n, d, k, tau):
        self.n, self.d, self.k = n, d, k
        self.layout = {"tau": tau, "batches": -(-k // tau)}
        self.calls = []
        self.kept = []

    def encrypt_inputs(self, X, A, y):
        self.X, self.A, self.y = X, A, y
        self.calls.append("encrypt")

    def fit(self, kappa):
        self.kappa = kappa
        self.calls.append("fit")

    def snp_stats(self, S, b0, b1):
        self.calls.append(("batches", b0, b1))
        self.kept.append((b0, b1, S))

    # the batch-invariant state: here the plaintext inputs the fit used,
    # as float64 words carried in an int64 buffer
    def _state(self):
        return np.concatenate([self.X.ravel(), self.A.ravel(), self.y.ravel(), [self.kappa]])

    def state_words(self):
        return self._state().size

    def export_state(self, buf):
        import torch
        self.calls.append("export")
        buf.copy_(torch.from_numpy(self._state().view(np.int64)))

    def import_state(self, buf):
        self.calls.append("import")
        v = buf.numpy().view(np.float64)
        n, d = self.n, self.d
        self.X = v[:n * d].reshape(n, d)
        self.A = v[n * d:n * d + d * d].reshape(d, d)
        self.y = v[n * d + d * d:n * d + d * d + n]
        self.kappa = int(v[-1])

    def decrypt_results(self):
        num = np.full(self.k, np.nan)
        den = np.full(self.k, np.nan)
        for b0, b1, S in self.kept:
            s0, s1 = snp_range(b0, b1, self.layout["tau"], self.k)
            ref = gwas_fp64.semi_parallel_fp64(self.X, self.y, S[:, s0:s1], kappa=self.kappa,
                                               A=self.A)
            num[s0:s1], den[s0:s1] = ref["num"], ref["den"]
        return num, den


def _job_main(rank, world, port, out_dir, share_state=True):
    import torch.distributed as dist

    from paper_1902_04303_gb300.sharding import run_sharded_job

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, d, k, tau = 32, 3, 200, 64
        data = make_gwas(n, d, k, seed=9)
        job = _PlainJob(n, d, k, tau)
        num, den, rng = run_sharded_job(None, job, data.X, gwas_fp64.xtx_inv(data.X), data.y,
                                        data.S, 1, rank, world, share_state=share_state)
        np.savez(os.path.join(out_dir, "job%d.npz" % rank), num=num, den=den, rng=np.array(rng),
                 calls=np.array([str(c) for c in job.calls]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("share_state", [True, False])
def test_run_sharded_job_on_gloo_ranks(tmp_path, share_state):
    """With share_state rank 0 alone fits and broadcasts the batch-invariant
    state, which rank 1 imports; without it every rank fits.  Each rank
    evaluates only its own batch range and ends with the complete results
    (4 batches over 2 ranks)."""
    import torch.multiprocessing as mp

    mp.start_processes(_job_main, args=(2, _free_port(), str(tmp_path), share_state), nprocs=2,
                       start_method="spawn", join=True)
    data = make_gwas(32, 3, 200, seed=9)
    full = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1,
                                        A=gwas_fp64.xtx_inv(data.X))
    want_ranges = [(0, 2), (2, 4)]
    for r in range(2):
        got = np.load(tmp_path / ("job%d.npz" % r))
        assert tuple(got["rng"]) == want_ranges[r]
        batches = str(("batches",) + want_ranges[r])
        if not share_state:
            want_calls = ["encrypt", "fit", batches]
        elif r == 0:
            want_calls = ["encrypt", "fit", "export", batches]
        else:
            want_calls = ["import", batches]
        assert list(got["calls"]) == want_calls
        assert np.allclose(got["num"], full["num"], rtol=1e-12, atol=1e-12)
        assert np.allclose(got["den"], full["den"], rtol=1e-12, atol=1e-12)
