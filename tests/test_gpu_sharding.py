"""Sharding one encrypted GWAS job by SNP-batch ranges with the covariate
phase's batch-invariant state computed once and broadcast: the state moves
through a flat buffer (host or device) into jobs that never ran the fit, and
their batches equal the fitting job's bit for bit.  The two-rank case runs as
two gloo processes on one GPU (their kernels never wait on each other: the
broadcast and the gather go through host memory)."""
import os
import socket

import numpy as np
import pytest

from oracle import gwas_fp64
from paper_1902_04303_gb300.datagen import make_gwas

pytestmark = pytest.mark.gpu

LOGN, L, K, DNUM, SEED = 10, 21, 7, 3, 17
N_, D_, K_ = 16, 3, 300  # five batches of 64 SNPs


@pytest.fixture(scope="module")
def g():
    import torch
    torch.cuda.set_device(0)
    from paper_1902_04303_gb300 import build
    build.build()
    from paper_1902_04303_gb300 import gwhe
    return gwhe


def _job(g, ctx, layout, data, A, fit=True):
    job = g.Job(ctx, N_, D_, K_, layout=layout)
    if fit:
        job.encrypt_inputs(data.X, A, data.y)
        job.fit(1)
    return job


@pytest.mark.parametrize("layout,host_tier", [("factored", 0), ("mccp", 0), ("mccp", 4)])
def test_state_moves_through_host_and_device_buffers(g, layout, host_tier):
    import torch
    data = make_gwas(N_, D_, K_, seed=21)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(LOGN, L, K=K, dnum=DNUM, seed=SEED)
    full = g.Job(ctx, N_, D_, K_, layout=layout)
    ctx.keygen(rot_steps=full.rotation_steps(), conj=True)
    full.encrypt_inputs(data.X, A, data.y)
    full.fit(1)
    host = full.export_state()
    assert host.dtype == np.uint64 and host.size == full.state_words()
    dev = torch.empty(full.state_words(), dtype=torch.int64, device="cuda")
    full.export_state(dev)
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), host)
    full.snp_stats(data.S)
    want = full.decrypt_results()
    for buf in (host, dev):
        job = _job(g, ctx, layout, data, A, fit=False)
        if host_tier:
            job.set_host_state(host_tier)
        with pytest.raises(g.GwheError):
            job.snp_stats(data.S)  # no state yet
        job.import_state(buf)
        job.snp_stats(data.S, 2, 5)  # a rank's range only
        job.snp_stats(data.S, 0, 2)
        for bi in range(5):
            for which in range(3):
                assert np.array_equal(job.ct(which, bi).export(), full.ct(which, bi).export())
        got = job.decrypt_results()
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    # a buffer made for another shape is refused
    other = g.Job(ctx, N_, D_ + 1, K_, layout=layout)
    with pytest.raises(g.GwheError) as e:
        other.import_state(host)
    assert e.value.code == -1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_1902_04303_gb300 import gwhe
    from paper_1902_04303_gb300.sharding import run_sharded_job

    torch.cuda.set_device(0)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data = make_gwas(N_, D_, K_, seed=21)
        A = gwas_fp64.xtx_inv(data.X)
        ctx = gwhe.Context(LOGN, L, K=K, dnum=DNUM, seed=SEED)  # same keys on every rank
        job = gwhe.Job(ctx, N_, D_, K_, layout="factored")
        ctx.keygen(rot_steps=job.rotation_steps(), conj=True)
        num, den, rng = run_sharded_job(ctx, job, data.X, A, data.y, data.S, 1, rank, world)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), num=num, den=den,
                 rng=np.array(rng), fitted=np.array(ctx.ks_histogram()[15:].sum() > 0))
        job.close()
        ctx.close()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_one_fit(g, tmp_path):
    """Rank 0 fits and broadcasts the state; rank 1 imports it, runs no
    covariate phase (no key switch above the batch levels) and evaluates
    its own batches; both end with the one-process job's statistics."""
    import torch.multiprocessing as mp

    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn", join=True)
    data = make_gwas(N_, D_, K_, seed=21)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(LOGN, L, K=K, dnum=DNUM, seed=SEED)
    full = g.Job(ctx, N_, D_, K_, layout="factored")
    ctx.keygen(rot_steps=full.rotation_steps(), conj=True)
    full.encrypt_inputs(data.X, A, data.y)
    full.fit(1)
    full.snp_stats(data.S)
    num, den = full.decrypt_results()
    for r, want_rng, fitted in ((0, (0, 3), True), (1, (3, 5), False)):
        got = np.load(tmp_path / ("rank%d.npz" % r))
        assert tuple(got["rng"]) == want_rng
        assert bool(got["fitted"]) == fitted
        assert np.array_equal(got["num"], num, equal_nan=True)
        assert np.array_equal(got["den"], den, equal_nan=True)
