"""Serving: continuous batching of GWAS jobs (worker threads with their own
streams sharing one context's keys, admission by HBM footprint).  Each
request's results must be the same alone and in the mix: bit for bit, since
a job's ciphertexts depend only on its inputs, its nonce and the shared keys;
and within the acceptance tolerances of the FP64 reference."""
import numpy as np
import pytest

from oracle import gwas_fp64
from paper_1902_04303_gb300.datagen import make_gwas

pytestmark = pytest.mark.gpu

SHAPES = [(16, 3, 100), (30, 2, 200), (12, 4, 64), (50, 3, 150), (16, 3, 100), (9, 5, 40)]


@pytest.fixture(scope="module")
def g():
    import torch
    torch.cuda.set_device(0)
    from paper_1902_04303_gb300 import build
    build.build()
    from paper_1902_04303_gb300 import gwhe
    return gwhe


@pytest.fixture(scope="module")
def setup(g):
    ctx = g.Context(10, 21, K=7, dnum=3, seed=41)
    steps = []
    for n, d, k in SHAPES:
        job = g.Job(ctx, n, d, k)
        steps += [r for r in job.rotation_steps() if r not in steps]
        job.close()
    ctx.keygen(rot_steps=steps, conj=True)
    reqs = []
    for i, (n, d, k) in enumerate(SHAPES):
        data = make_gwas(n, d, k, seed=500 + i)
        reqs.append((data, gwas_fp64.xtx_inv(data.X), i + 1))  # nonce i + 1
    alone = []
    for data, A, nonce in reqs:
        n, d = data.X.shape
        job = g.Job(ctx, n, d, data.S.shape[1])
        job.set_nonce(nonce)
        job.encrypt_inputs(data.X, A, data.y)
        job.fit(1)
        job.snp_stats(data.S)
        alone.append(job.decrypt_results())
        job.close()
    return ctx, reqs, alone


def test_results_are_the_same_alone_and_in_the_mix(g, setup):
    ctx, reqs, alone = setup
    srv = g.Server(ctx, workers=3, chunk_batches=2)
    ids = [srv.submit(data.X, A, data.y, data.S, nonce=nonce) for data, A, nonce in reqs]
    spans = []
    for rid, (data, A, nonce), (num0, den0) in zip(ids, reqs, alone):
        num, den, t = srv.wait(rid)
        assert np.array_equal(num, num0) and np.array_equal(den, den0), nonce
        assert t["latency_ms"] >= t["run_ms"] > 0
        assert t["device_end_ms"] > t["device_start_ms"] >= 0
        spans.append((t["device_start_ms"], t["device_end_ms"], t["high_priority"]))
        ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
        ok = np.abs(ref["den"]) > 1e-6
        assert np.max(np.abs(num[ok] / den[ok] - ref["b"][ok])) <= 5e-3
    st = srv.stats()
    assert st["admitted"] == len(reqs) and st["running"] == 0 and st["waiting"] == 0
    assert st["peak_bytes_claimed"] <= st["budget"]
    assert st["live_workers"] == 3
    # the jobs were resident at once and their work overlapped on the device:
    # at some device time at least two jobs' spans are open, and at most one
    # of the jobs running together holds the high-priority stream
    fps = [g.job_footprint(ctx, *data.X.shape, data.S.shape[1], chunk_batches=2)
           for data, _, _ in reqs]
    assert st["max_running"] >= 2 and st["peak_bytes_claimed"] > max(fps)
    overlap = max(sum(1 for a, b, _ in spans if a <= s0 < b) for s0, _, _ in spans)
    assert overlap >= 2, spans
    for s0, _, hi in spans:
        if hi:
            assert sum(1 for a, b, h in spans if h and a <= s0 < b) == 1
    srv.close()


def test_budget_admits_one_job_at_a_time(g, setup):
    """a budget below two jobs' footprints serialises them; results unchanged."""
    ctx, reqs, alone = setup
    fps = [g.job_footprint(ctx, *data.X.shape, data.S.shape[1], chunk_batches=2)
           for data, _, _ in reqs]
    budget = max(fps) + min(fps) - 1
    srv = g.Server(ctx, workers=3, hbm_budget=budget, chunk_batches=2)
    # the genotypes borrowed, not copied, at submission
    ids = [srv.submit(data.X, A, data.y, data.S, nonce=nonce, borrow=True)
           for data, A, nonce in reqs]
    for rid, (num0, den0) in zip(ids, alone):
        num, den, _ = srv.wait(rid)
        assert np.array_equal(num, num0) and np.array_equal(den, den0)
    st = srv.stats()
    assert st["peak_bytes_claimed"] <= budget < 2 * min(fps) + (max(fps) - min(fps))
    srv.close()


def test_oversized_request_is_refused(g, setup):
    ctx, reqs, _ = setup
    data, A, nonce = reqs[0]
    srv = g.Server(ctx, workers=1, hbm_budget=1 << 20)
    with pytest.raises(g.GwheError) as e:
        srv.submit(data.X, A, data.y, data.S, nonce=nonce)
    assert e.value.code == -2  # ENOMEM
    srv.close()


def test_mccp_job_over_budget_runs_in_host_tier(g, setup):
    """An M-CCP job whose footprint with Dup(M_j) on the device exceeds the
    budget is admitted with Dup(M_j) in the host tier; its results equal the
    same job run alone on the device, bit for bit."""
    ctx, reqs, _ = setup
    data, A, nonce = reqs[0]
    n, d = data.X.shape
    k = data.S.shape[1]
    job = g.Job(ctx, n, d, k, layout="mccp")
    job.set_nonce(nonce)
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    num0, den0 = job.decrypt_results()
    job.close()
    fp = g.job_footprint(ctx, n, d, k, layout="mccp", chunk_batches=2)
    srv = g.Server(ctx, workers=2, hbm_budget=fp - 1, chunk_batches=2)
    rid = srv.submit(data.X, A, data.y, data.S, layout="mccp", nonce=nonce)
    num, den, _ = srv.wait(rid)
    assert np.array_equal(num, num0) and np.array_equal(den, den0)
    st = srv.stats()
    assert st["host_tier_jobs"] == 1 and st["peak_bytes_claimed"] < fp
    srv.close()


def test_one_snp_loop_at_a_time(g, setup):
    """With GWHE_SERVER_ONE_SNP_LOOP the SNP loops run one after another on
    the device while other jobs' covariate phases overlap them; results are
    still those of the jobs alone."""
    ctx, reqs, alone = setup
    srv = g.Server(ctx, workers=3, chunk_batches=2, one_snp_loop=True)
    ids = [srv.submit(data.X, A, data.y, data.S, nonce=nonce) for data, A, nonce in reqs]
    loops, spans = [], []
    for rid, (num0, den0) in zip(ids, alone):
        num, den, t = srv.wait(rid)
        assert np.array_equal(num, num0) and np.array_equal(den, den0)
        assert t["high_priority"]
        assert t["device_start_ms"] <= t["snp_start_ms"] < t["snp_end_ms"] <= t["device_end_ms"]
        loops.append((t["snp_start_ms"], t["snp_end_ms"]))
        spans.append((t["device_start_ms"], t["device_end_ms"]))
    loops.sort()
    for (a0, a1), (b0, b1) in zip(loops, loops[1:]):
        assert b0 >= a1, loops  # never two loops at once
    overlap = max(sum(1 for a, b in spans if a <= s0 < b) for s0, _ in spans)
    assert overlap >= 2, spans
    srv.close()
