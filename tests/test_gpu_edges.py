"""Edge cases of the encrypted GWAS job on the GPU against the CPU oracle:
a single SNP (an odd SNP count leaves the imaginary half of the last packed
pair empty), the intercept alone (d = 1), a cohort that fills the slots
(n = M: one column block per ciphertext, two SNPs per batch), a cohort size
that is a power of two (nb = n), an empty batch range, and batch ranges
evaluated out of order.  Ciphertexts bit for bit with the oracle's circuit;
decrypted statistics within |d b'| <= 5e-3 of the FP64 reference."""
import numpy as np
import pytest

from oracle import gwas_fp64
from oracle.circuit import Circuit, Layout, rotation_steps
from oracle.ckks import OracleCKKS, galois_conj, galois_rot
from paper_1902_04303_gb300.datagen import make_gwas

pytestmark = pytest.mark.gpu

LOGN, L, K, DNUM, SEED = 10, 21, 7, 3, 23


@pytest.fixture(scope="module")
def g():
    import torch
    torch.cuda.set_device(0)
    from paper_1902_04303_gb300 import build
    build.build()
    from paper_1902_04303_gb300 import gwhe
    return gwhe


def run_both(g, n, d, k, seed, check_batches):
    """the factored job on the GPU and the oracle's circuit; returns
    (job, circuit, data, A, layout)"""
    data = make_gwas(n, d, k, seed=seed)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(LOGN, n, d, k)
    steps = rotation_steps(lay, factored=True)
    ctx = g.Context(LOGN, L, K=K, dnum=DNUM, seed=SEED)
    ctx.keygen(rot_steps=steps, conj=True)
    job = g.Job(ctx, n, d, k, layout="factored")
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    o = OracleCKKS(logN=LOGN, L=L, K=K, dnum=DNUM, seed=SEED)
    o.keygen(galois=[galois_rot(LOGN, r) for r in steps] + [galois_conj(LOGN)])
    c = Circuit(o, lay, factored=True)
    c.encrypt_inputs(data.X, A, data.y)
    c.fit(kappa=1)
    for bi in check_batches:
        want = c.snp_batch_factored(c.encrypt_snp_batch_ccp(data.S, bi))
        for which in range(3):
            assert np.array_equal(job.ct(which, bi).export(), want[which].c), (bi, which)
    return job, c, data, A, lay


def check_fp64(num, den, data, A, k):
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    assert np.all(np.isfinite(num[:k])) and np.all(np.isfinite(den[:k]))
    ok = np.abs(ref["den"]) > 1e-6
    assert np.max(np.abs(num[ok] / den[ok] - ref["b"][ok]), initial=0.0) <= 5e-3


def test_single_snp(g):
    job, c, data, A, lay = run_both(g, 16, 3, 1, seed=31, check_batches=[0])
    assert lay.batches == 1
    num, den = job.decrypt_results()
    assert num.shape == (1,) and den.shape == (1,)
    check_fp64(num, den, data, A, 1)


def test_intercept_only(g):
    job, c, data, A, lay = run_both(g, 16, 1, 40, seed=32, check_batches=[0])
    num, den = job.decrypt_results()
    check_fp64(num, den, data, A, 40)


def test_cohort_fills_the_slots(g):
    """n = M = 512 at N = 2^10: nb = M, one block per ciphertext, tau = 2;
    five SNPs make three batches, the last holding one SNP."""
    n = 1 << (LOGN - 1)
    job, c, data, A, lay = run_both(g, n, 2, 5, seed=33, check_batches=[0, 2])
    assert lay.nb == n and lay.B == 1 and lay.tau == 2 and lay.batches == 3
    num, den = job.decrypt_results()
    check_fp64(num, den, data, A, 5)


def test_power_of_two_cohort(g):
    job, c, data, A, lay = run_both(g, 32, 3, 70, seed=34, check_batches=[1])
    assert lay.nb == 32
    num, den = job.decrypt_results()
    check_fp64(num, den, data, A, 70)


def test_empty_and_out_of_order_ranges(g):
    """an empty range is a no-op; ranges in any order give the one-call
    ciphertexts"""
    n, d, k = 16, 3, 300  # five batches of 64 SNPs
    data = make_gwas(n, d, k, seed=35)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(LOGN, L, K=K, dnum=DNUM, seed=SEED)
    full = g.Job(ctx, n, d, k, layout="factored")
    ctx.keygen(rot_steps=full.rotation_steps(), conj=True)
    parts = g.Job(ctx, n, d, k, layout="factored")
    for j in (full, parts):
        j.encrypt_inputs(data.X, A, data.y)
        j.fit(1)
    full.snp_stats(data.S)
    ks0 = ctx.ks_histogram().copy()
    parts.snp_stats(data.S, 2, 2)
    assert np.array_equal(ctx.ks_histogram(), ks0)  # nothing issued
    for b0, b1 in ((3, 5), (0, 1), (1, 3)):
        parts.snp_stats(data.S, b0, b1)
    for bi in range(5):
        for which in range(3):
            assert np.array_equal(parts.ct(which, bi).export(), full.ct(which, bi).export())
    with pytest.raises(g.GwheError):
        parts.snp_stats(data.S, 4, 6)  # past the last batch


def test_sprime_beside_the_fit_with_any_later_chunking(g):
    """Batches encrypted before the fit get their S' during it; the SNP loop
    uses a precomputed chunk when its bounds match and otherwise computes
    S' from the kept encrypted batches: ranges that split the precomputed
    chunks, and a gap in the encrypted batches, give the fused job's
    ciphertexts bit for bit."""
    n, d, k = 16, 3, 300  # five batches of 64 SNPs
    data = make_gwas(n, d, k, seed=36)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(LOGN, L, K=K, dnum=DNUM, seed=SEED)
    full = g.Job(ctx, n, d, k, layout="factored")
    ctx.keygen(rot_steps=full.rotation_steps(), conj=True)
    full.encrypt_inputs(data.X, A, data.y)
    full.fit(1)
    full.snp_stats(data.S)
    want = [[full.ct(w, bi).export() for w in range(3)] for bi in range(5)]
    plans = (
        ([(0, 5)], [(0, 5)], []),                  # one chunk, used as computed
        ([(0, 5)], [(2, 5), (0, 2)], []),          # split ranges: computed again
        ([(0, 2), (3, 5)], [(0, 2), (2, 5)], [(2, 3)]),  # a gap, filled after the fit
    )
    for before, ranges, after in plans:
        job = g.Job(ctx, n, d, k, layout="factored")
        job.encrypt_inputs(data.X, A, data.y)
        for b0, b1 in before:
            job.encrypt_snps(data.S, b0, b1)
        job.fit(1)
        for b0, b1 in after:
            job.encrypt_snps(data.S, b0, b1)
        for b0, b1 in ranges:
            job.snp_stats(None, b0, b1)
        for bi in range(5):
            for w in range(3):
                assert np.array_equal(job.ct(w, bi).export(), want[bi][w]), (before, bi, w)
        with pytest.raises(g.GwheError):
            job.snp_stats(None, 0, 1)  # every batch consumed
        job.close()
