"""GPU parity of the encrypted GWAS job (Algorithms 1-11) against the CPU oracle:
ciphertexts bit for bit where the oracle can run the circuit, decrypted
results within |d b'| <= 5e-3 and |d(-log10 p)| <= 0.05 of the FP64 reference
at the paper's shape (245 samples, 5 covariates, 10643 SNPs, N = 2^16)."""
import numpy as np
import pytest

from oracle import gwas_fp64
from oracle.circuit import Circuit, Layout, ladder_groups, rotation_steps
from oracle.ckks import OracleCKKS, galois_conj, galois_rot
from oracle.trace import job_ks_histogram
from paper_1902_04303_gb300.datagen import WORKLOADS, make_gwas

pytestmark = pytest.mark.gpu

TOL_B = 5e-3
TOL_LOGP = 0.05


@pytest.fixture(scope="module")
def g():
    import torch
    torch.cuda.set_device(0)
    from paper_1902_04303_gb300 import build
    build.build()
    from paper_1902_04303_gb300 import gwhe
    return gwhe


def check_accuracy(num, den, ref, k):
    assert np.all(np.isfinite(num[:k])) and np.all(np.isfinite(den[:k]))
    ok = np.abs(ref["den"]) > 1e-6  # monomorphic SNPs: den = 0 (degenerate)
    assert np.max(np.abs(den[~ok]), initial=0.0) < 1e-3
    b = num[ok] / den[ok]
    db = np.abs(b - ref["b"][ok])
    assert np.max(db) <= TOL_B, np.max(db)
    dl = np.abs(gwas_fp64.neglog10p(b, 1.0 / den[ok])
                - gwas_fp64.neglog10p(ref["b"][ok], ref["err"][ok]))
    assert np.max(dl) <= TOL_LOGP, np.max(dl)
    return float(np.max(db)), float(np.max(dl))


def test_job_circuit_bit_exact(g):
    """Covariate fit + one ragged batch: every output ciphertext and the
    intermediate z', beta, Dup(M_j), Dup(w), Dup(w z') equal the oracle's."""
    logN, L, K, dnum, seed = 10, 21, 7, 3, 11
    n, d, k = 16, 3, 40
    data = make_gwas(n, d, k, seed=5)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(logN, n, d, k)
    steps = rotation_steps(lay)
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=seed)
    ctx.keygen(rot_steps=steps, conj=True)
    job = g.Job(ctx, n, d, k, layout="mccp")
    ks0 = ctx.ks_histogram().copy()
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    # same key switches at the same levels as the oracle circuit's level trace
    W = dict(logN=logN, L=L, q0_bits=60, scale_bits=40, K=K, sp_bits=60, dnum=dnum, n=n, d=d,
             k=k)
    want, _, _ = job_ks_histogram(W, 1)
    assert np.array_equal(ctx.ks_histogram() - ks0, want)
    o = OracleCKKS(logN=logN, L=L, K=K, dnum=dnum, seed=seed)
    o.keygen(galois=[galois_rot(logN, r) for r in steps] + [galois_conj(logN)])
    c = Circuit(o, lay)
    c.encrypt_inputs(data.X, A, data.y)
    c.fit(kappa=1)
    assert np.array_equal(job.ct(7).export(), c.beta.c)
    assert np.array_equal(job.ct(6).export(), c.zp.c)
    assert np.array_equal(job.ct(4).export(), c.DupW.c)
    assert np.array_equal(job.ct(5).export(), c.DupWZ.c)
    for jj in (0, 7, n - 1):
        assert np.array_equal(job.ct(3, jj).export(), c.DupM[jj].c), jj
    want = c.snp_batch(c.encrypt_snp_batch(data.S, 0))
    for which in range(3):
        assert np.array_equal(job.ct(which, 0).export(), want[which].c), which
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    check_accuracy(num, den, ref, k)


def test_job_split_mode_small_workload(g):
    """The small plain job (N = 2^13, 4 limbs, 1 special prime, n = 64, d = 4,
    k = 256, two batches): the client supplies M, w, w z' (split mode);
    batch outputs bit-exact with the oracle, decrypted within tolerance."""
    W = WORKLOADS["small-n64"]
    data = make_gwas(W["n"], W["d"], W["k"], seed=W["seed"])
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1)
    lay = Layout(W["logN"], W["n"], W["d"], W["k"])
    # colSum only, as its hoisted groups use them
    steps = [r for grp in ladder_groups([1 << i for i in range(int(np.log2(lay.nb)))]) for r in grp]
    ctx = g.Context(W["logN"], W["L"], K=W["K"], dnum=W["dnum"], seed=W["seed"])
    ctx.keygen(rot_steps=steps, conj=True)
    job = g.Job(ctx, W["n"], W["d"], W["k"])
    wz = ref["w"] * ref["zp"]
    job.set_fit_state(ref["M"], ref["w"], wz)
    job.snp_stats(data.S)
    num, den = job.decrypt_results()
    check_accuracy(num, den, ref, W["k"])
    o = OracleCKKS(logN=W["logN"], L=W["L"], K=W["K"], dnum=W["dnum"], seed=W["seed"])
    o.keygen(galois=[galois_rot(W["logN"], r) for r in steps] + [galois_conj(W["logN"])])
    c = Circuit(o, lay)
    c.load_split_state(ref["M"], ref["w"], wz)
    want = c.snp_batch(c.encrypt_snp_batch(data.S, 1))
    for which in range(3):
        assert np.array_equal(job.ct(which, 1).export(), want[which].c), which


def test_job_paper_shape_accuracy(g):
    """245 x 5 x 10643 at N = 2^16 (42 batches, ragged last batch of 147 SNPs):
    decrypted numerators/denominators against the FP64 reference; the
    ciphertexts of this size are checked op by op in test_gpu_parity."""
    W = WORKLOADS["paper-n245"]
    data = make_gwas(W["n"], W["d"], W["k"], seed=W["seed"])
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(W["logN"], W["L"], W["q0_bits"], W["scale_bits"], W["K"], W["sp_bits"],
                    W["dnum"], seed=W["seed"])
    job = g.Job(ctx, W["n"], W["d"], W["k"], layout="mccp")
    ctx.keygen(rot_steps=job.rotation_steps(), conj=True)
    assert job.layout["tau"] == 256 and job.layout["batches"] == 42 and job.layout["H"] == 2
    ks0 = ctx.ks_histogram().copy()
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    want, _, _ = job_ks_histogram(W, 1)
    assert np.array_equal(ctx.ks_histogram() - ks0, want)
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    db, dl = check_accuracy(num, den, ref, W["k"])
    print("paper shape: max |d b'| = %.3g, max |d -log10 p| = %.3g" % (db, dl))


def test_job_rejects_missing_state_and_depth(g):
    ctx = g.Context(10, 4, K=2, dnum=2, seed=1)
    job = g.Job(ctx, 16, 3, 40)
    ctx.keygen(rot_steps=job.rotation_steps(), conj=True)
    assert not job.factored  # four limbs: split-mode layout
    S = np.zeros((16, 40))
    with pytest.raises(g.GwheError):
        job.snp_stats(S)  # no covariate phase yet
    data = make_gwas(16, 3, 40, seed=2)
    job.encrypt_inputs(data.X, gwas_fp64.xtx_inv(data.X), data.y)
    with pytest.raises(g.GwheError) as e:
        job.fit(1)  # four limbs cannot hold the fit
    assert e.value.code == -3


def test_factored_layout_bit_exact(g):
    """Factored layout (second form of eq. Sprime, S as one CCP ciphertext per
    batch): Dup(X_c), Dup((XA)_c) and every batch output equal the oracle's
    factored circuit bit for bit, with the key switches of its level trace."""
    logN, L, K, dnum, seed = 10, 21, 7, 3, 12
    n, d, k = 16, 3, 100  # two batches of 64 SNPs, the second ragged
    data = make_gwas(n, d, k, seed=6)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(logN, n, d, k)
    steps = rotation_steps(lay, factored=True)
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=seed)
    job = g.Job(ctx, n, d, k, layout="factored")
    job.set_nonce(3)  # the encryption ids of a job with nonce 3, on both sides
    assert job.factored and sorted(job.rotation_steps()) == sorted(steps)
    assert job.layout["H"] == 0 and job.layout["batch_limbs"] == 6
    ctx.keygen(rot_steps=steps, conj=True)
    ks0 = ctx.ks_histogram().copy()
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    W = dict(logN=logN, L=L, q0_bits=60, scale_bits=40, K=K, sp_bits=60, dnum=dnum, n=n, d=d,
             k=k)
    want, _, _ = job_ks_histogram(W, 1, factored=True)
    assert np.array_equal(ctx.ks_histogram() - ks0, want)
    o = OracleCKKS(logN=logN, L=L, K=K, dnum=dnum, seed=seed)
    o.keygen(galois=[galois_rot(logN, r) for r in steps] + [galois_conj(logN)])
    c = Circuit(o, lay, factored=True, nonce=3)
    c.encrypt_inputs(data.X, A, data.y)
    c.fit(kappa=1)
    for cc in range(d):
        assert np.array_equal(job.ct(11, cc).export(), c.DupX[cc].c), cc
        assert np.array_equal(job.ct(12, cc).export(), c.DupB[cc].c), cc
    assert np.array_equal(job.ct(4).export(), c.DupW.c)
    assert np.array_equal(job.ct(5).export(), c.DupWZ.c)
    for bi in range(lay.batches):
        want = c.snp_batch_factored(c.encrypt_snp_batch_ccp(data.S, bi))
        for which in range(3):
            assert np.array_equal(job.ct(which, bi).export(), want[which].c), (bi, which)
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    check_accuracy(num, den, ref, k)


def test_factored_layout_paper_shape(g):
    """The paper's shape through the factored layout: 42 CCP batches, the same
    decrypted statistics within tolerance, key switches as the trace says."""
    W = WORKLOADS["paper-n245"]
    data = make_gwas(W["n"], W["d"], W["k"], seed=W["seed"])
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(W["logN"], W["L"], W["q0_bits"], W["scale_bits"], W["K"], W["sp_bits"],
                    W["dnum"], seed=W["seed"])
    job = g.Job(ctx, W["n"], W["d"], W["k"], layout="factored")
    ctx.keygen(rot_steps=job.rotation_steps(), conj=True)
    ks0 = ctx.ks_histogram().copy()
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    want, _, _ = job_ks_histogram(W, 1, factored=True)
    assert np.array_equal(ctx.ks_histogram() - ks0, want)
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    check_accuracy(num, den, ref, W["k"])


def test_large_cohort_auto_factored(g):
    """A cohort beyond the paper's 256-subject limit (n = 600, nb = 1024,
    tau = 64 at N = 2^16): the automatic layout is the factored one and the
    results meet the tolerances."""
    W = dict(WORKLOADS["paper-n245"])
    n, d, k = 600, 4, 1500
    data = make_gwas(n, d, k, seed=77)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(W["logN"], W["L"], W["q0_bits"], W["scale_bits"], W["K"], W["sp_bits"],
                    W["dnum"], seed=78)
    job = g.Job(ctx, n, d, k)
    assert job.factored and job.layout["tau"] == 64 and job.layout["batches"] == 24
    ctx.keygen(rot_steps=job.rotation_steps(), conj=True)
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    check_accuracy(num, den, ref, k)


def test_sharded_batch_ranges_merge_into_one_job(g):
    """The batch ranges two ranks would evaluate, run as two jobs here (one
    GPU: no cross-rank waits), merge into exactly the one-job results."""
    from paper_1902_04303_gb300.sharding import merge_shards, shard_batches, snp_range
    logN, L, K, dnum, seed = 10, 21, 7, 3, 13
    n, d, k = 16, 3, 300  # five batches of 64 SNPs
    data = make_gwas(n, d, k, seed=8)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=seed)
    full = g.Job(ctx, n, d, k)
    ctx.keygen(rot_steps=full.rotation_steps(), conj=True)
    full.encrypt_inputs(data.X, A, data.y)
    full.fit(1)
    full.snp_stats(data.S)
    want_num, want_den = full.decrypt_results()
    shards = []
    for rank in range(2):
        job = g.Job(ctx, n, d, k)
        job.encrypt_inputs(data.X, A, data.y)
        job.fit(1)
        b0, b1 = shard_batches(job.layout["batches"], 2, rank)
        job.snp_stats(data.S, b0, b1)
        num, den = job.decrypt_results()
        s0, s1 = snp_range(b0, b1, job.layout["tau"], k)
        assert np.isnan(num[:s0]).all() and np.isnan(num[s1:]).all()
        shards.append((s0, s1, num, den))
    num, den, complete = merge_shards(shards, k)
    assert complete
    assert np.array_equal(num, want_num) and np.array_equal(den, want_den)


def test_kappa3_circuit_bit_exact(g):
    """kappa = 3 Bohning iterations (Alg. 9) need about 40 limbs: the whole
    factored circuit at N = 2^10 with 40 limbs and 12 special primes, against
    the oracle bit for bit, and the FP64 reference with kappa = 3."""
    logN, L, K, dnum, seed = 10, 40, 12, 3, 14
    n, d, k = 16, 3, 64
    data = make_gwas(n, d, k, seed=15)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(logN, n, d, k)
    steps = rotation_steps(lay, factored=True)
    ctx = g.Context(logN, L, q0_bits=60, scale_bits=45, K=K, dnum=dnum, seed=seed)
    ctx.keygen(rot_steps=steps, conj=True)
    job = g.Job(ctx, n, d, k, layout="factored")
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(3)
    job.snp_stats(data.S)
    o = OracleCKKS(logN=logN, L=L, q0_bits=60, scale_bits=45, K=K, dnum=dnum, seed=seed)
    o.keygen(galois=[galois_rot(logN, r) for r in steps] + [galois_conj(logN)])
    c = Circuit(o, lay, factored=True)
    c.encrypt_inputs(data.X, A, data.y)
    c.fit(kappa=3)
    assert np.array_equal(job.ct(7).export(), c.beta.c)
    want = c.snp_batch_factored(c.encrypt_snp_batch_ccp(data.S, 0))
    for which in range(3):
        assert np.array_equal(job.ct(which, 0).export(), want[which].c), which
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=3, A=A)
    check_accuracy(num, den, ref, k)


def test_paper_ring_kappa3_accuracy(g):
    """The paper's own geometry for its most accurate run: N = 2^17, kappa = 3
    (tau = 512, 21 batches at n = 245), 40 limbs, against FP64 with kappa = 3."""
    n, d, k = 245, 5, 10643
    data = make_gwas(n, d, k, seed=1006)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(17, 40, q0_bits=60, scale_bits=45, K=12, dnum=3, seed=1006)
    job = g.Job(ctx, n, d, k)
    assert job.factored and job.layout["tau"] == 512 and job.layout["batches"] == 21
    ctx.keygen(rot_steps=job.rotation_steps(), conj=True)
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(3)
    job.snp_stats(data.S)
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=3, A=A)
    db, dl = check_accuracy(num, den, ref, k)
    print("N=2^17 kappa=3: max |d b'| = %.3g, max |d -log10 p| = %.3g" % (db, dl))


@pytest.mark.parametrize("layout", ["factored", "mccp"])
def test_host_genotypes_stream_in_chunks(g, layout):
    """Genotypes in host memory stay there: each chunk of 64 batches takes its
    columns through one of two pinned staging slots.  Over three chunks with a
    ragged tail (130 batches of 64 SNPs, the last short) every output
    ciphertext equals that of the same job with S on the device, and a batch
    of the last chunk equals the oracle's."""
    import torch
    logN, L, K, dnum, seed = 10, 21, 7, 3, 12
    n, d = 16, 3
    k = 130 * 64 - 21
    data = make_gwas(n, d, k, seed=8)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(logN, n, d, k)
    assert lay.batches == 130 and lay.tau == 64
    fact = layout == "factored"
    steps = rotation_steps(lay, factored=fact)
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=seed)
    ctx.keygen(rot_steps=steps, conj=True)
    outs, res = [], []
    for S in (data.S, torch.from_numpy(data.S).cuda()):
        job = g.Job(ctx, n, d, k, layout=layout)
        job.encrypt_inputs(data.X, A, data.y)
        job.fit(1)
        job.snp_stats(S)
        outs.append([[job.ct(w, bi).export() for w in range(3)] for bi in range(lay.batches)])
        res.append(job.decrypt_results())
        job.close()
    for bi in range(lay.batches):
        for w in range(3):
            assert np.array_equal(outs[0][bi][w], outs[1][bi][w]), (bi, w)
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    check_accuracy(res[0][0], res[0][1], ref, k)
    if fact:
        o = OracleCKKS(logN=logN, L=L, K=K, dnum=dnum, seed=seed)
        o.keygen(galois=[galois_rot(logN, r) for r in steps] + [galois_conj(logN)])
        c = Circuit(o, lay, factored=True)
        c.encrypt_inputs(data.X, A, data.y)
        c.fit(kappa=1)
        want = c.snp_batch_factored(c.encrypt_snp_batch_ccp(data.S, 129))
        for w in range(3):
            assert np.array_equal(outs[0][129][w], want[w].c), w


@pytest.mark.parametrize("chunk", [5, 16])
def test_mccp_host_tier_state(g, chunk):
    """Dup(M_j) in the host tier (pinned host memory, prefetched chunk columns
    at a time per set of 64 batches, partial tensor sums accumulated): every
    Dup(M_j) and every batch output equals the device-resident job's, over
    three sets of batches and ragged column chunks; split mode as well."""
    logN, L, K, dnum, seed = 10, 21, 7, 3, 11
    n, d = 16, 3
    k = 130 * 64 - 21
    data = make_gwas(n, d, k, seed=9)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(logN, n, d, k)
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=seed)
    ctx.keygen(rot_steps=rotation_steps(lay), conj=True)
    outs = []
    for host in (0, chunk):
        job = g.Job(ctx, n, d, k, layout="mccp")
        job.set_host_state(host)
        job.encrypt_inputs(data.X, A, data.y)
        job.fit(1)
        job.snp_stats(data.S)
        outs.append(([job.ct(3, jj).export() for jj in range(n)],
                     [[job.ct(w, bi).export() for w in range(3)] for bi in range(lay.batches)]))
        job.close()
    for jj in range(n):
        assert np.array_equal(outs[0][0][jj], outs[1][0][jj]), jj
    for bi in range(lay.batches):
        for w in range(3):
            assert np.array_equal(outs[0][1][bi][w], outs[1][1][bi][w]), (bi, w)
    # split mode: the client's Dup(M_j) encryptions go to the host tier too
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    res = []
    for host in (0, chunk):
        job = g.Job(ctx, n, d, k, layout="mccp")
        job.set_host_state(host)
        job.set_fit_state(ref["M"], ref["w"], ref["w"] * ref["zp"])
        job.snp_stats(data.S, 0, 3)
        res.append([[job.ct(w, bi).export() for w in range(3)] for bi in range(3)])
        job.close()
    assert all(np.array_equal(a, b) for ra, rb in zip(*res) for a, b in zip(ra, rb))
    with pytest.raises(g.GwheError):
        g.Job(ctx, n, d, k, layout="mccp").set_host_state(-1)


def _oracle_job(W, lay, steps, data, A, factored, nonce=0):
    o = OracleCKKS(logN=W["logN"], L=W["L"], K=W["K"], dnum=W["dnum"], seed=W["seed"])
    o.keygen(galois=[galois_rot(W["logN"], r) for r in steps] + [galois_conj(W["logN"])])
    c = Circuit(o, lay, factored=factored, nonce=nonce)
    c.encrypt_inputs(data.X, A, data.y)
    c.fit(kappa=1)
    return c


@pytest.mark.parametrize("snps_first", [False, True])
def test_factored_job_bit_exact_on_two_pass_transforms_and_full_groups(g, snps_first):
    """The factored job at N = 2^12, the smallest ring on the two-pass
    transform (with its ModDown epilogue) that the paper-shaped job runs on:
    12 batches in one set (the last ragged, 100 SNPs), so the colSum ladder's
    one-digit hoisted inner product walks 36 items (a full group of 32 and a
    ragged one).  The covariate state (beta, z, z', masked w, Dup(X_c),
    Dup((XA)_c), Dup(w), Dup(w z')) and the outputs of the first and the
    ragged last batch equal the oracle's circuit, which computes its own
    state batch by batch.  snps_first: the batches are encrypted before the
    fit, which then computes their S' on a second stream beside the
    covariate phase."""
    W = dict(logN=12, L=21, q0_bits=60, scale_bits=40, K=7, sp_bits=60, dnum=3, seed=14,
             n=16, d=3, k=11 * 256 + 100)
    data = make_gwas(W["n"], W["d"], W["k"], seed=8)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(W["logN"], W["n"], W["d"], W["k"])
    assert lay.tau == 256 and lay.batches == 12
    steps = rotation_steps(lay, factored=True)
    ctx = g.Context(W["logN"], W["L"], K=W["K"], dnum=W["dnum"], seed=W["seed"])
    ctx.keygen(rot_steps=steps, conj=True)
    job = g.Job(ctx, W["n"], W["d"], W["k"], layout="factored")
    job.set_nonce(5)
    ks0 = ctx.ks_histogram().copy()
    job.encrypt_inputs(data.X, A, data.y)
    if snps_first:
        job.encrypt_snps(data.S)
        job.fit(1)
        job.snp_stats(None)
    else:
        job.fit(1)
        job.snp_stats(data.S)
    want_h, _, _ = job_ks_histogram(W, 1, factored=True)
    assert np.array_equal(ctx.ks_histogram() - ks0, want_h)
    c = _oracle_job(W, lay, steps, data, A, factored=True, nonce=5)
    for which, ref in ((7, c.beta), (9, c.z), (6, c.zp), (10, c.w_m), (4, c.DupW),
                       (5, c.DupWZ)):
        assert np.array_equal(job.ct(which).export(), ref.c), which
    for cc in range(W["d"]):
        assert np.array_equal(job.ct(11, cc).export(), c.DupX[cc].c), cc
        assert np.array_equal(job.ct(12, cc).export(), c.DupB[cc].c), cc
    for bi in (0, lay.batches - 1):
        want = c.snp_batch_factored(c.encrypt_snp_batch_ccp(data.S, bi))
        for which in range(3):
            assert np.array_equal(job.ct(which, bi).export(), want[which].c), (bi, which)
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    check_accuracy(num, den, ref, W["k"])


def test_mccp_job_bit_exact_with_64_pair_tensor_sums(g):
    """The paper's own M-CCP layout at N = 2^12 with 64 samples: each batch's
    S' is a tensor sum of 64 pairs (two 32-pair partial reductions) over all
    four batches of one set, the last ragged (8 SNPs); Dup(M_j) spans both
    CCP ciphertexts of M.  M, Dup(M_j), beta, z' and the first and last
    batch outputs equal the oracle's circuit."""
    W = dict(logN=12, L=21, q0_bits=60, scale_bits=40, K=7, sp_bits=60, dnum=3, seed=13,
             n=64, d=3, k=200)
    data = make_gwas(W["n"], W["d"], W["k"], seed=7)
    A = gwas_fp64.xtx_inv(data.X)
    lay = Layout(W["logN"], W["n"], W["d"], W["k"])
    assert lay.nb == 64 and lay.B == 32 and lay.H == 2 and lay.batches == 4
    steps = rotation_steps(lay)
    ctx = g.Context(W["logN"], W["L"], K=W["K"], dnum=W["dnum"], seed=W["seed"])
    ctx.keygen(rot_steps=steps, conj=True)
    job = g.Job(ctx, W["n"], W["d"], W["k"], layout="mccp")
    ks0 = ctx.ks_histogram().copy()
    job.encrypt_inputs(data.X, A, data.y)
    job.fit(1)
    job.snp_stats(data.S)
    want_h, _, _ = job_ks_histogram(W, 1)
    assert np.array_equal(ctx.ks_histogram() - ks0, want_h)
    c = _oracle_job(W, lay, steps, data, A, factored=False)
    assert np.array_equal(job.ct(7).export(), c.beta.c)
    assert np.array_equal(job.ct(6).export(), c.zp.c)
    for h in range(lay.H):
        assert np.array_equal(job.ct(8, h).export(), c.Mct[h].c), h
    for jj in (0, 31, 32, 63):
        assert np.array_equal(job.ct(3, jj).export(), c.DupM[jj].c), jj
    for bi in (0, lay.batches - 1):
        want = c.snp_batch(c.encrypt_snp_batch(data.S, bi))
        for which in range(3):
            assert np.array_equal(job.ct(which, bi).export(), want[which].c), (bi, which)
    num, den = job.decrypt_results()
    ref = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1, A=A)
    check_accuracy(num, den, ref, W["k"])


@pytest.mark.parametrize("layout", ["factored", "mccp"])
def test_split_encryption_phase_equals_fused_path(g, layout):
    """The encryption phase as its own calls (covariates, phenotype, SNP
    batches in two streamed ranges) and the loop over the pre-encrypted
    batches give the fused path's ciphertexts bit for bit; the second job
    also moves to another CUDA stream midway (gwhe_ctx_set_stream)."""
    import torch
    logN, L, K, dnum, seed = 10, 21, 7, 3, 15
    n, d, k = 16, 3, 100  # two batches of 64 SNPs, the second ragged
    data = make_gwas(n, d, k, seed=9)
    A = gwas_fp64.xtx_inv(data.X)
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=seed)
    fused = g.Job(ctx, n, d, k, layout=layout)
    ctx.keygen(rot_steps=fused.rotation_steps(), conj=True)
    fused.encrypt_inputs(data.X, A, data.y)
    fused.fit(1)
    fused.snp_stats(data.S)
    split = g.Job(ctx, n, d, k, layout=layout)
    split.encrypt_covariates(data.X, A)
    split.encrypt_phenotype(data.y)
    with pytest.raises(g.GwheError) as e:
        split.snp_stats(None)  # no covariate phase, no encrypted batches
    assert e.value.code == -1
    split.fit(1)
    split.encrypt_snps(data.S, 0, 1)
    side = torch.cuda.Stream()
    ctx.set_stream(side)
    split.encrypt_snps(data.S, 1, 2)
    split.snp_stats(None)
    ctx.set_stream(None)
    with pytest.raises(g.GwheError):
        split.snp_stats(None)  # consumed: freed after the loop used them
    for which in (7, 6, 4, 5):
        assert np.array_equal(split.ct(which).export(), fused.ct(which).export()), which
    for bi in range(2):
        for which in range(3):
            assert np.array_equal(split.ct(which, bi).export(), fused.ct(which, bi).export()), \
                (bi, which)
    a, b = fused.decrypt_results(), split.decrypt_results()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
