"""Pins of O2 (FP64 approximated GWAS), O3 (exact references) and of the
oracle's encrypted circuit, against closed forms, invariants, the values the
paper prints, and brute force on tiny inputs."""
import json
import math
import os

import numpy as np
import pytest

from oracle import gwas_exact, gwas_fp64
from oracle.circuit import Circuit, Layout, rotation_steps
from oracle.ckks import OracleCKKS, galois_conj, galois_rot
from oracle.trace import job_ks_histogram
from paper_1902_04303_gb300.datagen import make_gwas

def _count_switches(o):
    """per-level key switches of the oracle evaluator o: one per switch, one
    per hoisted rotation group (shared ModUp and ModDown) and one per fused
    relinearisation-rescale"""
    hist = np.zeros(65, np.int64)
    real_ks, real_sum, real_rr = o.keyswitch, o.rotate_sum, o.relin_rescale

    def counting_ks(x, key_id):
        hist[x.shape[0]] += 1
        return real_ks(x, key_id)

    def counting_sum(a, rs):
        hist[a.level] += 1
        old = o.keyswitch
        o.keyswitch = real_ks
        try:
            return real_sum(a, rs)
        finally:
            o.keyswitch = old

    def counting_rr(t):
        hist[t.level] += 1
        return real_rr(t)

    o.keyswitch, o.rotate_sum, o.relin_rescale = counting_ks, counting_sum, counting_rr
    return hist


GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_sigma7_coefficients_and_values():
    g = GOLD["sigma7_coefficients"]
    assert gwas_fp64.SIGMA7_C0 == g["c0"]
    assert gwas_fp64.SIGMA7_C == (g["c1"], g["c3"], g["c5"], g["c7"])
    assert gwas_fp64.sigma7(0.0) == 0.5
    # at x = 8 the polynomial is the sum of its coefficients
    assert gwas_fp64.sigma7(8.0) == pytest.approx(0.5 - 1.73496 + 4.19407 - 5.43402 + 2.50739,
                                                  abs=1e-15)
    assert gwas_fp64.sigma7(2.0) == pytest.approx(0.1266391, abs=1e-6)
    # odd part: sigma7(x) + sigma7(-x) = 1
    x = np.linspace(-8, 8, 33)
    assert np.allclose(gwas_fp64.sigma7(x) + gwas_fp64.sigma7(-x), 1.0, atol=1e-15)
    # as printed it tracks the logistic function of -x on [-8, 8] (reading A-13)
    assert np.max(np.abs(gwas_fp64.sigma7(x) - gwas_exact.sigmoid(-x))) < 0.04


def test_inverse_slots_closed_form():
    g = GOLD["inverse_slots"]
    w = np.linspace(0.001, g["w_upper_bound"], 200)
    got = gwas_fp64.inverse_slots(w, guess=g["guess"], iters=g["iterations"])
    closed = (1.0 - (1.0 - 3.0 * w) ** 8) / w
    assert np.allclose(got, closed, rtol=1e-12)
    assert gwas_fp64.inverse_slots(np.array([0.25]))[0] == 3.99993896484375
    assert gwas_fp64.inverse_slots(np.array([0.01]))[0] == pytest.approx(21.6257, abs=1e-4)


def test_batch_geometry_matches_paper():
    g = GOLD["batch_geometry"]
    lay = Layout(g["logN"], g["n"], 5, g["k"])
    assert lay.tau == g["tau"] and lay.batches == g["batches"]
    for n, logN in GOLD["subject_limit"]["cases"]:
        nb = 1 << math.ceil(math.log2(n))
        # the paper's packed layout needs nb^2 slots, i.e. N >= 2 nb^2
        assert (1 << logN) >= 2 * nb * nb
        assert (1 << (logN - 1)) < 2 * nb * nb


def test_pow2_rotation_count():
    for r, cnt in GOLD["pow2_rotations"]["examples"]:
        assert bin(r).count("1") == cnt


@pytest.fixture(scope="module")
def data():
    d = make_gwas(64, 4, 48, seed=21)
    return d


def test_M_projection_invariants(data):
    res = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=1)
    M = res["M"]
    assert np.max(np.abs(M @ M - M)) < 1e-12
    assert np.max(np.abs(M @ data.X)) < 1e-12
    assert np.max(np.abs(M - M.T)) < 1e-12


def test_complex_route_equals_direct(data):
    res = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa=2)
    direct = (res["w"][:, None] * res["Sp"] ** 2).sum(axis=0)
    assert np.max(np.abs(res["den"] - direct) / direct) < 1e-12
    # odd k: the padded column is ignored
    den = gwas_fp64.complex_route_den(res["Sp"][:, :7], res["w"])
    assert np.allclose(den, direct[:7], rtol=1e-12)


def test_sign_slips_cancel(data):
    """reading A-13: literal beta = -corrected beta exactly; p, w, z', b' identical."""
    for kappa in (1, 2, 3):
        lit = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa)
        cor = gwas_fp64.semi_parallel_fp64(data.X, data.y, data.S, kappa, corrected=True)
        assert np.array_equal(lit["beta"], -cor["beta"])
        assert np.array_equal(lit["p"], cor["p"])
        assert np.allclose(lit["zp"], cor["zp"], atol=1e-11)
        assert np.allclose(lit["b"], cor["b"], atol=1e-11)


def test_bohning_fixed_point_is_mle(data):
    """with the exact logistic function the Bohning iteration converges to the MLE."""
    A = gwas_fp64.xtx_inv(data.X)
    # corrected=True evaluates f(-X beta); f(-x) = logistic(x) here
    beta, _ = gwas_fp64.hom_logreg(data.X, data.y, A, kappa=400, corrected=True,
                                   sigmoid=lambda x: gwas_exact.sigmoid(-x))
    mle = gwas_exact.newton_logreg(data.X, data.y)
    assert np.max(np.abs(beta - mle)) < 1e-8


def test_o2_tracks_exact_references(data):
    """reported, loose: the approximated GWAS follows the exact semi-parallel
    method and the per-SNP brute force (the paper's accuracy comparison)."""
    X, y, S = data.X, data.y, data.S[:, :24]
    o2 = gwas_fp64.semi_parallel_fp64(X, y, S, kappa=3)
    sp = gwas_exact.semi_parallel_exact(X, y, S)
    bf = gwas_exact.per_snp_logreg(X, y, S)
    assert np.corrcoef(o2["b"], sp["b"])[0, 1] > 0.95
    assert np.corrcoef(sp["b"], bf["b"])[0, 1] > 0.95
    assert np.max(np.abs(sp["b"] - bf["b"])) < 0.5


def test_encrypted_circuit_matches_o2():
    """the oracle's own encrypted circuit (Alg. 9-11 over O1) decrypts to O2
    within the acceptance tolerances |d b'| <= 5e-3, |d(-log10 p)| <= 0.05."""
    logN, n, d, k = 10, 16, 3, 40
    dat = make_gwas(n, d, k, seed=5)
    A = gwas_fp64.xtx_inv(dat.X)
    o = OracleCKKS(logN=logN, L=21, K=7, dnum=3, seed=11)
    lay = Layout(logN, n, d, k)
    o.keygen(galois=[galois_rot(logN, r) for r in rotation_steps(lay)] + [galois_conj(logN)])
    hist = _count_switches(o)
    c = Circuit(o, lay)
    c.encrypt_inputs(dat.X, A, dat.y)
    c.fit(kappa=1)
    nums, dens = [], []
    for i in range(lay.batches):
        num, de, do = c.snp_batch(c.encrypt_snp_batch(dat.S, i))
        a, b = c.extract(num, de, do, i)
        nums.append(a)
        dens.append(b)
    num = np.concatenate(nums)
    den = np.concatenate(dens)
    # the level tracer issues the same key switches at the same levels
    W = dict(logN=logN, L=21, q0_bits=60, scale_bits=40, K=7, sp_bits=60, dnum=3, n=n, d=d, k=k)
    want, _, _ = job_ks_histogram(W, 1)
    assert np.array_equal(hist, want)
    ref = gwas_fp64.semi_parallel_fp64(dat.X, dat.y, dat.S, kappa=1, A=A)
    ok = np.abs(ref["den"]) > 1e-6  # monomorphic SNPs have den = 0 (degenerate)
    assert np.max(np.abs(den[~ok])) < 1e-4
    b = num[ok] / den[ok]
    assert np.max(np.abs(b - ref["b"][ok])) < 5e-3
    dl = np.abs(gwas_fp64.neglog10p(b, 1 / den[ok]) - gwas_fp64.neglog10p(ref["b"][ok],
                                                                          ref["err"][ok]))
    assert np.max(dl) < 0.05


@pytest.mark.parametrize("n", [16, 64, 245])
def test_batch_key_switch_count_closed_form(n):
    """One SNP batch (Alg. 11 loop body) switches keys 6 + 3 ceil(log2(nb)/3)
    times: relinearisations of S', Dup(w z') S', Dup(w) S', WSS, WSC (5), the
    conjugation (1), and three column sums (Alg. 4) of log2(nb) rotation
    steps, evaluated three steps per hoisted switch."""
    W = dict(logN=16, L=24, q0_bits=60, scale_bits=45, K=8, sp_bits=60, dnum=3, n=n, d=5,
             k=10643)
    _, _, batch = job_ks_histogram(W, 1)
    nb = 1 << math.ceil(math.log2(n))
    assert batch.sum() == 6 + 3 * math.ceil(math.log2(nb) / 3)
    # every batch switch happens at or below the batch entry level
    assert batch[5:].sum() == 0


@pytest.mark.parametrize("n,d", [(16, 3), (245, 5), (1000, 6)])
def test_factored_batch_key_switch_count_closed_form(n, d):
    """The factored layout adds, per batch, d products, d column sums and d
    in-block broadcasts of log2(nb) rotation steps each (three steps per
    hoisted switch, h = ceil(log2(nb)/3) switches), and one relinearised tensor sum:
    d + 2 d h + 1 switches, then the body shared with the M-CCP layout
    (5 + 3 h: four relinearisations, the conjugation, three column sums); per
    level d at 6 limbs, d h at 5, d h + 1 at 4."""
    W = dict(logN=16, L=24, q0_bits=60, scale_bits=45, K=8, sp_bits=60, dnum=3, n=n, d=d,
             k=50000)
    _, fit_f, batch_f = job_ks_histogram(W, 1, factored=True)
    h = math.ceil(math.ceil(math.log2(n)) / 3)
    assert batch_f.sum() == (d + 2 * d * h + 1) + (5 + 3 * h)
    assert batch_f[6] == d and batch_f[5] == d * h and batch_f[4] == d * h + 1
    assert batch_f[7:].sum() == 0  # the CCP batch enters at 6 limbs


def test_sprime_forms_agree(data):
    """eq. Sprime: M S = S - X (X^T X)^-1 X^T S, and the packed complex batch
    of the factored layout carries two SNP columns per slot unchanged."""
    X, y, S = data.X, data.y, data.S
    A = gwas_fp64.xtx_inv(X)
    Mm = np.eye(X.shape[0]) - X @ A @ X.T
    assert np.max(np.abs(Mm @ S - (S - (X @ A) @ (X.T @ S)))) < 1e-10
    Sc = S[:, 0::2][:, : S.shape[1] // 2] + 1j * S[:, 1::2][:, : S.shape[1] // 2]
    Pc = Mm @ Sc
    assert np.allclose(Pc.real, Mm @ S[:, 0::2][:, : S.shape[1] // 2])
    assert np.allclose(Pc.imag, Mm @ S[:, 1::2][:, : S.shape[1] // 2])


def test_encrypted_factored_circuit_matches_o2():
    """the factored layout (second form of eq. Sprime, S in CCP) over O1
    decrypts to O2 within the acceptance tolerances, with the key switches
    the level trace predicts."""
    logN, n, d, k = 10, 16, 3, 100
    dat = make_gwas(n, d, k, seed=6)
    A = gwas_fp64.xtx_inv(dat.X)
    o = OracleCKKS(logN=logN, L=21, K=7, dnum=3, seed=12)
    lay = Layout(logN, n, d, k)
    o.keygen(galois=[galois_rot(logN, r) for r in rotation_steps(lay, factored=True)]
             + [galois_conj(logN)])
    hist = _count_switches(o)
    c = Circuit(o, lay, factored=True)
    c.encrypt_inputs(dat.X, A, dat.y)
    c.fit(kappa=1)
    assert not c.XtREP and not c.DupM
    nums, dens = [], []
    for i in range(lay.batches):
        Sct = c.encrypt_snp_batch_ccp(dat.S, i)
        num, de, do = c.snp_batch_factored(Sct)
        a, b = c.extract(num, de, do, i)
        nums.append(a)
        dens.append(b)
    num = np.concatenate(nums)
    den = np.concatenate(dens)
    W = dict(logN=logN, L=21, q0_bits=60, scale_bits=40, K=7, sp_bits=60, dnum=3, n=n, d=d, k=k)
    want, _, _ = job_ks_histogram(W, 1, factored=True)
    assert np.array_equal(hist, want)
    ref = gwas_fp64.semi_parallel_fp64(dat.X, dat.y, dat.S, kappa=1, A=A)
    ok = np.abs(ref["den"]) > 1e-6
    assert np.max(np.abs(den[~ok]), initial=0.0) < 1e-4
    b = num[ok] / den[ok]
    assert np.max(np.abs(b - ref["b"][ok])) < 5e-3
    dl = np.abs(gwas_fp64.neglog10p(b, 1 / den[ok]) - gwas_fp64.neglog10p(ref["b"][ok],
                                                                          ref["err"][ok]))
    assert np.max(dl) < 0.05


@pytest.mark.parametrize("m", [1, 3, 5, 8, 9])
def test_shared_replicate_equals_alg1(m):
    """Replicate (Alg. 1) of entries 0..m-1 through one shared ladder: every
    slot of result c decrypts to v_c (Alg. 1's definition), as Alg. 1's own
    mask-then-ladder gives, at the same level, with fewer hoisted switches:
    ceil(log2(M/P)/3) + m ceil(log2(P)/3) against m ceil(log2(M)/3).  A vector
    that is not zero beyond its entries breaks it (the precondition)."""
    from oracle.circuit import replicate_period
    logN = 10
    o = OracleCKKS(logN=logN, L=4, K=2, dnum=2, seed=21)
    M = 1 << (logN - 1)
    lay = Layout(logN, 16, m, 32)
    o.keygen(galois=[galois_rot(logN, r) for r in rotation_steps(lay)])
    c = Circuit(o, lay)
    rng = np.random.default_rng(m)
    v = rng.uniform(-1, 1, m)
    ct = c.encrypt_vector(v, 0x77)
    hist = _count_switches(o)
    reps = c.replicate_all(ct, m)
    shared = int(hist.sum())
    P = replicate_period(m, M)
    assert P >= m and P & (P - 1) == 0 and math.log2(P) % 3 == 0
    assert shared == math.ceil(math.log2(M // P) / 3) + m * math.ceil(math.log2(P) / 3)
    hist[:] = 0
    alg1 = [c.replicate(ct, j) for j in range(m)]
    assert int(hist.sum()) == m * math.ceil((logN - 1) / 3)
    for j in range(m):
        assert reps[j].level == alg1[j].level == ct.level - 1
        got = o.decrypt_decode(reps[j])
        ref = o.decrypt_decode(alg1[j])
        assert np.max(np.abs(got - v[j])) < 1e-5
        assert np.max(np.abs(got - ref)) < 1e-5
    # planted violation: a nonzero slot beyond the entries lands in its class
    bad = np.zeros(P + 1)
    bad[:m] = v
    bad[P] = 0.5
    reps_bad = c.replicate_all(c.encrypt_vector(bad, 0x78), m)
    assert np.max(np.abs(o.decrypt_decode(reps_bad[0]) - (v[0] + 0.5))) < 1e-5


def test_composed_rp_cp_matvec_equals_alg6_then_alg2():
    """A (X^T v) through Alg. 2 over Alg. 6's DotProds (the masks e_c and the
    replicates cancel) decrypts to the plaintext product and to Alg. 6 then
    Alg. 2, at the same level, without the replicate ladders: m (1 + h) + 1
    key switches (h = ceil(log2(M)/3) hoisted groups per DotProd ladder)
    against m (1 + h) + (ceil(log2(M/8)/3) + m) + 1."""
    logN, n, d = 10, 16, 3
    dat = make_gwas(n, d, 32, seed=31)
    A = gwas_fp64.xtx_inv(dat.X)
    o = OracleCKKS(logN=logN, L=8, K=3, dnum=2, seed=33)
    lay = Layout(logN, n, d, 32)
    o.keygen(galois=[galois_rot(logN, r) for r in rotation_steps(lay)])
    c = Circuit(o, lay)
    c.encrypt_inputs(dat.X, A, dat.y)
    rng = np.random.default_rng(5)
    v = rng.uniform(-1, 1, n)
    vct = c.encrypt_vector(v, 0x99)
    want = A @ (dat.X.T @ v)
    hist = _count_switches(o)
    fused = c.cp_rp_matvec(c.A, c.X, vct, d)
    n_fused = int(hist.sum())
    hist[:] = 0
    two = c.cp_matvec(c.A, c.rp_matvec(c.X, vct, d), d)
    n_two = int(hist.sum())
    assert fused.level == two.level == vct.level - 4
    got_f = o.decrypt_decode(fused).real[:d]
    got_t = o.decrypt_decode(two).real[:d]
    assert np.max(np.abs(got_f - want)) < 1e-4 and np.max(np.abs(got_t - want)) < 1e-4
    assert np.max(np.abs(got_f - got_t)) < 1e-4
    M = 1 << (logN - 1)
    per_ladder = math.ceil((logN - 1) / 3)
    assert n_fused == d * (1 + per_ladder) + 1
    assert n_two == d * (1 + per_ladder) + (math.ceil(math.log2(M // 8) / 3) + d) + 1
    # a planted error: a wrong column of A shows up in the result
    bad = c.cp_rp_matvec(c.A[::-1], c.X, vct, d)
    assert np.max(np.abs(o.decrypt_decode(bad).real[:d] - want)) > 1e-2


def test_encrypted_circuit_kappa3_matches_o2():
    """kappa = 3 Bohning iterations (Alg. 9; the paper's HEAAN setting) over
    O1 with 40 limbs (factored layout, N = 2^10): the decrypted beta equals the
    FP64 circuit's beta, and b' and -log10 p stay within the acceptance
    tolerances, with the key switches the level trace predicts."""
    logN, L, K, dnum = 10, 40, 12, 3
    n, d, k = 16, 3, 64
    dat = make_gwas(n, d, k, seed=15)
    A = gwas_fp64.xtx_inv(dat.X)
    lay = Layout(logN, n, d, k)
    o = OracleCKKS(logN=logN, L=L, q0_bits=60, scale_bits=45, K=K, dnum=dnum, seed=14)
    o.keygen(galois=[galois_rot(logN, r) for r in rotation_steps(lay, factored=True)]
             + [galois_conj(logN)])
    hist = _count_switches(o)
    c = Circuit(o, lay, factored=True)
    c.encrypt_inputs(dat.X, A, dat.y)
    c.fit(kappa=3)
    num, de, do = c.snp_batch_factored(c.encrypt_snp_batch_ccp(dat.S, 0))
    W = dict(logN=logN, L=L, q0_bits=60, scale_bits=45, K=K, sp_bits=60, dnum=dnum, n=n, d=d, k=k)
    want, _, _ = job_ks_histogram(W, 3, factored=True)
    assert np.array_equal(hist, want)
    ref = gwas_fp64.semi_parallel_fp64(dat.X, dat.y, dat.S, kappa=3, A=A)
    beta = o.decrypt_decode(c.beta).real[:d]
    assert np.max(np.abs(beta - ref["beta"])) < 1e-3
    a, b = c.extract(num, de, do, 0)
    ok = np.abs(ref["den"]) > 1e-6
    assert np.max(np.abs(a[ok] / b[ok] - ref["b"][ok])) < 5e-3
    dl = np.abs(gwas_fp64.neglog10p(a[ok] / b[ok], 1 / b[ok])
                - gwas_fp64.neglog10p(ref["b"][ok], ref["err"][ok]))
    assert np.max(dl) < 0.05
