"""Pins of the O1 oracle (textbook RNS-CKKS) against things other than itself:
library routines (sympy primality, the `cryptography` ChaCha20), schoolbook
negacyclic convolution, Python big-integer CRT, the definition of the
canonical embedding, and decryption invariants with noise bounds."""
import math

import numpy as np
import pytest

from oracle import ckks
from oracle.ckks import OracleCKKS, decode_naive, encode_naive_real, galois_conj, galois_rot

L = ckks.lib()


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------ primes
def test_is_prime_matches_sympy():
    sympy = pytest.importorskip("sympy")
    rng = _rng(1)
    vals = [int(v) | 1 for v in rng.integers(3, 2 ** 62, size=300, dtype=np.uint64)]
    vals += [2, 3, 4, 561, 1105, 2 ** 61 - 1, (2 ** 61 - 1) * 3, 3215031751, 341550071728321]
    for v in vals:
        assert bool(L.or_is_prime(v)) == bool(sympy.isprime(v)), v


@pytest.mark.parametrize("logN,Lq,K", [(4, 4, 2), (13, 4, 1), (16, 24, 8)])
def test_prime_generation_spec(logN, Lq, K):
    sympy = pytest.importorskip("sympy")
    q = np.zeros(Lq, np.uint64)
    p = np.zeros(K, np.uint64)
    assert L.or_gen_primes(logN, Lq, 60, 40, K, 60, q, p) == 0
    step = 2 << logN
    allp = [int(x) for x in q] + [int(x) for x in p]
    assert len(set(allp)) == len(allp)
    for x in allp:
        assert sympy.isprime(x) and x % step == 1
    # base prime: the largest candidate below 2^60
    assert int(q[0]) < 2 ** 60
    c = int(q[0]) + step
    while c < 2 ** 60:
        assert not sympy.isprime(c)
        c += step
    # scale primes alternate below / above 2^40, each the nearest unused one
    below = [int(x) for x in q[1::2]]
    above = [int(x) for x in q[2::2]]
    assert all(x < 2 ** 40 for x in below) and all(x > 2 ** 40 for x in above)
    assert below == sorted(below, reverse=True) and above == sorted(above)
    if below:
        c = below[0] + step
        while c < 2 ** 40:
            assert not sympy.isprime(c)
            c += step
    if above:
        c = 2 ** 40 + 1
        while c < above[0]:
            assert not sympy.isprime(c)
            c += step
    # special primes: descending below 2^60, the next ones after q0
    ps = [int(x) for x in p]
    assert ps == sorted(ps, reverse=True) and ps[0] < int(q[0])
    c = ps[0] + step
    while c < int(q[0]):
        assert not sympy.isprime(c)
        c += step


@pytest.mark.parametrize("logN", [4, 10, 16])
def test_primitive_root(logN):
    q = np.zeros(2, np.uint64)
    p = np.zeros(1, np.uint64)
    L.or_gen_primes(logN, 2, 60, 40, 1, 60, q, p)
    for m in [int(q[0]), int(q[1]), int(p[0])]:
        psi = L.or_primitive_root_2n(m, logN)
        N = 1 << logN
        assert pow(psi, N, m) == m - 1
        assert pow(psi, 2 * N, m) == 1


# ------------------------------------------------------------------ ring product
@pytest.mark.parametrize("logN", [1, 2, 3, 5, 8])
def test_polymul_equals_schoolbook(logN):
    N = 1 << logN
    q = np.zeros(1, np.uint64)
    p = np.zeros(1, np.uint64)
    L.or_gen_primes(max(logN, 2), 1, 60, 40, 1, 60, q, p)
    m = int(q[0])
    psi = L.or_primitive_root_2n(m, logN)
    rng = _rng(logN)
    a = rng.integers(0, m, size=N, dtype=np.uint64)
    b = rng.integers(0, m, size=N, dtype=np.uint64)
    o1 = np.zeros(N, np.uint64)
    o2 = np.zeros(N, np.uint64)
    L.or_polymul(a, b, o1, logN, m, psi)
    L.or_polymul_schoolbook(a, b, o2, logN, m)
    assert np.array_equal(o1, o2)
    # independent big-integer schoolbook (definition of X^N = -1)
    ai = [int(x) for x in a]
    bi = [int(x) for x in b]
    ref = [0] * N
    for i in range(N):
        for j in range(N):
            s = ai[i] * bi[j]
            if i + j < N:
                ref[i + j] += s
            else:
                ref[i + j - N] -= s
    assert [r % m for r in ref] == [int(x) for x in o1]


# ------------------------------------------------------------------ ChaCha20
def test_chacha20_matches_library():
    crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    from cryptography.hazmat.primitives.ciphers import Cipher, algorithms
    rng = _rng(3)
    for _ in range(8):
        key = rng.integers(0, 2 ** 32, size=8, dtype=np.uint64).astype(np.uint32)
        nonce = rng.integers(0, 2 ** 32, size=3, dtype=np.uint64).astype(np.uint32)
        counter = int(rng.integers(0, 2 ** 31))
        ours = ckks.chacha20_block(key, counter, nonce)
        iv = np.uint32(counter).tobytes() + nonce.tobytes()
        enc = Cipher(algorithms.ChaCha20(key.tobytes(), iv), mode=None).encryptor()
        ks = np.frombuffer(enc.update(bytes(64)), dtype=np.uint32)
        assert np.array_equal(ours, ks)


def test_samplers_distribution():
    logN = 14
    N = 1 << logN
    t = np.zeros(N, np.int64)
    L.or_sample_ternary(42, 1, logN, t)
    assert set(np.unique(t)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(t == v) - 1 / 3) < 0.02
    e = np.zeros(N, np.int64)
    L.or_sample_cbd(42, 3, logN, e)
    assert e.min() >= -21 and e.max() <= 21
    assert abs(e.mean()) < 0.15 and abs(e.var() - 10.5) < 0.6
    u = np.zeros(N, np.uint64)
    m = 1099511592961
    L.or_sample_uniform(42, 2, 5, m, logN, u)
    assert int(u.max()) < m
    assert abs(float(np.mean(u.astype(np.float64))) / m - 0.5) < 0.02
    # distinct objects / tags give distinct streams
    u2 = np.zeros(N, np.uint64)
    L.or_sample_uniform(42, 2, 6, m, logN, u2)
    assert not np.array_equal(u, u2)


# ------------------------------------------------------------------ encoding
@pytest.mark.parametrize("logN", [3, 5, 8, 10])
def test_encode_matches_definition(logN):
    M = 1 << (logN - 1)
    rng = _rng(logN + 100)
    z = rng.normal(size=M) + 1j * rng.normal(size=M)
    delta = 2.0 ** 40
    o = OracleCKKS(logN=max(logN, 4), L=2, K=1) if logN >= 4 else None
    m = np.zeros(1 << logN, np.int64)
    buf = np.ascontiguousarray(np.stack([z.real, z.imag], 1).reshape(-1))
    L.or_encode(logN, buf, delta, m)
    exact = encode_naive_real(z, logN, delta)
    # rounding of a value within the fixed-point procedure's error bound of the
    # definition: 0.5 plus scale * 2^-F, F = 61 - log2(M) - e fractional bits
    e = int(np.ceil(np.log2(max(np.max(np.abs(z.real)), np.max(np.abs(z.imag)), 1.0))))
    F = 61 - (logN - 1) - e
    assert np.max(np.abs(m - exact)) <= 0.5 + delta * 2.0 ** -F
    # decode by the definition recovers z within the rounding bound
    back = decode_naive(m, logN, delta)
    bound = (1 << logN) * 0.5 / delta
    assert np.max(np.abs(back - z)) <= bound
    if o is not None and o.logN == logN:
        assert np.max(np.abs(o.decode(o.to_rns(m, 2), delta) - z)) <= bound


def test_decode_fft_matches_definition():
    o = OracleCKKS(logN=9, L=2, K=1)
    rng = _rng(7)
    m = rng.integers(-2 ** 45, 2 ** 45, size=o.N)
    res = o.to_rns(m, 2)
    a = o.decode(res, 2.0 ** 40)
    b = decode_naive(m, 9, 2.0 ** 40)
    assert np.max(np.abs(a - b)) < 1e-6


# ------------------------------------------------------------------ scheme
@pytest.fixture(scope="module")
def small():
    o = OracleCKKS(logN=9, L=5, K=2, dnum=3, seed=5)
    o.keygen(galois=[galois_rot(9, 1), galois_rot(9, 8), galois_rot(9, -1), galois_conj(9)])
    return o


def test_encrypt_decrypt_roundtrip(small):
    o = small
    rng = _rng(8)
    z = rng.normal(size=o.M) + 1j * rng.normal(size=o.M)
    ct = o.encrypt(o.encode(z, o.delta, o.L), 1, o.delta)
    assert np.max(np.abs(o.decrypt_decode(ct) - z)) < 1e-6
    # decrypting the fresh ciphertext leaves m + (v e + e0 + e1 s): small noise
    m = o.encode_int(z, o.delta)
    diff = np.array(o.crt_centered(o.decrypt(ct)), dtype=object) - m.astype(object)
    assert max(abs(int(v)) for v in diff) < 2 ** 20
    # same id -> same ciphertext; different id -> different randomness
    ct2 = o.encrypt(o.encode(z, o.delta, o.L), 1, o.delta)
    ct3 = o.encrypt(o.encode(z, o.delta, o.L), 2, o.delta)
    assert np.array_equal(ct.c, ct2.c) and not np.array_equal(ct.c, ct3.c)


def test_homomorphic_identities(small):
    o = small
    rng = _rng(9)
    a = rng.normal(size=o.M) + 1j * rng.normal(size=o.M)
    b = rng.normal(size=o.M) + 1j * rng.normal(size=o.M)
    ca = o.encrypt(o.encode(a, o.delta, o.L), 1, o.delta)
    cb = o.encrypt(o.encode(b, o.delta, o.L), 2, o.delta)
    dd = o.decrypt_decode
    assert np.max(np.abs(dd(o.add(ca, cb)) - (a + b))) < 1e-6
    assert np.max(np.abs(dd(o.sub(ca, cb)) - (a - b))) < 1e-6
    assert np.max(np.abs(dd(o.mult(ca, cb)) - a * b)) < 1e-5
    assert np.max(np.abs(dd(o.rotate(ca, 1)) - np.roll(a, -1))) < 1e-6
    assert np.max(np.abs(dd(o.rotate(ca, 8)) - np.roll(a, -8))) < 1e-6
    assert np.max(np.abs(dd(o.rotate(ca, -1)) - np.roll(a, 1))) < 1e-6
    assert np.max(np.abs(dd(o.conj(ca)) - np.conj(a))) < 1e-6
    assert np.max(np.abs(dd(o.mul_int(ca, 3)) - 3 * a)) < 1e-6
    assert np.max(np.abs(dd(o.mul_const(ca, 0.125)) - 0.125 * a)) < 1e-6
    assert np.max(np.abs(dd(o.add_const(ca, 0.5)) - (a + 0.5))) < 1e-6
    mask = (np.arange(o.M) % 3 == 0).astype(float)
    assert np.max(np.abs(dd(o.mul_mask(ca, mask)) - a * mask)) < 1e-6


def test_rescale_equals_exact_division():
    """rescale = floor((C + floor(q_l/2)) / q_l) of the CRT integer C."""
    o = OracleCKKS(logN=4, L=4, K=1)
    rng = _rng(10)
    l = 4
    c = np.stack([rng.integers(0, o.q[i], size=o.N, dtype=np.uint64) for i in range(l)])
    ct = ckks.Ct(c[None].copy(), 1.0)
    out = o.rescale(ct).c[0]
    Q = math.prod(o.q[:l])
    ql = o.q[l - 1]
    for kk in range(o.N):
        C = sum(int(c[i, kk]) * (Q // o.q[i]) * pow(Q // o.q[i], -1, o.q[i]) for i in range(l)) % Q
        want = (C + ql // 2) // ql
        for i in range(l - 1):
            assert int(out[i, kk]) == want % o.q[i]


def _noise_of(o, u, target_res, x):
    """centred CRT of (u0 + u1 s) - x * target over the q-limbs."""
    l = x.shape[0]
    dec = o.decrypt(ckks.Ct(u, 1.0))
    prod = np.zeros_like(dec)
    for i in range(l):
        L.or_polymul(np.ascontiguousarray(x[i]), np.ascontiguousarray(target_res[i]), prod[i],
                     o.logN, o.q[i], L.or_primitive_root_2n(o.q[i], o.logN))
    diff = np.zeros_like(dec)
    for i in range(l):
        q = np.uint64(o.q[i])
        diff[i] = np.where(dec[i] >= prod[i], dec[i] - prod[i], dec[i] + q - prod[i])
    return max(abs(v) for v in o.crt_centered(diff))


@pytest.mark.parametrize("l", [5, 4, 2])
def test_keyswitch_noise_invariant(small, l):
    """u0 + u1 s = x s^2 + e with |e| far below the modulus, at every level."""
    o = small
    rng = _rng(11 + l)
    x = np.stack([rng.integers(0, o.q[i], size=o.N, dtype=np.uint64) for i in range(l)])
    u = o.keyswitch(x, 0)
    s2 = np.zeros((o.L + o.K, o.N), np.uint64)
    L.or_sk_square(o._ctx, s2)
    noise = _noise_of(o, u, s2, x)
    assert noise < 2 ** 24, noise
    # a key for a different target does not switch x s^2
    g = galois_rot(9, 1)
    u_bad = o.keyswitch(x, g)
    assert _noise_of(o, u_bad, s2, x) > math.prod(o.q[:l]) // 2 ** 8


@pytest.fixture(scope="module")
def wide():
    # K = 6 special primes, digits of 3 limbs: the switches at low levels use
    # fewer special primes than those at the top
    o = OracleCKKS(logN=9, L=6, K=6, dnum=2, seed=6)
    o.keygen(galois=[galois_rot(9, 1)])
    return o


def test_special_prime_counts_shrink_with_the_level(wide):
    """each level uses between one and K special primes, never fewer at a
    higher level, and at least two counts occur in this context."""
    o = wide
    ks = o.ks_k[1:]
    assert all(1 <= k <= o.K for k in ks)
    assert all(a <= b for a, b in zip(ks, ks[1:]))
    assert len(set(ks)) >= 2, ks
    # one key family per count, each covering the levels that use it
    assert set(o.keys[0]) == set(ks)
    for k, fam in o.keys[0].items():
        lmax = o.key_lmax[k]
        assert fam.shape == (-(-lmax // o.alpha), 2, lmax + k, o.N)


@pytest.mark.parametrize("l", [1, 2, 3, 4, 6])
def test_keyswitch_noise_invariant_reduced_special_primes(wide, l):
    """u0 + u1 s = x s^2 + e with |e| < 2^24 whatever the number of special
    primes the level uses; a key for another target fails the identity."""
    o = wide
    rng = _rng(31 + l)
    x = np.stack([rng.integers(0, o.q[i], size=o.N, dtype=np.uint64) for i in range(l)])
    u = o.keyswitch(x, 0)
    s2 = np.zeros((o.L + o.K, o.N), np.uint64)
    L.or_sk_square(o._ctx, s2)
    assert _noise_of(o, u, s2, x) < 2 ** 24
    u_bad = o.keyswitch(x, galois_rot(9, 1))
    assert _noise_of(o, u_bad, s2, x) > math.prod(o.q[:l]) // 2 ** 8


@pytest.mark.parametrize("l,rs", [(5, [1, 2, 3]), (3, [8, 16, 24]), (2, [-1, -2, -3]), (4, [2]),
                                  (3, list(range(1, 16))), (2, [-r for r in range(1, 16)])])
def test_hoisted_rotation_sum_is_the_sum_of_automorphisms(small_rot, l, rs):
    """Dec(rotate_sum(a, rs)) = Dec(a) + sum_r sigma_r(Dec(a)) + e with |e|
    < 2^24: the automorphism is exact on the decryption (sigma(c0 + c1 s) =
    sigma(c0) + sigma(c1) sigma(s)), so the one shared ModUp / ModDown must
    reproduce it up to switch noise; and a rotation set whose key is replaced
    fails the identity."""
    o = small_rot
    rng = _rng(50 + l)
    a = ckks.Ct(np.stack([np.stack([rng.integers(0, o.q[i], size=o.N, dtype=np.uint64)
                                    for i in range(l)]) for _ in range(2)]), o.delta)
    dec = o.decrypt(a)
    want = dec.copy()
    for r in rs:
        g = galois_rot(o.logN, r)
        for i in range(l):
            t = np.zeros(o.N, np.uint64)
            L.or_automorphism(np.ascontiguousarray(dec[i]), t, o.logN, g, o.q[i])
            q = np.uint64(o.q[i])
            ssum = want[i] + t
            want[i] = np.where(ssum >= q, ssum - q, ssum)
    got = o.decrypt(o.rotate_sum(a, rs))
    diff = np.zeros_like(got)
    for i in range(l):
        q = np.uint64(o.q[i])
        diff[i] = np.where(got[i] >= want[i], got[i] - want[i], got[i] + q - want[i])
    assert max(abs(v) for v in o.crt_centered(diff)) < 2 ** 24
    # swap in a wrong key for the first rotation: the identity breaks
    g0 = galois_rot(o.logN, rs[0])
    saved = o.keys[g0]
    o.keys[g0] = o.keys[0]
    try:
        bad = o.decrypt(o.rotate_sum(a, rs))
    finally:
        o.keys[g0] = saved
    for i in range(l):
        q = np.uint64(o.q[i])
        diff[i] = np.where(bad[i] >= want[i], bad[i] - want[i], bad[i] + q - want[i])
    assert max(abs(v) for v in o.crt_centered(diff)) > math.prod(o.q[:l]) // 2 ** 8


@pytest.fixture(scope="module")
def small_rot():
    o = OracleCKKS(logN=9, L=5, K=4, dnum=2, seed=7)
    # the rotations of two- and four-step hoisted ladder groups
    o.keygen(galois=[galois_rot(9, r) for r in sorted(set(range(1, 16)) | {16, 24}
                                                         | {-r for r in range(1, 16)})])
    return o


def _centred_crt(o, res, l):
    return np.array(o.crt_centered(res[:l]), dtype=object)


@pytest.mark.parametrize("l", [5, 3, 2])
def test_fused_relin_rescale_is_the_rounded_division(wide, l):
    """Dec(relin_rescale(t)) = round(Dec3(t) / q_{l-1}) + e, |e| < 2^24, where
    Dec3(t) = d0 + d1 s + d2 s^2 exactly (big-integer CRT): the one fused
    division by P q_{l-1} must reproduce the exact rounded rescale of the
    tensor's decryption up to switch noise; a wrong key breaks it."""
    o = wide
    rng = _rng(70 + l)
    t = ckks.Ct(np.stack([np.stack([rng.integers(0, o.q[i], size=o.N, dtype=np.uint64)
                                    for i in range(l)]) for _ in range(3)]), o.delta)
    s1 = np.zeros((o.L + o.K, o.N), np.uint64)
    s2 = np.zeros((o.L + o.K, o.N), np.uint64)
    sk = o.secret_key()
    L.or_to_rns(o._ctx, sk, o.L, s1[:o.L])
    L.or_sk_square(o._ctx, s2)
    dec3 = np.zeros((l, o.N), np.uint64)
    for i in range(l):
        q = o.q[i]
        psi = L.or_primitive_root_2n(q, o.logN)
        p1 = np.zeros(o.N, np.uint64)
        p2 = np.zeros(o.N, np.uint64)
        L.or_polymul(np.ascontiguousarray(t.c[1, i]), np.ascontiguousarray(s1[i]), p1, o.logN, q, psi)
        L.or_polymul(np.ascontiguousarray(t.c[2, i]), np.ascontiguousarray(s2[i]), p2, o.logN, q, psi)
        dec3[i] = ((t.c[0, i].astype(object) + p1.astype(object) + p2.astype(object)) % q).astype(np.uint64)
    exact = _centred_crt(o, dec3, l)
    ql = o.q[l - 1]
    want = np.array([(int(v) + ql // 2) // ql if v >= 0 else -((-int(v) + ql // 2) // ql)
                     for v in exact], dtype=object)
    got = _centred_crt(o, o.decrypt(o.relin_rescale(t)), l - 1)
    assert max(abs(int(a) - int(b)) for a, b in zip(got, want)) < 2 ** 24
    saved = o.keys[0]
    o.keys[0] = o.keys[galois_rot(9, 1)]
    try:
        bad = _centred_crt(o, o.decrypt(o.relin_rescale(t)), l - 1)
    finally:
        o.keys[0] = saved
    assert max(abs(int(a) - int(b)) for a, b in zip(bad, want)) > math.prod(o.q[:l - 1]) // 2 ** 8


def test_automorphism_rotates_slots():
    o = OracleCKKS(logN=8, L=2, K=1)
    rng = _rng(12)
    z = rng.normal(size=o.M) + 1j * rng.normal(size=o.M)
    m = o.encode_int(z, o.delta)
    res = o.to_rns(m, 2)
    for r in (1, 3, -2):
        ct = ckks.Ct(np.stack([res, np.zeros_like(res)]), o.delta)
        rot = o.automorphism(ct, galois_rot(8, r))
        assert np.max(np.abs(o.decode(rot.c[0], o.delta) - np.roll(z, -r))) < 1e-7
    ct = ckks.Ct(np.stack([res, np.zeros_like(res)]), o.delta)
    cj = o.automorphism(ct, galois_conj(8))
    assert np.max(np.abs(o.decode(cj.c[0], o.delta) - np.conj(z))) < 1e-7


# ------------------------------------------------- evaluation at a 2N-th root
def _root_2n(q, N, seed):
    """an element of multiplicative order 2N mod the prime q (2N | q - 1),
    found from random bases: h = b^((q-1)/2N) has order 2N iff h^N = -1"""
    import random
    rng = random.Random(seed)
    while True:
        h = pow(rng.randrange(2, q - 1), (q - 1) // (2 * N), q)
        if pow(h, N, q) == q - 1:
            return h


def _eval(poly, x, q):
    """poly(x) mod q by Horner's rule on Python integers"""
    acc = 0
    for c in reversed([int(v) for v in poly]):
        acc = (acc * x + c) % q
    return acc


def test_ring_maps_by_evaluation_at_a_root(small):
    """Evaluation at x with x^N = -1 mod q is a ring map Z_q[X]/(X^N + 1) -> Z_q.
    Through it: the plaintext product decrypts to Dec(ct)(x) pt(x) exactly (no
    noise term: Dec(c0 p, c1 p) = (c0 + c1 s) p), the Galois image of the secret
    key evaluates to s(x^g) and its square to s(x)^2 on every q- and special
    prime, and the RNS conversion of signed integers is the least residue."""
    o = small
    N = o.N
    rng = _rng(77)
    s = o.secret_key()
    l = 3
    ct = o.encrypt(o.encode(rng.uniform(-1, 1, o.M), o.delta, l), 0x5151, o.delta)
    coeffs = rng.integers(-1000, 1000, N)
    pt = o.to_rns(coeffs, l)
    for i in range(l):
        assert all(int(pt[i][j]) == int(coeffs[j]) % o.q[i] for j in range(N))
    m, mp = o.decrypt(ct), o.decrypt(o.mul_plain(ct, pt, 1.0))
    for i in range(l):
        q = o.q[i]
        x = _root_2n(q, N, i)
        assert _eval(mp[i], x, q) == _eval(m[i], x, q) * _eval(pt[i], x, q) % q
    mods = o.q + o.p
    s2 = np.zeros((len(mods), N), np.uint64)
    L.or_sk_square(o._ctx, s2)
    for g in (galois_rot(o.logN, 1), galois_rot(o.logN, 5), galois_conj(o.logN)):
        t = np.zeros((len(mods), N), np.uint64)
        L.or_sk_galois(o._ctx, g, t)
        for i, q in enumerate(mods):
            x = _root_2n(q, N, 100 + i)
            sq = [int(v) % q for v in s]
            assert _eval(t[i], x, q) == _eval(sq, pow(x, g, q), q), (g, i)
            # a planted wrong exponent does not match
            assert _eval(t[i], x, q) != _eval(sq, pow(x, g + 2, q), q), (g, i)
            if g == galois_conj(o.logN):
                assert _eval(s2[i], x, q) == _eval(sq, x, q) ** 2 % q, i
