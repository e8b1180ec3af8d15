"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work is compared bit for bit in the coefficient domain (ciphertexts,
keys, plaintexts).  Decrypted real results are compared within the stated
tolerances.  Inputs come from the seeded generators only; no expected value
comes from the CUDA path."""
import numpy as np
import pytest

from oracle import ckks as O
from oracle.ckks import OracleCKKS, galois_conj, galois_rot
from paper_1902_04303_gb300.datagen import make_residues, make_slots

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    torch.cuda.set_device(0)
    from paper_1902_04303_gb300 import build
    build.build()
    from paper_1902_04303_gb300 import gwhe
    return gwhe


def pair(g, logN, L, K, dnum, seed=3, rot=(1, -1, 2, 8, 3, 4, 5, 6, 7, -2, -3, 16, 24), conj=True,
         keys=True):
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=seed)
    o = OracleCKKS(logN=logN, L=L, K=K, dnum=dnum, seed=seed)
    if keys:
        ctx.keygen(rot_steps=rot, conj=conj)
        gal = [galois_rot(logN, r) for r in rot] + ([galois_conj(logN)] if conj else [])
        o.keygen(galois=gal)
    return ctx, o


def rand_ct(o, l, seed, npoly=2):
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.stack([np.stack([rng.integers(0, o.q[i], size=o.N, dtype=np.uint64) for i in range(l)])
                  for _ in range(npoly)])
    return O.Ct(c, o.delta)


# ------------------------------------------------------------------ NTT
@pytest.mark.parametrize("logN", [4, 7, 10, 12, 13, 14, 15, 16, 17])
def test_ntt_roundtrip_and_negacyclic_product(g, logN):
    import torch
    L = 4  # one-limb digits with one 60-bit special prime
    ctx, o = pair(g, logN, L, 1, L, keys=False)
    npoly = 3
    x = make_residues(npoly * L, ctx.N, [ctx.q[i % L] for i in range(npoly * L)], seed=logN)
    t = torch.from_numpy(x.view(np.int64)).cuda()
    ctx.ntt_batch(t, npoly, L, inverse=False)
    ctx.ntt_batch(t, npoly, L, inverse=True)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy().view(np.uint64), x)
    # products through the NTT domain equal the oracle's negacyclic products
    a = rand_ct(o, L, 100 + logN)
    b = rand_ct(o, L, 200 + logN)
    ga, gb = ctx.import_ct(a.c, 1.0), ctx.import_ct(b.c, 1.0)
    got = ctx.tensor(ga, gb).export()
    want = o.tensor(a, b).c
    assert np.array_equal(got, want)


# ------------------------------------------------------------------ keys, encoding
@pytest.mark.parametrize("logN,L,K,dnum", [(10, 6, 3, 3), (13, 4, 1, 4), (10, 9, 7, 2)])
def test_keygen_bit_exact(g, logN, L, K, dnum):
    ctx, o = pair(g, logN, L, K, dnum)
    assert np.array_equal(ctx.export_secret(), o.secret_key())
    pk = ctx.export_pk()
    assert np.array_equal(pk[0], o.pk_b) and np.array_equal(pk[1], o.pk_a)
    for l in range(1, L + 1):
        assert ctx.ks_special(l) == (o.ks_k[l], o.key_lmax[o.ks_k[l]]), l
    for kid in [0, galois_rot(logN, 1), galois_rot(logN, -1), galois_conj(logN)]:
        got, want = ctx.export_ksk(kid), o.keys[kid]
        assert set(got) == set(want), kid
        for k in want:
            assert np.array_equal(got[k], want[k]), (kid, k)


@pytest.mark.parametrize("logN", [5, 10, 13, 16, 17])
def test_encode_bit_exact(g, logN):
    ctx = g.Context(logN, 2, K=1)
    o = OracleCKKS(logN=logN, L=2, K=1)
    for seed, sc in [(1, 2.0 ** 40), (2, float(ctx.q[1])), (3, 2.0 ** 30)]:
        z = make_slots(ctx.M, seed, scale=3.0)
        assert np.array_equal(ctx.encode(z, sc), o.encode_int(z, sc))
    # a REP-like vector with exact small integers and a one-hot mask
    z = np.zeros(ctx.M, complex)
    z[: ctx.M // 2] = 2 + 1j
    assert np.array_equal(ctx.encode(z, 2.0 ** 40), o.encode_int(z, 2.0 ** 40))


@pytest.mark.parametrize("logN,L,K,dnum", [(10, 6, 3, 3), (16, 5, 2, 3), (17, 4, 2, 2)])
def test_encrypt_decrypt_bit_exact(g, logN, L, K, dnum):
    ctx, o = pair(g, logN, L, K, dnum, rot=(), conj=False)
    z = make_slots(ctx.M, 9)
    for lvl, eid in [(L, 7), (2, 0x1000000 + 5)]:
        gc = ctx.encrypt(z, o.delta, lvl, eid)
        oc = o.encrypt(o.encode(z, o.delta, lvl), eid, o.delta)
        assert np.array_equal(gc.export(), oc.c)
        assert np.array_equal(ctx.decrypt(gc), o.decrypt(oc))
        # fresh-encryption noise over the canonical embedding grows ~ N / Delta
        assert np.max(np.abs(ctx.decrypt_decode(gc) - z)) < 2e-5
    m = o.encode_int(z, o.delta)
    gc = ctx.encrypt_coeffs(m, o.delta, L, 99)
    assert np.array_equal(gc.export(), o.encrypt(o.to_rns(m, L), 99, o.delta).c)


# ------------------------------------------------------------------ operations
@pytest.fixture(scope="module")
def small(g):
    return pair(g, 10, 6, 3, 3, seed=21)


def test_elementwise_ops_bit_exact(g, small):
    ctx, o = small
    a, b = rand_ct(o, 6, 1), rand_ct(o, 6, 2)
    ga, gb = ctx.import_ct(a.c, a.scale), ctx.import_ct(b.c, b.scale)
    assert np.array_equal(ctx.add(ga, gb).export(), o.add(a, b).c)
    assert np.array_equal(ctx.sub(ga, gb).export(), o.sub(a, b).c)
    assert np.array_equal(ctx.negate(ga).export(), o.negate(a).c)
    ga2 = ctx.import_ct(a.c, a.scale)
    assert np.array_equal(ctx.add_const(ga2, 0.37).export(), o.add_const(a, 0.37).c)
    ga3 = ctx.import_ct(a.c, a.scale)
    assert np.array_equal(ctx.mul_int(ga3, -3).export(), o.mul_int(a, -3).c)
    ga4 = ctx.import_ct(a.c, a.scale)
    want = o.mul_const(a, -0.0271)
    got = ctx.mul_const(ga4, -0.0271)
    assert np.array_equal(got.export(), want.c) and got.scale == want.scale
    z = (np.arange(ctx.M) % 5 == 1).astype(float)
    got = ctx.mul_mask(ga, z)
    want = o.mul_mask(a, z)
    assert np.array_equal(got.export(), want.c) and got.scale == want.scale


def test_tensor_sum_relin_rescale_bit_exact(g, small):
    ctx, o = small
    A = [rand_ct(o, 6, 10 + i) for i in range(37)]
    B = [rand_ct(o, 6, 60 + i) for i in range(37)]
    gA = [ctx.import_ct(x.c, x.scale) for x in A]
    gB = [ctx.import_ct(x.c, x.scale) for x in B]
    t = ctx.tensor_sum(list(zip(gA, gB)))
    want = o.tensor(A[0], B[0])
    for x, y in zip(A[1:], B[1:]):
        want = o.add(want, o.tensor(x, y))
    assert np.array_equal(t.export(), want.c)
    r = ctx.relin(t)
    wr = o.relin(want)
    assert np.array_equal(r.export(), wr.c)
    ctx.rescale(r)
    wr = o.rescale(wr)
    assert np.array_equal(r.export(), wr.c) and r.scale == wr.scale


def test_mult_rotate_conj_bit_exact(g, small):
    ctx, o = small
    z1, z2 = make_slots(ctx.M, 31), make_slots(ctx.M, 32)
    a = o.encrypt(o.encode(z1, o.delta, 6), 1, o.delta)
    b = o.encrypt(o.encode(z2, o.delta, 6), 2, o.delta)
    ga, gb = ctx.import_ct(a.c, a.scale), ctx.import_ct(b.c, b.scale)
    m = ctx.mult(ga, gb)
    assert np.array_equal(m.export(), o.mult(a, b).c)
    for r in (1, -1, 2, 8):
        assert np.array_equal(ctx.rotate(ga, r).export(), o.rotate(a, r).c), r
    assert np.array_equal(ctx.conj(ga).export(), o.conj(a).c)
    assert np.max(np.abs(ctx.decrypt_decode(ctx.rotate(ga, 2)) - np.roll(z1, -2))) < 1e-6
    # at a lower level (shorter last digit)
    ga.drop(4)
    a4 = o.drop(a, 4)
    assert np.array_equal(ctx.rotate(ga, -1).export(), o.rotate(a4, -1).c)


@pytest.mark.parametrize("l", [6, 5, 3, 1])
def test_keyswitch_levels_bit_exact(g, small, l):
    ctx, o = small
    x = rand_ct(o, l, 70 + l, npoly=1).c[0]
    for kid in (0, galois_conj(10)):
        assert np.array_equal(ctx.keyswitch(x, kid), o.keyswitch(x, kid))


@pytest.fixture(scope="module")
def wide(g):
    # 7 special primes, digits of 5 limbs (two digits above level 5): levels
    # 1..9 use 2..5 of them
    return pair(g, 10, 9, 7, 2, seed=22)


def test_wide_context_uses_several_special_prime_counts(wide):
    ctx, o = wide
    ks = [ctx.ks_special(l)[0] for l in range(1, 10)]
    assert len(set(ks)) >= 3 and max(ks) < 7, ks


@pytest.mark.parametrize("l", range(1, 10))
def test_keyswitch_reduced_special_primes_bit_exact(g, wide, l):
    """every level of a context whose switches use 2..5 of the 7 special
    primes: relinearisation and rotation switches bit-exact, and a rotation
    plus rescale through the set path."""
    ctx, o = wide
    x = rand_ct(o, l, 90 + l, npoly=1).c[0]
    for kid in (0, galois_rot(10, 1)):
        assert np.array_equal(ctx.keyswitch(x, kid), o.keyswitch(x, kid)), kid
    if l >= 2:
        a = rand_ct(o, l, 120 + l)
        ga = ctx.import_ct(a.c, a.scale)
        assert np.array_equal(ctx.rotate(ga, -1).export(), o.rotate(a, -1).c)
        b = rand_ct(o, l, 140 + l)
        gb = ctx.import_ct(b.c, b.scale)
        assert np.array_equal(ctx.mult(ga, gb).export(), o.mult(a, b).c)


def test_errors_are_status_codes(g, small):
    ctx, o = small
    a = ctx.import_ct(rand_ct(o, 6, 1).c, o.delta)
    b = ctx.import_ct(rand_ct(o, 5, 2).c, o.delta)
    with pytest.raises(g.GwheError) as e:
        ctx.add(a, b)
    assert e.value.code == -3  # ELEVEL
    c = ctx.import_ct(rand_ct(o, 6, 3).c, o.delta * 1.5)
    with pytest.raises(g.GwheError) as e:
        ctx.add(a, c)
    assert e.value.code == -4  # ESCALE
    with pytest.raises(g.GwheError) as e:
        ctx.rotate(a, 11)  # no key for 11
    assert e.value.code == -5  # ENOKEY
    one = ctx.import_ct(rand_ct(o, 1, 4).c, o.delta)
    with pytest.raises(g.GwheError) as e:
        ctx.rescale(one)
    assert e.value.code == -3


# ------------------------------------------------------------------ full size
def test_full_size_keyswitch_and_rescale_bit_exact(g):
    """N = 2^16, 24 limbs, 8 special primes, dnum = 3: one relinearisation
    key switch at the top level and one rescale, sampled against the oracle."""
    logN, L, K, dnum = 16, 24, 8, 3
    ctx, o = pair(g, logN, L, K, dnum, seed=5, rot=(), conj=False)
    x = rand_ct(o, L, 77, npoly=1).c[0]
    assert np.array_equal(ctx.keyswitch(x, 0), o.keyswitch(x, 0))
    a = rand_ct(o, L, 78)
    ga = ctx.import_ct(a.c, a.scale)
    ctx.rescale(ga)
    assert np.array_equal(ga.export(), o.rescale(a).c)


@pytest.mark.parametrize("l,rs", [(6, [1, 2, 3]), (5, [8, 16, 24]), (3, [2, 4, 6]), (4, [-1, -2, -3]),
                                  (2, [1]), (1, [2, 4, 6]), (6, [1, 2, 3, 4, 5, 6, 7]),
                                  (2, [1, 2, 3, 4, 5, 6, 7])])
def test_hoisted_rotation_sum_bit_exact(g, small, l, rs):
    """a + sum_r Rotate(a, r) with one shared ModUp and ModDown, at levels
    with one and two key digits."""
    ctx, o = small
    a = rand_ct(o, l, 200 + l)
    ga = ctx.import_ct(a.c, a.scale)
    assert np.array_equal(ctx.rotate_sum(ga, rs).export(), o.rotate_sum(a, rs).c)


@pytest.mark.parametrize("l", [9, 7, 4, 2])
def test_hoisted_rotation_sum_reduced_special_primes(g, wide, l):
    ctx, o = wide
    a = rand_ct(o, l, 230 + l)
    ga = ctx.import_ct(a.c, a.scale)
    assert np.array_equal(ctx.rotate_sum(ga, [1, 2, 3]).export(), o.rotate_sum(a, [1, 2, 3]).c)
    rs = [1, 2, 3, 4, 5, 6, 7]
    assert np.array_equal(ctx.rotate_sum(ga, rs).export(), o.rotate_sum(a, rs).c)


def test_ring_2_17_switches_and_rotations_bit_exact(g):
    """N = 2^17 (the ring of the paper's own runs): relinearisation switch,
    hoisted rotation sum, mult and rescale against the oracle."""
    logN = 17
    ctx, o = pair(g, logN, 5, 3, 2, seed=31, rot=(1, 2, 3), conj=False)
    x = rand_ct(o, 5, 301, npoly=1).c[0]
    assert np.array_equal(ctx.keyswitch(x, 0), o.keyswitch(x, 0))
    a, b = rand_ct(o, 4, 302), rand_ct(o, 4, 303)
    ga, gb = ctx.import_ct(a.c, a.scale), ctx.import_ct(b.c, b.scale)
    assert np.array_equal(ctx.rotate_sum(ga, [1, 2, 3]).export(), o.rotate_sum(a, [1, 2, 3]).c)
    assert np.array_equal(ctx.mult(ga, gb).export(), o.mult(a, b).c)


def test_hoisted_rotation_sum_batch_bit_exact(g, small):
    """the batched entry point (one set of ciphertexts) equals the oracle's
    hoisted sum of each ciphertext, seven rotations."""
    ctx, o = small
    rs = [1, 2, 3, 4, 5, 6, 7]
    srcs = [rand_ct(o, 4, 400 + i) for i in range(11)]
    outs = ctx.rotate_sum_batch([ctx.import_ct(a.c, a.scale) for a in srcs], rs)
    for a, out in zip(srcs, outs):
        assert np.array_equal(out.export(), o.rotate_sum(a, rs).c)


@pytest.mark.parametrize("l", [2, 6])
def test_hoisted_sum_of_fifteen_rotations(g, l):
    """A hoisted sum of 15 rotations (inner products in chunks of 7, 7 and 1
    that accumulate before the one ModDown, the c0 automorphism sums the
    same way) over a set of 9 ciphertexts, at one key digit (l = 2) and at
    three (l = 6): every output equals the oracle's hoisted sum."""
    rs = list(range(1, 16))
    ctx, o = pair(g, 10, 6, 3, 3, seed=61, rot=tuple(rs), conj=False)
    srcs = [rand_ct(o, l, 9000 + 10 * l + i) for i in range(9)]
    outs = ctx.rotate_sum_batch([ctx.import_ct(a.c, a.scale) for a in srcs], rs)
    for a, out in zip(srcs, outs):
        assert np.array_equal(out.export(), o.rotate_sum(a, rs).c)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6])
def test_every_ntt_shape_is_bit_exact(g, variant):
    """each compiled shape of the N = 2^16 transform gives the oracle's
    residues (round trip, negacyclic product, one key switch)."""
    import torch
    ctx, o = pair(g, 16, 3, 2, 3, seed=41, rot=(1,), conj=False)
    ctx.set_ntt_variant(variant)
    x = rand_ct(o, 3, 500 + variant, npoly=1).c[0]
    assert np.array_equal(ctx.keyswitch(x, 0), o.keyswitch(x, 0))
    a, b = rand_ct(o, 3, 510), rand_ct(o, 3, 511)
    ga, gb = ctx.import_ct(a.c, a.scale), ctx.import_ct(b.c, b.scale)
    assert np.array_equal(ctx.mult(ga, gb).export(), o.mult(a, b).c)
    t = torch.from_numpy(np.ascontiguousarray(a.c.astype(np.int64))).cuda()
    ref = t.clone()
    ctx.ntt_batch(t, 2, 3)
    ctx.ntt_batch(t, 2, 3, inverse=True)
    assert torch.equal(t, ref)


def test_autotune_picks_a_shape(g):
    ctx = g.Context(16, 2, K=1, dnum=2, seed=1)
    for rows in (64, 512):  # the small- and the large-launch class
        v, ms = ctx.autotune(rows=rows)
        assert 0 <= v < g.NTT_SHAPES and len(ms) == g.NTT_SHAPES and all(x > 0 for x in ms)
        assert ms[v] == min(ms)


# ------------------------------------------------------------------ the job's basis, set widths
@pytest.fixture(scope="module")
def paper_basis(g):
    """The paper-shaped job's ring and basis: N = 2^16, 24 q-limbs (60 + 23 x
    45 bits), 8 special primes of 60 bits, dnum = 3, with the keys of one
    hoisted ladder group (rotations 1..7), on both sides."""
    logN, L, K, dnum, seed = 16, 24, 8, 3, 29
    rot = (1, 2, 3, 4, 5, 6, 7)
    ctx = g.Context(logN, L, q0_bits=60, scale_bits=45, K=K, sp_bits=60, dnum=dnum, seed=seed)
    ctx.keygen(rot_steps=rot, conj=False)
    o = OracleCKKS(logN=logN, L=L, q0_bits=60, scale_bits=45, K=K, sp_bits=60, dnum=dnum,
                   seed=seed)
    o.keygen(galois=[galois_rot(logN, r) for r in rot])
    return ctx, o


def test_job_width_hoisted_sum_batch_at_paper_basis(g, paper_basis):
    """66 ciphertexts at 5 limbs (one key digit): the one-digit hoisted inner
    product walks the set in groups of 32 items (two full groups and a ragged
    one of 2), as the SNP batches' colSum and broadcast ladders do.  Items
    from every group equal the oracle's hoisted sum of seven rotations."""
    ctx, o = paper_basis
    rs = [1, 2, 3, 4, 5, 6, 7]
    cnt, l = 66, 5
    srcs = [rand_ct(o, l, 4000 + i) for i in range(cnt)]
    outs = ctx.rotate_sum_batch([ctx.import_ct(a.c, a.scale) for a in srcs], rs)
    for i in (0, 1, 31, 32, 33, 63, 64, 65):
        assert np.array_equal(outs[i].export(), o.rotate_sum(srcs[i], rs).c), i


def test_job_width_tensor_sum_at_paper_basis(g, paper_basis):
    """A tensor sum of 70 pairs at 4 limbs (the CP-REP inner loop's width:
    two 32-pair partial reductions and a ragged tail) equals the sum of the
    oracle's exact negacyclic tensors."""
    ctx, o = paper_basis
    npairs, l = 70, 4
    a = [rand_ct(o, l, 5000 + i) for i in range(npairs)]
    b = [rand_ct(o, l, 6000 + i) for i in range(npairs)]
    got = ctx.tensor_sum([(ctx.import_ct(x.c, x.scale), ctx.import_ct(y.c, y.scale))
                          for x, y in zip(a, b)]).export()
    q = np.array(o.q[:l], dtype=np.uint64).reshape(1, l, 1)
    want = np.zeros((3, l, o.N), dtype=np.uint64)
    for x, y in zip(a, b):
        want = want + o.tensor(x, y).c  # both below q < 2^60: no wrap
        want = np.where(want >= q, want - q, want)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("cnt", [5, 6])
def test_few_item_multi_digit_hoisted_sum_at_paper_basis(g, paper_basis, cnt):
    """5 or 6 ciphertexts at 20 limbs (three key digits), seven rotations: the
    covariate phase's hoisted sums (five items take one group of five, six
    a group of four and one of two); the first and the last equal the
    oracle's."""
    ctx, o = paper_basis
    rs = [1, 2, 3, 4, 5, 6, 7]
    srcs = [rand_ct(o, 20, 7000 + 10 * cnt + i) for i in range(cnt)]
    outs = ctx.rotate_sum_batch([ctx.import_ct(a.c, a.scale) for a in srcs], rs)
    for i in (0, cnt - 1):
        assert np.array_equal(outs[i].export(), o.rotate_sum(srcs[i], rs).c), i
