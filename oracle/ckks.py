"""O1 -- textbook RNS-CKKS evaluator over the oracle's C core.

TEST INFRASTRUCTURE ONLY (tests/, the smoke check and the CPU-baseline leg of
the benchmark).  Ciphertexts are held in the COEFFICIENT domain as uint64
arrays [npoly][l][N]; every product is an exact negacyclic product mod q_i.

Scheme (paper section "Homomorphic Encryption"):
  KeyGen  -- s ternary; pk = (-a s + e, a); switching keys in hybrid form
  Encrypt -- v * pk + (m + e0, e1)
  Decrypt -- c0 + c1 s
  Add     -- limb-wise addition
  Mult    -- tensor (d0, d1, d2), d2 switched back to s (relinearisation)
  Rescale -- divide by the last prime with rounding (drops one limb)
  Encode / Decode -- canonical embedding phi over N/2 complex slots
  Rotate  -- Galois automorphism X -> X^(5^r) + key switch (slot i <- i + r)
and the complex conjugation X -> X^(2N-1) used for the packed SNP pairs.

Scale bookkeeping (identical op order on the CUDA side): a product multiplies
the scales, a rescale divides by float(q_last), a sum keeps the scale of its
first operand (operands whose scales differ by more than 2^-10 are rejected).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import build_oracle

_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")

_LIB = None


def lib():
    """Load (building if needed) the oracle's C core."""
    global _LIB
    if _LIB is not None:
        return _LIB
    L = ctypes.CDLL(build_oracle.build())
    u64, i32, u32, vp, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_double
    sig = {
        "or_is_prime": (i32, [u64]),
        "or_gen_primes": (i32, [i32, i32, i32, i32, i32, i32, _u64p, _u64p]),
        "or_primitive_root_2n": (u64, [u64, i32]),
        "or_polymul": (None, [_u64p, _u64p, _u64p, i32, u64, u64]),
        "or_polymul_schoolbook": (None, [_u64p, _u64p, _u64p, i32, u64]),
        "or_chacha20_block": (None, [_u32p, u32, _u32p, _u32p]),
        "or_sample_ternary": (None, [u64, u64, i32, _i64p]),
        "or_sample_cbd": (None, [u64, u64, i32, _i64p]),
        "or_sample_uniform": (None, [u64, u64, u32, u64, i32, _u64p]),
        "or_ctx_create": (vp, [i32, i32, i32, i32, i32, i32, i32, u64]),
        "or_ctx_destroy": (None, [vp]),
        "or_ctx_alpha": (i32, [vp]),
        "or_ctx_moduli": (None, [vp, _u64p]),
        "or_keygen_sk": (None, [vp, _i64p]),
        "or_keygen_pk": (None, [vp, _u64p, _u64p]),
        "or_keygen_ksk": (None, [vp, u32, i32, i32, _u64p, _u64p]),
        "or_ks_special": (i32, [vp, i32]),
        "or_sk_square": (None, [vp, _u64p]),
        "or_sk_galois": (None, [vp, u64, _u64p]),
        "or_automorphism": (None, [_u64p, _u64p, i32, u64, u64]),
        "or_encrypt": (None, [vp, _u64p, i32, u64, _u64p, _u64p, _u64p]),
        "or_decrypt": (None, [vp, _u64p, i32, _u64p]),
        "or_mul_plain": (None, [vp, _u64p, i32, _u64p, i32, _u64p]),
        "or_tensor": (None, [vp, _u64p, _u64p, i32, _u64p]),
        "or_rescale": (None, [vp, _u64p, i32, i32, _u64p]),
        "or_keyswitch": (None, [vp, _u64p, i32, _u64p, i32, _u64p]),
        "or_keyswitch_hoisted": (None, [vp, _u64p, i32, i32, _u64p, _u64p, i32, _u64p]),
        "or_relin_rescale": (None, [vp, _u64p, i32, _u64p, i32, _u64p]),
        "or_fft_twiddles": (None, [i32, i32, _f64p, _f64p]),
        "or_encode": (None, [i32, _f64p, dbl, _i64p]),
        "or_to_rns": (None, [vp, _i64p, i32, _u64p]),
        "or_to_rns_mods": (None, [i32, _i64p, _u64p, i32, _u64p]),
        "or_set_threads": (None, [i32]),
        "or_get_threads": (i32, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


# ---------------------------------------------------------------------------
# small helpers (definitions written out)
# ---------------------------------------------------------------------------
def chacha20_block(key_words, counter, nonce_words):
    """ChaCha20 block function (RFC 8439 section 2.3) -> 16 uint32 words."""
    out = np.zeros(16, np.uint32)
    lib().or_chacha20_block(np.ascontiguousarray(key_words, np.uint32), counter,
                            np.ascontiguousarray(nonce_words, np.uint32), out)
    return out


def slot_indices(logN: int) -> np.ndarray:
    """u_j = ((5^j mod 2N) - 1) / 4: the rotation-group position of slot j."""
    twoN = 2 << logN
    M = 1 << (logN - 1)
    u = np.zeros(M, np.int64)
    g = 1
    for j in range(M):
        u[j] = (g - 1) // 4
        g = (g * 5) % twoN
    return u


def galois_rot(logN: int, r: int) -> int:
    """Galois element of a left rotation by r slots: 5^(r mod N/2) mod 2N."""
    M = 1 << (logN - 1)
    return pow(5, r % M, 2 << logN)


def galois_conj(logN: int) -> int:
    return (2 << logN) - 1


def decode_naive(m_int, logN: int, scale: float) -> np.ndarray:
    """Definition of Decode: z_j = m(zeta^(5^j)) / scale, zeta = exp(i pi/N)."""
    N = 1 << logN
    M = N // 2
    m = np.asarray(m_int, dtype=np.float64)
    e5 = np.array([pow(5, j, 2 * N) for j in range(M)], dtype=np.int64)
    k = np.arange(N, dtype=np.int64)
    ang = np.pi * ((np.outer(e5, k)) % (2 * N)) / N
    return (np.exp(1j * ang) @ m) / scale


def encode_naive_real(z, logN: int, scale: float) -> np.ndarray:
    """Definition of Encode before rounding: the real m with m(zeta^(5^j)) =
    scale*z_j and m(conj) = conj, i.e. m_k = (2 scale / N) Re sum_j z_j zeta^(-k 5^j)."""
    N = 1 << logN
    M = N // 2
    zz = np.zeros(M, complex)
    zz[: len(z)] = z
    e5 = np.array([pow(5, j, 2 * N) for j in range(M)], dtype=np.int64)
    k = np.arange(N, dtype=np.int64)
    ang = -np.pi * ((np.outer(k, e5)) % (2 * N)) / N
    return (2.0 * scale / N) * np.real(np.exp(1j * ang) @ zz)


@dataclass
class Ct:
    """Ciphertext (npoly = 2) or tensor (npoly = 3), coefficient domain."""
    c: np.ndarray  # uint64 [npoly][l][N]
    scale: float

    @property
    def level(self) -> int:
        return self.c.shape[1]

    def copy(self) -> "Ct":
        return Ct(self.c.copy(), self.scale)


class ScaleMismatch(ValueError):
    pass


class OracleCKKS:
    """Textbook RNS-CKKS with hybrid key switching."""

    def __init__(self, logN, L, q0_bits=60, scale_bits=40, K=1, sp_bits=60, dnum=None,
                 seed=0):
        self.logN, self.L, self.K = logN, L, K
        self.N = 1 << logN
        self.M = self.N // 2
        self.dnum = L if dnum is None else dnum
        self.seed = seed
        self.delta = float(2 ** scale_bits)
        self._ctx = lib().or_ctx_create(logN, L, q0_bits, scale_bits, K, sp_bits, self.dnum, seed)
        if not self._ctx:
            raise ValueError("oracle context creation failed")
        mods = np.zeros(L + K, np.uint64)
        lib().or_ctx_moduli(self._ctx, mods)
        self.mods = mods
        self.q = [int(x) for x in mods[:L]]
        self.p = [int(x) for x in mods[L:]]
        self.alpha = lib().or_ctx_alpha(self._ctx)
        # key switches at level l use the first ks_k[l] special primes; one key
        # family per count k covers the levels up to key_lmax[k]
        self.ks_k = [0] + [lib().or_ks_special(self._ctx, l) for l in range(1, L + 1)]
        self.key_lmax = {}
        for l in range(1, L + 1):
            self.key_lmax[self.ks_k[l]] = l
        self.keys = {}

    def __del__(self):
        try:
            if self._ctx:
                lib().or_ctx_destroy(self._ctx)
                self._ctx = None
        except Exception:
            pass

    # ----------------------------------------------------------- keys
    def secret_key(self) -> np.ndarray:
        s = np.zeros(self.N, np.int64)
        lib().or_keygen_sk(self._ctx, s)
        return s

    def keygen(self, galois=()):
        """pk, relinearisation key (id 0) and one switching key per Galois element."""
        N, L = self.N, self.L
        self.pk_b = np.zeros((L, N), np.uint64)
        self.pk_a = np.zeros((L, N), np.uint64)
        lib().or_keygen_pk(self._ctx, self.pk_b, self.pk_a)
        t = np.zeros((L + self.K, N), np.uint64)
        lib().or_sk_square(self._ctx, t)
        self.keys[0] = self._ksk(0, t)
        for g in galois:
            self.add_galois_key(g)

    def add_galois_key(self, g: int):
        t = np.zeros((self.L + self.K, self.N), np.uint64)
        lib().or_sk_galois(self._ctx, g, t)
        self.keys[int(g)] = self._ksk(int(g), t)

    def _ksk(self, key_id, target):
        """{k: array [ceil(lmax/alpha)][2][lmax + k][N]} for every special-prime
        count k in use (target: residues over all L + K moduli)."""
        fam = {}
        for k, lmax in sorted(self.key_lmax.items()):
            dk = -(-lmax // self.alpha)
            out = np.zeros((dk, 2, lmax + k, self.N), np.uint64)
            lib().or_keygen_ksk(self._ctx, key_id, k, lmax, np.ascontiguousarray(target), out)
            fam[k] = out
        return fam

    # ----------------------------------------------------------- encoding
    def encode_int(self, z, scale: float) -> np.ndarray:
        """Encoding procedure -> signed integer coefficients (int64 [N])."""
        zz = np.zeros(self.M, complex)
        z = np.asarray(z)
        zz[: z.shape[0]] = z
        buf = np.ascontiguousarray(np.stack([zz.real, zz.imag], axis=1).reshape(-1), np.float64)
        out = np.zeros(self.N, np.int64)
        lib().or_encode(self.logN, buf, float(scale), out)
        return out

    def to_rns(self, coeffs, level: int) -> np.ndarray:
        out = np.zeros((level, self.N), np.uint64)
        lib().or_to_rns(self._ctx, np.ascontiguousarray(coeffs, np.int64), level, out)
        return out

    def encode(self, z, scale: float, level: int) -> np.ndarray:
        return self.to_rns(self.encode_int(z, scale), level)

    def encode_const_int(self, c: float, scale: float) -> int:
        """A constant in every slot encodes to the constant polynomial
        round(c * scale) (ties to even, as llrint)."""
        return int(np.rint(np.float64(c) * np.float64(scale)))

    def decode(self, res: np.ndarray, scale: float) -> np.ndarray:
        """CRT (exact, Python integers), centre, then the canonical embedding
        evaluated with numpy's FFT: z_j = sum_k c_k zeta^k w^(k u_j) / scale,
        c_k = m_k + i m_(k+M)."""
        m = self.crt_centered(res)
        mf = np.array([float(v) for v in m])
        N, M = self.N, self.M
        c = mf[:M] + 1j * mf[M:]
        k = np.arange(M)
        tw = np.exp(1j * np.pi * k / N)
        E = M * np.fft.ifft(c * tw)
        return E[slot_indices(self.logN)] / scale

    def crt_centered(self, res: np.ndarray):
        l = res.shape[0]
        qs = self.q[:l]
        Q = 1
        for x in qs:
            Q *= x
        terms = []
        for i, qi in enumerate(qs):
            Qi = Q // qi
            terms.append((Qi * pow(Qi, -1, qi)) % Q)
        out = []
        rows = [[int(v) for v in res[i]] for i in range(l)]
        for kk in range(self.N):
            v = 0
            for i in range(l):
                v += rows[i][kk] * terms[i]
            v %= Q
            if v > Q // 2:
                v -= Q
            out.append(v)
        return out

    # ----------------------------------------------------------- enc / dec
    def encrypt(self, pt: np.ndarray, enc_id: int, scale: float) -> Ct:
        l = pt.shape[0]
        ct = np.zeros((2, l, self.N), np.uint64)
        lib().or_encrypt(self._ctx, np.ascontiguousarray(pt), l, enc_id, self.pk_b, self.pk_a, ct)
        return Ct(ct, float(scale))

    def decrypt(self, ct: Ct) -> np.ndarray:
        assert ct.c.shape[0] == 2
        l = ct.level
        m = np.zeros((l, self.N), np.uint64)
        lib().or_decrypt(self._ctx, np.ascontiguousarray(ct.c), l, m)
        return m

    def decrypt_decode(self, ct: Ct) -> np.ndarray:
        return self.decode(self.decrypt(ct), ct.scale)

    # ----------------------------------------------------------- arithmetic
    def _qcol(self, l):
        return np.array(self.q[:l], dtype=object).reshape(1, l, 1)

    def _check_scales(self, a: Ct, b: Ct):
        if abs(a.scale / b.scale - 1.0) > 2.0 ** -10:
            raise ScaleMismatch((a.scale, b.scale))

    def _binop(self, a: Ct, b: Ct, sign: int) -> Ct:
        if a.level != b.level or a.c.shape[0] != b.c.shape[0]:
            raise ValueError("level/shape mismatch %s %s" % (a.c.shape, b.c.shape))
        self._check_scales(a, b)
        out = np.empty_like(a.c)
        for i in range(a.level):
            q = np.uint64(self.q[i])
            x = a.c[:, i, :]
            y = b.c[:, i, :]
            if sign > 0:
                s = x + y  # < 2^63, no wrap
                out[:, i, :] = np.where(s >= q, s - q, s)
            else:
                out[:, i, :] = np.where(x >= y, x - y, x + q - y)
        return Ct(out, a.scale)

    def add(self, a: Ct, b: Ct) -> Ct:
        return self._binop(a, b, +1)

    def sub(self, a: Ct, b: Ct) -> Ct:
        return self._binop(a, b, -1)

    def negate(self, a: Ct) -> Ct:
        out = np.empty_like(a.c)
        for i in range(a.level):
            q = np.uint64(self.q[i])
            x = a.c[:, i, :]
            out[:, i, :] = np.where(x == 0, x, q - x)
        return Ct(out, a.scale)

    def _scalar_mul(self, a: Ct, vals) -> Ct:
        """multiply limb i of every poly by the residue vals[i] (exact)."""
        out = np.empty_like(a.c)
        for i in range(a.level):
            q = self.q[i]
            v = vals[i] % q
            x = a.c[:, i, :].astype(object)
            out[:, i, :] = ((x * v) % q).astype(np.uint64)
        return Ct(out, a.scale)

    def add_const(self, a: Ct, c: float) -> Ct:
        """add the constant c (encoded at the ciphertext's scale) to every slot."""
        m0 = self.encode_const_int(c, a.scale)
        out = a.c.copy()
        for i in range(a.level):
            q = self.q[i]
            out[0, i, 0] = np.uint64((int(out[0, i, 0]) + m0) % q)
        return Ct(out, a.scale)

    def mul_int(self, a: Ct, k: int) -> Ct:
        """multiply by a small integer; no rescale, scale unchanged."""
        return self._scalar_mul(a, [k] * a.level)

    def mul_const(self, a: Ct, c: float) -> Ct:
        """multiply by a real constant encoded as round(c * q_last), then
        rescale: the scale is multiplied by float(q_last) and divided again."""
        ql = self.q[a.level - 1]
        m0 = self.encode_const_int(c, float(ql))
        t = self._scalar_mul(a, [m0] * a.level)
        t.scale = a.scale * float(ql)
        return self.rescale(t)

    def mul_plain(self, a: Ct, pt: np.ndarray, pt_scale: float) -> Ct:
        """product with a plaintext polynomial (no rescale)."""
        l = a.level
        npoly = a.c.shape[0]
        out = np.zeros_like(a.c)
        lib().or_mul_plain(self._ctx, np.ascontiguousarray(a.c), npoly,
                           np.ascontiguousarray(pt[:l]), l, out)
        return Ct(out, a.scale * pt_scale)

    def mul_mask(self, a: Ct, z) -> Ct:
        """slot-wise product with a public vector z encoded at scale q_last,
        then rescale (the ciphertext's scale is preserved up to rounding)."""
        ql = float(self.q[a.level - 1])
        pt = self.encode(z, ql, a.level)
        return self.rescale(self.mul_plain(a, pt, ql))

    def tensor(self, a: Ct, b: Ct) -> Ct:
        if a.level != b.level:
            raise ValueError("level mismatch")
        l = a.level
        out = np.zeros((3, l, self.N), np.uint64)
        lib().or_tensor(self._ctx, np.ascontiguousarray(a.c), np.ascontiguousarray(b.c), l, out)
        return Ct(out, a.scale * b.scale)

    def keyswitch(self, x: np.ndarray, key_id: int) -> np.ndarray:
        l = x.shape[0]
        k = self.ks_k[l]
        out = np.zeros((2, l, self.N), np.uint64)
        lib().or_keyswitch(self._ctx, np.ascontiguousarray(x), l,
                           np.ascontiguousarray(self.keys[key_id][k]), self.key_lmax[k], out)
        return out

    def relin(self, t: Ct) -> Ct:
        assert t.c.shape[0] == 3
        k = self.keyswitch(t.c[2], 0)
        return self.add(Ct(t.c[:2].copy(), t.scale), Ct(k, t.scale))

    def rescale(self, a: Ct) -> Ct:
        l = a.level
        if l < 2:
            raise ValueError("no level left to rescale")
        npoly = a.c.shape[0]
        out = np.zeros((npoly, l - 1, self.N), np.uint64)
        lib().or_rescale(self._ctx, np.ascontiguousarray(a.c), npoly, l, out)
        return Ct(out, a.scale / float(self.q[l - 1]))

    def relin_rescale(self, t: Ct) -> Ct:
        """relinearisation fused with the rescale after it: y = keyproduct(d2)
        + P (d0, d1) divided once by P q_{l-1}, rounding to nearest (one base
        conversion from the special primes and q_{l-1})."""
        assert t.c.shape[0] == 3
        l = t.level
        if l < 2:
            raise ValueError("no level left to rescale")
        k = self.ks_k[l]
        out = np.zeros((2, l - 1, self.N), np.uint64)
        lib().or_relin_rescale(self._ctx, np.ascontiguousarray(t.c), l,
                               np.ascontiguousarray(self.keys[0][k]), self.key_lmax[k], out)
        return Ct(out, t.scale / float(self.q[l - 1]))

    def mult(self, a: Ct, b: Ct) -> Ct:
        return self.relin_rescale(self.tensor(a, b))

    def drop(self, a: Ct, level: int) -> Ct:
        if level > a.level:
            raise ValueError("cannot raise a level")
        return Ct(a.c[:, :level, :].copy(), a.scale)

    def automorphism(self, a: Ct, g: int) -> Ct:
        out = np.zeros_like(a.c)
        for p in range(a.c.shape[0]):
            for i in range(a.level):
                lib().or_automorphism(np.ascontiguousarray(a.c[p, i]), out[p, i], self.logN,
                                      g, self.q[i])
        return Ct(out, a.scale)

    def apply_galois(self, a: Ct, g: int) -> Ct:
        t = self.automorphism(a, g)
        k = self.keyswitch(t.c[1], g)
        c0 = Ct(t.c[0:1].copy(), a.scale)
        k0 = Ct(k[0:1].copy(), a.scale)
        out = np.concatenate([self.add(c0, k0).c, k[1:2]], axis=0)
        return Ct(out, a.scale)

    def rotate(self, a: Ct, r: int) -> Ct:
        """left rotation: slot i <- slot i + r."""
        return self.apply_galois(a, galois_rot(self.logN, r))

    def conj(self, a: Ct) -> Ct:
        return self.apply_galois(a, galois_conj(self.logN))

    def rotate_sum(self, a: Ct, rs) -> Ct:
        """a + sum_r Rotate(a, r) with the rotations' key switches hoisted: one
        ModUp of c1, each rotation's automorphism applied to the ModUp digits,
        the inner products with the rotations' keys summed in the extended
        basis, one ModDown; c0 + sum_r sigma_r(c0) is added exactly."""
        l = a.level
        k = self.ks_k[l]
        gal = [galois_rot(self.logN, r) for r in rs]
        keys = np.ascontiguousarray(np.stack([self.keys[g][k] for g in gal]))
        ks = np.zeros((2, l, self.N), np.uint64)
        lib().or_keyswitch_hoisted(self._ctx, np.ascontiguousarray(a.c[1]), l, len(gal),
                                   np.array(gal, np.uint64), keys, self.key_lmax[k], ks)
        acc = Ct(np.stack([a.c[0], a.c[1]]), a.scale)
        for g in gal:
            rot0 = self.automorphism(Ct(a.c[0:1].copy(), a.scale), g)
            acc = self.add(acc, Ct(np.concatenate([rot0.c, np.zeros_like(rot0.c)]), a.scale))
        return self.add(acc, Ct(ks, a.scale))
