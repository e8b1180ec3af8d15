"""The encrypted semi-parallel GWAS circuit over the O1 evaluator.

TEST INFRASTRUCTURE ONLY.  Written from Algorithms 1-11 of the paper and the
readings listed in the design notes; the CUDA library implements the same
op sequence independently.  Every step below names the algorithm it follows.

Slot layouts (M = N/2 slots, nb = next power of two >= n, B = M/nb blocks):
  vector v (length n)        slots 0..n-1, zeros elsewhere
  CP matrix (Alg. 2)         one ciphertext per column
  REP row (section REP)      entry c repeated nb times: slot c*nb + t
  CCP matrix (Alg. 4)        column c in slots c*nb .. c*nb + nb - 1
  S batch (REP, complex)     row j of S_i: slot b*nb + t = S[j, 2b] + i S[j, 2b+1]
  S batch (CCP, complex)     one ciphertext: slot b*nb + t = S[t, 2b] + i S[t, 2b+1]

Two layouts of the SNP phase, both from eq. Sprime:
  M-CCP     S' = M S with M = I - X A X^T held as a CCP matrix and S in REP rows
            (Alg. 8; the first form of eq. Sprime, as in Alg. 11)
  factored  S' = S - (X A)(X^T S) with S in CCP (the second form of eq. Sprime):
            no n x n matrix, one SNP ciphertext per batch
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .ckks import Ct, OracleCKKS

# encryption ids (the nonce of each input ciphertext's randomness)
ENC_X = 0x100
ENC_A = 0x200
ENC_Y = 0x300
ENC_BETA0 = 0x301
ENC_DUPW = 0x302
ENC_DUPWZ = 0x303
ENC_XTREP = 0x10000
ENC_DUPM = 0x20000
ENC_S = 0x1000000
ENC_SCCP = 0x100000000
# a job's nonce (distinct per job under one key, so that no two jobs share
# encryption randomness) is added to every id above, shifted past them
ENC_NONCE_SHIFT = 36
MAX_NONCE = (1 << 12) - 1

SIGMA7_A = (-1.73496 / 8.0, 4.19407 / 8.0 ** 3, -5.43402 / 8.0 ** 5, 2.50739 / 8.0 ** 7)

BATCH_LEVEL = 4  # level at which a SNP batch enters (S', num, WS', WSS/WSC)
# M = I - X A X^T is only needed at BATCH_LEVEL + 1 limbs (the source of the
# Dup(M_j) masks); it is computed from X and A dropped to this level
M_LEVEL = BATCH_LEVEL + 4
# factored layout: a CCP SNP batch enters here and S' = S - (XA)(X^T S) leaves
# at BATCH_LEVEL - 1, where the M-CCP layout's S' is (product, mask, product)
FACT_LEVEL = BATCH_LEVEL + 2


@dataclass
class Layout:
    logN: int
    n: int
    d: int
    k: int

    @property
    def M(self):
        return 1 << (self.logN - 1)

    @property
    def nb(self):
        """next power of two >= n (the padded column length)."""
        return 1 << max(0, math.ceil(math.log2(self.n)))

    @property
    def B(self):
        """complex SNP columns per ciphertext (blocks of nb slots)."""
        return self.M // self.nb

    @property
    def tau(self):
        """SNPs per batch: eq. numSNPinBatch read as N / nb (two per slot)."""
        return 2 * self.B

    @property
    def batches(self):
        return -(-self.k // self.tau)

    @property
    def H(self):
        """ciphertexts holding the n x n CCP matrix M (nb^2 may exceed M)."""
        return -(-self.n // self.B)

    def check(self):
        if self.nb > self.M:
            raise ValueError("a column of nb slots does not fit one ciphertext")


LADDER_GROUP = 3  # ladder steps per hoisted key switch


def ladder_groups(steps):
    """Hoisted evaluation of a doubling ladder v += Rotate(v, s) over steps:
    up to LADDER_GROUP consecutive steps r, 2r, 4r merge into one group over
    the rotations r, 2r, ..., (2^m - 1) r (the same sum of rotations:
    v + Rot(v, r) + ... + Rot(v, (2^m - 1) r)); a shorter run of m steps gives
    2^m - 1 rotations."""
    out, i = [], 0
    while i < len(steps):
        m = 1
        while m < LADDER_GROUP and i + m < len(steps) and steps[i + m] == 2 * steps[i + m - 1]:
            m += 1
        out.append([t * steps[i] for t in range(1, 1 << m)])
        i += m
    return out


def replicate_period(m: int, M: int) -> int:
    """Period P of the shared replicate ladder for m entries: the smallest
    power of 2^LADDER_GROUP that is >= m (at most M).  Its step lists
    P, 2P, ..., M/2 and 1, 2, ..., P/2 split Alg. 1's ladder at a group
    boundary, so they need no rotation keys beyond Alg. 1's own."""
    P = 1 << LADDER_GROUP
    while P < m:
        P <<= LADDER_GROUP
    return min(P, M)


def circuit_ladders(layout: Layout, factored: bool = False):
    """The step lists of the circuit's ladders: Replicate/DotProd over all
    slots (Alg. 1, 5), colSum over nb (Alg. 4), Duplicate over the blocks
    (Alg. 7), and the factored layout's in-block broadcast."""
    lad = [[1 << i for i in range(layout.logN - 1)],
           [1 << i for i in range(int(math.log2(layout.nb)))],
           [layout.nb << i for i in range(int(math.log2(layout.B)))]]
    if factored:
        lad.append([-(1 << i) for i in range(int(math.log2(layout.nb)))])
    return lad


def rotation_steps(layout: Layout, factored: bool = False):
    """All rotations whose keys the circuit needs, as its hoisted ladder
    groups use them."""
    steps = []
    for lad in circuit_ladders(layout, factored):
        for g in ladder_groups(lad):
            for r in g:
                if r not in steps:
                    steps.append(r)
    return steps


class Circuit:
    def __init__(self, ev: OracleCKKS, layout: Layout, factored: bool = False, nonce: int = 0):
        if not 0 <= nonce <= MAX_NONCE:
            raise ValueError("job nonce out of range")
        self.ev = ev
        self.lay = layout
        self.factored = factored
        self.enc_base = nonce << ENC_NONCE_SHIFT
        layout.check()

    # --------------------------------------------------------- primitives
    def ladder(self, v: Ct, steps) -> Ct:
        """v += Rotate(v, s) for s in steps (the doubling ladders of Alg. 1, 4,
        5, 7), evaluated as hoisted rotation sums over ladder_groups(steps)."""
        for g in ladder_groups(steps):
            v = self.ev.rotate_sum(v, g)
        return v

    def e_slot(self, c):
        z = np.zeros(self.lay.M)
        z[c] = 1.0
        return z

    def mac_relin_rescale(self, pairs):
        """sum of tensors, one relinearisation, one rescale (Alg. 2, 8 bodies)."""
        ev = self.ev
        acc = None
        for a, b in pairs:
            t = ev.tensor(a, b)
            acc = t if acc is None else ev.add(acc, t)
        return ev.relin_rescale(acc)

    def replicate(self, v: Ct, c: int) -> Ct:
        """Alg. 1 for entry c: mask slot c, then a log2(M) rotate-and-add ladder."""
        ev = self.ev
        t = ev.mul_mask(v, self.e_slot(c))
        t = self.ladder(t, [1 << i for i in range(self.lay.logN - 1)])
        return t

    def replicate_all(self, v: Ct, m: int):
        """Alg. 1 for entries 0..m-1 of a vector that is zero beyond them,
        with one shared ladder.  Alg. 1's ladder sums the rotations of the
        masked slot by 0..M-1; here the steps P, 2P, ..., M/2 run first on v
        itself (slot s then holds the sum of v over the slots = s mod P, which
        is v_{s mod P}), the mask keeps the slots = c mod P, and the steps
        1, 2, ..., P/2 fill the rest: the same sum, with the first part done
        once for all m entries.  Same depth (one mask) and the same rotation
        keys as Alg. 1."""
        ev, M = self.ev, self.lay.M
        P = replicate_period(m, M)
        u = self.ladder(v, [P << i for i in range(int(math.log2(M // P)))])
        reps = []
        for c in range(m):
            mask = np.zeros(M)
            mask[c::P] = 1.0
            t = ev.mul_mask(u, mask)
            reps.append(self.ladder(t, [1 << i for i in range(int(math.log2(P)))]))
        return reps

    def cp_matvec(self, cols, v: Ct, m: int) -> Ct:
        """Alg. 2: sum_c A(c) * Replicate(v)(c), the m replicates of v (zero
        beyond its m entries in every use here) from one shared ladder."""
        reps = self.replicate_all(v, m)
        lv = reps[0].level
        return self.mac_relin_rescale([(self.ev.drop(cols[c], lv), reps[c]) for c in range(m)])

    def dotprod(self, a: Ct, b: Ct) -> Ct:
        """Alg. 5: C = A * B, then C += Rotate(C, 2^i) for i < log2(M)."""
        ev = self.ev
        t = ev.mult(a, b)
        t = self.ladder(t, [1 << i for i in range(self.lay.logN - 1)])
        return t

    def rp_matvec(self, rows, v: Ct, m: int) -> Ct:
        """Alg. 6: sum_c DotProd(A(c), v) * e_c, masks accumulated, one rescale."""
        ev = self.ev
        acc = None
        for c in range(m):
            dp = self.dotprod(ev.drop(rows[c], v.level), v)
            ql = float(ev.q[dp.level - 1])
            t = ev.mul_plain(dp, ev.encode(self.e_slot(c), ql, dp.level), ql)
            acc = t if acc is None else ev.add(acc, t)
        return ev.rescale(acc)

    def cp_rp_matvec(self, acols, rows, v: Ct, m: int) -> Ct:
        """A (R v): Alg. 2 over the DotProds of Alg. 6.  DotProd(R(c), v)
        (Alg. 5) ends with (R v)_c in every slot, which is what Replicate
        (Alg. 1) makes of entry c, so Alg. 6's masks e_c and Alg. 2's
        replicates cancel.  v is dropped two levels first: the result leaves at
        the level Alg. 6 then Alg. 2 would give."""
        ev = self.ev
        vv = ev.drop(v, v.level - 2)
        dps = [self.dotprod(ev.drop(rows[c], vv.level), vv) for c in range(m)]
        lv = dps[0].level
        return self.mac_relin_rescale([(ev.drop(acols[c], lv), dps[c]) for c in range(m)])

    def colsum(self, v: Ct) -> Ct:
        """Alg. 4: log2(nb) rotate-and-add steps; sums land at slots c*nb."""
        v = self.ladder(v, [1 << i for i in range(int(math.log2(self.lay.nb)))])
        return v

    def duplicate(self, v: Ct) -> Ct:
        """Alg. 7: doubling ladder v += Rotate(v, nb 2^i) over the M/nb blocks."""
        v = self.ladder(v, [self.lay.nb << i for i in range(int(math.log2(self.lay.B)))])
        return v

    def sigma7(self, x: Ct) -> Ct:
        """eq. sigma7 at depth 3: 0.5 + a1 x + a3 x^3 + a5 x^5 + a7 x^7 with
        a_k = c_k / 8^k; constants multiply at scale q_last (rescaled)."""
        ev = self.ev
        a1, a3, a5, a7 = SIGMA7_A
        x2 = ev.mult(x, x)
        x4 = ev.mult(x2, x2)
        b1 = ev.mul_const(x, a1)
        b3 = ev.mul_const(x, a3)
        b5 = ev.mul_const(x, a5)
        b7 = ev.mul_const(x, a7)
        t3 = ev.mult(b3, x2)
        t7a = ev.mult(b7, x2)
        t5 = ev.mult(ev.drop(b5, x4.level), x4)
        t7 = ev.mult(t7a, x4)
        lv = t7.level
        r = ev.add(ev.drop(b1, lv), ev.drop(t3, lv))
        r = ev.add(r, t5)
        r = ev.add(r, t7)
        return ev.add_const(r, 0.5)

    def add_plain_vec(self, ct: Ct, z) -> Ct:
        """add a public slot vector encoded at the ciphertext's scale."""
        ev = self.ev
        pt = ev.encode(z, ct.scale, ct.level)
        out = ct.c.copy()
        for i in range(ct.level):
            q = np.uint64(ev.q[i])
            s = out[0, i] + pt[i]
            out[0, i] = np.where(s >= q, s - q, s)
        return Ct(out, ct.scale)

    # --------------------------------------------------------- inputs
    def encrypt_vector(self, v, enc_id, level=None, scale=None):
        ev = self.ev
        level = ev.L if level is None else level
        scale = ev.delta if scale is None else scale
        z = np.zeros(self.lay.M, complex)
        z[: len(v)] = v
        return ev.encrypt(ev.encode(z, scale, level), self.enc_base + enc_id, scale)

    def encrypt_inputs(self, X, A, y):
        """X as CP, (X^T X)^-1 as CP, y, beta0 = Enc(0), X^T as REP (Alg. 11
        inputs and the walk-through after it)."""
        lay = self.lay
        n, d = X.shape
        self.X = [self.encrypt_vector(X[:, c], ENC_X + c) for c in range(d)]
        self.A = [self.encrypt_vector(A[:, c], ENC_A + c) for c in range(d)]
        self.y = self.encrypt_vector(y, ENC_Y)
        self.beta0 = self.encrypt_vector(np.zeros(1), ENC_BETA0)
        self.XtREP = []
        if self.factored:
            return  # X^T in REP only feeds the CCP matrix M
        for c in range(d):
            row = []
            for h in range(lay.H):
                z = np.zeros(lay.M)
                for b in range(lay.B):
                    col = h * lay.B + b
                    if col < n:
                        z[b * lay.nb:(b + 1) * lay.nb] = X[col, c]
                row.append(self.encrypt_vector(z, ENC_XTREP + c * 4096 + h))
            self.XtREP.append(row)

    def snp_batch_slots(self, S, i):
        """REP rows of batch i: list over samples j of M complex slot values."""
        lay = self.lay
        n, k = S.shape
        rows = []
        for j in range(n):
            z = np.zeros(lay.M, complex)
            for b in range(lay.B):
                c0 = i * lay.tau + 2 * b
                re = S[j, c0] if c0 < k else 0.0
                im = S[j, c0 + 1] if c0 + 1 < k else 0.0
                z[b * lay.nb:(b + 1) * lay.nb] = re + 1j * im
            rows.append(z)
        return rows

    def encrypt_snp_batch(self, S, i):
        lay = self.lay
        return [self.encrypt_vector(z, ENC_S + i * lay.n + j, level=BATCH_LEVEL)
                for j, z in enumerate(self.snp_batch_slots(S, i))]

    def snp_batch_ccp_slots(self, S, i):
        """CCP batch i (factored layout): slot b*nb + t = S[t, 2c] + i S[t, 2c+1]
        with c = i*B + b the complex column (section "Complex Space")."""
        lay = self.lay
        n, k = S.shape
        z = np.zeros(lay.M, complex)
        for b in range(lay.B):
            c0 = i * lay.tau + 2 * b
            re = S[:, c0] if c0 < k else np.zeros(n)
            im = S[:, c0 + 1] if c0 + 1 < k else np.zeros(n)
            z[b * lay.nb:b * lay.nb + n] = re + 1j * im
        return z

    def encrypt_snp_batch_ccp(self, S, i):
        return self.encrypt_vector(self.snp_batch_ccp_slots(S, i), ENC_SCCP + i,
                                   level=FACT_LEVEL)

    # --------------------------------------------------------- covariate phase
    def fit(self, kappa: int):
        """Alg. 9 then the preamble of Alg. 11: w, w^-1, z, z', M, Dup(M_j)."""
        ev, lay = self.ev, self.lay
        d, n = len(self.X), lay.n
        # Alg. 9
        beta = self.beta0
        p = ymp = None
        for _ in range(kappa):
            xb = self.cp_matvec(self.X, beta, d)
            p = self.sigma7(xb)
            ymp = ev.sub(ev.drop(self.y, p.level), p)
            ag = self.cp_rp_matvec(self.A, self.X, ymp, d)  # A g, g = X^T (y - p)
            ag4 = ev.mul_int(ag, 4)
            beta = ev.sub(ev.drop(beta, ag4.level), ag4)
        self.beta = beta
        # w = p(1 - p), masked copy for the duplicated weights
        w = ev.mult(p, ev.add_const(ev.negate(p), 1.0))
        mask_n = np.zeros(lay.M)
        mask_n[:n] = 1.0
        w_m = ev.mul_mask(w, mask_n)
        # Alg. 10 (first step uses the integer guess 3: no rescale)
        t = ev.mul_int(w, 3)
        u = ev.add_const(ev.negate(t), 2.0)
        g = ev.mul_int(u, 3)
        for _ in range(2):
            t = ev.mult(ev.drop(w, g.level), g)
            u = ev.add_const(ev.negate(t), 2.0)
            g = ev.mult(ev.drop(g, u.level), u)
        winv = g
        # eq. z
        xb = self.cp_matvec(self.X, beta, d)
        lv = min(winv.level, ymp.level)
        r = ev.mult(ev.drop(winv, lv), ev.drop(ymp, lv))
        lv = min(xb.level, r.level)
        z = ev.add(ev.drop(xb, lv), ev.drop(r, lv))
        # eq. zprime, second form: z' = z - X (A (X^T z))
        axtz = self.cp_rp_matvec(self.A, self.X, z, d)
        xaxtz = self.cp_matvec(self.X, axtz, d)
        zp = ev.sub(ev.drop(z, xaxtz.level), xaxtz)
        wzp = ev.mult(ev.drop(w_m, zp.level), zp)
        self.z, self.zp, self.w_m, self.wzp = z, zp, w_m, wzp
        # X A via Alg. 3 (CP-MatMult) from X and A dropped to M_LEVEL limbs,
        # each column duplicated into every block (Alg. 7)
        XA = [self.cp_matvec(self.X, ev.drop(self.A[r], M_LEVEL), d) for r in range(d)]
        dupXA = [self.duplicate(XA[r]) for r in range(d)]
        if self.factored:
            # second form of eq. Sprime: keep Dup((XA)_c) and Dup(X_c)
            self.DupB = dupXA
            self.DupX = [self.duplicate(ev.drop(self.X[c], FACT_LEVEL)) for c in range(d)]
            self.make_dup_state()
            return
        # eq. M: M = I - X A X^T via Alg. 8 (CP-REP) on the duplicated columns
        self.Mct = []
        for h in range(lay.H):
            lv = dupXA[0].level
            acc = self.mac_relin_rescale([(dupXA[r], ev.drop(self.XtREP[r][h], lv))
                                          for r in range(d)])
            eye = np.zeros(lay.M)
            for b in range(lay.B):
                col = h * lay.B + b
                if col < n:
                    eye[b * lay.nb + col] = 1.0
            self.Mct.append(self.add_plain_vec(ev.negate(acc), eye))
        self.make_dup_state()

    def make_dup_state(self):
        """Dup(M_j) for every column j (mask its block, Alg. 7), Dup(w), Dup(w z')."""
        ev, lay = self.ev, self.lay
        lb = BATCH_LEVEL
        if self.wzp.level < lb - 1:
            raise ValueError("depth exhausted before the SNP batches")
        self.DupM = []
        src = [] if self.factored else [ev.drop(m, lb + 1) for m in self.Mct]
        for j in range(0 if self.factored else lay.n):
            h, b = divmod(j, lay.B)
            mask = np.zeros(lay.M)
            mask[b * lay.nb:b * lay.nb + lay.n] = 1.0
            self.DupM.append(self.duplicate(ev.mul_mask(src[h], mask)))
        self.DupW = self.duplicate(ev.drop(self.w_m, lb - 1))
        self.DupWZ = self.duplicate(ev.drop(self.wzp, lb - 1))

    def load_split_state(self, M, w, wzp):
        """Split mode (small rings without the fit's depth): the client
        encrypts Dup(M_j), Dup(w), Dup(w z') computed in plaintext."""
        lay = self.lay
        n = lay.n
        lb = BATCH_LEVEL

        def dup(v):
            z = np.zeros(lay.M)
            for b in range(lay.B):
                z[b * lay.nb:b * lay.nb + n] = v
            return z

        self.DupM = [self.encrypt_vector(dup(M[:, j]), ENC_DUPM + j, level=lb)
                     for j in range(n)]
        self.DupW = self.encrypt_vector(dup(w), ENC_DUPW, level=lb - 1)
        self.DupWZ = self.encrypt_vector(dup(wzp), ENC_DUPWZ, level=lb - 1)

    # --------------------------------------------------------- per batch
    def snp_batch(self, Srow):
        """Alg. 11 loop body for one batch of the M-CCP layout:
        S' = sum_j Dup(M_j) S_ij (Alg. 8), then the common body."""
        Sp = self.mac_relin_rescale([(self.DupM[j], Srow[j]) for j in range(len(Srow))])
        return self.batch_body(Sp)

    def factored_sprime(self, Sct: Ct) -> Ct:
        """Second form of eq. Sprime for one CCP batch at FACT_LEVEL:
          U_c = Dup(X_c) S                       (product, one level)
          T_c = colSum(U_c) masked to the block heads b*nb   (Alg. 5, one level)
          R_c = T_c broadcast down its block: R += Rotate(R, -2^i), i < log2(nb)
          S'  = S - sum_c Dup((XA)_c) R_c        (tensor sum, relin, rescale)
        so slot b*nb + t of S' is S[t, .] - sum_c (XA)[t, c] (X^T S)[c, .]."""
        ev, lay = self.ev, self.lay
        d = len(self.DupX)
        heads = np.zeros(lay.M)
        heads[::lay.nb] = 1.0
        R = []
        for c in range(d):
            u = self.colsum(ev.mult(self.DupX[c], Sct))
            r = ev.mul_mask(u, heads)
            r = self.ladder(r, [-(1 << i) for i in range(int(math.log2(lay.nb)))])
            R.append(r)
        lv = R[0].level
        P = self.mac_relin_rescale([(ev.drop(self.DupB[c], lv), R[c]) for c in range(d)])
        return ev.sub(ev.drop(Sct, P.level), P)

    def snp_batch_factored(self, Sct: Ct):
        """Alg. 11 loop body for one CCP batch of the factored layout."""
        return self.batch_body(self.factored_sprime(Sct))

    def batch_body(self, Sp: Ct):
        """numerator = colSum(Dup(w z') S'), WSS, WSC, denEven/denOdd (the 1/2
        kept as scale metadata), colSum of each."""
        ev = self.ev
        lb = BATCH_LEVEL
        num = self.colsum(ev.mult(self.DupWZ, Sp))
        ws = ev.mult(self.DupW, Sp)
        s1 = ev.drop(Sp, lb - 2)
        wss = ev.mult(ws, s1)
        wsc = ev.mult(ws, ev.conj(s1))
        den_e = ev.add(wsc, wss)
        den_e.scale *= 2.0
        den_o = ev.sub(wsc, wss)
        den_o.scale *= 2.0
        return num, self.colsum(den_e), self.colsum(den_o)

    def extract(self, num: Ct, den_e: Ct, den_o: Ct, batch: int):
        """Decrypt and split the packed pairs: slot b*nb of num gives SNP 2b
        (real part) and 2b+1 (imaginary part); denEven / denOdd real parts."""
        lay = self.lay
        zn = self.ev.decrypt_decode(num)
        ze = self.ev.decrypt_decode(den_e)
        zo = self.ev.decrypt_decode(den_o)
        nums, dens = [], []
        for b in range(lay.B):
            s = b * lay.nb
            nums += [zn[s].real, zn[s].imag]
            dens += [ze[s].real, zo[s].real]
        lo = batch * lay.tau
        cnt = min(lay.tau, lay.k - lo)
        return np.array(nums[:cnt]), np.array(dens[:cnt])
