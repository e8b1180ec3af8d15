"""Level tracer for the oracle circuit: test and benchmark infrastructure.

Runs the oracle's GWAS circuit (Alg. 9 and Alg. 11 as written in
oracle/circuit.py) on ciphertexts of ONE coefficient per limb, so that only
the bookkeeping is real: the level of every ciphertext, its scale (product of
the operands' scales, divided by the dropped prime on each rescale, sect. 2.2)
and the number of key switches issued at each level (one per
relinearisation or conjugation, and one per hoisted group of ladder rotations,
which shares one ModUp and one ModDown).  No
ciphertext arithmetic is meaningful here; the tracer exists to count the
work of a job at full size in a fraction of a second.

Only tests/ and the benchmark's CPU arms use this module.
"""
from __future__ import annotations

import numpy as np

from .ckks import Ct, OracleCKKS


class LevelTrace(OracleCKKS):
    """OracleCKKS with every N-sized primitive replaced by a shape-only stand-in."""

    def __init__(self, *args, **kw):
        super().__init__(*args, **kw)
        self.ks_hist = np.zeros(65, np.int64)

    def _z(self, npoly, level):
        return np.zeros((npoly, level, 1), np.uint64)

    def keygen(self, galois=()):
        self.keys[0] = None

    def add_galois_key(self, g: int):
        self.keys[int(g)] = None

    def encode(self, z, scale: float, level: int) -> np.ndarray:
        return np.zeros((level, 1), np.uint64)

    def encrypt(self, pt: np.ndarray, enc_id: int, scale: float) -> Ct:
        return Ct(self._z(2, pt.shape[0]), float(scale))

    def decrypt_decode(self, ct: Ct) -> np.ndarray:
        return np.zeros(self.M, complex)

    def mul_plain(self, a: Ct, pt: np.ndarray, pt_scale: float) -> Ct:
        return Ct(np.zeros_like(a.c), a.scale * pt_scale)

    def tensor(self, a: Ct, b: Ct) -> Ct:
        if a.level != b.level:
            raise ValueError("level mismatch")
        return Ct(self._z(3, a.level), a.scale * b.scale)

    def keyswitch(self, x: np.ndarray, key_id: int) -> np.ndarray:
        self.ks_hist[x.shape[0]] += 1
        return np.zeros((2, x.shape[0], 1), np.uint64)

    def rescale(self, a: Ct) -> Ct:
        l = a.level
        if l < 2:
            raise ValueError("no level left to rescale")
        return Ct(self._z(a.c.shape[0], l - 1), a.scale / float(self.q[l - 1]))

    def automorphism(self, a: Ct, g: int) -> Ct:
        return Ct(np.zeros_like(a.c), a.scale)

    def relin_rescale(self, t: Ct) -> Ct:
        self.ks_hist[t.level] += 1
        l = t.level
        if l < 2:
            raise ValueError("no level left to rescale")
        return Ct(self._z(2, l - 1), t.scale / float(self.q[l - 1]))

    def rotate_sum(self, a: Ct, rs) -> Ct:
        self.ks_hist[a.level] += 1
        return Ct(np.zeros_like(a.c), a.scale)


def job_ks_histogram(W, kappa: int = 1, factored: bool = False):
    """Key switches per level of one job of workload W (dict with logN, L,
    q0_bits, scale_bits, K, sp_bits, dnum, n, d, k): the covariate phase once,
    then the SNP-batch body once per batch (every batch issues the same
    switches at the same levels), for the M-CCP or the factored layout.
    Returns (histogram[65], fit_part, batch_part)."""
    from .circuit import BATCH_LEVEL, FACT_LEVEL, Circuit, Layout

    ev = LevelTrace(logN=W["logN"], L=W["L"], q0_bits=W["q0_bits"],
                    scale_bits=W["scale_bits"], K=W["K"], sp_bits=W["sp_bits"],
                    dnum=W["dnum"], seed=0)
    lay = Layout(logN=W["logN"], n=W["n"], d=W["d"], k=W["k"])
    lay.check()
    circ = Circuit(ev, lay, factored=factored)
    n, d = W["n"], W["d"]
    X = np.zeros((n, d))
    X[:, 0] = 1.0
    circ.encrypt_inputs(X, np.eye(d), np.zeros(n))
    circ.fit(kappa)
    fit = ev.ks_hist.copy()
    if factored:
        circ.snp_batch_factored(ev.encrypt(np.zeros((FACT_LEVEL, 1), np.uint64), 0, ev.delta))
    else:
        Srow = [ev.encrypt(np.zeros((BATCH_LEVEL, 1), np.uint64), 0, ev.delta)
                for _ in range(n)]
        circ.snp_batch(Srow)
    batch = ev.ks_hist - fit
    return fit + batch * lay.batches, fit, batch
