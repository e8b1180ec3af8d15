"""Thin Python binding of the gwhe C ABI (include/gwhe.h).

Argument marshalling only: every step of the encrypted path runs in the CUDA
library.  Host arrays are numpy; device buffers may be torch CUDA tensors (or
raw device pointers) where the ABI accepts device memory.  If the compiled
library is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgwhe.so")

GWHE_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ELEVEL", -4: "ESCALE", -5: "ENOKEY",
          -6: "ETIMEOUT", -7: "ECUDA"}

_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_vp = ctypes.c_void_p
_i = ctypes.c_int
_l = ctypes.c_long
_d = ctypes.c_double
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t


class Params(ctypes.Structure):
    _fields_ = [("logN", _i), ("L", _i), ("q0_bits", _i), ("scale_bits", _i), ("K", _i),
                ("sp_bits", _i), ("dnum", _i)]


class GwheError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_SIGS = {
    "gwhe_gen_primes": [ctypes.POINTER(Params), _u64p, _u64p],
    "gwhe_fft_twiddles": [_i, _i, _f64p, _f64p],
    "gwhe_layout": [_i, _i, _l, ctypes.POINTER(_l)],
    "gwhe_ctx_create": [ctypes.POINTER(Params), _u64, _vp, ctypes.POINTER(_vp)],
    "gwhe_ctx_destroy": [_vp],
    "gwhe_ctx_moduli": [_vp, _u64p],
    "gwhe_sync": [_vp],
    "gwhe_keygen": [_vp, _i32p, _sz, _i],
    "gwhe_export_secret": [_vp, _i64p],
    "gwhe_export_pk": [_vp, _u64p],
    "gwhe_export_ksk": [_vp, _u32, _i, _u64p],
    "gwhe_ks_special": [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "gwhe_ct_create": [_vp, _i, _i, ctypes.POINTER(_vp)],
    "gwhe_ct_destroy": [_vp],
    "gwhe_ct_info": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_d)],
    "gwhe_ct_import": [_vp, _u64p, _i, _i, _d],
    "gwhe_ct_export": [_vp, _u64p],
    "gwhe_encode": [_vp, _f64p, _d, _i64p],
    "gwhe_encode_batch": [_vp, _vp, _i, _d, _vp],
    "gwhe_encrypt": [_vp, _f64p, _d, _i, _u64, _vp],
    "gwhe_encrypt_coeffs": [_vp, _i64p, _d, _i, _u64, _vp],
    "gwhe_decrypt": [_vp, _vp, _u64p],
    "gwhe_decrypt_decode": [_vp, _vp, _f64p],
    "gwhe_add": [_vp, _vp, _vp, _vp],
    "gwhe_sub": [_vp, _vp, _vp, _vp],
    "gwhe_negate": [_vp, _vp, _vp],
    "gwhe_add_const": [_vp, _vp, _d],
    "gwhe_mul_int": [_vp, _vp, ctypes.c_int64],
    "gwhe_mul_const": [_vp, _vp, _d],
    "gwhe_mul_mask": [_vp, _vp, _f64p, _vp],
    "gwhe_tensor": [_vp, _vp, _vp, _vp],
    "gwhe_tensor_sum": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _sz, _vp],
    "gwhe_relin": [_vp, _vp, _vp],
    "gwhe_rescale": [_vp, _vp],
    "gwhe_mult": [_vp, _vp, _vp, _vp],
    "gwhe_rotate": [_vp, _vp, _i, _vp],
    "gwhe_conjugate": [_vp, _vp, _vp],
    "gwhe_drop": [_vp, _i],
    "gwhe_keyswitch": [_vp, _u64p, _i, _u32, _u64p],
    "gwhe_keyswitch_noalloc": [_vp, _vp, _i, _u32, _vp],
    "gwhe_ntt_batch": [_vp, _vp, _i, _i, _i],
    "gwhe_job_create": [_vp, _i, _i, _l, ctypes.POINTER(_vp)],
    "gwhe_job_create_ex": [_vp, _i, _i, _l, _i, ctypes.POINTER(_vp)],
    "gwhe_job_info": [_vp, ctypes.POINTER(_l)],
    "gwhe_autotune": [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i)],
    "gwhe_set_ntt_variant": [_vp, _i],
    "gwhe_job_set_nonce": [_vp, _u32],
    "gwhe_job_set_host_state": [_vp, _i],
    "gwhe_job_release_results": [_vp],
    "gwhe_ctx_create_child": [_vp, _vp, ctypes.POINTER(_vp)],
    "gwhe_server_create": [_vp, _i, ctypes.c_uint64, _i, ctypes.POINTER(_vp)],
    "gwhe_server_create_ex": [_vp, _i, ctypes.c_uint64, _i, _i, ctypes.POINTER(_vp)],
    "gwhe_server_submit": [_vp, _i, _i, _l, _i, _i, _u32, _f64p, _f64p, _f64p, _f64p,
                           ctypes.POINTER(_l)],
    "gwhe_server_wait": [_vp, _l, _f64p, _f64p, _f64p],
    "gwhe_server_submit_borrowed": [_vp, _i, _i, _l, _i, _i, _u32, _f64p, _f64p, _f64p, _f64p,
                                    ctypes.POINTER(_l)],
    "gwhe_server_stats": [_vp, ctypes.POINTER(_l)],
    "gwhe_server_destroy": [_vp],
    "gwhe_rotate_sum": [_vp, _vp, ctypes.POINTER(ctypes.c_int32), _i, _vp],
    "gwhe_rotate_sum_batch": [_vp, ctypes.POINTER(_vp), _i, ctypes.POINTER(ctypes.c_int32), _i,
                              ctypes.POINTER(_vp)],
    "gwhe_probe_butterflies": [_vp, _i, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)],
    "gwhe_job_rotation_steps": [_vp, ctypes.POINTER(ctypes.c_int32), _i, ctypes.POINTER(_i)],
    "gwhe_job_destroy": [_vp],
    "gwhe_encrypt_inputs": [_vp, _vp, _vp, _vp],
    "gwhe_fit_covariates": [_vp, _i],
    "gwhe_set_fit_state": [_vp, _vp, _vp, _vp],
    "gwhe_snp_stats": [_vp, _vp, _l, _l, _i],
    "gwhe_decrypt_results": [_vp, _f64p, _f64p],
    "gwhe_job_ct": [_vp, _i, _l, ctypes.POINTER(_vp)],
    "gwhe_prof_enable": [_vp, _i],
    "gwhe_ks_histogram": [_vp, np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS"), _i],
    "gwhe_prof_read": [_vp, _f64p, _f64p, np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")],
    "gwhe_ctx_device": [_vp, ctypes.POINTER(_i)],
    "gwhe_ctx_set_stream": [_vp, _vp],
    "gwhe_rotate_batch": [_vp, ctypes.POINTER(_vp), _i, ctypes.c_int32, _i, ctypes.POINTER(_vp)],
    "gwhe_job_state_size": [_vp, ctypes.POINTER(_sz)],
    "gwhe_job_export_state": [_vp, _vp, _sz],
    "gwhe_job_import_state": [_vp, _vp, _sz],
    "gwhe_encrypt_covariates": [_vp, _vp, _vp],
    "gwhe_encrypt_phenotype": [_vp, _vp],
    "gwhe_encrypt_snps": [_vp, _vp, _l, _l],
    "gwhe_device_ok": [_i, _i],
    "gwhe_mem_info": [_vp, np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")],
}

PROF_CLASSES = ("ntt", "ks_inner", "tensor_mac", "baseconv", "elementwise", "encode", "sample")

_LIB = None


def lib():
    """The loaded libgwhe.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libgwhe.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _i
        L.gwhe_last_error.argtypes = [_vp]
        L.gwhe_last_error.restype = ctypes.c_char_p
        L.gwhe_job_keyswitches.argtypes = [_vp]
        L.gwhe_job_keyswitches.restype = _l
        L.gwhe_launch_count.argtypes = [_vp]
        L.gwhe_launch_count.restype = _l
        L.gwhe_job_footprint.argtypes = [_vp, _i, _i, _l, _i, _i]
        L.gwhe_job_footprint.restype = _l
        _LIB = L
    return _LIB


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(list(_SIGS) + ["gwhe_last_error", "gwhe_job_keyswitches", "gwhe_launch_count",
                                 "gwhe_job_footprint"])


def _check(rc, ctx=None):
    if rc != GWHE_OK:
        msg = ""
        if ctx is not None:
            m = lib().gwhe_last_error(ctx)
            msg = m.decode() if m else ""
        raise GwheError(rc, msg)


def _ptr(x):
    """device pointer of a torch tensor / integer, or a host array's address."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(x))


def _slots(z, M):
    z = np.asarray(z, dtype=complex)
    full = np.zeros(M, complex)
    full[: z.shape[0]] = z
    return np.ascontiguousarray(np.stack([full.real, full.imag], axis=1).reshape(-1))


# ----------------------------------------------------------------- host only
def params(logN, L, q0_bits=60, scale_bits=40, K=1, sp_bits=60, dnum=None):
    return Params(logN, L, q0_bits, scale_bits, K, sp_bits, L if dnum is None else dnum)


def gen_primes(prm: Params):
    q = np.zeros(prm.L, np.uint64)
    p = np.zeros(prm.K, np.uint64)
    _check(lib().gwhe_gen_primes(ctypes.byref(prm), q, p))
    return q, p


def fft_twiddles(logN, sign):
    M = 1 << (logN - 1)
    W = np.zeros(M, np.float64)  # M/2 complex
    T = np.zeros(2 * M, np.float64)
    _check(lib().gwhe_fft_twiddles(logN, sign, W, T))
    return W, T


def layout(logN, n, k):
    out = (_l * 5)()
    _check(lib().gwhe_layout(logN, n, k, out))
    return dict(zip(("nb", "B", "tau", "batches", "H"), list(out)))


# ----------------------------------------------------------------- objects
class Ciphertext:
    def __init__(self, ctx: "Context", handle):
        self.ctx = ctx
        self.h = handle
        ctx._children.add(self)

    def close(self):
        # a handle must not outlive its context (the context closes it first)
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            lib().gwhe_ct_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        npoly, l, sc = _i(), _i(), _d()
        _check(lib().gwhe_ct_info(self.h, ctypes.byref(npoly), ctypes.byref(l), ctypes.byref(sc)))
        return npoly.value, l.value, sc.value

    @property
    def level(self):
        return self.info()[1]

    @property
    def scale(self):
        return self.info()[2]

    def export(self):
        npoly, l, _ = self.info()
        out = np.zeros((npoly, l, self.ctx.N), np.uint64)
        _check(lib().gwhe_ct_export(self.h, out), self.ctx.h)
        return out

    def import_(self, coeffs, scale):
        coeffs = np.ascontiguousarray(coeffs, np.uint64)
        _check(lib().gwhe_ct_import(self.h, coeffs, coeffs.shape[0], coeffs.shape[1], scale),
               self.ctx.h)

    def drop(self, l):
        _check(lib().gwhe_drop(self.h, l), self.ctx.h)
        return self


class Context:
    def __init__(self, logN, L, q0_bits=60, scale_bits=40, K=1, sp_bits=60, dnum=None, seed=0,
                 stream=None):
        self.prm = params(logN, L, q0_bits, scale_bits, K, sp_bits, dnum)
        self.logN, self.L, self.K = logN, L, K
        self.N = 1 << logN
        self.M = self.N // 2
        self.dnum = self.prm.dnum
        self.delta = float(2 ** scale_bits)
        self._children = weakref.WeakSet()
        h = _vp()
        _check(lib().gwhe_ctx_create(ctypes.byref(self.prm), seed, _ptr(stream), ctypes.byref(h)))
        self.h = h
        mods = np.zeros(L + K, np.uint64)
        _check(lib().gwhe_ctx_moduli(self.h, mods))
        self.mods = mods
        self.q = [int(x) for x in mods[:L]]
        self.p = [int(x) for x in mods[L:]]

    def close(self):
        if getattr(self, "h", None):
            # servers first (their workers use the context), then jobs (they
            # own ciphertexts), then ciphertext handles
            kids = sorted(list(self._children),
                          key=lambda x: 0 if isinstance(x, Server) else 1 if isinstance(x, Job) else 2)
            for kid in kids:
                kid.close()
            lib().gwhe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        _check(rc, self.h)

    def sync(self):
        self._c(lib().gwhe_sync(self.h))

    # keys
    def keygen(self, rot_steps=(), conj=False):
        steps = np.ascontiguousarray(np.array(list(rot_steps), dtype=np.int32).reshape(-1))
        self._c(lib().gwhe_keygen(self.h, steps, len(steps), 1 if conj else 0))

    def export_secret(self):
        s = np.zeros(self.N, np.int64)
        self._c(lib().gwhe_export_secret(self.h, s))
        return s

    def export_pk(self):
        pk = np.zeros((2, self.L, self.N), np.uint64)
        self._c(lib().gwhe_export_pk(self.h, pk))
        return pk

    def ks_special(self, l):
        """(special primes a switch at level l uses, highest level of that count)."""
        k, lmax = _i(0), _i(0)
        self._c(lib().gwhe_ks_special(self.h, l, ctypes.byref(k), ctypes.byref(lmax)))
        return k.value, lmax.value

    def export_ksk(self, key_id):
        """{k: family [ceil(lmax/alpha)][2][lmax + k][N]} in the coefficient domain."""
        alpha = -(-self.L // self.dnum)
        fams = {}
        for l in range(1, self.L + 1):
            k, lmax = self.ks_special(l)
            fams[k] = lmax
        out = {}
        for k, lmax in fams.items():
            a = np.zeros((-(-lmax // alpha), 2, lmax + k, self.N), np.uint64)
            self._c(lib().gwhe_export_ksk(self.h, key_id, k, a))
            out[k] = a
        return out

    # ciphertexts
    def ct(self, npoly=2, cap=None):
        h = _vp()
        self._c(lib().gwhe_ct_create(self.h, npoly, self.L if cap is None else cap,
                                     ctypes.byref(h)))
        return Ciphertext(self, h)

    def import_ct(self, coeffs, scale):
        coeffs = np.ascontiguousarray(coeffs, np.uint64)
        c = self.ct(coeffs.shape[0], coeffs.shape[1])
        c.import_(coeffs, scale)
        return c

    def encode(self, z, scale):
        out = np.zeros(self.N, np.int64)
        self._c(lib().gwhe_encode(self.h, _slots(z, self.M), scale, out))
        return out

    def encode_batch(self, z_dev, count, scale, out_dev):
        """device-side encode of count x M complex slots (torch float64 [count, M, 2])."""
        self._c(lib().gwhe_encode_batch(self.h, _ptr(z_dev), count, scale, _ptr(out_dev)))

    def encrypt(self, z, scale, level, enc_id):
        c = self.ct(2, level)
        self._c(lib().gwhe_encrypt(self.h, _slots(z, self.M), scale, level, enc_id, c.h))
        return c

    def encrypt_coeffs(self, m, scale, level, enc_id):
        c = self.ct(2, level)
        self._c(lib().gwhe_encrypt_coeffs(self.h, np.ascontiguousarray(m, np.int64), scale,
                                          level, enc_id, c.h))
        return c

    def decrypt(self, ct):
        out = np.zeros((ct.level, self.N), np.uint64)
        self._c(lib().gwhe_decrypt(self.h, ct.h, out))
        return out

    def decrypt_decode(self, ct):
        out = np.zeros(2 * self.M, np.float64)
        self._c(lib().gwhe_decrypt_decode(self.h, ct.h, out))
        return out[0::2] + 1j * out[1::2]

    # arithmetic (results are new ciphertexts unless noted)
    def _out(self, a, npoly=2):
        return self.ct(npoly, a.level)

    def add(self, a, b):
        o = self._out(a)
        self._c(lib().gwhe_add(self.h, a.h, b.h, o.h))
        return o

    def sub(self, a, b):
        o = self._out(a)
        self._c(lib().gwhe_sub(self.h, a.h, b.h, o.h))
        return o

    def negate(self, a):
        o = self._out(a)
        self._c(lib().gwhe_negate(self.h, a.h, o.h))
        return o

    def add_const(self, a, v):  # in place
        self._c(lib().gwhe_add_const(self.h, a.h, v))
        return a

    def mul_int(self, a, k):  # in place
        self._c(lib().gwhe_mul_int(self.h, a.h, k))
        return a

    def mul_const(self, a, v):  # in place
        self._c(lib().gwhe_mul_const(self.h, a.h, v))
        return a

    def mul_mask(self, a, z):
        o = self._out(a)
        self._c(lib().gwhe_mul_mask(self.h, a.h, _slots(z, self.M), o.h))
        return o

    def tensor(self, a, b):
        o = self._out(a, 3)
        self._c(lib().gwhe_tensor(self.h, a.h, b.h, o.h))
        return o

    def tensor_sum(self, pairs):
        a = (_vp * len(pairs))(*[p[0].h for p in pairs])
        b = (_vp * len(pairs))(*[p[1].h for p in pairs])
        o = self._out(pairs[0][0], 3)
        self._c(lib().gwhe_tensor_sum(self.h, a, b, len(pairs), o.h))
        return o

    def relin(self, t3):
        o = self._out(t3)
        self._c(lib().gwhe_relin(self.h, t3.h, o.h))
        return o

    def rescale(self, a):  # in place
        self._c(lib().gwhe_rescale(self.h, a.h))
        return a

    def mult(self, a, b):
        o = self._out(a)
        self._c(lib().gwhe_mult(self.h, a.h, b.h, o.h))
        return o

    def rotate(self, a, r):
        o = self._out(a)
        self._c(lib().gwhe_rotate(self.h, a.h, r, o.h))
        return o

    def conj(self, a):
        o = self._out(a)
        self._c(lib().gwhe_conjugate(self.h, a.h, o.h))
        return o

    def rotate_sum_batch(self, cts, steps, outs=None):
        """[a + sum_r Rotate(a, r) for a in cts] as one set (shared level/scale),
        1 to 15 rotations."""
        outs = outs or [self._out(a) for a in cts]
        arr = (ctypes.c_int32 * len(steps))(*steps)
        ins = (_vp * len(cts))(*[a.h for a in cts])
        ous = (_vp * len(outs))(*[o.h for o in outs])
        self._c(lib().gwhe_rotate_sum_batch(self.h, ins, len(cts), arr, len(steps), ous))
        return outs

    def rotate_batch(self, cts, step, rescale=False, outs=None):
        """[Rotate(a, step) for a in cts] as one set (shared level/scale),
        each then rescaled if asked."""
        outs = outs or [self._out(a) for a in cts]
        ins = (_vp * len(cts))(*[a.h for a in cts])
        ous = (_vp * len(outs))(*[o.h for o in outs])
        self._c(lib().gwhe_rotate_batch(self.h, ins, len(cts), step, 1 if rescale else 0, ous))
        return outs

    def rotate_sum(self, a, steps):
        """a + sum_r Rotate(a, r) over 1 to 15 rotations, key switches hoisted."""
        o = self._out(a)
        arr = (ctypes.c_int32 * len(steps))(*steps)
        self._c(lib().gwhe_rotate_sum(self.h, a.h, arr, len(steps), o.h))
        return o

    def keyswitch(self, x, key_id):
        x = np.ascontiguousarray(x, np.uint64)
        l = x.shape[0]
        out = np.zeros((2, l, self.N), np.uint64)
        self._c(lib().gwhe_keyswitch(self.h, x, l, key_id, out))
        return out

    def autotune(self, rows=512):
        """time the compiled shapes of the N = 2^16 transform, keep the fastest;
        returns (chosen shape, ms per shape)."""
        ms = (ctypes.c_double * NTT_SHAPES)()
        ch = _i(0)
        self._c(lib().gwhe_autotune(self.h, rows, ms, ctypes.byref(ch)))
        return ch.value, [round(float(x), 4) for x in ms]

    def set_ntt_variant(self, v):
        self._c(lib().gwhe_set_ntt_variant(self.h, v))

    def probe_butterflies(self, rounds=2048):
        """butterflies/s of the NTT butterfly on register-resident data (the
        arithmetic ceiling of a butterfly kernel) and the launch's ms."""
        r, ms = ctypes.c_double(), ctypes.c_double()
        self._c(lib().gwhe_probe_butterflies(self.h, rounds, ctypes.byref(r), ctypes.byref(ms)))
        return r.value, ms.value

    def ks_histogram(self):
        out = np.zeros(65, np.int64)
        self._c(lib().gwhe_ks_histogram(self.h, out, 65))
        return out

    def launches(self):
        return lib().gwhe_launch_count(self.h)

    def prof_enable(self, on=True):
        self._c(lib().gwhe_prof_enable(self.h, 1 if on else 0))

    def prof_read(self):
        """{class: (ms, algorithmic bytes, launch groups)} since the last read."""
        ms = np.zeros(len(PROF_CLASSES))
        by = np.zeros(len(PROF_CLASSES))
        n = np.zeros(len(PROF_CLASSES), np.int64)
        self._c(lib().gwhe_prof_read(self.h, ms, by, n))
        return {k: (float(ms[i]), float(by[i]), int(n[i])) for i, k in enumerate(PROF_CLASSES)}

    def set_stream(self, stream):
        """later calls run on `stream` (torch stream, raw handle or None),
        ordered after the work already queued on the current one"""
        h = getattr(stream, "cuda_stream", stream)
        self._c(lib().gwhe_ctx_set_stream(self.h, _ptr(h)))

    def device(self):
        d = _i(0)
        self._c(lib().gwhe_ctx_device(self.h, ctypes.byref(d)))
        return d.value

    def mem_info(self):
        """{pool_used, pool_reserved, free, total} bytes of the context's device"""
        out = np.zeros(4, np.uint64)
        self._c(lib().gwhe_mem_info(self.h, out))
        return dict(zip(("pool_used", "pool_reserved", "free", "total"), (int(v) for v in out)))

    def keyswitch_noalloc(self, x_dev, l, key_id, out_dev):
        """Key switch of device rows x_dev[l][N] (NTT domain) into out_dev
        [2][l][N] using the library's static scratch (no device allocation)."""
        self._c(lib().gwhe_keyswitch_noalloc(self.h, _ptr(x_dev), l, key_id, _ptr(out_dev)))

    def ntt_batch(self, dev, npoly, nlimbs, inverse=False):
        """in-place NTT of device rows dev[npoly][nlimbs][N] (torch tensor or pointer)."""
        self._c(lib().gwhe_ntt_batch(self.h, _ptr(dev), npoly, nlimbs, 1 if inverse else 0))


LAYOUTS = {"auto": 0, "mccp": 1, "factored": 2}
NTT_SHAPES = 7  # compiled shapes of the N = 2^16 transform (gwhe_autotune)


class Job:
    """An encrypted semi-parallel GWAS job (Alg. 11) on a context.  layout:
    "mccp" (S' = M S, M as a CCP matrix, S in REP rows), "factored"
    (S' = S - XA(X^T S), S in CCP) or "auto" (factored on rings deep enough
    for the fit, M-CCP otherwise)."""

    def __init__(self, ctx: Context, n, d, k, layout="auto"):
        self.ctx = ctx
        self.n, self.d, self.k = n, d, k
        h = _vp()
        ctx._c(lib().gwhe_job_create_ex(ctx.h, n, d, k, LAYOUTS[layout], ctypes.byref(h)))
        self.h = h
        info = (_l * 8)()
        ctx._c(lib().gwhe_job_info(h, info))
        keys = ["M", "nb", "B", "tau", "H", "batches", "layout", "batch_limbs"]
        self.layout = {kk: int(v) for kk, v in zip(keys, info)}
        self.factored = self.layout["layout"] == LAYOUTS["factored"]
        ctx._children.add(self)

    def rotation_steps(self):
        """rotation steps whose Galois keys the job needs (with conjugation)."""
        cnt = _i(0)
        self.ctx._c(lib().gwhe_job_rotation_steps(self.h, None, 0, ctypes.byref(cnt)))
        out = (ctypes.c_int32 * cnt.value)()
        self.ctx._c(lib().gwhe_job_rotation_steps(self.h, out, cnt.value, ctypes.byref(cnt)))
        return [int(v) for v in out]

    def close(self):
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            # views taken from this job become invalid with it
            for kid in list(self.ctx._children):
                if isinstance(kid, Ciphertext) and getattr(kid, "job", None) is self:
                    kid.close()
            lib().gwhe_job_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _arr(x):
        if hasattr(x, "data_ptr"):
            return x, _ptr(x)
        a = np.ascontiguousarray(x, np.float64)
        return a, _ptr(a)

    def encrypt_inputs(self, X, XtX_inv, y):
        X, px = self._arr(X)
        A, pa = self._arr(XtX_inv)
        y, py = self._arr(y)
        self.ctx._c(lib().gwhe_encrypt_inputs(self.h, px, pa, py))

    def encrypt_covariates(self, X, XtX_inv):
        X, px = self._arr(X)
        A, pa = self._arr(XtX_inv)
        self.ctx._c(lib().gwhe_encrypt_covariates(self.h, px, pa))

    def encrypt_phenotype(self, y):
        y, py = self._arr(y)
        self.ctx._c(lib().gwhe_encrypt_phenotype(self.h, py))

    def encrypt_snps(self, S, b0=0, b1=None):
        """encrypt SNP batches [b0, b1) ahead of snp_stats(None, ...)"""
        S, ps = self._arr(S)
        b1 = self.layout["batches"] if b1 is None else b1
        self.ctx._c(lib().gwhe_encrypt_snps(self.h, ps, b0, b1))

    def fit(self, kappa):
        self.ctx._c(lib().gwhe_fit_covariates(self.h, kappa))

    def set_fit_state(self, M, w, wz):
        M, pm = self._arr(M)
        w, pw = self._arr(w)
        wz, pz = self._arr(wz)
        self.ctx._c(lib().gwhe_set_fit_state(self.h, pm, pw, pz))

    def snp_stats(self, S, b0=0, b1=None):
        """Alg. 11 loop over batches [b0, b1); S = None takes the batches
        encrypted by encrypt_snps"""
        S, ps = (None, None) if S is None else self._arr(S)
        b1 = self.layout["batches"] if b1 is None else b1
        self.ctx._c(lib().gwhe_snp_stats(self.h, ps, b0, b1, 1))

    def decrypt_results(self):
        num = np.full(self.k, np.nan)
        den = np.full(self.k, np.nan)
        self.ctx._c(lib().gwhe_decrypt_results(self.h, num, den))
        return num, den

    def state_words(self):
        """size (uint64 words) of the batch-invariant state after the fit"""
        w = _sz(0)
        self.ctx._c(lib().gwhe_job_state_size(self.h, ctypes.byref(w)))
        return w.value

    def export_state(self, out=None):
        """the covariate phase's batch-invariant state as a flat uint64 buffer
        (numpy array, or into `out`: a torch tensor of int64 on host or device)"""
        words = self.state_words()
        if out is None:
            out = np.zeros(words, np.uint64)
        self.ctx._c(lib().gwhe_job_export_state(self.h, _ptr(out), words))
        return out

    def import_state(self, buf):
        """take the state exported by a job of the same shape under the same
        keys (numpy uint64 array or torch int64 tensor, host or device)"""
        n = buf.numel() if hasattr(buf, "numel") else buf.size
        self.ctx._c(lib().gwhe_job_import_state(self.h, _ptr(buf), n))

    def set_nonce(self, nonce):
        """offset of this job's encryption ids (distinct per live job under one key)."""
        self.ctx._c(lib().gwhe_job_set_nonce(self.h, nonce))

    def set_host_state(self, chunk=32):
        """keep Dup(M_j) (M-CCP layout) in pinned host memory, prefetched back
        `chunk` columns at a time per set of SNP batches (0: on the device)."""
        self.ctx._c(lib().gwhe_job_set_host_state(self.h, chunk))

    def release_results(self):
        self.ctx._c(lib().gwhe_job_release_results(self.h))

    def ct(self, which, index=0):
        """a view of a job ciphertext (valid while the job lives)."""
        h = _vp()
        self.ctx._c(lib().gwhe_job_ct(self.h, which, index, ctypes.byref(h)))
        v = Ciphertext(self.ctx, h)
        v.job = self
        return v

    def keyswitches(self):
        return lib().gwhe_job_keyswitches(self.h)


def job_footprint(ctx: Context, n, d, k, layout="auto", chunk_batches=64):
    """estimated device bytes of one job beyond the shared keys."""
    v = lib().gwhe_job_footprint(ctx.h, n, d, k, LAYOUTS[layout], chunk_batches)
    if v < 0:
        raise GwheError(-1, "bad job shape")
    return v


class Server:
    """Continuous batching of GWAS jobs on the context's GPU: worker threads
    with their own streams share the context's keys; jobs are admitted by
    estimated HBM footprint as memory frees up and overlap on the device."""

    def __init__(self, ctx: Context, workers=4, hbm_budget=0, chunk_batches=64,
                 one_snp_loop=False):
        self.ctx = ctx
        h = _vp()
        ctx._c(lib().gwhe_server_create_ex(ctx.h, workers, hbm_budget, chunk_batches,
                                           1 if one_snp_loop else 0, ctypes.byref(h)))
        self.h = h
        self._k = {}
        ctx._children.add(self)

    def submit(self, X, XtX_inv, y, S, kappa=1, layout="auto", nonce=0, borrow=False):
        """queue one job; borrow=True leaves S in place (kept referenced here
        until wait) instead of copying it"""
        X = np.ascontiguousarray(X, np.float64)
        A = np.ascontiguousarray(XtX_inv, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        S = np.ascontiguousarray(S, np.float64)
        n, d = X.shape
        k = S.shape[1]
        rid = _l(0)
        f = lib().gwhe_server_submit_borrowed if borrow else lib().gwhe_server_submit
        self.ctx._c(f(self.h, n, d, k, LAYOUTS[layout], kappa, nonce, X, A, y, S,
                      ctypes.byref(rid)))
        self._k[rid.value] = (k, S if borrow else None)
        return rid.value

    def wait(self, rid):
        """(num[k], den[k], {"queue_ms", "run_ms", "latency_ms", "device_start_ms",
        "device_end_ms", "high_priority"})"""
        k, _held = self._k.pop(rid)  # a borrowed S stays referenced until here
        num = np.full(k, np.nan)
        den = np.full(k, np.nan)
        t = np.zeros(8)
        self.ctx._c(lib().gwhe_server_wait(self.h, rid, num, den, t))
        return num, den, {"queue_ms": t[0], "run_ms": t[1], "latency_ms": t[2],
                          "device_start_ms": t[3], "device_end_ms": t[4],
                          "high_priority": bool(t[5]), "snp_start_ms": t[6],
                          "snp_end_ms": t[7]}

    def stats(self):
        out = (_l * 9)()
        self.ctx._c(lib().gwhe_server_stats(self.h, out))
        keys = ["admitted", "running", "waiting", "bytes_claimed", "peak_bytes_claimed", "budget",
                "host_tier_jobs", "max_running", "live_workers"]
        return {kk: int(v) for kk, v in zip(keys, out)}

    def close(self):
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            lib().gwhe_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
