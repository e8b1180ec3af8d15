"""CPU checks of the C ABI: the library loads, exports every declared symbol,
and its host-only parameter code agrees with the oracle's independent
implementation of the same definitions (no GPU call is made)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    from paper_1902_04303_gb300 import build
    build.build()
    from paper_1902_04303_gb300 import gwhe
    gwhe.lib()
    return gwhe


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gwhe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gwhe_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(g):
    lib = g.lib()
    names = declared_functions()
    assert len(names) >= 40
    for name in names:
        assert hasattr(lib, name), name
    # and the binding covers exactly what the header declares
    assert set(g.exported_symbols()) == set(names)


@pytest.mark.parametrize("logN,L,K", [(4, 4, 2), (10, 21, 7), (13, 4, 1), (16, 24, 8)])
def test_primes_match_oracle(g, logN, L, K):
    from oracle import ckks
    q, p = g.gen_primes(g.params(logN, L, K=K))
    oq = np.zeros(L, np.uint64)
    op = np.zeros(K, np.uint64)
    assert ckks.lib().or_gen_primes(logN, L, 60, 40, K, 60, oq, op) == 0
    assert np.array_equal(q, oq) and np.array_equal(p, op)


@pytest.mark.parametrize("logN", [4, 10, 13, 16])
@pytest.mark.parametrize("sign", [-1, 1])
def test_encoding_twiddles_match_oracle_bitwise(g, logN, sign):
    from oracle import ckks
    W, T = g.fft_twiddles(logN, sign)
    M = 1 << (logN - 1)
    oW = np.zeros(M, np.float64)
    oT = np.zeros(2 * M, np.float64)
    ckks.lib().or_fft_twiddles(logN, sign, oW, oT)
    assert W.tobytes() == oW.tobytes() and T.tobytes() == oT.tobytes()


def test_layout_matches_paper_and_oracle(g):
    from oracle.circuit import Layout
    lay = g.layout(17, 245, 10643)
    assert lay["tau"] == 512 and lay["batches"] == 21  # section "Results"
    for logN, n, k in [(16, 245, 10643), (13, 64, 256), (10, 16, 40), (16, 1000, 5000)]:
        o = Layout(logN, n, 1, k)
        got = g.layout(logN, n, k)
        assert (got["nb"], got["B"], got["tau"], got["batches"], got["H"]) == \
            (o.nb, o.B, o.tau, o.batches, o.H)
    with pytest.raises(g.GwheError):
        g.layout(10, 600, 10)  # a column of 1024 slots does not fit 512


def test_bad_parameters_are_rejected_without_gpu(g):
    with pytest.raises(g.GwheError):
        g.gen_primes(g.params(16, 24, K=200))


def test_device_rule_without_gpu(g):
    """A call on a context is refused unless the context's device is current:
    the host-side check behind every entry point (no GPU is touched)."""
    lib = g.lib()
    assert lib.gwhe_device_ok(0, 0) == 0
    assert lib.gwhe_device_ok(3, 3) == 0
    assert lib.gwhe_device_ok(1, 0) == -1  # worker thread left on device 0
    assert lib.gwhe_device_ok(0, 1) == -1
    assert lib.gwhe_device_ok(-1, -1) == -1  # no device recorded
