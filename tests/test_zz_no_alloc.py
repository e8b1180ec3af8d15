"""The allocation-free key switch (gwhe_keyswitch_noalloc), for callers that
cannot let the library allocate device memory (a serving process whose memory
is reserved by its own pool, or a request path where an allocator call could
block).  Its output must equal the allocating gwhe_keyswitch bit for bit, on
consecutive calls that reuse the same static scratch array."""
import gc

import numpy as np
import pytest

from oracle.ckks import galois_conj
from paper_1902_04303_gb300.datagen import make_residues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    torch.cuda.set_device(0)
    from paper_1902_04303_gb300 import build
    build.build()
    from paper_1902_04303_gb300 import gwhe
    return gwhe


def noalloc_switch(ctx, x_coeff, key_id):
    """coefficient-domain host x -> device NTT -> no-alloc switch -> host coefficients"""
    import torch
    l = x_coeff.shape[0]
    xt = torch.from_numpy(np.ascontiguousarray(x_coeff).view(np.int64)).cuda()
    ctx.ntt_batch(xt, 1, l)
    out = torch.zeros(2 * l * ctx.N, dtype=torch.int64, device="cuda")
    ctx.keyswitch_noalloc(xt, l, key_id, out)
    ctx.ntt_batch(out, 2, l, inverse=True)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64).reshape(2, l, ctx.N)


def test_noalloc_keyswitch_allocates_nothing(g):
    """After a warm-up call, a second call at the same level leaves the
    device's stream-ordered pool (in use and reserved) and the device's free
    memory exactly as they were: the promise of the entry point."""
    import torch
    ctx = g.Context(16, 24, K=8, dnum=3, seed=19)
    ctx.keygen(rot_steps=[1], conj=False)
    l = 5
    x = make_residues(l, ctx.N, ctx.q[:l], seed=3)
    xt = torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
    ctx.ntt_batch(xt, 1, l)
    out = torch.zeros(2 * l * ctx.N, dtype=torch.int64, device="cuda")
    ctx.keyswitch_noalloc(xt, l, 0, out)  # warm-up: loads the kernels it launches
    ctx.sync()
    torch.cuda.synchronize()
    # no other object may free device memory meanwhile (a collected context
    # of an earlier test would): collect first, then keep the collector off
    gc.collect()
    gc.disable()
    try:
        before = ctx.mem_info()
        ctx.keyswitch_noalloc(xt, l, 0, out)
        ctx.sync()
        after = ctx.mem_info()
    finally:
        gc.enable()
    for key in ("pool_used", "pool_reserved", "free"):
        assert after[key] == before[key], (key, before, after)


@pytest.mark.parametrize("logN,L,K,dnum,levels", [(10, 6, 3, 3, (6, 3)), (16, 24, 8, 3, (4, 5))])
def test_noalloc_keyswitch_matches_allocating_keyswitch(g, logN, L, K, dnum, levels):
    ctx = g.Context(logN, L, K=K, dnum=dnum, seed=17)
    ctx.keygen(rot_steps=[1], conj=True)
    for call, l in enumerate(levels):  # two calls in a row share the scratch array
        for key_id in (0, galois_conj(logN)):
            x = make_residues(l, ctx.N, ctx.q[:l], seed=100 * call + key_id % 7)
            want = ctx.keyswitch(x, key_id)
            got = noalloc_switch(ctx, x, key_id)
            assert np.array_equal(got, want), (call, l, key_id)


def test_noalloc_keyswitch_rejects_requests_beyond_the_static_array(g):
    ctx = g.Context(16, 24, K=8, dnum=3, seed=17)
    ctx.keygen(rot_steps=[], conj=False)
    import torch
    x = torch.zeros(24 * ctx.N, dtype=torch.int64, device="cuda")
    out = torch.zeros(2 * 24 * ctx.N, dtype=torch.int64, device="cuda")
    with pytest.raises(g.GwheError) as e:
        ctx.keyswitch_noalloc(x, 24, 0, out)
    assert e.value.code == -1 and "scratch" in str(e.value)
