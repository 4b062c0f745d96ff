"""he_rescale_noalloc: the rescale for callers that cannot allocate device
memory (inside a stream capture, under a fixed memory budget, or next to an
allocator that owns the device).  Checked through the C ABI against the
allocating he_rescale on two calls in a row, and for its size limit.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_03060_gb300 import build
    build.build()
    import paper_2402_03060_gb300 as lib
    return lib


def test_rescale_noalloc_matches_rescale(G):
    import torch
    P = dict(logn=14, data_bits=[60, 40, 40, 40], special_bits=[60], dnum=4, log2_scale=40)
    ctx = G.Context(seed=3, **P)
    ctx.keygen([])
    L = G.load()
    M, N, B, lp = 1 << 13, 1 << 14, 3, 4
    for call in range(2):   # two calls in a row share (and overwrite) the scratch array
        x = np.random.default_rng(call).uniform(-1, 1, (B, M))
        ct = ctx.encrypt(x, 1, M, 500 + call)
        if call:
            ct = ctx.square([ct])[0]   # a different level and scale on the second call
        b, l, _ = ct.info()
        want = ctx.export(ctx.rescale(ct))
        coeff = ctx.export(ct)
        d_in = torch.from_numpy(coeff.view(np.int64).copy()).cuda()
        ctx.ntt(d_in.data_ptr(), b * 2 * l, [t for _ in range(2 * b) for t in range(l)])   # to evaluation form
        d_out = torch.zeros((b, 2, l - 1, N), dtype=torch.int64, device="cuda")
        ctx.sync()
        G.check(L.he_rescale_noalloc(ctx.h, ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                     b, l))
        ctx.ntt(d_out.data_ptr(), b * 2 * (l - 1), [t for _ in range(2 * b) for t in range(l - 1)], inverse=True)
        ctx.sync()
        got = d_out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want)
    # beyond the scratch size: a clear error, nothing launched
    with pytest.raises(G.HeError) as e:
        G.check(L.he_rescale_noalloc(ctx.h, ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                     17, 4))
    assert e.value.status == 1 and "scratch" in str(e.value)
    with pytest.raises(G.HeError) as e:
        G.check(L.he_rescale_noalloc(ctx.h, ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                     1, 1))
    assert e.value.status == 3
    # in and out overlapping (in place, or shifted by one word): refused on the host, nothing launched
    for shift in (0, 8):
        with pytest.raises(G.HeError) as e:
            G.check(L.he_rescale_noalloc(ctx.h, ctypes.c_void_p(d_in.data_ptr()),
                                         ctypes.c_void_p(d_in.data_ptr() + shift), 1, 4))
        assert e.value.status == 1 and "overlap" in str(e.value)
