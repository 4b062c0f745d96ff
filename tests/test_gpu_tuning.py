"""Autotuner: every launch shape it can choose gives bit-identical ciphertexts
(limb split over 2-CTA clusters, MAC output groups, key-switch tiling and grid
order), and its JSON cache round-trips."""
import json

import numpy as np
import pytest

import workloads as W

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


# limb layouts: 0 one CTA per limb, 1 a 2-CTA cluster, 2 the two-kernel form (outer stages over
# columns, inner stages over 1024-coefficient blocks)
SETTINGS = [
    dict(ntt_split=1, moddown_split=1, rescale_split=1, mac_group=4, lazy_bt=1, lazy_order=1, mac_bk=16, mac_split=1),
    dict(ntt_split=0, moddown_split=1, rescale_split=0, mac_group=6, lazy_bt=4, lazy_order=0, mac_bk=32, mac_split=2),
    dict(ntt_split=1, moddown_split=0, rescale_split=1, mac_group=12, lazy_bt=2, lazy_order=1, mac_bk=64, mac_split=2),
    dict(ntt_split=2, moddown_split=2, rescale_split=2, mac_group=8, lazy_bt=2, lazy_order=0, mac_bk=32, mac_split=1,
         comb_bt=2),
    dict(ntt_split=2, moddown_split=0, rescale_split=1, mac_group=12, lazy_bt=4, lazy_order=1, mac_bk=64, mac_split=1,
         comb_bt=4),
    # single-output weighted combinations with their weights folded into the keys from one
    # ciphertext on (the default folds from 16: not at these batch sizes)
    dict(ntt_split=2, moddown_split=2, rescale_split=2, mac_group=12, lazy_bt=4, lazy_order=0, mac_bk=64, mac_split=1,
         comb_bt=2, comb_fold=1),
    dict(ntt_split=2, moddown_split=2, rescale_split=2, mac_group=12, lazy_bt=4, lazy_order=0, mac_bk=64, mac_split=1,
         comb_bt=4, comb_fold=1),
    # the mask MAC of six or more outputs on the tensor cores: every limb, or the limbs of primes
    # of at most five bytes (the others on the integer units)
    dict(ntt_split=2, moddown_split=2, rescale_split=2, mac_group=12, lazy_bt=4, lazy_order=0, mac_bk=64, mac_split=1,
         comb_bt=4, mac_tc=8),
    dict(ntt_split=2, moddown_split=2, rescale_split=2, mac_group=8, lazy_bt=2, lazy_order=0, mac_bk=32, mac_split=2,
         comb_bt=2, mac_tc=5),
]


@pytest.mark.parametrize("params", ["lenet1", "serve_lenet1", "lenet1_2_14"])
def test_every_launch_shape_gives_the_same_ciphertexts(G, params):
    P = dict(W.SERVE_PARAMS["lenet1"] if params == "serve_lenet1" else W.PARAMS["lenet1"])
    if params != "lenet1_2_14":
        P["logn"] = 12                  # 2048 slots: two samples per ciphertext
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    imgs = W.images(6)
    m = ctx.compile(model, 28, 28, 2)
    ct = ctx.encrypt(imgs, 2, stride, W.ENC_SEED)
    ref = ctx.export(m.infer(ct))
    for s in SETTINGS:
        ctx.set_tuning(**s)
        got = ctx.export(m.infer(ct))
        assert np.array_equal(got, ref), s
    ctx.set_tuning(**{k: -1 for k in ctx.TUNE_KNOBS})


def test_autotune_and_cache(G, tmp_path):
    P = dict(W.SERVE_PARAMS["lenet1"])
    P["logn"] = 13
    ctx = G.Context(seed=1, **P)
    path = str(tmp_path / "tune.json")
    rep = ctx.autotune(path)
    assert "ntt_split" in rep and "mac_group" in rep and "lazy_order" in rep and "mac_bk" in rep and "comb_bt" in rep
    chosen = ctx.tuning()
    assert all(v >= 0 for v in chosen.values())
    assert chosen["mac_group"] == rep["mac_group"]["chosen"]
    cache = json.load(open(path))
    assert len(cache) == 1 and list(cache.values())[0] == chosen
    ctx2 = G.Context(seed=1, **P)
    rep2 = ctx2.autotune(path)
    assert "cached" in rep2 and ctx2.tuning() == chosen
