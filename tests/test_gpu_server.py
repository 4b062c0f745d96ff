"""The serving loop on the GPU: two models on two contexts (different chains),
requests submitted from the test thread while the loop runs; every result must
be bit-identical to the same request run alone through the compiled model, and
decrypt to the FP64 CNN's logits."""
import numpy as np
import pytest

import workloads as W
from oracle import cnn

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


def setup_model(G, layers, params, Wi, Hi, spc):
    stride, levels, steps = G.plan(layers, Wi, Hi)
    ctx = G.Context(seed=W.KEY_SEED, **params)
    ctx.keygen(steps)
    return ctx, ctx.compile(layers, Wi, Hi, spc), stride


@pytest.fixture(scope="module")
def two_models(G):
    lenet = W.lenet1()
    conv = W.single_conv()
    a = setup_model(G, lenet, W.small_params("lenet1", 11), 28, 28, 1)
    b = setup_model(G, conv, W.small_params("conv1", 11), 28, 28, 1)
    return (lenet, a), (conv, b)


@pytest.mark.parametrize("policy", [dict(), dict(max_inflight=1, exact_batches=True)])
def test_results_identical_alone_and_mixed(G, two_models, policy):
    (lenet, (ca, ma, sa)), (conv, (cb, mb, sb)) = two_models
    imgs = W.images(7)
    # requests: (model id, context, stride, images, seed); one request of two ciphertexts
    reqs = []
    for k in range(7):
        if k % 2 == 0:
            reqs.append((0, ca, sa, imgs[k:k + 1], W.ENC_SEED + k))
        else:
            reqs.append((1, cb, sb, imgs[k:k + 1], W.ENC_SEED + k))
    reqs.append((0, ca, sa, imgs[0:2], W.ENC_SEED + 50))
    models = [ma, mb]
    alone = []
    for mid, ctx, stride, x, seed in reqs:
        ct = ctx.encrypt(x, 1, stride, seed)
        alone.append(ctx.export(models[mid].infer(ct)))
    srv = G.Server(max_batch=4, **policy)
    assert srv.add_model(ma) == 0 and srv.add_model(mb) == 1
    ids = []
    for mid, ctx, stride, x, seed in reqs:
        ct = ctx.encrypt(x, 1, stride, seed)
        ids.append((mid, ctx, srv.submit(mid, ct)))
        del ct                     # the server keeps its own reference
    outs = []
    for (mid, ctx, rid), want in zip(ids, alone):
        assert srv.poll(rid) in (False, True)
        out, lat = srv.wait(rid)
        assert lat > 0
        got = ctx.export(out)
        assert got.shape == want.shape and np.array_equal(got, want)
        outs.append(out)
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["batches"] >= 2 and st["p50_ms"] <= st["p99_ms"]
    # decrypted results against the FP64 CNN
    for (mid, ctx, stride, x, seed), out in zip(reqs, outs):
        layers = lenet if mid == 0 else conv
        n_out = 10 if mid == 0 else 784
        dec = ctx.decrypt(out, n_out)
        for s in range(x.shape[0]):
            ref = cnn.forward(x[s], layers).reshape(-1)
            if mid == 0:
                assert np.abs(dec[s] - ref).max() < 1e-3
            else:   # the conv output sits at r*28 + c for r, c < 24
                v = dec[s].reshape(28, 28)[:24, :24].reshape(-1)
                assert np.abs(v - ref).max() < 1e-3
    srv.close()


def test_admission_and_errors(G, two_models):
    (_, (ca, ma, sa)), (_, (cb, mb, sb)) = two_models
    small = G.Server(max_batch=2, mem_budget=1 << 20)
    with pytest.raises(G.HeError) as e:
        small.add_model(ma)
    assert "HE_ENOMEM" in str(e.value)
    small.close()
    srv = G.Server(max_batch=2)
    srv.add_model(ma)
    ct_other = cb.encrypt(W.images(1), 1, sb, 1)
    with pytest.raises(G.HeError):
        srv.submit(0, ct_other)          # ciphertext of another context
    with pytest.raises(G.HeError):
        srv.submit(5, ct_other)          # unknown model
    big = ca.encrypt(W.images(3), 1, sa, 2)
    with pytest.raises(G.HeError):
        srv.submit(0, big)               # three ciphertexts > max_batch 2
    srv.close()
