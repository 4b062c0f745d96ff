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


def test_memory_admission_refuses_and_readmits(G):
    """A budget that holds the model plus exactly k = 2 request ciphertexts: two requests
    are admitted, the third gets HE_ENOMEM (the first two are not collected yet); after one
    he_server_wait collects a result the retried third request is admitted.  Every result
    is bit-identical to the same request run alone through the compiled model."""
    P = W.PARAMS["lenet1"]
    lenet = W.lenet1()
    ctx, m, stride = setup_model(G, lenet, P, 28, 28, 10)
    imgs = W.images(30)
    cts = [ctx.encrypt(imgs[10 * i: 10 * i + 10], 10, stride, W.ENC_SEED + i) for i in range(3)]
    alone = [ctx.export(m.infer(ct, use_graph=True)) for ct in cts]
    ct_bytes = 2 * ctx.n_data * ctx.n * 8          # one top-level ciphertext
    # the model's residency as the server counts it (the graphs are captured by the first add)
    probe = G.Server(max_batch=2, max_inflight=1, exact_batches=True)
    probe.add_model(m)
    probe.close()
    probe = G.Server(max_batch=2, max_inflight=1, exact_batches=True)
    probe.add_model(m)
    resident = probe.stats()["resident_bytes"]
    probe.close()
    srv = G.Server(max_batch=2, max_inflight=1, exact_batches=True, mem_budget=resident + 2 * ct_bytes + ct_bytes // 2)
    srv.add_model(m)
    assert abs(srv.stats()["resident_bytes"] - resident) < ct_bytes // 2
    r0 = srv.submit(0, cts[0])
    r1 = srv.submit(0, cts[1])
    with pytest.raises(G.HeError) as e:
        srv.submit(0, cts[2])
    assert e.value.status == 2 and "admission" in str(e.value)
    out0, _ = srv.wait(r0)
    r2 = srv.submit(0, cts[2])       # one result collected: room for one ciphertext again
    out1, _ = srv.wait(r1)
    out2, _ = srv.wait(r2)
    for out, want in zip((out0, out1, out2), alone):
        assert np.array_equal(ctx.export(out), want)
    logits = ctx.decrypt(out2, 10)
    for s in range(10):
        assert np.abs(logits[s] - cnn.forward(imgs[20 + s], lenet)).max() < 1e-3
    assert srv.stats()["requests"] == 3
    srv.close()
