"""GPU parity of the paper-order schedule: the CUDA library under
he_context_set_schedule(HE_SCHEDULE_LITERAL) -- every Rot its own key switch, masks
multiplied over Q_l after the rotations, Add, the centred rescale; square = tensor,
relinearise, rescale; flatten stages as mask, rotate, add -- compared limb by limb, in
coefficient form, with the oracle's literal backend on the same seeded inputs."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, cnn, layers as olayers

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


def slots_of(samples, stride, slots):
    x = np.zeros(slots)
    for b, s in enumerate(samples):
        f = np.asarray(s).reshape(-1)
        x[b * stride: b * stride + f.size] = f
    return x


def assert_same(ctx, gct, he, oct_, b=0):
    got = ctx.export(gct)[b]
    want = he.to_coeff(oct_)
    assert got.shape == want.shape, (got.shape, want.shape)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} residues differ, first at {bad[:3].tolist()}"


def literal_pair(G, P, steps):
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    ctx.set_schedule("literal")
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    he.keygen(steps)
    return ctx, he


def oracle_literal(he, model, samples, Wi, Hi, stride, spc, seed, dims=2, C=1):
    lay = olayers.input_layout(Wi, Hi, stride, spc, he.n // 2, dims, channels=C)
    ct = he.encrypt(slots_of(samples, stride, he.n // 2), seed)
    ys, _ = olayers.run_model(olayers.HeBackend(he, literal=True), ct, model, lay)
    return ys[0]


def test_literal_ops_bit_exact(G):
    """Square (tensor, relinearise, rescale) and the layer calls of a small ring."""
    P = dict(logn=10, data_bits=[60, 40, 40, 40], special_bits=[60], dnum=4, log2_scale=40)
    ctx, he = literal_pair(G, P, [1, 32, 33])
    x = np.random.default_rng(3).uniform(0, 1, (1, 16, 32))   # one 32 x 16 image, 512 slots
    g = ctx.encrypt(x, 1, 512, 77)
    o = he.encrypt(x[0].reshape(-1), 77)
    assert_same(ctx, g, he, o)
    assert_same(ctx, ctx.square([g])[0], he, he.square_literal(o))
    # a fused square of the same input differs in its bits (one division by q_top * P)
    assert not np.array_equal(he.to_coeff(he.square(o)), he.to_coeff(he.square_literal(o)))
    pool = ctx.avgpool([g], 2)[0]
    want = he.ct_add(he.ct_add(he.ct_add(o, he.rotate(o, 1)), he.rotate(o, 32)), he.rotate(o, 33))
    assert_same(ctx, pool, he, want)


def test_lenet1_literal_small_ring_bit_exact(G):
    """LeNet-1 in the paper's order at N = 2^11 (eager and graph replay), bit-exact against
    the literal oracle; its logits against the FP64 CNN."""
    P = W.small_params("lenet1", 11)
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28, schedule="literal")
    assert set(steps) == set(olayers.plan(model, 28, 28, schedule="literal")["steps"])
    ctx, he = literal_pair(G, P, steps)
    img = W.images(1)
    gct = ctx.encrypt(img, 1, stride, W.ENC_SEED)
    m = ctx.compile(model, 28, 28, 1)
    out_eager = m.infer(gct)
    out_graph = m.infer(gct, use_graph=True)
    want = oracle_literal(he, model, img, 28, 28, stride, 1, W.ENC_SEED)
    assert_same(ctx, out_eager, he, want)
    assert_same(ctx, out_graph, he, want)
    assert np.abs(ctx.decrypt(out_eager, 10)[0] - cnn.forward(img[0], model)).max() < 1e-3


@pytest.mark.parametrize("name", ["M1", "M3", "M6", "M7"])
def test_paper_models_literal_bit_exact(G, name):
    if name == "M3":
        model, Wi, Hi = W.m3_relu(), 28, 28
    else:
        model, Wi, Hi = W.paper_model(name)
    dims = 1 if Hi == 1 else 2
    ns = 2
    stride, levels, steps = G.plan(model, Wi, Hi, schedule="literal")
    logn = max(11, int(np.ceil(np.log2(stride * ns))) + 1)
    P = dict(logn=logn, data_bits=[60] + [40] * levels, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    ctx, he = literal_pair(G, P, steps)
    x = W.images(ns, Hi, Wi) if dims == 2 else W.signals(ns, Wi)[:, 0]
    out = ctx.compile(model, Wi, Hi, ns).infer(ctx.encrypt(x, ns, stride, W.ENC_SEED), use_graph=True)
    want = oracle_literal(he, model, x, Wi, Hi, stride, ns, W.ENC_SEED, dims)
    assert_same(ctx, out, he, want)
    n_out = model[-1]["w"].shape[0]
    logits = ctx.decrypt(out, n_out)
    for b in range(ns):
        assert np.abs(logits[b] - cnn.forward(x[b], model, dims=dims)).max() < 1e-3


def test_schedule_is_kept_by_the_compiled_model(G):
    """A model compiled under one schedule runs that schedule whatever the context is set to
    later; the fused and the literal results decrypt alike but differ in their bits."""
    P = W.small_params("lenet1", 11)
    model = W.lenet1()
    st_l = G.plan(model, 28, 28, schedule="literal")[2]
    st_f = G.plan(model, 28, 28)[2]
    stride = G.plan(model, 28, 28)[0]
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(sorted(set(st_l) | set(st_f)))
    img = W.images(1)
    gct = ctx.encrypt(img, 1, stride, W.ENC_SEED)
    m_f = ctx.compile(model, 28, 28, 1)
    ctx.set_schedule("literal")
    m_l = ctx.compile(model, 28, 28, 1)
    ctx.set_schedule("fused")
    a, b = ctx.export(m_l.infer(gct)), ctx.export(m_f.infer(gct))
    ctx.set_schedule("literal")
    c = ctx.export(m_f.infer(gct))
    assert np.array_equal(b, c) and not np.array_equal(a, b)
    la, lb = ctx.decrypt(m_l.infer(gct), 10)[0], ctx.decrypt(m_f.infer(gct), 10)[0]
    assert np.abs(la - lb).max() < 1e-5


@pytest.mark.slow
def test_lenet1_literal_full_size_bit_exact(G):
    """LeNet-1 at the benchmark's parameters (N = 2^14, chain [60, 40 x 7 | 60], dnum 8) in
    the paper's order: 21 samples in 3 ciphertexts (the last with one), one graph launch.
    The first ciphertext is compared limb by limb with the literal oracle run on it alone;
    every sample's logits with the FP64 CNN."""
    P = W.PARAMS["lenet1"]
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28, schedule="literal")
    ctx, he = literal_pair(G, P, steps)
    imgs = W.images(21)
    out = ctx.compile(model, 28, 28, 10).infer(ctx.encrypt(imgs, 10, stride, W.ENC_SEED), use_graph=True)
    assert out.batch == 3
    want = oracle_literal(he, model, imgs[:10], 28, 28, stride, 10, W.ENC_SEED)
    assert_same(ctx, out, he, want, 0)
    logits = ctx.decrypt(out, 10)
    for k in range(21):
        assert np.abs(logits[k] - cnn.forward(imgs[k], model)).max() < 1e-3
