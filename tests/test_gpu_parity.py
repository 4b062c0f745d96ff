"""GPU parity: every ciphertext the CUDA library produces is compared limb by
limb, in coefficient form, with the CPU oracle's on the same seeded inputs
(bit-exact), and decrypted logits with the FP64 CNN (max-abs 1e-3)."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, cnn, layers as olayers

pytestmark = pytest.mark.gpu

U64 = np.uint64


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_03060_gb300 import build
    build.build()
    import paper_2402_03060_gb300 as lib
    return lib


def make_pair(G, P, steps, seed=W.KEY_SEED):
    ctx = G.Context(seed=seed, **P)
    ctx.keygen(steps)
    he = ckks.Ckks(seed=seed, **P)
    he.keygen(steps)
    return ctx, he


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


P_SMALL = dict(logn=10, data_bits=[60, 40, 40, 40], special_bits=[60], dnum=4, log2_scale=40)
P_DIGITS = dict(logn=10, data_bits=[60, 40, 40, 40, 40], special_bits=[60, 60], dnum=3, log2_scale=40)
# N = 2^15: every limb is split over a 2-CTA cluster (NTT, ModDown, rescale, FFT)
P_BIG = dict(logn=15, data_bits=[60, 40, 40, 40], special_bits=[60, 60], dnum=2, log2_scale=40)
STEPS = {"small": [1, 3, 7, -2, 100, 511], "digits": [1, 5, -9], "big": [1, -3, 1000, 8191]}


def test_primes_match_oracle(G):
    for P in (P_SMALL, P_DIGITS, P_BIG, W.PARAMS["lenet1"], W.PARAMS["conv1"]):
        ctx = G.Context(seed=1, **P)
        assert ctx.primes() == ckks.gen_primes(list(P["data_bits"]) + list(P["special_bits"]), P["logn"])


# limb layouts: None the default for N, 0 one CTA per limb, 1 a 2-CTA cluster, 2 the two-kernel
# form (outer stages over columns, inner stages over 1024-coefficient blocks)
@pytest.mark.parametrize("logn,layout", [(4, None), (10, None), (13, None), (14, None), (15, None),
                                         (11, 2), (12, 2), (13, 2), (14, 0), (14, 1), (15, 1)])
def test_ntt_matches_oracle(G, logn, layout):
    import torch
    P = dict(logn=logn, data_bits=[60, 40], special_bits=[60], dnum=2, log2_scale=30)
    ctx = G.Context(seed=1, **P)
    if layout is not None:
        ctx.set_tuning(ntt_split=layout)
    he = ckks.Ckks(seed=1, **P)
    qs = ctx.primes()
    rng = np.random.default_rng(logn)
    idx = [0, 1, 2, 1, 0]   # ragged mix of primes
    a = np.stack([rng.integers(0, qs[i], 1 << logn, dtype=U64) for i in idx])
    d = torch.from_numpy(a.view(np.int64).copy()).cuda()
    ctx.ntt(d.data_ptr(), len(idx), idx)
    ctx.sync()
    got = d.cpu().numpy().view(U64)
    allpsi = he.qpsi + he.ppsi
    br = np.array([int(format(k, f"0{logn}b")[::-1], 2) for k in range(1 << logn)])
    for r, i in enumerate(idx):
        want = he.ntt(a[r][None], [qs[i]], [allpsi[i]])[0]
        assert np.array_equal(got[r], want[br]), f"row {r}"
    ctx.ntt(d.data_ptr(), len(idx), idx, inverse=True)
    ctx.sync()
    assert np.array_equal(d.cpu().numpy().view(U64), a)


@pytest.fixture(scope="module")
def pair_small(G):
    return make_pair(G, P_SMALL, [1, 3, 7, -2, 100, 511])


@pytest.fixture(scope="module")
def pair_digits(G):
    return make_pair(G, P_DIGITS, STEPS["digits"])


@pytest.fixture(scope="module")
def pair_big(G):
    return make_pair(G, P_BIG, STEPS["big"])


def enc_both(ctx, he, samples, stride, spc, seed=9000, lp=None):
    slots = he.n // 2
    gct = ctx.encrypt(np.asarray(samples), spc, stride, seed)
    oct_ = he.encrypt(slots_of(samples, stride, slots), seed)
    return gct, oct_


@pytest.mark.parametrize("which", ["small", "digits", "big"])
def test_encrypt_and_ops_bit_exact(G, pair_small, pair_digits, pair_big, which):
    ctx, he = {"small": pair_small, "digits": pair_digits, "big": pair_big}[which]
    rng = np.random.default_rng(3)
    M = he.n // 2
    samples = rng.uniform(-1, 1, (1, M))
    gct, oct_ = enc_both(ctx, he, samples, M, 1)
    assert_same(ctx, gct, he, oct_)
    # fresh-encryption noise in a slot grows about like N (coefficient noise ~ sqrt(N),
    # and each slot sums N coefficients): 2^-25 at N = 1024
    grow = max(1.0, M / 512)
    assert np.abs(ctx.decrypt(gct, M)[0] - samples[0]).max() < 2.0 ** -25 * grow
    steps = STEPS[which]
    for s in steps:
        assert_same(ctx, ctx.rotate(gct, s), he, he.rotate(oct_, s))
    hs = ctx.rotate_hoisted(gct, [0] + steps)
    ho = he.rotate_hoisted(oct_, [0] + steps)
    for i, s in enumerate([0] + steps):
        assert_same(ctx, hs[i], he, ho[s])
    assert_same(ctx, ctx.rescale(gct), he, he.rescale(oct_))
    assert_same(ctx, ctx.square([gct])[0], he, he.square(oct_))
    v = rng.uniform(-1, 1, M)
    pm = ctx.mul_plain(gct, v)
    po = he.ct_mul_plain(oct_, he.encode(v, he.scale, oct_.lp), he.scale)
    assert_same(ctx, pm, he, po)
    assert_same(ctx, ctx.add(pm, pm), he, he.ct_add(po, po))
    assert np.abs(ctx.decrypt(ctx.rescale(pm), M)[0] - samples[0] * v).max() < 1e-6 * grow
    # a lower level: the last digit becomes short / digits drop out
    low = ctx.rescale(ctx.rescale(gct))
    lowo = he.rescale(he.rescale(oct_))
    assert_same(ctx, ctx.rotate(low, steps[0]), he, he.rotate(lowo, steps[0]))
    assert_same(ctx, ctx.square([low])[0], he, he.square(lowo))


def test_single_conv_incremental_full_size(G):
    """Single 5x5 convolution, N=8192, [60,40,40 | 60], incremental rotations."""
    P = W.PARAMS["conv1"]
    model = W.single_conv()
    steps = [1, 24]
    ctx, he = make_pair(G, P, steps)
    img = W.images(1)
    gct, oct_ = enc_both(ctx, he, img, 784, 1)
    assert_same(ctx, gct, he, oct_)
    gout = ctx.conv2d([gct], model[0]["w"], model[0]["b"], 1, incremental=True)[0]
    lay = olayers.input_layout(28, 28, 784, 1, he.n // 2)
    oout, _ = olayers.conv(olayers.HeBackend(he), [oct_], model[0]["w"], model[0]["b"], 1, lay, "incremental")
    assert_same(ctx, gout, he, oout[0])
    dec = ctx.decrypt(gout, 784)[0]
    ref = cnn.forward(img[0], model)
    got = np.array([dec[r * 28 + c] for r in range(24) for c in range(24)])
    assert np.abs(got - ref).max() < 1e-6


def run_oracle_model(he, model, samples, Wi, Hi, stride, spc, seed, dims=2):
    lay = olayers.input_layout(Wi, Hi, stride, spc, he.n // 2, dims)
    x = slots_of(samples, stride, he.n // 2)
    ct = he.encrypt(x, seed)
    ys, _ = olayers.run_model(olayers.HeBackend(he), ct, model, lay)
    return ys[0]


def test_lenet1_small_ring_bit_exact(G):
    P = W.small_params("lenet1", 11)
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28)
    ctx, he = make_pair(G, P, steps)
    img = W.images(1)
    gct = ctx.encrypt(img, 1, stride, W.ENC_SEED)
    m = ctx.compile(model, 28, 28, 1)
    out_eager = m.infer(gct)
    out_graph1 = m.infer(gct, use_graph=True)
    out_graph2 = m.infer(gct, use_graph=True)
    want = run_oracle_model(he, model, img, 28, 28, stride, 1, W.ENC_SEED)
    assert_same(ctx, out_eager, he, want)
    assert_same(ctx, out_graph1, he, want)
    assert_same(ctx, out_graph2, he, want)
    logits = ctx.decrypt(out_eager, 10)[0]
    assert np.abs(logits - cnn.forward(img[0], model)).max() < 1e-3


def test_lenet5_dnum3_small_ring_bit_exact(G):
    """LeNet-5-shaped net (11 levels, FC -> x^2 -> FC chain) with the serving
    mix's dnum = 3 keys (four-prime digits, four special primes) at N = 4096:
    two samples per ciphertext, bit-exact against the oracle."""
    P = dict(W.SERVE_PARAMS["lenet5"])
    P["logn"] = 12
    model = W.lenet5_sq()
    stride, levels, steps = G.plan(model, 32, 32)
    assert (stride, levels) == (1024, 11)
    ctx, he = make_pair(G, P, steps)
    imgs = W.images(2, 32, 32)
    gct = ctx.encrypt(imgs, 2, stride, W.ENC_SEED)
    out = ctx.compile(model, 32, 32, 2).infer(gct, use_graph=True)
    want = run_oracle_model(he, model, imgs, 32, 32, stride, 2, W.ENC_SEED)
    assert_same(ctx, out, he, want)
    logits = ctx.decrypt(out, 10)
    for b in range(2):
        assert np.abs(logits[b] - cnn.forward(imgs[b], model)).max() < 1e-3


def test_lenet5_full_ring_logits(G):
    """The serving mix's LeNet-5 at N = 2^15 (every limb split over a 2-CTA
    cluster), 16 samples per ciphertext, 2 ciphertexts: logits of every sample
    against the FP64 CNN; the batch equals each ciphertext run alone."""
    P = W.SERVE_PARAMS["lenet5"]
    model = W.lenet5_sq()
    stride, levels, steps = G.plan(model, 32, 32)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    m = ctx.compile(model, 32, 32, 16)
    imgs = W.images(20, 32, 32)
    out = m.infer(ctx.encrypt(imgs, 16, stride, W.ENC_SEED), use_graph=True)
    logits = ctx.decrypt(out, 10)
    for k in range(20):
        assert np.abs(logits[k] - cnn.forward(imgs[k], model)).max() < 1e-3, k
    single = m.infer(ctx.encrypt(imgs[16:], 16, stride, W.ENC_SEED + 1))
    assert np.array_equal(ctx.export(out)[1], ctx.export(single)[0])


def test_cnn1d_tree_fc_dnum3_bit_exact(G):
    """The serving mix's 1-D CNN: dnum = 3 keys (three-prime digits, three special
    primes) and the FC's rotation sum in binary form, N = 8192 (one sample per
    ciphertext), bit-exact against the oracle."""
    P = dict(W.SERVE_PARAMS["cnn1d"])
    P["logn"] = 13
    model = W.cnn1d(fc_sum="tree")
    stride, levels, steps = G.plan(model, 1024, 1)
    assert len(steps) < 120
    ctx, he = make_pair(G, P, steps)
    x = W.signals(1)
    gct = ctx.encrypt(x, 1, stride, W.ENC_SEED)
    out = ctx.compile(model, 1024, 1, 1).infer(gct, use_graph=True)
    want = run_oracle_model(he, model, x[:, 0], 1024, 1, stride, 1, W.ENC_SEED, dims=1)
    assert_same(ctx, out, he, want)
    assert np.abs(ctx.decrypt(out, 5)[0] - cnn.forward(x[0, 0], model, dims=1)).max() < 1e-3


def test_m3_approx_relu_small_ring_bit_exact(G):
    """M3 (approximate ReLU after a convolution and after an FC, 9 levels) at N = 4096,
    dnum = 3, against the oracle; the approx_relu layer call gives the model's
    intermediate ciphertext; logits against the FP64 CNN."""
    P = dict(logn=12, data_bits=[60] + [40] * 9, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    model = W.m3_relu()
    stride, levels, steps = G.plan(model, 28, 28)
    assert levels == 9
    ctx, he = make_pair(G, P, steps)
    img = W.images(1)
    gct = ctx.encrypt(img, 1, stride, W.ENC_SEED)
    out = ctx.compile(model, 28, 28, 1).infer(gct, use_graph=True)
    want = run_oracle_model(he, model, img, 28, 28, stride, 1, W.ENC_SEED)
    assert_same(ctx, out, he, want)
    assert np.abs(ctx.decrypt(out, 10)[0] - cnn.forward(img[0], model)).max() < 1e-3
    # the layer calls: conv then approx_relu equals the first two layers of the model, which
    # first drops the input to the 3 levels they consume (Drop-Level)
    conv_out = ctx.conv2d([ctx.drop_level(gct, levels - 3)], model[0]["w"], model[0]["b"])
    relu_out = ctx.approx_relu(conv_out)
    ref = ctx.compile(model[:2], 28, 28, 1).infer(gct)
    got = np.stack([ctx.export(r) for r in relu_out])
    want2 = ctx.export(ref)
    # the model keeps the 6 channels as one batch, channel-major
    assert np.array_equal(got.reshape(want2.shape), want2)


def _paper_model_case(G, name, n_samples):
    model, Wi, Hi = W.paper_model(name)
    dims = 1 if Hi == 1 else 2
    stride, levels, steps = G.plan(model, Wi, Hi)
    logn = max(11, int(np.ceil(np.log2(stride * n_samples))) + 1)
    P = dict(logn=logn, data_bits=[60] + [40] * levels, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    ctx, he = make_pair(G, P, steps)
    x = W.images(n_samples, Hi, Wi) if dims == 2 else W.signals(n_samples, Wi)[:, 0]
    gct = ctx.encrypt(x, n_samples, stride, W.ENC_SEED)
    out = ctx.compile(model, Wi, Hi, n_samples).infer(gct, use_graph=True)
    want = run_oracle_model(he, model, x, Wi, Hi, stride, n_samples, W.ENC_SEED, dims=dims)
    assert_same(ctx, out, he, want)
    n_out = model[-1]["w"].shape[0]
    logits = ctx.decrypt(out, n_out)
    for b in range(n_samples):
        assert np.abs(logits[b] - cnn.forward(x[b], model, dims=dims)).max() < 1e-3


@pytest.mark.parametrize("name", ["M1", "M6", "M7"])
def test_paper_models_bit_exact(G, name):
    """The paper's M1 (conv K4 S3, flatten after the convolution), M6 (16x16, conv K4
    S2) and M7 (1-D, two strided convolutions): two samples per ciphertext, dnum = 3,
    bit-exact against the oracle; logits against the FP64 CNN."""
    _paper_model_case(G, name, 2)


@pytest.mark.slow
def test_lenet5_m4_bit_exact(G):
    """The paper's M4 (LeNet-5: conv3 16->120 leaves 1x1 per channel, so the
    flatten is channel packing alone, no level): bit-exact against the oracle."""
    _paper_model_case(G, "M4", 1)


def test_three_channel_input_bit_exact(G):
    """M5's layer sequence (channel-narrowed) on 3x32x32 inputs, the three channels
    in one ciphertext (the first convolution hoists 3 x 9 rotations of it): bit-exact
    against the oracle at N = 8192, logits against the FP64 CNN; a single-channel
    ciphertext is refused by the model."""
    model = W.m5_narrow()
    stride, levels, steps = G.plan(model, 32, 32)
    assert (stride, levels) == (3072, 8)
    P = dict(logn=13, data_bits=[60] + [40] * 8, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    ctx, he = make_pair(G, P, steps)
    img = W.images(1, 32, 32, C=3)
    gct = ctx.encrypt(img, 1, stride, W.ENC_SEED)
    m = ctx.compile(model, 32, 32, 1)
    out = m.infer(gct, use_graph=True)
    lay = olayers.input_layout(32, 32, stride, 1, he.n // 2, 2, channels=3)
    oct_ = he.encrypt(slots_of(img, stride, he.n // 2), W.ENC_SEED)
    assert_same(ctx, gct, he, oct_)
    want, _ = olayers.run_model(olayers.HeBackend(he), oct_, model, lay)
    assert_same(ctx, out, he, want[0])
    assert np.abs(ctx.decrypt(out, 10)[0] - cnn.forward(img[0], model)).max() < 1e-3
    from paper_2402_03060_gb300 import HeError
    with pytest.raises(HeError):
        m.infer(ctx.encrypt(img[:, 0], 1, stride, W.ENC_SEED))


def test_m5_full_logits(G):
    """The paper's M5 (CIFAR-10 shaped: 3 -> 16 -> 64 -> 128 channels, 8 levels) with
    the paper's 8192 slots (N = 2^14), two 3x32x32 samples per ciphertext: logits
    against the FP64 CNN.  The compiled model holds about 100 GB of encoded weight
    masks (90,544 masks over Q u P limbs)."""
    model, Wi, Hi = W.paper_model("M5")
    stride, levels, steps = G.plan(model, Wi, Hi)
    P = dict(logn=14, data_bits=[60] + [40] * levels, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    imgs = W.images(2, 32, 32, C=3)
    out = ctx.compile(model, Wi, Hi, 2).infer(ctx.encrypt(imgs, 2, stride, W.ENC_SEED))
    logits = ctx.decrypt(out, 10)
    for b in range(2):
        assert np.abs(logits[b] - cnn.forward(imgs[b], model)).max() < 1e-3


@pytest.mark.parametrize("name", ["M7", "lenet1"])
def test_power_of_two_keys_bit_exact(G, name):
    """Power-of-two Galois keys (the paper's SEAL key set): every rotation a chain of
    its non-adjacent form, every linear combination rotate-then-multiply.  M7 (two
    samples) and LeNet-1 (one sample, incl. the rotation calls) at small rings,
    bit-exact against the oracle in the same mode; logits against the FP64 CNN."""
    if name == "M7":
        model, Wi, Hi = W.paper_model("M7")
        dims, ns = 1, 2
    else:
        model, Wi, Hi = W.lenet1(), 28, 28
        dims, ns = 2, 1
    stride, levels, steps = G.plan(model, Wi, Hi)
    logn = max(11, int(np.ceil(np.log2(stride * ns))) + 1)
    P = dict(logn=logn, data_bits=[60] + [40] * levels, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen_pow2()
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    he.keygen(ckks.pow2_steps(he.n // 2))
    x = W.images(ns, Hi, Wi) if dims == 2 else W.signals(ns, Wi)[:, 0]
    gct = ctx.encrypt(x, ns, stride, W.ENC_SEED)
    out = ctx.compile(model, Wi, Hi, ns).infer(gct, use_graph=True)
    lay = olayers.input_layout(Wi, Hi, stride, ns, he.n // 2, dims)
    oct_ = he.encrypt(slots_of(x, stride, he.n // 2), W.ENC_SEED)
    want, _ = olayers.run_model(olayers.HeBackend(he, naf=True), oct_, model, lay)
    assert_same(ctx, out, he, want[0])
    n_out = model[-1]["w"].shape[0]
    logits = ctx.decrypt(out, n_out)
    for b in range(ns):
        assert np.abs(logits[b] - cnn.forward(x[b], model, dims=dims)).max() < 1e-3
    if name == "lenet1":
        for r in (1, 27, -100, 511):
            assert_same(ctx, ctx.rotate(gct, r), he, he.rotate_naf(oct_, r))
        hs = ctx.rotate_hoisted(gct, [3, 7, 0])
        cache = {}
        for g, r in zip(hs, [3, 7, 0]):
            assert_same(ctx, g, he, he.rotate_naf(oct_, r, cache))


@pytest.mark.parametrize("co", [16, 17])
def test_flatten_merge_boundary_bit_exact(G, co):
    """A pooled flatten with 8 rows over 16 channels (merged with the packing: 128 steps)
    and over 17 (stages and packing separate): bit-exact against the oracle."""
    rng = np.random.default_rng(co)
    model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (co, 1, 5, 5)), "b": rng.normal(0, 0.1, co), "stride": 1},
             {"op": "square"}, {"op": "avgpool", "k": 3}, {"op": "flatten"},
             {"op": "fc", "w": rng.normal(0, 0.1, (10, co * 64)), "b": rng.normal(0, 0.1, 10)}]
    stride, levels, steps = G.plan(model, 28, 28)
    P = dict(logn=12, data_bits=[60] + [40] * levels, special_bits=[60, 60], dnum=3, log2_scale=40)
    ctx, he = make_pair(G, P, steps)
    img = W.images(1)
    out = ctx.compile(model, 28, 28, 1).infer(ctx.encrypt(img, 1, stride, W.ENC_SEED), use_graph=True)
    want = run_oracle_model(he, model, img, 28, 28, stride, 1, W.ENC_SEED)
    assert_same(ctx, out, he, want)
    assert np.abs(ctx.decrypt(out, 10)[0] - cnn.forward(img[0], model)).max() < 1e-3


@pytest.mark.parametrize("case", ["one_channel_pool", "1d_pool_merged"])
def test_flatten_shapes_bit_exact(G, case):
    """A one-channel flatten after pooling (no packing) and a 1-D pooled flatten whose single
    stage is merged with the packing of 4 channels: bit-exact against the oracle."""
    rng = np.random.default_rng(7)
    if case == "one_channel_pool":
        model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (1, 1, 5, 5)), "b": rng.normal(0, 0.1, 1), "stride": 1},
                 {"op": "avgpool", "k": 2}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (10, 144)), "b": rng.normal(0, 0.1, 10)}]
        x, Wi, Hi, dims = W.images(1), 28, 28, 2
    else:
        model = [{"op": "conv1d", "w": rng.normal(0, 0.1, (4, 1, 3)), "b": rng.normal(0, 0.1, 4), "stride": 1},
                 {"op": "square"}, {"op": "avgpool", "k": 2}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (5, 124)), "b": rng.normal(0, 0.1, 5)}]
        x, Wi, Hi, dims = W.signals(1, 64)[:, 0], 64, 1, 1
    stride, levels, steps = G.plan(model, Wi, Hi)
    P = dict(logn=11, data_bits=[60] + [40] * levels, special_bits=[60, 60], dnum=3, log2_scale=40)
    ctx, he = make_pair(G, P, steps)
    out = ctx.compile(model, Wi, Hi, 1).infer(ctx.encrypt(x, 1, stride, W.ENC_SEED), use_graph=True)
    want = run_oracle_model(he, model, x, Wi, Hi, stride, 1, W.ENC_SEED, dims=dims)
    assert_same(ctx, out, he, want)
    n_out = model[-1]["w"].shape[0]
    assert np.abs(ctx.decrypt(out, n_out)[0] - cnn.forward(x[0], model, dims=dims)).max() < 1e-3


def test_fc_shapes_bit_exact(G):
    """Alg. 2 with DAT_in < DAT_out (12 -> 20: W_vec = DAT_out, a one-term rotation sum),
    DAT_in = DAT_out (20 -> 20) and a width that is not a multiple (20 -> 7): bit-exact
    against the oracle, logits against the FP64 CNN."""
    rng = np.random.default_rng(11)
    model = [{"op": "conv1d", "w": rng.normal(0, 0.3, (2, 1, 3)), "b": rng.normal(0, 0.1, 2), "stride": 1},
             {"op": "flatten"},
             {"op": "fc", "w": rng.normal(0, 0.3, (20, 12)), "b": rng.normal(0, 0.1, 20)},
             {"op": "fc", "w": rng.normal(0, 0.3, (20, 20)), "b": rng.normal(0, 0.1, 20)},
             {"op": "fc", "w": rng.normal(0, 0.3, (7, 20)), "b": rng.normal(0, 0.1, 7)}]
    stride, levels, steps = G.plan(model, 8, 1)
    P = dict(logn=11, data_bits=[60] + [40] * levels, special_bits=[60, 60], dnum=3, log2_scale=40)
    ctx, he = make_pair(G, P, steps)
    x = W.signals(2, 8)[:, 0]
    out = ctx.compile(model, 8, 1, 2).infer(ctx.encrypt(x, 2, stride, W.ENC_SEED), use_graph=True)
    want = run_oracle_model(he, model, x, 8, 1, stride, 2, W.ENC_SEED, dims=1)
    assert_same(ctx, out, he, want)
    logits = ctx.decrypt(out, 7)
    for b in range(2):
        assert np.abs(logits[b] - cnn.forward(x[b], model, dims=1)).max() < 1e-3


@pytest.mark.parametrize("name", ["lenet1", "m5n"])
def test_mask_budget_streams_masks_bit_identical(G, name):
    """With a mask budget smaller than a convolution's masks, the masks are encoded at
    every inference in output-channel groups (here one channel per group): the
    ciphertexts equal the cached-mask model's, eagerly and through a CUDA graph."""
    if name == "lenet1":
        model, Wi, Hi, C = W.lenet1(), 28, 28, 1
        P = W.small_params("lenet1", 11)
    else:
        model, Wi, Hi, C = W.m5_narrow(), 32, 32, 3
        P = dict(logn=13, data_bits=[60] + [40] * 8, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    stride, levels, steps = G.plan(model, Wi, Hi)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    ct = ctx.encrypt(W.images(1, Hi, Wi, C=C), 1, stride, W.ENC_SEED)
    ref = ctx.export(ctx.compile(model, Wi, Hi, 1).infer(ct, use_graph=True))
    m = ctx.compile(model, Wi, Hi, 1)
    m.set_mask_budget(1)
    assert np.array_equal(ctx.export(m.infer(ct)), ref)
    assert np.array_equal(ctx.export(m.infer(ct, use_graph=True)), ref)
    assert np.array_equal(ctx.export(m.infer(ct, use_graph=True)), ref)


@pytest.mark.slow
def test_m5_ring_2_15_with_mask_budget(G):
    """M5 at N = 2^15 (five 3x32x32 samples per ciphertext): its convolutions' masks
    (~200 GB if kept) are encoded per inference within a 24 GB budget; logits against the
    FP64 CNN."""
    model, Wi, Hi = W.paper_model("M5")
    stride, levels, steps = G.plan(model, Wi, Hi)
    P = dict(logn=15, data_bits=[60] + [40] * levels, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    imgs = W.images(5, 32, 32, C=3)
    m = ctx.compile(model, Wi, Hi, 5)
    m.set_mask_budget(24 << 30)
    logits = ctx.decrypt(m.infer(ctx.encrypt(imgs, 5, stride, W.ENC_SEED), use_graph=True), 10)
    for b in range(5):
        assert np.abs(logits[b] - cnn.forward(imgs[b], model)).max() < 1e-3


def test_pack_and_drop_level_bit_exact(G):
    """Batch combining (Sec. III-B) of three ciphertexts carrying 1, 2 and 1 samples,
    and Drop-Level (Sec. IV-A): the chain has two more levels than M7 consumes, so
    the model drops them first.  Every ciphertext bit-exact against the oracle."""
    model, Wi, Hi = W.paper_model("M7")
    stride, levels, steps = G.plan(model, Wi, Hi)
    P = dict(logn=11, data_bits=[60] + [40] * (levels + 2), special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    ctx, he = make_pair(G, P, sorted(set(steps) | set(G.pack_steps(stride, 4))))
    sig = W.signals(4, Wi)[:, 0]
    groups = [sig[0:1], sig[1:3], sig[3:4]]
    gcts = [ctx.encrypt(g, len(g), stride, W.ENC_SEED + k) for k, g in enumerate(groups)]
    octs = [he.encrypt(slots_of(g, stride, he.n // 2), W.ENC_SEED + k) for k, g in enumerate(groups)]
    lays = [olayers.input_layout(Wi, Hi, stride, len(g), he.n // 2, 1) for g in groups]
    for g, o in zip(gcts, octs):
        assert_same(ctx, g, he, o)
    gp = ctx.pack(gcts)
    be = olayers.HeBackend(he)
    op, lay = olayers.pack(be, octs, lays)
    assert_same(ctx, gp, he, op)
    assert_same(ctx, ctx.drop_level(gp, 2), he, he.drop_level(he.drop_level(op)))
    out = ctx.compile(model, Wi, Hi, 4).infer(gp, use_graph=True)
    want, _ = olayers.run_model(be, op, model, lay)
    assert_same(ctx, out, he, want[0])
    logits = ctx.decrypt(out, 5)
    for b in range(4):
        assert np.abs(logits[b] - cnn.forward(sig[b], model, dims=1)).max() < 1e-3
    from paper_2402_03060_gb300 import HeError
    other = ctx.encrypt(sig[:1], 1, stride + 8, W.ENC_SEED)
    with pytest.raises(HeError):
        ctx.pack([gcts[0], other])                      # another stride
    with pytest.raises(HeError) as e:
        ctx.pack([gcts[1]] * 5)                         # 10 samples x 128 slots > 1024
    assert "HE_ESLOTS" in str(e.value)
    with pytest.raises(HeError):
        ctx.drop_level(gp, levels + 3)                  # more levels than the ciphertext has


def test_batched_equals_single_and_uneven_tail(G):
    """3 ciphertexts x 2 samples (5 samples: an uneven last ciphertext) in one
    batch give the same ciphertexts as each ciphertext alone."""
    P = W.small_params("lenet1", 12)
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    imgs = W.images(5)
    m = ctx.compile(model, 28, 28, 2)
    batch = ctx.encrypt(imgs, 2, stride, W.ENC_SEED)
    assert batch.batch == 3
    out = m.infer(batch, use_graph=True)
    ob = ctx.export(out)
    for b in range(3):
        single = ctx.encrypt(imgs[2 * b: 2 * b + 2], 2, stride, W.ENC_SEED + b)
        os_ = ctx.export(m.infer(single))
        assert np.array_equal(ob[b], os_[0])
    logits = ctx.decrypt(out, 10)
    for k in range(5):
        assert np.abs(logits[k] - cnn.forward(imgs[k], model)).max() < 1e-3


def test_layer_calls_match_model(G):
    """The layer-by-layer C calls give the compiled model's ciphertext."""
    P = W.small_params("lenet1", 11)
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    img = W.images(1)
    ct = ctx.encrypt(img, 1, stride, W.ENC_SEED)
    ref = ctx.export(ctx.compile(model, 28, 28, 1).infer(ct))
    x = ctx.conv2d([ct], model[0]["w"], model[0]["b"], 1)
    x = ctx.square(x)
    x = ctx.avgpool(x, 2)
    x = ctx.conv2d(x, model[3]["w"], model[3]["b"], 1)
    x = ctx.square(x)
    x = ctx.avgpool(x, 2)
    f = ctx.flatten(x)
    y = ctx.fc(f, model[7]["w"], model[7]["b"])
    assert np.array_equal(ctx.export(y), ref)


def test_cnn1d_logits(G):
    """The 1-D CNN workload at its configured size: N = 2^14, [60, 40 x 6 | 60], 32
    ciphertexts of two signals each (64 samples) in one graph launch; every sample's
    logits against the FP64 CNN, and one ciphertext of the batch equals it run alone."""
    P = W.PARAMS["cnn1d"]
    model = W.cnn1d()
    stride, levels, steps = G.plan(model, 1024, 1)
    ctx = G.Context(seed=W.KEY_SEED, **P)
    ctx.keygen(steps)
    sig = W.signals(64)[:, 0]
    m = ctx.compile(model, 1024, 1, 2)
    out = m.infer(ctx.encrypt(sig, 2, stride, W.ENC_SEED), use_graph=True)
    assert out.batch == 32
    logits = ctx.decrypt(out, 5)
    for k in range(64):
        assert np.abs(logits[k] - cnn.forward(sig[k], model, dims=1)).max() < 1e-3, k
    alone = m.infer(ctx.encrypt(sig[62:], 2, stride, W.ENC_SEED + 31))
    assert np.array_equal(ctx.export(out)[31], ctx.export(alone)[0])


def test_error_codes(G, pair_small):
    from paper_2402_03060_gb300 import HeError
    ctx, he = pair_small
    M = he.n // 2
    ct = ctx.encrypt(np.zeros((1, M)), 1, M, 1)
    with pytest.raises(HeError) as e:
        ctx.rotate(ct, 2)                  # no key for step 2
    assert e.value.status == 6
    one = ctx.rescale(ctx.rescale(ctx.rescale(ct)))
    with pytest.raises(HeError) as e:
        ctx.rescale(one)                   # one limb left
    assert e.value.status == 3
    with pytest.raises(HeError) as e:
        ctx.encrypt(np.zeros((3, 400)), 3, 400, 1)   # 1200 slots > 512
    assert e.value.status == 5
    with pytest.raises(HeError) as e:
        ctx.add(ct, ctx.rescale(ct))       # level mismatch
    assert e.value.status == 1


def test_degenerate_cases(G, pair_small):
    """Rotation by 0 and by N/2 (the identity Galois element), a hoisted set made
    only of the identity, a 1x1 convolution, an empty or out-of-range encryption."""
    from paper_2402_03060_gb300 import HeError
    ctx, he = pair_small
    M = he.n // 2
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (1, M))
    ct = ctx.encrypt(x, 1, M, 3)
    ref = ctx.export(ct)
    assert np.array_equal(ctx.export(ctx.rotate(ct, 0)), ref)
    assert np.array_equal(ctx.export(ctx.rotate(ct, M)), ref)
    hs = ctx.rotate_hoisted(ct, [0, 0])
    assert np.array_equal(ctx.export(hs[0]), ref) and np.array_equal(ctx.export(hs[1]), ref)
    # 1x1 convolution: one plaintext product per output, no rotation, no key needed
    w = np.full((2, 1, 1, 1), 0.5)
    b = np.array([0.0, 0.25])
    img = rng.uniform(0, 1, (1, 4, 4))
    c2 = ctx.encrypt(img, 1, 16, 4)
    outs = ctx.conv2d([c2], w, b)
    for o in range(2):
        got = ctx.decrypt(outs[o], 16)[0]
        assert np.abs(got - (0.5 * img[0].reshape(-1) + b[o])).max() < 1e-6
    with pytest.raises(HeError):
        ctx.encrypt(np.zeros((0, 16)), 1, 16, 1)     # no samples
    with pytest.raises(HeError):
        ctx.conv2d([c2], np.zeros((1, 1, 5, 5)), np.zeros(1))   # kernel larger than the image


@pytest.mark.slow
def test_lenet1_full_size_bit_exact(G):
    """The benchmark's launch configuration: LeNet-1 at N=16384, 633 samples in 64
    ciphertexts (the last with 3), autotuned launch shapes, one graph launch.  The first
    and the ragged last ciphertext are compared with the oracle run on each alone."""
    P = W.PARAMS["lenet1"]
    model = W.lenet1()
    stride, levels, steps = G.plan(model, 28, 28)
    ctx, he = make_pair(G, P, steps)
    ctx.autotune()
    imgs = W.images(633)
    m = ctx.compile(model, 28, 28, 10)
    out = m.infer(ctx.encrypt(imgs, 10, stride, W.ENC_SEED), use_graph=True)
    assert out.batch == 64
    for b in (0, 63):
        want = run_oracle_model(he, model, imgs[10 * b: 10 * b + 10], 28, 28, stride, 10, W.ENC_SEED + b)
        assert_same(ctx, out, he, want, b)
    logits = ctx.decrypt(out, 10)
    for k in list(range(10)) + [630, 631, 632]:
        assert np.abs(logits[k] - cnn.forward(imgs[k], model)).max() < 1e-3


def test_maximum_sizes_bit_exact(G):
    """The largest chain the library takes (32 data primes, 4 special primes) with the
    widest digits (alpha = 8 limbs, dnum = 4) and with the most digits (dnum = 16):
    encrypt, hoisted and single rotations, square, rescale, bit-exact against the oracle."""
    for dnum in (4, 16):
        P = dict(logn=11, data_bits=[30] * 32, special_bits=[60] * 4, dnum=dnum, log2_scale=25)
        steps = [1, -7, 300]
        ctx, he = make_pair(G, P, steps)
        M = he.n // 2
        x = np.random.default_rng(dnum).uniform(-1, 1, (1, M))
        g = ctx.encrypt(x, 1, M, 11)
        o = he.encrypt(x[0], 11)
        assert_same(ctx, g, he, o)
        for r in steps:
            assert_same(ctx, ctx.rotate(g, r), he, he.rotate(o, r))
        # the chain is meaningful too: a digit of 8 x 30 bits against P of 240 bits
        assert np.abs(ctx.decrypt(ctx.rotate(g, 300), M)[0] - np.roll(x[0], -300)).max() < 0.05
        hs = ctx.rotate_hoisted(g, steps)
        ho = he.rotate_hoisted(o, steps)
        for gr, r in zip(hs, steps):
            assert_same(ctx, gr, he, ho[r])
        assert_same(ctx, ctx.square([g])[0], he, he.square(o))
        assert_same(ctx, ctx.rescale(g), he, he.rescale(o))
