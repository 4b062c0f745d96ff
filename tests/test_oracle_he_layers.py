"""The CKKS oracle running the paper's layers: decrypted results against the
FP64 direct CNN (paper Sec. VII validation), packed samples against single
samples, and levels consumed."""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, cnn, layers


def _enc_run(P, model, samples, Wi, Hi, dims=2, mode="hoisted", n_slots_samples=None):
    pl = layers.plan(model, Wi, Hi, dims)
    steps = pl["steps"]
    if mode == "incremental":
        steps = sorted(set(steps) | {1, Wi - np.asarray(model[0]["w"]).shape[-1] + 1})
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    he.keygen(steps)
    slots = he.n // 2
    ns = n_slots_samples or len(samples)
    lay = layers.input_layout(Wi, Hi, pl["stride"], ns, slots, dims)
    x = np.zeros(slots)
    for b, s in enumerate(samples):
        x[b * pl["stride"]: b * pl["stride"] + np.asarray(s).size] = np.asarray(s).reshape(-1)
    ct = he.encrypt(x, W.ENC_SEED)
    be = layers.HeBackend(he)
    ys, lay2 = layers.run_model(be, ct, model, lay, conv_mode=mode)
    return he, ys, lay2, pl, be


def test_single_conv_incremental_full_size():
    """Single-convolution workload: N=8192, [60,40,40 | 60], one 5x5 kernel, incremental rotations."""
    model = W.single_conv()
    img = W.images(1)[0]
    he, ys, lay, pl, be = _enc_run(W.PARAMS["conv1"], model, [img], 28, 28, mode="incremental")
    dec = he.decrypt(ys[0])
    ref = cnn.forward(img, model)             # 24 x 24
    got = np.array([dec[r * 28 + c] for r in range(24) for c in range(24)])
    assert np.abs(got - ref).max() < 1e-6
    # the chain has two levels, the model needs one: Drop-Level (Sec. IV-A) removes the other first
    assert ys[0].lp == 1 and be.count["rot"] == 24 and be.count["pmul"] == 25


def test_lenet1_small_ring_logits():
    P = W.small_params("lenet1", 11)
    model = W.lenet1()
    img = W.images(1)[0]
    he, ys, lay, pl, be = _enc_run(P, model, [img], 28, 28)
    assert ys[0].lp == 1       # 8 data primes, 7 levels consumed
    dec = he.decrypt(ys[0])[:10]
    assert np.abs(dec - cnn.forward(img, model)).max() < 1e-3


def test_packed_samples_equal_single():
    P = dict(W.PARAMS["conv1"])
    P["logn"] = 12            # 2048 slots: two 784-slot samples
    model = W.single_conv()
    imgs = W.images(2)
    he, ys, _, pl, _ = _enc_run(P, model, imgs, 28, 28, n_slots_samples=2)
    dec2 = he.decrypt(ys[0])
    he1, ys1, _, _, _ = _enc_run(P, model, imgs[:1], 28, 28, n_slots_samples=2)
    dec1 = he1.decrypt(ys1[0])
    idx = np.array([r * 28 + c for r in range(24) for c in range(24)])
    assert np.abs(dec2[idx] - dec1[idx]).max() < 1e-6
    for b in range(2):
        ref = cnn.forward(imgs[b], model)
        assert np.abs(dec2[b * 784 + idx] - ref.reshape(-1)).max() < 1e-6


def test_pack_on_the_slot_simulator_equals_packed_encryption():
    """Sec. III-B on cleartext: single-sample vectors rotated right by i*stride and
    added are exactly the multi-sample layout, and the model gives the same outputs."""
    from oracle import slotsim
    model, Wi, Hi = W.paper_model("M7")
    pl = layers.plan(model, Wi, Hi, 1)
    slots, n = 1024, 5
    sig = W.signals(n, Wi)[:, 0]
    be = slotsim.SlotSim()
    singles = []
    for s in sig:
        v = np.zeros(slots)
        v[:Wi] = s
        singles.append(be.wrap(v))
    lays = [layers.input_layout(Wi, Hi, pl["stride"], 1, slots, 1)] * n
    y, lay = layers.pack(be, singles, lays)
    assert lay.n_samples == n
    want = np.zeros(slots)
    for b, s in enumerate(sig):
        want[b * pl["stride"]: b * pl["stride"] + Wi] = s
    assert np.array_equal(y.v, want)
    out, _ = layers.run_model(be, y, model, lay)
    for b in range(n):
        ref = cnn.forward(sig[b], model, dims=1)
        assert np.abs(out[0].v[b * pl["stride"]: b * pl["stride"] + 5] - ref).max() < 1e-12


def test_pack_and_drop_level_on_ciphertexts():
    """Sec. III-B and IV-A on the CKKS oracle: three ciphertexts (1, 2 and 1 samples)
    packed into one decrypt to the concatenation; encrypted with two more levels than
    the model needs, the model drops them first (same final level as an exact chain)
    and every sample's logits match the FP64 CNN."""
    model, Wi, Hi = W.paper_model("M7")
    pl = layers.plan(model, Wi, Hi, 1)
    L = pl["levels"] + 2
    P = dict(logn=11, data_bits=[60] + [40] * L, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    stride, slots = pl["stride"], 1024
    he.keygen(sorted(set(pl["steps"]) | set(layers.pack_steps(stride, 4))))
    sig = W.signals(4, Wi)[:, 0]
    groups = [sig[0:1], sig[1:3], sig[3:4]]
    cts, lays = [], []
    for k, g in enumerate(groups):
        x = np.zeros(slots)
        for b, s in enumerate(g):
            x[b * stride: b * stride + Wi] = s
        cts.append(he.encrypt(x, W.ENC_SEED + k))
        lays.append(layers.input_layout(Wi, Hi, stride, len(g), slots, 1))
    be = layers.HeBackend(he)
    y, lay = layers.pack(be, cts, lays)
    assert lay.n_samples == 4 and y.lp == L + 1
    want = np.zeros(slots)
    for b, s in enumerate(sig):
        want[b * stride: b * stride + Wi] = s
    assert np.abs(he.decrypt(y) - want).max() < 1e-6
    # Drop-Level leaves the message untouched (decryption reads limb q_0 alone)
    assert np.array_equal(he.decrypt(he.drop_level(y)), he.decrypt(y))
    out, _ = layers.run_model(be, y, model, lay)
    assert out[0].lp == 1
    dec = he.decrypt(out[0])
    for b in range(4):
        ref = cnn.forward(sig[b], model, dims=1)
        assert np.abs(dec[b * stride: b * stride + 5] - ref).max() < 1e-3


def test_three_channel_input_logits():
    """M5's layer sequence (channel-narrowed) on a 3x32x32 input encrypted as one
    ciphertext, channel-major (Sec. III-A): the first convolution reads channel i
    through the extra rotation i*32*32; logits against the FP64 CNN."""
    model = W.m5_narrow()
    pl = layers.plan(model, 32, 32)
    assert pl["stride"] == 3 * 32 * 32 and pl["levels"] == 8
    P = dict(logn=13, data_bits=[60] + [40] * 8, special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    he.keygen(pl["steps"])
    img = W.images(1, 32, 32, C=3)
    x = np.zeros(he.n // 2)
    x[: img[0].size] = img[0].reshape(-1)
    lay = layers.input_layout(32, 32, pl["stride"], 1, he.n // 2, 2, channels=3)
    ys, _ = layers.run_model(layers.HeBackend(he), he.encrypt(x, W.ENC_SEED), model, lay)
    assert np.abs(he.decrypt(ys[0])[:10] - cnn.forward(img[0], model)).max() < 1e-3


def test_power_of_two_keys_model_logits():
    """The 1-D M7 with power-of-two Galois keys only (every rotation a chain of its
    non-adjacent form, linear combinations as rotate-then-multiply): logits against
    the FP64 CNN, with far fewer keys than the per-step set."""
    model, Wi, Hi = W.paper_model("M7")
    pl = layers.plan(model, Wi, Hi, 1)
    P = dict(logn=11, data_bits=[60] + [40] * pl["levels"], special_bits=[60, 60, 60], dnum=3, log2_scale=40)
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    keys = ckks.pow2_steps(he.n // 2)
    assert len(set(keys)) < len(pl["steps"])
    he.keygen(keys)
    sig = W.signals(2, Wi)[:, 0]
    x = np.zeros(he.n // 2)
    for b in range(2):
        x[b * pl["stride"]: b * pl["stride"] + Wi] = sig[b]
    lay = layers.input_layout(Wi, Hi, pl["stride"], 2, he.n // 2, 1)
    ys, _ = layers.run_model(layers.HeBackend(he, naf=True), he.encrypt(x, W.ENC_SEED), model, lay)
    dec = he.decrypt(ys[0])
    for b in range(2):
        ref = cnn.forward(sig[b], model, dims=1)
        assert np.abs(dec[b * pl["stride"]: b * pl["stride"] + 5] - ref).max() < 1e-3


def test_merged_flatten_packing_decrypts_like_separate_stages(monkeypatch):
    """The flatten's last masked stage merged with the channel packing (one combination,
    one ModDown) and evaluated separately (stage, rescale, then the packing) decrypt to
    the same values on the CKKS oracle; the ciphertexts differ only by key-switch rounding."""
    model = W.lenet1()[:7]                          # up to and including the flatten
    pl = layers.plan(W.lenet1(), 28, 28)
    P = W.small_params("lenet1", 11)
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    steps = set(pl["steps"])
    monkeypatch.setattr(layers, "MERGE_MAX_STEPS", 0)
    steps |= set(layers.plan(W.lenet1(), 28, 28)["steps"])
    he.keygen(sorted(steps))
    img = W.images(1)
    x = np.zeros(he.n // 2)
    x[:784] = img[0].reshape(-1)
    lay = layers.input_layout(28, 28, pl["stride"], 1, he.n // 2)
    ct = he.encrypt(x, W.ENC_SEED)
    sep, _ = layers.run_model(layers.HeBackend(he), ct, model, lay)
    monkeypatch.setattr(layers, "MERGE_MAX_STEPS", 128)
    mer, lay2 = layers.run_model(layers.HeBackend(he), ct, model, lay)
    assert mer[0].lp == sep[0].lp and abs(mer[0].scale - sep[0].scale) < 1e-9 * sep[0].scale
    a, b = he.decrypt(mer[0])[:192], he.decrypt(sep[0])[:192]
    assert np.abs(a - b).max() < 1e-6 and not np.array_equal(mer[0].d, sep[0].d)
    # and both are the FP64 CNN's flattened features
    feats = cnn.forward(img[0], model)
    assert np.abs(a - feats).max() < 1e-4
