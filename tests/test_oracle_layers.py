"""Pins of the layer algorithms (Alg. 1, Alg. 2, Sec. IV-C/E) on the cleartext
slot simulator: results equal the FP64 direct CNN (itself checked against
torch.nn.functional in float64), levels equal the paper's #Mult tables, and
operation counts follow the paper's complexity statements."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import cnn, layers, slotsim

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def build_model(spec_layers, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for l in spec_layers:
        if l[0] == "conv2d":
            _, ci, co, k, s = l
            out.append({"op": "conv2d", "w": rng.normal(0, 0.1, (co, ci, k, k)), "b": rng.normal(0, 0.1, co), "stride": s})
        elif l[0] == "conv1d":
            _, ci, co, k, s = l
            out.append({"op": "conv1d", "w": rng.normal(0, 0.1, (co, ci, k)), "b": rng.normal(0, 0.1, co), "stride": s})
        elif l[0] == "fc":
            _, din, dout = l
            out.append({"op": "fc", "w": rng.normal(0, 0.1, (dout, din)), "b": rng.normal(0, 0.1, dout)})
        elif l[0] == "avgpool":
            out.append({"op": "avgpool", "k": l[1]})
        else:
            out.append({"op": l[0]})
    return out


def pack(samples, stride, slots):
    x = np.zeros(slots)
    for b, s in enumerate(samples):
        f = np.asarray(s).reshape(-1)
        x[b * stride: b * stride + f.size] = f
    return x


def run_sim(model, samples, W_img, H_img, dims, slots, channels=1):
    pl = layers.plan(model, W_img, H_img, dims)
    lay = layers.input_layout(W_img, H_img, pl["stride"], len(samples), slots, dims, channels)
    be = slotsim.SlotSim()
    x = be.wrap(pack(samples, pl["stride"], slots))
    ys, lay = layers.run_model(be, x, model, lay)
    return ys[0], lay, be, pl


def test_cnn_against_torch():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    model = W.lenet1()
    x = W.images(1)[0]
    t = torch.tensor(x, dtype=torch.float64)[None, None]
    for l in model:
        if l["op"] == "conv2d":
            t = F.conv2d(t, torch.tensor(l["w"]), torch.tensor(l["b"]), stride=l["stride"])
        elif l["op"] == "square":
            t = t * t
        elif l["op"] == "avgpool":
            t = F.avg_pool2d(t, l["k"])
        elif l["op"] == "flatten":
            t = t.reshape(1, -1)
        elif l["op"] == "fc":
            t = F.linear(t, torch.tensor(l["w"]), torch.tensor(l["b"]))
    assert np.abs(t.numpy().reshape(-1) - cnn.forward(x, model)).max() < 1e-12
    m1 = W.cnn1d()
    s = W.signals(1)[0]
    t = torch.tensor(s, dtype=torch.float64)[None]
    for l in m1:
        if l["op"] == "conv1d":
            t = F.conv1d(t, torch.tensor(l["w"]), torch.tensor(l["b"]), stride=l["stride"])
        elif l["op"] == "square":
            t = t * t
        elif l["op"] == "avgpool":
            t = F.avg_pool1d(t, l["k"])
        elif l["op"] == "flatten":
            t = t.reshape(1, -1)
        elif l["op"] == "fc":
            t = F.linear(t.reshape(1, -1), torch.tensor(l["w"]), torch.tensor(l["b"]))
    assert np.abs(t.numpy().reshape(-1) - cnn.forward(s[0], m1, dims=1)).max() < 1e-12
    # three input channels (M5, CIFAR-10 shaped)
    m5, _, _ = W.paper_model("M5")
    x3 = W.images(1, 32, 32, C=3)[0]
    t = torch.tensor(x3, dtype=torch.float64)[None]
    for l in m5:
        if l["op"] == "conv2d":
            t = F.conv2d(t, torch.tensor(l["w"]), torch.tensor(l["b"]), stride=l["stride"])
        elif l["op"] == "square":
            t = t * t
        elif l["op"] == "avgpool":
            t = F.avg_pool2d(t, l["k"])
        elif l["op"] == "flatten":
            t = t.reshape(1, -1)
        elif l["op"] == "fc":
            t = F.linear(t, torch.tensor(l["w"]), torch.tensor(l["b"]))
    assert np.abs(t.numpy().reshape(-1) - cnn.forward(x3, m5)).max() < 1e-12


@pytest.mark.parametrize("name", ["lenet1", "cnn1d", "cnn1d_tree", "lenet5", "m3", "M1", "M4", "m5n", "M6", "M7"])
def test_slot_algorithms_equal_direct_cnn(name):
    channels = 1
    if name == "m5n":
        model, Wi, Hi, dims, slots, channels = W.m5_narrow(), 32, 32, 2, 8192, 3
        gen = lambda n: W.images(n, 32, 32, C=3)
    elif name in ("M4", "M6"):
        model, Wi, Hi = W.paper_model(name)
        dims, slots = 2, 8192
        gen = lambda n: W.images(n, Hi, Wi)
    elif name == "lenet1":
        model, Wi, Hi, dims, slots = W.lenet1(), 28, 28, 2, 8192
        gen = lambda n: W.images(n)
    elif name == "m3":
        model, Wi, Hi, dims, slots = W.m3_relu(), 28, 28, 2, 8192
        gen = lambda n: W.images(n)
    elif name.startswith("cnn1d"):
        model = W.cnn1d(fc_sum="tree" if name.endswith("tree") else "linear")
        Wi, Hi, dims, slots = 1024, 1, 1, 8192
        gen = lambda n: W.signals(n)[:, 0]
    elif name == "lenet5":
        model, Wi, Hi, dims, slots = W.lenet5_sq(), 32, 32, 2, 16384
        gen = lambda n: W.images(n, 32, 32)
    elif name == "M1":
        model, Wi, Hi, dims, slots = build_model(GOLD["mult_per_layer"]["M1"]["layers"]), 28, 28, 2, 8192
        gen = lambda n: W.images(n)
    else:
        model, Wi, Hi, dims, slots = build_model(GOLD["mult_per_layer"]["M7"]["layers"]), 128, 1, 1, 4096
        gen = lambda n: W.signals(n, 128)[:, 0]
    pl = layers.plan(model, Wi, Hi, dims)
    ns = slots // pl["stride"]
    samples = gen(ns)
    y, lay, be, _ = run_sim(model, samples, Wi, Hi, dims, slots, channels)
    for b in range(ns):
        ref = cnn.forward(samples[b], model, dims=dims)
        got = y.v[b * pl["stride"]: b * pl["stride"] + len(ref)]
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    # packing changes nothing: sample 0 alone gives the same numbers
    y1, _, _, _ = run_sim(model, samples[:1], Wi, Hi, dims, slots, channels)
    assert np.abs(y1.v[:len(ref)] - y.v[:len(ref)]).max() < 1e-12


def _narrow(spec, cap=8):
    """The same layer sequence with at most `cap` channels per convolution (levels
    and layouts do not depend on channel counts); the first FC shrinks with them."""
    out, ch, ch_orig = [], None, None
    for l in spec:
        if l[0] == "conv2d":
            co = min(l[2], cap)
            out.append(["conv2d", l[1] if ch is None else ch, co, l[3], l[4]])
            ch, ch_orig = co, l[2]
        elif l[0] == "fc" and ch_orig is not None:
            out.append(["fc", l[1] * ch // ch_orig, l[2]])
            ch_orig = None
        else:
            out.append(list(l))
    return out


@pytest.mark.parametrize("name", ["M1", "M2", "M3", "M4", "M5", "M6", "M7"])
def test_levels_per_layer_match_paper_tables(name):
    g = GOLD["mult_per_layer"][name]
    model = build_model(g["layers"])
    Wi, Hi = g["input"]
    C = g.get("channels", 1)
    dims = 1 if Hi == 1 else 2
    pl = layers.plan(model, Wi, Hi, dims)
    assert pl["levels"] == g["total"]
    if C > 1:        # run the channel-narrowed copy (128 full-size channels are too big here)
        model = build_model(_narrow(g["layers"]))
        pl = layers.plan(model, Wi, Hi, dims)
    slots = 1 << max(11, int(np.ceil(np.log2(pl["stride"]))))
    lay = layers.input_layout(Wi, Hi, pl["stride"], 1, slots, dims, C)
    be = slotsim.SlotSim()
    x0 = W.images(1, Hi, Wi, C=C) if dims == 2 else W.signals(1, Wi)[:, 0]
    xs = [be.wrap(pack(x0, pl["stride"], slots))]
    used = []
    for spec in model:
        before = xs[0].used
        xs, lay = layers.run_layers(be, xs, [spec], lay)
        used.append(xs[0].used - before)
    assert used == g["mult"], (used, g["mult"])
    assert sum(used) == g["total"] == pl["levels"]


def test_batch_capacity_matches_paper():
    g = GOLD["batch_capacity"]
    model = build_model(GOLD["mult_per_layer"][g["model"]]["layers"])
    pl = layers.plan(model, 28, 28)
    assert g["slots"] // pl["stride"] == g["samples"]
    # LeNet-1 (M2) packs the same 10 images per ciphertext
    assert 8192 // layers.plan(W.lenet1(), 28, 28)["stride"] == 10


def _counts(model, Wi, Hi, dims=2, slots=8192):
    _, _, be, _ = run_sim(model, W.images(1, Hi, Wi) if dims == 2 else W.signals(1, Wi)[:, 0], Wi, Hi, dims, slots)
    return be.count


@pytest.mark.parametrize("ci,co,k", [(1, 4, 5), (4, 12, 5), (2, 3, 3)])
def test_conv_operation_counts(ci, co, k):
    """Sec. IV-B: CH_in*CH_out*K^2 plaintext products, CH_in*K^2 rotations (one is the identity)."""
    model = [{"op": "conv2d", "w": np.ones((co, ci, k, k)) * 0.1, "b": np.zeros(co), "stride": 1}]
    rng = np.random.default_rng(0)
    pl = layers.plan(model, 28, 28)
    lay = layers.input_layout(28, 28, pl["stride"], 1, 8192)
    be = slotsim.SlotSim()
    xs = [be.wrap(pack([rng.uniform(size=(28, 28))], pl["stride"], 8192)) for _ in range(ci)]
    ys, lay = layers.conv(be, xs, model[0]["w"], model[0]["b"], 1, lay)
    assert be.count["pmul"] == ci * co * k * k
    assert be.count["rot"] == ci * (k * k - 1)
    assert be.count["rescale"] == co


@pytest.mark.parametrize("din,dout", [(64, 10), (192, 10), (648, 64), (120, 84), (4080, 5), (5, 10), (10, 10), (7, 3), (1, 4)])
def test_fc_operation_counts(din, dout):
    """Sec. IV-D: O(DAT_out) products and O(DAT_in/DAT_out + DAT_out) rotations."""
    rng = np.random.default_rng(1)
    M = rng.normal(size=(dout, din))
    Wv = -(-din // dout) * dout
    # slots >= 2 * W_vec, so that no step o - W_vec coincides with a step o modulo the slots
    lay = layers.Layout(W_img=din, H_img=1, W=din, H=1, I=1, stride=max(Wv, din), n_samples=1,
                        slots=1 << int(np.ceil(np.log2(2 * max(Wv, din)))), dims=1, prev="flatten", D=din)
    be = slotsim.SlotSim()
    x = np.zeros(lay.slots)
    x[:din] = rng.normal(size=din)
    ys, _ = layers.fc(be, [be.wrap(x)], M, np.zeros(dout), lay)
    assert np.abs(ys[0].v[:dout] - M @ x[:din]).max() < 1e-9
    assert be.count["pmul"] == 2 * dout - 1
    assert be.count["rot"] == 2 * (dout - 1) + (Wv // dout - 1)
    if (din, dout) == (GOLD["fc_example"]["din"], GOLD["fc_example"]["dout"]):
        assert be.count["pmul"] < 2 * dout and be.count["pmul"] < din


def test_avgpool_uses_no_level_and_leaves_invalid_values():
    lay = layers.input_layout(28, 28, 784, 1, 1024)
    be = slotsim.SlotSim()
    x = be.wrap(pack([W.images(1)[0]], 784, 1024))
    ys, lay2 = layers.avgpool(be, [x], 2, lay)
    assert ys[0].used == 0 and lay2.pending == 0.25 and lay2.I == 2
    img = W.images(1)[0]
    got = np.array([[ys[0].v[2 * (r * 28 + c)] for c in range(14)] for r in range(14)])
    want = 4 * cnn.avgpool(img[None], 2)[0]
    assert np.abs(got - want).max() < 1e-12
    # between the valid outputs the slots hold non-zero "invalid values" (Sec. IV-C)
    assert abs(ys[0].v[1]) > 0


def test_plan_stride_lenet1():
    pl = layers.plan(W.lenet1(), 28, 28)
    assert pl["stride"] == 784 and pl["levels"] == 7


@pytest.mark.parametrize("m", [1, 2, 3, 7, 8, 9, 20, 816])
def test_tree_rotation_sum(m):
    """The binary form of Alg. 2's final sum gives the slot sums of the printed
    form, with about log2(m) + popcount(m) rotations instead of m - 1."""
    rng = np.random.default_rng(m)
    slots, d = 8192, 5
    v = rng.normal(size=slots)
    lin, tree = slotsim.SlotSim(), slotsim.SlotSim()
    a = layers.rotation_sum(lin, lin.wrap(v), d, m, "linear")
    b = layers.rotation_sum(tree, tree.wrap(v), d, m, "tree")
    direct = sum(np.roll(v, -i * d) for i in range(m))
    assert np.abs(a.v - direct).max() < 1e-9 and np.abs(b.v - direct).max() < 1e-9
    n_rot = (m.bit_length() - 1) + bin(m).count("1") - 1
    assert tree.count["rot"] == n_rot == len(layers.tree_steps(d, m))


def test_approx_relu_folds_the_pooling_factor():
    """f(p x) for a pending factor p: approx_relu after avgpool equals the FP64
    f applied to the average (Sec. IV-C), and its constant term sits only at the
    valid slots."""
    rng = np.random.default_rng(9)
    model = [{"op": "conv2d", "w": rng.normal(0, 0.3, (2, 1, 3, 3)), "b": rng.normal(0, 0.1, 2), "stride": 1},
             {"op": "avgpool", "k": 2}, {"op": "approx_relu"}, {"op": "flatten"}]
    img = W.images(1)
    y, lay, be, _ = run_sim(model, img, 28, 28, 2, 2048)
    ref = cnn.forward(img[0], model)
    assert np.abs(y.v[:len(ref)] - ref).max() < 1e-12
    assert np.all(y.v[len(ref):lay.stride] == 0)


@pytest.mark.parametrize("co", [16, 17])
def test_flatten_merge_boundary_on_the_slot_simulator(co):
    """Pooled flatten with 8 rows: merged with the packing of 16 channels (128 steps), kept
    separate for 17 (136): both equal the FP64 CNN."""
    rng = np.random.default_rng(co)
    model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (co, 1, 5, 5)), "b": rng.normal(0, 0.1, co), "stride": 1},
             {"op": "square"}, {"op": "avgpool", "k": 3}, {"op": "flatten"},
             {"op": "fc", "w": rng.normal(0, 0.1, (10, co * 64)), "b": rng.normal(0, 0.1, 10)}]
    img = W.images(1)
    y, _, be, pl = run_sim(model, img, 28, 28, 2, 2048)
    ref = cnn.forward(img[0], model)
    assert np.abs(y.v[:10] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("case", ["1d_pool_merged", "1d_pool_separate", "conv_two_stages_separate",
                                  "one_channel_pool", "one_channel_conv", "odd_pool"])
def test_flatten_variants_on_the_slot_simulator(case):
    """Flatten after 1-D pooling (one masked stage, merged with the packing of 4 channels or
    kept separate for 40: 32 * 40 > 128 steps) and after a strided 2-D convolution with two
    masked stages over 17 channels (kept separate): equal to the FP64 CNN."""
    rng = np.random.default_rng(7)
    if case.startswith("1d"):
        co = 4 if case.endswith("merged") else 40
        model = [{"op": "conv1d", "w": rng.normal(0, 0.1, (co, 1, 3)), "b": rng.normal(0, 0.1, co), "stride": 1},
                 {"op": "square"}, {"op": "avgpool", "k": 2}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (5, co * 31)), "b": rng.normal(0, 0.1, 5)}]
        x, Wi, Hi, dims = W.signals(1, 64)[:, 0], 64, 1, 1
    elif case == "odd_pool":   # 27 x 27 after the convolution: pooling by 2 drops the last row and column
        model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (3, 1, 2, 2)), "b": rng.normal(0, 0.1, 3), "stride": 1},
                 {"op": "square"}, {"op": "avgpool", "k": 2}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (10, 3 * 169)), "b": rng.normal(0, 0.1, 10)}]
        x, Wi, Hi, dims = W.images(1), 28, 28, 2
    elif case == "one_channel_pool":
        model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (1, 1, 5, 5)), "b": rng.normal(0, 0.1, 1), "stride": 1},
                 {"op": "avgpool", "k": 2}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (10, 144)), "b": rng.normal(0, 0.1, 10)}]
        x, Wi, Hi, dims = W.images(1), 28, 28, 2
    elif case == "one_channel_conv":
        model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (1, 1, 4, 4)), "b": rng.normal(0, 0.1, 1), "stride": 3},
                 {"op": "flatten"}, {"op": "fc", "w": rng.normal(0, 0.1, (10, 81)), "b": rng.normal(0, 0.1, 10)}]
        x, Wi, Hi, dims = W.images(1), 28, 28, 2
    else:
        model = [{"op": "conv2d", "w": rng.normal(0, 0.1, (17, 1, 4, 4)), "b": rng.normal(0, 0.1, 17), "stride": 3},
                 {"op": "square"}, {"op": "flatten"},
                 {"op": "fc", "w": rng.normal(0, 0.1, (10, 17 * 81)), "b": rng.normal(0, 0.1, 10)}]
        x, Wi, Hi, dims = W.images(1), 28, 28, 2
    pl = layers.plan(model, Wi, Hi, dims)
    y, _, _, _ = run_sim(model, x, Wi, Hi, dims, 1 << max(11, int(np.ceil(np.log2(pl["stride"])))))
    ref = cnn.forward(x[0], model, dims=dims)
    assert np.abs(y.v[:len(ref)] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_approx_relu_coefficients_are_the_papers():
    """Both oracle parts (the layer algorithm and the FP64 CNN) use the printed polynomial,
    and after average pooling by c the layer's coefficients are the paper's folded ones."""
    g = GOLD["approx_relu"]
    assert (layers.RELU_C0, layers.RELU_C1, layers.RELU_C2) == (g["c0"], g["c1"], g["c2"])
    x = np.linspace(-3, 3, 13)
    got = cnn.forward(x.reshape(1, -1), [{"op": "approx_relu"}])
    assert np.array_equal(got, g["c0"] + g["c1"] * x + g["c2"] * x * x)
    # one pooled value v = mean of a c x c block: the layer sees the block sum s = c^2 v with p = 1/c^2
    for c in (2, 3):
        s = 1.7
        folded = g["c0"] + g["c1"] / c ** 2 * s + g["c2"] / c ** 4 * s * s
        p = 1.0 / c ** 2
        assert abs((layers.RELU_C0 + layers.RELU_C1 * p * s + layers.RELU_C2 * p * p * s * s) - folded) < 1e-15


@pytest.mark.parametrize("name", ["M1", "M4", "M5", "M6", "M7"])
def test_workload_shapes_are_the_paper_tables(name):
    """The workloads' model builders use exactly the layer parameters of the paper's tables
    (golden fixture), and the input size each table implies."""
    g = GOLD["mult_per_layer"][name]
    spec, Wi, Hi = W.PAPER_MODELS[name]
    assert [list(l) for l in spec] == g["layers"]
    assert [Wi, Hi] == g["input"]
    model, _, _ = W.paper_model(name)
    for l, m in zip(g["layers"], model):
        assert m["op"] == l[0]
        if l[0] in ("conv2d", "conv1d"):
            assert m["w"].shape[:2] == (l[2], l[1]) and m["w"].shape[-1] == l[3] and m["stride"] == l[4]
        elif l[0] == "fc":
            assert m["w"].shape == (l[2], l[1])
        elif l[0] == "avgpool":
            assert m["k"] == l[1]


@pytest.mark.parametrize("name,build", [("M2", W.lenet1), ("M3", W.m3_relu)])
def test_lenet1_and_m3_builders_are_the_paper_tables(name, build):
    g = GOLD["mult_per_layer"][name]
    model = build()
    assert [m["op"] for m in model] == [l[0] for l in g["layers"]]
    for l, m in zip(g["layers"], model):
        if l[0] == "conv2d":
            assert m["w"].shape == (l[2], l[1], l[3], l[3]) and m["stride"] == l[4]
        elif l[0] == "fc":
            assert m["w"].shape == (l[2], l[1])
        elif l[0] == "avgpool":
            assert m["k"] == l[1]
