"""The paper-order ("literal") schedule of the CKKS oracle, and the fused schedule
pinned against it.

The literal schedule evaluates each layer in the order the paper lists it (Alg. 1,
Sec. IV-C, Sec. IV-E, Alg. 2): every Rot is its own key switch, Mul (P) by the mask
over Q_l, Add, then the centred rescale of reading C7; square = tensor, relinearise,
rescale.  It is pinned by decryption against the FP64 CNN.  The fused schedule
(hoisting, one ModDown per output, ModDown and rescale as one division by q_top * P,
the merged flatten) is a different evaluation order of the same slot algebra: its
decrypted outputs must agree with the literal schedule's within the noise, while its
ciphertext bits differ.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ckks, cnn, layers


@pytest.fixture(scope="module")
def he():
    h = ckks.Ckks(logn=10, data_bits=[60, 40, 40], special_bits=[60], dnum=3, log2_scale=40, seed=7)
    h.keygen(rot_steps=[1, 5])
    return h


def _signed(v: np.ndarray, q: int) -> np.ndarray:
    v = v.astype(object)
    return np.array([int(x) - q if int(x) > q // 2 else int(x) for x in v], dtype=np.float64)


def test_relinearisation_decrypts_like_the_tensor(he):
    """(d0, d1) + KS(d2) decrypts with (1, s) to what the tensor decrypts to with
    (1, s, s^2), up to the small key-switching noise (coefficient units, limb q_0)."""
    M = he.n // 2
    z = np.random.default_rng(11).uniform(-1, 1, M)
    ct = he.encrypt(z, 9100)
    q = he.q[:ct.lp]
    s = he.keys.s[:ct.lp]
    d0, d1, d2 = he.tensor_square(ct)
    three = he.add(he.add(d0, he.mul(d1, s, q), q), he.mul(d2, he.mul(s, s, q), q), q)
    rl = he.relinearise((d0, d1, d2), ct.scale * ct.scale)
    two = he.add(rl.d[0], he.mul(rl.d[1], s, q), q)
    diff = he.intt(he.sub(two, three, q), q, he.qpsi)[0]
    assert np.abs(_signed(diff, q[0])).max() < 2.0 ** 30
    # and it decrypts to z^2: a dropped or doubled cross term of the tensor fails here
    assert np.abs(he.decrypt(he.rescale(rl)) - z * z).max() < 1e-6


def test_literal_square_is_relinearise_then_rescale(he):
    M = he.n // 2
    z = np.random.default_rng(12).uniform(-1, 1, M)
    ct = he.encrypt(z, 9101)
    lit = he.square_literal(ct)
    comp = he.rescale(he.relinearise(he.tensor_square(ct), ct.scale * ct.scale))
    assert np.array_equal(lit.d, comp.d) and lit.scale == comp.scale
    fused = he.square(ct)
    assert lit.lp == fused.lp == ct.lp - 1 and lit.scale == fused.scale
    assert not np.array_equal(lit.d, fused.d)           # other rounding (floor by q_top*P)
    assert np.abs(he.decrypt(lit) - he.decrypt(fused)).max() < 1e-7
    assert np.abs(he.decrypt(lit) - z * z).max() < 1e-6


def test_literal_rotation_sum_is_rotate_then_add(he):
    """A literal backend's plain sum of rotations is the sum of single rotations, bit for
    bit; the fused (hoisted, one ModDown) sum decrypts to the same slots."""
    M = he.n // 2
    z = np.random.default_rng(13).uniform(-1, 1, M)
    ct = he.encrypt(z, 9102)
    lit = layers.HeBackend(he, literal=True).lincomb([ct], [0, 1, 5], None)[0]
    acc = he.ct_add(he.ct_add(ct, he.rotate(ct, 1)), he.rotate(ct, 5))
    assert np.array_equal(lit.d, acc.d)
    fused = layers.HeBackend(he).lincomb([ct], [0, 1, 5], None)[0]
    want = z + np.roll(z, -1) + np.roll(z, -5)
    assert np.abs(he.decrypt(lit) - want).max() < 1e-6
    assert np.abs(he.decrypt(fused) - he.decrypt(lit)).max() < 1e-7


def _model_case(name):
    if name == "M2":
        return W.lenet1(), 28, 28, 1
    if name == "M3":
        return W.m3_relu(), 28, 28, 1
    if name == "M4n":
        return W.m4_narrow(), 32, 32, 1
    if name == "M5n":
        return W.m5_narrow(), 32, 32, 3
    model, Wi, Hi = W.paper_model(name)
    return model, Wi, Hi, 1


def _run_both(model, Wi, Hi, C, ns=1):
    """Both schedules on one encryption under one key set (the union of their plans' steps)."""
    dims = 1 if Hi == 1 else 2
    pl_l = layers.plan(model, Wi, Hi, dims, schedule="literal")
    pl_f = layers.plan(model, Wi, Hi, dims)
    logn = max(11, int(np.ceil(np.log2(pl_f["stride"] * ns))) + 1)
    P = dict(logn=logn, data_bits=[60] + [40] * pl_f["levels"], special_bits=[60, 60, 60], dnum=3,
             log2_scale=40)
    he = ckks.Ckks(seed=W.KEY_SEED, **P)
    he.keygen(sorted(set(pl_l["steps"]) | set(pl_f["steps"])))
    xs = W.images(ns, Hi, Wi, C=C) if dims == 2 else W.signals(ns, Wi)[:, 0]
    x = np.zeros(he.n // 2)
    for b in range(ns):
        x[b * pl_f["stride"]: b * pl_f["stride"] + xs[b].size] = np.asarray(xs[b]).reshape(-1)
    lay = layers.input_layout(Wi, Hi, pl_f["stride"], ns, he.n // 2, dims, channels=C)
    ct = he.encrypt(x, W.ENC_SEED)
    lit, _ = layers.run_model(layers.HeBackend(he, literal=True), ct, model, lay)
    fus, _ = layers.run_model(layers.HeBackend(he), ct, model, lay)
    return he, lit[0], fus[0], xs, dims


# every model shape of PAPER_MODELS plus LeNet-1 (M2) and M3; M4 and M5 with their layer
# sequences at fewer channels (the full channel counts take minutes per schedule here)
@pytest.mark.parametrize("name", ["M1", "M2", "M3", "M4n", "M5n", "M6", "M7"])
def test_fused_schedule_decrypts_like_the_literal_one(name):
    model, Wi, Hi, C = _model_case(name)
    he, lit, fus, xs, dims = _run_both(model, Wi, Hi, C)
    assert lit.lp == fus.lp and lit.scale == fus.scale
    n_out = model[-1]["w"].shape[0]
    a, b = he.decrypt(lit)[:n_out], he.decrypt(fus)[:n_out]
    ref = cnn.forward(xs[0], model, dims=dims)
    # the literal schedule is the paper's algorithm: pinned by the FP64 CNN
    assert np.abs(a - ref).max() < 1e-3
    # the fused one is the same slot algebra: within the noise of the literal one (both
    # carry key-switch and rescale rounding of about 1e-7 at Delta = 2^40 here)
    assert np.abs(a - b).max() < 1e-5
    # and a different evaluation order: other ciphertext bits
    assert not np.array_equal(lit.d, fus.d)


def test_literal_plan_never_merges_the_flatten():
    """The literal schedule's steps are the flatten stages' and the packing's own; the fused
    plan of LeNet-1 replaces the packing and the rows stage by their merged steps."""
    pl_f = layers.plan(W.lenet1(), 28, 28)
    pl_l = layers.plan(W.lenet1(), 28, 28, schedule="literal")
    assert pl_f["levels"] == pl_l["levels"] and pl_f["stride"] == pl_l["stride"]
    pack = {-o * 16 for o in range(1, 12)}
    rows = {r * (28 * 4 - 4) for r in range(1, 4)}
    merged = {r * (28 * 4 - 4) - o * 16 for r in range(4) for o in range(12)} - {0}
    lit, fus = set(pl_l["steps"]), set(pl_f["steps"])
    assert pack | rows <= lit and merged <= fus
    assert lit < fus and fus - lit <= merged
    assert not layers.merge_last_stage(4, 12, literal=True) and layers.merge_last_stage(4, 12)
