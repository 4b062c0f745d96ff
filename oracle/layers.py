"""UniHENN layer algorithms and layout planner, written once against a backend.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A backend supplies slot-vector operations:
    rot(x, r)            Rot(x, r): left rotation by r slots (paper Sec. II-B)
    rot_many(x, steps)   several rotations of one input (hoisted on ciphertexts)
    lincomb(xs, steps, w)  Y_o = sum_i sum_s w[o][i][s] * Rot(xs[i], steps[s]) (w None: a
                         single plain sum of the rotations); on ciphertexts all rotations
                         of an input share one ModUp and each output one ModDown
    add(x, y)            Add (C)
    mul_mask(x, v)       Mul (P) by the slot vector v encoded at scale Delta
    add_mask(x, v)       Add (P) of v encoded at x's current scale and level
    rescale(x)           drop one level (identity on cleartext)
    lincomb_rescale(xs, steps, w)  lincomb followed by rescale of every output
    square(x)            Mul (C) of x by itself, relinearised and rescaled
Two backends exist: ``slotsim.SlotSim`` (FP64 cleartext, O2) and
``HeBackend`` below (the CKKS oracle, O3).  Running the same layer code on
both is what lets the cleartext simulator pin the algorithm and the CKKS
oracle pin the ciphertexts.

Slot layout (paper Sec. III-A, III-B, V): sample b of a ciphertext starts at
slot b*stride; inside a sample the value at (row r, column c) of the current
feature map sits at I*(r*W_img + c), where I is the interval (product of the
strides and pool sizes so far) and W_img the width of the original input.
Masks are built over every sample position of the layout (``n_samples``),
whatever the number of samples a ciphertext actually carries (reading C17).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Layout:
    W_img: int
    H_img: int
    W: int
    H: int
    I: int
    stride: int
    n_samples: int
    slots: int
    dims: int = 2          # 2 (image) or 1 (signal: H_img = H = 1)
    pending: float = 1.0   # deferred factor of average pooling (Sec. IV-C)
    prev: str = "input"    # last layer that set the layout: input/conv/avgpool/flatten/fc
    D: int = 0             # after flatten / FC: values at slots [0, D) of each sample
    C: int = 1             # input channels in one ciphertext (channel i at i*W_img*H_img)

    @property
    def flat(self) -> bool:
        return self.prev in ("flatten", "fc")


def input_layout(W_img, H_img, stride, n_samples, slots, dims=2, channels=1) -> Layout:
    """A sample's channels flattened channel-major, row-major (Sec. III-A): value
    (i, r, c) at i*W_img*H_img + r*W_img + c of the sample."""
    assert stride * n_samples <= slots, "samples do not fit in the slots"
    assert channels * W_img * H_img <= stride, "a sample does not fit in the stride"
    return Layout(W_img, H_img, W_img, H_img, 1, stride, n_samples, slots, dims, C=channels)


def slot_vector(lay: Layout, positions, values) -> np.ndarray:
    """Slot vector with values[i] at positions[i] of every sample, zero elsewhere."""
    v = np.zeros(lay.slots)
    positions = np.asarray(positions, dtype=np.int64)
    values = np.broadcast_to(np.asarray(values, dtype=np.float64), positions.shape)
    for b in range(lay.n_samples):
        v[b * lay.stride + positions] = values
    return v


# --------------------------------------------------------------- layers
def conv(be, xs, w, bias, S: int, lay: Layout, mode: str = "hoisted"):
    """Algorithm 1 (Sec. IV-B).  w: [co][ci][K][K] (2-D) or [co][ci][K] (1-D).

    Rotations Rot(C_in(i), I*(k + W_img*j)); per output channel o the sum of
    Mul(C_rot(i,j,k), K(o,i,j,k)) with K(o,i,j,k) the weight (times the pending
    pooling factor) at every valid output slot (reading C1), then rescale and
    Add(bias at the valid output slots, reading C2).  I_out = I*S.
    mode "hoisted": all rotations of one input share one ModUp (Alg. 1 as printed).
    mode "incremental": each rotation is taken from the previous one, by I along a
    kernel row and by I*(W_img - K + 1) at a row change (reading C3 of the prose).
    """
    w = np.asarray(w, dtype=np.float64)
    if w.ndim == 3:
        w = w[:, :, None, :]
    co, ci, kh, kw = w.shape
    # an input of several channels in one ciphertext (Sec. III-A): input channel i is
    # read through the extra rotation i*W_img*H_img, all rotations hoisted together
    packed = len(xs) == 1 and ci > 1 and lay.prev == "input" and lay.C == ci
    assert packed or ci == len(xs)
    I = lay.I
    offs = [(j, k) for j in range(kh) for k in range(kw)]
    step = {o: I * (o[1] + lay.W_img * o[0]) for o in offs}
    Hout = (lay.H - kh) // S + 1
    Wout = (lay.W - kw) // S + 1
    Iout = I * S
    pos = [Iout * (r * lay.W_img + c) for r in range(Hout) for c in range(Wout)]
    def kvec(o, i, off):
        return slot_vector(lay, pos, float(w[o, i, off[0], off[1]]) * lay.pending)

    if packed:
        assert mode == "hoisted", "channels in one ciphertext: hoisted mode only"
        chan = lay.W_img * lay.H_img
        steps = [i * chan + step[off] for off in offs for i in range(ci)]
        weights = [[[kvec(o, i, off) for off in offs for i in range(ci)]] for o in range(co)]
        scaled = be.lincomb_rescale(xs, steps, weights)
    elif mode == "hoisted":
        # all rotations of every input channel and all products in one hoisted
        # linear combination per output channel, rescaled
        weights = [[[kvec(o, i, off) for off in offs] for i in range(ci)] for o in range(co)]
        scaled = be.lincomb_rescale(xs, [step[o] for o in offs], weights)
    elif mode == "incremental":
        rots = []
        for i in range(ci):
            rr = {offs[0]: xs[i]}
            prev = xs[i]
            for o in offs[1:]:
                s = I if o[1] > 0 else I * (lay.W_img - kw + 1)
                prev = be.rot(prev, s)
                rr[o] = prev
            rots.append(rr)
        sums = []
        for o in range(co):
            acc = None
            for i in range(ci):
                for off in offs:
                    t = be.mul_mask(rots[i][off], kvec(o, i, off))
                    acc = t if acc is None else be.add(acc, t)
            sums.append(acc)
        scaled = [be.rescale(x) for x in sums]
    else:
        raise ValueError(mode)
    outs = []
    for o in range(co):
        acc = be.add_mask(scaled[o], slot_vector(lay, pos, float(bias[o])))
        outs.append(acc)
    return outs, replace(lay, W=Wout, H=Hout, I=Iout, pending=1.0, prev="conv", C=1)


def conv_steps(lay: Layout, kh: int, kw: int, mode: str = "hoisted"):
    if mode == "incremental":
        return sorted({lay.I, lay.I * (lay.W_img - kw + 1)} if kh > 1 else {lay.I})
    return sorted({lay.I * (k + lay.W_img * j) for j in range(kh) for k in range(kw)} - {0})


def avgpool(be, xs, c: int, lay: Layout):
    """Sec. IV-C: a c x c all-ones 'convolution' with stride c by rotations and
    additions only (no mask, no level); 1/c^2 is deferred into ``pending``."""
    ch = c if lay.dims == 2 else 1
    steps = [lay.I * (k + lay.W_img * j) for j in range(ch) for k in range(c)]
    outs = [be.lincomb([x], steps, None)[0] for x in xs]
    Hout = lay.H // c if lay.dims == 2 else 1
    return outs, replace(lay, W=lay.W // c, H=Hout, I=lay.I * c,
                         pending=lay.pending / float(c ** lay.dims), prev="avgpool")


def square(be, xs, lay: Layout):
    """Square activation (Sec. IV-F, M2 table): one Mul (C) per channel, 1 level.
    A pending pooling factor p becomes p^2 (Sec. IV-C)."""
    return [be.square(x) for x in xs], replace(lay, pending=lay.pending * lay.pending)


# the degree-2 approximation of ReLU the paper uses (Sec. IV-F, Exp. 3 / M3): c0 + c1 x + c2 x^2
RELU_C0, RELU_C1, RELU_C2 = 0.375373, 0.5, 0.117071


def valid_positions(lay: Layout):
    """Slots of one sample that hold values: I*(r*W_img + c) for a feature map,
    [0, D) after flatten / FC."""
    if lay.flat:
        return np.arange(lay.D)
    H = lay.H if lay.dims == 2 else 1
    return np.array([lay.I * (r * lay.W_img + c) for r in range(H) for c in range(lay.W)])


def approx_relu(be, xs, lay: Layout):
    """Approximate ReLU f(x) = c0 + c1 x + c2 x^2 (Sec. IV-F), 2 levels.  A pending
    pooling factor p is folded in as f(p x) = c0 + (c1 p) x + (c2 p^2) x^2 (Sec. IV-C).
    Reading: a = Rescale(Mul(x^2, c2 p^2)); b = Rescale(Mul(x, c1 p)) with the
    plaintext encoded at the scale that lands b on a's scale, then its top limb
    dropped (Drop-Level as a modulus drop) to reach a's level; f = a + b + c0.  All
    three constants sit at the valid slots only, so every other slot ends at zero."""
    p = lay.pending
    pos = valid_positions(lay)
    m2 = slot_vector(lay, pos, RELU_C2 * p * p)
    m1 = slot_vector(lay, pos, RELU_C1 * p)
    m0 = slot_vector(lay, pos, RELU_C0)
    outs = []
    for x in xs:
        a = be.rescale(be.mul_mask(be.square(x), m2))
        b = be.mul_rescale_to(x, m1, a)
        outs.append(be.add_mask(be.add(a, b), m0))
    return outs, replace(lay, pending=1.0)


def flatten(be, xs, lay: Layout):
    """Sec. IV-E: gather every channel's W x H values into one contiguous block.

    After average pooling (IV-E-2): per column c' a mask carrying the pending
    factor at I*(r*W_img + c'), rescale, rotate left c'*(I-1), sum.
    After a convolution (IV-E-1, I > 1 and W > 1): sum of Rot(x, m*(I-1)) for
    m < I, then per block u < ceil(W/I) a mask of the block's columns, rescale,
    rotate left u*I*(I-1), sum.
    Then, when H > 1 (IV-E-3): per row r a mask of the row, rescale, rotate
    left r*(W_img*I - W), sum.  Finally (IV-E-4) channel o is rotated right by
    o*W*H and the channels are added.  Readings C12.

    Each mask-rotate-sum stage sum_k Rot(m_k (.) x, r_k) is evaluated as the
    single hoisted combination sum_k Rot(m_k, r_k) (.) Rot(x, r_k) (the same
    slot algebra: Rot is elementwise-multiplicative), followed by one rescale;
    the channel packing is one combination of the per-channel rotations.
    """
    I, W, H, Wi = lay.I, lay.W, lay.H, lay.W_img
    rows = range(H)
    cur = list(xs)
    pending = lay.pending

    literal = getattr(be, "literal", False)

    def masked_rotation_sum(x, masks, steps):
        if literal:
            # the steps of Sec. IV-E in their order: each mask multiplied with the
            # ciphertext, each product rotated left, the rotations added; one rescale
            acc = None
            for m, s in zip(masks, steps):
                t = be.rot(be.mul_mask(x, m), s)
                acc = t if acc is None else be.add(acc, t)
            return be.rescale(acc)
        rolled = [np.roll(m, -s) for m, s in zip(masks, steps)]
        return be.lincomb_rescale([x], steps, [[rolled]])[0]

    stages = []   # the masked rotation sums (masks, steps), in order
    if lay.prev == "avgpool":
        steps = [c * (I - 1) for c in range(W)]
        masks = [slot_vector(lay, [I * (r * Wi + c) for r in rows], pending) for c in range(W)]
        stages.append((masks, steps))
        pending = 1.0
    elif lay.prev == "conv":
        assert pending == 1.0
        if I > 1 and W > 1:
            nblk = -(-W // I)
            steps = [u * I * (I - 1) for u in range(nblk)]
            masks = []
            for u in range(nblk):
                cols = range(I * u, min(I * u + I, W))
                masks.append(slot_vector(lay, [I * r * Wi + I * I * u + (cc - I * u) for r in rows for cc in cols],
                                         1.0))
            cur = [be.lincomb([x], [m * (I - 1) for m in range(I)], None)[0] for x in cur]
            stages.append((masks, steps))
    else:
        raise ValueError("flatten must follow a convolution or an average pooling")
    if H > 1:
        steps = [r * (Wi * I - W) for r in rows]
        masks = [slot_vector(lay, [I * r * Wi + c for c in range(W)], 1.0) for r in rows]
        stages.append((masks, steps))
    for masks, steps in stages[:-1]:
        cur = [masked_rotation_sum(x, masks, steps) for x in cur]
    CH = len(cur)
    if stages and not merge_last_stage(len(stages[-1][1]), CH, literal):
        last = stages[-1]
        cur = [masked_rotation_sum(x, *last) for x in cur]
        stages = []            # every stage applied; the packing follows on its own
    if not stages:
        acc = be.lincomb_diag(cur, [-o * W * H for o in range(CH)]) if CH > 1 else cur[0]
    elif CH == 1:
        acc = masked_rotation_sum(cur[0], *stages[-1])
    else:
        # the last masked stage and the channel packing as one combination (reading C12):
        # channel o's term Rot(m_k (.) y_o, s_k) moved right by o*W*H is
        # Rot(m_k, s_k - o*W*H) (.) Rot(y_o, s_k - o*W*H); one ModDown and rescale for all
        masks, steps = stages[-1]
        st = [[s - o * W * H for s in steps] for o in range(CH)]
        ws = [[np.roll(m, -t) for m, t in zip(masks, st[o])] for o in range(CH)]
        acc = be.lincomb_chan_rescale(cur, st, ws)
    D = len(xs) * W * H
    return [acc], replace(lay, pending=pending, prev="flatten", D=D, W=D, H=1, I=1)


# The flatten's last masked stage (K steps) is merged with the packing of CH channels when the
# merged combination needs at most this many rotation steps (K*CH Galois keys instead of K + CH)
MERGE_MAX_STEPS = 128


def merge_last_stage(k: int, ch: int, literal: bool = False) -> bool:
    """Whether the fused schedule merges the flatten's last stage with the packing (the
    paper-order schedule never does)."""
    return not literal and ch > 1 and k * ch <= MERGE_MAX_STEPS


def fc_rot_matrix(M: np.ndarray):
    """Steps 1-4 of the FC figure (Sec. IV-D, reading C13): pad the columns of
    M (dout x din) with zeros to W_vec = ceil(din/dout)*dout and build
    M_rot[o][t] = M_pad[t mod dout][(t + o) mod W_vec]."""
    dout, din = M.shape
    Wv = -(-din // dout) * dout
    Mp = np.zeros((dout, Wv))
    Mp[:, :din] = M
    t = np.arange(Wv)
    Mr = np.stack([Mp[t % dout, (t + o) % Wv] for o in range(dout)])
    return Mr, Wv


def tree_steps(d: int, m: int):
    """Rotation steps of rotation_sum's binary form: the doublings k*d (k = 1, 2, 4, ..
    while 2k <= m) and the shifts off*d of the set bits of m below the highest."""
    steps, k = [], 1
    while 2 * k <= m:
        steps.append(k * d)
        k *= 2
    off = 0
    for b in reversed(range(m.bit_length())):
        if m >> b & 1:
            if off:
                steps.append(off * d)
            off += 1 << b
    return steps


def rotation_sum(be, x, d: int, m: int, mode: str = "linear"):
    """sum_{i<m} Rot(x, i*d), the last step of Algorithm 2.  "linear": the m
    rotations as one hoisted combination (as printed).  "tree": binary
    doubling, T_1 = x, T_2k = T_k + Rot(T_k, k*d), then the blocks T_{2^b} of
    the set bits b of m, high to low, each rotated by the total of the blocks
    before it: about log2(m) + popcount(m) rotations instead of m - 1.  Both
    compute the same slot sums; their ciphertexts differ (other key switches)."""
    if mode == "linear" or m == 1:
        return be.lincomb([x], [i * d for i in range(m)], None)[0]
    assert mode == "tree", mode
    T, k = [x], 1
    while 2 * k <= m:
        T.append(be.add(T[-1], be.rot(T[-1], k * d)))
        k *= 2
    acc, off = None, 0
    for b in reversed(range(len(T))):
        if m >> b & 1:
            term = T[b] if off == 0 else be.rot(T[b], off * d)
            acc = term if acc is None else be.add(acc, term)
            off += 1 << b
    return acc


def fc(be, xs, M, bias, lay: Layout, sum_mode: str = "linear"):
    """Algorithm 2 (Sec. IV-D): C_sum = sum_o Rot(C,o)*V1_o + Rot(C,o-W_vec)*V2_o,
    rescale, C_out = sum_{i < W_vec/dout} Rot(C_sum, i*dout) (rotation_sum, in
    sum_mode), then Add(bias) at slots [0, dout) of each sample."""
    assert len(xs) == 1 and lay.flat
    M = np.asarray(M, dtype=np.float64)
    dout, din = M.shape
    assert din == lay.D, f"FC expects {lay.D} inputs, got {din}"
    if lay.pending != 1.0:
        M = M * lay.pending
    Mr, Wv = fc_rot_matrix(M)
    x = xs[0]
    # rotations by o (with V1_o) then by o - W_vec (with V2_o, o >= 1): one hoisted combination
    steps = [o for o in range(dout)] + [o - Wv for o in range(1, dout)]
    t_idx = np.arange(Wv)
    vecs = [slot_vector(lay, t_idx, np.where(t_idx < Wv - o, Mr[o], 0.0)) for o in range(dout)]
    vecs += [slot_vector(lay, t_idx, np.where(t_idx >= Wv - o, Mr[o], 0.0)) for o in range(1, dout)]
    acc = be.lincomb_rescale([x], steps, [[vecs]])[0]
    nsum = Wv // dout
    out = rotation_sum(be, acc, dout, nsum, sum_mode)
    out = be.add_mask(out, slot_vector(lay, np.arange(dout), np.asarray(bias, dtype=np.float64)))
    return [out], replace(lay, pending=1.0, prev="fc", D=dout, W=dout)


# --------------------------------------------------------------- batch combining
def pack_steps(stride: int, n: int):
    """Rotation steps pack() uses for n single-sample ciphertexts: right by i*stride."""
    return [-i * stride for i in range(1, n)]


def pack(be, xs, lays):
    """Sec. III-B: combine ciphertexts into one: the i-th input is rotated right by
    (the samples before it) * stride and the rotations are added.  Every input
    has the input layout of the same image size and stride; the result carries
    all their samples in order.  Evaluated as one combination of the per-input
    rotations with a single ModDown (as the channel packing of the flatten)."""
    l0 = lays[0]
    off, steps = 0, []
    for lay in lays:
        assert lay.prev == "input" and (lay.W_img, lay.H_img, lay.stride, lay.dims, lay.slots) == \
            (l0.W_img, l0.H_img, l0.stride, l0.dims, l0.slots), "pack: inputs differ in layout"
        steps.append(-off * l0.stride)
        off += lay.n_samples
    assert off * l0.stride <= l0.slots, "pack: the samples do not fit in the slots"
    y = be.lincomb_diag(list(xs), steps) if len(xs) > 1 else xs[0]
    return y, replace(l0, n_samples=off)


# --------------------------------------------------------------- model
def run_model(be, x, layers, lay: Layout, conv_mode: str = "hoisted"):
    """Evaluate a layer list (dicts as produced by ``workloads``) on [x].

    Drop-Level (Sec. IV-A): when x has more levels left than the model consumes,
    its top levels are dropped first (reading C11: as a modulus drop), so every
    layer runs on the fewest limbs."""
    left = be.levels_left(x)
    if left is not None:
        need = plan(layers, lay.W_img, lay.H_img, lay.dims)["levels"]
        assert left >= need, "not enough levels for this model"
        for _ in range(left - need):
            x = be.drop_level(x)
    return run_layers(be, [x], layers, lay, conv_mode)


def run_layers(be, xs, layers, lay: Layout, conv_mode: str = "hoisted"):
    """Evaluate a layer list on the channel list xs."""
    for spec in layers:
        op = spec["op"]
        if op in ("conv2d", "conv1d"):
            xs, lay = conv(be, xs, spec["w"], spec["b"], spec["stride"], lay, conv_mode)
        elif op == "square":
            xs, lay = square(be, xs, lay)
        elif op == "approx_relu":
            xs, lay = approx_relu(be, xs, lay)
        elif op == "avgpool":
            xs, lay = avgpool(be, xs, spec["k"], lay)
        elif op == "flatten":
            xs, lay = flatten(be, xs, lay)
        elif op == "fc":
            if not lay.flat:
                xs, lay = flatten(be, xs, lay)
            xs, lay = fc(be, xs, spec["w"], spec["b"], lay, spec.get("sum", "linear"))
        else:
            raise ValueError(op)
    return xs, lay


def plan(layers, W_img: int, H_img: int, dims: int = 2, schedule: str = "fused"):
    """Layout sizes of Sec. V: the slots one sample needs (the stride), the number
    of levels the model consumes, and the rotation steps it uses.

    Stride = max(input W_img*H_img (Theorem 1 keeps every later valid value
    inside it), CH*W*H of each flatten (V-C), W_vec of each FC (V-D)).
    schedule "literal" (the paper's order, ``HeBackend(literal=True)``) never merges the
    flatten's last stage with the packing, so its steps are the stages' and the packing's.
    """
    assert schedule in ("fused", "literal"), schedule
    W, H, I, ch = W_img, H_img, 1, 1
    prev = "input"
    # the input's channels: CH_in of a first convolution (all in one ciphertext)
    C = np.asarray(layers[0]["w"]).shape[1] if layers and layers[0]["op"] in ("conv2d", "conv1d") else 1
    need = C * W_img * H_img
    levels = 0
    steps: set[int] = set()
    flat_D = 0
    for spec in layers:
        op = spec["op"]
        if op in ("conv2d", "conv1d"):
            w = np.asarray(spec["w"])
            kh = w.shape[2] if w.ndim == 4 else 1
            kw = w.shape[-1]
            S = spec["stride"]
            chans = range(w.shape[1]) if prev == "input" else [0]
            steps |= {i * W_img * H_img + I * (k + W_img * j) for i in chans for j in range(kh) for k in range(kw)}
            H, W, I = (H - kh) // S + 1, (W - kw) // S + 1, I * S
            ch = w.shape[0]
            levels += 1
            prev = "conv"
        elif op == "square":
            levels += 1
        elif op == "approx_relu":
            levels += 2
        elif op == "avgpool":
            c = spec["k"]
            ckh = c if dims == 2 else 1
            steps |= {I * (k + W_img * j) for j in range(ckh) for k in range(c)}
            W, H, I = W // c, (H // c if dims == 2 else 1), I * c
            prev = "avgpool"
        elif op in ("flatten", "fc"):
            if prev in ("conv", "avgpool"):
                stage_steps = []   # steps of the masked stages, in order
                if prev == "avgpool":
                    levels += 1
                    stage_steps.append([c * (I - 1) for c in range(W)])
                elif I > 1 and W > 1:
                    levels += 1
                    steps |= {m * (I - 1) for m in range(I)}
                    stage_steps.append([u * I * (I - 1) for u in range(-(-W // I))])
                if H > 1:
                    levels += 1
                    stage_steps.append([r * (W_img * I - W) for r in range(H)])
                if stage_steps and merge_last_stage(len(stage_steps[-1]), ch, schedule == "literal"):
                    for st in stage_steps[:-1]:
                        steps |= set(st)
                    steps |= {s - o * W * H for s in stage_steps[-1] for o in range(ch)}
                else:
                    for st in stage_steps:
                        steps |= set(st)
                    steps |= {-o * W * H for o in range(ch)}
                flat_D = ch * W * H
                need = max(need, flat_D)
                prev = "flatten"
            if op == "fc":
                dout, din = np.asarray(spec["w"]).shape
                Wv = -(-din // dout) * dout
                need = max(need, Wv)
                steps |= set(range(dout)) | {o - Wv for o in range(1, dout)}
                if spec.get("sum", "linear") == "tree":
                    steps |= set(tree_steps(dout, Wv // dout))
                else:
                    steps |= {i * dout for i in range(Wv // dout)}
                levels += 1
                prev = "fc"
                flat_D = dout
    steps.discard(0)
    return {"stride": need, "levels": levels, "steps": sorted(steps)}


# --------------------------------------------------------------- CKKS backend
class HeBackend:
    """The CKKS oracle as a layer backend; counts the operations it performs.

    Three schedules, each bit-compared with the GPU library in the same mode:

    * default ("fused"): the rotations of one input share one ModUp (hoisting), a
      linear combination of rotations is accumulated over Q_l u P with one ModDown
      per output, ModDown and rescale are one division by q_top * P, and the
      flatten's last stage may be merged with the channel packing.  Each of these is
      an evaluation order of the same slot algebra, pinned against the literal
      schedule by decryption.
    * literal=True: the paper's order, one operation at a time (Alg. 1, Sec. IV-C,
      Sec. IV-E, Alg. 2 as printed): every Rot is its own key switch (ModUp, inner
      product, ModDown, + sigma(c0)); Mul (P) by the mask over Q_l; Add; the rescale
      of reading C7; square = tensor, relinearise, rescale; the flatten's stages are
      mask, rotate, add, and the packing follows them.
    * naf=True: the context holds power-of-two Galois keys only (the key set SEAL
      generates by default).  Every rotation is then a chain of power-of-two rotations
      (``Ckks.rotate_naf``), and a linear combination of rotations is evaluated as
      rotate-then-multiply: the rotated ciphertexts of one input (chains sharing their
      prefixes), the products with the plaintexts over Q_l (Mul (P)) summed, then the
      rescale (reading C7)."""

    def __init__(self, he, naf: bool = False, literal: bool = False):
        self.he = he
        self.naf = naf
        self.literal = literal
        self.count = {"rot": 0, "pmul": 0, "rescale": 0, "square": 0}

    @property
    def _seq(self) -> bool:
        """rotate-then-multiply, one rotation at a time (literal or power-of-two keys)"""
        return self.naf or self.literal

    def _rot1(self, x, r, cache=None):
        return self.he.rotate_naf(x, r, cache) if self.naf else self.he.rotate(x, r)

    def _rots(self, x, steps):
        cache = {} if self.naf else None
        return [self._rot1(x, s, cache) for s in steps]

    def rot(self, x, r):
        self.count["rot"] += 1 if r % (self.he.n // 2) else 0
        return self._rot1(x, r)

    def rot_many(self, x, steps):
        self.count["rot"] += len({s for s in steps if s % (self.he.n // 2)})
        if self._seq:
            return dict(zip(steps, self._rots(x, steps)))
        return self.he.rotate_hoisted(x, steps)

    def lincomb_diag(self, xs, steps):
        m = self.he.n // 2
        self.count["rot"] += len([s for s in steps if s % m])
        if self._seq:
            ys = [self._rot1(x, s) for x, s in zip(xs, steps)]
            acc = ys[0]
            for y in ys[1:]:
                acc = self.he.ct_add(acc, y)
            return acc
        return self.he.lincomb_diag(xs, steps)

    def _seq_lincomb(self, xs, steps, weights):
        rots = [self._rots(x, steps) for x in xs]
        if weights is None:
            outs = []
            for r in rots:
                acc = r[0]
                for y in r[1:]:
                    acc = self.he.ct_add(acc, y)
                outs.append(acc)
            return outs
        lp = xs[0].lp
        outs = []
        for wo in weights:
            acc = None
            for i, wi in enumerate(wo):
                for s, v in enumerate(wi):
                    t = self.he.ct_mul_plain(rots[i][s], self.he.encode(v, self.he.scale, lp), self.he.scale)
                    acc = t if acc is None else self.he.ct_add(acc, t)
            outs.append(acc)
        return outs

    def lincomb(self, xs, steps, weights):
        m = self.he.n // 2
        self.count["rot"] += len(xs) * len({s % m for s in steps if s % m})
        if weights is not None:
            self.count["pmul"] += sum(len(wi) for wo in weights for wi in wo)
        if self._seq:
            return self._seq_lincomb(xs, steps, weights)
        if weights is None:
            return self.he.lincomb(xs, steps, None)
        lp = xs[0].lp
        enc = [[[self.he.encode_ext(v, self.he.scale, lp) for v in wi] for wi in wo] for wo in weights]
        return self.he.lincomb(xs, steps, enc, self.he.scale)

    def lincomb_rescale(self, xs, steps, weights):
        m = self.he.n // 2
        self.count["rot"] += len(xs) * len({s % m for s in steps if s % m})
        self.count["pmul"] += sum(len(wi) for wo in weights for wi in wo)
        self.count["rescale"] += len(weights)
        if self._seq:
            return [self.he.rescale(y) for y in self._seq_lincomb(xs, steps, weights)]
        lp = xs[0].lp
        enc = [[[self.he.encode_ext(v, self.he.scale, lp) for v in wi] for wi in wo] for wo in weights]
        return self.he.lincomb(xs, steps, enc, self.he.scale, rescale=True)

    def lincomb_chan_rescale(self, xs, steps, weights):
        """Rescale(sum_i sum_k w[i][k] (.) Rot(x_i, steps[i][k])): one output, each input
        with its own steps."""
        m = self.he.n // 2
        self.count["rot"] += sum(len({s % m for s in st if s % m}) for st in steps)
        self.count["pmul"] += sum(len(w) for w in weights)
        self.count["rescale"] += 1
        lp = xs[0].lp
        if self._seq:
            acc = None
            for x, st, ws in zip(xs, steps, weights):
                rots = self._rots(x, st)
                for y, v in zip(rots, ws):
                    t = self.he.ct_mul_plain(y, self.he.encode(v, self.he.scale, lp), self.he.scale)
                    acc = t if acc is None else self.he.ct_add(acc, t)
            return self.he.rescale(acc)
        enc = [[self.he.encode_ext(v, self.he.scale, lp) for v in ws] for ws in weights]
        return self.he.lincomb_chan(xs, steps, enc, self.he.scale, rescale=True)

    def mul_rescale_to(self, x, v, target):
        """x (.) v rescaled onto target's scale and level: the plaintext is encoded at
        target.scale * q_top / x.scale, the product rescaled and its top limbs
        dropped down to target's level; the scale is then set to target's (equal up
        to the rounding of that quotient)."""
        self.count["pmul"] += 1
        self.count["rescale"] += 1
        s = target.scale * float(self.he.q[x.lp - 1]) / x.scale
        y = self.he.rescale(self.he.ct_mul_plain(x, self.he.encode(v, s, x.lp), s))
        while y.lp > target.lp:
            y = self.he.drop_level(y)
        y.scale = target.scale
        return y

    def levels_left(self, x):
        return x.lp - 1

    def drop_level(self, x):
        return self.he.drop_level(x)

    def add(self, x, y):
        return self.he.ct_add(x, y)

    def mul_mask(self, x, v):
        self.count["pmul"] += 1
        pt = self.he.encode(v, self.he.scale, x.lp)
        return self.he.ct_mul_plain(x, pt, self.he.scale)

    def add_mask(self, x, v):
        pt = self.he.encode(v, x.scale, x.lp)
        return self.he.ct_add_plain(x, pt)

    def rescale(self, x):
        self.count["rescale"] += 1
        return self.he.rescale(x)

    def square(self, x):
        self.count["square"] += 1
        return self.he.square_literal(x) if self.literal else self.he.square(x)
