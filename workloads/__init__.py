"""Seeded synthetic workloads shaped like the paper's experiments.

Shared by the tests, the benchmark and the oracle as INPUT GENERATORS ONLY:
nothing here performs homomorphic-encryption arithmetic.  MNIST, USPS, CIFAR-10 and the
ECG set are not available, so (paper Sec. VI datasets -> stand-ins):
  * MNIST 28x28 gray images      -> U[0,1] 28x28 images, sample i seeded 1000+i
  * USPS 16x16, CIFAR-10 3x32x32  -> U[0,1] images of those shapes, seeded the same way
  * 1-D ECG beats                -> N(0,1) signals of length 1024, seeded 1000+i
  * trained weights               -> N(0, 0.1^2) weights and biases, seed 42
Model shapes: a single 5x5 convolution
(Exp. 1 style), the LeNet-1-shaped net of Exp. 2 (Table M2: conv 1->4 K5,
x^2, avgpool 2, conv 4->12 K5, x^2, avgpool 2, flatten, FC 192->10) and a 1-D
CNN in the family of Exp. 7, and a LeNet-5-shaped net (x^2 activations) at
N = 2^15 for the serving mix.
"""
from __future__ import annotations

import numpy as np

WEIGHT_SEED = 42
INPUT_SEED = 1000
KEY_SEED = 7
ENC_SEED = 9000


def _normal(rng, shape, sd=0.1):
    return rng.normal(0.0, sd, size=shape)


def single_conv(seed: int = WEIGHT_SEED, K: int = 5):
    rng = np.random.default_rng(seed)
    return [{"op": "conv2d", "w": _normal(rng, (1, 1, K, K)), "b": np.zeros(1), "stride": 1}]


def lenet1(seed: int = WEIGHT_SEED):
    rng = np.random.default_rng(seed)
    return [
        {"op": "conv2d", "w": _normal(rng, (4, 1, 5, 5)), "b": _normal(rng, (4,)), "stride": 1},
        {"op": "square"},
        {"op": "avgpool", "k": 2},
        {"op": "conv2d", "w": _normal(rng, (12, 4, 5, 5)), "b": _normal(rng, (12,)), "stride": 1},
        {"op": "square"},
        {"op": "avgpool", "k": 2},
        {"op": "flatten"},
        {"op": "fc", "w": _normal(rng, (10, 192)), "b": _normal(rng, (10,))},
    ]


def cnn1d(seed: int = WEIGHT_SEED, length: int = 1024, fc_sum: str = "linear"):
    """fc_sum: how the FC's final rotation sum is evaluated ("linear" as in Alg. 2,
    or "tree": binary doubling, the form the serving mix uses)."""
    rng = np.random.default_rng(seed)
    l1 = length - 2          # conv k3 s1
    l2 = l1 // 2             # avgpool 2
    l3 = (l2 - 3) // 2 + 1   # conv k3 s2
    return [
        {"op": "conv1d", "w": _normal(rng, (8, 1, 3)), "b": _normal(rng, (8,)), "stride": 1},
        {"op": "square"},
        {"op": "avgpool", "k": 2},
        {"op": "conv1d", "w": _normal(rng, (16, 8, 3)), "b": _normal(rng, (16,)), "stride": 2},
        {"op": "square"},
        {"op": "flatten"},
        {"op": "fc", "w": _normal(rng, (5, 16 * l3)), "b": _normal(rng, (5,)), "sum": fc_sum},
    ]


def lenet5_sq(seed: int = WEIGHT_SEED):
    rng = np.random.default_rng(seed)
    return [
        {"op": "conv2d", "w": _normal(rng, (6, 1, 5, 5)), "b": _normal(rng, (6,)), "stride": 1},
        {"op": "square"},
        {"op": "avgpool", "k": 2},
        {"op": "conv2d", "w": _normal(rng, (16, 6, 5, 5)), "b": _normal(rng, (16,)), "stride": 1},
        {"op": "square"},
        {"op": "avgpool", "k": 2},
        {"op": "flatten"},
        {"op": "fc", "w": _normal(rng, (120, 400)), "b": _normal(rng, (120,))},
        {"op": "square"},
        {"op": "fc", "w": _normal(rng, (84, 120)), "b": _normal(rng, (84,))},
        {"op": "square"},
        {"op": "fc", "w": _normal(rng, (10, 84)), "b": _normal(rng, (10,))},
    ]


def m3_relu(seed: int = WEIGHT_SEED):
    """The paper's M3 shape (Exp. 3, Sec. VII-C): conv 1->6 K3, approximate ReLU, avgpool 2,
    flatten, FC 1014->120, approximate ReLU, FC 120->10 (9 levels)."""
    rng = np.random.default_rng(seed)
    return [
        {"op": "conv2d", "w": _normal(rng, (6, 1, 3, 3)), "b": _normal(rng, (6,)), "stride": 1},
        {"op": "approx_relu"},
        {"op": "avgpool", "k": 2},
        {"op": "flatten"},
        {"op": "fc", "w": _normal(rng, (120, 1014)), "b": _normal(rng, (120,))},
        {"op": "approx_relu"},
        {"op": "fc", "w": _normal(rng, (10, 120)), "b": _normal(rng, (10,))},
    ]


def _from_shapes(spec, seed):
    rng = np.random.default_rng(seed)
    out = []
    for l in spec:
        if l[0] == "conv2d":
            _, ci, co, k, s = l
            out.append({"op": "conv2d", "w": _normal(rng, (co, ci, k, k)), "b": _normal(rng, (co,)), "stride": s})
        elif l[0] == "conv1d":
            _, ci, co, k, s = l
            out.append({"op": "conv1d", "w": _normal(rng, (co, ci, k)), "b": _normal(rng, (co,)), "stride": s})
        elif l[0] == "fc":
            _, din, dout = l
            out.append({"op": "fc", "w": _normal(rng, (dout, din)), "b": _normal(rng, (dout,))})
        elif l[0] == "avgpool":
            out.append({"op": "avgpool", "k": l[1]})
        else:
            out.append({"op": l[0]})
    return out


# The paper's other model shapes (Sec. VII, tables of detailed parameters), as
# (op, CH_in, CH_out, K, S) / (fc, DAT_in, DAT_out) lists, with the input size each implies.
PAPER_MODELS = {
    # Exp. 1: conv 1->8 K4 S3 on 28x28 (8x8 outputs), flatten after the convolution
    "M1": ([("conv2d", 1, 8, 4, 3), ("square",), ("flatten",), ("fc", 648, 64), ("square",), ("fc", 64, 10)],
           28, 28),
    # Exp. 4: LeNet-5 with x^2; conv3 16->120 K5 leaves 1x1 per channel (32x32 input)
    "M4": ([("conv2d", 1, 6, 5, 1), ("square",), ("avgpool", 2), ("conv2d", 6, 16, 5, 1), ("square",),
            ("avgpool", 2), ("conv2d", 16, 120, 5, 1), ("square",), ("flatten",), ("fc", 120, 84), ("square",),
            ("fc", 84, 10)], 32, 32),
    # Exp. 5: CIFAR-10 3x32x32 (the three channels in one ciphertext); pool 4 leaves 1x1x128
    "M5": ([("conv2d", 3, 16, 3, 1), ("square",), ("avgpool", 2), ("conv2d", 16, 64, 4, 1), ("square",),
            ("avgpool", 2), ("conv2d", 64, 128, 3, 1), ("square",), ("avgpool", 4), ("flatten",),
            ("fc", 128, 10)], 32, 32),
    # Exp. 6: USPS 16x16, conv 1->6 K4 S2 (7x7 outputs, 294 = DAT_in of FC1)
    "M6": ([("conv2d", 1, 6, 4, 2), ("square",), ("flatten",), ("fc", 294, 64), ("square",), ("fc", 64, 10)],
           16, 16),
    # Exp. 7: 1-D CNN on length 128 (flatten 4 x 32 = 128 = DAT_in of FC1)
    "M7": ([("conv1d", 1, 2, 2, 2), ("square",), ("conv1d", 2, 4, 2, 2), ("flatten",), ("fc", 128, 32),
            ("square",), ("fc", 32, 5)], 128, 1),
}


def m5_narrow(seed: int = WEIGHT_SEED):
    """M5's layer sequence (3-channel 32x32 input, kernels 3/4/3, pools 2/2/4) with
    4, 8 and 8 channels instead of 16, 64 and 128: the same levels and layouts at a
    size the oracle runs in seconds."""
    return _from_shapes([("conv2d", 3, 4, 3, 1), ("square",), ("avgpool", 2), ("conv2d", 4, 8, 4, 1), ("square",),
                         ("avgpool", 2), ("conv2d", 8, 8, 3, 1), ("square",), ("avgpool", 4), ("flatten",),
                         ("fc", 8, 10)], seed)


def m4_narrow(seed: int = WEIGHT_SEED):
    """M4's layer sequence (LeNet-5 with x^2 on 32x32: three 5x5 convolutions, the last to 1x1,
    pools 2/2, FC, x^2, FC) with 2, 4 and 8 channels instead of 6, 16 and 120."""
    return _from_shapes([("conv2d", 1, 2, 5, 1), ("square",), ("avgpool", 2), ("conv2d", 2, 4, 5, 1), ("square",),
                         ("avgpool", 2), ("conv2d", 4, 8, 5, 1), ("square",), ("flatten",), ("fc", 8, 6),
                         ("square",), ("fc", 6, 10)], seed)


def paper_model(name: str, seed: int = WEIGHT_SEED):
    """(layers with N(0, 0.1^2) weights, W_img, H_img) of one of PAPER_MODELS."""
    spec, Wi, Hi = PAPER_MODELS[name]
    return _from_shapes(spec, seed), Wi, Hi


def images(n: int, H: int = 28, W: int = 28, seed: int = INPUT_SEED, C: int = 1) -> np.ndarray:
    """[n][H][W] (C = 1) or [n][C][H][W] U[0,1] images (CIFAR-10 -> C = 3)."""
    shape = (H, W) if C == 1 else (C, H, W)
    return np.stack([np.random.default_rng(seed + i).uniform(0.0, 1.0, shape) for i in range(n)])


def signals(n: int, length: int = 1024, seed: int = INPUT_SEED) -> np.ndarray:
    return np.stack([np.random.default_rng(seed + i).normal(0.0, 1.0, (1, length)) for i in range(n)])


# CKKS parameter sets of the workloads (bit sizes of the data chain, then the
# special primes; dnum digits; log2 of the scale Delta).
PARAMS = {
    "conv1": dict(logn=13, data_bits=[60, 40, 40], special_bits=[60], dnum=3, log2_scale=40),
    "lenet1": dict(logn=14, data_bits=[60] + [40] * 7, special_bits=[60], dnum=8, log2_scale=40),
    "cnn1d": dict(logn=14, data_bits=[60] + [40] * 6, special_bits=[60], dnum=7, log2_scale=40),
    # M3 with approximate ReLU: 9 levels
    "m3": dict(logn=14, data_bits=[60] + [40] * 9, special_bits=[60], dnum=10, log2_scale=40),
    # LeNet-5-shaped net with x^2 activations: 11 levels at N = 2^15
    "lenet5": dict(logn=15, data_bits=[60] + [40] * 11, special_bits=[60], dnum=12, log2_scale=40),
}

# Serving mix: every model's keys with dnum = 3 digits.  A digit then spans up to
# three (LeNet-1, 1-D CNN) or four (LeNet-5) data primes, so the special modulus
# P must cover it: three 50-bit primes (150 bits > 140) and three 60-bit primes
# (180 bits, the size of LeNet-5's widest digit).  At N = 2^14 that makes log QP =
# 490 bits, above the 438 bits of the 128-bit HE-standard bound; recorded, not hidden.
SERVE_PARAMS = {
    "lenet1": dict(logn=14, data_bits=[60] + [40] * 7, special_bits=[50] * 3, dnum=3, log2_scale=40),
    "lenet5": dict(logn=15, data_bits=[60] + [40] * 11, special_bits=[60] * 3, dnum=3, log2_scale=40),
    "cnn1d": dict(logn=14, data_bits=[60] + [40] * 6, special_bits=[50] * 3, dnum=3, log2_scale=40),
}
ARRIVAL_SEED = 12345


def small_params(name: str, logn: int) -> dict:
    """The same chain at a smaller ring degree (for oracle-speed parity cases)."""
    p = dict(PARAMS[name])
    p["logn"] = logn
    return p
