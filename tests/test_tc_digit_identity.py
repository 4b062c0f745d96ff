"""The integer identity behind the tensor-core form of the mask MAC, checked on the host in exact
Python integers: a residue v < 256^C written as C signed byte digits d_a = (byte a of v) - 128,
v = sum_a d_a 256^a + Cc with Cc = 128 (256^C - 1) / 255, gives for T' terms

    sum_t w_t x_t = sum_{k<2C-1} 2^(8k) S_k + Cc sum_t w_t + Cc sum_t x_t - T' Cc^2,
    S_k = sum_{a+b=k} sum_t e_a(w_t) d_b(x_t),

and every partial sum of S_k stays below 2^24 in magnitude for T' <= 112 (so fp32 accumulation
of fp16 digit products is exact).  A dropped correction term, a wrong offset or a shift off by
one digit fails here."""
import random

import pytest


def digits(v, C):
    assert 0 <= v < 256 ** C
    return [((v >> (8 * a)) & 255) - 128 for a in range(C)]


def cc(C):
    return 128 * (256 ** C - 1) // 255


@pytest.mark.parametrize("bits", [20, 40, 50, 60])
def test_byte_digits_reconstruct(bits):
    C = (bits + 7) // 8
    rng = random.Random(bits)
    for _ in range(200):
        v = rng.randrange(0, 1 << bits)
        d = digits(v, C)
        assert all(-128 <= x <= 127 for x in d)
        assert sum(x * 256 ** a for a, x in enumerate(d)) + cc(C) == v


@pytest.mark.parametrize("bits,T", [(40, 100), (60, 100), (60, 112), (36, 7)])
def test_shift_sums_reconstruct_the_dot_product(bits, T):
    C = (bits + 7) // 8
    rng = random.Random(1000 * bits + T)
    q = rng.randrange(1 << (bits - 1), 1 << bits) | 1
    Tp = 16 * ((T + 15) // 16)                       # terms staged, zero padding included
    w = [rng.randrange(q) for _ in range(T)] + [0] * (Tp - T)
    x = [rng.randrange(q) for _ in range(T)] + [0] * (Tp - T)
    S = [0] * (2 * C - 1)
    for wt, xt in zip(w, x):
        e, d = digits(wt, C), digits(xt, C)
        for a in range(C):
            for b in range(C):
                S[a + b] += e[a] * d[b]
    # exact fp32 accumulation: every S_k (and every partial sum, bounded by the same count of
    # |e d| <= 2^14 products) below 2^24
    bound = min(C, 8) * Tp * 128 * 128
    assert bound < 1 << 24
    assert all(abs(s) <= bound for s in S)
    got = sum(s << (8 * k) for k, s in enumerate(S)) + cc(C) * sum(w) + cc(C) * sum(x) - Tp * cc(C) ** 2
    assert got == sum(a * b for a, b in zip(w, x))
    assert got % q == sum(a * b for a, b in zip(w, x)) % q
    # the offset terms are required: without them the digits alone do not give the product
    assert sum(s << (8 * k) for k, s in enumerate(S)) != got
