"""The residue identity behind the one-pass lazy combination (ks_comb_lazy_kernel), checked on the
host in exact integers with the kernel's own steps: 128-bit sums of products (wrapping at 2^128
would be a bug, so the sum is asserted to stay below it), a fold to a residue before 63 products
could overflow, one reduction and one Montgomery reduction at the end.

Per-step form (ks_comb_kernel):  Z = sum_s w_s * (REDC(sum_j d_j K~_j) + P c0)  mod q
Lazy folded form:                 Z = REDC( sum_s [ sum_j d_j (K~_j w_s mod q) + c0 ([P 2^64]_q w_s mod q) ] mod q )
with K~ = K 2^64 mod q (Montgomery keys) and REDC(x) = x 2^-64 mod q.  The plain sum is the
same with w_s = 1.  A dropped 2^64 factor, a missing P, or a fold that loses the carry fails here."""
import random

import pytest

R = 1 << 64


def redc(x, q):
    """Montgomery reduction of x < q * 2^64 as the kernel computes it: x * 2^-64 mod q in [0, q)."""
    assert 0 <= x < q * R
    qneginv = (-pow(q, -1, R)) % R
    m = (x % R) * qneginv % R
    t = (x + m * q) >> 64
    return t - q if t >= q else t


def lazy(terms, q, fold_at=63):
    """sum of products with the kernel's fold rule, then reduce and REDC."""
    acc, n = 0, 0
    for per_step in terms:
        if n + len(per_step) > fold_at:
            acc, n = acc % q, 0
        for a, b in per_step:
            acc += a * b
            assert acc < 1 << 128
        n += len(per_step)
    return redc(acc % q, q)


@pytest.mark.parametrize("bits,beta,S", [(40, 6, 25), (60, 8, 64), (61, 3, 7), (50, 1, 40)])
def test_lazy_folded_combination_equals_the_per_step_form(bits, beta, S):
    rng = random.Random(bits * 1000 + beta * 10 + S)
    q = rng.randrange(1 << (bits - 1), 1 << bits) | 1
    P = rng.randrange(1 << 59, 1 << 60)
    Km = [[rng.randrange(q) for _ in range(beta)] for _ in range(S)]          # K~ (Montgomery form)
    d = [[rng.randrange(q) for _ in range(beta)] for _ in range(S)]           # gathered digits
    c0 = [rng.randrange(q) for _ in range(S)]                                 # gathered c0
    w = [rng.randrange(q) for _ in range(S)]                                  # weights
    ident = [rng.random() < 0.2 for _ in range(S)]                            # identity steps: P c0 only
    # per-step form
    ref = 0
    for s in range(S):
        a = (P * c0[s]) % q if ident[s] else (redc(sum(x * k for x, k in zip(d[s], Km[s])), q) + P * c0[s]) % q
        ref = (ref + w[s] * a) % q
    # lazy folded form: folded keys K~ w_s mod q, c0 multiplier [P 2^64]_q w_s mod q
    pm = (P % q) * R % q
    terms = []
    for s in range(S):
        step = [] if ident[s] else [(x, k * w[s] % q) for x, k in zip(d[s], Km[s])]
        step.append((c0[s], pm * w[s] % q))
        terms.append(step)
    assert lazy(terms, q) == ref
    # the plain sum: weights 1, keys as they are, c0 times [P 2^64]_q
    ref_plain = sum((P * c0[s]) % q if ident[s] else redc(sum(x * k for x, k in zip(d[s], Km[s])), q) + P * c0[s]
                    for s in range(S)) % q
    plain = [([] if ident[s] else list(zip(d[s], Km[s]))) + [(c0[s], pm)] for s in range(S)]
    assert lazy(plain, q) == ref_plain
    # without the 2^64 factor on the c0 multiplier the result is wrong
    bad = [([] if ident[s] else list(zip(d[s], Km[s]))) + [(c0[s], P % q)] for s in range(S)]
    assert lazy(bad, q) != ref_plain


def test_fold_rule_keeps_the_sum_below_2_128():
    """63 products of 61-bit residues plus a folded residue stay below 2^128; 64 more would not
    be guaranteed."""
    q = (1 << 61) - 1
    assert 63 * (q - 1) ** 2 + q < 1 << 128
    assert 300 * (q - 1) ** 2 > 1 << 128
