"""Pins of the oracle's ring arithmetic against definitions it does not use:
Python big-integer schoolbook products, exact CRT, brute force on tiny moduli."""
import numpy as np
import pytest

from oracle import ckks

U64 = np.uint64


def negacyclic_schoolbook(a, b, q):
    n = len(a)
    c = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                c[k] += int(a[i]) * int(b[j])
            else:
                c[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in c]


@pytest.mark.parametrize("logn,bits", [(3, 60), (4, 40), (6, 60), (10, 40)])
def test_ntt_product_equals_schoolbook(logn, bits):
    he = ckks.Ckks(logn=logn, data_bits=[bits], special_bits=[], dnum=1, log2_scale=30, seed=1)
    q, psi = he.q[0], he.qpsi[0]
    rng = np.random.default_rng(logn)
    a = rng.integers(0, q, he.n, dtype=U64)
    b = rng.integers(0, q, he.n, dtype=U64)
    A = he.ntt(a[None], [q], [psi])
    B = he.ntt(b[None], [q], [psi])
    c = he.intt(he.mul(A, B, [q]), [q], [psi])[0]
    assert [int(x) for x in c] == negacyclic_schoolbook(a, b, q)


@pytest.mark.parametrize("logn", [3, 4, 6])
def test_ntt_is_the_definition(logn):
    he = ckks.Ckks(logn=logn, data_bits=[60], special_bits=[], dnum=1, log2_scale=30, seed=1)
    q, psi, n = he.q[0], he.qpsi[0], he.n
    a = np.random.default_rng(5).integers(0, q, n, dtype=U64)
    A = he.ntt(a[None], [q], [psi])[0]
    ref = [sum(int(a[j]) * pow(psi, j * (2 * k + 1), q) for j in range(n)) % q for k in range(n)]
    assert [int(x) for x in A] == ref
    assert np.array_equal(he.intt(A[None], [q], [psi])[0], a)


def test_primes_are_the_largest_of_their_class():
    logn = 13
    m = 2 << logn
    bits = [60, 40, 40, 60]
    ps = ckks.gen_primes(bits, logn)
    assert len(set(ps)) == len(ps)
    taken = []
    for b, q in zip(bits, ps):
        assert q < (1 << b) and q % m == 1 and ckks.is_prime(q)
        c = q + m
        while c < (1 << b):  # nothing larger of the class is a prime not already taken
            assert c in taken or not ckks.is_prime(c)
            c += m
        taken.append(q)


def test_is_prime_against_sympy():
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(3)
    cands = [int(x) | 1 for x in rng.integers(1 << 40, 1 << 62, 300, dtype=np.int64)]
    cands += [561, 1105, 1729, 2465, 2821, 6601, 3215031751, 341550071728321]  # Carmichael / strong pseudoprimes
    for c in cands:
        assert ckks.is_prime(c) == bool(sympy.isprime(c)), c


@pytest.mark.parametrize("q,logn", [(17, 2), (97, 3), (257, 4), (7681, 8)])
def test_smallest_psi_brute_force(q, logn):
    n = 1 << logn
    roots = [x for x in range(1, q) if pow(x, n, q) == q - 1]
    assert ckks.smallest_psi(q, logn) == min(roots)


def test_psi_order():
    he = ckks.Ckks(logn=14, data_bits=[60, 40], special_bits=[60], dnum=2, log2_scale=40, seed=1)
    for q, psi in zip(he.q + he.p, he.qpsi + he.ppsi):
        assert pow(psi, he.n, q) == q - 1


def _poly_mul(he, a, b, q, psi):
    return he.intt(he.mul(he.ntt(a[None], [q], [psi]), he.ntt(b[None], [q], [psi]), [q]), [q], [psi])[0]


def test_automorphism_properties():
    he = ckks.Ckks(logn=5, data_bits=[40], special_bits=[], dnum=1, log2_scale=30, seed=1)
    q, psi, n = he.q[0], he.qpsi[0], he.n
    rng = np.random.default_rng(7)
    a = rng.integers(0, q, n, dtype=U64)
    b = rng.integers(0, q, n, dtype=U64)
    for g, h in [(5, 25), (3, 7), (2 * n - 1, 5)]:
        sa = he.automorph_coeff(a[None], g, [q])
        # coefficient and evaluation forms agree
        assert np.array_equal(he.ntt(sa, [q], [psi]), he.automorph_eval(he.ntt(a[None], [q], [psi]), g))
        # composition
        assert np.array_equal(he.automorph_coeff(sa, h, [q]), he.automorph_coeff(a[None], g * h % (2 * n), [q]))
        # ring homomorphism: sigma(a*b) = sigma(a)*sigma(b), products checked by schoolbook
        ab = np.array(negacyclic_schoolbook(a, b, q), dtype=U64)
        lhs = he.automorph_coeff(ab[None], g, [q])[0]
        sb = he.automorph_coeff(b[None], g, [q])[0]
        rhs = negacyclic_schoolbook(sa[0], sb, q)
        assert [int(x) for x in lhs] == rhs
    # 5 has order N/2 modulo 2N: sigma_{5^(N/2)} is the identity
    assert pow(5, n // 2, 2 * n) == 1
    # X^g literally: a(X) = X^1 -> X^g (sign flip past degree n)
    x = np.zeros(n, dtype=U64)
    x[1] = 1
    for g in (5, 3 * n // 2 + 1):
        y = he.automorph_coeff(x[None], g, [q])[0]
        e = g % (2 * n)
        want = np.zeros(n, dtype=U64)
        if e < n:
            want[e] = 1
        else:
            want[e - n] = q - 1
        assert np.array_equal(y, want)


def _crt(res, mods):
    M = 1
    for m in mods:
        M *= m
    x = 0
    for r, m in zip(res, mods):
        Mi = M // m
        x += int(r) * Mi * pow(Mi, -1, m)
    return x % M, M


def test_bconv_is_crt_plus_small_multiple():
    he = ckks.Ckks(logn=3, data_bits=[60, 40, 40], special_bits=[60, 50], dnum=1, log2_scale=30, seed=1)
    qin, qout = he.q, he.p
    rng = np.random.default_rng(11)
    x = np.stack([rng.integers(0, q, he.n, dtype=U64) for q in qin])
    out = np.zeros((len(qout), he.n), dtype=U64)
    ckks.lib().o_bconv(ckks._p(out), ckks._p(x), len(qin), ckks._p(ckks._u(qin)), len(qout),
                       ckks._p(ckks._u(qout)), he.n)
    for c in range(he.n):
        X, Q = _crt([x[i, c] for i in range(len(qin))], qin)
        ok = False
        for e in range(len(qin)):
            if all((X + e * Q) % p == int(out[t, c]) for t, p in enumerate(qout)):
                ok = True
        assert ok


def test_moddown_is_floor_division_up_to_small_error():
    he = ckks.Ckks(logn=3, data_bits=[60, 40, 40], special_bits=[60, 55], dnum=3, log2_scale=30, seed=1)
    qs, ps = he.q, he.p
    basis = qs + ps
    rng = np.random.default_rng(12)
    coef = np.stack([rng.integers(0, m, he.n, dtype=U64) for m in basis])
    acc = np.concatenate([he.ntt(coef[:3], qs, he.qpsi), he.ntt(coef[3:], ps, he.ppsi)])
    out = he.intt(he.moddown(acc), qs, he.qpsi)
    P = ps[0] * ps[1]
    for c in range(he.n):
        X, QP = _crt([coef[i, c] for i in range(len(basis))], basis)
        Y, Q = _crt([out[i, c] for i in range(3)], qs)
        d = (Y - X // P) % Q
        assert d == 0 or Q - d < len(ps), (c, d)


def test_rescale_is_rounded_division():
    he = ckks.Ckks(logn=4, data_bits=[60, 40, 40, 40], special_bits=[], dnum=1, log2_scale=30, seed=1)
    rng = np.random.default_rng(13)
    coef = np.stack([rng.integers(0, q, he.n, dtype=U64) for q in he.q])
    ct = ckks.Ct(np.stack([he.ntt(coef, he.q, he.qpsi)] * 2), 2.0 ** 80)
    r = he.rescale(ct)
    assert r.scale == 2.0 ** 80 / he.q[-1]
    out = he.intt(r.d[0], he.q[:3], he.qpsi[:3])
    ql = he.q[-1]
    for c in range(he.n):
        X, Q = _crt([coef[i, c] for i in range(4)], he.q)
        want = (2 * X + ql) // (2 * ql)   # nearest integer to X/ql (no ties: ql odd)
        Y, Q3 = _crt([out[i, c] for i in range(3)], he.q[:3])
        assert Y == want % Q3


def _splitmix64_reference(seed, count):
    """Steele-Lea-Flood SplitMix64 as published (state += gamma; mix13 finaliser)."""
    M = (1 << 64) - 1
    G = 0x9E3779B97F4A7C15
    s, out = seed, []
    for _ in range(count):
        s = (s + G) & M
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_reference_vector():
    # widely published first outputs of SplitMix64 seeded with 0
    assert _splitmix64_reference(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_rand_word_is_splitmix_of_splitmix():
    for seed, stream in [(7, 0), (9000, ckks.stream_id("enc_u")), (42, ckks.stream_id("ksk_a", 3125, 2, 5))]:
        state = _splitmix64_reference(seed, stream + 1)[-1] if stream < 50 else None
        if state is None:  # jump directly: output #stream is mix(seed + (stream+1)*gamma)
            M = (1 << 64) - 1
            z = (seed + (stream + 1) * 0x9E3779B97F4A7C15) & M
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
            state = z ^ (z >> 31)
        want = _splitmix64_reference(state, 5)
        got = [ckks.lib().o_rand_word(seed, stream, i) for i in range(5)]
        assert got == want


def test_sampler_distributions():
    n = 1 << 16
    t = ckks.sample_ternary(5, 1, n)
    assert set(np.unique(t)) <= {-1, 0, 1}
    assert abs(np.mean(t)) < 0.02 and abs(np.mean(t == 0) - 1 / 3) < 0.01
    e = ckks.sample_cbd(5, 2, n)
    assert np.abs(e).max() <= 21 and abs(np.var(e) - 10.5) < 0.4 and abs(np.mean(e)) < 0.05
    q = (1 << 40) - 87
    u = ckks.sample_uniform(5, 3, n, q)
    assert int(u.max()) < q and abs(float(np.mean(u.astype(np.float64))) / q - 0.5) < 0.01


def test_moddown_rescale_is_floor_division_by_q_top_times_P():
    """The fused ModDown + rescale divides by D = q_top * P in one base conversion:
    out = floor(X / D) - e with 0 <= e < K + 1, X the CRT value over Q_l u P."""
    he = ckks.Ckks(logn=3, data_bits=[60, 40, 40], special_bits=[60, 55], dnum=3, log2_scale=30, seed=1)
    qs, ps = he.q, he.p
    basis = qs + ps
    rng = np.random.default_rng(14)
    coef = np.stack([rng.integers(0, m, he.n, dtype=U64) for m in basis])
    acc = np.concatenate([he.ntt(coef[:3], qs, he.qpsi), he.ntt(coef[3:], ps, he.ppsi)])
    out = he.intt(he.moddown_rescale(acc), qs[:2], he.qpsi[:2])
    D = qs[2] * ps[0] * ps[1]
    for c in range(he.n):
        X, _ = _crt([coef[i, c] for i in range(len(basis))], basis)
        Y, Q2 = _crt([out[i, c] for i in range(2)], qs[:2])
        d = (Y - X // D) % Q2
        assert d == 0 or Q2 - d < len(ps) + 1, (c, d)
