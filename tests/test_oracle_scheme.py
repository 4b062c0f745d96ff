"""Pins of the CKKS oracle: decrypt(encrypt(x)) round trips, rotation
composition, key switching and the ciphertext product, all against cleartext."""
import numpy as np
import pytest

from oracle import ckks


@pytest.fixture(scope="module")
def he():
    h = ckks.Ckks(logn=10, data_bits=[60, 40, 40], special_bits=[60], dnum=3, log2_scale=40, seed=7)
    h.keygen(rot_steps=[1, 3, 4, 7, -2, 100, 511])
    return h


@pytest.fixture(scope="module")
def he_dnum():
    # alpha = 2 limbs per digit, two special primes, a short last digit
    h = ckks.Ckks(logn=10, data_bits=[60, 40, 40, 40, 40], special_bits=[60, 60], dnum=3, log2_scale=40, seed=8)
    h.keygen(rot_steps=[1, 5])
    return h


def test_round_trip(he):
    M = he.n // 2
    z = np.random.default_rng(0).uniform(-1, 1, M)
    ct = he.encrypt(z, 9000)
    assert np.abs(he.decrypt(ct) - z).max() < 2.0 ** -25
    # deterministic under the same seeds
    assert np.array_equal(he.encrypt(z, 9000).d, ct.d)
    assert not np.array_equal(he.encrypt(z, 9001).d, ct.d)


def test_rotation_composition(he):
    M = he.n // 2
    z = np.random.default_rng(1).uniform(-1, 1, M)
    ct = he.encrypt(z, 9000)
    for a, b in [(1, 3), (4, -2), (7, 100)]:
        r = he.rotate(he.rotate(ct, a), b)
        assert np.abs(he.decrypt(r) - np.roll(z, -(a + b))).max() < 1e-6
    # rotation by N/2 slots is the identity element (no key switch)
    assert np.array_equal(he.rotate(ct, M).d, ct.d)


def test_hoisted_equals_single_up_to_noise(he):
    M = he.n // 2
    z = np.random.default_rng(2).uniform(-1, 1, M)
    ct = he.encrypt(z, 9002)
    rr = he.rotate_hoisted(ct, [0, 1, 511, -2])
    for r in [1, 511, -2]:
        assert np.abs(he.decrypt(rr[r]) - np.roll(z, -r)).max() < 1e-6
    assert np.array_equal(rr[0].d, ct.d)


def test_general_digits(he_dnum):
    he = he_dnum
    M = he.n // 2
    z = np.random.default_rng(3).uniform(-1, 1, M)
    for lp in (5, 4, 3):   # full, short last digit, fewer digits
        ct = he.encrypt(z, 9003, lp=lp)
        assert np.abs(he.decrypt(he.rotate(ct, 5)) - np.roll(z, -5)).max() < 1e-6
        sq = he.square(ct)
        assert sq.lp == lp - 1
        assert np.abs(he.decrypt(sq) - z * z).max() < 1e-6


def test_square_and_plain_mult(he):
    M = he.n // 2
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, M)
    v = rng.uniform(-1, 1, M)
    ct = he.encrypt(z, 9004)
    sq = he.square(ct)
    assert sq.lp == 2 and abs(sq.scale - he.scale ** 2 / he.q[2]) == 0
    assert np.abs(he.decrypt(sq) - z * z).max() < 1e-6
    pm = he.rescale(he.ct_mul_plain(ct, he.encode(v, he.scale, 3), he.scale))
    assert np.abs(he.decrypt(pm) - z * v).max() < 1e-6
    s = he.ct_add_plain(pm, he.encode(v, pm.scale, pm.lp))
    assert np.abs(he.decrypt(s) - (z * v + v)).max() < 1e-6


def test_keyswitch_relation(he):
    """KS(x) decrypts to x*s' for the relinearisation key (s' = s^2)."""
    n = he.n
    q = he.q
    rng = np.random.default_rng(5)
    x = np.stack([rng.integers(0, qi, n, dtype=np.uint64) for qi in q])
    k0, k1 = he.keyswitch(x, he.keys.rlk)
    lhs = he.add(k0, he.mul(k1, he.keys.s[:3], q), q)
    s2 = he.mul(he.keys.s[:3], he.keys.s[:3], q)
    rhs = he.mul(x, s2, q)
    diff = he.intt(he.sub(lhs, rhs, q), q, he.qpsi)[0]
    c = np.where(diff > q[0] // 2, diff.astype(np.float64) - q[0], diff.astype(np.float64))
    assert np.abs(c).max() < 2.0 ** 30   # small key-switching noise, x is uniform mod Q


def test_moddown_absorbs_multiples_of_P(he_dnum):
    """ModDown(A + P*x) = ModDown(A) + x exactly: the identity the hoisted linear
    combination relies on to fold sigma(c0) into the Q u P accumulator."""
    he = he_dnum
    lp = 4
    basis, psis = he.ext_basis(lp)
    rng = np.random.default_rng(8)
    A = np.stack([rng.integers(0, m, he.n, dtype=np.uint64) for m in basis])
    x = np.stack([rng.integers(0, qi, he.n, dtype=np.uint64) for qi in he.q[:lp]])
    Pq = np.array([[he.P_mod(qi)] * he.n for qi in he.q[:lp]], dtype=np.uint64)
    Px = np.concatenate([he.mul(x, Pq, he.q[:lp]), np.zeros((he.K, he.n), dtype=np.uint64)])
    lhs = he.moddown(he.add(A, Px, basis))
    rhs = he.add(he.moddown(A), x, he.q[:lp])
    assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("which", ["he", "he_dnum"])
def test_lincomb_decrypts_to_weighted_rotation_sum(request, which):
    he = request.getfixturevalue(which)
    M = he.n // 2
    rng = np.random.default_rng(9)
    steps = [0, 1, 5] if which == "he_dnum" else [0, 1, 7, -2]
    zs = [rng.uniform(-1, 1, M) for _ in range(2)]
    cts = [he.encrypt(z, 9100 + i) for i, z in enumerate(zs)]
    w = [[[rng.uniform(-1, 1, M) for _ in steps] for _ in zs] for _ in range(2)]
    enc = [[[he.encode_ext(v, he.scale, cts[0].lp) for v in wi] for wi in wo] for wo in w]
    outs = he.lincomb(cts, steps, enc, he.scale)
    for o in range(2):
        want = sum(w[o][i][k] * np.roll(zs[i], -s) for i in range(2) for k, s in enumerate(steps))
        got = he.decrypt(he.rescale(outs[o]))
        assert np.abs(got - want).max() < 1e-5
    plain = he.lincomb(cts[:1], steps, None)[0]
    assert np.abs(he.decrypt(plain) - sum(np.roll(zs[0], -s) for s in steps)).max() < 1e-6


def test_lincomb_diag_decrypts_to_sum_of_rotations(he):
    M = he.n // 2
    rng = np.random.default_rng(10)
    zs = [rng.uniform(-1, 1, M) for _ in range(3)]
    cts = [he.encrypt(z, 9200 + i) for i, z in enumerate(zs)]
    steps = [0, -2, 7]
    out = he.lincomb_diag(cts, steps)
    want = sum(np.roll(z, -s) for z, s in zip(zs, steps))
    assert np.abs(he.decrypt(out) - want).max() < 1e-6


@pytest.mark.parametrize("which", ["he", "he_dnum"])
def test_lincomb_with_rescale_matches_lincomb_then_rescale(which, request):
    """The fused division gives the message of ModDown followed by rescale."""
    he = request.getfixturevalue(which)
    rng = np.random.default_rng(21)
    M = he.n // 2
    x = rng.uniform(-1, 1, M)
    ct = he.encrypt(x, 5)
    steps = [0, 1]
    ws = [rng.uniform(-1, 1, M) for _ in steps]
    enc = [[[he.encode_ext(w, he.scale, ct.lp) for w in ws]]]
    fused = he.lincomb([ct], steps, enc, he.scale, rescale=True)[0]
    plain = he.rescale(he.lincomb([ct], steps, enc, he.scale)[0])
    assert fused.lp == plain.lp == ct.lp - 1 and fused.scale == plain.scale
    want = sum(np.roll(x, -s) * w for s, w in zip(steps, ws))
    assert np.abs(he.decrypt(fused)[:M] - want).max() < 1e-5
    assert np.abs(he.decrypt(fused)[:M] - he.decrypt(plain)[:M]).max() < 1e-5


def test_naf_terms_are_the_minimal_signed_binary_form():
    """naf_terms: the terms sum to r mod the slots, are signed powers of two at
    strictly increasing, non-adjacent positions, and their count equals the minimal
    number of signed powers of two summing to r (brute force over small r)."""
    M = 64
    # minimal weight of r as a sum of +-2^k (k < 8), by breadth-first search over sums
    best, frontier = {0: 0}, [0]
    terms = [s * (1 << k) for k in range(8) for s in (1, -1)]
    for w in range(1, 6):
        nxt = []
        for v in frontier:
            for t in terms:
                u = v + t
                if abs(u) <= 256 and u not in best:
                    best[u] = w
                    nxt.append(u)
        frontier = nxt
    for r in range(-2 * M, 2 * M):
        t = ckks.naf_terms(r, M)
        assert sum(t) % M == r % M
        v = sum(t)
        assert -M // 2 < v <= M // 2
        pos = [abs(x).bit_length() - 1 for x in t]
        assert all(abs(x) == 1 << p for x, p in zip(t, pos))
        assert all(b - a >= 2 for a, b in zip(pos, pos[1:]))
        assert len(t) == best[v], (r, t)
    assert ckks.naf_terms(0, M) == [] and ckks.naf_terms(M, M) == []
    assert sorted(set(ckks.pow2_steps(M))) == sorted({s * (1 << k) for k in range(6) for s in (1, -1)})


def test_rotation_with_power_of_two_keys_only():
    """With the power-of-two key set alone, every rotation (composed from its
    non-adjacent form) decrypts to the rolled slots; shared prefixes are reused."""
    h = ckks.Ckks(logn=10, data_bits=[60, 40, 40], special_bits=[60], dnum=3, log2_scale=40, seed=11)
    M = h.n // 2
    h.keygen(rot_steps=ckks.pow2_steps(M))
    z = np.random.default_rng(5).uniform(-1, 1, M)
    ct = h.encrypt(z, 9000)
    cache = {}
    for r in [1, 3, 7, 100, -45, 255, 511, -511, 512, 1000]:
        y = h.rotate_naf(ct, r, cache)
        assert np.abs(h.decrypt(y) - np.roll(z, -r)).max() < 1e-6, r
    # the chain for 7 = 8 - 1 reuses the cached rotation by -1 of the chain for 3 = 4 - 1
    assert -1 in cache and 3 in cache and 7 in cache
    assert np.array_equal(h.rotate_naf(ct, 0).d, ct.d)


@pytest.mark.parametrize("rescale", [False, True])
def test_lincomb_chan_decrypts_to_per_input_rotation_sums(he, rescale):
    """Each input with its own steps (the flatten's merged stage): the combination
    decrypts to sum_i sum_k w_ik * roll(x_i, -s_ik); with one input and shared steps it
    is exactly (bit for bit) the one-output lincomb."""
    M = he.n // 2
    rng = np.random.default_rng(31)
    zs = [rng.uniform(-1, 1, M) for _ in range(2)]
    cts = [he.encrypt(z, 9300 + i) for i, z in enumerate(zs)]
    steps = [[0, 3], [-2, 100]]
    ws = [[rng.uniform(-1, 1, M) for _ in st] for st in steps]
    enc = [[he.encode_ext(w, he.scale, cts[0].lp) for w in wi] for wi in ws]
    out = he.lincomb_chan(cts, steps, enc, he.scale, rescale=rescale)
    want = sum(w * np.roll(z, -s) for z, st, wi in zip(zs, steps, ws) for s, w in zip(st, wi))
    got = he.decrypt(out if rescale else he.rescale(out))
    assert np.abs(got - want).max() < 1e-5
    one = he.lincomb_chan(cts[:1], [[1, 7]], [enc[0]], he.scale, rescale=rescale)
    ref = he.lincomb(cts[:1], [1, 7], [[enc[0]]], he.scale, rescale=rescale)[0]
    assert np.array_equal(one.d, ref.d) and one.scale == ref.scale
