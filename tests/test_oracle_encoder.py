"""Pins of the FP64 canonical-embedding encoder against the O(N^2) textbook
evaluation m(zeta^(5^j)) and against closed forms."""
import numpy as np
import pytest

from oracle import ckks


def _he(logn):
    return ckks.Ckks(logn=logn, data_bits=[60], special_bits=[], dnum=1, log2_scale=40, seed=1)


@pytest.mark.parametrize("logn", [3, 6, 8])
def test_encode_matches_textbook_embedding(logn):
    he = _he(logn)
    N, M = he.n, he.n // 2
    rng = np.random.default_rng(logn)
    z = rng.uniform(-1, 1, M) + 1j * rng.uniform(-1, 1, M)
    scale = 2.0 ** 40
    m = he.encode_coeffs(z, scale).astype(np.float64)
    zeta = np.exp(1j * np.pi / N)
    for j in range(M):
        t = pow(5, j, 2 * N)
        val = np.sum(m * zeta ** (t * np.arange(N)))
        # rounding each coefficient moves the evaluation by at most N/2
        assert abs(val - scale * z[j]) <= N / 2 + 1e-6 * scale
    # the conjugate points hold the conjugate values (real coefficients)
    for j in range(3):
        t = (2 * N - pow(5, j, 2 * N)) % (2 * N)
        val = np.sum(m * zeta ** (t * np.arange(N)))
        assert abs(val - scale * np.conj(z[j])) <= N / 2 + 1e-6 * scale


def test_decode_is_the_textbook_evaluation():
    he = _he(6)
    N, M = he.n, he.n // 2
    coef = np.random.default_rng(2).normal(size=N)
    z = he.decode_coeffs(coef)
    zeta = np.exp(1j * np.pi / N)
    ref = np.array([np.sum(coef * zeta ** (pow(5, j, 2 * N) * np.arange(N))) for j in range(M)])
    assert np.abs(z - ref).max() < 1e-12 * N


def test_closed_forms():
    he = _he(10)
    N, M = he.n, he.n // 2
    # a constant vector c encodes to the constant polynomial round(c*Delta)
    m = he.encode_coeffs(np.full(M, 0.75), 2.0 ** 40)
    assert m[0] == round(0.75 * 2 ** 40) and np.all(m[1:] == 0)
    # the monomial X^k decodes to zeta^(5^j k) at slot j
    coef = np.zeros(N)
    coef[3] = 1.0
    z = he.decode_coeffs(coef)
    ref = np.exp(1j * np.pi / N * 3 * np.array([pow(5, j, 2 * N) for j in range(M)]))
    assert np.abs(z - ref).max() < 1e-12


@pytest.mark.parametrize("logn", [11, 14])
def test_round_trip(logn):
    he = _he(logn)
    M = he.n // 2
    z = np.random.default_rng(logn).uniform(-1, 1, M)
    m = he.encode_coeffs(z, 2.0 ** 40)
    back = he.decode_coeffs(m.astype(np.float64) / 2.0 ** 40)
    assert np.abs(back - z).max() < 2.0 ** -30
