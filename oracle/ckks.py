"""RNS-CKKS oracle (O3): the scheme the paper evaluates its CNNs with.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper uses CKKS through SEAL (Sec. II-B: Add, Mul and Rot on ciphertexts,
levels and depth; Table II parameters).  It does not spell out the RNS
details, so this module fixes them from the published scheme descriptions and
records each choice (the "readings"):

* Primes (reading C8): for each requested bit size, in order (data primes, then
  special primes), the largest prime q < 2^bits with q = 1 mod 2N not already
  taken.  psi = the smallest primitive 2N-th root of unity mod q.
* Ciphertexts are (c0, c1) with m = c0 + c1*s, limbs q_0..q_{L'-1} in natural
  order evaluation form.  Comparisons with other implementations are made in
  coefficient form (``to_coeff``), which is independent of any NTT ordering.
* Randomness (reading C9): counter-based SplitMix64 words (``o_rand_word``);
  stream id = purpose<<56 | key_id<<32 | digit<<16 | limb.  Secret s and
  encryption u ternary, errors centred binomial eta=21, uniform a = floor(r*q/2^64),
  all sampled in coefficient form.
* Hybrid key switching (reading C6, Han-Ki 2020): digits are consecutive groups
  of alpha = ceil((L+1)/dnum) active limbs; ModUp is fast base conversion
  without correction; inner product over Q_l u P; ModDown without rounding
  correction.  Hoisted rotations apply sigma_g to the ModUp'ed digits.
* Rotation (reading C5): Rot(v, r) moves slot j+r to slot j (paper Sec. II-B),
  Galois element g = 5^(r mod N/2) mod 2N.
* Rescale (reading C7): centred remainder of the top limb; new scale =
  (scale)/q_top in FP64.
* Public-key encryption (reading C14): c = (u*pk0 + e0 + m, u*pk1 + e1).
* Decryption decodes from limb q_0 alone (valid while |m| < q_0/2).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dp = ctypes.POINTER(ctypes.c_double)

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(_build.build())
        u64, i32, vp, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
        sig = {
            "o_mulmod": (u64, [u64, u64, u64]),
            "o_powmod": (u64, [u64, u64, u64]),
            "o_invmod": (u64, [u64, u64]),
            "o_ntt": (None, [vp, i32, u64, u64]),
            "o_intt": (None, [vp, i32, u64, u64]),
            "o_ntt_limbs": (None, [vp, i32, i32, vp, vp]),
            "o_intt_limbs": (None, [vp, i32, i32, vp, vp]),
            "o_mul": (None, [vp, vp, vp, i32, i32, vp]),
            "o_add": (None, [vp, vp, vp, i32, i32, vp]),
            "o_sub": (None, [vp, vp, vp, i32, i32, vp]),
            "o_muladd": (None, [vp, vp, vp, i32, i32, vp]),
            "o_reduce_signed": (None, [vp, vp, i32, i32, vp]),
            "o_automorph_coeff": (None, [vp, vp, i32, i32, u64, vp]),
            "o_automorph_eval": (None, [vp, vp, i32, i32, u64]),
            "o_bconv": (None, [vp, vp, i32, vp, i32, vp, i32]),
            "o_rescale": (None, [vp, vp, i32, i32, vp, vp]),
            "o_moddown": (None, [vp, vp, i32, i32, i32, vp, vp, vp, vp]),
            "o_modup_digit": (None, [vp, vp, i32, i32, i32, i32, i32, vp, vp, vp, vp]),
            "o_rand_word": (u64, [u64, u64, u64]),
            "o_sample_ternary": (None, [vp, u64, u64, i32]),
            "o_sample_cbd": (None, [vp, u64, u64, i32]),
            "o_sample_uniform": (None, [vp, u64, u64, i32, u64]),
            "o_encode": (ctypes.c_int, [vp, vp, vp, i32, dbl]),
            "o_decode": (None, [vp, vp, vp, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    # data_as keeps a reference to the array for as long as the pointer lives
    return a.ctypes.data_as(ctypes.c_void_p)


def _u(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


# ----------------------------------------------------------------- primes
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin; the first twelve prime bases are exact for n < 3.3e24."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def gen_primes(bit_sizes, logn: int) -> list[int]:
    """Largest primes q < 2^bits with q = 1 mod 2N, distinct, in request order."""
    m = 2 << logn
    taken: list[int] = []
    for bits in bit_sizes:
        c = ((1 << bits) - 1) // m * m + 1
        if c >= (1 << bits):
            c -= m
        while c > m:
            if c not in taken and is_prime(c):
                taken.append(c)
                break
            c -= m
        else:
            raise ValueError(f"no {bits}-bit prime = 1 mod {m}")
    return taken


def smallest_psi(q: int, logn: int) -> int:
    """Smallest primitive 2N-th root of unity modulo q."""
    n = 1 << logn
    m = 2 * n
    assert (q - 1) % m == 0
    root = None
    for g in range(2, 1 << 20):
        r = pow(g, (q - 1) // m, q)
        if pow(r, n, q) == q - 1:
            root = r
            break
    assert root is not None
    best, x, r2 = root, root, root * root % q
    for _ in range(n - 1):  # all odd powers root^(2k+1)
        x = x * r2 % q
        if x < best:
            best = x
    return best


# ------------------------------------------------------------- randomness
PURPOSE = {"sk": 1, "pk_a": 2, "pk_e": 3, "ksk_a": 4, "ksk_e": 5,
           "enc_u": 6, "enc_e0": 7, "enc_e1": 8}


def stream_id(purpose: str, key_id: int = 0, digit: int = 0, limb: int = 0) -> int:
    return (PURPOSE[purpose] << 56) | (key_id << 32) | (digit << 16) | limb


def sample_ternary(seed, stream, n):
    out = np.zeros(n, dtype=np.int64)
    lib().o_sample_ternary(_p(out), seed, stream, n)
    return out


def sample_cbd(seed, stream, n):
    out = np.zeros(n, dtype=np.int64)
    lib().o_sample_cbd(_p(out), seed, stream, n)
    return out


def sample_uniform(seed, stream, n, q):
    out = np.zeros(n, dtype=np.uint64)
    lib().o_sample_uniform(_p(out), seed, stream, n, q)
    return out


def galois_elt(r: int, logn: int) -> int:
    """Galois element of a left rotation by r slots: 5^(r mod N/2) mod 2N."""
    m = 1 << (logn - 1)
    return pow(5, r % m, 2 << logn)


def naf_terms(r: int, slots: int):
    """The rotation r (taken mod the slot count, in (-slots/2, slots/2]) as the signed
    powers of two of its non-adjacent form (Reitwiesner 1960), lowest first: every
    nonzero digit d_i in {-1, 1}, no two adjacent, r = sum d_i 2^i."""
    v = r % slots
    if v > slots // 2:
        v -= slots
    out, i = [], 0
    while v != 0:
        if v % 2:
            d = 2 - v % 4          # v = 1 (mod 4) -> +1, v = 3 (mod 4) -> -1
            v -= d
            out.append(d * (1 << i))
        v //= 2
        i += 1
    return out


def pow2_steps(slots: int):
    """The rotation steps of a power-of-two key set: +-2^k for 2^k < slots."""
    k, out = 1, []
    while k < slots:
        out += [k, -k]
        k *= 2
    return out


# ------------------------------------------------------------ the scheme
@dataclass
class Ct:
    """A ciphertext (c0, c1): array [2][L'][N] of residues, natural-order eval form."""
    d: np.ndarray
    scale: float

    @property
    def lp(self) -> int:
        return self.d.shape[1]

    def copy(self) -> "Ct":
        return Ct(self.d.copy(), self.scale)


@dataclass
class Keys:
    s: np.ndarray                     # [L+1+K][N] eval
    pk: np.ndarray                    # [2][L+1][N]
    rlk: tuple | None = None          # (b [dnum][L+1+K][N], a [...])
    gk: dict = field(default_factory=dict)  # galois element -> (b, a)


class Ckks:
    def __init__(self, logn: int, data_bits, special_bits, dnum: int, log2_scale: float, seed: int):
        self.logn = logn
        self.n = 1 << logn
        allp = gen_primes(list(data_bits) + list(special_bits), logn)
        self.q = allp[: len(data_bits)]
        self.p = allp[len(data_bits):]
        self.L1 = len(self.q)            # number of data primes (L+1)
        self.K = len(self.p)
        self.dnum = dnum
        self.alpha = -(-self.L1 // dnum)
        self.scale = 2.0 ** log2_scale
        self.seed = seed
        self.qpsi = [smallest_psi(q, logn) for q in self.q]
        self.ppsi = [smallest_psi(p, logn) for p in self.p]
        self.keys: Keys | None = None

    # ---- bases
    def primes_all(self):
        return self.q + self.p

    def qa(self, lp):
        return _u(self.q[:lp])

    def qpsia(self, lp):
        return _u(self.qpsi[:lp])

    def ext_basis(self, lp):
        """(primes, psis) of Q_l u P as arrays."""
        return _u(self.q[:lp] + self.p), _u(self.qpsi[:lp] + self.ppsi)

    # ---- transforms
    def ntt(self, a: np.ndarray, primes, psis) -> np.ndarray:
        a = _u(a).copy()
        lib().o_ntt_limbs(_p(a), a.shape[0], self.logn, _p(_u(primes)), _p(_u(psis)))
        return a

    def intt(self, a: np.ndarray, primes, psis) -> np.ndarray:
        a = _u(a).copy()
        lib().o_intt_limbs(_p(a), a.shape[0], self.logn, _p(_u(primes)), _p(_u(psis)))
        return a

    def reduce_signed(self, v: np.ndarray, primes) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.int64)
        primes = _u(primes)
        out = np.zeros((len(primes), self.n), dtype=np.uint64)
        lib().o_reduce_signed(_p(out), _p(v), len(primes), self.n, _p(primes))
        return out

    def _bin(self, fn, a, b, primes):
        primes = _u(primes)
        a, b = _u(a), _u(b)
        out = np.zeros_like(a)
        getattr(lib(), fn)(_p(out), _p(a), _p(b), a.shape[0], self.n, _p(primes))
        return out

    def mul(self, a, b, primes):
        return self._bin("o_mul", a, b, primes)

    def add(self, a, b, primes):
        return self._bin("o_add", a, b, primes)

    def sub(self, a, b, primes):
        return self._bin("o_sub", a, b, primes)

    def neg(self, a, primes):
        return self.sub(np.zeros_like(a), a, primes)

    def automorph_eval(self, a, g):
        a = _u(a)
        out = np.zeros_like(a)
        lib().o_automorph_eval(_p(out), _p(a), a.shape[0], self.logn, g)
        return out

    def automorph_coeff(self, a, g, primes):
        a = _u(a)
        out = np.zeros_like(a)
        lib().o_automorph_coeff(_p(out), _p(a), a.shape[0], self.logn, g, _p(_u(primes)))
        return out

    # ---- encoding
    def encode_coeffs(self, z, scale: float) -> np.ndarray:
        """Slot values (length N/2, real or complex) -> rounded integer coefficients."""
        z = np.asarray(z)
        m = self.n // 2
        assert z.shape == (m,)
        zre = np.ascontiguousarray(z.real, dtype=np.float64)
        zim = np.ascontiguousarray(z.imag if np.iscomplexobj(z) else np.zeros(m), dtype=np.float64)
        out = np.zeros(self.n, dtype=np.int64)
        rc = lib().o_encode(_p(out), _p(zre), _p(zim), self.logn, float(scale))
        if rc != 0:
            raise OverflowError("encoded coefficient exceeds 2^63")
        return out

    def encode(self, z, scale: float, lp: int) -> np.ndarray:
        """Plaintext at level lp in eval form: [lp][N]."""
        return self.ntt(self.reduce_signed(self.encode_coeffs(z, scale), self.q[:lp]),
                        self.q[:lp], self.qpsi[:lp])

    def decode_coeffs(self, coef: np.ndarray) -> np.ndarray:
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        m = self.n // 2
        zre = np.zeros(m)
        zim = np.zeros(m)
        lib().o_decode(_p(zre), _p(zim), _p(coef), self.logn)
        return zre + 1j * zim

    # ---- keys
    def keygen(self, rot_steps=()):
        n, seed = self.n, self.seed
        allq = self.primes_all()
        allpsi = self.qpsi + self.ppsi
        s_int = sample_ternary(seed, stream_id("sk"), n)
        s = self.ntt(self.reduce_signed(s_int, allq), allq, allpsi)
        # public key over the data primes
        qd = self.q
        a = np.stack([sample_uniform(seed, stream_id("pk_a", 0, 0, l), n, qd[l]) for l in range(self.L1)])
        a = self.ntt(a, qd, self.qpsi)
        e = self.ntt(self.reduce_signed(sample_cbd(seed, stream_id("pk_e"), n), qd), qd, self.qpsi)
        pk0 = self.add(self.neg(self.mul(a, s[: self.L1], qd), qd), e, qd)
        self.keys = Keys(s=s, pk=np.stack([pk0, a]))
        s2 = self.mul(s, s, allq)
        self.keys.rlk = self.make_ksk(s2, key_id=0)
        for r in rot_steps:
            self.add_galois_key(galois_elt(r, self.logn))
        return self.keys

    def add_galois_key(self, g: int):
        if g in self.keys.gk or g == 1:
            return
        sg = self.automorph_eval(self.keys.s, g)
        self.keys.gk[g] = self.make_ksk(sg, key_id=g)

    def P_mod(self, qi: int) -> int:
        v = 1
        for p in self.p:
            v = v * p % qi
        return v

    def make_ksk(self, sprime: np.ndarray, key_id: int):
        """Hybrid key-switching key: b_j = -a_j s + e_j + P*Qtilde_j*s' over Q u P."""
        n, seed = self.n, self.seed
        allq = self.primes_all()
        allpsi = self.qpsi + self.ppsi
        nt = len(allq)
        bs, as_ = [], []
        for j in range(self.dnum):
            a = np.stack([sample_uniform(seed, stream_id("ksk_a", key_id, j, t), n, allq[t]) for t in range(nt)])
            a = self.ntt(a, allq, allpsi)
            e = self.ntt(self.reduce_signed(sample_cbd(seed, stream_id("ksk_e", key_id, j), n), allq), allq, allpsi)
            b = self.add(self.neg(self.mul(a, self.keys.s, allq), allq), e, allq)
            for t in range(j * self.alpha, min((j + 1) * self.alpha, self.L1)):
                pm = np.full(n, self.P_mod(self.q[t]), dtype=np.uint64)
                term = self.mul(pm[None, :], sprime[t:t + 1], [self.q[t]])
                b[t:t + 1] = self.add(b[t:t + 1], term, [self.q[t]])
            bs.append(b)
            as_.append(a)
        return np.stack(bs), np.stack(as_)

    # ---- encryption
    def encrypt_coeffs(self, m_int: np.ndarray, scale: float, enc_seed: int, lp: int | None = None) -> Ct:
        lp = self.L1 if lp is None else lp
        n = self.n
        q, psi = self.q[:lp], self.qpsi[:lp]
        u = self.ntt(self.reduce_signed(sample_ternary(enc_seed, stream_id("enc_u"), n), q), q, psi)
        e0 = sample_cbd(enc_seed, stream_id("enc_e0"), n)
        e1 = sample_cbd(enc_seed, stream_id("enc_e1"), n)
        me = self.ntt(self.reduce_signed(m_int + e0, q), q, psi)
        e1 = self.ntt(self.reduce_signed(e1, q), q, psi)
        c0 = self.add(self.mul(u, self.keys.pk[0][:lp], q), me, q)
        c1 = self.add(self.mul(u, self.keys.pk[1][:lp], q), e1, q)
        return Ct(np.stack([c0, c1]), scale)

    def encrypt(self, slots, enc_seed: int, lp: int | None = None) -> Ct:
        return self.encrypt_coeffs(self.encode_coeffs(slots, self.scale), self.scale, enc_seed, lp)

    def decrypt_coeffs(self, ct: Ct) -> np.ndarray:
        """Centred integer coefficients of m = c0 + c1*s, from limb q_0."""
        lp = ct.lp
        q = self.q[:lp]
        m = self.add(ct.d[0], self.mul(ct.d[1], self.keys.s[:lp], q), q)
        m0 = self.intt(m[:1], q[:1], self.qpsi[:1])[0]
        q0 = self.q[0]
        return np.where(m0 > q0 // 2, m0.astype(np.int64) - np.int64(q0), m0.astype(np.int64))

    def decrypt(self, ct: Ct) -> np.ndarray:
        coef = self.decrypt_coeffs(ct)
        return self.decode_coeffs(coef.astype(np.float64) / ct.scale).real

    # ---- ciphertext arithmetic
    def to_coeff(self, ct: Ct) -> np.ndarray:
        q, psi = self.q[: ct.lp], self.qpsi[: ct.lp]
        return np.stack([self.intt(ct.d[0], q, psi), self.intt(ct.d[1], q, psi)])

    def ct_add(self, a: Ct, b: Ct) -> Ct:
        assert a.lp == b.lp and a.scale == b.scale, "level/scale mismatch"
        q = self.q[: a.lp]
        return Ct(np.stack([self.add(a.d[0], b.d[0], q), self.add(a.d[1], b.d[1], q)]), a.scale)

    def drop_level(self, a: Ct) -> Ct:
        """Drop-Level (Sec. IV-A, reading C11) as a modulus drop: the top limb of each
        polynomial is discarded; message and scale are unchanged."""
        assert a.lp >= 2, "level exhausted"
        return Ct(np.ascontiguousarray(a.d[:, : a.lp - 1]), a.scale)

    def ct_add_plain(self, a: Ct, pt: np.ndarray) -> Ct:
        q = self.q[: a.lp]
        return Ct(np.stack([self.add(a.d[0], pt, q), a.d[1].copy()]), a.scale)

    def ct_mul_plain(self, a: Ct, pt: np.ndarray, pt_scale: float) -> Ct:
        q = self.q[: a.lp]
        return Ct(np.stack([self.mul(a.d[0], pt, q), self.mul(a.d[1], pt, q)]), a.scale * pt_scale)

    def rescale(self, a: Ct) -> Ct:
        lp = a.lp
        assert lp >= 2, "level exhausted"
        q, psi = _u(self.q[:lp]), _u(self.qpsi[:lp])
        out = np.zeros((2, lp - 1, self.n), dtype=np.uint64)
        for k in range(2):
            src = np.ascontiguousarray(a.d[k])
            dst = np.zeros((lp - 1, self.n), dtype=np.uint64)
            lib().o_rescale(_p(dst), _p(src), lp, self.logn, _p(q), _p(psi))
            out[k] = dst
        return Ct(out, a.scale / float(self.q[lp - 1]))

    # ---- key switching
    def digits(self, lp: int):
        return [(lo, min(lo + self.alpha, lp)) for lo in range(0, lp, self.alpha)]

    def modup(self, x: np.ndarray) -> np.ndarray:
        """x [lp][N] eval -> [beta][lp+K][N] eval (one extended copy per digit)."""
        lp = x.shape[0]
        x = _u(x)
        q, qpsi, p, ppsi = _u(self.q[:lp]), _u(self.qpsi[:lp]), _u(self.p), _u(self.ppsi)
        ds = self.digits(lp)
        out = np.zeros((len(ds), lp + self.K, self.n), dtype=np.uint64)
        for j, (lo, hi) in enumerate(ds):
            o = np.zeros((lp + self.K, self.n), dtype=np.uint64)
            lib().o_modup_digit(_p(o), _p(x), lo, hi, lp, self.K, self.logn,
                                _p(q), _p(qpsi), _p(p), _p(ppsi))
            out[j] = o
        return out

    def key_limbs(self, key_poly: np.ndarray, lp: int) -> np.ndarray:
        """Restrict a key polynomial over Q u P to Q_l u P."""
        return np.ascontiguousarray(np.concatenate([key_poly[:lp], key_poly[self.L1:]], axis=0))

    def ks_inner(self, digs: np.ndarray, key, g: int = 1):
        lp = digs.shape[1] - self.K
        basis, _ = self.ext_basis(lp)
        kb, ka = key
        acc0 = np.zeros((lp + self.K, self.n), dtype=np.uint64)
        acc1 = np.zeros_like(acc0)
        for j in range(digs.shape[0]):
            d = digs[j] if g == 1 else self.automorph_eval(digs[j], g)
            d = _u(d)
            lib().o_muladd(_p(acc0), _p(d), _p(self.key_limbs(kb[j], lp)), lp + self.K, self.n, _p(basis))
            lib().o_muladd(_p(acc1), _p(d), _p(self.key_limbs(ka[j], lp)), lp + self.K, self.n, _p(basis))
        return acc0, acc1

    def moddown(self, acc: np.ndarray) -> np.ndarray:
        lp = acc.shape[0] - self.K
        out = np.zeros((lp, self.n), dtype=np.uint64)
        lib().o_moddown(_p(out), _p(_u(acc)), lp, self.K, self.logn,
                        _p(_u(self.q[:lp])), _p(_u(self.qpsi[:lp])), _p(_u(self.p)), _p(_u(self.ppsi)))
        return out

    def moddown_rescale(self, acc: np.ndarray) -> np.ndarray:
        """ModDown and rescale as one division by D = q_top * P: the dropped basis is
        the top data prime and the special primes, and (reading C6/C7 applied to
        that basis) out_i = (acc_i - BConv_{D->q_i}([acc]_D)) * D^{-1} mod q_i for
        the lp - 1 remaining limbs, fast base conversion without correction.
        acc [lp+K][N] over Q_l u P (data limbs, then special) -> [lp-1][N]:
        floor(x / D) - e with 0 <= e < K + 1.  Equals ModDown then rescale up to
        that rounding (one base conversion instead of two)."""
        lp = acc.shape[0] - self.K
        assert lp >= 2, "level exhausted"
        out = np.zeros((lp - 1, self.n), dtype=np.uint64)
        drop = [self.q[lp - 1]] + list(self.p)
        dpsi = [self.qpsi[lp - 1]] + list(self.ppsi)
        lib().o_moddown(_p(out), _p(_u(acc)), lp - 1, self.K + 1, self.logn,
                        _p(_u(self.q[:lp - 1])), _p(_u(self.qpsi[:lp - 1])), _p(_u(drop)), _p(_u(dpsi)))
        return out

    def keyswitch(self, x: np.ndarray, key):
        acc0, acc1 = self.ks_inner(self.modup(x), key)
        return self.moddown(acc0), self.moddown(acc1)

    def rotate(self, ct: Ct, r: int) -> Ct:
        """Single rotation: sigma_g on (c0, c1), then key switching of sigma_g(c1)."""
        g = galois_elt(r, self.logn)
        if g == 1:
            return ct.copy()
        q = self.q[: ct.lp]
        c0 = self.automorph_eval(ct.d[0], g)
        c1 = self.automorph_eval(ct.d[1], g)
        k0, k1 = self.keyswitch(c1, self.keys.gk[g])
        return Ct(np.stack([self.add(c0, k0, q), k1]), ct.scale)

    def rotate_naf(self, ct: Ct, r: int, cache=None) -> Ct:
        """Rot(ct, r) with power-of-two keys only: the rotations of naf_terms(r) applied
        one after another, lowest first.  cache maps a partial sum of those terms to its
        ciphertext, so the rotations of one input share their common prefixes (the
        prefix of a non-adjacent form is the non-adjacent form of the partial sum)."""
        cur, acc = ct, 0
        for t in naf_terms(r, self.n // 2):
            acc += t
            if cache is not None and acc in cache:
                cur = cache[acc]
                continue
            cur = self.rotate(cur, t)
            if cache is not None:
                cache[acc] = cur
        return cur if acc else ct.copy()

    def rotate_hoisted(self, ct: Ct, steps) -> dict:
        """Several rotations of one ciphertext sharing one ModUp of c1."""
        out = {}
        digs = None
        q = self.q[: ct.lp]
        for r in steps:
            g = galois_elt(r, self.logn)
            if g == 1:
                out[r] = ct.copy()
                continue
            if digs is None:
                digs = self.modup(ct.d[1])
            acc0, acc1 = self.ks_inner(digs, self.keys.gk[g], g)
            c0 = self.automorph_eval(ct.d[0], g)
            out[r] = Ct(np.stack([self.add(c0, self.moddown(acc0), q), self.moddown(acc1)]), ct.scale)
        return out

    def encode_ext(self, z, scale: float, lp: int) -> np.ndarray:
        """Plaintext over Q_l u P (eval form, [lp+K][N]): the same rounded integer
        polynomial as ``encode`` reduced into the special primes as well."""
        basis, psis = self.ext_basis(lp)
        return self.ntt(self.reduce_signed(self.encode_coeffs(z, scale), basis), basis, psis)

    def lincomb(self, cts, steps, weights=None, pt_scale: float = 1.0, rescale: bool = False):
        """Hoisted linear combination of rotations with one ModDown per output:

            Y_o = sum_i sum_s w[o][i][s] (.) Rot(ct_i, steps[s])

        computed as Y_o = ModDown(Z_o), Z_o = sum_{i,s} w[o][i][s] (.) A_{i,s} over Q_l u P, where
            A_{i,s} = (sum_j sigma_g(D_j) (.) ksk_g,j,0 + P*sigma_g(c0),  sum_j sigma_g(D_j) (.) ksk_g,j,1)
        (D = ModUp(c1) of ct_i, g = 5^steps[s]) and A_{i,s} = (P*c0, P*c1) for a step of 0.
        Because ModDown(A + P*x) = ModDown(A) + x exactly, Y_o decrypts to the same
        message as the rotate-then-multiply composition; only the rounding of the
        single ModDown differs.  w[o][i][s] are plaintexts over Q_l u P (``encode_ext``)
        or None (all ones, a plain sum of rotations); the output scale is
        ct.scale * pt_scale.  With rescale, each output is also rescaled: the
        single division by q_top * P of ``moddown_rescale`` replaces ModDown."""
        lp = cts[0].lp
        K = self.K
        E = lp + K
        basis, _ = self.ext_basis(lp)
        q = self.q[:lp]
        pq = np.array([self.P_mod(qi) for qi in q], dtype=np.uint64)
        Pq = np.repeat(pq[:, None], self.n, axis=1)
        zero_p = np.zeros((K, self.n), dtype=np.uint64)
        A = []   # A[i][s] = (a0, a1) over E limbs
        for ct in cts:
            assert ct.lp == lp and ct.scale == cts[0].scale
            digs = None
            row = []
            for r in steps:
                g = galois_elt(r, self.logn)
                if g == 1:
                    a0 = np.concatenate([self.mul(ct.d[0], Pq, q), zero_p])
                    a1 = np.concatenate([self.mul(ct.d[1], Pq, q), zero_p])
                else:
                    if digs is None:
                        digs = self.modup(ct.d[1])
                    a0, a1 = self.ks_inner(digs, self.keys.gk[g], g)
                    c0g = self.automorph_eval(ct.d[0], g)
                    a0 = np.concatenate([self.add(a0[:lp], self.mul(c0g, Pq, q), q), a0[lp:]])
                row.append((a0, a1))
            A.append(row)
        n_out = 1 if weights is None else len(weights)
        outs = []
        for o in range(n_out):
            z0 = np.zeros((E, self.n), dtype=np.uint64)
            z1 = np.zeros_like(z0)
            for i in range(len(cts)):
                for s in range(len(steps)):
                    a0, a1 = A[i][s]
                    if weights is None:
                        z0 = self.add(z0, a0, basis)
                        z1 = self.add(z1, a1, basis)
                    else:
                        w = weights[o][i][s]
                        lib().o_muladd(_p(z0), _p(_u(a0)), _p(_u(w)), E, self.n, _p(basis))
                        lib().o_muladd(_p(z1), _p(_u(a1)), _p(_u(w)), E, self.n, _p(basis))
            if rescale:
                outs.append(Ct(np.stack([self.moddown_rescale(z0), self.moddown_rescale(z1)]),
                               cts[0].scale * pt_scale / float(self.q[lp - 1])))
            else:
                outs.append(Ct(np.stack([self.moddown(z0), self.moddown(z1)]), cts[0].scale * pt_scale))
        return outs

    def lincomb_diag(self, cts, steps) -> Ct:
        """sum_i Rot(ct_i, steps[i]) with one ModDown: each input contributes the
        accumulator A_i of its own step (as in ``lincomb``), the A_i are added over
        Q_l u P and ModDown is applied once."""
        lp = cts[0].lp
        basis, _ = self.ext_basis(lp)
        E = lp + self.K
        z0 = np.zeros((E, self.n), dtype=np.uint64)
        z1 = np.zeros_like(z0)
        for ct, r in zip(cts, steps):
            assert ct.lp == lp and ct.scale == cts[0].scale
            # a one-step combination with no weights gives exactly the accumulator pair
            a0, a1 = self._lazy_acc(ct, r)
            z0 = self.add(z0, a0, basis)
            z1 = self.add(z1, a1, basis)
        return Ct(np.stack([self.moddown(z0), self.moddown(z1)]), cts[0].scale)

    def lincomb_chan(self, cts, steps, weights, pt_scale: float, rescale: bool = False) -> Ct:
        """One output from inputs that each have their own rotation steps:

            Y = sum_i sum_k w[i][k] (.) Rot(ct_i, steps[i][k])

        Each input's rotations share one ModUp (hoisting); the weighted accumulator pairs
        (see ``lincomb``) of every input and step are summed over Q_l u P and ModDown runs
        once -- or, with rescale, the single division by q_top * P.  w[i][k] are plaintexts
        over Q_l u P; the output scale is ct.scale * pt_scale (then / q_top)."""
        lp = cts[0].lp
        E = lp + self.K
        basis, _ = self.ext_basis(lp)
        z0 = np.zeros((E, self.n), dtype=np.uint64)
        z1 = np.zeros_like(z0)
        for ct, st, ws in zip(cts, steps, weights):
            assert ct.lp == lp and ct.scale == cts[0].scale and len(st) == len(ws)
            digs = self.modup(ct.d[1]) if any(galois_elt(r, self.logn) != 1 for r in st) else None
            for r, w in zip(st, ws):
                a0, a1 = self._lazy_acc(ct, r, digs)
                lib().o_muladd(_p(z0), _p(_u(a0)), _p(_u(w)), E, self.n, _p(basis))
                lib().o_muladd(_p(z1), _p(_u(a1)), _p(_u(w)), E, self.n, _p(basis))
        if rescale:
            return Ct(np.stack([self.moddown_rescale(z0), self.moddown_rescale(z1)]),
                      cts[0].scale * pt_scale / float(self.q[lp - 1]))
        return Ct(np.stack([self.moddown(z0), self.moddown(z1)]), cts[0].scale * pt_scale)

    def _lazy_acc(self, ct: Ct, r: int, digs=None):
        """The Q_l u P accumulator pair of Rot(ct, r) before ModDown (see ``lincomb``)."""
        lp = ct.lp
        q = self.q[:lp]
        zero_p = np.zeros((self.K, self.n), dtype=np.uint64)
        Pq = np.repeat(np.array([self.P_mod(qi) for qi in q], dtype=np.uint64)[:, None], self.n, axis=1)
        g = galois_elt(r, self.logn)
        if g == 1:
            return (np.concatenate([self.mul(ct.d[0], Pq, q), zero_p]),
                    np.concatenate([self.mul(ct.d[1], Pq, q), zero_p]))
        if digs is None:
            digs = self.modup(ct.d[1])
        a0, a1 = self.ks_inner(digs, self.keys.gk[g], g)
        c0g = self.automorph_eval(ct.d[0], g)
        return np.concatenate([self.add(a0[:lp], self.mul(c0g, Pq, q), q), a0[lp:]]), a1

    def tensor_square(self, ct: Ct):
        """(d0, d1, d2) = (a0^2, 2 a0 a1, a1^2): decrypts with (1, s, s^2) to m^2."""
        q = self.q[: ct.lp]
        a0, a1 = ct.d[0], ct.d[1]
        return (self.mul(a0, a0, q), self.add(self.mul(a0, a1, q), self.mul(a1, a0, q), q),
                self.mul(a1, a1, q))

    def relinearise(self, d, scale: float) -> Ct:
        """(d0, d1) + KS(d2): the key switch of d2 with the relinearisation key (ModUp,
        inner product, ModDown of each polynomial) added to (d0, d1)."""
        d0, d1, d2 = d
        q = self.q[: d0.shape[0]]
        k0, k1 = self.keyswitch(d2, self.keys.rlk)
        return Ct(np.stack([self.add(d0, k0, q), self.add(d1, k1, q)]), scale)

    def square_literal(self, ct: Ct) -> Ct:
        """Mul (C) of a ciphertext by itself in the textbook order (reading C15), one step
        at a time: the tensor, relinearisation, then the centred rescale of reading C7."""
        assert ct.lp >= 2, "level exhausted"
        return self.rescale(self.relinearise(self.tensor_square(ct), ct.scale * ct.scale))

    def square(self, ct: Ct) -> Ct:
        """Ciphertext tensor with itself, relinearisation, rescale (reading C15).
        Relinearisation and rescale end in one division by q_top * P: the key-switch
        accumulators of d2 over Q_l u P get P*(d0, d1) added on the data limbs
        (ModDown(A + P*d) = ModDown(A) + d) and go through ``moddown_rescale``."""
        lp = ct.lp
        assert lp >= 2, "level exhausted"
        q = self.q[:lp]
        a0, a1 = ct.d[0], ct.d[1]
        d0 = self.mul(a0, a0, q)
        d1 = self.add(self.mul(a0, a1, q), self.mul(a1, a0, q), q)
        d2 = self.mul(a1, a1, q)
        acc0, acc1 = self.ks_inner(self.modup(d2), self.keys.rlk)
        Pq = np.repeat(np.array([self.P_mod(qi) for qi in q], dtype=np.uint64)[:, None], self.n, axis=1)
        acc0 = np.concatenate([self.add(acc0[:lp], self.mul(d0, Pq, q), q), acc0[lp:]])
        acc1 = np.concatenate([self.add(acc1[:lp], self.mul(d1, Pq, q), q), acc1[lp:]])
        return Ct(np.stack([self.moddown_rescale(acc0), self.moddown_rescale(acc1)]),
                  ct.scale * ct.scale / float(self.q[lp - 1]))
