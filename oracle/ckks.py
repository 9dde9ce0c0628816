"""Leveled RNS-CKKS, step by step (test infrastructure only).

Follows Sec. 2.2 of the paper: R_Q = Z_Q[x]/(x^N+1), Q = q_0*...*q_L held as
L+1 residue polynomials of native 64-bit words; encoding scales by Delta and
rounds; add/mult act slot-wise; rotation shifts the N/2 slots cyclically;
rescale divides by the last prime and drops one level; a special modulus P
(here alpha primes) serves hybrid key switching.  The paper uses SEAL and does
not spell out the scheme's internal conventions, so this module fixes them as
follows (each is a reading of a silent point):

* ciphertexts are (c0, c1) with c0 + c1*s = m + e, kept in the NTT domain;
* secret key s is ternary; errors are centered-binomial with eta = 21;
* "uniform" polynomials (key and encryption masks) are drawn directly in the
  NTT domain, which has the same distribution as drawing them in the
  coefficient domain;
* hybrid key switching splits the active primes into digits of alpha
  consecutive primes; ModUp is the fast approximate basis conversion, the key
  of digit j encrypts P * e_j * s' where e_j is the CRT idempotent of digit j;
  ModDown subtracts the centred P-part and multiplies by P^-1;
* rotation by r uses the Galois element 5^r mod 2N (slots move left by r);
* rescale subtracts the centred top residue and multiplies by q_l^-1.

Every modular operation goes through ckks_ref.c, whose routines are the plain
definitions.  Nothing here is blocked, fused or reordered.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import build as _build

_lib = None

U64P = ctypes.POINTER(ctypes.c_uint64)
I64P = ctypes.POINTER(ctypes.c_int64)
U32P = ctypes.POINTER(ctypes.c_uint32)
DBLP = ctypes.POINTER(ctypes.c_double)

# random-stream domains (key word 2 of the ChaCha20 key)
DOM_SECRET = 1
DOM_KEY_A = 2
DOM_KEY_E = 3
DOM_ENC_A = 4
DOM_ENC_E = 5


def lib():
    """Load (building if needed) the oracle's C routines."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u64, i32, sz, u32, dbl = (ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t,
                                  ctypes.c_uint32, ctypes.c_double)
        sig = {
            "orc_mulmod": (u64, [u64, u64, u64]),
            "orc_powmod": (u64, [u64, u64, u64]),
            "orc_invmod": (u64, [u64, u64]),
            "orc_is_prime": (i32, [u64]),
            "orc_gen_primes": (i32, [i32, i32, u64, U64P, i32, U64P]),
            "orc_root_2n": (u64, [u64, u64]),
            "orc_ntt_naive": (None, [U64P, U64P, i32, u64, u64]),
            "orc_ntt": (None, [U64P, i32, u64, u64]),
            "orc_intt": (None, [U64P, i32, u64, u64]),
            "orc_negacyclic_naive": (None, [U64P, U64P, U64P, i32, u64]),
            "orc_vec_add": (None, [U64P, U64P, U64P, sz, u64]),
            "orc_vec_sub": (None, [U64P, U64P, U64P, sz, u64]),
            "orc_vec_neg": (None, [U64P, U64P, sz, u64]),
            "orc_vec_mul": (None, [U64P, U64P, U64P, sz, u64]),
            "orc_vec_mul_scalar": (None, [U64P, u64, U64P, sz, u64]),
            "orc_vec_add_scalar": (None, [U64P, u64, U64P, sz, u64]),
            "orc_vec_from_signed": (None, [I64P, U64P, sz, u64]),
            "orc_basis_convert": (None, [U64P, U64P, i32, u64, U64P, sz]),
            "orc_conv_overflow": (None, [U64P, U64P, i32, U64P, sz]),
            "orc_chacha20_block": (None, [U32P, u32, U32P, U32P]),
            "orc_stream_words": (None, [u64, u32, u32, u32, U32P, sz]),
            "orc_sample_uniform": (None, [u64, u32, u32, u32, u64, U64P, sz]),
            "orc_sample_ternary": (None, [u64, u32, u32, u32, I64P, sz]),
            "orc_sample_cbd": (None, [u64, u32, u32, u32, I64P, sz]),
            "orc_encode": (None, [DBLP, DBLP, i32, dbl, DBLP]),
            "orc_vec_from_double": (None, [DBLP, U64P, sz, u64]),
            "orc_encode_naive": (None, [DBLP, DBLP, i32, dbl, DBLP]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray, ptr):
    assert a.flags["C_CONTIGUOUS"], "array must be contiguous"
    return a.ctypes.data_as(ptr)


# ------------------------------------------------------------ small helpers

def mulmod(a, b, q):
    return lib().orc_mulmod(a, b, q)


def invmod(a, q):
    return lib().orc_invmod(a % q, q)


def is_prime(n: int) -> bool:
    return bool(lib().orc_is_prime(n))


def gen_primes(bits: int, count: int, two_n: int, exclude: Sequence[int] = ()) -> List[int]:
    out = np.zeros(count, dtype=np.uint64)
    ex = np.array(list(exclude) or [0], dtype=np.uint64)
    got = lib().orc_gen_primes(bits, count, two_n, _p(ex, U64P), len(exclude), _p(out, U64P))
    if got != count:
        raise ValueError("not enough %d-bit primes = 1 mod %d" % (bits, two_n))
    return [int(x) for x in out]


def ntt(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().orc_ntt(_p(out, U64P), int(out.size).bit_length() - 1, q, psi)
    return out


def intt(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.uint64).copy()
    lib().orc_intt(_p(out, U64P), int(out.size).bit_length() - 1, q, psi)
    return out


def ntt_naive(a: np.ndarray, q: int, psi: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().orc_ntt_naive(_p(a, U64P), _p(out, U64P), int(a.size).bit_length() - 1, q, psi)
    return out


def negacyclic_naive(a, b, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.zeros_like(a)
    lib().orc_negacyclic_naive(_p(a, U64P), _p(b, U64P), _p(out, U64P),
                               int(a.size).bit_length() - 1, q)
    return out


def _vec2(fn, a, b, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.empty_like(a)
    getattr(lib(), fn)(_p(a, U64P), _p(b, U64P), _p(out, U64P), a.size, q)
    return out


def vadd(a, b, q):
    return _vec2("orc_vec_add", a, b, q)


def vsub(a, b, q):
    return _vec2("orc_vec_sub", a, b, q)


def vmul(a, b, q):
    return _vec2("orc_vec_mul", a, b, q)


def vneg(a, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_vec_neg(_p(a, U64P), _p(out, U64P), a.size, q)
    return out


def vmul_scalar(a, c, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_vec_mul_scalar(_p(a, U64P), int(c) % q, _p(out, U64P), a.size, q)
    return out


def vadd_scalar(a, c, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.empty_like(a)
    lib().orc_vec_add_scalar(_p(a, U64P), int(c) % q, _p(out, U64P), a.size, q)
    return out


def from_signed(a: np.ndarray, q: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int64)
    out = np.empty(a.shape, dtype=np.uint64)
    lib().orc_vec_from_signed(_p(a, I64P), _p(out, U64P), a.size, q)
    return out


def basis_convert(x: np.ndarray, q_in: Sequence[int], t: int) -> np.ndarray:
    """Fast (approximate) basis conversion of limbs x[i] mod q_in[i] to mod t."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    qi = np.array(q_in, dtype=np.uint64)
    n = x.shape[-1]
    out = np.empty(n, dtype=np.uint64)
    lib().orc_basis_convert(_p(x, U64P), _p(qi, U64P), len(q_in), t, _p(out, U64P), n)
    return out


def conv_overflow(x: np.ndarray, q_in: Sequence[int]) -> np.ndarray:
    """u with basis_convert(x, q_in, t) = x + u*Qin (mod t): the number of
    times the fast conversion overshoots, found exactly (0 <= u < len(q_in))."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    qi = np.array(q_in, dtype=np.uint64)
    n = x.shape[-1]
    out = np.empty(n, dtype=np.uint64)
    lib().orc_conv_overflow(_p(x, U64P), _p(qi, U64P), len(q_in), _p(out, U64P), n)
    return out


def stream_words(seed, domain, id0, id1, n_words):
    out = np.empty(n_words, dtype=np.uint32)
    lib().orc_stream_words(seed, domain, id0, id1, _p(out, U32P), n_words)
    return out


def chacha20_block(key_words, counter, nonce_words):
    k = np.array(key_words, dtype=np.uint32)
    nn = np.array(nonce_words, dtype=np.uint32)
    out = np.empty(16, dtype=np.uint32)
    lib().orc_chacha20_block(_p(k, U32P), counter, _p(nn, U32P), _p(out, U32P))
    return out


def sample_uniform(seed, domain, id0, id1, q, n):
    out = np.empty(n, dtype=np.uint64)
    lib().orc_sample_uniform(seed, domain, id0, id1, q, _p(out, U64P), n)
    return out


def sample_ternary(seed, domain, id0, id1, n):
    out = np.empty(n, dtype=np.int64)
    lib().orc_sample_ternary(seed, domain, id0, id1, _p(out, I64P), n)
    return out


def sample_cbd(seed, domain, id0, id1, n):
    out = np.empty(n, dtype=np.int64)
    lib().orc_sample_cbd(seed, domain, id0, id1, _p(out, I64P), n)
    return out


def from_double(a: np.ndarray, q: int) -> np.ndarray:
    """Integral doubles -> residues mod q (exact at any magnitude)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty(a.shape, dtype=np.uint64)
    lib().orc_vec_from_double(_p(a, DBLP), _p(out, U64P), a.size, q)
    return out


def encode_coeffs(z: np.ndarray, logn: int, scale: float) -> np.ndarray:
    """Integer coefficients round(scale * sigma^-1(z)) in the fixed FFT order,
    as integral doubles."""
    n = 1 << (logn - 1)
    z = np.asarray(z, dtype=np.complex128)
    zz = np.zeros(n, dtype=np.complex128)
    zz[: z.size] = z
    re = np.ascontiguousarray(zz.real)
    im = np.ascontiguousarray(zz.imag)
    out = np.empty(2 * n, dtype=np.float64)
    lib().orc_encode(_p(re, DBLP), _p(im, DBLP), logn, float(scale), _p(out, DBLP))
    return out


def encode_naive(z: np.ndarray, logn: int, scale: float) -> np.ndarray:
    n = 1 << (logn - 1)
    zz = np.zeros(n, dtype=np.complex128)
    zz[: np.asarray(z).size] = z
    re = np.ascontiguousarray(zz.real)
    im = np.ascontiguousarray(zz.imag)
    out = np.empty(2 * n, dtype=np.float64)
    lib().orc_encode_naive(_p(re, DBLP), _p(im, DBLP), logn, float(scale), _p(out, DBLP))
    return out


def decode_coeffs(m: Sequence[float], logn: int, scale: float) -> np.ndarray:
    """Slots z_j = m(zeta^(5^j)) / scale, evaluated through numpy's FFT:
    with v_k = m_k + i m_{k+n}, z_j = sum_k (v_k zeta^k) exp(2 pi i k t_j / n)."""
    N = 1 << logn
    n = N // 2
    m = np.asarray(m, dtype=np.float64)
    v = (m[:n] + 1j * m[n:]) / scale
    k = np.arange(n)
    y = np.fft.ifft(v * np.exp(1j * np.pi * k / N)) * n
    e = np.empty(n, dtype=np.int64)
    acc = 1
    for j in range(n):
        e[j] = acc
        acc = acc * 5 % (2 * N)
    return y[(e - 1) // 4]


def galois_elt(step: int, N: int) -> int:
    """Galois element 5^r mod 2N of a left rotation by r slots."""
    n = N // 2
    return pow(5, step % n, 2 * N)


def automorphism_coeff(a: np.ndarray, k: int, q: int) -> np.ndarray:
    """a(x) -> a(x^k) in Z_q[x]/(x^N+1), by its definition on coefficients."""
    N = a.size
    out = np.zeros_like(a)
    for i in range(N):
        e = (i * k) % (2 * N)
        v = int(a[i])
        if e < N:
            out[e] = v
        else:
            out[e - N] = (q - v) % q
    return out


# ------------------------------------------------------------ parameters

@dataclass
class Params:
    """RNS-CKKS parameters.  Q primes are ordered q_0 (output prime) ... q_L,
    then the alpha special primes p_0..p_{alpha-1} (Appendix on FHE parameters:
    moduli ordered q_0..q_L, P)."""
    logn: int
    q: List[int]
    p: List[int]
    alpha: int
    scale: float

    def __post_init__(self):
        self.N = 1 << self.logn
        self.L = len(self.q) - 1
        self.primes = list(self.q) + list(self.p)
        self.psi = [lib().orc_root_2n(t, 2 * self.N) for t in self.primes]
        self.P = 1
        for t in self.p:
            self.P *= t

    def digits(self, level: int) -> List[List[int]]:
        """Active-prime index sets of the key-switching digits at `level`:
        alpha consecutive primes each, the last one truncated."""
        out = []
        for j in range(0, self.L + 1, self.alpha):
            d = [i for i in range(j, min(j + self.alpha, self.L + 1)) if i <= level]
            if d:
                out.append(d)
        return out


def make_params(logn: int, L: int, q_bits: int, q0_bits: int, p_bits: int, alpha: int,
                log_scale: float) -> Params:
    """Prime chain: L primes of q_bits (descending from 2^q_bits) are q_1..q_L,
    then q_0 of q0_bits, then alpha special primes of p_bits, each list skipping
    primes already taken.  All primes are = 1 mod 2N."""
    two_n = 2 << logn
    rest = gen_primes(q_bits, L, two_n) if L > 0 else []
    q0 = gen_primes(q0_bits, 1, two_n, exclude=rest)
    p = gen_primes(p_bits, alpha, two_n, exclude=rest + q0)
    return Params(logn, q0 + rest, p, alpha, float(2.0 ** log_scale))


# ------------------------------------------------------------ containers

@dataclass
class Ciphertext:
    """(c0, c1[, c2]) in the NTT domain: array [n_poly][level+1][N]."""
    c: np.ndarray
    level: int
    scale: float

    def copy(self):
        return Ciphertext(self.c.copy(), self.level, self.scale)


@dataclass
class Plaintext:
    m: np.ndarray   # [level+1][N], NTT domain
    level: int
    scale: float


@dataclass
class SwitchKey:
    """digit j -> array [2][L+1+alpha][N] (b_j, a_j), NTT domain."""
    key_id: int
    digits: List[np.ndarray]


@dataclass
class Keys:
    s_coef: np.ndarray                 # ternary, int64 [N]
    s_ntt: np.ndarray                  # [L+1+alpha][N]
    relin: Optional[SwitchKey] = None
    galois: Dict[int, SwitchKey] = field(default_factory=dict)


# ------------------------------------------------------------ the scheme

class CKKS:
    def __init__(self, prm: Params):
        self.prm = prm

    # -- limb helpers
    def to_ntt(self, limbs: np.ndarray, idx: Sequence[int]) -> np.ndarray:
        prm = self.prm
        return np.stack([ntt(limbs[k], prm.primes[t], prm.psi[t]) for k, t in enumerate(idx)])

    def from_ntt(self, limbs: np.ndarray, idx: Sequence[int]) -> np.ndarray:
        prm = self.prm
        return np.stack([intt(limbs[k], prm.primes[t], prm.psi[t]) for k, t in enumerate(idx)])

    def signed_to_ntt(self, v: np.ndarray, idx: Sequence[int]) -> np.ndarray:
        prm = self.prm
        return np.stack([ntt(from_signed(v, prm.primes[t]), prm.primes[t], prm.psi[t]) for t in idx])

    # -- keys
    def keygen(self, seed: int, rot_steps: Sequence[int] = (), relin: bool = True) -> Keys:
        prm = self.prm
        s = sample_ternary(seed, DOM_SECRET, 0, 0, prm.N)
        all_idx = list(range(len(prm.primes)))
        keys = Keys(s, self.signed_to_ntt(s, all_idx))
        if relin:
            s2 = np.stack([vmul(keys.s_ntt[t], keys.s_ntt[t], prm.primes[t]) for t in all_idx])
            keys.relin = self._switch_key(seed, 0, s2, keys)
        for r in rot_steps:
            k = galois_elt(r, prm.N)
            if k in keys.galois or k == 1:
                continue
            sk = np.stack([automorphism_coeff(from_signed(s, prm.primes[t]), k, prm.primes[t])
                           for t in all_idx])
            sk = self.to_ntt(sk, all_idx)
            keys.galois[k] = self._switch_key(seed, k, sk, keys)
        return keys

    def _switch_key(self, seed: int, key_id: int, s_new: np.ndarray, keys: Keys) -> SwitchKey:
        """For each digit j (top level): (b_j, a_j) with
        b_j = -a_j*s + e_j + P*e_j(CRT idempotent)*s_new  over all primes Q_L, P.
        The idempotent is 1 on digit j's primes and 0 on every other prime, so
        the gadget term is (P mod q_t) * s_new[t] on digit j's limbs only."""
        prm = self.prm
        n_all = len(prm.primes)
        digits = []
        for j, dj in enumerate(prm.digits(prm.L)):
            e = sample_cbd(seed, DOM_KEY_E, key_id, j, prm.N)
            e_ntt = self.signed_to_ntt(e, range(n_all))
            kj = np.empty((2, n_all, prm.N), dtype=np.uint64)
            for t in range(n_all):
                qt = prm.primes[t]
                a = sample_uniform(seed, DOM_KEY_A, key_id, j * 65536 + t, qt, prm.N)
                b = vsub(e_ntt[t], vmul(a, keys.s_ntt[t], qt), qt)
                if t in dj:
                    b = vadd(b, vmul_scalar(s_new[t], prm.P % qt, qt), qt)
                kj[0, t] = b
                kj[1, t] = a
            digits.append(kj)
        return SwitchKey(key_id, digits)

    # -- encode / encrypt / decrypt / decode
    def encode(self, z, scale: float, level: int) -> Plaintext:
        m = encode_coeffs(z, self.prm.logn, scale)
        prm = self.prm
        limbs = np.stack([ntt(from_double(m, prm.primes[t]), prm.primes[t], prm.psi[t])
                          for t in range(level + 1)])
        return Plaintext(limbs, level, float(scale))

    def encrypt(self, keys: Keys, pt: Plaintext, seed: int) -> Ciphertext:
        """c1 = a (uniform), c0 = -a*s + e + m, all at the plaintext's level."""
        prm = self.prm
        lv = pt.level
        e = sample_cbd(seed, DOM_ENC_E, 0, 0, prm.N)
        e_ntt = self.signed_to_ntt(e, range(lv + 1))
        c = np.empty((2, lv + 1, prm.N), dtype=np.uint64)
        for t in range(lv + 1):
            qt = prm.primes[t]
            a = sample_uniform(seed, DOM_ENC_A, 0, t, qt, prm.N)
            c[1, t] = a
            c[0, t] = vadd(vsub(e_ntt[t], vmul(a, keys.s_ntt[t], qt), qt), pt.m[t], qt)
        return Ciphertext(c, lv, pt.scale)

    def decrypt_residues(self, keys: Keys, ct: Ciphertext) -> np.ndarray:
        """m = c0 + c1*s (+ c2*s^2), returned as coefficient-domain residues."""
        prm = self.prm
        m = np.empty((ct.level + 1, prm.N), dtype=np.uint64)
        for t in range(ct.level + 1):
            qt = prm.primes[t]
            acc = ct.c[0, t].copy()
            sp = keys.s_ntt[t]
            for k in range(1, ct.c.shape[0]):
                acc = vadd(acc, vmul(ct.c[k, t], sp, qt), qt)
                sp = vmul(sp, keys.s_ntt[t], qt)
            m[t] = intt(acc, qt, prm.psi[t])
        return m

    def crt(self, residues: np.ndarray) -> List[int]:
        """Exact centred CRT reconstruction to Python integers in (-Q/2, Q/2]."""
        prm = self.prm
        idx = range(residues.shape[0])
        qs = [prm.primes[t] for t in idx]
        Q = 1
        for q in qs:
            Q *= q
        terms = []
        for k, q in enumerate(qs):
            Qk = Q // q
            terms.append((Qk * pow(Qk % q, -1, q)) % Q)
        out = []
        for i in range(residues.shape[1]):
            x = 0
            for k in range(len(qs)):
                x += int(residues[k, i]) * terms[k]
            x %= Q
            if x > Q // 2:
                x -= Q
            out.append(x)
        return out

    def decrypt_decode(self, keys: Keys, ct: Ciphertext) -> np.ndarray:
        res = self.decrypt_residues(keys, ct)
        m = self.crt(res)
        return decode_coeffs([float(x) for x in m], self.prm.logn, ct.scale)

    # -- elementwise homomorphic ops
    def add(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        assert a.level == b.level and a.c.shape == b.c.shape
        prm = self.prm
        c = np.empty_like(a.c)
        for k in range(a.c.shape[0]):
            for t in range(a.level + 1):
                c[k, t] = vadd(a.c[k, t], b.c[k, t], prm.primes[t])
        return Ciphertext(c, a.level, a.scale)

    def mul_plain(self, a: Ciphertext, pt: Plaintext) -> Ciphertext:
        prm = self.prm
        c = np.empty_like(a.c)
        for k in range(a.c.shape[0]):
            for t in range(a.level + 1):
                c[k, t] = vmul(a.c[k, t], pt.m[t], prm.primes[t])
        return Ciphertext(c, a.level, a.scale * pt.scale)

    def mul_const(self, a: Ciphertext, value: int, const_scale: float) -> Ciphertext:
        """Multiply by the integer constant `value` (a constant polynomial)."""
        prm = self.prm
        c = np.empty_like(a.c)
        for k in range(a.c.shape[0]):
            for t in range(a.level + 1):
                c[k, t] = vmul_scalar(a.c[k, t], int(value) % prm.primes[t], prm.primes[t])
        return Ciphertext(c, a.level, a.scale * const_scale)

    def add_plain(self, a: Ciphertext, pt: Plaintext) -> Ciphertext:
        """c0 + m (the plaintext must be at the ciphertext's scale)."""
        prm = self.prm
        c = a.c.copy()
        for t in range(a.level + 1):
            c[0, t] = vadd(a.c[0, t], pt.m[t], prm.primes[t])
        return Ciphertext(c, a.level, a.scale)

    def add_const(self, a: Ciphertext, value: int) -> Ciphertext:
        """Add the integer constant polynomial `value` (its NTT is the constant)."""
        prm = self.prm
        c = a.c.copy()
        for t in range(a.level + 1):
            c[0, t] = vadd_scalar(a.c[0, t], int(value) % prm.primes[t], prm.primes[t])
        return Ciphertext(c, a.level, a.scale)

    def tensor_square(self, a: Ciphertext) -> Ciphertext:
        """(c0, c1)^2 = (c0^2, 2 c0 c1, c1^2)."""
        prm = self.prm
        c = np.empty((3, a.level + 1, prm.N), dtype=np.uint64)
        for t in range(a.level + 1):
            q = prm.primes[t]
            c0, c1 = a.c[0, t], a.c[1, t]
            c[0, t] = vmul(c0, c0, q)
            x = vmul(c0, c1, q)
            c[1, t] = vadd(x, x, q)
            c[2, t] = vmul(c1, c1, q)
        return Ciphertext(c, a.level, a.scale * a.scale)

    def drop_to(self, a: Ciphertext, level: int) -> Ciphertext:
        """Mod-drop: discard the limbs above `level` (scale unchanged)."""
        assert level <= a.level
        return Ciphertext(a.c[:, : level + 1].copy(), level, a.scale)

    # -- key switching
    def ext_primes(self, level: int) -> List[int]:
        """indices of the extended basis Q_level u P"""
        prm = self.prm
        return list(range(level + 1)) + list(range(prm.L + 1, prm.L + 1 + prm.alpha))

    def modup(self, d: np.ndarray, level: int) -> List[np.ndarray]:
        """ModUp of one polynomial (NTT domain, limbs 0..level): for every
        digit j, the digit's residues extended to Q_level u P by the fast
        basis conversion, NTT domain.  Returns [digit][ext limb][N]."""
        prm = self.prm
        Qidx = list(range(level + 1))
        ext = self.ext_primes(level)
        d_coef = self.from_ntt(d, Qidx)
        out = []
        for dj in prm.digits(level):
            qd = [prm.primes[i] for i in dj]
            limbs = np.empty((len(ext), prm.N), dtype=np.uint64)
            for k, t in enumerate(ext):
                qt = prm.primes[t]
                if t in dj:
                    limbs[k] = d[t]
                else:
                    limbs[k] = ntt(basis_convert(d_coef[dj], qd, qt), qt, prm.psi[t])
            out.append(limbs)
        return out

    def galois_ext(self, limbs: np.ndarray, level: int, k: int) -> np.ndarray:
        """sigma_k applied to NTT-domain limbs of the extended basis, through
        the coefficient-domain definition on each limb."""
        prm = self.prm
        ext = self.ext_primes(level)
        out = np.empty_like(limbs)
        for r, t in enumerate(ext):
            qt = prm.primes[t]
            coef = intt(limbs[r], qt, prm.psi[t])
            out[r] = ntt(automorphism_coeff(coef, k, qt), qt, prm.psi[t])
        return out

    def inner_product(self, ext_digits: List[np.ndarray], level: int, key: SwitchKey) -> np.ndarray:
        """sum_j ext_j * key_j over Q_level u P: [2][ext][N]"""
        prm = self.prm
        ext = self.ext_primes(level)
        acc = np.zeros((2, len(ext), prm.N), dtype=np.uint64)
        for j, x in enumerate(ext_digits):
            for k, t in enumerate(ext):
                qt = prm.primes[t]
                for r in range(2):
                    acc[r, k] = vadd(acc[r, k], vmul(x[k], key.digits[j][r, t], qt), qt)
        return acc

    def moddown(self, acc: np.ndarray, level: int) -> np.ndarray:
        """(acc - [acc]_P centred) * P^-1 over Q_level: [2][level+1][N], i.e.
        acc / P rounded to the nearest integer.  [acc]_P + floor(P/2) is
        brought from the special primes to each q_i exactly: the fast
        conversion's overshoot u*P is removed (conv_overflow), then floor(P/2)
        is subtracted, which centres the representative."""
        prm = self.prm
        Qidx = list(range(level + 1))
        Pidx = list(range(prm.L + 1, prm.L + 1 + prm.alpha))
        pq = [prm.primes[t] for t in Pidx]
        half_p = prm.P // 2
        out = np.empty((2, level + 1, prm.N), dtype=np.uint64)
        for r in range(2):
            p_part = self.from_ntt(acc[r, len(Qidx):], Pidx)
            p_part = np.stack([vadd_scalar(p_part[m], half_p % pq[m], pq[m]) for m in range(len(pq))])
            u = conv_overflow(p_part, pq)
            for i in Qidx:
                qi = prm.primes[i]
                conv = basis_convert(p_part, pq, qi)
                conv = vsub(conv, vmul_scalar(u, prm.P % qi, qi), qi)
                conv = vsub(conv, np.full(prm.N, half_p % qi, dtype=np.uint64), qi)
                conv = ntt(conv, qi, prm.psi[i])
                out[r, i] = vmul_scalar(vsub(acc[r, i], conv, qi), invmod(prm.P % qi, qi), qi)
        return out

    def key_switch(self, d: np.ndarray, level: int, key: SwitchKey) -> np.ndarray:
        """Hybrid key switch of one polynomial d (NTT domain, limbs 0..level):
        ModUp, inner product with the key, ModDown.  Returns [2][level+1][N]."""
        return self.moddown(self.inner_product(self.modup(d, level), level, key), level)

    def _galois_key(self, step: int, keys: Keys):
        k = galois_elt(step, self.prm.N)
        if k not in keys.galois:
            raise KeyError("no Galois key for step %d" % step)
        return k, keys.galois[k]

    def rotate_hoisted(self, ct: Ciphertext, steps: Sequence[int], keys: Keys) -> Dict[int, Ciphertext]:
        """Rotations of one ciphertext by several steps sharing one ModUp:
        ModUp(c1) once; for each step, sigma applied to the extended limbs,
        inner product with that step's key, ModDown, plus sigma(c0)."""
        prm = self.prm
        lv = ct.level
        ext = self.modup(ct.c[1], lv)
        out = {}
        for step in steps:
            k, key = self._galois_key(step, keys)
            rot_ext = [self.galois_ext(x, lv, k) for x in ext]
            ks = self.moddown(self.inner_product(rot_ext, lv, key), lv)
            g0 = self.galois_ext(np.concatenate([ct.c[0], np.zeros((prm.alpha, prm.N), dtype=np.uint64)]), lv, k)
            c = np.empty_like(ct.c)
            for t in range(lv + 1):
                c[0, t] = vadd(g0[t], ks[0, t], prm.primes[t])
                c[1, t] = ks[1, t]
            out[step] = Ciphertext(c, lv, ct.scale)
        return out

    # -- double hoisting: rotations left in the extended basis
    def encode_ext(self, z, scale: float, level: int) -> np.ndarray:
        """encode()'s integer polynomial reduced modulo every prime of
        Q_level u P, NTT domain: [ext][N]."""
        m = encode_coeffs(z, self.prm.logn, scale)
        prm = self.prm
        return np.stack([ntt(from_double(m, prm.primes[t]), prm.primes[t], prm.psi[t])
                         for t in self.ext_primes(level)])

    def rotate_hoisted_ext(self, ct: Ciphertext, steps: Sequence[int], keys: Keys) -> Dict[int, np.ndarray]:
        """Rotations of one ciphertext sharing one ModUp, left in Q_l u P:
        for each step the inner product of sigma_k(ModUp(c1)) with that
        step's key, plus P sigma_k(c0) on the Q limbs (P is 0 modulo the
        special primes).  [2][ext][N] per step; its ModDown is exactly the
        rotation of rotate_hoisted, since P sigma_k(c0) divides by P with
        no remainder."""
        prm = self.prm
        lv = ct.level
        ext = self.modup(ct.c[1], lv)
        out = {}
        for step in steps:
            k, key = self._galois_key(step, keys)
            acc = self.inner_product([self.galois_ext(x, lv, k) for x in ext], lv, key)
            g0 = self.galois_ext(np.concatenate([ct.c[0], np.zeros((prm.alpha, prm.N), dtype=np.uint64)]), lv, k)
            for t in range(lv + 1):
                qt = prm.primes[t]
                acc[0, t] = vadd(acc[0, t], vmul_scalar(g0[t], prm.P % qt, qt), qt)
            out[step] = acc
        return out

    def mul_plain_ext(self, pair: np.ndarray, pt_ext: np.ndarray, level: int) -> np.ndarray:
        """[2][ext][N] pair times a plaintext over Q_level u P, limb by limb."""
        prm = self.prm
        out = np.empty_like(pair)
        for r in range(2):
            for k, t in enumerate(self.ext_primes(level)):
                out[r, k] = vmul(pair[r, k], pt_ext[k], prm.primes[t])
        return out

    def add_ext(self, a: np.ndarray, b: np.ndarray, level: int) -> np.ndarray:
        prm = self.prm
        out = np.empty_like(a)
        for r in range(2):
            for k, t in enumerate(self.ext_primes(level)):
                out[r, k] = vadd(a[r, k], b[r, k], prm.primes[t])
        return out

    def rotate_sum_lazy(self, terms: Sequence, keys: Keys, base: Ciphertext) -> Ciphertext:
        """base + sum_g rot(ct_g, g) with one ModDown: each term's ModUp and
        inner product (sigma_g on the extended limbs) are summed over Q_l u P,
        the sigma_g(c0) parts over Q_l, then a single ModDown."""
        prm = self.prm
        lv = base.level
        ext_n = len(self.ext_primes(lv))
        acc = np.zeros((2, ext_n, prm.N), dtype=np.uint64)
        c0 = np.zeros((lv + 1, prm.N), dtype=np.uint64)
        for ct, step in terms:
            k, key = self._galois_key(step, keys)
            rot_ext = [self.galois_ext(x, lv, k) for x in self.modup(ct.c[1], lv)]
            ip = self.inner_product(rot_ext, lv, key)
            ext = self.ext_primes(lv)
            for r in range(2):
                for q in range(ext_n):
                    acc[r, q] = vadd(acc[r, q], ip[r, q], prm.primes[ext[q]])
            g0 = self.galois_ext(np.concatenate([ct.c[0], np.zeros((prm.alpha, prm.N), dtype=np.uint64)]), lv, k)
            for t in range(lv + 1):
                c0[t] = vadd(c0[t], g0[t], prm.primes[t])
        ks = self.moddown(acc, lv)
        c = np.empty_like(base.c)
        for t in range(lv + 1):
            qt = prm.primes[t]
            c[0, t] = vadd(vadd(base.c[0, t], c0[t], qt), ks[0, t], qt)
            c[1, t] = vadd(base.c[1, t], ks[1, t], qt)
        return Ciphertext(c, lv, base.scale)

    def relinearize(self, ct: Ciphertext, keys: Keys) -> Ciphertext:
        assert ct.c.shape[0] == 3
        prm = self.prm
        ks = self.key_switch(ct.c[2], ct.level, keys.relin)
        c = np.empty((2, ct.level + 1, prm.N), dtype=np.uint64)
        for r in range(2):
            for t in range(ct.level + 1):
                c[r, t] = vadd(ct.c[r, t], ks[r, t], prm.primes[t])
        return Ciphertext(c, ct.level, ct.scale)

    def apply_galois(self, ct: Ciphertext, k: int) -> np.ndarray:
        """sigma_k applied to every polynomial, through the coefficient domain."""
        prm = self.prm
        idx = list(range(ct.level + 1))
        out = np.empty_like(ct.c)
        for r in range(ct.c.shape[0]):
            coef = self.from_ntt(ct.c[r], idx)
            coef = np.stack([automorphism_coeff(coef[t], k, prm.primes[t]) for t in idx])
            out[r] = self.to_ntt(coef, idx)
        return out

    def rotate(self, ct: Ciphertext, step: int, keys: Keys) -> Ciphertext:
        """Slots move left by `step`: sigma_{5^step} then switch sigma(s) -> s."""
        prm = self.prm
        k = galois_elt(step, prm.N)
        if k == 1:
            return ct.copy()
        if k not in keys.galois:
            raise KeyError("no Galois key for step %d" % step)
        g = self.apply_galois(ct, k)
        ks = self.key_switch(g[1], ct.level, keys.galois[k])
        c = np.empty_like(ct.c)
        for t in range(ct.level + 1):
            c[0, t] = vadd(g[0, t], ks[0, t], prm.primes[t])
            c[1, t] = ks[1, t]
        return Ciphertext(c, ct.level, ct.scale)

    def rescale(self, ct: Ciphertext) -> Ciphertext:
        """c_i <- q_l^-1 (c_i - [c_l]_centred) mod q_i; scale / q_l; level - 1."""
        prm = self.prm
        lv = ct.level
        assert lv >= 1
        ql = prm.primes[lv]
        out = np.empty((ct.c.shape[0], lv, prm.N), dtype=np.uint64)
        for r in range(ct.c.shape[0]):
            top = intt(ct.c[r, lv], ql, prm.psi[lv]).astype(np.int64)
            # centred representative in (-q_l/2, q_l/2]
            top = np.where(top > (ql - 1) // 2, top - np.int64(ql), top)
            for i in range(lv):
                qi = prm.primes[i]
                t = ntt(from_signed(top, qi), qi, prm.psi[i])
                out[r, i] = vmul_scalar(vsub(ct.c[r, i], t, qi), invmod(ql % qi, qi), qi)
        return Ciphertext(out, lv - 1, ct.scale / ql)
