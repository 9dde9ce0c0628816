"""Pins of the CPU oracle against values and identities fixed outside it.

Each test checks the oracle against something other than itself: numbers the
paper prints (tests/golden/), brute-force definitions on tiny inputs, exact
big-integer arithmetic, an independent library (sympy, cryptography), or
algebraic identities of the scheme.
"""
import math
import os

import numpy as np
import pytest

import paper_chains
from oracle import ckks as C
from oracle import planner

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ primes

def _paper_chains():
    return paper_chains.rows()


def test_paper_prime_chains_are_ntt_primes():
    """Every modulus printed in the appendix is prime, = 1 mod 2N, and the
    chain sizes add up to Table 4's log2 Q and log2 P."""
    rows = _paper_chains()
    assert [r[0] for r in rows] == ["VGG-16", "ResNet-18", "ResNet-20", "ResNet-32"]
    for name, logn, d, L, lq, lp, qs, p in rows:
        assert len(qs) == L + 1, name
        for q in qs + [p]:
            assert C.is_prime(q), (name, hex(q))
            assert (q - 1) % (2 << logn) == 0, (name, hex(q))
        assert round(sum(math.log2(q) for q in qs)) == lq, name
        assert round(math.log2(p)) == lp, name


def test_is_prime_matches_sympy():
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(5)
    cands = [int(x) | 1 for x in rng.integers(2 ** 40, 2 ** 62, 300, dtype=np.int64)]
    cands += [2 ** 61 - 1, 3215031751, 341550071728321, 3825123056546413051]
    for n in cands:
        assert C.is_prime(n) == sympy.isprime(n), n


def test_prime_generator_descending_ntt_primes():
    two_n = 2 << 13
    ps = C.gen_primes(40, 6, two_n)
    assert ps == sorted(ps, reverse=True)
    for p in ps:
        assert C.is_prime(p) and p < 2 ** 40 and (p - 1) % two_n == 0
    # nothing skipped: no prime = 1 mod 2N lies between consecutive outputs
    sympy = pytest.importorskip("sympy")
    for hi, lo in zip([2 ** 40 + 1] + ps[:-1], ps):
        for c in range(lo + two_n, hi, two_n):
            assert not sympy.isprime(c)


def test_root_has_order_2n():
    for logn in (4, 10, 16):
        two_n = 2 << logn
        q = C.gen_primes(50, 1, two_n)[0]
        psi = C.lib().orc_root_2n(q, two_n)
        assert pow(psi, two_n // 2, q) == q - 1
        assert pow(psi, two_n, q) == 1


# ------------------------------------------------------------------ NTT

@pytest.mark.parametrize("logn", [1, 2, 4, 7, 10])
def test_ntt_is_evaluation_at_odd_roots(logn):
    """NTT(a)[j] = a(psi^(2 brv(j) + 1)): checked by brute force with Python
    integers, not through the C routine's own naive form only."""
    N = 1 << logn
    q = C.gen_primes(45, 1, 2 * N)[0]
    psi = C.lib().orc_root_2n(q, 2 * N)
    a = np.random.default_rng(logn).integers(0, q, N, dtype=np.uint64)
    got = C.ntt(a, q, psi)
    assert np.array_equal(got, C.ntt_naive(a, q, psi))
    if logn <= 7:
        for j in range(N):
            brv = int(format(j, "0%db" % logn)[::-1], 2) if logn else 0
            x = pow(psi, 2 * brv + 1, q)
            assert int(got[j]) == sum(int(a[i]) * pow(x, i, q) for i in range(N)) % q


@pytest.mark.parametrize("logn", [3, 6, 10])
def test_ntt_product_is_negacyclic_convolution(logn):
    N = 1 << logn
    q = C.gen_primes(50, 1, 2 * N)[0]
    psi = C.lib().orc_root_2n(q, 2 * N)
    rng = np.random.default_rng(10 + logn)
    a = rng.integers(0, q, N, dtype=np.uint64)
    b = rng.integers(0, q, N, dtype=np.uint64)
    prod = C.intt(C.vmul(C.ntt(a, q, psi), C.ntt(b, q, psi), q), q, psi)
    assert np.array_equal(prod, C.negacyclic_naive(a, b, q))
    # schoolbook with Python ints, independent of the C routine
    if logn <= 6:
        ref = [0] * N
        for i in range(N):
            for j in range(N):
                k = i + j
                s = -1 if k >= N else 1
                ref[k % N] = (ref[k % N] + s * int(a[i]) * int(b[j])) % q
        assert [int(x) for x in prod] == ref


def test_intt_inverts_ntt_at_full_size():
    N = 1 << 16
    q = C.gen_primes(60, 1, 2 * N)[0]
    psi = C.lib().orc_root_2n(q, 2 * N)
    a = np.random.default_rng(3).integers(0, q, N, dtype=np.uint64)
    assert np.array_equal(C.intt(C.ntt(a, q, psi), q, psi), a)


# ------------------------------------------------------------------ sampling

def test_chacha20_block_matches_cryptography_library():
    """The stream's block function equals RFC 8439 ChaCha20 as implemented by
    the `cryptography` package (keystream = encryption of zeros)."""
    crypto = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    algos = pytest.importorskip("cryptography.hazmat.primitives.ciphers.algorithms")
    rng = np.random.default_rng(9)
    for _ in range(4):
        key = rng.integers(0, 2 ** 32, 8, dtype=np.uint64).astype(np.uint32)
        nonce = rng.integers(0, 2 ** 32, 3, dtype=np.uint64).astype(np.uint32)
        counter = int(rng.integers(0, 2 ** 31))
        ours = C.chacha20_block(key, counter, nonce).tobytes()
        full_nonce = np.array([counter], dtype="<u4").tobytes() + nonce.astype("<u4").tobytes()
        cipher = crypto.Cipher(algos.ChaCha20(key.astype("<u4").tobytes(), full_nonce), mode=None)
        assert ours == cipher.encryptor().update(b"\0" * 64)


def test_stream_words_are_consecutive_blocks():
    w = C.stream_words(0x1234567890ABCDEF, 3, 5, 6, 40)
    key = [0x90ABCDEF, 0x12345678, 3, 0, 0, 0, 0, 0]
    for b in range(3):
        blk = C.chacha20_block(key, b, [5, 6, 0])
        n = min(16, 40 - 16 * b)
        assert np.array_equal(w[16 * b:16 * b + n], blk[:n])


def test_samplers_follow_their_definitions_and_moments():
    seed = 77
    n = 1 << 15
    w = C.stream_words(seed, 9, 1, 2, 4 * n)
    q = C.gen_primes(50, 1, 2 << 14)[0]
    u = C.sample_uniform(seed, 9, 1, 2, q, n)
    for k in range(0, n, 997):
        v = sum(int(w[4 * k + i]) << (32 * i) for i in range(4))
        assert int(u[k]) == v % q
    assert abs(u.astype(np.float64).mean() / q - 0.5) < 0.01
    t = C.sample_ternary(seed, 9, 1, 2, n)
    assert set(np.unique(t)) <= {-1, 0, 1}
    for k in range(0, n, 991):
        assert t[k] == (int(w[k]) * 3 >> 32) - 1
    assert np.all(np.abs(np.bincount(t + 1) / n - 1 / 3) < 0.01)
    e = C.sample_cbd(seed, 9, 1, 2, n)
    for k in range(0, n, 983):
        a = bin(int(w[2 * k]) & 0x1FFFFF).count("1")
        b = bin(int(w[2 * k + 1]) & 0x1FFFFF).count("1")
        assert e[k] == a - b
    assert abs(e.mean()) < 0.1 and abs(e.var() - 10.5) < 0.4 and np.abs(e).max() <= 21


# ------------------------------------------------------------------ encoding

@pytest.mark.parametrize("logn", [2, 4, 7, 9])
def test_encode_matches_definition(logn):
    N = 1 << logn
    rng = np.random.default_rng(logn)
    z = rng.uniform(-1, 1, N // 2) + 1j * rng.uniform(-1, 1, N // 2)
    scale = 2.0 ** 30
    m = C.encode_coeffs(z, logn, scale)
    ref = C.encode_naive(z, logn, scale)
    assert np.max(np.abs(m - ref)) <= 0.5 + 1e-6
    # and the definition itself, written with numpy: m(zeta^(5^j)) = scale*z_j
    zeta = np.exp(1j * np.pi / N)
    e = [pow(5, j, 2 * N) for j in range(N // 2)]
    vals = np.array([np.sum(ref * zeta ** (np.arange(N) * ej % (2 * N))) for ej in e])
    assert np.max(np.abs(vals / scale - z)) < 1e-9


def test_encode_constant_is_constant_polynomial():
    """A constant slot vector w encodes exactly to the constant round(Delta*w)."""
    for logn in (4, 13):
        N = 1 << logn
        for w in (0.3, -1.25, 7.0):
            m = C.encode_coeffs(np.full(N // 2, w), logn, 2.0 ** 40)
            assert m[0] == round(w * 2 ** 40)
            assert np.all(m[1:] == 0)


def test_decode_inverts_encode_and_big_scales():
    logn = 13
    N = 1 << logn
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, N // 2)
    for scale in (2.0 ** 25, 2.0 ** 40, 2.0 ** 80):
        m = C.encode_coeffs(z, logn, scale)
        back = C.decode_coeffs(m, logn, scale)
        assert np.max(np.abs(back - z)) < max(1e-12, N / scale)
        # residues of big integral doubles are exact
        q = C.gen_primes(50, 1, 2 * N)[0]
        r = C.from_double(m[:64], q)
        assert [int(x) for x in r] == [int(v) % q for v in m[:64]]


def test_galois_automorphism_rotates_slots():
    """sigma_{5^r}(m) decodes to the slots rotated left by r (canonical
    embedding identity), checked on the coefficient-domain definition."""
    logn = 6
    N = 1 << logn
    q = C.gen_primes(55, 1, 2 * N)[0]
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, N // 2) + 1j * rng.uniform(-1, 1, N // 2)
    scale = 2.0 ** 40
    m = C.encode_coeffs(z, logn, scale)
    res = C.from_double(m, q)
    for r in (1, 3, -1, 17):
        k = C.galois_elt(r, N)
        rot = C.automorphism_coeff(res, k, q).astype(np.int64)
        rot = np.where(rot > q // 2, rot - np.int64(q), rot)
        back = C.decode_coeffs(rot.astype(np.float64), logn, scale)
        assert np.max(np.abs(back - np.roll(z, -r))) < 1e-9


def test_galois_map_in_the_ntt_domain_keeps_aligned_pairs():
    """The NTT-domain form of sigma_k, derived here from the coefficient
    definition (NTT of a(x^k) against NTT of a), is a permutation of slots
    that (1) sends every aligned pair of slots onto an aligned pair and (2)
    is inverted by the map of k^-1 mod 2N.  The key-switching kernels rely on
    both: a gather reads two slots with one 16-byte load, and the batched
    baby-step inner product scatters to the pair that the inverse map
    gives."""
    logn = 8
    N = 1 << logn
    prm = C.make_params(logn=logn, L=1, q_bits=50, q0_bits=50, p_bits=50, alpha=1, log_scale=20)
    q, psi = prm.primes[0], prm.psi[0]
    a = np.random.default_rng(5).integers(0, q, N, dtype=np.uint64)
    base = C.ntt(a, q, psi)
    where = {int(v): i for i, v in enumerate(base)}
    assert len(where) == N                       # distinct values: positions identify slots

    def slot_map(k):
        # out[j] = in[src[j]] for the NTT of a(x^k)
        img = C.ntt(C.automorphism_coeff(a, k, q), q, psi)
        return np.array([where[int(v)] for v in img])

    for r in (1, 3, -1, 17, N // 4 - 1):
        k = C.galois_elt(r, N)
        src = slot_map(k)
        assert sorted(src) == list(range(N))
        for j in range(0, N, 2):
            assert src[j] ^ 1 == src[j + 1]
        kinv = pow(k, -1, 2 * N)
        inv = slot_map(kinv)
        assert all(src[inv[i]] == i for i in range(N))


# ------------------------------------------------------------------ RNS

def test_basis_conversion_is_crt_plus_small_multiple():
    rng = np.random.default_rng(4)
    qs = C.gen_primes(50, 3, 2 << 10)
    t = C.gen_primes(60, 1, 2 << 10)[0]
    Q = qs[0] * qs[1] * qs[2]
    xs = [int(v) for v in rng.integers(0, 2 ** 62, 64, dtype=np.int64)]
    xs = [(x * 12345678910111) % Q for x in xs]
    limbs = np.array([[x % q for x in xs] for q in qs], dtype=np.uint64)
    got = C.basis_convert(limbs, qs, t)
    for x, g in zip(xs, got):
        assert any((x + u * Q) % t == int(g) for u in range(3))


def test_crt_reconstruction_exact():
    prm = C.make_params(logn=4, L=3, q_bits=50, q0_bits=45, p_bits=55, alpha=2, log_scale=30)
    S = C.CKKS(prm)
    Q = 1
    for q in prm.q:
        Q *= q
    rng = np.random.default_rng(6)
    vals = [int(v) * int(w) - Q // 3 for v, w in zip(rng.integers(0, 2 ** 62, 16, dtype=np.int64),
                                                    rng.integers(0, 2 ** 62, 16, dtype=np.int64))]
    res = np.array([[v % q for v in vals] for q in prm.q], dtype=np.uint64)
    assert S.crt(res) == vals


# ------------------------------------------------------------------ scheme

@pytest.fixture(scope="module")
def small():
    prm = C.make_params(logn=5, L=3, q_bits=40, q0_bits=45, p_bits=50, alpha=2, log_scale=30)
    S = C.CKKS(prm)
    keys = S.keygen(11, [1, -1, 3, 5])
    return prm, S, keys


def test_decrypt_encrypt_is_m_plus_e_exactly(small):
    prm, S, keys = small
    z = np.random.default_rng(0).uniform(-1, 1, prm.N // 2)
    pt = S.encode(z, prm.scale, prm.L)
    ct = S.encrypt(keys, pt, 7)
    dec = S.crt(S.decrypt_residues(keys, ct))
    m = C.encode_coeffs(z, prm.logn, prm.scale)
    e = C.sample_cbd(7, C.DOM_ENC_E, 0, 0, prm.N)
    assert [int(x) for x in dec] == [int(a) + int(b) for a, b in zip(m, e)]


def test_keyswitch_relin_rotate_noise_bounded(small):
    prm, S, keys = small
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, prm.N // 2) + 1j * rng.uniform(-1, 1, prm.N // 2)
    ct = S.encrypt(keys, S.encode(z, prm.scale, prm.L), 8)
    for r in (1, 3, -1, 5):
        out = S.rotate(ct, r, keys)
        assert np.max(np.abs(S.decrypt_decode(keys, out) - np.roll(z, -r))) < 1e-6
    back = S.rotate(S.rotate(ct, 1, keys), -1, keys)
    assert np.max(np.abs(S.decrypt_decode(keys, back) - z)) < 1e-6
    sq = S.relinearize(S.tensor_square(ct), keys)
    assert np.max(np.abs(S.decrypt_decode(keys, sq) - z * z)) < 1e-6
    # the tensor before relinearisation decrypts with s^2 as well
    t3 = S.tensor_square(ct)
    assert np.max(np.abs(S.decrypt_decode(keys, t3) - z * z)) < 1e-6


def test_keyswitch_output_is_d_times_sprime_over_p(small):
    """KS(d) decrypts to d*s' plus noise far below the modulus: compare the
    integer polynomial c0 + c1*s against d*s' computed with Python ints."""
    prm, S, keys = small
    lv = prm.L
    rng = np.random.default_rng(3)
    d = np.stack([rng.integers(0, prm.q[t], prm.N, dtype=np.uint64) for t in range(lv + 1)])
    ks = S.key_switch(d, lv, keys.relin)
    ct = C.Ciphertext(ks, lv, 1.0)
    got = S.crt(S.decrypt_residues(keys, ct))
    s2 = np.stack([C.vmul(keys.s_ntt[t], keys.s_ntt[t], prm.q[t]) for t in range(lv + 1)])
    want = S.crt(np.stack([C.intt(C.vmul(d[t], s2[t], prm.q[t]), prm.q[t], prm.psi[t])
                           for t in range(lv + 1)]))
    Q = 1
    for q in prm.q:
        Q *= q
    diffs = [((g - w + Q // 2) % Q) - Q // 2 for g, w in zip(got, want)]
    assert max(abs(x) for x in diffs) < 2 ** 20


def test_rescale_is_rounded_division(small):
    """rescale(c) equals round(c / q_l) computed with big integers
    (coefficient domain, centred representatives)."""
    prm, S, keys = small
    rng = np.random.default_rng(4)
    lv = prm.L
    c = np.stack([np.stack([rng.integers(0, prm.q[t], prm.N, dtype=np.uint64) for t in range(lv + 1)])
                  for _ in range(2)])
    ct = C.Ciphertext(c, lv, 2.0 ** 60)
    out = S.rescale(ct)
    Ql = 1
    for q in prm.q[:lv]:
        Ql *= q
    ql = prm.q[lv]
    for r in range(2):
        big = S.crt(np.stack([C.intt(c[r, t], prm.q[t], prm.psi[t]) for t in range(lv + 1)]))
        res = S.crt(np.stack([C.intt(out.c[r, t], prm.q[t], prm.psi[t]) for t in range(lv)]))
        for x, y in zip(big, res):
            rounded = (2 * x + ql) // (2 * ql)          # floor(x/q + 1/2)
            assert (y - rounded) % Ql == 0
    assert out.level == lv - 1 and out.scale == 2.0 ** 60 / ql


def test_moddown_is_rounded_division_by_p():
    """ModDown(acc) equals round(acc / P) for every coefficient, with acc taken
    as its centred integer in (-PQ/2, PQ/2] (big integers; three special primes
    so that the fast conversion from P overshoots by up to 2P)."""
    prm = C.make_params(logn=5, L=2, q_bits=40, q0_bits=45, p_bits=50, alpha=3, log_scale=30)
    S = C.CKKS(prm)
    lv = prm.L
    ext = S.ext_primes(lv)
    rng = np.random.default_rng(9)
    acc_coef = np.stack([np.stack([rng.integers(0, prm.primes[t], prm.N, dtype=np.uint64) for t in ext])
                         for _ in range(2)])
    acc = np.stack([np.stack([C.ntt(acc_coef[r, k], prm.primes[t], prm.psi[t]) for k, t in enumerate(ext)])
                    for r in range(2)])
    out = S.moddown(acc, lv)
    PQ = prm.P
    Q = 1
    for q in prm.q[:lv + 1]:
        Q *= q
        PQ *= q
    terms = []
    for k, t in enumerate(ext):
        pt = prm.primes[t]
        Mk = PQ // pt
        terms.append((Mk * pow(Mk % pt, -1, pt)) % PQ)
    for r in range(2):
        got = S.crt(np.stack([C.intt(out[r, t], prm.q[t], prm.psi[t]) for t in range(lv + 1)]))
        for c in range(prm.N):
            x = sum(int(acc_coef[r, k, c]) * terms[k] for k in range(len(ext))) % PQ
            if x > PQ // 2:
                x -= PQ
            rounded = (2 * x + prm.P) // (2 * prm.P)        # floor(x/P + 1/2)
            assert (got[c] - rounded) % Q == 0


def test_conv_overflow_counts_the_overshoot():
    """basis_convert(x) - conv_overflow(x)*Qin reproduces x exactly (CRT)."""
    qs = C.gen_primes(50, 4, 1 << 13)
    rng = np.random.default_rng(10)
    Qin = 1
    for q in qs:
        Qin *= q
    xs = [int(a) * int(b) % Qin for a, b in zip(rng.integers(1, 2 ** 62, 64, dtype=np.int64),
                                                 rng.integers(1, 2 ** 62, 64, dtype=np.int64))]
    res = np.array([[x % q for x in xs] for q in qs], dtype=np.uint64)
    u = C.conv_overflow(res, qs)
    assert u.max() < len(qs)
    t = C.gen_primes(58, 1, 1 << 13)[0]
    conv = C.basis_convert(res, qs, t)
    for k, x in enumerate(xs):
        assert (int(conv[k]) - int(u[k]) * Qin) % t == x % t


def test_rotation_error_not_concentrated_in_one_slot():
    """After an exact ModDown the key-switching error has no constant bias:
    the decoded error of a rotation at slot 0 (where a per-coefficient bias
    times s would concentrate) is of the size of the other slots'."""
    prm = C.make_params(logn=12, L=3, q_bits=50, q0_bits=40, p_bits=58, alpha=3, log_scale=25)
    S = C.CKKS(prm)
    keys = S.keygen(11, [1])
    z = np.random.default_rng(0).uniform(-0.01, 0.01, prm.N // 2)
    ct = S.encrypt(keys, S.encode(z, 2.0 ** 25, prm.L), 5)
    e = S.decrypt_decode(keys, S.rotate(ct, 1, keys)).real - np.roll(z, -1)
    assert abs(e[0]) < 2 * np.abs(e[1:]).max()
    assert np.abs(e).max() < 1e-3


# ------------------------------------------------------------------ planner

def test_table1_levels():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_levels.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[f[0]] = [int(x) for x in f[1:]]
    assert set(rows) == set(planner.PROFILES)
    for model, want in rows.items():
        got = [planner.table1_levels(**planner.PROFILES[model], variant=v) for v in planner.VARIANTS]
        assert got == want, model


def test_tower_reuse_worked_example():
    """Sec. 4.3 example: lambda(x)=1, q ~ Delta^2; activation -> 2 (no
    rescale); convolution with lambda(omega)=1 -> 3 > 2 -> rescale -> 1."""
    n, trace = planner.tower_reuse([("square", 0), ("mul", 1)], lam_q=2, lam_in=1)
    assert trace == [2, 1] and n == 1


def test_tower_reuse_count_matches_table1_last_column():
    """The rule applied along each model's longest path reproduces P2FRT."""
    want = {"VGG-16": 16, "ResNet-18": 18, "ResNet-20": 20, "ResNet-32": 32}
    n_lin = {"VGG-16": 16, "ResNet-18": 18, "ResNet-20": 20, "ResNet-32": 32}
    n_act = {"VGG-16": 15, "ResNet-18": 17, "ResNet-20": 19, "ResNet-32": 31}
    for m in want:
        n, _ = planner.tower_reuse(planner.alternating_path(n_lin[m], n_act[m]), lam_q=2)
        assert n == want[m], m


def test_hoisted_rotations_decrypt_to_rotated_slots(small):
    """Rotations sharing one ModUp decrypt to the rotated slots (the
    extended-basis automorphism of ModUp(c1) is a valid key-switch input)."""
    prm, S, keys = small
    rng = np.random.default_rng(11)
    z = rng.uniform(-1, 1, prm.N // 2) + 1j * rng.uniform(-1, 1, prm.N // 2)
    ct = S.encrypt(keys, S.encode(z, prm.scale, prm.L), 12)
    rots = S.rotate_hoisted(ct, [1, 3, -1], keys)
    for step, r in rots.items():
        assert np.max(np.abs(S.decrypt_decode(keys, r) - np.roll(z, -step))) < 1e-6
    # one step alone: same plaintext as the plain rotation, different noise
    plain = S.rotate(ct, 3, keys)
    d1 = S.decrypt_decode(keys, rots[3])
    d2 = S.decrypt_decode(keys, plain)
    assert np.max(np.abs(d1 - d2)) < 1e-6


def test_extended_basis_rotations_moddown_to_the_hoisted_ones(small):
    """Double hoisting: a rotation kept in Q_l u P (inner product plus
    P sigma(c0)) brought down by ModDown is bit for bit the single-hoisted
    rotation, since P sigma(c0) is divided by P exactly; its special-prime
    limbs hold only the inner product (P is 0 modulo each special prime)."""
    prm, S, keys = small
    rng = np.random.default_rng(13)
    z = rng.uniform(-1, 1, prm.N // 2)
    ct = S.encrypt(keys, S.encode(z, prm.scale, prm.L), 14)
    steps = [1, 3, -1]
    ext = S.rotate_hoisted_ext(ct, steps, keys)
    single = S.rotate_hoisted(ct, steps, keys)
    lv = ct.level
    xd = S.modup(ct.c[1], lv)
    for step in steps:
        assert np.array_equal(S.moddown(ext[step], lv), single[step].c)
        k, key = S._galois_key(step, keys)
        ip = S.inner_product([S.galois_ext(x, lv, k) for x in xd], lv, key)
        assert np.array_equal(ext[step][:, lv + 1:], ip[:, lv + 1:])
        assert np.array_equal(ext[step][1], ip[1])


def test_double_hoisted_sum_of_products_decrypts_to_the_sum(small):
    """sum_b pt_b (.) rot_b(ct) formed in Q_l u P with plaintexts encoded over
    Q_l u P, then one ModDown: decrypts to sum_b w_b * rotate(z, b), and
    differs from the single-hoisted sum only by rounding (a few units of
    the ciphertext modulus' last place after decoding)."""
    prm, S, keys = small
    rng = np.random.default_rng(14)
    z = rng.uniform(-1, 1, prm.N // 2)
    ws = {b: rng.uniform(-1, 1, prm.N // 2) for b in (1, 3, 5)}
    ct = S.encrypt(keys, S.encode(z, prm.scale, prm.L), 15)
    lv = ct.level
    ext = S.rotate_hoisted_ext(ct, list(ws), keys)
    acc = None
    for b, w in ws.items():
        term = S.mul_plain_ext(ext[b], S.encode_ext(w, prm.scale, lv), lv)
        acc = term if acc is None else S.add_ext(acc, term, lv)
    dh = C.Ciphertext(S.moddown(acc, lv), lv, prm.scale * prm.scale)
    want = sum(w * np.roll(z, -b) for b, w in ws.items())
    assert np.max(np.abs(S.decrypt_decode(keys, dh).real - want)) < 1e-6
    single = S.rotate_hoisted(ct, list(ws), keys)
    sacc = None
    for b, w in ws.items():
        term = S.mul_plain(single[b], S.encode(w, prm.scale, lv))
        sacc = term if sacc is None else S.add(sacc, term)
    assert np.max(np.abs(S.decrypt_decode(keys, dh) - S.decrypt_decode(keys, sacc))) < 1e-6
    # the Q limbs of an extended-basis plaintext are the ordinary plaintext
    assert np.array_equal(S.encode_ext(z, prm.scale, lv)[: lv + 1], S.encode(z, prm.scale, lv).m)


def test_lazy_rotation_sum_decrypts_to_the_sum(small):
    """base + sum_g rot(ct_g, g) with a single ModDown decrypts to the sum."""
    prm, S, keys = small
    rng = np.random.default_rng(12)
    zs = [rng.uniform(-1, 1, prm.N // 2) for _ in range(3)]
    cts = [S.encrypt(keys, S.encode(z, prm.scale, prm.L), 20 + i) for i, z in enumerate(zs)]
    out = S.rotate_sum_lazy([(cts[1], 1), (cts[2], 5)], keys, cts[0])
    want = zs[0] + np.roll(zs[1], -1) + np.roll(zs[2], -5)
    assert np.max(np.abs(S.decrypt_decode(keys, out).real - want)) < 1e-6


def test_oracle_with_the_paper_resnet32_chain():
    """The paper's ResNet-32 chain (q_0 of 28 bits, 32 primes of ~52 bits, one
    54-bit special prime, so one prime per digit: 33 digits at the top) at
    N = 2^10: the key switch of a uniform d is d*s^2 plus noise of a fresh
    error's size; a rotation decrypts to the rotated slots; a rescale from
    Delta^3 leaves Delta and the values."""
    logn, d, q, p = paper_chains.chain("ResNet-32")
    prm = C.Params(10, q, p, 1, 2.0 ** d)
    assert len(prm.digits(prm.L)) == 33 and q[0].bit_length() == 28
    S = C.CKKS(prm)
    keys = S.keygen(11, [1])
    lv = prm.L
    rng = np.random.default_rng(3)
    dd = np.stack([rng.integers(0, prm.q[t], prm.N, dtype=np.uint64) for t in range(lv + 1)])
    got = S.crt(S.decrypt_residues(keys, C.Ciphertext(S.key_switch(dd, lv, keys.relin), lv, 1.0)))
    s2 = np.stack([C.vmul(keys.s_ntt[t], keys.s_ntt[t], prm.q[t]) for t in range(lv + 1)])
    want = S.crt(np.stack([C.intt(C.vmul(dd[t], s2[t], prm.q[t]), prm.q[t], prm.psi[t]) for t in range(lv + 1)]))
    Q = math.prod(prm.q)
    assert max(abs(((g - w + Q // 2) % Q) - Q // 2) for g, w in zip(got, want)) < 2 ** 20
    z = rng.uniform(-1, 1, prm.N // 2)
    ct = S.encrypt(keys, S.encode(z, 2.0 ** (3 * d), lv), 8)
    assert np.max(np.abs(S.decrypt_decode(keys, S.rotate(ct, 1, keys)) - np.roll(z, -1))) < 1e-6
    r = S.rescale(ct)
    assert r.level == lv - 1 and abs(math.log2(r.scale) - d) < 0.01
    # the rescale's rounding (1/2 per coefficient, times s) decodes to about
    # sqrt(N) * 13 / Delta ~ 1e-5 in the slots at Delta = 2^26, N = 2^10
    assert np.max(np.abs(S.decrypt_decode(keys, r) - z)) < 1e-4


def test_rotation_steps_repeat_with_period_half_n(small):
    """5 has multiplicative order exactly N/2 modulo 2N (the slot rotations
    form a cyclic group of order N/2), so rotations by r and r + N/2 are one
    automorphism and a rotation by N/2 leaves the slots unchanged."""
    prm, S, keys = small
    for logn in (5, 10, 12, 16):
        N = 1 << logn
        assert pow(5, N // 2, 2 * N) == 1 and pow(5, N // 4, 2 * N) != 1
    N = prm.N
    z = np.random.default_rng(11).uniform(-1, 1, N // 2)
    ct = S.encrypt(keys, S.encode(z, prm.scale, prm.L), 12)
    assert np.array_equal(S.rotate(ct, 1 + N // 2, keys).c, S.rotate(ct, 1, keys).c)
    assert np.array_equal(S.rotate(ct, N // 2, keys).c, ct.c)
    assert np.max(np.abs(S.decrypt_decode(keys, S.rotate(ct, -N // 2, keys)) - z)) < 1e-6


def test_degenerate_inputs(small):
    """An empty slot vector encodes to the zero plaintext; a ciphertext on
    q_0 alone still decrypts; there is no rescale below level 0."""
    prm, S, keys = small
    assert not S.encode(np.zeros(0), prm.scale, prm.L).m.any()
    z = np.random.default_rng(12).uniform(-1, 1, prm.N // 2)
    ct0 = S.encrypt(keys, S.encode(z, prm.scale, 0), 13)
    assert ct0.level == 0 and np.max(np.abs(S.decrypt_decode(keys, ct0) - z)) < 1e-6
    with pytest.raises(AssertionError):
        S.rescale(ct0)
