"""GPU parity of the CKKS primitives: every ciphertext limb computed by the
CUDA library through the C ABI equals the oracle's, bit for bit, on the same
seeded randomness."""
import numpy as np
import pytest

from oracle import ckks as O

pytestmark = pytest.mark.gpu

# small ring, several digits and a ragged last digit (L+1 = 5 primes, alpha 2)
SMALL = dict(logn=12, L=4, q_bits=45, q0_bits=50, p_bits=55, alpha=2, log_scale=35)
# the ring of the tiny network (one prime per digit)
TINY = dict(logn=13, L=4, q_bits=40, q0_bits=40, p_bits=40, alpha=1, log_scale=40)
# prime widths of the ResNet-20 chain (40-bit q0, 50-bit q_i, 58-bit p_j):
# basis conversions between primes of different widths
WIDE = dict(logn=12, L=6, q_bits=50, q0_bits=40, p_bits=58, alpha=3, log_scale=25)
# the ResNet-20 chain and digits (21 Q primes, dnum = 3 digits of 7 primes,
# 7 special primes) on a small ring; lower levels have a ragged last digit
DNUM3 = dict(logn=12, L=20, q_bits=50, q0_bits=40, p_bits=58, alpha=7, log_scale=25)
CFGS = {"small": SMALL, "tiny": TINY, "wide": WIDE, "dnum3": DNUM3}


@pytest.fixture(scope="module", params=list(CFGS))
def pair(request):
    from paper_2509_22857_gb300 import _lib as F
    cfg = CFGS[request.param]
    prm = O.make_params(**cfg)
    ctx = F.fhe_ctx_create(cfg["logn"], cfg["L"], cfg["q_bits"], cfg["q0_bits"], cfg["p_bits"],
                           cfg["alpha"], cfg["log_scale"])
    S = O.CKKS(prm)
    steps = [1, -1, 5, 300, 1000]
    keys = S.keygen(11, steps)
    sk, evk = F.fhe_keygen(ctx, 11, steps)
    yield F, ctx, prm, S, keys, sk, evk
    F.fhe_evk_free(evk)
    F.fhe_sk_free(sk)
    F.fhe_ctx_destroy(ctx)


def _coef(S, ct):
    """oracle ciphertext -> canonical coefficient-domain residues"""
    prm = S.prm
    return np.stack([np.stack([O.intt(ct.c[r, t], prm.primes[t], prm.psi[t]) for t in range(ct.level + 1)])
                     for r in range(ct.c.shape[0])])


def _encrypt_both(F, ctx, S, keys, sk, z, level, seed):
    prm = S.prm
    pt_o = S.encode(z, prm.scale, level)
    ct_o = S.encrypt(keys, pt_o, seed)
    pt_g = F.fhe_encode(ctx, z, prm.scale, level)
    ct_g = F.fhe_encrypt(ctx, sk, pt_g, seed)
    F.fhe_pt_free(pt_g)
    return ct_o, ct_g


def _assert_same(F, S, ct_o, ct_g):
    buf, lv, sc = F.fhe_ct_export(ct_g, S.prm.N)
    assert lv == ct_o.level
    assert sc == ct_o.scale
    ref = _coef(S, ct_o)
    assert buf.shape == ref.shape
    bad = np.argwhere(buf != ref)
    assert bad.size == 0, "first mismatch at %s" % (bad[:3].tolist(),)


def test_primes_match(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    assert F.fhe_ctx_primes(ctx) == prm.primes


def test_ntt_parity(pair):
    import torch
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(0)
    idx = list(range(len(prm.primes)))
    a = np.stack([rng.integers(0, prm.primes[t], prm.N, dtype=np.uint64) for t in idx])
    dev = torch.from_numpy(a.view(np.int64).copy()).cuda()
    F.fhe_ntt_device(ctx, dev.data_ptr(), idx, inverse=False)
    torch.cuda.synchronize()
    got = dev.cpu().numpy().view(np.uint64)
    want = np.stack([O.ntt(a[t], prm.primes[t], prm.psi[t]) for t in idx])
    assert np.array_equal(got, want)
    F.fhe_ntt_device(ctx, dev.data_ptr(), idx, inverse=True)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), a)


def test_encoder_bit_exact(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(1)
    for scale in (prm.scale, prm.scale ** 2, 2.0 ** 20):
        z = rng.uniform(-1, 1, prm.N // 2) + 1j * rng.uniform(-1, 1, prm.N // 2)
        assert np.array_equal(F.fhe_encode_coeffs(ctx, z, scale, prm.N), O.encode_coeffs(z, prm.logn, scale))


def test_keys_bit_exact(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    s = F.fhe_sk_export(sk, len(prm.primes) * prm.N).reshape(len(prm.primes), prm.N)
    assert np.array_equal(s, keys.s_ntt)
    relin = F.fhe_evk_export(evk, 0).reshape(-1, 2, len(prm.primes), prm.N)
    assert np.array_equal(relin, np.stack(keys.relin.digits))
    assert sorted(F.fhe_evk_galois(evk)) == sorted(keys.galois)
    for k, key in keys.galois.items():
        g = F.fhe_evk_export(evk, k).reshape(-1, 2, len(prm.primes), prm.N)
        assert np.array_equal(g, np.stack(key.digits)), k


def test_encrypt_and_decrypt(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(2)
    z = rng.uniform(-1, 1, prm.N // 2)
    for level in (prm.L, 1):
        ct_o, ct_g = _encrypt_both(F, ctx, S, keys, sk, z, level, 7 + level)
        _assert_same(F, S, ct_o, ct_g)
        pt = F.fhe_decrypt(ctx, sk, ct_g)
        back = F.fhe_decode(ctx, pt, prm.N // 2)
        F.fhe_pt_free(pt)
        # fresh-encryption noise: a few sqrt(N) in the coefficients, over the scale
        assert np.max(np.abs(back.real - z)) < max(1e-6, 40 * prm.N ** 0.5 / prm.scale)
        F.fhe_ct_free(ct_g)


def test_rotate_bit_exact(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(3)
    z = rng.uniform(-1, 1, prm.N // 2)
    for level in (prm.L, 2, 0):
        ct_o, ct_g = _encrypt_both(F, ctx, S, keys, sk, z, level, 20 + level)
        for step in (1, -1, 300):
            r_o = S.rotate(ct_o, step, keys)
            r_g = F.fhe_rotate(ctx, evk, ct_g, step)
            _assert_same(F, S, r_o, r_g)
            F.fhe_ct_free(r_g)
        F.fhe_ct_free(ct_g)


def test_missing_rotation_key_is_an_error(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    ct_o, ct_g = _encrypt_both(F, ctx, S, keys, sk, np.ones(4), prm.L, 5)
    with pytest.raises(F.FheError) as e:
        F.fhe_rotate(ctx, evk, ct_g, 2)
    assert e.value.code == -3
    F.fhe_ct_free(ct_g)


def test_square_relin_bit_exact(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, prm.N // 2)
    for level in (prm.L, 1):
        ct_o, ct_g = _encrypt_both(F, ctx, S, keys, sk, z, level, 30 + level)
        sq_o = S.relinearize(S.tensor_square(ct_o), keys)
        sq_g = F.fhe_square(ctx, evk, ct_g)
        _assert_same(F, S, sq_o, sq_g)
        F.fhe_ct_free(sq_g)
        F.fhe_ct_free(ct_g)


def test_rescale_bit_exact(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, prm.N // 2)
    ct_o, ct_g = _encrypt_both(F, ctx, S, keys, sk, z, prm.L, 40)
    sq_o = S.relinearize(S.tensor_square(ct_o), keys)
    sq_g = F.fhe_square(ctx, evk, ct_g)
    for _ in range(prm.L):
        sq_o = S.rescale(sq_o)
        F.fhe_rescale(ctx, sq_g)
        _assert_same(F, S, sq_o, sq_g)
    with pytest.raises(F.FheError) as e:
        F.fhe_rescale(ctx, sq_g)
    assert e.value.code == -2
    F.fhe_ct_free(sq_g)
    F.fhe_ct_free(ct_g)


def test_add_and_mul_plain_bit_exact(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(6)
    z1, z2 = rng.uniform(-1, 1, prm.N // 2), rng.uniform(-1, 1, prm.N // 2)
    a_o, a_g = _encrypt_both(F, ctx, S, keys, sk, z1, 3, 50)
    b_o, b_g = _encrypt_both(F, ctx, S, keys, sk, z2, 3, 51)
    s_g = F.fhe_add(ctx, a_g, b_g)
    _assert_same(F, S, S.add(a_o, b_o), s_g)
    w = rng.uniform(-1, 1, prm.N // 2)
    pt_g = F.fhe_encode(ctx, w, prm.scale, 3)
    m_g = F.fhe_mul_plain(ctx, a_g, pt_g)
    _assert_same(F, S, S.mul_plain(a_o, S.encode(w, prm.scale, 3)), m_g)
    for h in (s_g, m_g, a_g, b_g):
        F.fhe_ct_free(h)
    F.fhe_pt_free(pt_g)


def test_import_export_roundtrip(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    rng = np.random.default_rng(7)
    buf = np.stack([np.stack([rng.integers(0, prm.primes[t], prm.N, dtype=np.uint64) for t in range(3)])
                    for _ in range(2)])
    ct = F.fhe_ct_import(ctx, buf, 2, 123.0)
    back, lv, sc = F.fhe_ct_export(ct, prm.N)
    assert lv == 2 and sc == 123.0 and np.array_equal(back, buf)
    F.fhe_ct_free(ct)
    bad = buf.copy()
    bad[0, 1, 5] = prm.primes[1]
    with pytest.raises(F.FheError):
        F.fhe_ct_import(ctx, bad, 2, 1.0)


def test_add_rejects_a_scale_mismatch(pair):
    F, ctx, prm, S, keys, sk, evk = pair
    z = np.random.default_rng(8).uniform(-1, 1, prm.N // 2)
    pa = F.fhe_encode(ctx, z, prm.scale, 2)
    pb = F.fhe_encode(ctx, z, 2 * prm.scale, 2)
    a, b = F.fhe_encrypt(ctx, sk, pa, 61), F.fhe_encrypt(ctx, sk, pb, 62)
    with pytest.raises(F.FheError) as e:
        F.fhe_add(ctx, a, b)
    assert e.value.code == F.FHE_E_LEVEL
    for h in (a, b):
        F.fhe_ct_free(h)
    for h in (pa, pb):
        F.fhe_pt_free(h)


def test_injected_allocation_failure_leaves_the_context_usable(pair):
    """A refused device allocation (host-side injection) fails the call with
    FHE_E_OOM; the same calls afterwards give the same bits as before."""
    F, ctx, prm, S, keys, sk, evk = pair
    z = np.random.default_rng(9).uniform(-1, 1, prm.N // 2)
    pt = F.fhe_encode(ctx, z, prm.scale, prm.L)
    ct = F.fhe_encrypt(ctx, sk, pt, 70)
    rot = F.fhe_rotate(ctx, evk, ct, 1)
    want_ct, want_rot = F.fhe_ct_export(ct, prm.N)[0], F.fhe_ct_export(rot, prm.N)[0]
    for after in (0, 1):            # the ciphertext buffer, then the error polynomial
        F.fhe_ctx_inject_alloc_failure(ctx, after)
        with pytest.raises(F.FheError) as e:
            F.fhe_encrypt(ctx, sk, pt, 70)
        assert e.value.code == F.FHE_E_OOM and "injected" in str(e.value)
    F.fhe_ctx_inject_alloc_failure(ctx, 0)
    with pytest.raises(F.FheError) as e:
        F.fhe_rotate(ctx, evk, ct, 1)
    assert e.value.code == F.FHE_E_OOM
    # the injection turned itself off
    ct2 = F.fhe_encrypt(ctx, sk, pt, 70)
    rot2 = F.fhe_rotate(ctx, evk, ct2, 1)
    assert np.array_equal(F.fhe_ct_export(ct2, prm.N)[0], want_ct)
    assert np.array_equal(F.fhe_ct_export(rot2, prm.N)[0], want_rot)
    F.fhe_ctx_inject_alloc_failure(ctx, 5)
    F.fhe_ctx_inject_alloc_failure(ctx, -1)   # armed, then off: nothing is refused
    rot3 = F.fhe_rotate(ctx, evk, ct2, 1)
    for h in (ct, rot, ct2, rot2, rot3):
        F.fhe_ct_free(h)
    F.fhe_pt_free(pt)
