"""Key transport on the device: a key set saved by the client and loaded
into a context gives the same bits as the original keys (rotation,
relinearised square, decryption); corrupted or secret-less sets are refused."""
import json
import os
import shutil

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CFG = dict(logn=12, L=4, q_bits=45, q0_bits=50, p_bits=55, alpha=2, log_scale=35)


def test_saved_keys_give_the_same_bits(tmp_path):
    from paper_2509_22857_gb300 import _lib as F
    from paper_2509_22857_gb300 import checkpoint as K
    c = CFG
    N = 1 << c["logn"]
    ctx = F.fhe_ctx_create(c["logn"], c["L"], c["q_bits"], c["q0_bits"], c["p_bits"], c["alpha"], c["log_scale"])
    sk, evk = F.fhe_keygen(ctx, 11, [1, -1, 5])
    par = (c["logn"], c["L"], c["alpha"])
    client, server = str(tmp_path / "client"), str(tmp_path / "server")
    K.save_keys(client, ctx, evk, *par, sk=sk)
    K.save_keys(server, ctx, evk, *par)
    evk2 = K.load_evk(server, ctx, *par)
    sk2 = K.load_sk(client, ctx, *par)
    handles = []
    try:
        assert F.fhe_evk_galois(evk2) == F.fhe_evk_galois(evk)
        z = np.random.default_rng(1).uniform(-1, 1, N // 2)
        pt = F.fhe_encode(ctx, z, 2.0 ** c["log_scale"], c["L"])
        ct = F.fhe_encrypt(ctx, sk, pt, 5)
        handles.append(ct)
        for step in (1, -1, 5):
            a, b = F.fhe_rotate(ctx, evk, ct, step), F.fhe_rotate(ctx, evk2, ct, step)
            handles += [a, b]
            assert np.array_equal(F.fhe_ct_export(a, N)[0], F.fhe_ct_export(b, N)[0])
        a, b = F.fhe_square(ctx, evk, ct), F.fhe_square(ctx, evk2, ct)
        handles += [a, b]
        assert np.array_equal(F.fhe_ct_export(a, N)[0], F.fhe_ct_export(b, N)[0])
        ct2 = F.fhe_encrypt(ctx, sk2, pt, 5)       # the loaded secret key encrypts to the same bits
        handles.append(ct2)
        assert np.array_equal(F.fhe_ct_export(ct, N)[0], F.fhe_ct_export(ct2, N)[0])
        F.fhe_pt_free(pt)
        # the server's set holds no secret key
        with pytest.raises(ValueError, match="no secret"):
            K.load_sk(server, ctx, *par)
        # other parameters
        with pytest.raises(ValueError):
            K.load_evk(server, ctx, c["logn"], c["L"] + 1, c["alpha"])
        # a residue at or above its prime
        bad = str(tmp_path / "bad")
        shutil.copytree(server, bad)
        g = json.load(open(os.path.join(bad, "meta.json")))["galois"][0]
        key = np.load(os.path.join(bad, "g%d.npy" % g))
        key[7] = F.fhe_ctx_primes(ctx)[0]
        np.save(os.path.join(bad, "g%d.npy" % g), key)
        with pytest.raises(F.FheError) as e:
            K.load_evk(bad, ctx, *par)
        assert e.value.code == F.FHE_E_INVAL
        # no relinearisation key / a duplicate element
        relin = np.load(os.path.join(server, "relin.npy"))
        with pytest.raises(F.FheError):
            F.fhe_evk_import(ctx, {g: key * 0})
        with pytest.raises(F.FheError):
            F.fhe_evk_import(ctx, {0: relin, 4: relin})    # 4 is not a Galois element (even)
    finally:
        for h in handles:
            F.fhe_ct_free(h)
        F.fhe_evk_free(evk2)
        F.fhe_sk_free(sk2)
        F.fhe_evk_free(evk)
        F.fhe_sk_free(sk)
        F.fhe_ctx_destroy(ctx)
