"""fhe_rescale_noalloc, the rescale for callers that cannot allocate device
memory (their memory belongs to another pool or budget, or they cannot take
cudaMalloc's synchronisation): called through the C ABI on caller-owned
device buffers, twice in a row, it must give exactly the ciphertexts of the
allocating fhe_rescale."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _to_device_ntt(F, ctx, coef, level):
    import torch
    n_poly = coef.shape[0]
    dev = torch.from_numpy(np.ascontiguousarray(coef).view(np.int64).copy()).cuda()
    F.fhe_ntt_device(ctx, dev.data_ptr(), list(range(level + 1)) * n_poly, inverse=False)
    return dev


def _to_host_coef(F, ctx, dev, level, n_poly, N):
    import torch
    tmp = dev.clone()
    F.fhe_ntt_device(ctx, tmp.data_ptr(), list(range(level + 1)) * n_poly, inverse=True)
    torch.cuda.synchronize()
    return tmp.cpu().numpy().view(np.uint64).reshape(n_poly, level + 1, N)


def test_rescale_noalloc_matches_rescale_twice():
    import torch
    from paper_2509_22857_gb300 import _lib as F
    pre = synth.PRESETS["resnet20"]          # N = 2^16: the largest ring the scratch serves
    N = 1 << pre["logn"]
    ctx = F.fhe_ctx_create(pre["logn"], pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"],
                           pre["log_scale"])
    try:
        sk, evk = F.fhe_keygen(ctx, 11, [])
        z = np.random.default_rng(0).uniform(-1, 1, N // 2)
        pt = F.fhe_encode(ctx, z, 2.0 ** 50, pre["L"])
        ct = F.fhe_encrypt(ctx, sk, pt, 3)
        coef, lv, _ = F.fhe_ct_export(ct, N)
        cur = _to_device_ntt(F, ctx, coef, lv)
        stream = torch.cuda.current_stream()
        for call in range(2):
            out = torch.zeros((2 * lv * N,), dtype=torch.int64, device="cuda")
            F.fhe_rescale_noalloc(ctx, cur.data_ptr(), out.data_ptr(), 2, lv, stream)
            F.fhe_rescale(ctx, ct)                       # the allocating entry point
            want, lv2, _ = F.fhe_ct_export(ct, N)
            assert lv2 == lv - 1
            got = _to_host_coef(F, ctx, out, lv - 1, 2, N)
            assert np.array_equal(got, want), "call %d differs" % call
            cur, lv = out, lv - 1
        # beyond the fixed scratch: three polynomials of N = 2^16
        big = torch.zeros((3 * (lv + 1) * N,), dtype=torch.int64, device="cuda")
        res = torch.zeros((3 * lv * N,), dtype=torch.int64, device="cuda")
        with pytest.raises(F.FheError) as e:
            F.fhe_rescale_noalloc(ctx, big.data_ptr(), res.data_ptr(), 3, lv, stream)
        assert e.value.code == -1
        F.fhe_ct_free(ct)
        F.fhe_pt_free(pt)
        F.fhe_evk_free(evk)
        F.fhe_sk_free(sk)
    finally:
        torch.cuda.synchronize()
        F.fhe_ctx_destroy(ctx)
