"""The autotuner's host logic: which digit widths are admissible (checked
against the oracle's exact key-switching noise), the result cache, and the
tuning loops against a fake C binding (the GPU runs are in
test_gpu_autotune.py)."""
import json
import time

import numpy as np
import pytest

import synth
from oracle import ckks as C
from paper_2509_22857_gb300 import autotune as A


def test_digit_bits_and_rule_at_resnet20_parameters():
    pre = synth.PRESETS["resnet20"]
    assert A.digit_bits(20, 58, 40, 7) == [40 + 6 * 58, 7 * 58, 7 * 58]
    assert A.digit_bits(20, 58, 40, 3)[-1] == 3 * 58 and len(A.digit_bits(20, 58, 40, 3)) == 7
    # width 1 gives 21 digits, above the 16 that 58-bit primes admit (2^(62-58));
    # every width from 2 on covers its digits with 58-bit P primes
    assert A.max_digits(58) == 16 and A.max_digits(54) == 64
    assert A.admissible_widths(pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"]) == [2, 3, 4, 5, 6, 7, 8]
    # P smaller than a digit is rejected
    assert not A.admissible(4, 50, 40, 30, 2)
    assert A.admissible(4, 50, 40, 50, 2)


@pytest.mark.parametrize("name", sorted(synth.PRESETS))
def test_every_preset_uses_an_admissible_width(name):
    pre = synth.PRESETS[name]
    assert A.admissible(pre["L"], pre["q_bits"], pre["q0_bits"], pre["p_bits"], pre["alpha"])


def _keyswitch_noise_bits(p_bits, alpha):
    """log2 of the largest coefficient of KS(d) - d * s^2 (relinearisation
    key, Python integers), for a uniformly random d at the top level."""
    prm = C.make_params(logn=6, L=3, q_bits=40, q0_bits=45, p_bits=p_bits, alpha=alpha, log_scale=30)
    S = C.CKKS(prm)
    keys = S.keygen(11, [])
    lv = prm.L
    rng = np.random.default_rng(3)
    d = np.stack([rng.integers(0, prm.q[t], prm.N, dtype=np.uint64) for t in range(lv + 1)])
    ks = S.key_switch(d, lv, keys.relin)
    got = S.crt(S.decrypt_residues(keys, C.Ciphertext(ks, lv, 1.0)))
    s2 = np.stack([C.vmul(keys.s_ntt[t], keys.s_ntt[t], prm.q[t]) for t in range(lv + 1)])
    want = S.crt(np.stack([C.intt(C.vmul(d[t], s2[t], prm.q[t]), prm.q[t], prm.psi[t]) for t in range(lv + 1)]))
    Q = 1
    for q in prm.q:
        Q *= q
    return max(abs(((g - w + Q // 2) % Q) - Q // 2) for g, w in zip(got, want)).bit_length()


@pytest.mark.parametrize("p_bits,alpha", [(50, 2), (55, 2), (50, 1), (43, 2), (40, 2), (25, 2), (20, 1)])
def test_rule_matches_the_oracles_keyswitch_noise(p_bits, alpha):
    """The admissibility rule rests on the key-switching noise being about
    digit * e / P.  With the oracle's exact hybrid key switch (q_0 45-bit,
    q_1..q_3 40-bit, N = 64): admissible widths leave noise at the size of a
    fresh error (under 2^12), and a special modulus s bits short of the
    largest digit leaves s to s + 12 bits of noise."""
    noise = _keyswitch_noise_bits(p_bits, alpha)
    short = max(A.digit_bits(3, 40, 45, alpha)) - alpha * p_bits
    if A.admissible(3, 40, 45, p_bits, alpha):
        assert short <= 0 and noise < 12, noise
    else:
        assert short <= noise <= short + 12, (noise, short)


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    t = A.Tuner(path)
    t.record("k|dev|a=1", {"best": 3})
    assert json.load(open(path)) == {"k|dev|a=1": {"best": 3}}
    assert A.Tuner(path).lookup("k|dev|a=1") == {"best": 3}
    assert A.Tuner(path).lookup("other") is None


class FakeLib:
    """Stands in for the binding: key-switch time per (alpha, level) from a
    table; inference time per chunk size by sleeping; outputs as arrays."""

    def __init__(self, ks_us=None, infer_ms=None, bad_chunk=None):
        self.ks_us, self.infer_ms, self.bad_chunk = ks_us or {}, infer_ms or {}, bad_chunk
        self.live, self.calls, self.alpha, self.chunk = set(), 0, {}, None
        self.n = 0

    def _new(self, tag):
        self.n += 1
        h = (tag, self.n)
        self.live.add(h)
        return h

    def _free(self, h):
        self.live.remove(h)

    def fhe_ctx_create(self, logn, L, q, q0, p, alpha, log_scale, device=0):
        h = self._new("ctx")
        self.alpha[h] = alpha
        return h

    def fhe_ctx_destroy(self, h):
        self._free(h)

    def fhe_keygen(self, ctx, seed, rots):
        return self._new("sk"), ("evk", ctx)

    def fhe_sk_free(self, h):
        self._free(h)

    def fhe_evk_free(self, h):
        pass

    def fhe_profile_keyswitch(self, ctx, evk, level, items, iters):
        self.calls += 1
        t = self.ks_us[(self.alpha[ctx], level)] * items / 1e3
        return [t / 8] * 8

    def fhe_ctx_set_linear_chunk(self, ctx, c):
        self.chunk = c

    # the other bit-neutral knobs drive the same fake timing table
    fhe_ctx_set_mac_images = fhe_ctx_set_linear_chunk
    fhe_ctx_set_keyswitch_batch = fhe_ctx_set_linear_chunk

    def fhe_infer(self, ctx, model, evk, cts, n_img, n_out):
        time.sleep(self.infer_ms[self.chunk] / 1e3)
        return [self._new(("ct", self.chunk, k)) for k in range(n_img * n_out)]

    def fhe_ct_export(self, h, N):
        v = 7 if h[0][1] == self.bad_chunk else 1
        return np.full(4, v + h[0][2], dtype=np.uint64), 0, 1.0

    def fhe_ct_free(self, h):
        self._free(h)


def test_digit_width_tuner_weights_levels_and_caches():
    # width 3 is faster at the low level, 4 at the top: the weights decide; L = 20
    # gives width 1 twenty-one digits (more than 2^(62-58) = 16): never measured
    us = {(3, 20): 50.0, (3, 2): 10.0, (4, 20): 40.0, (4, 2): 30.0, (1, 20): 1.0, (1, 2): 1.0}
    F = FakeLib(ks_us=us)
    t = A.Tuner()
    kw = dict(logn=12, L=20, q_bits=50, q0_bits=40, p_bits=58, log_scale=25, candidates=(1, 3, 4), F=F,
              device="fake")
    top = A.tune_digit_width(t, levels=[(20, 1.0)], **kw)
    assert top["best"] == 4 and set(top["cost_us"]) == {"3", "4"}
    low = A.tune_digit_width(t, levels=[(20, 1.0), (2, 5.0)], **kw)
    assert low["best"] == 3
    assert low["cost_us"]["3"] == pytest.approx(50 + 5 * 10) and low["cost_us"]["4"] == pytest.approx(40 + 5 * 30)
    assert not F.live                        # every context and key freed
    n = F.calls
    assert A.tune_digit_width(t, levels=[(20, 1.0), (2, 5.0)], **kw) == low and F.calls == n   # cached
    with pytest.raises(ValueError):
        A.tune_digit_width(t, levels=None, **dict(kw, candidates=(1,)))


def test_linear_chunk_tuner_picks_fastest_and_checks_outputs():
    F = FakeLib(infer_ms={8: 30.0, 40: 5.0, 160: 15.0})
    t = A.Tuner()
    rec = A.tune_linear_chunk(t, "ctx", "model", "evk", [], 2, 3, 4, candidates=(8, 40, 160), reps=1, F=F,
                              device="fake", sync=lambda: None)
    assert rec["best"] == 40 and F.chunk == 40 and not F.live
    F.chunk = None
    assert A.tune_linear_chunk(t, "ctx", "model", "evk", [], 2, 3, 4, candidates=(8, 40, 160), F=F,
                               device="fake", sync=lambda: None) == rec and F.chunk == 40   # cached, applied
    bad = FakeLib(infer_ms={8: 1.0, 40: 1.0}, bad_chunk=40)
    with pytest.raises(RuntimeError, match="chunk size 40"):
        A.tune_linear_chunk(A.Tuner(), "ctx", "m", "evk", [], 1, 2, 4, candidates=(8, 40), reps=1, F=bad,
                            device="fake", sync=lambda: None)
    assert not bad.live


@pytest.mark.parametrize("tune, label", [("tune_mac_images", "images per MAC block"),
                                         ("tune_keyswitch_batch", "key-switch batch")])
def test_other_knob_tuners_pick_fastest_and_check_outputs(tune, label):
    fn = getattr(A, tune)
    F = FakeLib(infer_ms={1: 9.0, 2: 3.0, 4: 6.0})
    rec = fn(A.Tuner(), "ctx", "model", "evk", [], 2, 3, 4, candidates=(1, 2, 4), reps=1, F=F, device="fake",
             sync=lambda: None)
    assert rec["best"] == 2 and F.chunk == 2 and not F.live
    bad = FakeLib(infer_ms={1: 1.0, 4: 1.0}, bad_chunk=4)
    with pytest.raises(RuntimeError, match="%s 4" % label):
        fn(A.Tuner(), "ctx", "m", "evk", [], 1, 2, 4, candidates=(1, 4), reps=1, F=bad, device="fake",
           sync=lambda: None)


def test_keyswitch_census_of_a_small_network():
    """Levels of the census lie in [0, L]; the first linear step switches at
    the top level; the weights the tuner gets are the census, top first."""
    from paper_2509_22857_gb300 import model as M
    pre = synth.PRESETS["resnet_mini"]
    prm = C.make_params(**pre)
    net = synth.resnet_mini()
    prog = M.compile_network(net, synth.params(net), prm.q, pre["logn"], pre["log_scale"], "packed", pre["alpha"])
    census = M.keyswitch_census(prog)
    assert census and all(0 <= lv <= pre["L"] for lv in census) and pre["L"] in census
    lv = A.keyswitch_levels(prog)
    assert [l for l, _ in lv] == sorted(census, reverse=True) and sum(k for _, k in lv) == sum(census.values())
    acts = [st for st in prog.steps if st["kind"] == 3]
    assert all(M.keyswitches_of_step(prog, st) == prog.tensors[st["src"]].layout.n_ct for st in acts)


class FakePipeLib:
    """Pipelines whose tick sleeps per group size; sizes in `oom` are refused
    at creation, as fhe_pipeline_create refuses a pipeline that does not fit."""
    FheError = None
    FHE_E_OOM = -4

    def __init__(self, tick_ms, oom=()):
        from paper_2509_22857_gb300 import _lib
        self.FheError = _lib.FheError
        self.tick_ms, self.oom, self.live, self.n = tick_ms, set(oom), set(), 0

    def fhe_pipeline_create(self, ctx, model, evk, g, graphs):
        if g in self.oom:
            raise self.FheError(self.FHE_E_OOM, "out of memory")
        self.n += 1
        h = ("pipe", g, self.n)
        self.live.add(h)
        return h

    def fhe_pipeline_info(self, pipe):
        return (3, 0, 1, 1)

    def fhe_pipeline_tick(self, pipe, grp, g, n):
        time.sleep(self.tick_ms[pipe[1]] / 1e3)
        return [], 0, -1

    def fhe_pipeline_free(self, pipe):
        self.live.remove(pipe)


def test_pipeline_group_tuner_skips_sizes_that_do_not_fit():
    F = FakePipeLib({2: 4.0, 4: 5.0, 8: 6.0}, oom=(16,))
    rec = A.tune_pipeline_group(A.Tuner(), "ctx", "m", "evk", [[1], [2]], 1, 4, candidates=(2, 4, 8, 16), F=F,
                                device="fake", sync=lambda: None)
    # images per second: 2/4 ms, 4/5 ms, 8/6 ms -> 8 is best; 16 refused
    assert rec["best"] == 8 and set(rec["img_s"]) == {"2", "4", "8"} and "16" in rec["refused"]
    assert not F.live
    with pytest.raises(RuntimeError, match="fits"):
        A.tune_pipeline_group(A.Tuner(), "ctx", "m", "evk", [[1]], 1, 4, candidates=(16,), F=FakePipeLib({}, (16,)),
                              device="fake", sync=lambda: None)
