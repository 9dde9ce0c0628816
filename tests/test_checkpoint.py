"""Checkpoints without a GPU: compiled programs survive a save / load round
trip exactly (no pickle), and a key set is refused for other parameters."""
import json

import numpy as np
import pytest

import synth
from oracle import ckks as C
from paper_2509_22857_gb300 import checkpoint as K
from paper_2509_22857_gb300 import model as M


def _compile(arch, preset, layout, members=1):
    pre = synth.PRESETS[preset]
    prm = C.make_params(**pre)
    net = synth.ARCHS[arch]()
    raw = synth.cluster_joint([synth.params(net, m) for m in range(members)], net, 4) if members > 1 else \
        synth.params(net)
    return net, M.compile_network(net, raw, prm.q, pre["logn"], pre["log_scale"], layout, pre["alpha"]), prm


@pytest.mark.parametrize("arch,preset,layout,members", [("resnet_mini", "resnet_mini", "packed", 1),
                                                        ("tiny", "tiny", "hw", 1),
                                                        ("resnet18_mini", "resnet18_mini", "hw_ens", 3)])
def test_program_round_trip(tmp_path, arch, preset, layout, members):
    net, prog, prm = _compile(arch, preset, layout, members)
    path = str(tmp_path / "prog.npz")
    K.save_program(prog, path)
    back = K.load_program(path)
    ok, where = K.programs_equal(prog, back)
    assert ok, where
    assert M.giant_steps(back) == M.giant_steps(prog) and M.keyswitch_census(back) == M.keyswitch_census(prog)
    img = synth.image(0, net[0]["c"], net[0]["h"], net[0]["w"])
    for a, b in zip(M.input_slots(prog, img, prm.N // 2), M.input_slots(back, img, prm.N // 2)):
        assert np.array_equal(a, b)
    # the file holds no pickled objects
    with np.load(path, allow_pickle=False) as z:
        assert all(z[k].dtype != object for k in z.files)


def test_programs_equal_sees_a_changed_weight(tmp_path):
    _, prog, _ = _compile("resnet_mini", "resnet_mini", "packed")
    path = str(tmp_path / "p.npz")
    K.save_program(prog, path)
    back = K.load_program(path)
    st = next(s for s in back.steps if "vecs" in s)
    st["vecs"][0] = st["vecs"][0].copy()
    st["vecs"][0][3] += 1e-12
    assert not K.programs_equal(prog, back)[0]


def test_unknown_program_format_is_refused(tmp_path):
    path = str(tmp_path / "p.npz")
    blob = np.frombuffer(json.dumps({"format": 99}).encode(), dtype=np.uint8)
    np.savez(path, __meta__=blob)
    with pytest.raises(ValueError, match="format"):
        K.load_program(path)


def test_key_set_parameters_are_checked():
    meta = {"format": K.FORMAT, "log_n": 12, "L": 4, "alpha": 2, "primes": [97, 193, 257]}
    K.check_meta(meta, 12, 4, 2, [97, 193, 257])
    for args in [(13, 4, 2, [97, 193, 257]), (12, 5, 2, [97, 193, 257]), (12, 4, 3, [97, 193, 257]),
                 (12, 4, 2, [97, 257, 193])]:
        with pytest.raises(ValueError):
            K.check_meta(meta, *args)
    with pytest.raises(ValueError, match="format"):
        K.check_meta(dict(meta, format=0), 12, 4, 2, [97, 193, 257])
