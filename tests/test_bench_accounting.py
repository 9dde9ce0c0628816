"""The bench's work accounting (the roofline's algorithmic products and
bytes) against counts done by hand on a toy program, for a single- and a
double-hoisted linear step."""
import os
import sys
from types import SimpleNamespace

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

N, LOGN, ALPHA, LV = 16, 4, 2, 3


def _prog(hoist):
    lay = SimpleNamespace(n_ct=1)
    tensors = [SimpleNamespace(level=LV, layout=lay), SimpleNamespace(level=LV, layout=lay)]
    # one output; giant steps {0, 4}; terms (input, baby): (0,0) (0,1) (0,2) in
    # group 0, (0,0) (0,1) in group 4
    st = {"kind": 1, "src": 0, "dst": 1, "hoist": hoist,
          "t_out": np.zeros(5, dtype=np.int64), "t_giant": np.array([0, 0, 0, 4, 4]),
          "t_ct": np.zeros(5, dtype=np.int64), "t_baby": np.array([0, 1, 2, 0, 1]),
          "t_vid": np.arange(5), "vecs": [None] * 5, "bias": {0: None}}
    return SimpleNamespace(tensors=tensors, steps=[st])


@pytest.mark.parametrize("hoist", [1, 2])
def test_mac_products_count_the_extended_limbs_of_rotated_terms(hoist):
    nl = LV + 1
    rot_limbs = nl + (ALPHA if hoist == 2 else 0)
    # 2 unrotated terms over Q_l, 3 rotated ones over Q_l (u P when double-hoisted)
    assert bench.mac_products(_prog(hoist), N, ALPHA) == 2 * N * (2 * nl + 3 * rot_limbs)


@pytest.mark.parametrize("hoist", [1, 2])
def test_mac_bytes_by_hand(hoist):
    W = (LV + 1) * N * 8
    WX = (LV + 1 + (ALPHA if hoist == 2 else 0)) * N * 8
    B = 3
    n_in, n_rot, n_out = 1, 2, 1          # input 0 unrotated; rotations (0,1) (0,2)
    n_grp = 2 if hoist == 2 else 0        # groups (0,0) and (0,4) hold rotated terms
    want = B * (2 * W * n_in + 2 * WX * n_rot + 2 * W * n_out + 2 * WX * n_grp) + WX * 5 + W * 1
    assert bench.mac_bytes(_prog(hoist), N, B, ALPHA) == want


@pytest.mark.parametrize("hoist", [1, 2])
def test_keyswitch_work_counts_one_moddown_per_rotated_group(hoist):
    mu, ip, md = bench.ks_parts(LV, ALPHA, LOGN)
    # one input with babies {1, 2}; one giant step (4) for one output
    # single hoisting: a ModDown per baby rotation, (0,1) and (0,2); double:
    # one per output group with rotated terms, (0,0) and (0,4): two either way
    want = mu + 2 * ip + 1 * (mu + ip) + 1 * md + 2 * md
    n_ks, mm = bench.image_modmuls(_prog(hoist), ALPHA, LOGN)
    assert n_ks == 3 and mm == want


def test_double_hoisting_counts_fewer_moddowns_when_groups_share_babies():
    prog = _prog(2)
    st = prog.steps[0]
    # three babies feeding one group: single hoisting pays 3 ModDowns, double 1
    st["t_giant"] = np.zeros(5, dtype=np.int64)
    st["t_baby"] = np.array([0, 1, 2, 3, 0])
    mu, ip, md = bench.ks_parts(LV, ALPHA, LOGN)
    _, mm2 = bench.image_modmuls(prog, ALPHA, LOGN)
    st["hoist"] = 1
    _, mm1 = bench.image_modmuls(prog, ALPHA, LOGN)
    assert mm2 == mu + 3 * ip + 1 * md
    assert mm1 == mu + 3 * (ip + md)
