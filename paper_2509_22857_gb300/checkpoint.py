"""Checkpoints on disk: key sets and compiled network programs.

Key generation and the offline compilation (diagonals, baby-step /
giant-step split, level plan) need not be redone between runs, and a client
can hand its evaluation keys to a server, which never sees the secret key
(Sec. 2.2: the server holds the model and the public evaluation keys).

A key set is a directory:

* ``meta.json``: format version, log N, L, alpha, the prime chain
  (q_0..q_L, p_0..), the Galois elements present, words per key;
* ``relin.npy`` and ``g<element>.npy``: one key each, uint64 in the layout
  of ``fhe_evk_export`` ([dnum][2][L+1+alpha][N], NTT domain);
* ``sk.npy``: the secret key, only when saved with ``secret=True`` (a
  client-side file; the server-side set has none).

Loading checks the directory against the context (same parameters and the
same primes, in order); the library rejects out-of-range residues.

A program is one ``.npz`` file: its structure as JSON plus its arrays as
members, read back with ``allow_pickle=False`` (no code runs on load).
"""
from __future__ import annotations

import json
import os
from typing import Dict, Tuple

import numpy as np

from . import _lib as F
from . import model as M

FORMAT = 1


# ============================================================ key sets

def _ctx_meta(ctx, log_n: int, L: int, alpha: int) -> dict:
    return {"format": FORMAT, "log_n": log_n, "L": L, "alpha": alpha, "primes": [int(p) for p in F.fhe_ctx_primes(ctx)]}


def check_meta(meta: dict, log_n: int, L: int, alpha: int, primes) -> None:
    """Raise ValueError unless a saved key set belongs to these parameters."""
    if meta.get("format") != FORMAT:
        raise ValueError("unknown key-set format %r" % meta.get("format"))
    for k, v in (("log_n", log_n), ("L", L), ("alpha", alpha)):
        if meta.get(k) != v:
            raise ValueError("key set has %s = %r, the context %r" % (k, meta.get(k), v))
    if [int(p) for p in meta.get("primes", [])] != [int(p) for p in primes]:
        raise ValueError("key set was made for another prime chain")


def save_keys(path: str, ctx, evk, log_n: int, L: int, alpha: int, sk=None) -> None:
    """Write the evaluation keys (and the secret key if given) to directory `path`."""
    os.makedirs(path, exist_ok=True)
    meta = _ctx_meta(ctx, log_n, L, alpha)
    galois = F.fhe_evk_galois(evk)
    relin = F.fhe_evk_export(evk, 0)
    np.save(os.path.join(path, "relin.npy"), relin)
    for g in galois:
        np.save(os.path.join(path, "g%d.npy" % g), F.fhe_evk_export(evk, g))
    if sk is not None:
        n = (L + 1 + alpha) << log_n
        np.save(os.path.join(path, "sk.npy"), F.fhe_sk_export(sk, n))
    meta.update(galois=[int(g) for g in galois], words_per_key=int(relin.size), secret=sk is not None)
    with open(os.path.join(path, "meta.json"), "w") as f:
        json.dump(meta, f, indent=1)


def _load_meta(path: str, ctx, log_n: int, L: int, alpha: int) -> dict:
    with open(os.path.join(path, "meta.json")) as f:
        meta = json.load(f)
    check_meta(meta, log_n, L, alpha, F.fhe_ctx_primes(ctx))
    return meta


def load_evk(path: str, ctx, log_n: int, L: int, alpha: int) -> int:
    """Evaluation key set of directory `path` on the context's device."""
    meta = _load_meta(path, ctx, log_n, L, alpha)
    keys: Dict[int, np.ndarray] = {0: np.load(os.path.join(path, "relin.npy"), allow_pickle=False)}
    for g in meta["galois"]:
        keys[int(g)] = np.load(os.path.join(path, "g%d.npy" % g), allow_pickle=False)
    return F.fhe_evk_import(ctx, keys)


def load_sk(path: str, ctx, log_n: int, L: int, alpha: int) -> int:
    meta = _load_meta(path, ctx, log_n, L, alpha)
    if not meta.get("secret"):
        raise ValueError("this key set holds no secret key")
    return F.fhe_sk_import(ctx, np.load(os.path.join(path, "sk.npy"), allow_pickle=False))


# ============================================================ programs

def _enc(v, name: str, arrays: Dict[str, np.ndarray]):
    if isinstance(v, np.ndarray):
        arrays[name] = v
        return {"nd": name}
    if isinstance(v, list) and v and all(isinstance(x, np.ndarray) for x in v):
        keys = []
        for i, x in enumerate(v):
            arrays["%s.%d" % (name, i)] = x
            keys.append("%s.%d" % (name, i))
        return {"ndl": keys}
    if isinstance(v, dict):
        out = []
        for k in sorted(v):
            if not isinstance(v[k], np.ndarray):
                raise TypeError("dict values must be arrays (%s)" % name)
            arrays["%s.%d" % (name, k)] = v[k]
            out.append([int(k), "%s.%d" % (name, k)])
        return {"ndd": out}
    if isinstance(v, (bool, int, float, str)) or v is None:
        return v
    if isinstance(v, (list, tuple)) and all(isinstance(x, (int, float)) for x in v):
        return list(v)
    if isinstance(v, (np.integer, np.floating)):
        return v.item()
    raise TypeError("cannot store %s (%s)" % (name, type(v).__name__))


def _dec(v, z):
    if isinstance(v, dict):
        if "nd" in v:
            return z[v["nd"]]
        if "ndl" in v:
            return [z[k] for k in v["ndl"]]
        if "ndd" in v:
            return {int(k): z[n] for k, n in v["ndd"]}
    return v


def save_program(prog: M.Program, path: str) -> None:
    arrays: Dict[str, np.ndarray] = {}
    tensors = [{"layout": {"n_ct": t.layout.n_ct, "copies": [[list(c) for c in cs] for cs in t.layout.copies],
                           "H": t.layout.H, "W": t.layout.W, "st": t.layout.st, "row": t.layout.row,
                           "block": t.layout.block},
                "level": t.level, "scale": t.scale} for t in prog.tensors]
    steps = [{k: _enc(v, "s%d.%s" % (i, k), arrays) for k, v in st.items()} for i, st in enumerate(prog.steps)]
    meta = {"format": FORMAT, "tensors": tensors, "steps": steps, "rotations": sorted(int(r) for r in prog.rotations),
            "input": prog.input, "output": prog.output}
    blob = np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8)
    with open(path, "wb") as f:
        np.savez(f, __meta__=blob, **arrays)


def load_program(path: str) -> M.Program:
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(bytes(z["__meta__"]).decode())
        if meta.get("format") != FORMAT:
            raise ValueError("unknown program format %r" % meta.get("format"))
        tensors = []
        for t in meta["tensors"]:
            lay = dict(t["layout"])
            lay["copies"] = [[tuple(c) for c in cs] for cs in lay["copies"]]
            tensors.append(M.TInfo(M.SlotMap(**lay), int(t["level"]), float(t["scale"])))
        steps = [{k: _dec(v, z) for k, v in st.items()} for st in meta["steps"]]
    return M.Program(tensors=tensors, steps=steps, rotations=set(meta["rotations"]), input=meta["input"],
                     output=meta["output"])


def programs_equal(a: M.Program, b: M.Program) -> Tuple[bool, str]:
    """(equal, first difference): tensors, steps (arrays element by element), rotations."""
    if a.input != b.input or a.output != b.output or a.rotations != b.rotations:
        return False, "input / output / rotations"
    if len(a.tensors) != len(b.tensors) or len(a.steps) != len(b.steps):
        return False, "lengths"
    for i, (x, y) in enumerate(zip(a.tensors, b.tensors)):
        if x != y:
            return False, "tensor %d" % i
    for i, (x, y) in enumerate(zip(a.steps, b.steps)):
        if set(x) != set(y):
            return False, "step %d keys" % i
        for k in x:
            u, v = x[k], y[k]
            if isinstance(u, np.ndarray):
                same = isinstance(v, np.ndarray) and u.dtype == v.dtype and np.array_equal(u, v)
            elif isinstance(u, list) and u and isinstance(u[0], np.ndarray):
                same = len(u) == len(v) and all(p.dtype == q.dtype and np.array_equal(p, q) for p, q in zip(u, v))
            elif isinstance(u, dict):
                same = set(u) == set(v) and all(np.array_equal(u[j], v[j]) for j in u)
            else:
                same = u == v
            if not same:
                return False, "step %d field %s" % (i, k)
    return True, ""
