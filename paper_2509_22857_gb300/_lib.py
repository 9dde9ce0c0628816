"""ctypes binding of libfhecnn.so (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments and check the return code; all computation
happens in the CUDA library.  Loading fails loudly when the library has not
been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfhecnn.so")

c_int, c_size, c_u64, c_double, c_void = (ctypes.c_int, ctypes.c_size_t, ctypes.c_uint64,
                                          ctypes.c_double, ctypes.c_void_p)
P_U64 = ctypes.POINTER(ctypes.c_uint64)
P_I32 = ctypes.POINTER(ctypes.c_int32)
P_DBL = ctypes.POINTER(ctypes.c_double)
P_I64 = ctypes.POINTER(ctypes.c_int64)
PP = ctypes.POINTER(ctypes.c_void_p)


class FheParams(ctypes.Structure):
    _fields_ = [("log_n", c_int), ("L", c_int), ("q_bits", c_int), ("q0_bits", c_int),
                ("p_bits", c_int), ("alpha", c_int), ("log_scale", c_double), ("device", c_int),
                ("primes", P_U64)]


class FheStepDesc(ctypes.Structure):
    _fields_ = [("kind", c_int), ("src", c_int), ("src2", c_int), ("dst", c_int),
                ("w_scale", c_double), ("bias_scale", c_double),
                ("n_groups", c_int), ("group_out", P_I32), ("group_giant", P_I32),
                ("group_term_begin", P_I32), ("term_ct", P_I32), ("term_baby", P_I32),
                ("term_vec_id", P_I32), ("n_vecs", c_int), ("vecs", P_DBL),
                ("n_bias", c_int), ("bias_out", P_I32), ("bias_vec", P_DBL),
                ("c1", c_double), ("c0", c_double), ("value", c_double),
                ("n_steps", c_int), ("steps", P_I32), ("level", c_int),
                ("sparse_vec_begin", P_I64), ("sparse_slot", P_I32), ("sparse_val", P_DBL),
                ("act_c1_vecs", P_DBL), ("act_c0_vecs", P_DBL), ("act_c1_scale", c_double),
                ("act_c0_scale", c_double), ("double_hoist", c_int)]


class FheModelDesc(ctypes.Structure):
    _fields_ = [("n_tensors", c_int), ("tensor_n_ct", P_I32), ("tensor_level", P_I32),
                ("tensor_scale", P_DBL), ("input_tensor", c_int), ("output_tensor", c_int),
                ("n_steps", c_int), ("steps", ctypes.POINTER(FheStepDesc))]


STEP_LINEAR, STEP_RESCALE, STEP_ACT, STEP_ROTSUM, STEP_CMUL, STEP_DROP, STEP_ADD = 1, 2, 3, 4, 5, 6, 7

_lib = None


# error codes of include/fhecnn.h
FHE_OK, FHE_E_INVAL, FHE_E_LEVEL, FHE_E_NOKEY, FHE_E_OOM, FHE_E_CUDA, FHE_E_TIMEOUT = 0, -1, -2, -3, -4, -5, -6


class FheError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libfhecnn error %d: %s" % (code, msg))
        self.code = code


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfhecnn.so is not built (run paper_2509_22857_gb300/build.py); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        V = c_void
        sigs = {
            "fhe_last_error": (ctypes.c_char_p, []),
            "fhe_kernel_launches": (ctypes.c_uint64, []),
            "fhe_ctx_create": (c_int, [ctypes.POINTER(FheParams), PP]),
            "fhe_ctx_destroy": (c_int, [V]),
            "fhe_ctx_set_encode_scratch": (c_int, [V, c_size]),
            "fhe_ctx_set_keyswitch_batch": (c_int, [V, c_int]),
            "fhe_ctx_set_mac_images": (c_int, [V, c_int]),
            "fhe_ctx_set_linear_chunk": (c_int, [V, c_int]),
            "fhe_ctx_inject_alloc_failure": (c_int, [V, c_int]),
            "fhe_ctx_primes": (c_int, [V, P_U64, c_size, ctypes.POINTER(c_size)]),
            "fhe_keygen": (c_int, [V, c_u64, P_I32, c_size, PP, PP]),
            "fhe_sk_free": (c_int, [V]),
            "fhe_evk_free": (c_int, [V]),
            "fhe_evk_galois": (c_int, [V, P_I32, c_size, ctypes.POINTER(c_size)]),
            "fhe_encode": (c_int, [V, P_DBL, P_DBL, c_size, c_double, c_int, PP]),
            "fhe_pt_free": (c_int, [V]),
            "fhe_encrypt": (c_int, [V, V, V, c_u64, PP]),
            "fhe_decrypt": (c_int, [V, V, V, PP]),
            "fhe_decode": (c_int, [V, V, P_DBL, P_DBL, c_size]),
            "fhe_ct_free": (c_int, [V]),
            "fhe_ct_info": (c_int, [V, ctypes.POINTER(c_int), ctypes.POINTER(c_int), P_DBL]),
            "fhe_ct_export": (c_int, [V, P_U64, c_size, ctypes.POINTER(c_int), P_DBL, ctypes.POINTER(c_int)]),
            "fhe_ct_import": (c_int, [V, P_U64, c_int, c_int, c_double, PP]),
            "fhe_rotate": (c_int, [V, V, V, c_int, PP, V]),
            "fhe_square": (c_int, [V, V, V, PP, V]),
            "fhe_rescale": (c_int, [V, V, V]),
            "fhe_rescale_noalloc": (c_int, [V, V, V, c_int, c_int, V]),
            "fhe_add": (c_int, [V, V, V, PP, V]),
            "fhe_mul_plain": (c_int, [V, V, V, PP, V]),
            "fhe_model_load": (c_int, [V, ctypes.POINTER(FheModelDesc), PP]),
            "fhe_model_free": (c_int, [V]),
            "fhe_eval_conv": (c_int, [V, V, V, c_int, PP, c_size, PP, c_size, V]),
            "fhe_eval_quad_act": (c_int, [V, V, V, c_int, PP, c_size, V]),
            "fhe_eval_pool_dense": (c_int, [V, V, V, c_int, PP, c_size, PP, c_size, V]),
            "fhe_infer": (c_int, [V, V, V, PP, c_size, PP, V]),
            "fhe_infer_profiled": (c_int, [V, V, V, PP, c_size, PP, V, P_DBL]),
            "fhe_pipeline_create": (c_int, [V, V, V, c_int, c_int, PP]),
            "fhe_pipeline_info": (c_int, [V, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                          ctypes.POINTER(c_int)]),
            "fhe_pipeline_tick": (c_int, [V, PP, c_size, PP, ctypes.POINTER(c_size),
                                          ctypes.POINTER(ctypes.c_int64)]),
            "fhe_pipeline_ticks": (c_int, [V, ctypes.POINTER(ctypes.c_int64)]),
            "fhe_pipeline_free": (c_int, [V]),
            "fhe_server_create": (c_int, [V, V, PP]),
            "fhe_server_add_model": (c_int, [V, V, c_int, c_size, ctypes.POINTER(c_int)]),
            "fhe_server_submit": (c_int, [V, c_int, PP, ctypes.POINTER(c_u64)]),
            "fhe_server_poll": (c_int, [V, c_u64, c_int, PP, c_size, ctypes.POINTER(c_size), P_DBL]),
            "fhe_server_stats": (c_int, [V, ctypes.POINTER(c_u64), P_DBL, P_DBL]),
            "fhe_server_pause": (c_int, [V, c_int]),
            "fhe_server_destroy": (c_int, [V]),
            "fhe_ntt_device": (c_int, [V, V, c_size, P_I32, c_int, V]),
            "fhe_evk_export": (c_int, [V, c_int, P_U64, c_size, ctypes.POINTER(c_size)]),
            "fhe_sk_export": (c_int, [V, P_U64, c_size]),
            "fhe_sk_import": (c_int, [V, P_U64, c_size, PP]),
            "fhe_evk_import": (c_int, [V, P_I32, c_size, ctypes.POINTER(P_U64), c_size, PP]),
            "fhe_profile_keyswitch": (c_int, [V, V, c_int, c_int, c_int, ctypes.POINTER(ctypes.c_float), V]),
            "fhe_encode_coeffs": (c_int, [V, P_DBL, P_DBL, c_size, c_double, P_DBL]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise FheError(rc, lib().fhe_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(t)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


# ------------------------------------------------------------------ context

def fhe_kernel_launches() -> int:
    return int(lib().fhe_kernel_launches())


def fhe_ctx_create(log_n, L, q_bits, q0_bits, p_bits, alpha, log_scale, device=0, primes=None) -> int:
    """primes: optional explicit chain q_0..q_L, p_0..p_{alpha-1} (the bit
    sizes are then ignored)"""
    arr = None
    if primes is not None:
        arr = np.ascontiguousarray(np.array([int(x) for x in primes], dtype=np.uint64))
        if arr.size != L + 1 + alpha:
            raise ValueError("an explicit chain has L + 1 + alpha primes")
    p = FheParams(log_n, L, q_bits, q0_bits, p_bits, alpha, float(log_scale), device,
                  _ptr(arr, P_U64) if arr is not None else None)
    h = c_void()
    _check(lib().fhe_ctx_create(ctypes.byref(p), ctypes.byref(h)))
    return h.value


def fhe_ctx_destroy(ctx):
    _check(lib().fhe_ctx_destroy(ctx))


def fhe_ctx_set_linear_chunk(ctx, lin_chunk_srcs: int):
    _check(lib().fhe_ctx_set_linear_chunk(ctx, int(lin_chunk_srcs)))


def fhe_ctx_inject_alloc_failure(ctx, after: int):
    _check(lib().fhe_ctx_inject_alloc_failure(ctx, int(after)))


def fhe_ctx_set_encode_scratch(ctx, n_bytes: int):
    _check(lib().fhe_ctx_set_encode_scratch(ctx, int(n_bytes)))


def fhe_ctx_set_keyswitch_batch(ctx, max_items: int):
    _check(lib().fhe_ctx_set_keyswitch_batch(ctx, int(max_items)))


def fhe_ctx_set_mac_images(ctx, images_per_cta: int):
    _check(lib().fhe_ctx_set_mac_images(ctx, int(images_per_cta)))


def fhe_ctx_primes(ctx) -> List[int]:
    n = c_size()
    _check(lib().fhe_ctx_primes(ctx, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.uint64)
    _check(lib().fhe_ctx_primes(ctx, _ptr(out, P_U64), n.value, ctypes.byref(n)))
    return [int(x) for x in out]


# ------------------------------------------------------------------ client

def fhe_keygen(ctx, seed: int, rot_steps: Sequence[int]) -> Tuple[int, int]:
    st = np.ascontiguousarray(np.array(list(rot_steps) or [0], dtype=np.int32))
    sk, evk = c_void(), c_void()
    _check(lib().fhe_keygen(ctx, seed, _ptr(st, P_I32), len(rot_steps), ctypes.byref(sk), ctypes.byref(evk)))
    return sk.value, evk.value


def fhe_sk_free(sk):
    _check(lib().fhe_sk_free(sk))


def fhe_evk_free(evk):
    _check(lib().fhe_evk_free(evk))


def fhe_evk_galois(evk) -> List[int]:
    n = c_size()
    _check(lib().fhe_evk_galois(evk, None, 0, ctypes.byref(n)))
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(lib().fhe_evk_galois(evk, _ptr(out, P_I32), n.value, ctypes.byref(n)))
    return [int(x) for x in out[: n.value]]


def fhe_sk_import(ctx, words: np.ndarray) -> int:
    """secret key from the words of fhe_sk_export"""
    w = np.ascontiguousarray(words, dtype=np.uint64)
    h = c_void()
    _check(lib().fhe_sk_import(ctx, _ptr(w, P_U64), w.size, ctypes.byref(h)))
    return h.value


def fhe_evk_import(ctx, keys) -> int:
    """evaluation key set from {galois element: words of fhe_evk_export}
    (element 0: the relinearisation key)"""
    items = sorted(keys.items())
    arrs = [np.ascontiguousarray(v, dtype=np.uint64) for _, v in items]
    words = arrs[0].size if arrs else 0
    if any(a.size != words for a in arrs):
        raise ValueError("keys of different sizes")
    gal = np.ascontiguousarray([g for g, _ in items] or [0], dtype=np.int32)
    ptrs = (P_U64 * max(len(arrs), 1))(*[_ptr(a, P_U64) for a in arrs])
    h = c_void()
    _check(lib().fhe_evk_import(ctx, _ptr(gal, P_I32), len(arrs), ptrs, words, ctypes.byref(h)))
    return h.value


def fhe_encode(ctx, z, scale: float, level: int) -> int:
    z = np.asarray(z)
    re = np.ascontiguousarray(z.real, dtype=np.float64)
    im = np.ascontiguousarray(z.imag, dtype=np.float64) if np.iscomplexobj(z) else None
    h = c_void()
    _check(lib().fhe_encode(ctx, _ptr(re, P_DBL), _ptr(im, P_DBL) if im is not None else None, re.size,
                            float(scale), level, ctypes.byref(h)))
    return h.value


def fhe_encode_coeffs(ctx, z, scale: float, n_coeffs: int) -> np.ndarray:
    z = np.asarray(z)
    re = np.ascontiguousarray(z.real, dtype=np.float64)
    im = np.ascontiguousarray(z.imag, dtype=np.float64) if np.iscomplexobj(z) else None
    out = np.zeros(n_coeffs, dtype=np.float64)
    _check(lib().fhe_encode_coeffs(ctx, _ptr(re, P_DBL), _ptr(im, P_DBL) if im is not None else None,
                                   re.size, float(scale), _ptr(out, P_DBL)))
    return out


def fhe_pt_free(pt):
    _check(lib().fhe_pt_free(pt))


def fhe_encrypt(ctx, sk, pt, seed: int) -> int:
    h = c_void()
    _check(lib().fhe_encrypt(ctx, sk, pt, seed, ctypes.byref(h)))
    return h.value


def fhe_decrypt(ctx, sk, ct) -> int:
    h = c_void()
    _check(lib().fhe_decrypt(ctx, sk, ct, ctypes.byref(h)))
    return h.value


def fhe_decode(ctx, pt, n: int) -> np.ndarray:
    re = np.zeros(n, dtype=np.float64)
    im = np.zeros(n, dtype=np.float64)
    _check(lib().fhe_decode(ctx, pt, _ptr(re, P_DBL), _ptr(im, P_DBL), n))
    return re + 1j * im


# ------------------------------------------------------------------ ciphertexts

def fhe_ct_free(ct):
    _check(lib().fhe_ct_free(ct))


def fhe_ct_info(ct) -> Tuple[int, int, float]:
    lv, npoly, sc = c_int(), c_int(), c_double()
    _check(lib().fhe_ct_info(ct, ctypes.byref(lv), ctypes.byref(npoly), ctypes.byref(sc)))
    return lv.value, npoly.value, sc.value


def fhe_ct_export(ct, N: int) -> Tuple[np.ndarray, int, float]:
    lv, npoly, sc = fhe_ct_info(ct)
    buf = np.zeros((npoly, lv + 1, N), dtype=np.uint64)
    l2, s2, n2 = c_int(), c_double(), c_int()
    _check(lib().fhe_ct_export(ct, _ptr(buf, P_U64), buf.size, ctypes.byref(l2), ctypes.byref(s2),
                               ctypes.byref(n2)))
    return buf, l2.value, s2.value


def fhe_ct_import(ctx, buf: np.ndarray, level: int, scale: float) -> int:
    buf = np.ascontiguousarray(buf, dtype=np.uint64)
    h = c_void()
    _check(lib().fhe_ct_import(ctx, _ptr(buf, P_U64), buf.shape[0], level, float(scale), ctypes.byref(h)))
    return h.value


# ------------------------------------------------------------------ evaluation

def fhe_rotate(ctx, evk, ct, step: int, stream=None) -> int:
    h = c_void()
    _check(lib().fhe_rotate(ctx, evk, ct, step, ctypes.byref(h), _stream(stream)))
    return h.value


def fhe_square(ctx, evk, ct, stream=None) -> int:
    h = c_void()
    _check(lib().fhe_square(ctx, evk, ct, ctypes.byref(h), _stream(stream)))
    return h.value


def fhe_rescale(ctx, ct, stream=None):
    _check(lib().fhe_rescale(ctx, ct, _stream(stream)))


def fhe_rescale_noalloc(ctx, in_dev_ptr: int, out_dev_ptr: int, n_poly: int, level: int, stream=None):
    _check(lib().fhe_rescale_noalloc(ctx, in_dev_ptr, out_dev_ptr, n_poly, level, _stream(stream)))


def fhe_add(ctx, a, b, stream=None) -> int:
    h = c_void()
    _check(lib().fhe_add(ctx, a, b, ctypes.byref(h), _stream(stream)))
    return h.value


def fhe_mul_plain(ctx, a, pt, stream=None) -> int:
    h = c_void()
    _check(lib().fhe_mul_plain(ctx, a, pt, ctypes.byref(h), _stream(stream)))
    return h.value


def _handles(hs) -> ctypes.Array:
    arr = (c_void * max(len(hs), 1))()
    for i, h in enumerate(hs):
        arr[i] = h
    return arr


def fhe_model_load(ctx, desc: FheModelDesc) -> int:
    h = c_void()
    _check(lib().fhe_model_load(ctx, ctypes.byref(desc), ctypes.byref(h)))
    return h.value


def fhe_model_free(m):
    _check(lib().fhe_model_free(m))


def fhe_eval_conv(ctx, model, evk, step: int, cts, n_out: int, stream=None) -> List[int]:
    out = (c_void * n_out)()
    _check(lib().fhe_eval_conv(ctx, model, evk, step, _handles(cts), len(cts), out, n_out, _stream(stream)))
    return [out[i] for i in range(n_out)]


def fhe_eval_pool_dense(ctx, model, evk, step: int, cts, n_out: int, stream=None) -> List[int]:
    out = (c_void * n_out)()
    _check(lib().fhe_eval_pool_dense(ctx, model, evk, step, _handles(cts), len(cts), out, n_out,
                                     _stream(stream)))
    return [out[i] for i in range(n_out)]


def fhe_eval_quad_act(ctx, model, evk, step: int, cts, stream=None):
    _check(lib().fhe_eval_quad_act(ctx, model, evk, step, _handles(cts), len(cts), _stream(stream)))


def fhe_infer(ctx, model, evk, cts, n_img: int, n_out_per_img: int, stream=None) -> List[int]:
    out = (c_void * (n_img * n_out_per_img))()
    _check(lib().fhe_infer(ctx, model, evk, _handles(cts), n_img, out, _stream(stream)))
    return [out[i] for i in range(n_img * n_out_per_img)]


PHASES = {2: "rescale", 3: "activation", 4: "rotsum", 5: "cmul", 6: "drop", 7: "add",
          10: "linear_baby_rotations", 11: "linear_mac", 12: "linear_giant_rotations",
          13: "linear_encode_on_demand"}


def fhe_infer_profiled(ctx, model, evk, cts, n_img: int, n_out_per_img: int, stream=None):
    """(output handles, {phase: ms})"""
    out = (c_void * (n_img * n_out_per_img))()
    ms = np.zeros(16, dtype=np.float64)
    _check(lib().fhe_infer_profiled(ctx, model, evk, _handles(cts), n_img, out, _stream(stream), _ptr(ms, P_DBL)))
    return [out[i] for i in range(n_img * n_out_per_img)], {PHASES[k]: float(ms[k]) for k in PHASES}


def fhe_pipeline_create(ctx, model, evk, group: int, use_graphs: bool = True) -> int:
    h = c_void()
    _check(lib().fhe_pipeline_create(ctx, model, evk, group, int(use_graphs), ctypes.byref(h)))
    return h.value


def fhe_pipeline_info(pipe) -> Tuple[int, int, int, int]:
    a, b, c_, d = c_int(), c_int(), c_int(), c_int()
    _check(lib().fhe_pipeline_info(pipe, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c_), ctypes.byref(d)))
    return a.value, b.value, c_.value, d.value


def fhe_pipeline_tick(pipe, cts, n_in: int, out_capacity: int) -> Tuple[List[int], int, int]:
    """returns (output handles, images completed, entry tick of that group or -1)"""
    out = (c_void * max(out_capacity, 1))()
    n_out, tag = c_size(), ctypes.c_int64()
    _check(lib().fhe_pipeline_tick(pipe, _handles(cts), n_in, out, ctypes.byref(n_out), ctypes.byref(tag)))
    n_ct_out = fhe_pipeline_info(pipe)[3]
    return [out[i] for i in range(n_out.value * n_ct_out)], n_out.value, tag.value


def fhe_pipeline_ticks(pipe) -> int:
    t = ctypes.c_int64()
    _check(lib().fhe_pipeline_ticks(pipe, ctypes.byref(t)))
    return t.value


def fhe_pipeline_free(pipe):
    _check(lib().fhe_pipeline_free(pipe))


def fhe_server_create(ctx, evk) -> int:
    h = c_void()
    _check(lib().fhe_server_create(ctx, evk, ctypes.byref(h)))
    return h.value


def fhe_server_add_model(server, model, group: int, reserve_bytes: int = 0) -> int:
    mid = c_int()
    _check(lib().fhe_server_add_model(server, model, group, reserve_bytes, ctypes.byref(mid)))
    return mid.value


def fhe_server_submit(server, model_id: int, cts) -> int:
    t = c_u64()
    _check(lib().fhe_server_submit(server, model_id, _handles(cts), ctypes.byref(t)))
    return t.value


def fhe_server_poll(server, ticket: int, wait, cap: int) -> Tuple[List[int], float]:
    """returns (output handles, latency ms); no handles while pending.
    wait: True (until done), False (not at all) or a timeout in milliseconds,
    after which FheError with code FHE_E_TIMEOUT is raised."""
    timeout_ms = -1 if wait is True else 0 if wait is False else int(wait)
    out = (c_void * max(cap, 1))()
    n, lat = c_size(), c_double()
    _check(lib().fhe_server_poll(server, ticket, timeout_ms, out, cap, ctypes.byref(n), ctypes.byref(lat)))
    return [out[i] for i in range(n.value)], lat.value


def fhe_server_pause(server, paused: bool):
    _check(lib().fhe_server_pause(server, int(bool(paused))))


def fhe_server_stats(server) -> Tuple[int, float, float]:
    n, p50, p99 = c_u64(), c_double(), c_double()
    _check(lib().fhe_server_stats(server, ctypes.byref(n), ctypes.byref(p50), ctypes.byref(p99)))
    return n.value, p50.value, p99.value


def fhe_server_destroy(server):
    _check(lib().fhe_server_destroy(server))


# ------------------------------------------------------------------ test hooks

def fhe_ntt_device(ctx, dev_ptr: int, prime_idx: Sequence[int], inverse: bool, stream=None):
    p = np.ascontiguousarray(np.array(prime_idx, dtype=np.int32))
    _check(lib().fhe_ntt_device(ctx, dev_ptr, len(prime_idx), _ptr(p, P_I32), int(inverse), _stream(stream)))


def fhe_evk_export(evk, galois: int) -> np.ndarray:
    n = c_size()
    _check(lib().fhe_evk_export(evk, galois, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.uint64)
    _check(lib().fhe_evk_export(evk, galois, _ptr(out, P_U64), n.value, ctypes.byref(n)))
    return out


def fhe_profile_keyswitch(ctx, evk, level: int, n_items: int, iters: int, stream=None) -> List[float]:
    ms = (ctypes.c_float * 8)()
    _check(lib().fhe_profile_keyswitch(ctx, evk, level, n_items, iters, ms, _stream(stream)))
    return [float(x) for x in ms]


def fhe_sk_export(sk, n_words: int) -> np.ndarray:
    out = np.zeros(n_words, dtype=np.uint64)
    _check(lib().fhe_sk_export(sk, _ptr(out, P_U64), n_words))
    return out


EXPORTED = ["fhe_last_error", "fhe_kernel_launches", "fhe_ctx_create", "fhe_ctx_destroy", "fhe_ctx_primes",
            "fhe_ctx_set_linear_chunk", "fhe_ctx_set_encode_scratch", "fhe_ctx_set_keyswitch_batch", "fhe_ctx_set_mac_images",
            "fhe_ctx_inject_alloc_failure", "fhe_keygen",
            "fhe_sk_free", "fhe_evk_free", "fhe_evk_galois", "fhe_encode", "fhe_pt_free", "fhe_encrypt",
            "fhe_decrypt", "fhe_decode", "fhe_ct_free", "fhe_ct_info", "fhe_ct_export", "fhe_ct_import",
            "fhe_rotate", "fhe_square", "fhe_rescale", "fhe_add", "fhe_mul_plain", "fhe_model_load",
            "fhe_model_free", "fhe_eval_conv", "fhe_eval_quad_act", "fhe_eval_pool_dense", "fhe_infer",
            "fhe_ntt_device", "fhe_evk_export", "fhe_sk_export", "fhe_encode_coeffs",
            "fhe_profile_keyswitch", "fhe_rescale_noalloc", "fhe_infer_profiled", "fhe_pipeline_create", "fhe_pipeline_info",
            "fhe_pipeline_tick", "fhe_pipeline_ticks", "fhe_pipeline_free", "fhe_server_create", "fhe_server_add_model",
            "fhe_sk_import", "fhe_evk_import", "fhe_server_submit", "fhe_server_poll", "fhe_server_pause", "fhe_server_stats", "fhe_server_destroy"]
