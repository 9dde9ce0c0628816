"""CPU oracle for leveled RNS-CKKS CNN inference (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked
against.  It is used by the tests, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``; the product library never imports, links or
calls it, and it imports nothing from the product package.

Layout:
  ckks_ref.c  -- modular arithmetic, textbook NTT, fast basis conversion,
                 ChaCha20 (RFC 8439), the slot encoder (C, compiled by build.py)
  ckks.py     -- parameters, keys, encryption, key switching, rotation,
                 relinearisation, rescale (Sec. 2.2 of the paper), in the
                 algorithm's own order, on top of ckks_ref.c
  planner.py  -- level accounting of Table 1 and the tower-reuse rule (Sec. 4.3)
  cnn.py      -- float64 plaintext network and the homomorphic CNN layers
                 (Sec. 4.1-4.2 transforms, Sec. 5.1 slot layouts)
"""
