"""The prime chains printed in the paper's appendix on FHE parameters
(tests/golden/paper_primes.txt), parsed.  Each line prints q_1..q_L first
and the small output prime q_0 last (the moduli are q_0..q_L, then P)."""
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rows():
    out = []
    for line in open(os.path.join(GOLDEN, "paper_primes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, qs, p = [x.strip() for x in line.split("|")]
        name, logn, d, L, lq, lp = head.split()
        out.append((name, int(logn), int(d), int(L), int(lq), int(lp), [int(x, 16) for x in qs.split()], int(p, 16)))
    return out


def chain(name):
    """(log N, log2 Delta, [q_0, q_1, .., q_L], [P]) of one model's chain"""
    for r in rows():
        if r[0] == name:
            qs = r[6]
            return r[1], r[2], [qs[-1]] + qs[:-1], [r[7]]
    raise KeyError(name)
