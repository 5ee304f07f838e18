"""The arithmetic behind inline records (every substring one 32-bit word,
m = q/32): a candidate reached by table j at ring rho differs from the query
in exactly rho bits of word j, so its distance is rho plus the popcounts of
the other words, and "first discovered at step m*rho + j" (reading c8) is
"every other word i of the record has at least rho + [i < j] differing
bits".  Checked here by brute force on random words, independently of the
kernels."""
import numpy as np
import pytest


def popc(x):
    return bin(int(x)).count("1")


@pytest.mark.parametrize("nw", [2, 4, 8])
def test_record_distance_and_first_discovery(nw):
    rng = np.random.default_rng(nw)
    m = nw
    for _ in range(3000):
        g = rng.integers(0, 2**32, size=nw, dtype=np.uint64)
        # a code near the query: each word gets a few flipped bits
        flips = rng.integers(0, 4, size=nw)
        c = g.copy()
        for w in range(nw):
            for b in rng.choice(32, size=flips[w], replace=False):
                c[w] ^= np.uint64(1 << int(b))
        d_words = [popc(c[w] ^ g[w]) for w in range(nw)]
        d = sum(d_words)
        first_step = min(m * d_words[jj] + jj for jj in range(m))
        for j in range(m):
            rho = d_words[j]          # the ring at which table j reaches this code
            rec = [c[i] for i in range(nw) if i != j]
            gq = [g[i] for i in range(nw) if i != j]
            pc = [popc(r ^ q) for r, q in zip(rec, gq)]
            assert rho + sum(pc) == d
            th = [rho + (1 if i < j else 0) for i in range(nw - 1)]
            keep = all(p >= t for p, t in zip(pc, th))
            assert keep == (first_step == m * rho + j), (d_words, j)
