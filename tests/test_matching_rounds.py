"""The merger's pair selection on the GPU takes, in rounds, every pair that
is the smallest still-free pair at both of its ends.  For a strict order of
the pairs this equals the sequential greedy matching (ascending (chi2, a, b),
each end used once) that the merge step defines.  Checked here on random
bipartite pair sets with many ties in chi2, by emulating the rounds in
Python against the sequential pass."""
import numpy as np


def greedy(pairs):
    nxt, prv = {}, {}
    for c, a, b in sorted(pairs):
        if a in nxt or b in prv:
            continue
        nxt[a], prv[b] = b, a
    return nxt


def rounds(pairs):
    nxt, prv = {}, {}
    n_rounds = 0
    while True:
        free = [(c, a, b) for c, a, b in pairs if a not in nxt and b not in prv]
        if not free:
            return nxt, n_rounds
        n_rounds += 1
        min_a, min_b = {}, {}
        for c, a, b in free:  # keys: (chi2, b) at end a, (chi2, a) at end b
            min_a[a] = min(min_a.get(a, (np.inf, 0)), (c, b))
            min_b[b] = min(min_b.get(b, (np.inf, 0)), (c, a))
        for c, a, b in free:
            if min_a[a] == (c, b) and min_b[b] == (c, a):
                nxt[a], prv[b] = b, a


def test_rounds_equal_sequential_greedy():
    rng = np.random.default_rng(7)
    for trial in range(300):
        na, nb = rng.integers(1, 30, 2)
        m = int(rng.integers(0, 120))
        cand = {(int(rng.integers(na)), int(rng.integers(nb))) for _ in range(m)}
        # coarse chi2 values: many exact ties, broken by (a, b)
        pairs = [(float(rng.integers(0, 6)) * 0.5, a, b) for a, b in cand]
        got, n_rounds = rounds(pairs)
        assert got == greedy(pairs)
        assert n_rounds <= max(1, len(pairs))
