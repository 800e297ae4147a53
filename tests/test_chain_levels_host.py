"""The decomposition of the large-set hull's chain phase, checked on the CPU.

The device path sorts the survivors by (x, y) key, with equal keys in no
index order (survivors arrive in compaction order), then chains them in
levels: each chunk keeps the first point of every x column for its lower
chain and the last key of every column for its upper chain (each with the
lowest index among the copies of its key), adds its last key to the lower
list and its first point to the upper list, and chains each list in two
levels (short runs chained separately, then one walk over the run chains'
vertices); later levels concatenate groups of chunk chains and chain them
again, window by window, onto a running stack.  This test replays those
steps in plain Python with small chunk, run, group and window sizes (so
that every boundary case occurs often) and checks the emitted hull against
the oracle's on random and degenerate sets.  It checks the decomposition
argument, not the kernel; the GPU parity tests check the kernel.
"""
import numpy as np
import pytest

import oracle


def cross(o, a, b):
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def chain(entries, sg, stack=None):
    """Monotone chain of (key, index) entries in key order onto `stack`
    (sg = +1 lower: pop unless strictly left; -1 upper), the lowest index
    standing for equal keys."""
    st = [] if stack is None else stack
    for k, v in entries:
        if st and st[-1][0] == k:
            if v < st[-1][1]:
                st[-1] = (k, v)
            continue
        while len(st) >= 2 and sg * cross(st[-2][0], st[-1][0], k) <= 0:
            st.pop()
        st.append((k, v))
    return st


def window_chain(entries, sg, stack, lanes, run_min):
    """Two levels: runs of S entries chained apart, then their vertices
    pushed in order onto the running stack."""
    n = len(entries)
    if n == 0:
        return stack
    S = max(-(-n // lanes), run_min)
    verts = []
    for lo in range(0, n, S):
        verts.extend(chain(entries[lo:lo + S], sg))
    return chain(verts, sg, stack)


def level0(keys, vals, c0, lanes, run_min):
    """Per chunk of c0 sorted elements: its lower and upper chains."""
    lows, ups = [], []
    for tb in range(0, len(keys), c0):
        k = keys[tb:tb + c0]
        v = list(vals[tb:tb + c0])
        tn = len(k)
        # the first slot of every run of equal keys takes the run's lowest index
        e = 0
        while e < tn:
            f = e
            while f + 1 < tn and k[f + 1] == k[e]:
                f += 1
            v[e] = min(v[e:f + 1])
            e = f + 1

        def run_start(i):
            while i > 0 and k[i - 1] == k[i]:
                i -= 1
            return i

        lo_pos = [i for i in range(tn) if i == 0 or k[i - 1][0] != k[i][0]] + [run_start(tn - 1)]
        up_pos = [0] + [run_start(i) for i in range(tn) if i == tn - 1 or k[i + 1][0] != k[i][0]]
        lows.append(window_chain([(k[i], v[i]) for i in lo_pos], 1, [], lanes, run_min))
        ups.append(window_chain([(k[i], v[i]) for i in up_pos], -1, [], lanes, run_min))
    return lows, ups


def merge_levels(chains, sg, fan, window, lanes, run_min):
    while len(chains) > 1:
        nxt = []
        for g in range(0, len(chains), fan):
            cat = [e for c in chains[g:g + fan] for e in c]
            st = []
            for w0 in range(0, len(cat), window):
                window_chain(cat[w0:w0 + window], sg, st, lanes, run_min)
            nxt.append(st)
        chains = nxt
    return chains[0]


def large_path_hull(xy, rng, c0=16, fan=4, window=8, lanes=4, run_min=2):
    xi = np.rint(xy).astype(np.int64)
    keys = [(int(a), int(b)) for a, b in xi]
    order = sorted(range(len(keys)), key=lambda i: keys[i])
    # equal keys in no index order, as the survivors arrive
    i = 0
    while i < len(order):
        j = i
        while j + 1 < len(order) and keys[order[j + 1]] == keys[order[i]]:
            j += 1
        if j > i:
            seg = order[i:j + 1]
            rng.shuffle(seg)
            order[i:j + 1] = seg
        i = j + 1
    sk = [keys[i] for i in order]
    sv = list(order)
    lows, ups = level0(sk, sv, c0, lanes, run_min)
    lower = merge_levels(lows, 1, fan, window, lanes, run_min)
    upper = merge_levels(ups, -1, fan, window, lanes, run_min)
    a, b = len(lower), len(upper)
    if a <= 1:
        return [lower[0][1]]
    # counter-clockwise from the lexicographic minimum: the lower chain
    # without its last point, then the upper chain from its last point back
    # to its second
    return [v for _, v in lower[:a - 1]] + [upper[k][1] for k in range(b - 1, 0, -1)]


def sets():
    rng = np.random.default_rng(20)
    yield "disk", np.round(rng.normal(0, 1, (3000, 2)) * 1000)
    yield "square", rng.integers(-50, 51, (2500, 2)).astype(np.float64)
    yield "tiny_lattice", rng.integers(-3, 4, (600, 2)).astype(np.float64)
    t = rng.integers(-200, 200, 800)
    yield "collinear", np.stack([3 * t, -2 * t], 1).astype(np.float64)
    a = np.arange(500) * (2 * np.pi / 500)
    ring = np.round(np.stack([1e6 * np.cos(a), 1e6 * np.sin(a)], 1))
    yield "ring_repeated", np.concatenate([ring, ring, ring])[rng.permutation(1500)]
    yield "all_equal", np.tile(np.array([[5.0, -2.0]]), (300, 1))
    yield "two_columns", np.stack([rng.integers(0, 2, 900) * 7, rng.integers(-40, 41, 900)], 1).astype(np.float64)
    # several points in the first and in the last column, the last column
    # starting exactly at a chunk boundary (16 points before it): the chunk
    # end points the chains must add
    first = np.stack([np.full(4, -10), np.arange(4) * 3], 1)
    mid = np.stack([rng.integers(-9, 10, 12), rng.integers(-20, 21, 12)], 1)
    last = np.stack([np.full(5, 10), np.arange(5) * 2 - 4], 1)
    yield "end_columns", np.concatenate([first, mid, last]).astype(np.float64)


@pytest.mark.parametrize("name,xy", list(sets()), ids=lambda v: v if isinstance(v, str) else "")
@pytest.mark.parametrize("sizes", [dict(), dict(c0=8, fan=2, window=4, lanes=2, run_min=1),
                                   dict(c0=64, fan=8, window=32, lanes=8, run_min=8)])
def test_chunked_two_level_chains_give_the_hull(name, xy, sizes):
    rng = np.random.default_rng(7)
    xy = np.asarray(xy, np.float32)
    got = large_path_hull(xy, rng, **sizes)
    assert got == oracle.hull(xy).tolist()
