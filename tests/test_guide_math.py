"""The arithmetic of guided ITS (CPU only), restated in exact integers: the
draw-space bounds U_j, the first candidates of the d draw cells written edge
by edge, and the bounded search give, for every draw (random ones and every
cell boundary), the ITS answer of Section 2.3 -- the smallest i with
x < p'_i, x = floor(r64 * S / 2^64).  The device kernels build and search the
same tables; the GPU tests compare their records and walks with this and with
the oracle."""
import random

M = 1 << 64


def its_answer(P, r64):
    x = r64 * P[-1] >> 64
    return next(i for i, p in enumerate(P) if x < p)


def build(W):
    d = len(W)
    P, acc = [], 0
    for w in W:
        acc += w
        P.append(acc)
    S = acc
    U = [0 if p == 0 else ((p << 64) - 1) // S for p in P]
    first, last = [-1] * d, [-1] * d
    for j in range(d):
        if U[j] == 0:
            continue
        Up = 0 if j == 0 else U[j - 1]
        k0 = 0 if Up == 0 else (Up * d >> 64) + 1
        k1 = U[j] * d >> 64
        for k in range(k0, k1 + 1):
            first[k] = j
            if k >= 1:
                last[k - 1] = j
    last[d - 1] = d - 1
    return P, U, first, last


def guided(U, first, last, r64, d):
    r = max(r64, 1)
    k = r64 * d >> 64
    a, hi = first[k], last[k]
    assert 0 <= a <= hi < d
    if r <= U[a]:
        return a
    n, a = hi - a - 1, a + 1
    while n > 0:
        half = n >> 1
        if U[a + half] < r:
            a, n = a + half + 1, n - half - 1
        else:
            n = half
    return a


def test_guided_search_is_its():
    rng = random.Random(3)
    rows = [[1], [0, 5], [5, 0], [0, 0, 7, 0], [2 ** 32 - 1, 1, 2 ** 32 - 1], [1] * 50, list(range(1, 40))]
    for _ in range(1500):
        d = rng.randint(1, 40)
        rows.append([rng.choice([0, 0, 1, 2, 3, 65536, 2 ** 32 - 1, rng.randint(1, 10 ** 6)]) for _ in range(d)])
    for W in rows:
        if sum(W) == 0:
            continue
        P, U, first, last = build(W)
        d = len(W)
        assert all(f >= 0 for f in first) and U[-1] == M - 1
        draws = [0, 1, M - 1, M // 2] + [rng.randrange(M) for _ in range(64)]
        for k in range(d):
            b = -(-k * M // d)  # the smallest draw of cell k
            draws += [b, max(b - 1, 0), min(b + 1, M - 1)]
        for r in draws:
            assert guided(U, first, last, r, d) == its_answer(P, r), (W, r)


def test_zero_weight_edges_are_never_first():
    P, U, first, last = build([0, 0, 3, 0, 5, 0])
    assert set(first) <= {2, 4}
    assert first[0] == 2  # the draw 0 takes the first positive edge
