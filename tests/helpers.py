"""Small instance builders shared by the tests (no decoder arithmetic here)."""
import itertools
import math

import numpy as np

from paper_2601_19041_gb300.synth import Instance, Params


def csr_from_dense(Hd, dtype=np.float32):
    Hd = np.asarray(Hd, np.float64)
    n = Hd.shape[0]
    rowptr = [0]
    col, val = [], []
    for i in range(n):
        js = [j for j in range(n) if j != i and Hd[i, j] != 0.0]
        col += js
        val += [Hd[i, j] for j in js]
        rowptr.append(len(col))
    return (np.asarray(rowptr, np.int32), np.asarray(col, np.int32),
            np.asarray(val, dtype))


def euclid(coords, Hd=None, symmetrize=1, dtype=np.float32):
    coords = np.asarray(coords, np.float32)
    n = len(coords)
    if Hd is None:
        Hd = np.zeros((n, n))
    rp, c, v = csr_from_dense(Hd, dtype)
    return Instance(n=n, kind=0, coords=coords, cost=None, rowptr=rp, col=c, val=v,
                    symmetrize=symmetrize)


def atsp(cost, Hd=None):
    cost = np.asarray(cost, np.float32)
    n = cost.shape[0]
    if Hd is None:
        Hd = np.zeros((n, n))
    rp, c, v = csr_from_dense(Hd)
    return Instance(n=n, kind=1, coords=None, cost=cost, rowptr=rp, col=c, val=v, symmetrize=0)


def dmat(coords):
    p = np.asarray(coords, np.float32).astype(np.float64)
    dx = p[None, :, 0] - p[:, None, 0]
    dy = p[None, :, 1] - p[:, None, 1]
    return np.sqrt(dx * dx + dy * dy)


def tour_len(D, tour):
    L = 0.0
    for s in range(1, len(tour)):
        L += D[tour[s - 1], tour[s]]
    return L + D[tour[-1], tour[0]]


def strided_partials_len(D, tour):
    """The decoder's tour-length order, restated: edge e into partial e mod 32
    (sequential within a partial), then a pairwise tree over the 32 partials."""
    n = len(tour)
    P = [0.0] * 32
    for e in range(n):
        P[e % 32] = P[e % 32] + float(D[tour[e], tour[(e + 1) % n]])
    w = 1
    while w < 32:
        for q in range(0, 32, 2 * w):
            P[q] = P[q] + P[q + w]
        w *= 2
    return P[0]


def brute_force_opt(D):
    """Exact optimum by enumerating (n-1)!/2 cycles (node 0 fixed)."""
    n = D.shape[0]
    best, arg = math.inf, None
    for perm in itertools.permutations(range(1, n)):
        if perm[0] > perm[-1]:
            continue
        t = (0,) + perm
        L = tour_len(D, t)
        if L < best:
            best, arg = L, t
    return best, list(arg)


def cycle_heat(n, tour, value=1.0):
    H = np.zeros((n, n))
    for s in range(n):
        u, v = tour[s], tour[(s + 1) % n]
        H[u, v] = value
        H[v, u] = value
    return H


def is_perm(t, n):
    return sorted(int(x) for x in t) == list(range(n))


def params(**kw):
    return Params(**kw)
