"""The FP32 decision rule of the GPU 2-opt is sound.

The kernel decides most candidate moves from FP32 copies of the distances
and falls back to FP64 only inside an error band (Sec. III-D's 2-opt with the
FP64 gain; the band is this implementation's).  This test restates that rule
with numpy float32 operations (IEEE, each rounded once, as the kernel's _rn
intrinsics) and checks, on millions of candidate moves, that

  * each FP32 distance is within 4 units of 2^-24 (relative) of the FP64 one,
  * "certainly not improving" never meets an FP64 gain above 1e-10,
  * "certainly improving" never meets an FP64 gain at or below 1e-10,
  * the d(a, b) < d(a, dir a) margin is certain in both directions,

on point sets chosen to stress it: uniform, exact grids (many gains exactly
zero), tiny scales (gains near the 1e-10 threshold), large scales, clusters of
near-duplicates and exact duplicates.
"""
import numpy as np
import pytest

LS_GAIN = 1e-10
G1_LO = np.float32(0.999996)
F = np.float32


def d64(p, q):
    dx = q[:, 0].astype(np.float64) - p[:, 0].astype(np.float64)
    dy = q[:, 1].astype(np.float64) - p[:, 1].astype(np.float64)
    return np.sqrt(dx * dx + dy * dy)


def d32(p, q):
    dx = q[:, 0] - p[:, 0]
    dy = q[:, 1] - p[:, 1]
    return np.sqrt(dx * dx + dy * dy)


def gain_class(da, dab, dbb, dn):
    # 0: FP64 gain certainly <= LS_GAIN, 2: certainly above, 1: undecided
    est = ((da - dab) + dbb) - dn
    mag = (da + dab) + (dbb + dn)
    tol = F(4e-6) * mag + F(1e-18)
    lo = F(LS_GAIN) - tol
    hi = F(LS_GAIN) + tol
    return np.where(~(est > lo), 0, np.where(est > hi, 2, 1))


def point_sets():
    rng = np.random.default_rng(2601)
    g = np.stack(np.meshgrid(np.arange(24), np.arange(24)), -1).reshape(-1, 2)
    base = rng.random((400, 2))
    yield "uniform", rng.random((3000, 2)).astype(np.float32)
    yield "grid", (g / 16.0).astype(np.float32)
    yield "grid_offset", (g / 64.0 + 0.37).astype(np.float32)
    yield "tiny", (rng.random((3000, 2)) * 1e-5).astype(np.float32)
    yield "tiny_offset", (0.5 + rng.random((3000, 2)) * 2e-4).astype(np.float32)
    yield "large", (rng.random((3000, 2)) * 1e4).astype(np.float32)
    # the largest coordinates accepted with local search (|x|, |y| <= 1e18):
    # FP32 squared differences stay finite
    yield "huge", ((rng.random((3000, 2)) * 2.0 - 1.0) * 1e18).astype(np.float32)
    yield "near_dup", (np.repeat(base, 4, axis=0) + rng.normal(0, 1e-7, (1600, 2))).astype(np.float32)
    yield "dup", np.repeat(base, 3, axis=0).astype(np.float32)


@pytest.mark.parametrize("name,pts", list(point_sets()), ids=[n for n, _ in point_sets()])
def test_fp32_classes_never_contradict_fp64(name, pts):
    rng = np.random.default_rng(7)
    m = 1_000_000
    ia, ian, ib, ibn = (rng.integers(0, len(pts), m) for _ in range(4))
    a, an, b, bn = pts[ia], pts[ian], pts[ib], pts[ibn]
    Da, Dab, Dbb, Dn = d64(a, an), d64(a, b), d64(b, bn), d64(an, bn)
    gain = ((Da - Dab) + Dbb) - Dn

    # FP32 distances: computed in FP32, or FP64 rounded once (both kinds are stored)
    with np.errstate(over="raise"):
        for x in (d32(a, an), d32(an, bn), Dab.astype(np.float32)):
            assert np.all(np.isfinite(x)), name
    for x32, x64 in ((d32(a, an), Da), (d32(an, bn), Dn), (Dab.astype(np.float32), Dab)):
        ok = x64 > 1e-30
        rel = np.abs(x32[ok].astype(np.float64) - x64[ok]) / x64[ok]
        assert rel.max() <= 4 * 2.0 ** -24, (name, rel.max())

    # the edge lengths el[] may hold either kind: try both for the two tour edges
    for da, dbb in ((d32(a, an), d32(b, bn)), (Da.astype(np.float32), Dbb.astype(np.float32))):
        dab, dn = Dab.astype(np.float32), d32(an, bn)
        c = gain_class(da, dab, dbb, dn)
        assert not np.any((c == 0) & (gain > LS_GAIN)), name
        assert not np.any((c == 2) & ~(gain > LS_GAIN)), name
        # the certain-accept path also needs d(a, b) < d(a, dir a) for certain
        sure_g1 = (da * G1_LO) > dab
        maybe_g1 = da > (dab * G1_LO)
        assert not np.any(sure_g1 & ~(Da > Dab)), name
        assert not np.any(~maybe_g1 & (Da > Dab)), name
        if name in ("grid", "grid_offset", "dup"):
            # exact ties: zero gains must stay undecided (or certainly not
            # improving), and the set must contain many of them
            zero = gain == 0.0
            assert zero.sum() > 1000
            assert not np.any(c[zero] == 2)


def test_band_is_narrow():
    # on generic inputs the FP32 classes decide almost every candidate, which is
    # what makes the FP64 fallback rare
    rng = np.random.default_rng(11)
    pts = rng.random((5000, 2)).astype(np.float32)
    m = 1_000_000
    idx = rng.integers(0, 5000, (4, m))
    # four distinct cities, as in a real move (the kernel skips b = dir a and dir b = a)
    keep = np.ones(m, bool)
    for i in range(4):
        for j in range(i + 1, 4):
            keep &= idx[i] != idx[j]
    a, an, b, bn = (pts[i[keep]] for i in idx)
    c = gain_class(d32(a, an), d64(a, b).astype(np.float32), d32(b, bn), d32(an, bn))
    assert np.mean(c == 1) < 1e-4


def test_local_search_rejects_coordinates_beyond_the_fp32_range(orc):
    """Above |x| = 1e18 the FP32 squared differences of the pre-test could
    overflow, so the decoder refuses such instances when it runs 2-opt (and
    accepts them without local search)."""
    from helpers import euclid, params
    pts = np.random.default_rng(3).random((12, 2)).astype(np.float32)
    ok = orc.Oracle(euclid(pts * np.float32(1e18)), params(m=2, k=4, iterations=1, rho=0.2, local_search=1, ls_k=5))
    assert ok.n == 12
    big = pts.copy()
    big[3, 1] = np.float32(3e18)
    with pytest.raises(ValueError):
        orc.Oracle(euclid(big), params(m=2, k=4, iterations=1, rho=0.2, local_search=1, ls_k=5))
    orc.Oracle(euclid(big), params(m=2, k=4, iterations=1, rho=0.2))
