"""The input generators: the SoftDist heatmap (the non-learned control of
Sec. V-C) is the row softmax of the negated distances; the kNN recipe's rows
are normalised."""
import numpy as np

from helpers import dmat
from paper_2601_19041_gb300 import synth


def test_softdist_is_the_row_softmax_of_negated_distances():
    pts = np.random.default_rng(4).random((40, 2)).astype(np.float32)
    rowptr, col, val = synth.softdist_heatmap(pts, t_rel=2.0, floor=0.0, k_max=39, dtype=np.float64)
    D = dmat(pts)
    np.fill_diagonal(D, np.inf)
    T = 2.0 * D.min(axis=1).mean()
    ref = np.exp(-D / T)
    ref /= ref.sum(axis=1, keepdims=True)
    H = np.zeros((40, 40))
    for i in range(40):
        cols = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i not in cols
        H[i, cols] = val[rowptr[i]:rowptr[i + 1]]
    assert np.allclose(H, ref, rtol=1e-12, atol=1e-300)
    assert np.allclose(H.sum(axis=1), 1.0, rtol=1e-12)


def test_softdist_truncation_keeps_the_largest_entries():
    pts = np.random.default_rng(5).random((300, 2)).astype(np.float32)
    rowptr, col, val = synth.softdist_heatmap(pts, t_rel=1.0, floor=1e-6, k_max=16)
    D = dmat(pts)
    np.fill_diagonal(D, np.inf)
    for i in (0, 17, 299):
        cols = col[rowptr[i]:rowptr[i + 1]]
        assert 1 <= len(cols) <= 16
        near = np.argsort(D[i], kind="stable")[:len(cols)]
        assert set(cols.tolist()) == set(near.tolist())      # monotone in the distance
        assert np.all(val[rowptr[i]:rowptr[i + 1]] >= 1e-6)


def test_knn_heatmap_rows_are_normalised():
    inst = synth.euclid_instance(6, 200, K=20)
    sums = np.add.reduceat(inst.val.astype(np.float64), inst.rowptr[:-1])
    assert np.allclose(sums, 1.0, rtol=1e-5)
    assert np.all(np.diff(inst.rowptr) == 20)
