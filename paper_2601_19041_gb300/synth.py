"""Seeded synthetic TSP / ATSP instances and heatmaps.

This module only draws inputs: point sets, cost matrices and sparse
edge-confidence heatmaps in CSR form. It holds none of the decoder's
arithmetic, so both the CUDA library and the CPU oracle can consume its
output without sharing any decoding code.

The heatmaps stand in for the learned heatmaps of Sec. IV-A (AttGCN, DIMES,
UTSP, DIFUSCO on the ML4CO-Bench-101 suites), which are not available here.
The recipe mimics their structure: mass concentrated on the nearest
neighbours of each node, with multiplicative noise, row-normalised.

    w_ij = exp(-d_ij / dbar) * LogNormal(0, 0.5)   for j in kNN(i)
    H_ij = w_ij / sum_j w_ij                         (zero elsewhere)

dbar is the mean of the n*K neighbour distances of the instance. The
symmetrisation (H + H^T)/2 of Sec. II-B is left to the decoder
(``symmetrize=1``), so that it runs inside the library.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# the five synthetic workloads: symmetric n=500; batched n~U{500..2000};
# large n=10000 with 2-opt; ATSP n=1000; a serving stream of mixed sizes.
# Paper-setting runs (Sec. IV-D parameters: m=32, k=20, I=5000, rho=0.8, the
# MMAS schedule) on 128 instances of n=500 or n=1000, without local search
# and with 2-opt on every ant, for comparison with the paper's decode times.
WORKLOADS = ("tsp500", "batch128", "tsp10k_2opt", "atsp1000", "serve",
             "paper_tsp500", "paper_tsp500_2opt", "paper_tsp1k")


@dataclass
class Instance:
    """One decode problem: geometry (or costs) plus a CSR heatmap."""
    n: int
    kind: int                      # 0 = Euclidean from coords, 1 = explicit cost matrix
    coords: np.ndarray | None      # (n, 2) float32
    cost: np.ndarray | None        # (n, n) float32, row-major c_ij
    rowptr: np.ndarray             # (n+1,) int32
    col: np.ndarray                # (nnz,) int32, strictly increasing per row
    val: np.ndarray                # (nnz,) float32 or float16
    symmetrize: int = 1
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def h_dtype(self) -> int:
        return 1 if self.val.dtype == np.float16 else 0


@dataclass
class Params:
    """Decoder parameters; defaults follow Sec. IV-D except where a workload overrides."""
    m: int = 32
    k: int = 20
    iterations: int = 5000
    alpha: float = 1.0
    beta: float = 2.0
    rho: float = 0.8
    theta_h: float = 1e-4
    eps: float = 1e-9
    c_cap: float = 0.5
    q_level: float = 0.90
    p_best: float = 0.05
    logw_clip: float = 30.0
    degree_target: int = 2
    local_search: int = 0
    baseline_scope: int = 0
    ls_k: int = 20
    seed: int = 0
    schedule: int = 0                 # 1: MMAS u_gb schedule and restarts (Sec. III-B)
    kappa_mode: int = 0               # 0: eq. kappa; 1: fixed kappa = 1; 2: no cap factor (Sec. V-D)


# ----------------------------------------------------------------------------- points

def uniform_points(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.random((n, 2)).astype(np.float32)


def gaussian_mixture_points(rng: np.random.Generator, n: int, comps: int = 8,
                            sigma: float = 0.05) -> np.ndarray:
    centres = rng.random((comps, 2))
    which = rng.integers(0, comps, size=n)
    pts = centres[which] + sigma * rng.standard_normal((n, 2))
    return pts.astype(np.float32)


def perturbed_grid_points(rng: np.random.Generator, n: int, jitter: float = 0.1) -> np.ndarray:
    side = int(math.ceil(math.sqrt(n)))
    s = 1.0 / side
    gx, gy = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    lattice = np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.float64) * s
    order = rng.permutation(side * side)[:n]
    pts = lattice[order] + rng.uniform(-jitter * s, jitter * s, size=(n, 2))
    return pts.astype(np.float32)


# ----------------------------------------------------------------------------- kNN

def _knn_rows(dist_rows: np.ndarray, row_ids: np.ndarray, K: int):
    """K smallest of each row (self excluded), ties broken by column index."""
    d = dist_rows.copy()
    d[np.arange(len(row_ids)), row_ids] = np.inf
    part = np.argpartition(d, K - 1, axis=1)[:, :K]
    pd = np.take_along_axis(d, part, axis=1)
    o = np.lexsort((part, pd), axis=1)
    return np.take_along_axis(part, o, axis=1), np.take_along_axis(pd, o, axis=1)


def knn_euclid(pts: np.ndarray, K: int, chunk: int = 1024):
    p = pts.astype(np.float64)
    n = len(p)
    K = min(K, n - 1)
    idx = np.empty((n, K), np.int64)
    dd = np.empty((n, K), np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        dx = p[s:e, 0:1] - p[None, :, 0]
        dy = p[s:e, 1:2] - p[None, :, 1]
        d = np.sqrt(dx * dx + dy * dy)
        idx[s:e], dd[s:e] = _knn_rows(d, np.arange(s, e), K)
    return idx, dd


def knn_cost(cost: np.ndarray, K: int):
    n = cost.shape[0]
    K = min(K, n - 1)
    return _knn_rows(cost.astype(np.float64), np.arange(n), K)


def knn_heatmap(rng: np.random.Generator, nbr: np.ndarray, nd: np.ndarray,
                dtype=np.float32):
    """Row-normalised exp(-d/dbar)*LogNormal(0,0.5) weights on the kNN pattern, as CSR."""
    n, K = nbr.shape
    dbar = float(nd.mean()) if nd.size else 1.0
    noise = rng.lognormal(mean=0.0, sigma=0.5, size=(n, K))
    w = np.exp(-nd / max(dbar, 1e-12)) * noise
    w /= w.sum(axis=1, keepdims=True)
    order = np.argsort(nbr, axis=1, kind="stable")
    col = np.take_along_axis(nbr, order, axis=1).astype(np.int32)
    val = np.take_along_axis(w, order, axis=1).astype(dtype)
    rowptr = (np.arange(n + 1, dtype=np.int64) * K).astype(np.int32)
    return rowptr, col.ravel(), val.ravel()


# ----------------------------------------------------------------------------- instances

def euclid_instance(seed: int, n: int, K: int = 50, family: str = "uniform",
                    dtype=np.float32, symmetrize: int = 1) -> Instance:
    rng = np.random.default_rng(seed)
    if family == "uniform":
        pts = uniform_points(rng, n)
    elif family == "gmm":
        pts = gaussian_mixture_points(rng, n)
    elif family == "grid":
        pts = perturbed_grid_points(rng, n)
    else:
        raise ValueError(family)
    nbr, nd = knn_euclid(pts, K)
    rowptr, col, val = knn_heatmap(rng, nbr, nd, dtype)
    return Instance(n=n, kind=0, coords=pts, cost=None, rowptr=rowptr, col=col, val=val,
                    symmetrize=symmetrize, seed=seed, meta={"family": family, "knn": K})


def atsp_instance(seed: int, n: int, K: int = 50, noise_hi: float = 0.5) -> Instance:
    rng = np.random.default_rng(seed)
    p = rng.random((n, 2)).astype(np.float64)
    dx = p[:, None, 0] - p[None, :, 0]
    dy = p[:, None, 1] - p[None, :, 1]
    c = np.sqrt(dx * dx + dy * dy) + rng.uniform(0.0, noise_hi, size=(n, n))
    np.fill_diagonal(c, 0.0)
    cost = c.astype(np.float32)
    nbr, nd = knn_cost(cost, K)
    rowptr, col, val = knn_heatmap(rng, nbr, nd, np.float32)
    return Instance(n=n, kind=1, coords=None, cost=cost, rowptr=rowptr, col=col, val=val,
                    symmetrize=0, seed=seed, meta={"family": "atsp", "knn": K})


def softdist_heatmap(pts: np.ndarray, t_rel: float = 1.0, floor: float = 1e-6, k_max: int = 64,
                     dtype=np.float32, chunk: int = 1024):
    """SoftDist heatmap (the non-learned control of Sec. V-C): row i is the
    softmax of the negated distances, H_ij = exp(-d_ij/T) / sum_{l != i}
    exp(-d_il/T), over all j != i.  The paper does not state the temperature;
    here T = t_rel times the instance's mean nearest-neighbour distance, a
    documented parameter.  Entries below ``floor`` (far under the decoder's
    threshold theta_h = 1e-4) are not stored, and at most the ``k_max``
    largest of a row are kept.  Returns CSR (rowptr, col, val)."""
    p = pts.astype(np.float64)
    n = len(p)
    nn, nd = knn_euclid(pts, 1)
    T = max(t_rel * float(nd.mean()), 1e-300)
    K = min(k_max, n - 1)
    rows_c, rows_v = [], []
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        dx = p[s:e, 0:1] - p[None, :, 0]
        dy = p[s:e, 1:2] - p[None, :, 1]
        d = np.sqrt(dx * dx + dy * dy)
        d[np.arange(e - s), np.arange(s, e)] = np.inf          # j != i
        z = -(d - d.min(axis=1, keepdims=True)) / T             # shifted for a stable softmax
        w = np.exp(z)
        w /= w.sum(axis=1, keepdims=True)
        top = np.argpartition(-w, K - 1, axis=1)[:, :K]
        for r in range(e - s):
            js = top[r][w[r, top[r]] >= floor]
            js.sort()
            rows_c.append(js.astype(np.int32))
            rows_v.append(w[r, js].astype(dtype))
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum([len(c) for c in rows_c])
    return (rowptr.astype(np.int32), np.concatenate(rows_c) if rows_c else np.zeros(0, np.int32),
            np.concatenate(rows_v) if rows_v else np.zeros(0, dtype))


def softdist_instance(seed: int, n: int, t_rel: float = 1.0, family: str = "uniform",
                      symmetrize: int = 1) -> Instance:
    """Uniform (or other family) points with a SoftDist heatmap."""
    rng = np.random.default_rng(seed)
    pts = {"uniform": uniform_points, "gmm": gaussian_mixture_points,
           "grid": perturbed_grid_points}[family](rng, n)
    rowptr, col, val = softdist_heatmap(pts, t_rel)
    return Instance(n=n, kind=0, coords=pts, cost=None, rowptr=rowptr, col=col, val=val,
                    symmetrize=symmetrize, seed=seed, meta={"family": family, "heatmap": "softdist",
                                                            "t_rel": t_rel})


def empty_heatmap(n: int):
    return np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32)


# ----------------------------------------------------------------------------- workloads

def workload(name: str, count: int | None = None, base_seed: int | None = None):
    """(instances, params-per-instance) for one of WORKLOADS.

    ``count`` truncates a multi-instance workload (the first ``count`` instances
    are identical to the full workload's first ones).
    """
    if name == "tsp500":
        inst = [euclid_instance(0, 500, K=50)]
        ps = [Params(m=50, k=20, iterations=100, rho=0.2, seed=0)]
        return inst, ps
    if name == "batch128":
        total = 128
        ns = np.random.default_rng(1).integers(500, 2001, size=total)
        cnt = total if count is None else count
        b0 = 1000 if base_seed is None else base_seed
        inst = [euclid_instance(b0 + b, int(ns[b]), K=50) for b in range(cnt)]
        ps = [Params(m=64, k=20, iterations=200, rho=0.2, seed=b0 + b) for b in range(cnt)]
        return inst, ps
    if name == "tsp10k_2opt":
        cnt = 16 if count is None else count
        b0 = 2000 if base_seed is None else base_seed
        inst = [euclid_instance(b0 + b, 10000, K=10) for b in range(cnt)]
        ps = [Params(m=64, k=10, iterations=300, rho=0.2, local_search=1, seed=b0 + b)
              for b in range(cnt)]
        return inst, ps
    if name == "atsp1000":
        cnt = 64 if count is None else count
        b0 = 3000 if base_seed is None else base_seed
        inst = [atsp_instance(b0 + b, 1000, K=50) for b in range(cnt)]
        ps = [Params(m=50, k=20, iterations=200, rho=0.2, degree_target=1, seed=b0 + b)
              for b in range(cnt)]
        return inst, ps
    if name in ("paper_tsp500", "paper_tsp500_2opt", "paper_tsp1k"):
        cnt = 128 if count is None else count
        n = 1000 if name == "paper_tsp1k" else 500
        b0 = (6000 if n == 1000 else 5000) if base_seed is None else base_seed
        ls = 2 if name.endswith("2opt") else 0
        inst = [euclid_instance(b0 + b, n, K=50) for b in range(cnt)]
        ps = [Params(m=32, k=20, iterations=5000, rho=0.8, local_search=ls, ls_k=20, schedule=1, seed=b0 + b)
              for b in range(cnt)]
        return inst, ps
    raise ValueError(name)


@dataclass
class Request:
    arrival: float
    inst: Instance
    params: Params


def serving_stream(num: int = 2000, rate: float = 200.0, seed: int = 4,
                   sizes=(500, 1000, 2000, 5000, 10000), iters=(100, 300)):
    """Poisson arrivals of mixed-size decode requests with FP16 heatmaps."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=num))
    fams = ("uniform", "gmm", "grid")
    out = []
    for r in range(num):
        n = int(sizes[rng.integers(0, len(sizes))])
        fam = fams[rng.integers(0, 3)]
        it = int(rng.integers(iters[0], iters[1] + 1))
        s = 40000 + r
        inst = euclid_instance(s, n, K=50, family=fam, dtype=np.float16)
        out.append(Request(float(t[r]), inst, Params(m=64, k=20, iterations=it, rho=0.2, seed=s)))
    return out
