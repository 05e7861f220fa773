"""Seeded synthetic workloads for graph segmentation.

This module only builds *inputs*: a symmetric weighted adjacency matrix W in
CSR form (no self loops), the fidelity labels (-1 = unlabelled) and the ground
truth used for accuracy reports.  It holds none of the segmentation method's
arithmetic (no degrees, no Laplacian, no energy): both the CUDA path and the
FP64 oracle consume the same `Graph` objects.

The three families stand in for the paper's workloads (Sec. 5.1, Tables 1-2),
whose datasets are not available here:

* `blobs_knn`  -- K isotropic Gaussian blobs, symmetrised k-NN graph with the
                  self-tuning weights exp(-d^2/(sigma_i sigma_j)); stands in for
                  the paper's smaller networks (LFR, Amazon, LastFM).
* `sbm`        -- stochastic block model with unit weights; stands in for the
                  paper's large networks (LFR 100k, Twitch).
* `voronoi_image` -- noisy piecewise-constant colour image with an
                  8-neighbour pixel graph, weights exp(-||c_i-c_j||^2/s); stands
                  in for the paper's colour-segmentation images (Table 2),
                  with a sparse graph in place of the paper's NFFT dense one.

Every generator is deterministic given its seed (numpy PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = ["Graph", "blobs_knn", "sbm", "voronoi_image", "pick_labels",
           "batched_blobs", "from_edges"]


@dataclasses.dataclass
class Graph:
    """A segmentation input: symmetric W (CSR, int32 indices, float64 weights)."""
    n: int
    row_ptr: np.ndarray          # int32[n+1]
    col: np.ndarray              # int32[nnz], sorted within each row
    w: np.ndarray                # float64[nnz], w_ij = w_ji > 0
    K: int
    labels: np.ndarray           # int32[n], class in [0,K) or -1
    truth: np.ndarray            # int32[n], ground-truth class
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def from_edges(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray) -> tuple:
    """CSR of the symmetric matrix with entries (i,j,w) and (j,i,w).

    Duplicate (i,j) pairs are merged keeping the first weight; self loops are
    dropped.  Returns (row_ptr int32, col int32, w float64) with columns sorted.
    """
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    keep = i != j
    i, j, w = i[keep], j[keep], w[keep]
    # merge undirected duplicates on the canonical (min, max) pair first, so
    # (i,j) and (j,i) always carry the same weight
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    ukey, first = np.unique(lo * n + hi, return_index=True)
    lo, hi, w = ukey // n, ukey % n, w[first]
    ii = np.concatenate([lo, hi])
    jj = np.concatenate([hi, lo])
    ww = np.concatenate([w, w])
    key = ii * n + jj
    order = np.argsort(key, kind="stable")
    key = key[order]
    ww = ww[order]
    rows = key // n
    cols = key % n
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr.astype(np.int32), cols.astype(np.int32), ww


def pick_labels(truth: np.ndarray, K: int, rng: np.random.Generator,
                frac: Optional[float] = None, per_class: Optional[int] = None,
                total_frac: Optional[float] = None) -> np.ndarray:
    """Fidelity labels: a uniformly random subset of nodes keeps its class.

    `frac` labels round(frac*|class|) (>=1) nodes of every class; `per_class`
    labels exactly that many per class; `total_frac` labels round(frac*n)
    nodes drawn from all nodes, then adds one node of any class left without.
    """
    n = truth.shape[0]
    labels = np.full(n, -1, dtype=np.int32)
    if total_frac is not None:
        m = max(1, int(round(total_frac * n)))
        pick = rng.choice(n, size=m, replace=False)
        labels[pick] = truth[pick]
        for c in range(K):
            if not np.any(labels == c):
                members = np.flatnonzero(truth == c)
                if members.size:
                    v = members[rng.integers(members.size)]
                    labels[v] = c
        return labels
    for c in range(K):
        members = np.flatnonzero(truth == c)
        if per_class is not None:
            m = min(per_class, members.size)
        else:
            m = max(1, int(round(frac * members.size)))
        pick = rng.choice(members, size=m, replace=False)
        labels[pick] = c
    return labels


def _knn(X: np.ndarray, k: int, device: Optional[str]):
    """Exact k nearest neighbours (self excluded) by brute force.

    Selection runs in float32 (torch, chunked) when `device` is given, else in
    float64 numpy; the returned squared distances are recomputed in float64.
    """
    n = X.shape[0]
    if device is None:
        sq = np.einsum("ij,ij->i", X, X)
        idx = np.empty((n, k), dtype=np.int64)
        chunk = max(1, min(n, (1 << 25) // max(n, 1)))
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            d2 = sq[a:b, None] + sq[None, :] - 2.0 * (X[a:b] @ X.T)
            d2[np.arange(b - a), np.arange(a, b)] = np.inf
            part = np.argpartition(d2, k, axis=1)[:, :k]
            pd = np.take_along_axis(d2, part, axis=1)
            order = np.argsort(pd, axis=1, kind="stable")
            idx[a:b] = np.take_along_axis(part, order, axis=1)
    else:
        import torch
        Xt = torch.as_tensor(X, dtype=torch.float32, device=device)
        sq = (Xt * Xt).sum(1)
        idx = np.empty((n, k), dtype=np.int64)
        chunk = max(1, min(n, (1 << 27) // max(n, 1)))
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            d2 = sq[a:b, None] + sq[None, :] - 2.0 * (Xt[a:b] @ Xt.T)
            ar = torch.arange(b - a, device=device)
            d2[ar, ar + a] = float("inf")
            _, top = torch.topk(d2, k, dim=1, largest=False, sorted=True)
            idx[a:b] = top.cpu().numpy()
    diff = X[:, None, :] - X[idx]
    d2 = np.einsum("ijk,ijk->ij", diff, diff)
    order = np.argsort(d2, axis=1, kind="stable")
    return np.take_along_axis(idx, order, axis=1), np.take_along_axis(d2, order, axis=1)


def blobs_knn(n: int = 2000, K: int = 5, dim: int = 10, knn: int = 10,
              sigma_rank: int = 7, label_frac: float = 0.05, seed: int = 0,
              centre_std: float = 2.0, device: Optional[str] = None) -> Graph:
    """K isotropic unit-variance Gaussian blobs in R^dim, centres ~ N(0, centre_std^2 I).

    Graph: union-symmetrised `knn`-NN (self excluded); w_ij = exp(-d_ij^2 /
    (sigma_i sigma_j)) with sigma_i the distance to the `sigma_rank`-th nearest
    neighbour.  Classes have sizes n//K (+1 for the first n%K).
    """
    rng = np.random.default_rng(seed)
    sizes = np.full(K, n // K, dtype=np.int64)
    sizes[: n % K] += 1
    centres = rng.normal(0.0, centre_std, size=(K, dim))
    truth = np.repeat(np.arange(K, dtype=np.int32), sizes)
    X = centres[truth] + rng.normal(0.0, 1.0, size=(n, dim))
    idx, d2 = _knn(X, knn, device)
    sigma = np.sqrt(d2[:, sigma_rank - 1])
    sigma = np.maximum(sigma, 1e-12)
    ii = np.repeat(np.arange(n, dtype=np.int64), knn)
    jj = idx.reshape(-1)
    ww = np.exp(-d2.reshape(-1) / (sigma[ii] * sigma[jj]))
    row_ptr, col, w = from_edges(n, ii, jj, ww)
    labels = pick_labels(truth, K, rng, frac=label_frac)
    return Graph(n, row_ptr, col, w, K, labels, truth,
                 dict(kind="blobs_knn", dim=dim, knn=knn, sigma_rank=sigma_rank,
                      label_frac=label_frac, seed=seed))


def sbm(n: int = 200_000, K: int = 10, deg_in: float = 20.0, deg_out: float = 2.0,
        label_frac: float = 0.01, seed: int = 0) -> Graph:
    """Stochastic block model with K equal blocks and unit weights.

    Every unordered pair inside a block is an edge with probability
    p_in = deg_in/(m-1), across blocks with p_out = deg_out/(n-m) (m = n/K), so
    the expected in-block and out-of-block degrees are deg_in and deg_out.
    Sampling: per block pair a Binomial edge count, then that many uniform pairs
    (duplicates merged).  A node left with no edge is joined to a uniformly
    chosen member of its block.
    """
    rng = np.random.default_rng(seed)
    m = n // K
    assert m * K == n, "sbm wants n divisible by K"
    truth = np.repeat(np.arange(K, dtype=np.int32), m)
    p_in = deg_in / (m - 1)
    p_out = deg_out / (n - m)
    I, J = [], []
    for a in range(K):
        for b in range(a, K):
            if a == b:
                npairs = m * (m - 1) // 2
                cnt = rng.binomial(npairs, p_in)
                i = rng.integers(0, m, size=cnt) + a * m
                j = rng.integers(0, m, size=cnt) + a * m
            else:
                npairs = m * m
                cnt = rng.binomial(npairs, p_out)
                i = rng.integers(0, m, size=cnt) + a * m
                j = rng.integers(0, m, size=cnt) + b * m
            I.append(i)
            J.append(j)
    I = np.concatenate(I)
    J = np.concatenate(J)
    keep = I != J
    I, J = I[keep], J[keep]
    deg = np.bincount(I, minlength=n) + np.bincount(J, minlength=n)
    lonely = np.flatnonzero(deg == 0)
    if lonely.size:
        blk = lonely // m
        partner = rng.integers(0, m - 1, size=lonely.size) + blk * m
        partner = np.where(partner >= lonely, partner + 1, partner)
        I = np.concatenate([I, lonely])
        J = np.concatenate([J, partner])
    row_ptr, col, w = from_edges(n, I, J, np.ones(I.shape[0]))
    labels = pick_labels(truth, K, rng, frac=label_frac)
    return Graph(n, row_ptr, col, w, K, labels, truth,
                 dict(kind="sbm", deg_in=deg_in, deg_out=deg_out,
                      label_frac=label_frac, seed=seed))


# raster-order neighbour offsets: column indices come out sorted in each row
_OFF8 = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def voronoi_image(side: int = 2048, K: int = 4, noise: float = 0.1,
                  scale: float = 0.05, label_frac: float = 0.005, seed: int = 0,
                  height: Optional[int] = None) -> Graph:
    """Noisy piecewise-constant RGB image on `side` x `height` pixels.

    K seed points uniform in the image define Voronoi cells (ties to the lowest
    seed index), one class and one colour ~ U[0,1]^3 per cell; i.i.d.
    N(0, noise^2) is added per channel (not clipped).  Graph: 8-neighbour
    pixels, w = exp(-||c_i - c_j||^2 / scale) on the noisy colours.  Labels:
    round(label_frac * n) pixels uniformly, at least one per class.
    """
    rng = np.random.default_rng(seed)
    Wd = side
    H = side if height is None else height
    n = Wd * H
    seeds = rng.uniform(0.0, 1.0, size=(K, 2)) * np.array([H, Wd])
    colours = rng.uniform(0.0, 1.0, size=(K, 3))
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64) + 0.5,
                         np.arange(Wd, dtype=np.float64) + 0.5, indexing="ij")
    best = np.full((H, Wd), np.inf)
    truth = np.zeros((H, Wd), dtype=np.int32)
    for c in range(K):
        d = (yy - seeds[c, 0]) ** 2 + (xx - seeds[c, 1]) ** 2
        better = d < best
        truth[better] = c
        best[better] = d[better]
    img = colours[truth] + rng.normal(0.0, noise, size=(H, Wd, 3))
    flat = img.reshape(n, 3)
    ids = np.arange(n, dtype=np.int64).reshape(H, Wd)
    cols = np.full((n, 8), -1, dtype=np.int64)
    for t, (dy, dx) in enumerate(_OFF8):
        y0, y1 = max(0, -dy), H - max(0, dy)
        x0, x1 = max(0, -dx), Wd - max(0, dx)
        src = ids[y0:y1, x0:x1].reshape(-1)
        dst = ids[y0 + dy:y1 + dy, x0 + dx:x1 + dx].reshape(-1)
        cols[src, t] = dst
    valid = cols >= 0
    counts = valid.sum(1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    src = np.repeat(np.arange(n, dtype=np.int64), counts)
    dst = cols[valid]
    diff = flat[src] - flat[dst]
    w = np.exp(-np.einsum("ij,ij->i", diff, diff) / scale)
    truth = truth.reshape(-1)
    labels = pick_labels(truth, K, rng, total_frac=label_frac)
    return Graph(n, row_ptr.astype(np.int32), dst.astype(np.int32), w, K, labels,
                 truth, dict(kind="voronoi_image", side=Wd, height=H, noise=noise,
                             scale=scale, label_frac=label_frac, seed=seed))


def batched_blobs(P: int = 256, n_min: int = 1000, n_max: int = 200_000,
                  K_min: int = 3, K_max: int = 10, label_frac: float = 0.02,
                  seed: int = 0, device: Optional[str] = None,
                  n_scale: float = 1.0) -> list:
    """P independent blob problems: n log-uniform in [n_min, n_max] (times
    `n_scale`, for reduced test sizes), K uniform in {K_min..K_max}; problem p
    uses seed + 1 + p."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(P):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * n_scale))
        K = int(rng.integers(K_min, K_max + 1))
        n = max(n, 4 * K)
        out.append(blobs_knn(n=n, K=K, label_frac=label_frac, seed=seed + 1 + p,
                             device=device))
    return out


# --------------------------------------------------------------- configs --
# The benchmark workloads: generator recipe, seed and solver parameters.
# eps / omega0 are the paper's network values (Sec. 5.2) unless noted; the
# image workload runs at eps = 50 for multi-iteration throughput, and its
# one-shot setting (eps = 0.1, omega0 = 1e5, Sec. 5.2) is a separate entry.
SEED0 = 20250813

CONFIGS = {
    # 2,000 points in R^10, 5 blobs, symmetrised 10-NN, FP64 parity case
    "blobs2k": dict(gen="blobs", seed=SEED0 + 0, n=2000, K=5, label_frac=0.05,
                    eps=50.0, omega0=1000.0, iters=500, weights="f64"),
    # SBM n = 200,000, K = 10 blocks, in/out degree 20/2, unit weights, FP32
    "sbm200k": dict(gen="sbm", seed=SEED0 + 1, n=200_000, K=10, label_frac=0.01,
                    eps=50.0, omega0=1000.0, iters=500, weights="f32"),
    # 2048 x 2048 noisy Voronoi image, K = 4, 8-neighbour graph
    # (measured with FP32 weights and, in the same run, with BF16 weights)
    "voronoi2048": dict(gen="voronoi", seed=SEED0 + 2, side=2048, K=4, label_frac=0.005,
                        eps=50.0, omega0=1e5, iters=200, weights="f32", arms=("f32", "bf16")),
    "voronoi2048_oneshot": dict(gen="voronoi", seed=SEED0 + 2, side=2048, K=4,
                                label_frac=0.005, eps=0.1, omega0=1e5, iters=10,
                                weights="f32"),
}


def make_config_graph(name: str, device: Optional[str] = None, **override) -> Graph:
    """Generate the input graph of a named workload (sizes overridable)."""
    c = dict(CONFIGS[name])
    c.update(override)
    if c["gen"] == "blobs":
        return blobs_knn(n=c["n"], K=c["K"], label_frac=c["label_frac"], seed=c["seed"],
                         device=device)
    if c["gen"] == "sbm":
        return sbm(n=c["n"], K=c["K"], label_frac=c["label_frac"], seed=c["seed"])
    if c["gen"] == "voronoi":
        return voronoi_image(side=c["side"], K=c["K"], label_frac=c["label_frac"],
                             seed=c["seed"])
    raise ValueError(name)
