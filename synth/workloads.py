"""Seeded generators for the five reverse k-ranks workloads.

Every array is produced by numpy's PCG64 generator from an explicit seed, in
float32, C-contiguous.  Row recipe ("gaussian"): g ~ N(0, I/d), direction
g/||g||, norm exp(sigma * z) with z ~ N(0, 1).  Mixture recipe: centres
c ~ N(0, I/d) * center_scale, a row is c + N(0, within_std^2 I/d), then
normalised and given a log-normal norm.

Nothing here computes an inner product, a rank or a threshold.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


def gaussian_rows(rng: np.random.Generator, count: int, d: int, sigma: float) -> np.ndarray:
    """Rows with isotropic Gaussian direction and log-normal(0, sigma) norm."""
    out = np.empty((count, d), dtype=np.float32)
    chunk = 1 << 16
    for lo in range(0, count, chunk):
        hi = min(count, lo + chunk)
        g = rng.standard_normal((hi - lo, d))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        g *= np.exp(sigma * rng.standard_normal((hi - lo, 1)))
        out[lo:hi] = g
    return out


def mixture_rows(rng: np.random.Generator, centers: np.ndarray, count: int,
                 within_std: float, sigma: float) -> np.ndarray:
    """Rows drawn around uniformly chosen centres, then given log-normal norms."""
    ncent, d = centers.shape
    out = np.empty((count, d), dtype=np.float32)
    chunk = 1 << 16
    for lo in range(0, count, chunk):
        hi = min(count, lo + chunk)
        which = rng.integers(0, ncent, size=hi - lo)
        g = centers[which] + rng.standard_normal((hi - lo, d)) * (within_std / math.sqrt(d))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        g *= np.exp(sigma * rng.standard_normal((hi - lo, 1)))
        out[lo:hi] = g
    return out


def sample_positions(seed: int, sizes: np.ndarray, s: int) -> np.ndarray:
    """Positions of the per-bucket random samples (Alg. 1, the sampling step).

    ``sizes`` are the bucket sizes, supplied by the caller (each side derives
    them from m and omega itself).  Returns an int32 array of shape (omega, s).  Row l holds s distinct
    positions in [0, sizes[l]) drawn uniformly without replacement; when a
    bucket holds s items or fewer every position is taken (in order) and the
    rest of the row is -1.
    """
    rng = np.random.default_rng(np.random.PCG64([seed, 0x5A4D]))
    omega = len(sizes)
    out = np.full((omega, s), -1, dtype=np.int32)
    for l in range(omega):
        size = int(sizes[l])
        if size <= s:
            out[l, :size] = np.arange(size, dtype=np.int32)
        else:
            out[l] = rng.choice(size, size=s, replace=False).astype(np.int32)
    return out


@dataclasses.dataclass
class Workload:
    name: str
    U: np.ndarray
    P: np.ndarray
    Q: np.ndarray
    k: np.ndarray                 # int32 per query
    c: float = 2.0
    tau: int = 500
    omega: int = 10
    s: int = 100
    query_from_P: Optional[np.ndarray] = None   # item index of queries drawn from P, -1 if fresh
    subsets_given: Optional[list] = None        # per-query sorted int32 user ids, or None
    seed: int = 0
    subset_blocks: Optional[list] = None        # per-query ids of 1,024-user blocks (uneven)

    @property
    def subsets(self):
        """Per-query sorted int32 user ids (None = all users); for block subsets the
        ids are expanded on first use (large: avoid at full size, use bitmaps)."""
        if self.subsets_given is None and self.subset_blocks is not None:
            n = self.U.shape[0]
            out = []
            for blocks in self.subset_blocks:
                ids = (blocks[:, None] * 1024 + np.arange(1024)[None, :]).ravel()
                out.append(ids[ids < n].astype(np.int32))
            self.subsets_given = out
        return self.subsets_given

    def subset_bitmaps(self) -> np.ndarray:
        """(nq, (n + 31) // 32) uint32: bit u of row q set iff user u is in query q's subset."""
        n = self.U.shape[0]
        words = (n + 31) // 32
        nq = self.Q.shape[0]
        out = np.zeros((nq, words), dtype=np.uint32)
        if self.subset_blocks is not None:
            nblk = (n + 1023) // 1024
            full = np.zeros((nq, nblk, 32), dtype=np.uint32)   # 32 words per 1,024-user block
            for q, blocks in enumerate(self.subset_blocks):
                full[q, blocks, :] = 0xFFFFFFFF
            out = np.ascontiguousarray(full.reshape(nq, nblk * 32)[:, :words])
            if n % 32:
                out[:, words - 1] &= np.uint32((1 << (n % 32)) - 1)
            return out
        for q in range(nq):
            ids = np.arange(n) if self.subsets is None else np.asarray(self.subsets[q])
            np.bitwise_or.at(out[q], ids >> 5, (np.uint32(1) << (ids & 31).astype(np.uint32)))
        return out

    @property
    def n(self):
        return self.U.shape[0]

    @property
    def m(self):
        return self.P.shape[0]

    @property
    def d(self):
        return self.U.shape[1]


def _queries_from_P(rng, P, count):
    idx = rng.choice(P.shape[0], size=count, replace=False)
    return P[idx].copy(), idx.astype(np.int64)


def make_workload(name: str, *, n: Optional[int] = None, m: Optional[int] = None,
                  nq: Optional[int] = None, d: Optional[int] = None,
                  seed: Optional[int] = None) -> Workload:
    """Build one of the named workloads; n, m, nq, d may be overridden to shrink it.

    Names and full sizes:
      ``exact_small``   n=2,000  m=5,000  d=32,  sigma 0.5, 16 queries from P, k=10, seed 0
      ``exact_batched`` n=500,000 m=20,000 d=100, sigma 0.7, 512 queries from P + 512 fresh, k=100
      ``approx``        n=1,000,000 m=100,000 d=200, mixture of 256 centres (scale 1, within std 0.3,
                        log-normal sigma 0.5), 10,000 queries from P, k uniform in {10, 50, 100},
                        c=2, tau=500, omega=10, s=100
      ``uneven``        n=2,000,000 m=1,000,000 d=128, mixture of 1,024 centres, 4,096 queries,
                        k log-uniform in [1, 1000], per-query user subsets of 10%-100% of U chosen
                        per block of 1,024 users
    """
    if name == "exact_small":
        n = n or 2000; m = m or 5000; d = d or 32; nq = nq or 16
        seed = 0 if seed is None else seed
        rng = np.random.default_rng(seed)
        U = gaussian_rows(rng, n, d, 0.5)
        P = gaussian_rows(rng, m, d, 0.5)
        Q, qidx = _queries_from_P(rng, P, nq)
        k = np.full(nq, 10, dtype=np.int32)
        return Workload(name, U, P, Q, k, query_from_P=qidx, seed=seed)
    if name == "exact_batched":
        n = n or 500_000; m = m or 20_000; d = d or 100; nq = nq or 1024
        seed = 1 if seed is None else seed
        rng = np.random.default_rng(seed)
        U = gaussian_rows(rng, n, d, 0.7)
        P = gaussian_rows(rng, m, d, 0.7)
        half = nq // 2
        Qp, qidx = _queries_from_P(rng, P, half)
        Qf = gaussian_rows(rng, nq - half, d, 0.7)
        Q = np.ascontiguousarray(np.vstack([Qp, Qf]))
        qidx = np.concatenate([qidx, np.full(nq - half, -1, dtype=np.int64)])
        k = np.full(nq, 100, dtype=np.int32)
        return Workload(name, U, P, Q, k, query_from_P=qidx, seed=seed)
    if name in ("approx", "learned"):
        n = n or 1_000_000; m = m or 100_000; d = d or 200; nq = nq or 10_000
        seed = 2 if seed is None else seed
        rng = np.random.default_rng(seed)
        centers = rng.standard_normal((256, d)) / math.sqrt(d) * 1.0
        U = mixture_rows(rng, centers, n, 0.3, 0.5)
        P = mixture_rows(rng, centers, m, 0.3, 0.5)
        Q, qidx = _queries_from_P(rng, P, nq)
        k = rng.choice(np.array([10, 50, 100], dtype=np.int32), size=nq)
        return Workload(name, U, P, Q, k, c=2.0, tau=500, omega=10, s=100,
                        query_from_P=qidx, seed=seed)
    if name == "uneven":
        n = n or 2_000_000; m = m or 1_000_000; d = d or 128; nq = nq or 4096
        seed = 4 if seed is None else seed
        rng = np.random.default_rng(seed)
        centers = rng.standard_normal((1024, d)) / math.sqrt(d)
        U = mixture_rows(rng, centers, n, 0.3, 0.5)
        P = mixture_rows(rng, centers, m, 0.3, 0.5)
        Q = mixture_rows(rng, centers, nq, 0.3, 0.5)
        k = np.clip(np.rint(np.exp(rng.uniform(0.0, math.log(1000.0), size=nq))), 1, 1000).astype(np.int32)
        nblk = (n + 1023) // 1024
        blocks_q, sizes = [], []
        for _ in range(nq):
            frac = rng.uniform(0.1, 1.0)
            keep = rng.random(nblk) < frac
            if not keep.any():
                keep[rng.integers(0, nblk)] = True
            blocks = np.nonzero(keep)[0]
            blocks_q.append(blocks)
            sizes.append(int(np.minimum(blocks * 1024 + 1024, n).sum() - (blocks * 1024).sum()))
        k = np.minimum(k, np.array(sizes, dtype=np.int32))
        return Workload(name, U, P, Q, k, query_from_P=np.full(nq, -1, dtype=np.int64),
                        subset_blocks=blocks_q, seed=seed)
    raise ValueError(f"unknown workload {name!r}")


def disjoint_queries(w: Workload, count: int, seed: int):
    """`count` further queries drawn from P without replacement, none of them an item
    that the workload already uses as a query; k uniform in {10, 50, 100}.
    Returns (Q, item indices, k)."""
    rng = np.random.default_rng(seed)
    used = w.query_from_P[w.query_from_P >= 0]
    pool = np.setdiff1d(np.arange(w.m, dtype=np.int64), used)
    idx = rng.choice(pool, size=count, replace=False)
    k = rng.choice(np.array([10, 50, 100], dtype=np.int32), size=count)
    return w.P[idx].copy(), idx, k


WORKLOADS = ("exact_small", "exact_batched", "approx", "learned", "uneven")
