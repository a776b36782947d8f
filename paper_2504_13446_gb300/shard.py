"""Users split by rows across processes, merged by a host exchange.

Each rank holds a contiguous block of the users (``shard_range``) and builds its
own index from its rows, the same items P and the same build parameters and
sample positions, so every per-user quantity (f_min, f_max, the Eq. 1 table
row, every rank) equals that of one index over all users.

* Exact queries (Def. 2): every rank answers with its min(k, n_rank) best users
  (global ids), the lists are gathered, and ``rkr_merge_exact`` keeps the k
  smallest (rank, user).
* c-approximate queries (Section 4.3): every rank sends the candidates of
  ``rkr_query_approx_candidates`` (its users whose lower bound can matter, with
  bounds and step-3 estimates); ``rkr_merge_approx`` runs steps 1-3 on the union.

Both give the single-index answer bit for bit.  The exchange is one
``all_gather_object`` per batch over ``torch.distributed`` (gloo on CPU ranks,
or NCCL); it moves O(k) entries per query and rank, not user rows.  The
merge is the library's host code; the rank-local parts run on the rank's GPU.
"""

from __future__ import annotations

import numpy as np

from . import (Index, rkr_merge_approx, rkr_merge_exact)


def shard_range(n: int, world: int, rank: int):
    """Rows [start, stop) of rank `rank` when n users are split into `world` blocks
    (the first n % world blocks get one more row)."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def concat_parts(parts, keys):
    """Per query, the concatenation of every part's entries (parts in rank order).

    parts: list of dicts with "offsets" (nq + 1) and per-entry arrays named in keys.
    Returns (offsets, {key: array})."""
    nq = len(parts[0]["offsets"]) - 1
    counts = np.stack([np.diff(p["offsets"]) for p in parts])      # parts x nq
    offs = np.concatenate([[0], np.cumsum(counts.sum(axis=0), dtype=np.int64)])
    out = {}
    for key in keys:
        chunks = []
        for q in range(nq):
            for p in parts:
                chunks.append(p[key][p["offsets"][q]:p["offsets"][q + 1]])
        out[key] = np.concatenate(chunks) if chunks else np.zeros(0)
    return offs, out


def _gather(obj, group=None):
    import torch.distributed as dist
    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, obj, group=group)
    return got


def exchange_exact(local: dict, k, group=None):
    """Merge the ranks' exact answers.  local: offsets, users (global ids), ranks of
    this rank's min(k, n_rank) best per query.  Every rank gets (users, ranks, offsets)."""
    parts = _gather(local, group)
    offs, cat = concat_parts(parts, ("users", "ranks"))
    return rkr_merge_exact(k, offs, cat["users"], cat["ranks"])


def exchange_approx(local: dict, k, c: float, s: int, group=None) -> dict:
    """Merge the ranks' approximate candidates (rkr_query_approx_candidates output)."""
    parts = _gather(local, group)
    offs, cat = concat_parts(parts, ("users", "n_low", "n_up", "est"))
    return rkr_merge_approx(k, c, s, offs, cat["users"], cat["n_low"], cat["n_up"], cat["est"])


class ShardedIndex:
    """This rank's block of users with its own index; queries merge over all ranks."""

    def __init__(self, U_rows, P, *, n_total: int, user_offset: int, s: int = 100, group=None,
                 **build_kw):
        self.n_local = int(U_rows.shape[0])
        self.n_total = int(n_total)
        self.offset = int(user_offset)
        self.s = int(s)
        self.group = group
        self.index = Index(U_rows, P, s=s, **build_kw)

    def _local_k(self, Q, k):
        nq = Q.shape[0]
        kk = np.broadcast_to(np.asarray(k, np.int32), (nq,))
        return kk, np.minimum(kk, self.n_local).astype(np.int32)

    def query_exact(self, Q, k):
        kk, kl = self._local_k(Q, k)
        users, ranks, offs, _ = self.index.query_exact(Q, kl)
        local = {"offsets": offs, "users": users.astype(np.int64) + self.offset, "ranks": ranks}
        return exchange_exact(local, kk, self.group)

    def query_approx(self, Q, k, c: float) -> dict:
        kk, kl = self._local_k(Q, k)
        local = self.index.query_approx_candidates(Q, kl, user_offset=self.offset)
        return exchange_approx(local, kk, c, self.s, self.group)

    def close(self):
        self.index.close()
