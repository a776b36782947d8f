"""Users split across two CPU ranks (gloo), merged by the host exchange.

Each rank's part comes from the oracle on that rank's rows (the same items and
sample positions); paper_2504_13446_gb300.shard gathers the parts and the
library's host merge (rkr_merge_exact, rkr_merge_approx) combines them.  The
merged answer must equal the oracle's answer over all users, bit for bit, for
exact queries (Def. 2) and for the c-approximate steps of Section 4.3, with
either the tight candidate set (lower bound at most the part's R_up_k) or every
user of the part.
"""

import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

TAU, OMEGA, S, C = 24, 4, 30, 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    w = synth.make_workload("approx", n=601, m=400, d=16, nq=9)
    w.k = np.array([1, 5, 10, 40, 300, 301, 601, 3, 50], np.int32)
    pos = synth.sample_positions(5, oracle.bucket_sizes(w.m, OMEGA), S)
    return w, pos


def _local_exact(U, P, Q, k, offset):
    users, ranks, offs = [], [], [0]
    for u, r in oracle.exact_query(U, P, Q, k):
        users.append(u.astype(np.int64) + offset)
        ranks.append(r)
        offs.append(offs[-1] + len(u))
    return {"offsets": np.array(offs, np.int64), "users": np.concatenate(users),
            "ranks": np.concatenate(ranks).astype(np.int32)}


def _local_candidates(U, P, Q, k, pos, offset, tight):
    ora = oracle.build_index(U, P, TAU, OMEGA, S, pos)
    th = oracle.scores(U, Q)
    cols = {"users": [], "n_low": [], "n_up": [], "est": []}
    offs = [0]
    ids = np.arange(U.shape[0])
    for q in range(Q.shape[0]):
        j, lo, up = oracle.lookup(ora, th[:, q])
        est = oracle.interpolate(ora, th[:, q], j, lo, up, ids)
        keep = lo <= np.partition(up, k[q] - 1)[k[q] - 1] if tight else np.ones(len(ids), bool)
        cols["users"].append(ids[keep] + offset)
        cols["n_low"].append(lo[keep])
        cols["n_up"].append(up[keep])
        cols["est"].append(est[keep])
        offs.append(offs[-1] + int(keep.sum()))
    out = {key: np.concatenate(v) for key, v in cols.items()}
    out["offsets"] = np.array(offs, np.int64)
    return out


def _worker(rank, world, port, tight, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2504_13446_gb300 import shard
    w, pos = _workload()
    a, b = shard.shard_range(w.n, world, rank)
    kl = np.minimum(w.k, b - a)
    ex = shard.exchange_exact(_local_exact(w.U[a:b], w.P, w.Q, kl, a), w.k)
    ap = shard.exchange_approx(_local_candidates(w.U[a:b], w.P, w.Q, kl, pos, a, tight), w.k, C, S)
    results[rank] = (ex, {key: v for key, v in ap.items()})
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("tight", [True, False])
def test_two_rank_merge_equals_single_process(tight):
    from paper_2504_13446_gb300 import buildlib
    buildlib.build()
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), tight, results), nprocs=2, join=True)
    w, pos = _workload()
    want_ex = oracle.exact_query(w.U, w.P, w.Q, w.k)
    ora = oracle.build_index(w.U, w.P, TAU, OMEGA, S, pos)
    want_ap = oracle.approx_query(ora, w.U, w.Q, w.k, C)
    for rank in range(2):
        (users, ranks, off), ap = results[rank]
        for q in range(w.Q.shape[0]):
            sl = slice(off[q], off[q + 1])
            assert (users[sl] == want_ex[q][0]).all() and (ranks[sl] == want_ex[q][1]).all(), q
            sl = slice(ap["offsets"][q], ap["offsets"][q + 1])
            a = want_ap[q]
            assert (ap["users"][sl] == a["users"]).all(), q
            assert (ap["n_low"][sl] == a["n_low"]).all(), q
            assert (ap["n_up"][sl] == a["n_up"]).all(), q
            assert (ap["est"][sl] == a["est"]).all(), q
            assert ap["case"][q] == a["case"] and ap["nc"][q] == a["nc"], q


def test_shard_range_covers_every_row_once():
    from paper_2504_13446_gb300 import shard
    for n in (1, 7, 601, 1000):
        for world in (1, 2, 3, 8):
            if world > n:
                continue
            spans = [shard.shard_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1


def test_merge_rejects_bad_input():
    import paper_2504_13446_gb300 as rkr
    rkr.buildlib.build()
    with pytest.raises(rkr.RKRError):   # fewer entries than k
        rkr.rkr_merge_exact([3], [0, 2], [5, 6], [1, 2])
    with pytest.raises(rkr.RKRError):   # a user listed twice
        rkr.rkr_merge_exact([2], [0, 2], [5, 5], [1, 2])
    with pytest.raises(rkr.RKRError):   # c < 1
        rkr.rkr_merge_approx([1], 0.5, 10, [0, 1], [0], [1], [2], [1.5])
