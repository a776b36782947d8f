"""Benchmark: reverse k-ranks on the |U| = 1M, |P| = 100k, d = 200 workload.

One step is one pass of the whole path over one batch of 10,000 queries:
pre-processing (norms, sort, buckets, samples, f_min/f_max, rank table, level
tables, exact count table) followed by the c-approximate query batch
(Section 4.3, c = 2) and the exact query batch (Def. 2) of the same queries.
The metric is queries per second of that pass; the index build is part of it.

Inputs are resident in HBM when the timed region starts and are larger than
L2 (U alone is 800 MB).  Device time is measured with CUDA events on the
stream the library runs on.  ``e2e`` repeats the step through the C ABI with
inputs in pinned host memory and results returned to host arrays, host-device
copies included.  ``cpu_baseline`` times the FP64
oracle on a bounded sample of users and queries and scales it to the workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                      [--case full|small|learned|latency|sweep|uneven]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "approx"
C = 2.0


# DRAM bytes (read + written) per screened row, per launch, of the screens whose
# traffic was captured with ncu (dram__bytes_read.sum + dram__bytes_write.sum) on
# the small profiling case (`--case small`: 40k users, all 100k items), where
# the rows a launch screens are known.  A full-size launch of the same kernel
# reads the same item side per row block, so its traffic scales with its rows;
# the bench multiplies this figure by the rows of the timed launches.  Empty
# until a capture of the current kernel exists (traffic is then reported null).
TRAFFIC_PER_ROW = {
    # k_screen_pair<EpiXT> (concatenated split operands), 40,000 rows of the 1M x 100k
    # workload's generator with all items: 495.6 MB read + 2,235.0 MB written in one
    # launch; the tail-list writes (about 55 KB per user) dominate and scale with rows
    "k_screen<EpiXT>": 68_265.0,
}

# Products the tensor cores issue per pair of each screen, relative to the
# method's one inner product of length d: the split screens issue three
# products over K padded to a multiple of 16.
SPLIT_SCREENS = ("k_screen<EpiRC>", "k_screen<EpiXT>", "k_screen<EpiSkim>",
                 "k_screen<EpiTable>", "k_screen<EpiTableSm>", "k_screen<EpiTheta>")


def _load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("RKR_BENCH_GLOO") is None else "gloo")
        return dist, rank, ws
    return None, 0, 1


def job_ms(ms_local: float, dist) -> float:
    """The job's step time: the maximum over ranks (each rank runs its own replica)."""
    if not dist:
        return ms_local
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size: int, queries_per_rank: int, ms: float) -> float:
    """Whole-job throughput: queries processed by all ranks per second of the slowest rank."""
    return world_size * queries_per_rank / (ms / 1000.0)


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to a scratch file; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"rkr_clocks_{os.getpid()}_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(case="full"):
    if case == "small":
        # profiling case: 40k users, all 100k items, 2,000 queries; two of them shrunk to a
        # tiny norm so that u.q lies mid-range for every user and the recount screen runs
        w = synth.make_workload(WORKLOAD, n=40_000, nq=2000)
        w.Q[:2] *= np.float32(1e-3)
    else:
        w = synth.make_workload(WORKLOAD)
    sizes = np.array([w.m // w.omega + (1 if l < w.m % w.omega else 0) for l in range(w.omega)])
    pos = synth.sample_positions(w.seed, sizes, w.s)
    return w, pos


def run_step(rkr, U, P, Q, k, pos, w, device=True, keep=False):
    idx = rkr.Index(U, P, tau=w.tau, omega=w.omega, s=w.s, fbounds="exact", exact_table=True,
                    sample_pos=pos)
    a = idx.query_approx(Q, k, C, device=device)
    e = idx.query_exact(Q, k, device=device)
    t = idx.timings()
    if keep:
        return a, e, t, idx
    idx.close()
    return a, e, t


def roofline_of(kernels, steps, peaks, peak_src, launches_rows=None):
    """Roofline entry of the kernel with the largest device time in the timed region.

    For a tensor-core screen, achieved = the method's flops (one inner product of
    length d per screened pair: 2 * rows * cols * d) / its device time, against the
    measured dense BF16 peak; the products the tensor cores actually issue (three
    for the split form, K padded to a multiple of 16) are reported beside it."""
    name = max(kernels, key=lambda kk: kernels[kk][1])
    n_l, t_ms, work = kernels[name]
    if work <= 0:
        return {"kernel": name, "bound": None, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None, "launches_per_step": n_l / steps,
                "ms_per_launch": t_ms / n_l}
    peak = peaks["bf16_tflops"]
    achieved = work / (t_ms / 1000.0) / 1e12
    out = {"kernel": name, "bound": "tensor", "achieved": achieved, "peak": peak,
           "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
           "launches_per_step": n_l / steps, "ms_per_launch": t_ms / n_l,
           "peak_source": f"{peak_src} bf16 dense burst peak (MEASURED_PEAKS.json bf16_tflops); "
                          "achieved = 2 x rows x cols x d (the method's inner products) / "
                          "CUDA-event time of the launches"}
    if "bf16_tflops_sustained" in peaks:
        out["frac_of_sustained"] = achieved / peaks["bf16_tflops_sustained"]
    if name in SPLIT_SCREENS:
        out["tensor_products_issued_per_pair"] = "3 x K' (K' = d rounded up to 16)"
    if name in TRAFFIC_PER_ROW and launches_rows:
        out["traffic"] = TRAFFIC_PER_ROW[name] * launches_rows / n_l
    return out


def bench_ours(args):
    import torch
    import paper_2504_13446_gb300 as rkr

    dist, rank, ws = _dist()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    peaks, peak_src = _load_peaks()
    w, pos = make_inputs(args.case)
    U = torch.from_numpy(w.U).cuda()
    P = torch.from_numpy(w.P).cuda()
    Q = torch.from_numpy(w.Q).cuda()
    k = torch.from_numpy(w.k.astype(np.int32)).cuda()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        run_step(rkr, U, P, Q, k, pos, w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = rkr.kernel_launches()
    rkr.rkr_profile_start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage = []
    qstats = []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        a, e, t = run_step(rkr, U, P, Q, k, pos, w)
        stage.append(t)
        qstats.append((a["stats"].as_dict(), e[3].as_dict()))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = rkr.kernel_launches() - launches0
    prof = rkr.rkr_profile_stop()
    clocks = sampler.stop()
    ms = job_ms(ev0.elapsed_time(ev1) / args.steps, dist)
    kernels = {kk: v for kk, v in prof.items() if not kk.startswith("span:")}
    spans = {kk[5:]: v for kk, v in prof.items() if kk.startswith("span:")}

    if args.case == "small":
        if rank == 0:
            print(json.dumps({"case": "small (profiling)", "ms_per_step": ms,
                              "kernels_ms_per_step": {kk: round(v[1] / args.steps, 3)
                                                      for kk, v in kernels.items()},
                              "screen_rows_per_step": {
                                  kk: v[2] / (2.0 * w.m * w.d) / args.steps
                                  for kk, v in kernels.items() if v[2] > 0},
                              "exact_stats": qstats[-1][1]}))
        return
    # end to end through the C ABI with host buffers: inputs in pinned host memory,
    # copied to the device inside the library, results read back to host arrays
    Uh, Ph, Qh = (torch.from_numpy(a_).pin_memory() for a_ in (w.U, w.P, w.Q))
    kh = w.k.astype(np.int32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    a_h, e_h, _, idx = run_step(rkr, Uh, Ph, Qh, kh, pos, w, device=False, keep=True)
    e2e_s = time.perf_counter() - t0
    h2d = w.U.nbytes + w.P.nbytes + w.Q.nbytes + 4 * w.Q.shape[0] + pos.nbytes
    d2h = sum(v.nbytes for kk, v in a_h.items() if isinstance(v, np.ndarray) and kk != "offsets")
    d2h += e_h[0].nbytes + e_h[1].nbytes

    # quality of the approximate answers of the step against its exact answers
    # (after the timed region): exact ranks of every returned user by the exact path
    nq = w.Q.shape[0]
    qid = np.repeat(np.arange(nq, dtype=np.int32), np.diff(a_h["offsets"]))
    r_c = idx.rank_pairs(w.Q, a_h["users"], qid)
    quality = approx_quality(r_c, a_h["offsets"], e_h[1], C)
    quality["case_b_queries"] = int(np.sum(a_h["case"] == 2))
    precision = screen_precision(rkr, U, P)
    learned = None
    if os.environ.get("RKR_BENCH_LEARNED", "1") != "0":
        # the learned cut against the plain exact batch on the same index
        # (outside the timed region)
        learned = learned_comparison(rkr, w, U, P, Q, pos, 2, idx=idx)
    idx.close()

    if rank != 0:
        return
    value = job_value(ws, nq, ms)
    mean = lambda key: float(np.mean([s_[key] for s_ in stage]))  # noqa: E731
    rows_of = {kk: v[2] / (2.0 * w.m * w.d) for kk, v in kernels.items() if v[2] > 0}
    name = max(kernels, key=lambda kk: kernels[kk][1])
    roof = roofline_of(kernels, args.steps, peaks, peak_src, rows_of.get(name))
    top = sorted(kernels.items(), key=lambda kv: -kv[1][1])[:14]
    qa0, qe0 = qstats[-1]
    cpu = cpu_baseline(w, pos)
    out = {
        "metric": "queries/s",
        "value": value,
        "unit": "queries/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16+f32+f64",
        "data": "synthetic",
        "config": {
            "workload": "c-approximate + exact reverse k-ranks, index build included: "
                        "|U|=1,000,000 |P|=100,000 d=200 Gaussian mixture (256 centres), "
                        "10,000 queries from P, k in {10,50,100}, c=2, tau=500, omega=10, s=100",
            "l2": "inputs larger than L2 (U is 800 MB)",
            "parallelism": f"replicas x{ws}",
            "tuning": rkr.rkr_tuning_get(),
        },
        "user_item_scores_per_s": w.n * w.m / (ms / 1000.0),
        "phases_ms": {
            "build": {kk: mean(kk) for kk in stage[0]},
            "approx": {kk: qa0[kk] for kk in ("ms_theta", "ms_resolve", "ms_select")},
            "exact": {kk: qe0[kk] for kk in ("ms_theta", "ms_resolve", "ms_select")},
        },
        "candidates": {"approx": qa0["candidates"], "exact": qe0["candidates"],
                       "exact_recounted": qe0["recounted"],
                       "exact_recount_users": qe0["recount_users"],
                       "exact_recount_split": qe0["recount_split"],
                       "exact_recount_open": qe0["recount_open"],
                       "exact_prefix_rows": qe0["prefix_rows"],
                       "exact_prefix_pruned": qe0["prefix_pruned"],
                       "wide_queries": [qa0["wide_queries"], qe0["wide_queries"]],
                       "deep_queries": [qa0["deep_queries"], qe0["deep_queries"]]},
        "approx_quality": quality,
        "learned_cut": learned,
        "precision": {
            "screen_sample": precision,
            "exact_path": {
                "near_ties": qe0["near_ties"],
                "flagged_fraction": (qe0["near_ties"] / (qe0["recount_open"] * w.m)
                                     if qe0["recount_open"] else 0.0),
                "flagged_fraction_definition": "item scores of the exact recount that needed "
                                               "canonical FP64 / item scores it screened",
                "fp64_dots": qe0["fp64_dots"],
                "max_rel_screen_err": qe0["max_rel_screen_err"],
                "max_screen_err_over_bound": qe0["max_screen_err_ratio"]},
            "approx_path": {"fp64_dots": qa0["fp64_dots"], "candidates": qa0["candidates"]},
        },
        "roofline": roof,
        "kernels_ms_per_step": {kk: round(v[1] / args.steps, 3) for kk, v in top},
        "spans_ms_per_step": {kk: round(v[1] / args.steps, 3) for kk, v in spans.items()},
        "cpu_baseline": cpu,
        "e2e": {"value": nq / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "library": rkr.version(),
    }
    print(json.dumps(out))


def learned_comparison(rkr, w, U, P, Q, pos, steps, idx=None):
    """The learned cut on the 1M x 100k x 200 workload: a monotone rank regressor
    (65 -> 256 -> 256 -> 1) trained on the GPU on 10M exact (query, user, rank)
    samples that the GPU path itself produces for 1,000 training queries (each
    query's 2,000 best users plus 8,000 random ones), the keep factor calibrated
    on 200 held-out queries (the smallest on a grid whose cut needs no more than
    1 % of its candidates revived), then the 10,000 bench queries answered with
    and without the cut.  With its exact fallback the cut returns the exact
    answer; the comparison reports time, candidates and revived candidates.
    All training and calibration queries are items of P disjoint from the bench
    queries."""
    import torch

    k = w.k.astype(np.int32)
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    own = idx is None
    ms_build = None
    if own:
        idx, ms_build = timed(lambda: rkr.Index(U, P, tau=w.tau, omega=w.omega, s=w.s,
                                                fbounds="exact", exact_table=True,
                                                sample_pos=pos))
    rng = np.random.default_rng(7)
    Rp = (rng.standard_normal((64, w.d)) / math.sqrt(w.d)).astype(np.float32)
    n_train, n_cal, top, rand = 1000, 200, 2000, 8000
    Qx, _, kx = synth.disjoint_queries(w, n_train + n_cal, seed=8)
    Qtr, Qcal, kcal = Qx[:n_train], Qx[n_train:], kx[n_train:]
    (tu, tr, toff, _), ms_top = timed(lambda: idx.query_exact(Qtr, top))
    ru = rng.integers(0, w.n, size=n_train * rand).astype(np.int32)
    rq = np.repeat(np.arange(n_train, dtype=np.int32), rand)
    rr, ms_pairs = timed(lambda: idx.rank_pairs(Qtr, ru, rq))
    pu = np.concatenate([tu, ru]).astype(np.int32)
    pq = np.concatenate([np.repeat(np.arange(n_train, dtype=np.int32), top), rq])
    target = np.log(np.concatenate([tr, rr]).astype(np.float64)).astype(np.float32)
    (X, t), ms_feat = timed(lambda: idx.pair_features(Rp, Qtr, pu, pq))
    net = rkr.Pruner(65, 256, seed=2)
    epochs = int(os.environ.get("RKR_LEARNED_EPOCHS", "4"))
    loss, ms_train = timed(lambda: net.train(X, t, target, epochs=epochs, batch=4096, lr=1e-3,
                                             seed=3))
    del X, t
    # keep factor of the plain cut: the smallest alpha on the grid with recall >= 0.99
    # on the held-out queries (judged by the exact query)
    def recall_of(lr_, loff_, plain_r_):
        hits = viol = 0
        for q in range(len(loff_) - 1):
            sl = slice(loff_[q], loff_[q + 1])
            kth = plain_r_[sl].max()
            hits += int(np.sum(lr_[sl] <= kth))
            viol += int(np.sum(lr_[sl] > C * kth))
        return hits / float(loff_[-1]), viol

    _, cal_r, _, _ = idx.query_exact(Qcal, kcal)
    grid = [1.0, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0]
    cal = {}
    alpha = grid[-1]
    for a in grid:
        keep = np.ceil(a * kcal).astype(np.int32)
        _, lr_c, loff_c, _ = idx.query_exact_learned(net, Rp, Qcal, kcal, keep, certify=False)
        cal[a] = recall_of(lr_c, loff_c, cal_r)[0]
        if cal[a] >= 0.99:
            alpha = a
            break
    keep = np.ceil(alpha * k).astype(np.int32)
    for _ in range(2):
        idx.query_exact(Q, k)
        idx.query_exact_learned(net, Rp, Q, k, keep, certify=False)
        idx.query_exact_learned(net, Rp, Q, k, keep, certify=True)
    ms_plain, ms_cut, ms_cert = [], [], []
    for _ in range(steps):
        (pu_, pr_, poff, pst), t_plain = timed(lambda: idx.query_exact(Q, k))
        ms_plain.append(t_plain)
        (lu, lr, loff, lst), t_cut = timed(
            lambda: idx.query_exact_learned(net, Rp, Q, k, keep, certify=False))
        ms_cut.append(t_cut)
        (cu_, cr_, coff, cst), t_cert = timed(
            lambda: idx.query_exact_learned(net, Rp, Q, k, keep, certify=True))
        ms_cert.append(t_cert)
    recall, viol = recall_of(lr, loff, pr_)
    same_cert = bool((cu_ == pu_).all() and (cr_ == pr_).all())
    # the network tabulated per user (rkr_pruner_invert): one lookup per candidate
    G = 64
    _, ms_invert = timed(lambda: net.invert(idx, Rp, G))
    for _ in range(2):
        idx.query_exact_learned(net, Rp, Q, k, keep, certify=False)
    ms_tcut, ms_tcert = [], []
    for _ in range(steps):
        (tu_, tr_, toff_, tst), t_tc = timed(
            lambda: idx.query_exact_learned(net, Rp, Q, k, keep, certify=False))
        ms_tcut.append(t_tc)
        (tcu, tcr, _, tcst), t_tk = timed(
            lambda: idx.query_exact_learned(net, Rp, Q, k, keep, certify=True))
        ms_tcert.append(t_tk)
    t_recall, t_viol = recall_of(tr_, toff_, pr_)
    mtc, mtk = statistics.median(ms_tcut), statistics.median(ms_tcert)
    mplain = statistics.median(ms_plain)
    table = {"grid_points": G, "ms_invert": ms_invert,
             "ms_per_batch": {"learned_cut": mtc, "learned_certified": mtk},
             "speedup_over_plain_exact": {"cut": mplain / mtc, "certified": mplain / mtk},
             "recall_at_k": t_recall, "c_bound_violations": t_viol,
             "certified_answers_equal_plain_exact": bool((tcu == pu_).all() and
                                                         (tcr == pr_).all()),
             "recounted_cut": tst.recounted}
    net.invert(idx, Rp, 0)
    if own:
        idx.close()
    mp, mc, mk = (statistics.median(v) for v in (ms_plain, ms_cut, ms_cert))
    return {
        "ms_per_batch": {"learned_cut": mc, "learned_certified": mk, "plain_exact": mp},
        "speedup": {"cut": mp / mc, "certified": mp / mk},
        "recall_at_k": recall, "c_bound_violations": viol,
        "certified_answers_equal_plain_exact": same_cert,
        "keep": f"ceil({alpha} * k) per query",
        "candidates": {"plain": pst.candidates, "cut": lst.candidates,
                       "certified": cst.candidates,
                       "revived_by_fallback": cst.learned_revived,
                       "recounted_plain": pst.recounted, "recounted_cut": lst.recounted,
                       "recounted_certified": cst.recounted},
        "per_user_tables": table,
        "calibration_recall": {str(a): r for a, r in cal.items()},
        "training": {"queries": n_train, "samples": int(len(pu)), "epochs": epochs,
                     "batch": 4096, "final_loss": loss,
                     "ms": {"index_build": ms_build, "top_users": ms_top,
                            "rank_pairs": ms_pairs, "features": ms_feat, "train": ms_train}},
    }


def bench_learned(args):
    """The learned case on its own JSON line (see learned_comparison)."""
    import torch
    import paper_2504_13446_gb300 as rkr

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w, pos = make_inputs("full")
    U = torch.from_numpy(w.U).cuda()
    P = torch.from_numpy(w.P).cuda()
    Q = torch.from_numpy(w.Q).cuda()
    rkr.rkr_profile_start()
    res = learned_comparison(rkr, w, U, P, Q, pos, args.steps)
    kernels = rkr.rkr_profile_stop()
    nq = w.Q.shape[0]
    top_k = sorted(((kk, v) for kk, v in kernels.items() if not kk.startswith("span:")),
                   key=lambda kv: -kv[1][1])[:12]
    print(json.dumps({
        "case": "learned",
        "metric": "queries/s", "value": nq / (res["ms_per_batch"]["learned_cut"] / 1000.0),
        "unit": "queries/s",
        "plain_exact_value": nq / (res["ms_per_batch"]["plain_exact"] / 1000.0),
        "steps": args.steps, "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "exact reverse k-ranks with and without the learned cut: "
                               "|U|=1,000,000 |P|=100,000 d=200 mixture, 10,000 queries from P, "
                               "k in {10,50,100}; regressor 65->256->256->1"},
        **res,
        "kernels_ms_total": {kk: round(v[1], 3) for kk, v in top_k}}))


def bench_uneven(args):
    """The uneven batch at full size: |U| = 2M, |P| = 1M, d = 128 (mixture of 1,024
    centres), 4,096 queries with k log-uniform in [1, 1000] and a user subset per
    query (10-100 % of U in blocks of 1,024 users, passed as bitmaps).  The index
    (tau 500, omega 10, s 100, exact tables with floor rank 2,048) is built once,
    timed apart; a step is the exact batch and the c-approximate batch (c = 2) of
    all 4,096 queries.  User-item scores/s counts |subset| * m per query."""
    import torch
    import paper_2504_13446_gb300 as rkr

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    peaks, peak_src = _load_peaks()
    t_start = time.perf_counter()

    def note(msg):   # progress on stderr, flushed (the JSON line stays the only stdout)
        print(f"[uneven {time.perf_counter() - t_start:8.1f} s] {msg}", file=sys.stderr,
              flush=True)

    t0 = time.perf_counter()
    size = os.environ.get("RKR_UNEVEN_SIZE")   # "n,m,nq" for a reduced case
    if size:
        n_, m_, q_ = (int(v) for v in size.split(","))
        w = synth.make_workload("uneven", n=n_, m=m_, nq=q_)
    else:
        w = synth.make_workload("uneven")
    bm = w.subset_bitmaps()
    t_gen = time.perf_counter() - t0
    note(f"generated n={w.n} m={w.m} nq={w.Q.shape[0]}")
    U = torch.from_numpy(w.U).cuda()
    P = torch.from_numpy(w.P).cuda()
    Q = torch.from_numpy(w.Q).cuda()
    k = torch.from_numpy(w.k.astype(np.int32)).cuda()
    member = torch.from_numpy(bm.view(np.int32)).cuda()
    sizes = np.array([int(np.unpackbits(r.view(np.uint8)).sum()) for r in bm[:64]])
    subset_users = float(sum(int(np.minimum(b * 1024 + 1024, w.n).sum() - (b * 1024).sum())
                             for b in w.subset_blocks))
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    note("inputs on the device")
    rkr.rkr_profile_start()
    # the exact tables with the deep count grid below the tail lists (exact_table = 2):
    # the queries' k reaches 1,000, far below the floor rank for many users
    xt = int(os.environ.get("RKR_UNEVEN_EXACT_TABLE", "2"))
    idx, ms_build = timed(lambda: rkr.Index(U, P, tau=w.tau, omega=w.omega, s=w.s,
                                            fbounds="exact", exact_table=xt, floor_rank=2048))
    note(f"index built in {ms_build:.0f} ms: {idx.timings()}")
    build_prof = rkr.rkr_profile_stop()
    note("build kernels: " + json.dumps({kk: round(v[1], 1) for kk, v in
                                         sorted(build_prof.items(), key=lambda kv: -kv[1][1])[:8]}))
    for _ in range(max(1, args.warmup)):
        (_, _, _, wst), t_w = timed(lambda: idx.query_exact(Q, k, member=member, device=True))
        note(f"warm-up exact batch {t_w:.0f} ms: {json.dumps(wst.as_dict())}")
        _, t_w = timed(lambda: idx.query_approx(Q, k, C, member=member, device=True))
        note(f"warm-up approximate batch {t_w:.0f} ms")
    rkr.rkr_profile_start()
    ms_e, ms_a = [], []
    for _ in range(args.steps):
        (eu, er, eoff, est_), t_e = timed(lambda: idx.query_exact(Q, k, member=member,
                                                                  device=True))
        a, t_a = timed(lambda: idx.query_approx(Q, k, C, member=member, device=True))
        ms_e.append(t_e)
        ms_a.append(t_a)
        note(f"step: exact {t_e:.0f} ms, approximate {t_a:.0f} ms")
    prof = rkr.rkr_profile_stop()
    mem = idx.device_bytes()
    note("screen forms against the floor thresholds")
    forms = screen_forms_at_floor(rkr, idx, w)
    idx.close()
    kernels = {kk: v for kk, v in prof.items() if not kk.startswith("span:")}
    rows_of = {kk: v[2] / (2.0 * w.m * w.d) for kk, v in kernels.items() if v[2] > 0}
    name = max(kernels, key=lambda kk: kernels[kk][1])
    roof = roofline_of(kernels, args.steps, peaks, peak_src, rows_of.get(name))
    me, ma = statistics.median(ms_e), statistics.median(ms_a)
    nq = w.Q.shape[0]
    print(json.dumps({
        "case": "uneven (config 4)",
        "metric": "queries/s", "unit": "queries/s",
        "value": 2 * nq / ((me + ma) / 1000.0),
        "exact_queries_per_s": nq / (me / 1000.0), "approx_queries_per_s": nq / (ma / 1000.0),
        "user_item_scores_per_s": {"exact": subset_users * w.m / (me / 1000.0),
                                   "approx": subset_users * w.m / (ma / 1000.0)},
        "ms_per_batch": {"exact": me, "approx": ma, "index_build": ms_build},
        "steps": args.steps, "higher_is_better": True, "data": "synthetic",
        "dtype": "bf16+f32+f64",
        "config": {"workload": f"|U|={w.n:,} |P|={w.m:,} d={w.d} mixture (1,024 centres), "
                               f"{nq:,} queries, k log-uniform in [1,1000], per-query subsets of "
                               "10-100% of U in 1,024-user blocks (bitmaps), tau=500, omega=10, "
                               "s=100, exact tables with floor rank 2,048"
                               + (" and the deep count grid" if xt == 2 else "") + ", c=2",
                   "tuning": rkr.rkr_tuning_get(),
                   "subset_users_total": subset_users, "k_max": int(w.k.max()),
                   "k_mean": float(w.k.mean()), "first_subset_sizes": sizes[:4].tolist()},
        "index_device_gb": mem / 1e9,
        "stats_exact": est_.as_dict(),
        "roofline": roof,
        "kernels_ms_per_step": {kk: round(v[1] / args.steps, 3) for kk, v in
                                sorted(kernels.items(), key=lambda kv: -kv[1][1])[:14]},
        "generation_s": t_gen,
        "screen": "BF16 single and split products; the E4M3 screen is not on this path",
        "screen_forms_at_floor": forms}))


def screen_forms_at_floor(rkr, idx, w, users=128, seed=5):
    """After the timed region: for a sample of users and every item, the fraction
    of (user, item) pairs whose screened interval [s_hat - b, s_hat + b] contains
    the user's floor threshold x_0 (the comparison the exact table and the recount
    must settle), for the E4M3 screen, the single and the split BF16 products."""
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(w.n, size=min(users, w.n), replace=False))
    x0 = idx.export("xgrid")[sample, 0][:, None]
    out = {"users": int(len(sample)), "items": int(w.m), "threshold": "x_0 (floor rank)"}
    for name, split in (("e4m3", 2), ("bf16_single", False), ("bf16_split", True)):
        sc, b = rkr.rkr_screen_scores(w.U[sample], w.P, split=split)
        open_ = np.abs(sc.astype(np.float64) - x0) <= b
        out[name] = {"undecided_fraction": float(open_.mean()),
                     "median_bound_over_abs_score":
                         float(np.median(b / np.maximum(np.abs(sc), 1e-30)))}
        del sc, b, open_
    return out


def bench_latency(args):
    """Queries one at a time (rkr_query_approx_single) on the 1M x 100k x 200
    index: the paper's per-query protocol (1,000 random items of P as queries,
    each answered on its own).  Reports ms per query and the HBM bandwidth of the
    scan kernel (its algorithmic bytes: U once, per-user bin data, two table
    cells and the bound arrays it writes) against the measured copy bandwidth."""
    import torch
    import paper_2504_13446_gb300 as rkr

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    peaks, peak_src = _load_peaks()
    n_users = int(os.environ.get("RKR_LATENCY_USERS", "0"))   # profiling: fewer users
    if n_users:
        w = synth.make_workload(WORKLOAD, n=n_users)
        sizes = np.array([w.m // w.omega + (1 if l < w.m % w.omega else 0)
                          for l in range(w.omega)])
        pos = synth.sample_positions(w.seed, sizes, w.s)
    else:
        w, pos = make_inputs("full")
    U = torch.from_numpy(w.U).cuda()
    P = torch.from_numpy(w.P).cuda()
    nq = int(os.environ.get("RKR_LATENCY_QUERIES", "1000"))
    Q = torch.from_numpy(w.Q[:nq]).cuda()
    k = torch.from_numpy(w.k[:nq].astype(np.int32)).cuda()
    stream = torch.cuda.current_stream()
    idx = rkr.Index(U, P, tau=w.tau, omega=w.omega, s=w.s, fbounds="exact", exact_table=False,
                    sample_pos=pos)
    for _ in range(max(args.warmup, 1)):
        idx.query_approx(Q[:50], k[:50], C, single=True, device=True)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    rkr.rkr_profile_start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        one = idx.query_approx(Q, k, C, single=True, device=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = rkr.rkr_profile_stop()
    clocks = sampler.stop()
    ms_q = ev0.elapsed_time(ev1) / (args.steps * nq)
    batch = idx.query_approx(Q, k, C, device=True)
    same = all(bool((one[key] == batch[key]).all()) for key in
               ("users", "n_low", "n_up", "est", "case", "nc"))
    st1 = one["stats"]
    # end to end per query through a graph-captured session: host query in, host
    # answer out, copies and synchronization included
    kh = w.k[:nq].astype(np.int32)
    bu = batch["users"].cpu().numpy()
    boff = batch["offsets"]
    sess = rkr.Session(idx, max_k=int(kh.max()), c=C)
    for q in range(min(20, nq)):
        sess.query(w.Q[q], int(kh[q]))
    lat = []
    same_sess = True
    for q in range(nq):
        t0 = time.perf_counter()
        got = sess.query(w.Q[q], int(kh[q]))
        lat.append((time.perf_counter() - t0) * 1000.0)
        same_sess &= bool((got["users"] == bu[boff[q]:boff[q + 1]]).all())
    sess.close()
    idx.close()
    n_l, t_ms, work = prof["k_latency_scan"]
    gbs = work / (t_ms / n_l / 1000.0) / n_l / 1e9
    print(json.dumps({
        "case": "latency (one query at a time)",
        "metric": "ms/query", "value": ms_q, "unit": "ms/query", "higher_is_better": False,
        "queries_per_s": 1000.0 / ms_q, "queries": nq, "steps": args.steps,
        "config": {"workload": "c-approximate reverse k-ranks, one query at a time: "
                               "|U|=1,000,000 |P|=100,000 d=200 mixture, tau=500, omega=10, "
                               "s=100, c=2, 1,000 queries from P, k in {10,50,100}"},
        "equals_batched_answer": same,
        "session_e2e_ms": {"mean": float(np.mean(lat)), "p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)),
                           "note": "rkr_session_query: host query in, host answer out, one "
                                   "CUDA graph replay per query",
                           "equals_batched_answer": same_sess},
        "canonical_fp64_fraction": st1.fp64_dots / max(st1.pairs, 1),
        "roofline": {"kernel": "k_latency_scan", "bound": "hbm", "achieved": gbs,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                     "traffic": None, "ms_per_launch": t_ms / n_l,
                     "bytes_per_launch": work / n_l,
                     "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
        "kernels_ms_per_query": {kk: round(v[1] / (args.steps * nq), 5) for kk, v in prof.items()
                                 if not kk.startswith("span:")},
        "clocks": clocks,
        "paper_context": "the paper's one-thread CPU query time at tau=500 is 57.8-501.9 ms on "
                         "its datasets (Table 1; i9-10980XE)"}))


SWEEP = [(100, 10, 100), (500, 10, 100), (1000, 10, 100),     # tau at omega 10, s 100
         (500, 1, 1000), (500, 10, 10), (500, 10, 1000), (500, 100, 100)]


def bench_sweep(args):
    """The analogue of the paper's Table 1 on the 1M x 100k x 200 workload: for each
    (tau, omega, s) of SWEEP, the build time of the c-approximate index, the time of
    the 10,000-query batch (c = 2), the index's device memory, and the quality of the
    answers against the exact ones (accuracy, overall ratio, recall, c-bound
    violations).  The exact answers and the exact ranks of every returned user come
    from one exact index (they do not depend on tau, omega or s)."""
    import torch
    import paper_2504_13446_gb300 as rkr

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w, pos0 = make_inputs("full")
    U = torch.from_numpy(w.U).cuda()
    P = torch.from_numpy(w.P).cuda()
    Q = torch.from_numpy(w.Q).cuda()
    k = w.k.astype(np.int32)
    nq = w.Q.shape[0]
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    exact = rkr.Index(U, P, tau=w.tau, omega=w.omega, s=w.s, fbounds="exact", exact_table=True,
                      sample_pos=pos0)
    _, best, off, _ = exact.query_exact(Q, k)
    qid = np.repeat(np.arange(nq, dtype=np.int32), np.diff(off))
    rows = []
    for tau, omega, s_ in SWEEP:
        sizes = np.array([w.m // omega + (1 if l < w.m % omega else 0) for l in range(omega)])
        pos = synth.sample_positions(w.seed, sizes, s_)
        kw = dict(tau=tau, omega=omega, s=s_, fbounds="exact", exact_table=False, sample_pos=pos)
        rkr.Index(U, P, **kw).close()                      # warm-up build
        idx, ms_build = timed(lambda: rkr.Index(U, P, **kw))
        idx.query_approx(Q, k, C, device=True)              # warm-up batch
        a, ms_query = timed(lambda: idx.query_approx(Q, k, C, device=True))
        mem = idx.device_bytes()
        idx.close()
        users = a["users"].cpu().numpy()
        r_c = exact.rank_pairs(w.Q, users, qid)
        qual = approx_quality(r_c, off, best, C)
        rows.append({"tau": tau, "omega": omega, "s": s_, "build_ms": ms_build,
                     "query_batch_ms": ms_query, "ms_per_query": ms_query / nq,
                     "index_device_gb": mem / 1e9,
                     "case_b_queries": int((a["case"].cpu().numpy() == 2).sum()),
                     **{kk: qual[kk] for kk in ("accuracy", "overall_ratio", "recall_at_k",
                                                 "c_bound_violations",
                                                 "queries_with_violations")}})
    exact.close()
    print(json.dumps({
        "case": "sweep (Table 1 analogue)",
        "config": {"workload": "c-approximate reverse k-ranks: |U|=1,000,000 |P|=100,000 d=200 "
                               "mixture (256 centres), 10,000 queries from P, k in {10,50,100}, "
                               "c=2, exact f-bounds; one batch of all queries per setting"},
        "rows": rows,
        "paper_context": "Table 1 of the paper: query time, overall ratio and memory at tau = "
                         "100/500/1000 on Amazon-Kindle, MovieLens and Netflix (real data, one "
                         "CPU thread per query)"}))


def cpu_baseline(w, pos, n_sample=None, q_sample=None):
    """The oracle on a user sample (all items), scaled by n / n_sample; queries of the
    approximate step on a query sample, scaled by nq / q_sample."""
    import oracle
    cores = os.cpu_count() or 1
    n_sample = n_sample or int(os.environ.get("RKR_CPU_USERS", "2000"))
    q_sample = q_sample or int(os.environ.get("RKR_CPU_QUERIES", "500"))
    rng = np.random.default_rng(0)
    users = np.sort(rng.choice(w.n, size=n_sample, replace=False))
    Us = np.ascontiguousarray(w.U[users])
    nq = w.Q.shape[0]
    t0 = time.perf_counter()
    ora = oracle.build_index(Us, w.P, w.tau, w.omega, w.s, pos)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    R = oracle.ranks(Us, w.P, w.Q)
    for q in range(nq):
        oracle.select_exact(R[:, q], min(int(w.k[q]), n_sample))
    t_exact = time.perf_counter() - t0
    qs = np.arange(q_sample)
    t0 = time.perf_counter()
    oracle.approx_query(ora, Us, w.Q[qs], np.minimum(w.k[qs], n_sample), C)
    t_approx = (time.perf_counter() - t0) * nq / q_sample
    step = (t_build + t_exact + t_approx) * w.n / n_sample
    return {"value": nq / step, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} of {w.n} users with all {w.m} items; approximate queries on "
                      f"{q_sample} of {nq} queries; scaled linearly to the full step",
            "seconds": {"build": t_build, "exact": t_exact, "approx_scaled": t_approx}}


def bench_reference(args):
    dist, rank, ws = _dist()
    if rank != 0:
        return
    w, pos = make_inputs()
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(cpu_baseline(w, pos, n_sample=400, q_sample=100))
    vals = vals[args.warmup:]
    value = statistics.mean(v["value"] for v in vals)
    cb = dict(vals[-1])
    cb["value"] = value
    out = {"impl": "reference", "metric": "queries/s", "value": value, "unit": "queries/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 * w.Q.shape[0] / value, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "c-approximate + exact reverse k-ranks, index build included: "
                                  "|U|=1,000,000 |P|=100,000 d=200, 10,000 queries (oracle "
                                  "on a user sample, scaled)"},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def approx_quality(ranks_c, off, best, c):
    """Quality of c-approximate answers against the exact ones (Def. 3; the
    accuracy and overall ratio of Section 5, "Criteria"), per query, aggregated.

    ranks_c: exact ranks of the users each approximate answer returned; best: the
    exact answer's ranks (the k smallest, ascending); off: per-query offsets of
    both.  Position i pairs the i-th smallest rank of the returned set with the
    i-th smallest rank overall.  Recall counts returned users whose rank is at
    most the k-th smallest; a c-bound violation is a returned user ranked above
    c times the k-th smallest rank."""
    ranks_c = np.asarray(ranks_c, np.float64)
    best = np.asarray(best, np.float64)
    nq = len(off) - 1
    acc = np.empty(nq)
    ratio = np.empty(nq)
    rec = np.empty(nq)
    viol = np.zeros(nq, np.int64)
    for q in range(nq):
        sl = slice(int(off[q]), int(off[q + 1]))
        got = np.sort(ranks_c[sl], kind="stable")
        b = best[sl]
        kth = b[-1]
        acc[q] = np.mean(got <= c * b)
        ratio[q] = np.mean(got / b)
        rec[q] = np.mean(got <= kth)
        viol[q] = int(np.sum(got > c * kth))
    worst = int(np.argmax(ratio)) if nq else -1
    return {"queries": nq, "accuracy": float(acc.mean()), "overall_ratio": float(ratio.mean()),
            "recall_at_k": float(rec.mean()), "c_bound_violations": int(viol.sum()),
            "queries_with_violations": int(np.sum(viol > 0)),
            "queries_below_accuracy_1": int(np.sum(acc < 1.0)),
            "worst_query": {"index": worst, "overall_ratio": float(ratio[worst]) if nq else None,
                            "accuracy": float(acc[worst]) if nq else None}}


def screen_precision(rkr, U, P, rows=256):
    """Error of the tensor-core screen against FP64 on a sample: the first `rows`
    users against every item, single and split products.  The FP64 reference is
    a float64 product of the float32 inputs on the GPU (its own rounding, about
    1e-16 relative, is far below the screen's)."""
    import torch
    Us = U[:rows].contiguous()
    ref = (Us.double() @ P.double().T).cpu().numpy()
    nu = torch.linalg.vector_norm(Us.double(), dim=1).cpu().numpy()
    npn = torch.linalg.vector_norm(P.double(), dim=1).cpu().numpy()
    scale = np.outer(nu, npn)
    out = {"sample": f"{rows} users x {P.shape[0]} items"}
    for name, split in (("single_bf16", False), ("split_bf16", True)):
        s_, b_ = rkr.rkr_screen_scores(Us, P, split=split)
        err = np.abs(s_.astype(np.float64) - ref)
        out[name] = {"max_abs_err": float(err.max()),
                     "max_rel_err": float((err / scale).max()),
                     "max_err_over_bound": float((err / b_.astype(np.float64)).max()),
                     "mean_bound_rel": float((b_ / scale).mean())}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="full",
                    choices=["full", "small", "learned", "latency", "sweep", "uneven"],
                    help="small: a 40k-user profiling case (no CPU baseline, no e2e); "
                         "learned: train the rank regressor and compare the learned cut "
                         "with the plain exact query")
    ap.add_argument("--tuning", default=None,
                    help='rkr_tuning fields as JSON (e.g. \'{"rc_seg_min": 4}\'), set before '
                         "the run; the line reports the tuning in effect")
    args = ap.parse_args()
    if args.tuning and args.impl == "ours":
        import paper_2504_13446_gb300 as rkr
        rkr.rkr_tuning_set(**json.loads(args.tuning))
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and args.impl == "ours":
        # one rank per GPU: load the build without cluster multicast
        os.environ["RKR_LIB_VARIANT"] = "replica"
        from paper_2504_13446_gb300 import buildlib
        buildlib.build(variant="replica")
    if args.impl == "reference":
        bench_reference(args)
    elif args.case == "learned":
        bench_learned(args)
    elif args.case == "latency":
        bench_latency(args)
    elif args.case == "sweep":
        bench_sweep(args)
    elif args.case == "uneven":
        bench_uneven(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
