"""Benchmark of the query-time hot path: APS search over a two-level index.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (seeded, synthetic): 1,000,000 x 128 FP32 vectors from a 1,000-component
Gaussian mixture (centres ~ N(0, I), sigma 1.5), a two-level index (1,000 leaf partitions under 32 parents,
10 Lloyd iterations), 10,000 queries per step whose component is Zipf(1.1),
L2, k = 10, APS with recall target 0.9 (raised in steps of 0.01 until mean
recall@10 against an FP64 brute force reaches 0.9).  One step = one search of
the 10,000 queries: root scoring, APS at both levels and the fused scan, all in
the library's kernels.  The arena (640 MB) is larger than L2, so no flush is
needed between steps.

With N > 1 (torchrun) every rank holds a replica of the index and searches its
own 10,000 queries: weak scaling, no collective on the data path.

--impl reference times the CPU oracle (FP64 numpy) on a bounded sample of the
same workload on the host cores.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time


def _impl_arg(argv):
    for i, a in enumerate(argv):
        if a == "--impl" and i + 1 < len(argv):
            return argv[i + 1]
        if a.startswith("--impl="):
            return a.split("=", 1)[1]
    return None


if _impl_arg(sys.argv) == "reference":
    # the reference arm times the oracle in this process on one BLAS thread ("cores": 1); the
    # variables must be set before numpy loads its BLAS
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_03437_b300 import synth  # noqa: E402

D, SIGMA, K = 128, 1.5, 10   # sigma 1.5: APS at target 0.9 needs ~24 of 1,000 partitions, as on Sift1M
ITERS, SEED = 10, 1234
N, N_COMP, NQ, N_LEAF, N_PARENT = 1_000_000, 1000, 10_000, 1000, 32   # set from the flags in main()
F_M_LEAF, F_M_PARENT = 0.1, 0.25
METRIC = "QPS at recall@10>=0.9 vs FP64 brute force (APS, two-level index)"
WORKLOAD = "aps_search_1Mx128_1000leaf_32parent_10kq_zipf1.1_k10"
ORACLE_BUILD_ITERS = 3   # Lloyd iterations of the index the CPU-baseline leg searches
STORAGE = "f32"


# DRAM traffic of one aps_search_kernel launch on the full workload, from the
# single-pass ncu capture summarised in profiles/aps_search_kernel_aps_1Mx128.md
# (dram__bytes_read.sum + dram__bytes_write.sum).  It belongs to the kernel
# sources with this hash; once they change the figure is no longer reported.
TRAFFIC_BYTES = 120.52e9 + 0.411e9
TRAFFIC_KERNEL_HASH = "bfca0f4e553054f7"
KERNEL_SOURCES = ["search_impl.cuh", "common.cuh", "capvol.cuh", "index.cuh"]
# DRAM traffic of the grouped scans of one batched APS step on the full workload
# (its four launches, one per round, summed: the lane-split layout in round 1,
# whole rows after it), from the single-pass ncu capture summarised in
# profiles/aps_batch_launches_1Mx128.md, with tiles (2, 64, 4096, 2) as the
# autotuner picks them; it belongs to these sources with this hash.
SCAN_TRAFFIC_BYTES = (457.54 + 7.10 + 546.75 + 33.38 + 0.218 + 0.217) * 1e6
SCAN_TRAFFIC_HASH = "f0470d2c84a97926"
SCAN_SOURCES = ["grouped.cuh", "common.cuh", "index.cuh", "aps_batch.cu"]


def kernel_hash(sources=None):
    import hashlib
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2506_03437_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    def __init__(self, gpu):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def gt_fp64(torch, Xd, Qd, k, chunk=512):
    """Exact top-k by FP64 brute force on the device (evaluation only)."""
    X64 = Xd.double()
    xn = (X64 * X64).sum(1)
    outD = torch.empty((Qd.shape[0], k), dtype=torch.float64, device=Xd.device)
    for s in range(0, Qd.shape[0], chunk):
        Q64 = Qd[s:s + chunk].double()
        Dm = (Q64 * Q64).sum(1, keepdim=True) - 2.0 * (Q64 @ X64.T) + xn[None, :]
        v, _ = torch.topk(Dm, k, dim=1, largest=False, sorted=True)
        outD[s:s + chunk] = v
        del Dm
    return outD, X64


def recall(torch, X64, Qd, ids, gtD, k, rtol=1e-5):
    """Recall@k with distance ties counted (a returned id within the k-th GT distance)."""
    Q64 = Qd.double()
    ok = ids >= 0
    rows = X64[ids.clamp(min=0)]
    dist = ((rows - Q64[:, None, :]) ** 2).sum(-1)
    kth = gtD[:, k - 1]
    thr = kth + rtol * kth.abs() + rtol
    hit = ok & (dist <= thr[:, None])
    return (hit.sum(1).double() / k).mean().item()


def max_over_ranks(values, world, device):
    """Every rank's timings replaced by their maximum over the ranks (the job ends with the
    slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(units_per_rank, world, seconds):
    """Units of all ranks (each rank processes its own units_per_rank) per second."""
    return world * units_per_rank / seconds


def rank_queries(rank):
    """The queries of one rank: rank 0 searches the workload's own queries, rank r > 0 an
    independent batch from the same mixture (weak scaling, no shared data path)."""
    if rank == 0:
        return synth.aps_queries(1236, D, N_COMP, SIGMA, NQ)
    return synth.aps_queries(1236, D, N_COMP, SIGMA, NQ, stream=rank)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2506_03437_b300 import index as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    X, ids, Q = synth.aps_search(n=N, d=D, n_comp=N_COMP, sigma=SIGMA, nq=NQ)
    if rank > 0:   # each rank searches its own queries from the same mixture
        Q = rank_queries(rank)
    Xd = torch.from_numpy(X).to(dev)
    idd = torch.from_numpy(ids).to(dev)
    Qd = torch.from_numpy(Q).to(dev)
    storage = {"f32": 0, "bf16": 1, "fp8": 2}[args.storage]
    ix = I.Index(D, n_leaf=N_LEAF, n_parent=N_PARENT, kmeans_iters=ITERS, seed=SEED,
                 f_M_leaf=F_M_LEAF, f_M_parent=F_M_PARENT, storage=storage, rerank=args.rerank)
    ix.set_search_upper(args.search_upper)
    t0 = time.time()
    ix.build(Xd, idd)
    torch.cuda.synchronize()
    build_s = time.time() - t0

    gtD, X64 = gt_fp64(torch, Xd, Qd, K)
    stream = torch.cuda.current_stream()

    # recall target: 0.9, raised by 0.01 until mean recall@10 >= 0.9
    tau = 0.90
    while True:
        oi, od, on, orr = ix.search(Qd, K, recall_target=tau, stream=stream)
        ix.check(stream)
        bad = int(((oi < -1) | (oi >= N)).sum().item())
        if bad:
            raise RuntimeError(f"search returned {bad} out-of-range ids")
        rec = recall(torch, X64, Qd, oi, gtD, K)
        if rec >= 0.9 or tau >= 0.999:
            break
        tau = round(tau + 0.01, 2)
    mean_nprobe = on.double().mean().item()
    # the fixed-nprobe path for comparison: the smallest nprobe whose mean recall@10 is >= 0.9
    fixed = None
    if not args.no_fixed:
        lo, hi = 1, N_LEAF
        while lo < hi:
            mid = (lo + hi) // 2
            fi, _, _, _ = ix.search(Qd, K, recall_target=0.0, nprobe=mid, stream=stream)
            if recall(torch, X64, Qd, fi, gtD, K) >= 0.9:
                hi = mid
            else:
                lo = mid + 1
        fo = ix.search(Qd, K, recall_target=0.0, nprobe=lo, stream=stream)
        frec = recall(torch, X64, Qd, fo[0], gtD, K)
        for _ in range(args.warmup):
            ix.search(Qd, K, recall_target=0.0, nprobe=lo, out=fo, stream=stream)
        fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for a_, b_ in fev:
            a_.record(stream)
            ix.search(Qd, K, recall_target=0.0, nprobe=lo, out=fo, stream=stream)
            b_.record(stream)
        torch.cuda.synchronize()
        fs = sum(a_.elapsed_time(b_) for a_, b_ in fev) / 1e3 / args.steps
        fixed = {"nprobe": lo, "recall_at_10": round(frec, 4), "value": round(NQ / fs, 1), "unit": "queries/s",
                 "ms_per_step": round(1e3 * fs, 4)}
    del X64

    sizes0, _, _ = ix.export_level(0)
    sizes1, _, _ = ix.export_level(1)
    # the per-query kernel (one CTA per query runs Algorithm 1 alone), for comparison
    out = (oi, od, on, orr)
    for _ in range(args.warmup):
        ix.search(Qd, K, recall_target=tau, out=out, stream=stream)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for a_, b_ in pev:
        a_.record(stream)
        ix.search(Qd, K, recall_target=tau, out=out, stream=stream)
        b_.record(stream)
    torch.cuda.synchronize()
    pq_s = sum(a_.elapsed_time(b_) for a_, b_ in pev) / 1e3 / args.steps
    per_query = {"value": round(NQ / pq_s, 1), "unit": "queries/s", "ms_per_step": round(1e3 * pq_s, 4),
                 "kernel": "aps_search_kernel, one CTA per query"}

    # the hot path: batched APS (the same decisions and results, the leaf scans
    # of all queries grouped by partition)
    batched = args.storage == "f32"
    tiles = None
    if batched:
        plan = I.ApsBatchPlan(ix, NQ, K, rounds=args.rounds)
        bout = plan.outputs(Qd)
        if args.tiles:
            tiles = tuple(int(x) for x in args.tiles.split(","))
            plan.set_tiles(*tiles)
        else:
            tiles = plan.autotune(Qd, tau, out=bout, reps=2, stream=stream)

        def step(q_, o_=None):
            plan.search(q_, tau, out=bout if o_ is None else o_, stream=stream)
    else:   # low-precision storage: the per-query kernel is the path
        plan, bout = None, out

        def step(q_, o_=None):
            ix.search(q_, K, recall_target=tau, out=bout if o_ is None else o_, stream=stream)
    step(Qd)
    torch.cuda.synchronize()
    same = {"ids": float((bout[0] == oi).all(dim=1).float().mean().item()),
            "nprobe": float((bout[2] == on).float().mean().item())}
    for _ in range(args.warmup):
        step(Qd)
    torch.cuda.synchronize()
    ix.hits(0, reset=True)
    ix.hits(1, reset=True)
    if plan:
        plan.set_timing(True)
    peak, peak_kind = peaks()
    # the K steps back to back on one stream, between two events; the library's
    # stage events time the last step's kernels (scan, prepare, replay, grouping)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        ev[0].record(stream)
        for i in range(args.steps):
            step(Qd)
        ev[1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if plan:
        stages = plan.stage_times()
        scan_ms = [stages["scan"]] * args.steps
        plan.set_timing(False)
        a_items, t_items = plan.round_stats()
    else:
        stages, scan_ms, a_items, t_items = {}, [], np.zeros(0, np.int64), np.zeros(0, np.int64)
    ix.check(stream)
    dev_s = ev[0].elapsed_time(ev[1]) / 1e3
    if world > 1:
        dist.barrier()
    h0 = ix.hits(0)
    h1 = ix.hits(1)
    pairs_first = None
    if plan:   # (evaluation only, after the hit counts are read) the first round's pairs
        s0 = plan.search(Qd, tau, cap0=1, stream=stream)[4]
        torch.cuda.synchronize()
        first = s0[:, 0].cpu().numpy()
        pairs_first = int(sizes0[first[first >= 0]].sum())
    eb = {"f32": 4, "bf16": 2, "fp8": 1}[args.storage]
    bytes_unique, bytes_items = algorithmic_bytes(h0, h1, sizes0, sizes1, eb, args.steps, 0)
    avg_step_s = dev_s / args.steps
    # the grouped scan, the dominant kernel: 2 FP32 instructions (subtract, fused
    # multiply-add) per element of every (query, row) pair of the items Algorithm 1 took in
    pairs = float((h0 * sizes0).sum()) / args.steps
    scan_s = sum(scan_ms) / 1e3 / args.steps if plan else None
    clock_mhz = clk.summary().get("sm_max_mhz") or 2032.0
    peak_ops = 148 * 128 * clock_mhz * 1e6 / 1e12

    # end to end: pinned host queries copied in, the batch, results copied out, every step
    Qh = torch.from_numpy(Q).pin_memory()
    oh = (torch.empty((NQ, K), dtype=torch.int64).pin_memory(), torch.empty((NQ, K), dtype=torch.float32).pin_memory(),
          torch.empty(NQ, dtype=torch.int32).pin_memory(), torch.empty(NQ, dtype=torch.float32).pin_memory())
    # Two query and two result buffers: a second stream copies step i + 1's
    # queries in and step i's results out while step i runs, so every step
    # still moves its own bytes both ways inside the timed region.
    qbuf = [torch.empty_like(Qd), torch.empty_like(Qd)]
    obuf = [tuple(torch.empty_like(t_) for t_ in bout[:4]), tuple(torch.empty_like(t_) for t_ in bout[:4])]
    xs = torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_run = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_run(n):
        with torch.cuda.stream(xs):
            qbuf[0].copy_(Qh, non_blocking=True)
            ev_in[0].record(xs)
        for i in range(n):
            j = i % 2
            stream.wait_event(ev_in[j])
            if i >= 2:
                stream.wait_event(ev_out[j])   # step i - 2's results are out of this buffer
            step(qbuf[j], obuf[j])
            ev_run[j].record(stream)
            with torch.cuda.stream(xs):
                if i + 1 < n:
                    if i >= 1:
                        xs.wait_event(ev_run[1 - j])   # step i - 1 has read that query buffer
                    qbuf[1 - j].copy_(Qh, non_blocking=True)
                    ev_in[1 - j].record(xs)
                xs.wait_event(ev_run[j])
                for h_, d_ in zip(oh, obuf[j]):
                    h_.copy_(d_, non_blocking=True)
                ev_out[j].record(xs)
    e2e_run(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_run(args.steps)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_same = bool((oh[0] == bout[0].cpu()).all().item())

    dev_s, e2e_s = max_over_ranks([dev_s, e2e_s], world, dev)
    qps = whole_job_rate(NQ * args.steps, world, dev_s)
    e2e_qps = whole_job_rate(NQ * args.steps, world, e2e_s)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(qps, 1), "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dev_s / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "bf16": "bf16 storage, f32 accumulate + f32 re-rank",
                      "fp8": "fp8-e4m3 storage, f32 accumulate + f32 re-rank"}[args.storage],
            "data": "synthetic (seeded Gaussian mixture; stands in for Sift1M-shaped data)",
            "config": {"workload": WORKLOAD, "n": N, "d": D, "n_leaf": N_LEAF, "n_parent": N_PARENT,
                       "queries_per_step": NQ, "k": K, "recall_target": tau, "recall_at_10": round(rec, 4),
                       "fixed_nprobe_path": fixed, "per_query_kernel": per_query,
                       "path": (f"batched APS, {args.rounds} rounds (qk_aps_batch_search)" if plan else
                                "per-query kernel (qk_search)"),
                       "tiles": ({"queries_per_warp": tiles[0], "tile_rows": tiles[1], "chunk_rows": tiles[2],
                                  "rows_per_thread": tiles[3] if len(tiles) > 3 else 0,
                                  "chosen_by": "flag" if args.tiles else "autotuner (qk_aps_batch_autotune)"}
                                 if tiles else None),
                       "same_as_per_query_kernel": same,
                       "stage_ms": {k_: (round(v_, 4) if isinstance(v_, float) else [round(x, 4) for x in v_])
                                    for k_, v_ in stages.items()},
                       "items_asked_per_round": a_items.tolist(), "items_taken_per_round": t_items.tolist(),
                       "pairs_first_round": pairs_first,
                       "mean_nprobe": round(mean_nprobe, 2), "f_M": [F_M_LEAF, F_M_PARENT],
                       "tau_rho": 0.01, "upper_recall": 0.99, "beta": "table", "build_s": round(build_s, 2),
                       "storage": args.storage, "rerank": args.rerank if args.storage != "f32" else None,
                       "l2": "no flush: 640 MB arena > 126 MB L2",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": round(e2e_qps, 1), "unit": "queries/s",
                    "h2d_bytes_per_step": NQ * D * 4,
                    "d2h_bytes_per_step": NQ * K * (8 + 4) + NQ * 8, "results_equal_device_run": e2e_same,
                    "copies": "pinned host buffers; a second stream copies step i+1's queries in and step i's "
                              "results out while step i runs"},
            # per step: the prepare kernel, the first replay, then per round the grouping,
            # the fill, the grouped scan and the replay
            "gpu_launches": args.steps * (2 + 4 * args.rounds) if plan else args.steps,
            "roofline": (scan_roofline(pairs, scan_s, peak_ops, bytes_unique, bytes_items, avg_step_s, peak,
                                       peak_kind) if plan else
                         roofline(bytes_unique, bytes_items, peak, peak_kind, avg_step_s)),
            "clocks": clk.summary(),
        }
        if args.serve_ops > 0 and world == 1:
            st, scfg, sclk = serve_stream(args.serve_ops, args.serve_load, args.server, args.update_wait,
                                          args.start, maintain_every=args.serve_ops)
            line["p50_ms"] = st["search"]["p50_ms"]
            line["p99_ms"] = st["search"]["p99_ms"]
            line["serving"] = {"config": scfg, "search_qps": st["search_qps"], "search": st["search"],
                               "recall_at_10_sample": st["recall_at_10_sample"],
                               "insert": st.get("insert"), "delete": st.get("delete"),
                               "maintenance_passes": st["maintenance_passes"],
                               "driver_lag_p99_ms": st["driver_lag_p99_ms"], "clocks": sclk,
                               "note": ("latency from each request's scheduled arrival to its completion, "
                                        "through the library's serving loop (qk_server_*)")}
            # the same sample at 90% of the saturation (the stream's second load level)
            st9, scfg9, sclk9 = serve_stream(args.serve_ops, 0.9, args.server, args.update_wait, args.start,
                                             maintain_every=args.serve_ops)
            line["serving"]["at_90pct_load"] = {
                "arrival_rate_ops": scfg9["arrival_rate_ops"], "search_qps": st9["search_qps"],
                "search": st9["search"], "insert": st9.get("insert"), "delete": st9.get("delete"),
                "recall_at_10_sample": st9["recall_at_10_sample"], "clocks": sclk9}
            if args.server == "native":   # the same sample with the slots' batched APS plans
                st2, scfg2, sclk2 = serve_stream(args.serve_ops, args.serve_load, args.server, args.update_wait,
                                                 args.start, maintain_every=args.serve_ops, batched_from=256)
                line["serving"]["with_batched_plans"] = {
                    "batched_from": 256, "saturation_qps": scfg2["saturation_qps"],
                    "arrival_rate_ops": scfg2["arrival_rate_ops"], "search_qps": st2["search_qps"],
                    "search": st2["search"], "insert": st2.get("insert"), "delete": st2.get("delete"),
                    "recall_at_10_sample": st2["recall_at_10_sample"],
                    "driver_lag_p99_ms": st2["driver_lag_p99_ms"], "clocks": sclk2}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(X, ids, Q, tau, args.cpu_seconds, workers=cpu_workers(args))
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def algorithmic_bytes(h0, h1, sizes0, sizes1, eb, steps, rerank):
    """Per-launch algorithmic bytes of the search (per item: s_p (d b + 8), rows and int64 ids).

    unique: every partition the launch touches, read once: the level-0 partitions with
      a hit (rows + ids), the touched parents' rows (leaf centroids + their int64 leaf
      ids), the top partition, the queries and the results.  The minimum traffic.
    items: every scanned (query, partition) item's rows + ids (the paper's effective
      scan rate, Sec. 8 "Scalability"), plus the same top partition, queries and results.
    Both add the FP32 re-rank rows of low-precision storage (rerank * k per query).
    h0/h1 are hit counts summed over `steps` identical launches."""
    row0 = D * eb + 8
    row1 = D * 4 + 8
    fixed = NQ * N_PARENT * D * 4 + NQ * D * 4 + NQ * K * 12 + NQ * min(1024, rerank * K) * D * 4
    unique = float(sizes0[h0 > 0].sum()) * row0 + float(sizes1[h1 > 0].sum()) * row1 + fixed
    items = (float((h0 * sizes0).sum()) * row0 + float((h1 * sizes1).sum()) * row1) / steps + fixed
    return unique, items


def scan_roofline(pairs, scan_s, peak_ops, bytes_unique, bytes_items, step_s, hbm_peak, hbm_kind):
    """Roofline of the grouped scan (grouped_scan_kernel), the dominant kernel of a
    batched APS step.  It is bound by FP32 issue: every (query, row) pair costs d
    subtractions and d fused multiply-adds on the FP32 lanes (148 SMs x 128 lanes
    x clock).  achieved = those instructions for the items Algorithm 1 took in,
    over the grouped scans' device time in the step (CUDA events around each
    scan launch, summed over the rounds).  The HBM figures of the whole step sit
    beside it: unique bytes (each touched partition once) and the per-item bytes
    of the paper's effective scan rate."""
    ops = 2.0 * pairs * D
    achieved = ops / scan_s / 1e12
    full = N == 1_000_000 and NQ == 10_000 and D == 128
    traffic = SCAN_TRAFFIC_BYTES if (full and kernel_hash(SCAN_SOURCES) == SCAN_TRAFFIC_HASH) else None
    extra = {}
    if traffic is not None:
        extra = {"dram_gbs": round(traffic / scan_s / 1e9, 1), "dram_frac": round(traffic / scan_s / 1e9 / hbm_peak, 4),
                 "reread_factor": round(traffic / bytes_unique, 2),
                 "traffic_note": "ncu DRAM read + write bytes of the step's grouped-scan launches, summed"}
    return {"bound": "alu", "kernel": "grouped_scan_rows_kernel + grouped_scan_kernel (the step's scans)",
            "achieved": round(achieved, 2),
            "peak": round(peak_ops, 2), "unit": "Tops/s", "frac": round(achieved / peak_ops, 4),
            "traffic": traffic, **extra, "peak_kind": "derived: 148 SMs x 128 FP32 lanes x max SM clock",
            "scan_ms_per_step": round(1e3 * scan_s, 4),
            "scan_timing": "library CUDA events around the scans of the last timed step", "pairs_per_step": round(pairs),
            "hbm": {"unique_gbs": round(bytes_unique / step_s / 1e9, 1),
                    "unique_frac": round(bytes_unique / step_s / 1e9 / hbm_peak, 4),
                    "effective_scan_gbs": round(bytes_items / step_s / 1e9, 1),
                    "effective_frac": round(bytes_items / step_s / 1e9 / hbm_peak, 4),
                    "peak": hbm_peak, "peak_kind": hbm_kind, "unique_bytes": round(bytes_unique),
                    "item_bytes": round(bytes_items)},
            "note": ("achieved counts 2 FP32 instructions per element of every scanned (query, row) pair; "
                     "hbm.unique counts every touched partition's rows and ids once per step, "
                     "hbm.effective every (query, partition) item's")}


def roofline(bytes_unique, bytes_items, peak, peak_kind, launch_s):
    """Roofline of aps_search_kernel.  achieved = the launch's unique algorithmic bytes
    (every touched partition once) over its duration, so frac <= 1 is a fraction of HBM;
    effective_scan_gbs counts every (query, partition) item's bytes, re-reads included;
    traffic is the ncu DRAM bytes of one launch when a capture of these kernel sources
    exists."""
    full = (N, NQ, N_LEAF, N_PARENT) == (1_000_000, 10_000, 1000, 32) and STORAGE == "f32"
    traffic = TRAFFIC_BYTES if (full and kernel_hash() == TRAFFIC_KERNEL_HASH) else None
    achieved = bytes_unique / launch_s / 1e9
    eff = bytes_items / launch_s / 1e9
    out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
           "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
           "unique_bytes": round(bytes_unique), "item_bytes": round(bytes_items),
           "effective_scan_gbs": round(eff, 1), "effective_frac": round(eff / peak, 4),
           "note": ("achieved = unique algorithmic bytes (each touched partition's rows and ids once) per "
                    "launch / launch time; effective_scan_gbs counts every scanned (query, partition) item, "
                    "so reads served from L2 count too; traffic = ncu DRAM bytes per launch")}
    if traffic is not None:
        out["dram_gbs"] = round(traffic / launch_s / 1e9, 1)
        out["dram_frac"] = round(traffic / launch_s / 1e9 / peak, 4)
        out["reread_factor"] = round(traffic / bytes_unique, 2)
    return out


def oracle_index(X, ids):
    from oracle import kmeans
    return kmeans.build_index(X, ids, N_LEAF, N_PARENT, iters=ORACLE_BUILD_ITERS, seed=SEED)


def cpu_workers(args):
    if args.cpu_workers >= 0:
        return args.cpu_workers
    from oracle import pool
    return min(64, pool.available_cores())


def cpu_baseline(X, ids, Q, tau, seconds, levels=None, workers=0):
    """The oracle's APS search timed on a bounded sample of the same queries: 1 host thread, and
    with workers > 1 also over that many processes (the queries split between them)."""
    from oracle import aps
    if levels is None:
        levels = oracle_index(X, ids)
    from oracle import pool
    prm = aps.Params(k=K, recall_target=tau, f_M=(F_M_LEAF, F_M_PARENT))
    rate1, done = pool.search_rate(levels, Q, prm, seconds, 1)
    out = {"value": round(rate1, 3), "unit": "queries/s", "cores": 1, "kind": "oracle",
           "sample": (f"first {done} of {Q.shape[0]} queries, FP64 numpy APS search in one spawned process on one "
                      f"BLAS thread, over an index the oracle built itself ({ORACLE_BUILD_ITERS} Lloyd iterations)")}
    if workers > 1:
        rate, n_done = pool.search_rate(levels, Q, prm, seconds, workers)
        out["parallel"] = {"value": round(rate, 3), "unit": "queries/s", "cores": workers, "kind": "oracle",
                           "sample": (f"{n_done} of {Q.shape[0]} queries split over {workers} spawned processes "
                                      f"(one BLAS thread each), at most {seconds:g} s each")}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    X, ids, Q = synth.aps_search(n=N, d=D, n_comp=N_COMP, sigma=SIGMA, nq=NQ)
    levels = oracle_index(X, ids)
    from oracle import aps
    prm = aps.Params(k=K, recall_target=0.9, f_M=(F_M_LEAF, F_M_PARENT))
    per_step = max(1, args.ref_queries)
    for w in range(args.warmup):
        aps.search(levels, Q[:1], prm)
    t0 = time.perf_counter()
    for s in range(args.steps):
        lo = (s * per_step) % NQ
        aps.search(levels, Q[lo:lo + per_step], prm)
    el = time.perf_counter() - t0
    qps = per_step * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": round(qps, 3), "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian mixture)",
            "config": {"workload": WORKLOAD, "n": N, "d": D, "n_leaf": N_LEAF, "n_parent": N_PARENT,
                       "queries_per_step": per_step, "k": K, "recall_target": 0.9},
            "cpu_baseline": {"value": round(qps, 3), "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} queries per step of the {NQ}-query batch"},
            "e2e": {"value": round(qps, 3), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_assign(args):
    """Tensor-core nearest-centroid assignment (k-means step of the build): 1M x 128 rows, 1,000 centroids."""
    import torch
    from paper_2506_03437_b300 import _lib as L
    torch.cuda.set_device(0)
    n, d, K = args.n, D, args.leaves
    X, _, _ = synth.aps_search(n=n, d=d, n_comp=max(1, n // 1000), sigma=SIGMA, nq=1)
    C = X[np.random.default_rng(SEED).choice(n, K, replace=False)].copy()
    Xd, Cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    idx = torch.empty((n, 1), dtype=torch.int32, device="cuda")
    dist = torch.empty((n, 1), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        L.check(L.lib.qk_nearest_centroids(Xd.data_ptr(), n, d, Cd.data_ptr(), K, 0, 1, idx.data_ptr(),
                                           dist.data_ptr(), stream.cuda_stream))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(0) as clk:
        for a, b in ev:
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
    s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    flops = 2.0 * n * K * d
    peak_bf16 = 1767.5
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    kind = "fallback"
    if os.path.exists(p):
        with open(p) as f:
            peak_bf16 = float(json.load(f)["bf16_tflops"])
        kind = "measured"
    peak_tf32 = peak_bf16 * (1.1 / 2.25)   # nominal TF32 / BF16 dense ratio
    tf = flops * args.steps / s / 1e12
    print(json.dumps({
        "metric": "rows assigned per second (tensor-core nearest centroid, exact FP32 re-score)",
        "value": round(n * args.steps / s, 1), "unit": "rows/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * s / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "tf32 operands, f32 accumulate",
        "data": "synthetic", "config": {"workload": f"nearest_centroid_{n}x{d}_K{K}", "n": n, "d": d, "K": K},
        "roofline": {"bound": "tensor", "achieved": round(tf, 1), "peak": round(peak_tf32, 1), "unit": "TFLOP/s",
                     "frac": round(tf / peak_tf32, 4), "traffic": None,
                     "peak_kind": f"{kind} bf16 burst x nominal tf32/bf16 ratio 1.1/2.25",
                     "note": "achieved counts the 2*n*K*d dot-product flops over the whole call "
                             "(GEMM, candidate selection and exact re-score)"},
        "clocks": clk.summary()}), flush=True)


def run_batch(args):
    """Batching workload: 5M x 256 rows in 20,000 Zipf(1.0)-sized partitions (10 to 100,000 rows),
    4,096 queries per launch, each with its own log-uniform nprobe in 1..500, k = 10.  One
    CUDA-graph replay of the batched search per step, tile shapes from the autotuner; compared
    with the per-query kernel in one launch and with a per-query launch loop."""
    import torch
    from paper_2506_03437_b300 import index as I
    torch.cuda.set_device(0)
    n, d, n_part, nq, k, np_hi = args.n_batch, 256, args.parts, 4096, 10, 500
    t0 = time.time()
    X, ids, lab, Q, nprobe = synth.zipf_partitions(n=n, d=d, n_part=n_part, nq=nq, nprobe_hi=np_hi)
    gen_s = time.time() - t0
    Xd, labd = torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda()
    sizes = np.bincount(lab, minlength=n_part)
    C = torch.zeros((n_part, d), dtype=torch.float64, device="cuda")
    for s in range(0, n, 1 << 20):   # FP64 partition means, rounded to FP32
        C.index_add_(0, labd[s:s + (1 << 20)], Xd[s:s + (1 << 20)].double())
    C = (C / torch.from_numpy(sizes).cuda().double()[:, None]).float()
    ix = I.Index(d, n_leaf=n_part, n_parent=0)
    ix.load(Xd, torch.from_numpy(ids).cuda(), leaf_centroids=C, leaf_of_row=labd.int())
    Qd, npd = torch.from_numpy(Q).cuda(), torch.from_numpy(nprobe).cuda()
    plan = I.BatchPlan(ix, nq, k, np_hi)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        if args.tiles:
            plan.tiles = tuple(int(x) for x in args.tiles.split(","))
            tiles = plan.tiles
        else:
            tiles = plan.autotune(Qd, npd, reps=1, stream=stream)
        # stage times of uncaptured runs (CUDA events between the steps)
        plan.set_timing(True)
        stages = []
        for _ in range(3):
            plan.search(Qd, npd, stream=stream)
            stages.append(plan.stage_times())
        plan.set_timing(False)
        stage_ms = {s: round(float(np.median([x[s] for x in stages])), 4) for s in stages[0]}
        out = (torch.empty((nq, k), dtype=torch.int64, device="cuda"),
               torch.empty((nq, k), dtype=torch.float32, device="cuda"))
        plan.capture(Qd, npd, out, stream)
        for _ in range(args.warmup):
            plan.replay(stream)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with Clocks(0) as clk:
            for a, b_ in ev:
                a.record(stream)
                plan.replay(stream)
                b_.record(stream)
            stream.synchronize()
        ix.check(stream)
        step_s = sum(a.elapsed_time(b_) for a, b_ in ev) / 1e3 / args.steps
        qps = nq / step_s
        # end to end: queries and nprobe from pinned host memory, results back, copies
        # timed.  Two plans, each with its graph over its own buffers, take the steps in
        # turn; a second stream copies step i + 1's inputs in and step i's results out
        # while step i runs.
        Qh, nph = torch.from_numpy(Q).pin_memory(), torch.from_numpy(nprobe).pin_memory()
        oh = (torch.empty((nq, k), dtype=torch.int64).pin_memory(), torch.empty((nq, k), dtype=torch.float32).pin_memory())
        plan2 = I.BatchPlan(ix, nq, k, np_hi)
        plan2.tiles = plan.tiles
        Qd2, npd2 = Qd.clone(), npd.clone()
        out2 = (torch.empty_like(out[0]), torch.empty_like(out[1]))
        plan2.capture(Qd2, npd2, out2, stream)
        P = [(plan, Qd, npd, out), (plan2, Qd2, npd2, out2)]
        xs = torch.cuda.Stream()
        ev_in, ev_run, ev_out = ([torch.cuda.Event(), torch.cuda.Event()] for _ in range(3))

        def e2e_run(n_):
            with torch.cuda.stream(xs):
                Qd.copy_(Qh, non_blocking=True)
                npd.copy_(nph, non_blocking=True)
                ev_in[0].record(xs)
            for i in range(n_):
                j = i % 2
                stream.wait_event(ev_in[j])
                if i >= 2:
                    stream.wait_event(ev_out[j])   # step i - 2's results are out of this buffer
                P[j][0].replay(stream)
                ev_run[j].record(stream)
                with torch.cuda.stream(xs):
                    if i + 1 < n_:
                        if i >= 1:
                            xs.wait_event(ev_run[1 - j])   # step i - 1 has read those inputs
                        P[1 - j][1].copy_(Qh, non_blocking=True)
                        P[1 - j][2].copy_(nph, non_blocking=True)
                        ev_in[1 - j].record(xs)
                    xs.wait_event(ev_run[j])
                    oh[0].copy_(P[j][3][0], non_blocking=True)
                    oh[1].copy_(P[j][3][1], non_blocking=True)
                    ev_out[j].record(xs)
        e2e_run(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_run(args.steps)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        e2e_same = bool((oh[0] == out[0].cpu()).all().item())
        # the per-query kernel (one CTA per query) in one launch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ix.search_nprobe(Qd, k, npd, stream=stream)
        e0.record(stream)
        pq = ix.search_nprobe(Qd, k, npd, stream=stream)
        e1.record(stream)
        stream.synchronize()
        perq_s = e0.elapsed_time(e1) / 1e3
        # a per-query launch loop on a sample
        m = args.loop_queries
        e0.record(stream)
        for j in range(m):   # nprobe from host memory: a device slice of it is not 16-byte aligned
            ix.search_nprobe(Qd[j:j + 1], k, nprobe[j:j + 1], stream=stream)
        e1.record(stream)
        stream.synchronize()
        loop_s = e0.elapsed_time(e1) / 1e3 / m
    same = float((pq[0] == out[0]).all(1).double().mean().item())
    # recall@10 against FP64 brute force on a sample of queries (evaluation only)
    ns = 256
    gtD, X64 = gt_fp64(torch, Xd, Qd[:ns], k)
    rec = recall(torch, X64, Qd[:ns], out[0][:ns], gtD, k)
    del X64
    # algorithmic work of the scan: every (query, partition) item's rows
    Cn = (C * C).sum(1)
    sel_rows, uniq = 0.0, torch.zeros(n_part, dtype=torch.bool, device="cuda")
    sz = torch.from_numpy(sizes).cuda()
    for s in range(0, nq, 512):
        Dq = Cn[None, :] - 2.0 * (Qd[s:s + 512] @ C.T)
        top = torch.topk(Dq, np_hi, dim=1, largest=False).indices
        mask = torch.arange(np_hi, device="cuda")[None, :] < npd[s:s + 512, None]
        sel_rows += float(sz[top][mask].double().sum().item())
        uniq[top[mask]] = True
    uniq_bytes = float(sz[uniq].double().sum().item()) * d * 4
    scan_s = stage_ms["scan"] / 1e3
    ops = sel_rows * d * 2.0                      # one subtract and one fused multiply-add per element
    clock_mhz = (clk.summary().get("sm_max_mhz") or 2032.0)
    peak_ops = 148 * 128 * clock_mhz * 1e6 / 1e12   # FP32 lanes x clock, Tops/s
    achieved = ops / scan_s / 1e12
    hbm_peak, hbm_kind = peaks()
    line = {
        "metric": "queries/s, batched fixed-nprobe search (4,096 queries, own nprobe each, k=10)",
        "value": round(qps, 1), "unit": "queries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * step_s, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (tf32 centroid scoring + exact f32 re-score)",
        "data": "synthetic (seeded Gaussian mixture, Zipf(1.0) partition sizes)",
        "config": {"workload": f"batch_{n}x{d}_{n_part}part_zipf1.0_{nq}q_nprobe1-{np_hi}_k{k}",
                   "n": n, "d": d, "partitions": n_part, "sizes_min_max": [int(sizes.min()), int(sizes.max())],
                   "queries": nq, "nprobe_mean": round(float(nprobe.mean()), 2), "k": k,
                   "tiles": {"queries_per_warp": tiles[0], "tile_rows": tiles[1], "chunk_rows": tiles[2],
                             "rows_per_thread": tiles[3], "chosen_by": "flag" if args.tiles else "autotuner"},
                   "stage_ms": stage_ms, "recall_at_10_vs_fp64": round(rec, 4),
                   "items": int(sum(min(int(x), n_part) for x in nprobe)), "rows_scanned": int(sel_rows),
                   "unique_partition_bytes": int(uniq_bytes),
                   "per_query_kernel": {"value": round(nq / perq_s, 1), "unit": "queries/s",
                                        "same_ids_fraction": round(same, 4)},
                   "per_query_launch_loop": {"value": round(1.0 / loop_s, 1), "unit": "queries/s",
                                             "sample": f"first {m} queries, one launch each"},
                   "l2": "no flush: 5.1 GB arena > 126 MB L2", "data_gen_s": round(gen_s, 1)},
        "e2e": {"value": round(nq / e2e_s, 1), "unit": "queries/s", "h2d_bytes_per_step": nq * d * 4 + nq * 4,
                "d2h_bytes_per_step": nq * k * 12, "results_equal_device_run": e2e_same,
                "copies": "pinned host buffers; two graphs take the steps in turn while a second stream "
                          "copies step i+1's inputs in and step i's results out"},
        "gpu_launches": 8 * args.steps,
        "roofline": {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak_ops, 2), "unit": "Tops/s",
                     "frac": round(achieved / peak_ops, 4), "traffic": None,
                     "peak_kind": f"148 SMs x 128 FP32 lanes x {clock_mhz:.0f} MHz",
                     "kernel": "grouped_scan_kernel", "kernel_ms": stage_ms["scan"],
                     "hbm_unique_gbs": round(uniq_bytes / scan_s / 1e9, 1), "hbm_peak": hbm_peak,
                     "hbm_peak_kind": hbm_kind,
                     "note": "achieved counts 2 FP32 operations (subtract, fused multiply-add) per element of "
                             "every scanned (query, row) pair; the scan reads each partition tile once per "
                             "group of queries, so its unique-byte rate is far below the HBM peak"},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(X, ids, lab, sizes, C.cpu().numpy(), Q, nprobe, k, args.cpu_seconds)
    print(json.dumps(line), flush=True)


def batch_cpu_baseline(X, ids, lab, sizes, C, Q, nprobe, k, seconds):
    """The oracle's per-query fixed-nprobe IVF search timed on a bounded sample (1 host thread)."""
    from oracle import aps, kmeans
    off = np.concatenate([[0], np.cumsum(sizes)])   # rows are grouped by partition already
    level = kmeans.Level(C, [X[off[j]:off[j + 1]] for j in range(len(sizes))],
                         [ids[off[j]:off[j + 1]] for j in range(len(sizes))])
    from oracle import pool
    rate, done = pool.ivf_rate(level, Q, k, nprobe, seconds, 1)
    return {"value": round(rate, 3), "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": (f"first {done} of {Q.shape[0]} queries, FP64 numpy per-query IVF in one spawned process on "
                       "one BLAS thread")}


def run_precision(args):
    """Precision workload: 10M x 768 unit-norm rows from 5,000 directions, inner product,
    100 parents over 10,000 leaves, batches of 1,024 queries, k = 100.  FP32, BF16 and FP8-E4M3
    (per-partition scale) storage, the low-precision forms with an FP32 re-rank of the top 4k.
    Each form is timed at the smallest recall target (from 0.9 in steps of 0.01) whose mean
    recall@10 against FP64 brute force is >= 0.9; recall@100 and the distance error of the
    returned results are reported beside it."""
    import torch
    from paper_2506_03437_b300 import _lib as L
    from paper_2506_03437_b300 import index as I
    torch.cuda.set_device(0)
    n, d, nq, k = args.n_prec, 768, 1024, 100
    n_leaf, n_parent = args.prec_leaves, args.prec_parents
    t0 = time.time()
    Xd, Qd = synth.unit_mixture_cuda(n=n, d=d, nq=nq, s=args.prec_spread)
    gen_s = time.time() - t0
    ids = torch.arange(n, dtype=torch.int64, device="cuda")
    # FP64 brute-force top-k by inner product (evaluation only)
    Q64 = Qd.double()
    best_s = torch.full((nq, k), -float("inf"), dtype=torch.float64, device="cuda")
    best_i = torch.full((nq, k), -1, dtype=torch.int64, device="cuda")
    for a in range(0, n, 1 << 20):
        S = Q64 @ Xd[a:a + (1 << 20)].double().T
        v, i = torch.topk(S, k, dim=1)
        cs, ci = torch.cat([best_s, v], 1), torch.cat([best_i, i + a], 1)
        v2, j = torch.topk(cs, k, dim=1)
        best_s, best_i = v2, torch.gather(ci, 1, j)
        del S
    gt10 = best_s[:, 9]
    gt100 = best_s[:, k - 1]
    torch.cuda.synchronize()
    gt_s = time.time() - t0 - gen_s

    def evaluate(oi, od):
        rows = Xd[oi.clamp(min=0)].double()
        sc = (rows * Q64[:, None, :]).sum(-1)                       # FP64 inner products of the results
        ok = oi >= 0
        tol10 = gt10 - 1e-5 * gt10.abs() - 1e-5
        tol100 = gt100 - 1e-5 * gt100.abs() - 1e-5
        r10 = ((sc[:, :10] >= tol10[:, None]) & ok[:, :10]).sum(1).double().mean().item() / 10
        r100 = ((sc >= tol100[:, None]) & ok).sum(1).double().mean().item() / k
        err = ((od.double() + sc).abs() / sc.abs().clamp(min=1e-12))[ok]   # dist = -<q, x>
        return r10, r100, err.max().item(), err.mean().item()

    stream = torch.cuda.current_stream()
    forms, cfg_base, assign = {}, None, None
    peak, peak_kind = peaks()
    with Clocks(0) as clk:
        for storage in args.prec_forms.split(","):
            st = {"f32": L.STORE_F32, "bf16": L.STORE_BF16, "fp8": L.STORE_FP8}[storage]
            ix = I.Index(d, metric=L.METRIC_IP, n_leaf=n_leaf, n_parent=n_parent, kmeans_iters=args.prec_iters,
                         seed=SEED, f_M_leaf=args.prec_fm, f_M_parent=F_M_PARENT, storage=st, rerank=4)
            ix.set_search_upper(args.search_upper)
            tb = time.time()
            if assign is None:
                ix.build(Xd, ids)
                s0, C0, i0 = ix.export_level(0)
                s1, C1, i1 = ix.export_level(1)
                lor = np.empty(n, np.int32)
                lor[i0] = np.repeat(np.arange(n_leaf, dtype=np.int32), s0)
                pol = np.empty(n_leaf, np.int32)
                pol[i1] = np.repeat(np.arange(n_parent, dtype=np.int32), s1)
                assign = (C0, lor, C1, pol)
            else:   # the same partitions, stored in another form
                ix.load(Xd, ids, leaf_centroids=assign[0], leaf_of_row=torch.from_numpy(assign[1]).cuda(),
                        parent_centroids=assign[2], parent_of_leaf=assign[3])
            torch.cuda.synchronize()
            build_s = time.time() - tb
            tau = 0.90
            while True:
                oi, od, on, orr = ix.search(Qd, k, recall_target=tau, stream=stream)
                ix.check(stream)
                r10, r100, emax, emean = evaluate(oi, od)
                if r10 >= 0.9 or tau >= 0.999:
                    break
                tau = round(tau + 0.01, 3)
            out = (oi, od, on, orr)
            for _ in range(args.warmup):
                ix.search(Qd, k, recall_target=tau, out=out, stream=stream)
            torch.cuda.synchronize()
            ix.hits(0, reset=True)
            ix.hits(1, reset=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for a_, b_ in ev:
                a_.record(stream)
                ix.search(Qd, k, recall_target=tau, out=out, stream=stream)
                b_.record(stream)
            torch.cuda.synchronize()
            ix.check(stream)
            s_step = sum(a_.elapsed_time(b_) for a_, b_ in ev) / 1e3 / args.steps
            h0, h1 = ix.hits(0), ix.hits(1)
            sz0, _, _ = ix.export_level(0)
            sz1, _, _ = ix.export_level(1)
            eb = {"f32": 4, "bf16": 2, "fp8": 1}[storage]
            bytes_step = (float((h0 * sz0).sum()) * d * eb + float((h1 * sz1).sum()) * d * 4) / args.steps \
                + nq * n_parent * d * 4 + (nq * 4 * k * d * 4 if storage != "f32" else 0)
            forms[storage] = {"qps": round(nq / s_step, 1), "ms_per_batch": round(1e3 * s_step, 4),
                              "recall_target": tau, "recall_at_10": round(r10, 4), "recall_at_100": round(r100, 4),
                              "dist_rel_err_max": emax, "dist_rel_err_mean": emean,
                              "mean_nprobe": round(float(on.double().mean().item()), 2),
                              "scan_gbs": round(bytes_step / s_step / 1e9, 1), "build_s": round(build_s, 1)}
            del ix, out, oi, od, on, orr
            torch.cuda.empty_cache()
    best = max(forms, key=lambda s: forms[s]["qps"])
    v = forms[best]
    line = {
        "metric": "QPS at recall@10>=0.9 vs FP64 brute force (inner product, k=100, BF16/FP8 storage + FP32 re-rank)",
        "value": v["qps"], "unit": "queries/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": v["ms_per_batch"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16 storage, f32 accumulate + f32 re-rank",
                  "fp8": "fp8-e4m3 storage, f32 accumulate + f32 re-rank"}[best],
        "data": "synthetic (seeded unit-norm mixture around 5,000 directions, generated on the GPU)",
        "config": {"workload": f"precision_{n}x{d}_ip_{n_parent}p_{n_leaf}l_{nq}q_k{k}", "n": n, "d": d,
                   "n_leaf": n_leaf, "n_parent": n_parent, "queries_per_batch": nq, "k": k,
                   "kmeans_iters": args.prec_iters, "best_form": best, "forms": forms,
                   "fp32_vs_best_speedup": round(v["qps"] / forms["f32"]["qps"], 3) if "f32" in forms else None,
                   "spread_s": args.prec_spread, "f_M": [args.prec_fm, F_M_PARENT],
                   "search_upper": args.search_upper,
                   "l2": "no flush: 30.7 GB FP32 arena > 126 MB L2", "data_gen_s": round(gen_s, 1),
                   "ground_truth_s": round(gt_s, 1)},
        "roofline": {"bound": "hbm", "achieved": v["scan_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": round(v["scan_gbs"] / peak, 4), "traffic": None, "peak_kind": peak_kind,
                     "kernel": "aps_search_kernel",
                     "note": "achieved counts every scanned (query, partition) item's stored rows, the parent level, "
                             "the root and the FP32 re-rank rows over the whole launch"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """Per-level recall targets on the APS workload (the synthetic counterpart of the paper's
    per-level sweep, Sec. 8): the index is built once; for every upper-level target tau_1 the same
    partitions are loaded with that target, and every leaf target tau_0 is timed.  Reports
    recall@10 against FP64 brute force, mean nprobe and queries/s for each pair."""
    import torch
    from paper_2506_03437_b300 import index as I
    torch.cuda.set_device(0)
    X, ids, Q = synth.aps_search(n=N, d=D, n_comp=N_COMP, sigma=SIGMA, nq=NQ)
    Xd, idd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(ids).cuda(), torch.from_numpy(Q).cuda()
    base = I.Index(D, n_leaf=N_LEAF, n_parent=N_PARENT, kmeans_iters=ITERS, seed=SEED,
                   f_M_leaf=F_M_LEAF, f_M_parent=F_M_PARENT)
    base.build(Xd, idd)
    s0, C0, i0 = base.export_level(0)
    s1, C1, i1 = base.export_level(1)
    lor = np.empty(N, np.int32)
    lor[i0] = np.repeat(np.arange(N_LEAF, dtype=np.int32), s0)
    pol = np.empty(N_LEAF, np.int32)
    pol[i1] = np.repeat(np.arange(N_PARENT, dtype=np.int32), s1)
    del base
    gtD, X64 = gt_fp64(torch, Xd, Qd, K)
    stream = torch.cuda.current_stream()
    grid = []
    with Clocks(0) as clk:
        for t1 in (0.8, 0.9, 0.95, 0.99, 1.0):
            ix = I.Index(D, n_leaf=N_LEAF, n_parent=N_PARENT, kmeans_iters=ITERS, seed=SEED,
                         f_M_leaf=F_M_LEAF, f_M_parent=F_M_PARENT, upper_recall=t1)
            ix.load(Xd, idd, leaf_centroids=C0, leaf_of_row=lor, parent_centroids=C1, parent_of_leaf=pol)
            for t0 in (0.8, 0.9, 0.95, 0.99):
                oi, od, on, orr = ix.search(Qd, K, recall_target=t0, stream=stream)
                rec = recall(torch, X64, Qd, oi, gtD, K)
                out = (oi, od, on, orr)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    ix.search(Qd, K, recall_target=t0, out=out, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                grid.append({"tau_1": t1, "tau_0": t0, "recall_at_10": round(rec, 4),
                             "mean_nprobe": round(on.double().mean().item(), 2), "qps": round(NQ / ms * 1e3, 1)})
            ix.check(stream)
            del ix
    # Early-termination comparators on the default upper target (tau_1 = 0.99), the
    # synthetic counterpart of Table 6, at recall targets 0.8, 0.9 and 0.95:
    #   fixed   the smallest nprobe whose mean recall@10 reaches the target;
    #   SPANN   the ratio rule (qk_search_ratio) with eps bisected to the smallest whose
    #           mean recall@10 reaches the target, as its threshold is tuned;
    #   oracle  each query's smallest nprobe whose own recall@10 reaches it (nprobe 1..64);
    #   APS     the grid's (0.99, target) entry.
    ix = I.Index(D, n_leaf=N_LEAF, n_parent=N_PARENT, kmeans_iters=ITERS, seed=SEED,
                 f_M_leaf=F_M_LEAF, f_M_parent=F_M_PARENT)
    ix.load(Xd, idd, leaf_centroids=C0, leaf_of_row=lor, parent_centroids=C1, parent_of_leaf=pol)
    kth = gtD[:, K - 1]
    thr = kth + 1e-5 * kth.abs() + 1e-5
    Q64 = Qd.double()

    def per_query_recall(fi):
        rows = X64[fi.clamp(min=0)]
        return ((fi >= 0) & (((rows - Q64[:, None, :]) ** 2).sum(-1) <= thr[:, None])).sum(1).double() / K

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return round(NQ / (e0.elapsed_time(e1) / args.steps) * 1e3, 1)

    per_n = {}
    for n_ in range(1, 65):
        fi, _, _, _ = ix.search(Qd, K, recall_target=0.0, nprobe=n_, stream=stream)
        per_n[n_] = per_query_recall(fi)
    table = []
    for target in (0.8, 0.9, 0.95):
        row = {"target": target}
        aps_g = next((g for g in grid if g["tau_1"] == 0.99 and g["tau_0"] == target), None)
        if aps_g:
            row["aps"] = {k_: aps_g[k_] for k_ in ("recall_at_10", "mean_nprobe", "qps")}
        fixed_np = next((n_ for n_ in range(1, 65) if per_n[n_].mean().item() >= target), None)
        if fixed_np:
            fo = ix.search(Qd, K, recall_target=0.0, nprobe=fixed_np, stream=stream)
            row["fixed"] = {"nprobe": fixed_np, "recall_at_10": round(per_n[fixed_np].mean().item(), 4),
                            "qps": timed(lambda: ix.search(Qd, K, recall_target=0.0, nprobe=fixed_np, out=fo,
                                                           stream=stream))}
        lo, hi = 1e-4, 4.0
        if per_query_recall(ix.search_ratio(Qd, K, hi, stream=stream)[0]).mean().item() >= target:
            for _ in range(24):
                mid = (lo * hi) ** 0.5
                if per_query_recall(ix.search_ratio(Qd, K, mid, stream=stream)[0]).mean().item() >= target:
                    hi = mid
                else:
                    lo = mid
            so = ix.search_ratio(Qd, K, hi, stream=stream)
            row["spann"] = {"eps": round(hi, 5), "mean_nprobe": round(so[2].double().mean().item(), 2),
                            "recall_at_10": round(per_query_recall(so[0]).mean().item(), 4),
                            "qps": timed(lambda: ix.search_ratio(Qd, K, hi, stream=stream))}
        oracle_np = torch.full((NQ,), 64, dtype=torch.int32, device="cuda")
        for n_ in range(64, 0, -1):
            oracle_np[per_n[n_] >= target] = n_
        oi, od = ix.search_nprobe(Qd, K, oracle_np, stream=stream)
        row["oracle"] = {"mean_nprobe": round(oracle_np.double().mean().item(), 2),
                         "recall_at_10": round(recall(torch, X64, Qd, oi, gtD, K), 4),
                         "qps": timed(lambda: ix.search_nprobe(Qd, K, oracle_np, out=(oi, od), stream=stream))}
        table.append(row)
        print(json.dumps({"early_termination": row}), file=sys.stderr, flush=True)
    best = max((g for g in grid if g["recall_at_10"] >= 0.9), key=lambda g: g["qps"], default=None)
    print(json.dumps({
        "metric": "per-level recall-target sweep (QPS and recall@10 per (tau_1, tau_0))",
        "value": best["qps"] if best else None, "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian mixture; stands in for Sift1M-shaped data)",
        "config": {"workload": WORKLOAD, "best_at_recall_0.9": best, "grid": grid,
                   "early_termination": table,
                   "note": "oracle nprobe is known only after the fact: a lower bound on the partitions any "
                           "early-termination rule must scan"},
        "clocks": clk.summary()}), flush=True)


def serving_recall(X, ids, ops, out_ids, k, frac=0.01, seed=1244, dev="cuda"):
    """(evaluation only) recall@k of a served stream's searches on a seeded 1% sample, against
    an FP64 brute force over the rows live when each sampled search arrived: the starting rows,
    plus the inserts and minus the deletes that precede it in the stream.  The server applies
    updates in groups (within the group wait), so a search may miss the last few milliseconds of
    updates; that staleness counts against the recall.  Returns (recall, sampled searches)."""
    import torch
    from paper_2506_03437_b300.serving import DELETE, INSERT, SEARCH
    q_ops = np.flatnonzero(ops.kind == SEARCH)
    g = np.random.default_rng(seed)
    pick = np.sort(g.choice(q_ops, size=max(1, int(round(frac * q_ops.size))), replace=False))
    ins = np.flatnonzero(ops.kind == INSERT)
    rows = np.concatenate([X, ops.vec[ins]]).astype(np.float32)
    row_ids = np.concatenate([ids, ops.ref[ins]]).astype(np.int64)
    born = np.concatenate([np.full(X.shape[0], -1, np.int64), ins.astype(np.int64)])   # op that made the row live
    died = np.full(rows.shape[0], np.iinfo(np.int64).max, np.int64)                      # op that deleted it
    order = np.argsort(row_ids, kind="stable")
    dels = np.flatnonzero(ops.kind == DELETE)
    at = np.clip(np.searchsorted(row_ids[order], ops.ref[dels]), 0, order.size - 1)
    ok = row_ids[order][at] == ops.ref[dels]          # stream ids are never reused
    died[order[at[ok]]] = dels[ok]
    A = torch.from_numpy(rows).to(dev, torch.float64)
    an = (A * A).sum(1)
    born_t, died_t = torch.from_numpy(born).to(dev), torch.from_numpy(died).to(dev)
    ids_t = torch.from_numpy(row_ids).to(dev)
    hits = 0
    for c in range(0, pick.size, 64):
        js = pick[c:c + 64]
        Qc = torch.from_numpy(ops.vec[js]).to(dev, torch.float64)
        dist = (Qc * Qc).sum(1, keepdim=True) - 2.0 * (Qc @ A.T) + an[None, :]
        jt = torch.from_numpy(js.astype(np.int64)).to(dev)[:, None]
        live = (born_t[None, :] < jt) & (died_t[None, :] > jt)
        dist = torch.where(live, dist, torch.full_like(dist, float("inf")))
        gt = ids_t[torch.topk(dist, k, dim=1, largest=False).indices].cpu().numpy()
        for r, j in enumerate(js):
            hits += len(set(gt[r].tolist()) & set(out_ids[j].tolist()))
    del A, an, born_t, died_t, ids_t
    if dev == "cuda":
        torch.cuda.empty_cache()
    return hits / (k * pick.size), int(pick.size)


def serve_stream(n_ops, load, server="native", update_wait=0.01, start=2_000_000, maintain_every=100_000,
                 batched_from=0, search_upper=-1):
    """The dynamic skewed stream of the serving workload (start 2M x 128 from 2,000
    components; 90% queries, 5% inserts, 5% deletes; Zipf(1.2) over a hot set of 100
    components rotating every 100,000 operations; maintenance every 100,000 operations),
    open-loop Poisson arrivals at `load` x the saturation rate measured by a closed burst.
    batched_from > 0 (native server): batches of that many searches or more run through the
    slots' batched APS plans.  Returns (latency summary, config, clocks)."""
    import torch
    from paper_2506_03437_b300 import index as I
    from paper_2506_03437_b300.serving import NativeServer, Server, skewed_stream
    if server == "native":
        def Srv(*a, **kw):
            return NativeServer(*a, batched_from=batched_from, **kw)
    else:
        Srv = Server
    n0, n_comp = start, 2000
    C = synth.mixture_centers(n_comp, D, 1240)
    X, _ = synth.mixture_samples(C, n0, SIGMA, 1241)
    ids = np.arange(n0, dtype=np.int64)
    n_leaf = int(round(n0 ** 0.5))
    ix = I.Index(D, n_leaf=n_leaf, n_parent=int(round(n_leaf ** 0.5)), kmeans_iters=ITERS, seed=SEED,
                 f_M_leaf=F_M_LEAF, f_M_parent=F_M_PARENT)
    ix.set_search_upper(search_upper)
    ix.build(torch.from_numpy(X).cuda(), torch.from_numpy(ids).cuda())
    # scan latency lambda(s) per (query, partition): 2 us + 45 ns per 128-d FP32 row, from the
    # search kernel's per-CTA scan rate measured by bench.py (about 11 GB/s per resident query)
    maint = dict(lam_sizes=[0, 100_000], lam_us=[2.0, 2.0 + 0.045 * 100_000], tau_us=0.25, alpha=0.9,
                 refine_radius=50, refine_iters=1, s_min=max(1, n0 // n_leaf // 8))
    print(f"serve: built {n0} x {D} ({n_leaf} leaves)", file=sys.stderr, flush=True)
    # saturation: a closed burst of queries
    burst = skewed_stream(C, ids, 20_000, SIGMA, 1242, p_query=1.0, p_insert=0.0, rate=None)
    srv = Srv(ix, D, k=K, recall_target=0.9, max_batch=2048, streams=4)
    sat = srv.run(burst)["search_qps"]
    sat = max(sat, srv.run(burst)["search_qps"])
    rate = load * sat / 0.9          # ops/s so that queries arrive at load x saturation
    ops = skewed_stream(C, ids, n_ops, SIGMA, 1243, rate=rate)
    srv = Srv(ix, D, k=K, recall_target=0.9, max_batch=2048, streams=4, maintain_every=maintain_every,
              maint_args=maint, update_wait_s=update_wait)
    with Clocks(0) as clk:
        st = srv.run(ops, keep_results=True)
    rec, n_s = serving_recall(X, ids, ops, srv.out_ids, K)
    st["recall_at_10_sample"] = {"value": round(rec, 4), "searches": n_s,
                                 "against": "FP64 brute force over the rows live at each search's arrival"}
    cfg = {"workload": f"serve_{n0}x{D}_{n_ops}ops", "start_vectors": n0, "ops": n_ops,
           "load": load, "saturation_qps": sat, "arrival_rate_ops": round(rate, 1),
           "update_wait_s": update_wait, "server": server, "maintain_every": maintain_every,
           "n_leaf": n_leaf, "streams": 4, "max_batch": 2048,
           "batched_from": batched_from if server == "native" else None}
    del ix
    torch.cuda.empty_cache()
    return st, cfg, clk.summary()


def run_serve(args):
    """The serving workload on the whole stream: reports p50/p99 latency and QPS."""
    import torch
    torch.cuda.set_device(0)
    st, cfg, clocks = serve_stream(args.ops, args.serve_load, args.server, args.update_wait, args.start,
                                   batched_from=args.serve_batched_from, search_upper=args.search_upper)
    line = {"metric": "serving p50/p99 latency and QPS (dynamic skewed stream)",
            "value": st["search_qps"], "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": round(1e3 * st["wall_s"], 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic skewed stream",
            "config": cfg, "latency": st, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="aps", choices=["aps", "assign", "serve", "batch", "precision", "sweep"],
                    help="aps: the APS search (default); assign: tensor-core nearest-centroid assignment; "
                         "serve: the continuous-batching request loop on a dynamic skewed stream")
    ap.add_argument("--ops", type=int, default=1_000_000, help="operations of the serving stream")
    ap.add_argument("--serve-load", type=float, default=0.5, help="query arrival rate / saturation")
    ap.add_argument("--serve-ops", type=int, default=100_000,
                    help="operations of the bounded serving sample in the default run (0: none)")
    ap.add_argument("--start", type=int, default=2_000_000, help="vectors in the index when the stream starts")
    ap.add_argument("--server", default="native", choices=["native", "python"],
                    help="the scheduler in the library (qk_server_*) or the Python loop of serving.py")
    ap.add_argument("--serve-batched-from", type=int, default=0,
                    help="serve workload: batches from this size run through batched APS plans (0: never)")
    ap.add_argument("--update-wait", type=float, default=0.01,
                    help="seconds the oldest pending update may wait before a group is applied")
    ap.add_argument("--n-batch", type=int, default=5_000_000, help="rows of the batching workload")
    ap.add_argument("--parts", type=int, default=20_000, help="partitions of the batching workload")
    ap.add_argument("--loop-queries", type=int, default=128, help="queries timed in the per-query launch loop")
    ap.add_argument("--n-prec", type=int, default=10_000_000, help="rows of the precision workload")
    ap.add_argument("--prec-leaves", type=int, default=10_000)
    ap.add_argument("--prec-parents", type=int, default=100)
    ap.add_argument("--prec-iters", type=int, default=5, help="Lloyd iterations of the precision index")
    ap.add_argument("--prec-spread", type=float, default=2.0,
                    help="noise s of the precision mixture: x = normalize(mu + s g / sqrt(d))")
    ap.add_argument("--prec-forms", default="f32,bf16,fp8", help="storage forms of the precision workload")
    ap.add_argument("--prec-fm", type=float, default=0.02, help="f_M of the leaf level (candidate fraction)")
    ap.add_argument("--search-upper", type=int, default=-1, choices=[-1, 0, 1],
                    help="qk_set_search_upper mode of the per-query search (aps and precision workloads): "
                         "-1 auto, 0 in each query's CTA, 1 prepare kernel")
    ap.add_argument("--tiles", default="", help="queries_per_warp,tile_rows,chunk_rows of the grouped scan "
                                                 "(aps and batch workloads) instead of the autotuner's choice")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-workers", type=int, default=-1,
                    help="processes of the parallel oracle leg (-1: the host's cores, at most 64; 0 or 1: skip)")
    ap.add_argument("--ref-queries", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fixed", action="store_true", help="skip the fixed-nprobe comparison of the APS workload")
    ap.add_argument("--n", type=int, default=1_000_000, help="vectors (smaller for profiling runs)")
    ap.add_argument("--nq", type=int, default=10_000, help="queries per step")
    ap.add_argument("--leaves", type=int, default=1000)
    ap.add_argument("--parents", type=int, default=32)
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "fp8"],
                    help="leaf storage: FP32, or BF16 / FP8 E4M3 with an FP32 re-rank of 4k candidates")
    ap.add_argument("--rerank", type=int, default=4)
    ap.add_argument("--rounds", type=int, default=4, help="rounds of the batched APS search")
    args = ap.parse_args()
    global N, N_COMP, NQ, N_LEAF, N_PARENT, WORKLOAD, STORAGE
    N, NQ, N_LEAF, N_PARENT = args.n, args.nq, args.leaves, args.parents
    STORAGE = args.storage
    N_COMP = max(1, N // 1000)
    if (N, NQ, N_LEAF, N_PARENT) != (1_000_000, 10_000, 1000, 32):
        WORKLOAD = f"aps_search_{N}x128_{N_LEAF}leaf_{N_PARENT}parent_{NQ}q_zipf1.1_k10"
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "assign":
        run_assign(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
