"""Benchmark: exact 1-NN queries/s and p50/p99 latency at 100M x 256 fp32.

Workload (default): 100M random-walk series of 256 points (fp32, generated on the
device from seed 0, ~102 GB resident in HBM), indexed with 16 segments and
cardinality 256, leaf capacity 2000; 100 queries: 50 fresh random walks (seed 1) and
50 collection members plus N(0, sigma^2) noise, sigma cycling 0.01 / 0.1 / 1 (ids and
noise from seed 2). One step answers the 100 queries (k = 1) in one msi_knn call on
a stream (the batched form); the plain form answers them one call and one wait at a
time and gives the p50/p99 latency.

Prints one JSON line. `--impl reference` times the CPU oracle (FP64 serial scan) on a
bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
METRIC = "exact 1-NN queries/s and p50/p99 ms at 100M x 256 fp32, batched vs plain"


MIXED_SEED = 4  # the mixed-shape collection


def workload(n_total, length, nq, k, leaf, kind="walks"):
    if kind == "mixed":
        return (f"{n_total // 1_000_000}M x {length} fp32 mixed shapes (seed {MIXED_SEED}: 50% noisy sinusoids, "
                f"50% Laplace-step walks with spike bursts), {nq} queries (fresh draws + N(0, 0.1) noise), k={k}, "
                f"16 segments, cardinality 256, leaf capacity {leaf}")
    return (f"{n_total // 1_000_000}M x {length} fp32 random walks (seed 0), {nq} queries (50% fresh walks, "
            f"50% noisy members), k={k}, 16 segments, cardinality 256, leaf capacity {leaf}")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default 100 for the headline, about 0.3 s of GPU time; 10 otherwise)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=100_000_000)
    p.add_argument("--len", type=int, default=256)
    p.add_argument("--queries", type=int, default=100)
    p.add_argument("--k", type=int, default=1)
    p.add_argument("--leaf", type=int, default=2000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=2_000_000, help="series in the oracle's timed sample")
    p.add_argument("--cpu-queries", type=int, default=10)
    p.add_argument("--serving", action="store_true", help="Poisson-arrival serving sweep over three collections")
    p.add_argument("--dtw", action="store_true", help="exact k-NN under DTW (window 10%%) on the same workload")
    p.add_argument("--query-slots", type=int, default=0,
                   help="concurrent query slots of the index (0: the autotuner's choice, default schedule 16)")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default batched schedule (the batched chain, groups of 128, share 4)")
    p.add_argument("--schedule", default="auto", choices=["auto", "chain", "dense", "slots"],
                   help="batched form: auto (the autotuner's choice), the batched chain with the iSAX filters, "
                        "the batched chain with the tensor-core filter, or query slots (no autotuning)")
    p.add_argument("--tune-reps", type=int, default=10, help="timed calls per schedule candidate of the autotuner")
    p.add_argument("--batch-order", action="store_true",
                   help="batched chain: refine each query's survivors in ascending lower-bound order")
    p.add_argument("--slot-capacity", type=int, default=0,
                   help="entries of each bounded query slot's candidate and survivor lists (0: the defaults)")
    p.add_argument("--workload", default="walks", choices=["walks", "mixed"],
                   help="random walks (the headline) or the mixed-shape family (use --n 60000000)")
    p.add_argument("--window", type=int, default=-1, help="DTW half-width (default len / 10)")
    p.add_argument("--serve-scale", type=float, default=1.0, help="collection sizes x this (serving mode)")
    p.add_argument("--rates", default="1000,3000,10000,30000,100000")
    p.add_argument("--serve-slots", type=int, default=8, help="query slots per collection (serving mode)")
    p.add_argument("--serve-requests", type=int, default=3000, help="most requests per rate")
    p.add_argument("--load-rates", default="5000,10000,15000",
                   help="offered Poisson rates (queries/s) of the under-load leg on the benchmark's collection "
                        "(empty: skip the leg)")
    p.add_argument("--load-requests", type=int, default=3000, help="requests per offered rate of the under-load leg")
    args = p.parse_args()
    if args.steps is None:
        args.steps = 10 if (args.dtw or args.serving or args.impl == "reference") else 100
    return args


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def bf16_peak():
    """Dense bf16 TFLOP/s, measured (burst) when the file holds it, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index=0):
        self.samples = []
        self._stop = threading.Event()
        self._index = index
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self._index), f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                vals = [v.strip() for v in out.stdout.strip().split(",")]
                if len(vals) == 6:
                    self.samples.append(vals)
            except Exception:
                pass
            self._stop.wait(0.05)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def cpu_baseline(args, length, n_total, seconds_budget=None):
    """The oracle's FP64 serial-scan 1-NN on a bounded sample of the workload: the
    first `cpu_sample` series (regenerated on the host) and `cpu_queries` queries of
    the same mix; time per query scaled to the full collection size."""
    import datagen
    import oracle
    ns = min(args.cpu_sample, n_total)
    mixed = getattr(args, "workload", "walks") == "mixed"
    X = datagen.mixed(MIXED_SEED, 0, ns, length) if mixed else datagen.walks(0, 0, ns, length)
    t0 = time.perf_counter()
    Z = oracle.summarise(X, 16, 256, want_paa=False)[0]
    t_sum = time.perf_counter() - t0
    if mixed:
        Q = datagen.mixed_queries(count=args.queries, length=length)[: args.cpu_queries]
    else:
        Q = datagen.paper_queries(n_total, length, count=args.queries)[: args.cpu_queries]
    t0 = time.perf_counter()
    for q in Q:
        oracle.knn_scan(Z, oracle.znorm(q)[0], args.k)
    t_scan = (time.perf_counter() - t0) / len(Q)
    per_query_full = t_scan * (n_total / ns)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    return {"value": 1.0 / per_query_full, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 serial scan of {ns} of the {n_total} series (regenerated on the host, z-normalised by "
                      f"the oracle in {t_sum:.2f} s) for {len(Q)} queries; {t_scan * 1e3:.1f} ms/query scaled "
                      f"x{n_total / ns:g} to the full collection"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    length = args.len
    times = []
    base = None
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        base = cpu_baseline(args, length, args.n)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = base["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.n, length, args.queries, args.k, args.leaf, args.workload),
                       "sample": base["sample"]},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def serving(args):
    """Continuous batching vs one query at a time, under Poisson arrivals: three
    resident random-walk collections (80M x 128, 40M x 256, 8M x 1024 at scale 1),
    each request targeting a uniform collection with k uniform in 1..100."""
    import random

    import torch

    import datagen
    import paper_2009_00786_gb300 as msi
    dev = torch.device("cuda:0")
    shapes = [(int(80e6 * args.serve_scale), 128), (int(40e6 * args.serve_scale), 256),
              (int(8e6 * args.serve_scale), 1024)]
    s = torch.cuda.Stream()
    cols, indexes, pools = [], [], []
    for ci, (n, length) in enumerate(shapes):
        X = torch.empty((n, length), dtype=torch.float32, device=dev)
        datagen.walks_device(10 + ci, 0, n, length, X.data_ptr(), s.cuda_stream)
        s.synchronize()
        cols.append(X)
        indexes.append(msi.msi_build(X, segments=16, cardinality=256, leaf_capacity=2000,
                                     flags=msi.MSI_BUILD_BORROW, query_slots=1))
        n_fresh, ids, sig = datagen.query_plan(n, 64, fresh_seed=20 + ci, pick_seed=30 + ci)
        pools.append(np.concatenate([datagen.walks(20 + ci, 0, n_fresh, length),
                                     datagen.noisy_copies(10 + ci, 30 + ci, ids, sig, length)]))
    rates = [float(r) for r in args.rates.split(",")]
    out = {"metric": "serving: exact k-NN queries/s and p50/p99 ms under Poisson arrivals, continuous batching "
                     "vs one query at a time",
           "unit": "queries/s", "data": "synthetic",
           "config": {"workload": " + ".join(f"{n // 1_000_000}M x {l}" for n, l in shapes) +
                      " fp32 random walks, k uniform in 1..100, uniform collection per request"},
           "rates": []}
    for name, opts in (("continuous", dict(slots_per_index=args.serve_slots)), ("one_at_a_time", dict(slots_per_index=1,
                                                                                        max_inflight=1))):
        srv = msi.Server(indexes, **opts)
        for rate in rates:
            rng = random.Random(int(rate))
            nreq = int(min(args.serve_requests, max(200, rate * 2)))
            t = 0.0
            plan = []
            for _ in range(nreq):
                t += rng.expovariate(rate)
                ci = rng.randrange(3)
                plan.append((t, ci, pools[ci][rng.randrange(64)], rng.randint(1, 100)))
            tickets = []
            t0 = time.perf_counter()
            for at, ci, q, k in plan:
                while time.perf_counter() - t0 < at:
                    pass
                tickets.append((srv.submit(ci, q, k), k))
            lat = [srv.wait(tk, k)[2] for tk, k in tickets]
            wall = time.perf_counter() - t0
            out["rates"].append({"server": name, "offered_qps": rate, "requests": nreq,
                                 "achieved_qps": nreq / wall, "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99)), **{f"srv_{kk}": v for kk, v in srv.stats().items()}})
            print(json.dumps(out["rates"][-1]), file=sys.stderr, flush=True)
        srv.close()
    print(json.dumps(out))


def under_load_leg(msi, index, pool, k, args):
    """Poisson arrivals at each offered rate through msi_server_* on the benchmark's
    index: continuous batching (16 slots) against one query at a time
    (max_inflight = 1). Each request is a query of the benchmark's mix; the latency of
    a request runs from its submission to its completion."""
    import random
    rates = [float(r) for r in args.load_rates.split(",") if r]
    out = []
    for name, opts in (("continuous", dict(slots_per_index=16)), ("one_at_a_time", dict(slots_per_index=1,
                                                                                         max_inflight=1))):
        srv = msi.Server([index], **opts)
        for q in pool[:8]:  # warm the slots
            srv.wait(srv.submit(0, q, k), k)
        for rate in rates:
            rng = random.Random(int(rate) + 17)
            plan, t = [], 0.0
            for _ in range(args.load_requests):
                t += rng.expovariate(rate)
                plan.append((t, pool[rng.randrange(len(pool))]))
            tickets = []
            t0 = time.perf_counter()
            for at, q in plan:
                while time.perf_counter() - t0 < at:
                    pass
                tickets.append(srv.submit(0, q, k))
            lat = [srv.wait(tk, k)[2] for tk in tickets]
            wall = time.perf_counter() - t0
            out.append({"server": name, "offered_qps": rate, "requests": len(plan), "achieved_qps": len(plan) / wall,
                        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))})
        srv.close()
    return out


def dtw_bench(args):
    """Exact k-NN under DTW (Section IV, MESSI with DTW) on the benchmark's collection
    and query mix: the same index, a Sakoe-Chiba window of 10% of the length."""
    import torch

    import datagen
    import oracle
    import paper_2009_00786_gb300 as msi
    dev = torch.device("cuda:0")
    n, length, nq, k = args.n, args.len, args.queries, args.k
    r = args.window if args.window >= 0 else length // 10
    stream = torch.cuda.Stream()
    X = torch.empty((n, length), dtype=torch.float32, device=dev)
    datagen.walks_device(0, 0, n, length, X.data_ptr(), stream.cuda_stream)
    n_fresh, ids, sig = datagen.query_plan(n, nq)
    Q = torch.empty((nq, length), dtype=torch.float32, device=dev)
    datagen.walks_device(1, 0, n_fresh, length, Q.data_ptr(), stream.cuda_stream)
    ids_d, sig_d = torch.from_numpy(ids).to(dev), torch.from_numpy(sig).to(dev)
    datagen.noisy_copies_device(0, 2, ids_d.data_ptr(), sig_d.data_ptr(), nq - n_fresh, length,
                                Q[n_fresh:].data_ptr(), stream.cuda_stream)
    stream.synchronize()
    index = msi.msi_build(X, segments=16, cardinality=256, leaf_capacity=args.leaf, flags=msi.MSI_BUILD_BORROW,
                          stream=stream)
    for _ in range(args.warmup):
        msi.msi_knn_dtw(index, Q, k, window=r, stream=stream)
    stream.synchronize()
    msi.msi_query_stats_get(index, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            msi.msi_knn_dtw(index, Q, k, window=r, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1)
    st = msi.msi_query_stats_get(index, reset=True)
    lat = []
    qe0, qe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(nq):
        qe0.record(stream)
        msi.msi_knn_dtw(index, Q[i:i + 1], k, window=r, stream=stream)
        qe1.record(stream)
        qe1.synchronize()
        lat.append(qe0.elapsed_time(qe1))
    # the oracle's FP64 DTW scan on a bounded sample, scaled to the collection
    ns = min(args.cpu_sample // 10, n)
    Z = oracle.summarise(datagen.walks(0, 0, ns, length), 16, 256, want_paa=False)[0]
    Qh = Q[: args.cpu_queries // 2].cpu().numpy()
    t0 = time.perf_counter()
    for q in Qh:
        oracle.knn_scan_dtw(Z, oracle.znorm(q)[0], k, r)
    t_scan = (time.perf_counter() - t0) / len(Qh)
    line = {
        "metric": f"exact {k}-NN DTW queries/s and p50/p99 ms at {n // 1_000_000}M x {length} fp32 "
                  f"(Sakoe-Chiba window {r})",
        "value": nq * args.steps / (ms / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload(n, length, nq, k, args.leaf) + f", DTW window {r}"},
        "plain": {"qps": nq / (sum(lat) / 1e3), "p50_ms": float(np.percentile(lat, 50)),
                  "p99_ms": float(np.percentile(lat, 99))},
        "gpu_launches": st["kernel_launches"],
        "work_per_query": {kk: v / max(1, st["queries"]) for kk, v in st.items() if not kk.endswith("_ms")},
        "clocks": clocks.summary(),
        "cpu_baseline": {"value": 1.0 / (t_scan * n / ns), "unit": "queries/s",
                         "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())), "kind": "oracle",
                         "sample": f"FP64 DTW scan of {ns} of the {n} series for {len(Qh)} queries; "
                                   f"{t_scan * 1e3:.1f} ms/query scaled x{n / ns:g}"},
    }
    index.close()
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.serving:
        serving(args)
        return
    if args.dtw:
        dtw_bench(args)
        return
    import torch
    import torch.distributed as dist

    import datagen
    import paper_2009_00786_gb300 as msi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, length, nq, k = args.n, args.len, args.queries, args.k
    stream = torch.cuda.Stream(device=dev)

    # ---- collection (this rank's shard of the weak-scaled job) and queries, in HBM
    first_id = rank * n
    X = torch.empty((n, length), dtype=torch.float32, device=dev)
    if args.workload == "mixed":
        datagen.mixed_device(MIXED_SEED, first_id, n, length, X.data_ptr(), stream.cuda_stream)
        Q = torch.from_numpy(datagen.mixed_queries(count=nq, length=length)).to(dev)
    else:
        datagen.walks_device(0, first_id, n, length, X.data_ptr(), stream.cuda_stream)
        n_fresh, ids, sig = datagen.query_plan(n, nq)
        Q = torch.empty((nq, length), dtype=torch.float32, device=dev)
        datagen.walks_device(1, 0, n_fresh, length, Q.data_ptr(), stream.cuda_stream)
        ids_d = torch.from_numpy(ids).to(dev)
        sig_d = torch.from_numpy(sig).to(dev)
        datagen.noisy_copies_device(0, 2, ids_d.data_ptr(), sig_d.data_ptr(), nq - n_fresh, length,
                                    Q[n_fresh:].data_ptr(), stream.cuda_stream)
    stream.synchronize()

    # ---- build (timed once; the collection is borrowed in place)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        b0.record(stream)
        index = msi.msi_build(X, segments=16, cardinality=256, leaf_capacity=args.leaf, flags=msi.MSI_BUILD_BORROW,
                              stream=stream, query_slots=args.query_slots, slot_capacity=args.slot_capacity)
        b1.record(stream)
    stream.synchronize()
    build_ms = b0.elapsed_time(b1)

    out_ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    out_d = torch.empty((nq, k), dtype=torch.float32, device=dev)

    # ---- the batched schedule (query slots x grid share), chosen by the library's
    # autotuner before the warm-up (answers do not depend on it), on a query set of the
    # same mix drawn from other seeds than the timed queries
    if args.workload == "mixed":
        Qt = torch.from_numpy(datagen.mixed_queries(count=nq, length=length, query_seed=7, noise_seed=8)).to(dev)
    else:
        Qt = torch.from_numpy(datagen.paper_queries(n, length, count=nq, data_seed=0, fresh_seed=7,
                                                    pick_seed=8)).to(dev) if first_id == 0 else Q
    if args.query_slots or args.schedule == "slots":
        msi.msi_schedule_set(index, batch_chain=0)
    elif args.schedule in ("chain", "dense"):
        msi.msi_schedule_set(index, batch_chain=1, batch_group=min(128, nq), batch_share=4,
                             batch_dense=1 if args.schedule == "dense" else 0)
    if args.batch_order:
        msi.msi_schedule_set(index, batch_order=1)
    schedule = dict(msi.msi_schedule_get(index), autotuned=False)
    if not args.no_autotune and not args.query_slots and args.schedule == "auto":
        tr = msi.msi_autotune(index, Qt, k, reps=args.tune_reps, stream=stream)
        schedule = {"batch_chain": tr["batch_chain"], "batch_group": tr["batch_group"],
                    "batch_share": tr["batch_share"], "batch_dense": tr["batch_dense"], "query_slots": tr["query_slots"],
                    "grid_share": tr["grid_share"], "autotuned": True,
                    "candidates": tr["candidates"], "tuned_qps": tr["queries_per_s"],
                    "untuned_schedule_qps": tr["default_queries_per_s"],
                    "tuning_queries": "a disjoint set of the same mix (seeds 7 and 8)"}

    def step():
        if world > 1:  # answers over every rank's shard, merged by (FP64 distance, id)
            from paper_2009_00786_gb300 import shard
            shard.sharded_knn(index, Q, k, first_id)
        else:
            msi.msi_knn(index, Q, k, out_ids, out_d, stream=stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    msi.msi_query_stats_get(index, reset=True)

    # ---- timed region: K batched steps
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # an event after every step: a query of the batched form is answered when its
    # call completes, so its latency is its call's (from the call's start on the
    # stream to its completion)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        e0.record(stream)
        for i in range(args.steps):
            step()
            step_ev[i].record(stream)
        e1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    call_lat = [e0.elapsed_time(step_ev[0])] + [step_ev[i - 1].elapsed_time(step_ev[i])
                                                 for i in range(1, args.steps)]
    timed_launches = msi.msi_query_stats_get(index)["kernel_launches"]  # counted by the library
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
        dist.barrier()
    qps = nq * args.steps / (elapsed_ms / 1e3)  # queries answered over the whole (sharded) collection

    # ---- plain form: one call and one wait per query, for p50 / p99
    lat = []
    qe0, qe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(nq):
        qe0.record(stream)
        msi.msi_knn(index, Q[i:i + 1], k, out_ids[i:i + 1], out_d[i:i + 1], stream=stream)
        qe1.record(stream)
        qe1.synchronize()
        lat.append(qe0.elapsed_time(qe1))
    plain_qps = nq / (sum(lat) / 1e3)

    # ---- under load: Poisson arrivals through the serving loop on this collection,
    # continuous batching against one query at a time
    under_load = under_load_leg(msi, index, Q.cpu().numpy(), k, args) if (args.load_rates and world == 1) else None

    # ---- end to end: host queries in, host results out, through the C ABI
    Qh = torch.empty((nq, length), dtype=torch.float32, pin_memory=True)
    Qh.copy_(Q.cpu())
    ids_h = torch.empty((nq, k), dtype=torch.int64, pin_memory=True)
    d_h = torch.empty((nq, k), dtype=torch.float32, pin_memory=True)
    msi.msi_knn(index, Qh, k, ids_h, d_h, stream=stream)
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    for _ in range(args.steps):
        msi.msi_knn(index, Qh, k, ids_h, d_h, stream=stream)
    ee1.record(stream)
    ee1.synchronize()
    e2e_qps = nq * args.steps / (ee0.elapsed_time(ee1) / 1e3)

    # ---- refinement kernels, timed with CUDA events recorded on the query stream
    batched_st = msi.msi_query_stats_get(index, reset=True)  # the timed and end-to-end batched steps
    msi.msi_set_timing(index, True)
    step()
    stream.synchronize()
    msi.msi_set_timing(index, False)
    st = msi.msi_query_stats_get(index, reset=True)
    launches = max(1, st["refine_launches"])
    main_refined = st["series_refined"] - st["seed_series"]
    sched = msi.msi_schedule_get(index)
    wf = msi.msi_index_info_get(index)["fine_segments"]
    peak, peak_kind = peaks()
    filt_s = st["filter_ms"] / launches / 1e3
    rows_s = (st["refine_ms"] - st["filter_ms"]) / launches / 1e3
    # algorithmic bytes per launch (a launch covers one group of queries in the
    # batched chain, one query in the slot form):
    # row refinement: 8 per survivor read + 4 len + 4 + 8 per refined series (row,
    # perm, moments) + 8 per kept candidate
    rows_bytes = ((8 + 4 * length + 4 + 8) * main_refined + 8 * st["candidates"]) / launches
    kernels = {"q_refine_rows": {"alg_bytes_per_launch": rows_bytes, "avg_launch_us": rows_s * 1e6,
                                 "achieved_gbs": rows_bytes / rows_s / 1e9 if rows_s > 0 else 0.0}}
    tensor = None
    if sched["batch_chain"] and sched["batch_dense"]:
        # q_tc_filter: every pass reads the whole collection (4 len per series) and its
        # id -> position map and moments (12 per series), and writes 8 per survivor;
        # 2 len flops per (series, query) pair on the tensor cores (TF32)
        per = next(m for m in (128, 64, 32, 16) if -(-length // 32) * m * 128 <= 128 * 1024)
        groups = [min(sched["batch_group"], nq - g0) for g0 in range(0, nq, sched["batch_group"])]
        passes = sum(-(-g // per) for g in groups)
        tc_bytes = (passes * n * (4 * length + 12) + 8 * st["survivors"]) / launches
        tc_flops = 2.0 * length * st["tc_pairs"] / launches
        kernels["q_tc_filter"] = {"alg_bytes_per_launch": tc_bytes, "avg_launch_us": filt_s * 1e6,
                                  "achieved_gbs": tc_bytes / filt_s / 1e9 if filt_s > 0 else 0.0,
                                  "passes_per_launch": passes / launches, "flops_per_launch": tc_flops}
        # TF32 dense peak taken as half the measured bf16 peak (the nominal ratio)
        tf32_peak = bf16_peak() / 2.0
        tensor = {"achieved_tflops": tc_flops / filt_s / 1e12 if filt_s > 0 else 0.0, "peak_tflops": tf32_peak,
                  "peak_kind": "measured bf16 x 0.5 (nominal TF32 / BF16 ratio)",
                  "frac": tc_flops / filt_s / 1e12 / tf32_peak if filt_s > 0 else 0.0}
    else:
        # the series filter (qb_filter_series in the batched chain): 16 per SAX word
        # bounded + 8 per block task read + 2 wf per fine PAA read (wf fp16 means) + 8 per
        # survivor written (survivors counted by the rows they became)
        filt_bytes = (16 * st["series_lower_bounded"] + 8 * st["blocks_examined"] + 2 * wf * st["fine_bounded"]
                      + 8 * main_refined) / launches
        name = "qb_filter_series" if sched["batch_chain"] else "q_filter_series"
        kernels[name] = {"alg_bytes_per_launch": filt_bytes, "avg_launch_us": filt_s * 1e6,
                         "achieved_gbs": filt_bytes / filt_s / 1e9 if filt_s > 0 else 0.0}
    dom = max(kernels, key=lambda kk: kernels[kk]["avg_launch_us"])
    achieved = kernels[dom]["achieved_gbs"]
    alg_bytes, refine_s = kernels[dom]["alg_bytes_per_launch"], kernels[dom]["avg_launch_us"] / 1e6
    traffic = None
    import hashlib
    dom_src = "msi_tc.cu" if dom == "q_tc_filter" else "msi_query.cu"
    dom_sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2009_00786_gb300", "csrc", dom_src), "rb").read()
                             ).hexdigest()[:16]
    tpath = os.path.join(ROOT, "profiles", f"{dom}_traffic.txt")
    if os.path.exists(tpath):
        kv = dict(l.split(":", 1) for l in open(tpath).read().splitlines() if ":" in l and not l.startswith("#"))
        if kv.get("source", dom_src).strip() == dom_src and kv.get("source_sha256_16", "").strip() == dom_sha:
            # a capture on a smaller collection, scaled to this launch by its units
            # (the algorithmic bytes) when the file gives the ratio
            if "dram_bytes_per_alg_byte" in kv:
                traffic = float(kv["dram_bytes_per_alg_byte"]) * alg_bytes
            else:
                traffic = float(kv["dram_bytes_per_launch"])

    line = {
        "metric": METRIC,
        "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload(n * world, length, nq, k, args.leaf, args.workload),
                   "n_series": n * world, "len": length, "queries_per_step": nq, "k": k,
                   "l2": "inputs larger than L2 (102 GB collection)", "collection": "borrowed in place (MSI_BUILD_BORROW)",
                   "query_slots": schedule["query_slots"], "schedule": schedule},
        "plain": {"qps": plain_qps, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))},
        "batched": {"qps": qps, "p50_ms": float(np.percentile(call_lat, 50)),
                    "p99_ms": float(np.percentile(call_lat, 99)), "latency": "per call (every query of a call "
                    "is answered when the call completes), over the timed steps", "queries_per_call": nq,
                    "overflow_reruns_per_query": batched_st["overflow_reruns"] / max(1, batched_st["queries"])},
        "build": {"ms": build_ms, "input_gbs": n * length * 4 / (build_ms / 1e3) / 1e9,
                  "input_frac_of_hbm": n * length * 4 / (build_ms / 1e3) / 1e9 / peak,
                  "index_device_gb": msi.msi_index_info_get(index)["device_bytes"] / 1e9},
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": nq * length * 4,
                "d2h_bytes_per_step": nq * k * 12},
        "gpu_launches": timed_launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_us": refine_s * 1e6,
                     "source": dom_src, "source_sha256_16": dom_sha,
                     **({"tensor": tensor} if tensor else {})},
        "refine_kernels": kernels,
        # every kernel of the chain together, over the timed batched steps: leaves (40 B
        # each), block envelopes and tasks (40 B per block bounded), SAX words (16 B),
        # fine PAA means (2 wf B per series or front row bounded by them), rows of the
        # seed, front leaves and survivors (4 len + 12 B), candidates (8 B)
        "step_alg_gbs": (40 * st["leaves_total"] + 40 * st["blocks_examined"] + 16 * st["series_lower_bounded"]
                         + 2 * wf * (st["fine_bounded"] + st["front_fine_bounded"])
                         + (4 * length + 12) * st["series_refined"] + 8 * st["candidates"])
                        / max(1, st["queries"]) * qps / 1e9,
        "work_per_query": {kk: v / max(1, st["queries"]) for kk, v in st.items() if not kk.endswith("_ms")},
        "clocks": clocks.summary(),
    }
    if under_load is not None:
        line["under_load"] = under_load
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, length, n * world)
    index.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
