"""Benchmark: exact k-NN queries/s on one GB300 (or N replicas).

Workload (default "large"): 100,000,000 random-walk series x 256 float32
(z-normalised, seed 0) indexed with leaf capacity 100,000; 10,000 hard queries
(a dataset series plus N(0, sigma^2) noise, sigma alternating 0.5 / 1.0,
re-z-normalised, seed 1); k = 10.  A step answers one batch of queries (1,000
by default) through the whole path: query preparation, LB_EAPCA, the
approximate search, leaf pruning, the distance step, top-k, and the binary64
boundary rescore.  Consecutive steps take consecutive batches of the 10,000
queries.  The distance step is the tensor-core form on a float16 copy by
default (`--form fp16`; `bf16` and the float32 scan `plain` are the others);
the float32 path is also timed on the same index and reported under `forms`.
Every answer is exact (ids equal to brute force).

Prints one JSON line.  `--impl reference` times the oracle (plain binary64
brute force on the host cores) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: N, n, leaf capacity, total queries, noise sigmas, k, queries per step
    "large": dict(N=100_000_000, n=256, tau=100_000, nq=10_000, sigmas=[0.5, 1.0], k=10, batch=2000,
                  desc="100M random walks x 256, leaf 100K, 10K hard queries (sigma 0.5/1.0), k=10"),
    "precision": dict(N=10_000_000, n=256, tau=10_000, nq=1024, sigmas=("uniform", 0.01, 1.0), k=100, batch=1024,
                      desc="10M random walks x 256, leaf 10K, 1024 queries (sigma uniform in [0.01, 1.0]), k=100"),
    "mid": dict(N=10_000_000, n=256, tau=10_000, nq=100, sigmas=[0.01, 0.1, 0.5, 1.0], k=10, batch=100,
                desc="10M random walks x 256, leaf 10K, 100 queries (sigma 0.01/0.1/0.5/1.0), k=10"),
    # 2-6 GB cases of the large workload's shape, for profiler captures
    "tcprofile": dict(N=2_000_000, n=256, tau=20_000, nq=1000, sigmas=[0.5, 1.0], k=10, batch=1000,
                      desc="2M random walks x 256, leaf 20K, 1000 hard queries (sigma 0.5/1.0), k=10"),
    "tcleaf100k": dict(N=4_000_000, n=256, tau=100_000, nq=1000, sigmas=[0.5, 1.0], k=10, batch=1000,
                       desc="4M random walks x 256, leaf 100K, 1000 hard queries (sigma 0.5/1.0), k=10"),
    "tcleaf100k2k": dict(N=4_000_000, n=256, tau=100_000, nq=2000, sigmas=[0.5, 1.0], k=10, batch=2000,
                         desc="4M random walks x 256, leaf 100K, 2000 hard queries (sigma 0.5/1.0), k=10"),
    "precprofile": dict(N=2_000_000, n=256, tau=10_000, nq=1024, sigmas=("uniform", 0.01, 1.0), k=100,
                        batch=1024,
                        desc="2M random walks x 256, leaf 10K, 1024 queries (sigma uniform in [0.01, 1.0]), k=100"),
    "profile": dict(N=2_000_000, n=256, tau=10_000, nq=200, sigmas=[0.5, 1.0], k=10, batch=200,
                    desc="2M random walks x 256, leaf 10K, 200 hard queries (sigma 0.5/1.0), k=10"),
    "small": dict(N=100_000, n=256, tau=1_000, nq=10, sigmas=[0.1], k=1, batch=10,
                  desc="100K random walks x 256, leaf 1K, 10 queries (sigma 0.1), k=1"),
}

# DRAM traffic of the dominant kernel per launch, as a multiple of the
# launch's algorithmic DRAM bytes (for k_tc_scan: the 16-bit rows and norms of
# every leaf the step scans, each once), from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of a small case of the same
# shape; a full launch's traffic is that multiple of its own algorithmic bytes.
# Each entry holds the SHA-256 prefix of the kernel source it was taken on;
# once the source differs, traffic is reported as null until re-captured.
TRAFFIC_RATIO = {   # (kernel, form): dict(exact=r, approx=r, src=sha16, capture=description)
    ("k_tc_scan", "fp16"): dict(
        exact=3.1739e9 / 2.08e9, approx=None, src="4893367fad87e23e",
        capture="the exact-step launch of bench.py --workload tcleaf100k2k (4M random walks x 256, leaf 100K, "
                "2000 hard queries: 3.1739 GB of DRAM, L2 hit 73.5%, against 2.08 GB of 16-bit rows and norms)"),
}
# each kernel's source file and the first line of its definition; the hash
# covers the definition's text, up to the closing brace at the start of a line
KERNEL_SOURCE = {
    "k_tc_scan": ("paper_2212_13297_gb300/csrc/hk_tc.cu",
                  "__global__ void __launch_bounds__(kTcThreads, 1) k_tc_scan(TcArgs A) {"),
    "k_scan": ("paper_2212_13297_gb300/csrc/hk_query.cu",
               "__global__ void __launch_bounds__(kBT, 4) k_scan(ScanArgs A) {"),
}


def source_sha(kernel):
    """SHA-256 prefix of the kernel definition's source text."""
    import hashlib
    path, head = KERNEL_SOURCE[kernel]
    text = open(os.path.join(ROOT, path)).read()
    a = text.index(head)
    b = text.index("\n}\n", a)
    return hashlib.sha256(text[a:b].encode()).hexdigest()[:16]


def traffic_ratio(kernel, form):
    r = TRAFFIC_RATIO.get((kernel, form))
    return r if r and r["src"] == source_sha(kernel) else None


SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=d["hbm_gbs"], sm_max_mhz=d.get("sm_max_mhz", 2070.0),
                    bf16_tflops=d.get("bf16_tflops"), bf16_tflops_sustained=d.get("bf16_tflops_sustained"),
                    source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0,
                source="fallback")


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(smax) if smax else None, reasons=sorted(reasons),
                    samples=len(sm))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t, ws):
    """The largest of each rank's t (the job's time): one all-reduce over the
    default process group (NCCL tensors on the GPU, gloo on the CPU)."""
    if ws <= 1:
        return t
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([float(t)], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def rank_batch(i, rank, nbatches):
    """The query batch rank `rank` answers at step i: replicas answer
    different batches (weak scaling: each rank adds its own queries)."""
    return (i + rank) % nbatches


def metric_name(wl):
    N, n, k = wl["N"], wl["n"], wl["k"]
    size = "%dM x %d" % (N // 1_000_000, n) if N >= 1_000_000 else "%d x %d" % (N, n)
    return "exact %d-NN queries/s (%s)" % (k, size)


def cpu_oracle_rate(X_sample, Q, N_full, budget_s=10.0, chunk=250_000):
    """Oracle queries/s over a collection of N_full series, extrapolated from
    the time the oracle takes to scan the sample rows for blocks of queries
    (Q's rows, block after block, until about budget_s of CPU time)."""
    import oracle
    nb = max(1, min(16, Q.shape[0]))
    t0 = time.perf_counter()
    queries = 0
    while True:
        qb = Q[(queries % Q.shape[0]):(queries % Q.shape[0]) + nb]
        s = oracle.KnnStream(qb, 10)
        for done in range(0, X_sample.shape[0], chunk):
            s.update(X_sample[done:done + chunk], done)
        queries += qb.shape[0]
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    qps = queries / (dt * (N_full / X_sample.shape[0]))
    return qps, dt, X_sample.shape[0], s.nthreads, queries


def run_reference(args, wl):
    """The reference arm: the oracle as it stands, on the host cores."""
    import numpy as np
    import torch
    from paper_2212_13297_gb300 import workload
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    rows = min(4_000_000, wl["N"])   # rows scanned per step (the collection's first rows)
    X = workload.random_walk(rows, wl["n"], seed=0, device="cpu").numpy()
    cores = len(os.sched_getaffinity(0))
    nqb = max(1, min(16, cores))
    sig = wl["sigmas"]
    if isinstance(sig, tuple) and sig[0] == "uniform":
        sig = workload.uniform_sigmas(nqb * (args.steps + args.warmup), sig[1], sig[2], seed=1)
    Qt, _ = workload.queries(torch.from_numpy(X), nqb * (args.steps + args.warmup), sig, seed=1)
    Q = Qt.numpy()
    import oracle
    oracle._lib()
    times = []
    for i in range(args.warmup + args.steps):
        q = Q[i * nqb:(i + 1) * nqb]
        t0 = time.perf_counter()
        s = oracle.KnnStream(q, wl["k"], nthreads=cores)
        s.update(X, 0)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    # one step = nqb queries over `rows` rows; scale to the full collection
    scale = wl["N"] / rows
    per_step = statistics.mean(times) * scale
    value = nqb / per_step
    line = dict(impl="reference", metric=metric_name(wl), value=value,
                unit="queries/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
                ms_per_step=per_step * 1e3, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=wl["desc"], N=wl["N"], n=wl["n"], k=wl["k"]),
                cpu_baseline=dict(value=value, unit="queries/s", cores=cores, kind="oracle",
                                  sample="%d queries x %d of the series per step, "
                                         "time scaled by %.0fx to %d series" % (nqb, rows, scale, wl["N"])),
                e2e=dict(value=value, unit="queries/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def serve(binding, idx, Q_all, k, max_batch, qflags, rate, seconds, form, persistent=0):
    """Open-loop serving: requests arrive one query at a time (Poisson at
    `rate` requests/s for `seconds`) and are answered by the
    continuous-batching server (batch-level, or with the tensor-core scans of
    all batches in flight in one resident launch when `persistent`); reports
    arrival-to-answer latency and the rate at which answers came back."""
    import threading
    import numpy as np
    Qh = Q_all.cpu().numpy()
    rng = np.random.default_rng(11)
    n_req = max(1, int(rate * seconds))
    gaps = rng.exponential(1.0 / rate, n_req)
    sv = binding.Server(max_batch=max_batch, max_wait_us=0, query_flags=qflags,
                        workers=3 if persistent else 2, persistent=persistent)
    coll = sv.add(idx)
    # warm the workers' buffers
    for t in [sv.submit(coll, Qh[i], k) for i in range(min(64, len(Qh)))]:
        sv.poll(t, k, timeout_us=60_000_000)
    tickets = [None] * n_req
    ready = threading.Semaphore(0)
    lat = np.zeros(n_req)
    t_done = [0.0]

    def submitter():
        t0 = time.perf_counter()
        due = t0
        for i in range(n_req):
            due += gaps[i]
            d = due - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets[i] = sv.submit(coll, Qh[i % len(Qh)], k)
            ready.release()

    def poller():
        for i in range(n_req):
            ready.acquire()
            r = None
            while r is None:
                r = sv.poll(tickets[i], k, timeout_us=10_000_000)
            lat[i] = r[2] / 1e9
        t_done[0] = time.perf_counter()

    t_start = time.perf_counter()
    ths = [threading.Thread(target=submitter), threading.Thread(target=poller)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    wall = t_done[0] - t_start
    st = sv.stats()
    sv.close()
    ls = np.sort(lat)
    return dict(kind="open loop, Poisson arrivals, one query per request, %s" % (
                    "persistent scan, 3 workers" if persistent else "batch-level, 2 workers"), form=form,
                scan_launches=st["scan_launches"], scan_jobs=st["scan_jobs"],
                scan_jobs_inflight=st["scan_jobs_inflight"],
                offered_rate=rate, requests=n_req, answered_per_s=n_req / wall,
                latency_ms=dict(p50=float(ls[n_req // 2]) * 1e3,
                                p99=float(ls[min(n_req - 1, int(0.99 * n_req))]) * 1e3,
                                max=float(ls[-1]) * 1e3),
                batches=st["batches"], mean_batch=st["served"] / max(1, st["batches"]),
                max_batch=st["max_batch"], errors=st["errors"])


def serve_mix(args):
    """Four device-resident collections behind one continuous-batching server:
    Poisson arrivals at args.serve_mix requests/s, each request a uniformly
    chosen collection, k uniform in {1, 10, 100}, noise sigma uniform in
    [0.01, 1.0]; the precision form where a collection has a 16-bit copy
    (n <= 256), the float32 path otherwise.  Prints one JSON line."""
    import threading
    import numpy as np
    import torch
    from paper_2212_13297_gb300 import binding, workload
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(2)
    sv_flags = binding.HK_Q_BF16
    idxs, pools, builds = [], [], []
    MIX = workload.SERVED_MIX
    for ci, (name, N, n, kind, tau) in enumerate(MIX):
        t0 = time.perf_counter()
        X = workload.collection(kind, N, n, seed=10 + ci, device="cuda")
        nqp = 2048
        sig = workload.uniform_sigmas(nqp, 0.01, 1.0, seed=20 + ci)
        Q, _ = workload.queries(X, nqp, sig, seed=20 + ci, norm=workload.query_norm(kind))
        flags = binding.HK_BUILD_FP16 if n <= 256 else 0
        idxs.append(binding.Index(X, tau, flags=flags))
        pools.append(Q.cpu().numpy())
        del X
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        builds.append(time.perf_counter() - t0)
    sv = binding.Server(max_batch=1024, max_wait_us=0, query_flags=sv_flags,
                        workers=3 if args.persistent else 2, persistent=1 if args.persistent else 0)
    colls = [sv.add(ix) for ix in idxs]
    for ci in range(len(MIX)):   # warm each collection's path
        for t in [sv.submit(colls[ci], pools[ci][i], kk) for i, kk in enumerate((1, 10, 100))]:
            sv.poll(t, 100, timeout_us=120_000_000)
    n_req = max(1, int(args.serve_mix * args.serve_seconds))
    gaps = rng.exponential(1.0 / args.serve_mix, n_req)
    which = rng.integers(0, len(MIX), n_req)
    ks = rng.choice([1, 10, 100], n_req)
    qi = rng.integers(0, 2048, n_req)
    tickets = [None] * n_req
    ready = threading.Semaphore(0)
    lat = np.zeros(n_req)
    t_done = [0.0]

    def submitter():
        due = time.perf_counter()
        for i in range(n_req):
            due += gaps[i]
            d = due - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets[i] = sv.submit(colls[which[i]], pools[which[i]][qi[i]], int(ks[i]))
            ready.release()

    def poller():
        for i in range(n_req):
            ready.acquire()
            r = None
            while r is None:
                r = sv.poll(tickets[i], int(ks[i]), timeout_us=10_000_000)
            lat[i] = r[2] / 1e9
        t_done[0] = time.perf_counter()

    t_start = time.perf_counter()
    ths = [threading.Thread(target=submitter), threading.Thread(target=poller)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    wall = t_done[0] - t_start
    st = sv.stats()
    sv.close()

    def pct(a, p):
        a = np.sort(a)
        return float(a[min(len(a) - 1, int(p * len(a)))]) * 1e3 if len(a) else None

    per = []
    for ci, (name, N, n, kind, tau) in enumerate(MIX):
        m = which == ci
        per.append(dict(collection=name, requests=int(m.sum()), p50_ms=pct(lat[m], 0.5), p99_ms=pct(lat[m], 0.99),
                        form="tensor cores (float16 copy)" if n <= 256 else "float32", build_s=builds[ci]))
    line = dict(metric="served mix: arrival-to-answer latency, exact k-NN", value=n_req / wall, unit="answers/s",
                offered_rate=args.serve_mix, requests=n_req, higher_is_better=True, n_gpus=1,
                latency_ms=dict(p50=pct(lat, 0.5), p99=pct(lat, 0.99), max=float(lat.max()) * 1e3),
                per_collection=per, batches=st["batches"], mean_batch=st["served"] / max(1, st["batches"]),
                max_batch=st["max_batch"], errors=st["errors"], data="synthetic",
                scan_launches=st["scan_launches"], scan_jobs=st["scan_jobs"],
                scan_jobs_inflight=st["scan_jobs_inflight"], scan_max_collections=st["scan_max_collections"],
                config=dict(workload="served mix: " + "; ".join(m[0] for m in MIX), k=[1, 10, 100],
                            sigma="uniform [0.01, 1.0]", arrivals="Poisson, seed 2",
                            server="persistent scan, 3 workers" if args.persistent else "batch-level, 2 workers"))
    print(json.dumps(line), flush=True)


def ablation(args):
    """The paper's ablation (Sec. 4.2): the float32 path with and without
    LB_SAX filtering (NoSAX) and the EAPCA_TH / SAX_TH switches (NoThresh),
    on the mid workload (10M x 256, 100 queries of mixed difficulty, k = 10)
    or the one --ablation-workload names.  Prints one JSON line."""
    import torch
    from paper_2212_13297_gb300 import binding, workload
    import __graft_entry__
    __graft_entry__.build()
    wl = WORKLOADS[args.ablation_workload]
    X = workload.random_walk(wl["N"], wl["n"], seed=0, device="cuda")
    Q, _ = workload.queries(X, wl["nq"], wl["sigmas"], seed=1)
    idx = binding.Index(X, wl["tau"])
    del X
    torch.cuda.empty_cache()
    out = []
    for name, f in [("Hercules", 0), ("NoSAX", binding.HK_Q_NOSAX), ("NoThresh", binding.HK_Q_NOTHRESH),
                    ("NoSAX+NoThresh", binding.HK_Q_NOSAX | binding.HK_Q_NOTHRESH)]:
        for _ in range(args.warmup):
            idx.query(Q, wl["k"], flags=f)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        agg = {}
        for _ in range(args.steps):
            _, _, st = idx.query(Q, wl["k"], flags=f | binding.HK_Q_TIMING)
            for key, v in st.items():
                agg[key] = agg.get(key, 0) + v
        ev1.record()
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        out.append(dict(variant=name, queries_per_s=wl["nq"] * args.steps / t, ms_per_batch=t / args.steps * 1e3,
                        leaves_candidate_frac=agg["leaves_candidate"] / max(1, agg["leaves_total"]),
                        sax_pruned_frac=agg["series_sax_pruned"] / max(1, agg["series_candidate"]),
                        points_per_query=agg["points_computed"] / max(1, agg["queries"]),
                        skip_sequential=agg["skip_sequential"] / args.steps,
                        scan_GBps=agg["scan_bytes"] / max(1, agg["scan_ns"])))
    print(json.dumps(dict(metric="ablation: exact 10-NN queries/s, float32 path", unit="queries/s",
                          config=dict(workload=wl["desc"]), data="synthetic", variants=out)), flush=True)


def tune_graph(args):
    """Form (2) measured: hk_tune's choice against the library's defaults, and
    CUDA-graph replay (HK_Q_GRAPH) against ordinary calls, on a 10M x 256
    random-walk collection (leaf 10K, float16 copy), queries of mixed
    difficulty (sigma 0.01 / 0.1 / 0.5 / 1.0), k = 10.  The tuner sees one
    batch; the configurations are timed on the next.  Prints one JSON line."""
    import torch
    from paper_2212_13297_gb300 import binding, workload
    import __graft_entry__
    __graft_entry__.build()
    N, n, tau, k = 10_000_000, 256, 10_000, 10
    X = workload.random_walk(N, n, seed=0, device="cuda")
    Qall, _ = workload.queries(X, 4096, [0.01, 0.1, 0.5, 1.0], seed=1)
    idx = binding.Index(X, tau, flags=binding.HK_BUILD_FP16)
    del X
    torch.cuda.empty_cache()

    def ms_per_call(Q, kw, reps):
        ids = torch.empty((Q.shape[0], k), dtype=torch.int64, device="cuda")
        dist = torch.empty((Q.shape[0], k), dtype=torch.float32, device="cuda")
        for _ in range(max(3, args.warmup)):
            idx.query(Q, k, out=(ids, dist), **kw)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(reps):
            idx.query(Q, k, out=(ids, dist), **kw)
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    tune_rows = []
    for batch in (64, 512):
        sample, Q = Qall[:batch].contiguous(), Qall[batch:2 * batch].contiguous()
        t0 = time.perf_counter()
        tuned = idx.tune(sample, k)
        tune_s = time.perf_counter() - t0
        kw = {key: tuned[key] for key in ("l_max", "eapca_th", "sax_th", "flags", "query_group", "series_tile")}
        row = dict(batch=batch, tune_s=tune_s, tried=tuned["tried"], chosen=dict(kw, tensor_cores=tuned["tensor_cores"]))
        for name, qkw in (("default_float32", dict(flags=0)), ("default_precision", dict(flags=binding.HK_Q_BF16)),
                          ("tuned", kw)):
            ms = ms_per_call(Q, qkw, 5)
            row[name] = dict(ms_per_batch=ms, queries_per_s=batch / ms * 1e3)
        tune_rows.append(row)
    graph_rows = []
    for batch in (1, 8, 64, 512):
        Q = Qall[:batch].contiguous()
        plain = ms_per_call(Q, dict(flags=binding.HK_Q_BF16), 20)
        graph = ms_per_call(Q, dict(flags=binding.HK_Q_BF16 | binding.HK_Q_GRAPH), 20)
        graph_rows.append(dict(batch=batch, ms_per_batch_launches=plain, ms_per_batch_graph=graph,
                               speedup=plain / graph))
    print(json.dumps(dict(metric="form (2): autotuned configuration and CUDA-graph replay, exact 10-NN",
                          unit="ms per batch", data="synthetic",
                          config=dict(workload="10M random walks x 256, leaf 10K, float16 copy, "
                                               "sigma 0.01/0.1/0.5/1.0, k=10"),
                          autotune=tune_rows, graphs=graph_rows)), flush=True)


def tree_compare(args):
    """Row f3 measured: pruning with the tree's internal-node synopses
    (HK_Q_TREE) against the flat pass over all leaves, on a collection with
    >= 1e5 leaves (N random walks x 256, leaf capacity args.tree_leaf, float16
    copy), 2,000 hard queries (sigma 0.5 / 1.0) and 2,000 easy ones (sigma
    0.01 / 0.1), k = 10, through the precision form and the float32 path.
    Prints one JSON line."""
    import torch
    from paper_2212_13297_gb300 import binding, workload
    import __graft_entry__
    __graft_entry__.build()
    N, n, tau, k, B = args.tree_n, 256, args.tree_leaf, 10, 2000
    X = workload.random_walk(N, n, seed=0, device="cuda")
    t0 = time.perf_counter()
    idx = binding.Index(X, tau, flags=binding.HK_BUILD_FP16)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    batches = {"hard": workload.queries(X, B, [0.5, 1.0], seed=1)[0],
               "easy": workload.queries(X, B, [0.01, 0.1], seed=3)[0]}
    del X
    torch.cuda.empty_cache()
    info = idx.info()
    rows = []
    for name, Q in batches.items():
        for form, f in (("precision", binding.HK_Q_BF16), ("float32", 0)):
            if form == "float32" and name == "hard":
                continue   # minutes per batch at this size; the precision form shows the same pruning
            for mode, tf in (("flat", 0), ("tree", binding.HK_Q_TREE)):
                for _ in range(max(1, args.warmup)):
                    idx.query(Q, k, flags=f | tf)
                torch.cuda.synchronize()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record()
                agg = {}
                for _ in range(args.steps):
                    _, _, st = idx.query(Q, k, flags=f | tf)
                    for key, v in st.items():
                        agg[key] = agg.get(key, 0) + v
                ev1.record()
                torch.cuda.synchronize()
                t = ev0.elapsed_time(ev1) / 1e3
                rows.append(dict(queries=name, form=form, mode=mode, queries_per_s=B * args.steps / t,
                                 ms_per_batch=t / args.steps * 1e3,
                                 lb_evaluations_per_query=agg["lb_evaluations"] / agg["queries"],
                                 leaves_candidate_per_query=agg["leaves_candidate"] / agg["queries"]))
    print(json.dumps(dict(metric="row f3: flat LB_EAPCA over every leaf vs tree pruning (HK_Q_TREE), exact 10-NN",
                          unit="queries/s", data="synthetic",
                          config=dict(workload="%d random walks x %d, leaf %d, float16 copy, 2000 queries per "
                                               "batch (hard: sigma 0.5/1.0, easy: 0.01/0.1), k=%d" % (N, n, tau, k),
                                      leaves=info["leaves"], depth=info["depth"], build_s=build_s),
                          rows=rows)), flush=True)


def dtw_bench(args):
    """Row f4 measured: exact k-NN under DTW (Sakoe-Chiba band) through the
    index, 1M random walks x 256, leaf 1K, band 12 (about 5% of n), 100
    queries (sigma 0.1 / 0.5), k = 10; the same batch under the Euclidean
    distance for comparison.  Prints one JSON line."""
    import torch
    from paper_2212_13297_gb300 import binding, workload
    import __graft_entry__
    __graft_entry__.build()
    N, n, tau, k, band, B = 1_000_000, 256, 1000, 10, 12, 100
    X = workload.random_walk(N, n, seed=0, device="cuda")
    Q, _ = workload.queries(X, B, [0.1, 0.5], seed=1)
    idx = binding.Index(X, tau)
    del X
    torch.cuda.empty_cache()
    out = {}
    for name, call in (("dtw", lambda: idx.query_dtw(Q, k, band)), ("euclidean", lambda: idx.query(Q, k))):
        for _ in range(max(1, args.warmup)):
            call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        agg = {}
        for _ in range(args.steps):
            _, _, st = call()
            for key, v in st.items():
                agg[key] = agg.get(key, 0) + v
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out[name] = dict(queries_per_s=B * args.steps / t, ms_per_batch=t / args.steps * 1e3,
                         leaves_candidate_frac=agg["leaves_candidate"] / max(1, agg["leaves_total"]),
                         series_candidate_per_query=agg["series_candidate"] / agg["queries"],
                         word_bound_pruned_frac=agg["series_sax_pruned"] / max(1, agg["series_candidate"]),
                         keogh_or_abandoned_frac=agg["series_abandoned"] / max(1, agg["series_candidate"]),
                         full_per_query=agg["series_full"] / agg["queries"],
                         points_per_query=agg["points_computed"] / agg["queries"],
                         points_per_s=agg["points_computed"] / t)
    # DTW cells: a difference, a square and an addition each (3 flops), against
    # the derived FP32 ALU peak the float32 scan reports against
    alu_peak = 152 * 128 * 2 * 2070e6
    out["dtw"]["alu_frac"] = 3 * out["dtw"]["points_per_s"] / alu_peak
    print(json.dumps(dict(metric="row f4: exact 10-NN under DTW (band %d) through the index" % band,
                          unit="queries/s", data="synthetic",
                          config=dict(workload="1M random walks x 256, leaf 1K, 100 queries (sigma 0.1/0.5), "
                                               "k=10, band 12"),
                          results=out)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="queries per step (0 = workload default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--query-group", type=int, default=0)
    ap.add_argument("--series-tile", type=int, default=0)
    ap.add_argument("--l-max", type=int, default=0)
    ap.add_argument("--plain-steps", type=int, default=2,
                    help="steps of the float32 path measured beside the headline form")
    ap.add_argument("--plain-groups", default="0,4",
                    help="query groups of the float32 measurements (0 = the library's choice)")
    ap.add_argument("--form", default="fp16", choices=["plain", "bf16", "fp16"],
                    help="plain float32 scan, or the tensor-core form on a bfloat16 / float16 copy")
    ap.add_argument("--serve", type=float, default=2000.0,
                    help="also drive the continuous-batching server with the headline form at this "
                         "Poisson arrival rate (requests/s) and report arrival-to-answer latency (0: off)")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-plain", type=float, default=500.0,
                    help="the same for the float32 path, at a rate it sustains (0: off)")
    ap.add_argument("--serve-plain-seconds", type=float, default=2.5)
    ap.add_argument("--timing-steps", type=int, default=3,
                    help="instrumented steps (kernel times by CUDA events) after the timed steps; "
                         "at least 1 (the roofline needs them)")
    ap.add_argument("--ablation", action="store_true",
                    help="instead of the step benchmark, the NoSAX / NoThresh ablation on the mid workload")
    ap.add_argument("--ablation-workload", default="mid", choices=sorted(WORKLOADS))
    ap.add_argument("--tune-graph", action="store_true",
                    help="instead of the step benchmark, hk_tune's choice against the defaults and "
                         "CUDA-graph replay against ordinary calls (10M x 256)")
    ap.add_argument("--tree", action="store_true",
                    help="instead of the step benchmark, flat vs tree pruning (HK_Q_TREE) on >= 1e5 leaves")
    ap.add_argument("--tree-n", type=int, default=100_000_000)
    ap.add_argument("--tree-leaf", type=int, default=1000)
    ap.add_argument("--dtw", action="store_true",
                    help="instead of the step benchmark, exact k-NN under DTW through the index")
    ap.add_argument("--persistent", action="store_true",
                    help="--serve-mix: serve with the resident tensor-core scan")
    ap.add_argument("--serve-mix", type=float, default=0.0,
                    help="instead of the step benchmark, serve the four-collection mix at this "
                         "rate (requests/s) and print its latency line")
    args = ap.parse_args()
    args.timing_steps = max(1, args.timing_steps)
    wl = dict(WORKLOADS[args.workload])
    if args.batch:
        wl["batch"] = args.batch

    if args.impl == "reference":
        run_reference(args, wl)
        return
    if args.serve_mix > 0:
        serve_mix(args)
        return
    if args.ablation:
        ablation(args)
        return
    if args.tune_graph:
        tune_graph(args)
        return
    if args.tree:
        tree_compare(args)
        return
    if args.dtw:
        dtw_bench(args)
        return

    import numpy as np
    import torch
    from paper_2212_13297_gb300 import binding, workload
    import __graft_entry__
    __graft_entry__.build()

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local

    N, n, k, B = wl["N"], wl["n"], wl["k"], wl["batch"]
    t0 = time.perf_counter()
    X = workload.random_walk(N, n, seed=0, device="cuda")
    sig = wl["sigmas"]
    if isinstance(sig, tuple) and sig[0] == "uniform":
        sig = workload.uniform_sigmas(wl["nq"], sig[1], sig[2], seed=1)
    Q_all, _ = workload.queries(X, wl["nq"], sig, seed=1)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    sample = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample = X[:min(N, 4_000_000)].cpu().numpy()
    t0 = time.perf_counter()
    bflags = {"plain": 0, "bf16": binding.HK_BUILD_BF16, "fp16": binding.HK_BUILD_FP16}[args.form]
    qflags = binding.HK_Q_BF16 if args.form != "plain" else 0
    idx = binding.Index(X, wl["tau"], flags=bflags)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    info = idx.info()
    del X
    torch.cuda.empty_cache()

    nb = max(1, wl["nq"] // B)
    batches = [Q_all[(i % nb) * B:(i % nb + 1) * B].contiguous() for i in range(args.warmup + args.steps)]
    ids = torch.empty((B, k), dtype=torch.int64, device="cuda")
    dist_out = torch.empty((B, k), dtype=torch.float32, device="cuda")
    qkw = dict(l_max=args.l_max, query_group=args.query_group, series_tile=args.series_tile)

    def timed(flags, steps, warmup, first, **over):
        """Device time of `steps` batches (after `warmup`), summed stats, and
        each step's time between CUDA events recorded on the query stream
        before and after its call (ms)."""
        kw = dict(qkw, **over)
        for i in range(warmup):
            idx.query(batches[rank_batch(first + i, rank, len(batches))], k, flags=flags,
                      out=(ids, dist_out), **kw)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        stream = torch.cuda.current_stream()
        evs[0].record(stream)
        agg = {}
        for i in range(steps):
            _, _, st = idx.query(batches[rank_batch(first + warmup + i, rank, len(batches))], k,
                                 flags=flags, out=(ids, dist_out), **kw)
            evs[i + 1].record(stream)
            for key, v in st.items():
                agg[key] = agg.get(key, 0) + v
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        t = max_over_ranks(evs[0].elapsed_time(evs[-1]) / 1e3, ws)
        return t, agg, [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]

    sampler = ClockSampler(dev_index)
    sampler.start()
    time.sleep(1.0)   # nvidia-smi starts up and takes its first samples before the timed region
    t_dev, agg, step_ms = timed(qflags, args.steps, args.warmup, 0)
    clocks = sampler.stop()
    value = ws * B * args.steps / t_dev
    # kernel times (CUDA events around the scan launches) from a separate,
    # instrumented pass over the same batches, so the headline carries none
    t_ins, agg_ins, _ = timed(qflags | binding.HK_Q_TIMING, args.timing_steps, 0, args.warmup)

    # end to end through the C ABI with host buffers (pinned queries in,
    # host results out; the copies are inside each call)
    e2e = None
    if not args.no_e2e:
        hq = [batches[rank_batch(args.warmup + i, rank, len(batches))].cpu().pin_memory()
              for i in range(args.steps)]
        hid = np.empty((B, k), np.int64)
        hdi = np.empty((B, k), np.float32)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        te = time.perf_counter()
        for i in range(args.steps):
            idx.query(hq[i], k, flags=qflags, out=(hid, hdi), **qkw)
        t_e2e = max_over_ranks(time.perf_counter() - te, ws)
        e2e = dict(value=ws * B * args.steps / t_e2e, unit="queries/s",
                   h2d_bytes_per_step=B * n * 4, d2h_bytes_per_step=B * k * 12)

    # the plain float32 path on the same index, for comparison, at each query
    # group asked for (0 = the library's choice): more queries per series read
    # means fewer bytes per query but more arithmetic per byte
    forms = {args.form: dict(value=value, ms_per_step=t_dev / args.steps * 1e3)}
    plain_runs = []
    if args.plain_steps > 0:
        for gsz in [int(x) for x in args.plain_groups.split(",") if x.strip()]:
            if args.form == "plain" and gsz == args.query_group:
                continue   # the headline run already is this one
            tp, aggp, _ = timed(binding.HK_Q_TIMING, args.plain_steps, 1, args.warmup, query_group=gsz)
            name = "plain" if gsz == 0 else "plain_group%d" % gsz
            forms[name] = dict(value=ws * B * args.plain_steps / tp, ms_per_step=tp / args.plain_steps * 1e3,
                               query_group=gsz or "auto (8)")
            plain_runs.append((name, aggp))

    # served: Poisson arrivals through the continuous-batching server, the
    # headline form and the float32 path at a rate it sustains
    serving = None
    if args.serve > 0 or args.serve_plain > 0:
        serving = {}
        if args.serve > 0:
            serving[args.form] = serve(binding, idx, Q_all, k, B, qflags, args.serve, args.serve_seconds,
                                       args.form)
            if args.form != "plain":
                serving[args.form + "_persistent"] = serve(binding, idx, Q_all, k, B, qflags, args.serve,
                                                           args.serve_seconds, args.form, persistent=1)
        if args.serve_plain > 0 and args.form != "plain":
            serving["plain"] = serve(binding, idx, Q_all, k, B, 0, args.serve_plain,
                                     args.serve_plain_seconds, "plain")

    if rank != 0:
        return
    pk = peaks()
    alu_peak = SM_COUNT_GB300 * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12

    def plain_roof(a):
        """The float32 scan: FP32 ALU rate on its (q-x)^2 points (what bounds it:
        it is issue-bound), the rate of its algorithmic scan bytes (per work
        item; L2 serves the query groups' repeats, so not an HBM figure), and
        DRAM GB/s from a capture's DRAM-to-algorithmic ratio when one exists
        for this kernel source."""
        scan_s = a["scan_ns"] / 1e9
        alu_ach = 3.0 * a["points_computed"] / scan_s / 1e12 if scan_s else None
        rate = a["scan_bytes"] / scan_s / 1e9 if scan_s else None
        tr = traffic_ratio("k_scan", "plain")
        dram = None
        if tr and rate:
            dram = dict(achieved=tr["exact"] * rate, peak=pk["hbm_gbs"], unit="GB/s",
                        frac=tr["exact"] * rate / pk["hbm_gbs"],
                        note="DRAM bytes = %.3f x the algorithmic scan bytes (ncu capture of %s)" % (
                            tr["exact"], tr["capture"]))
        return dict(kernel="k_scan", alu=dict(achieved=alu_ach, peak=alu_peak, unit="TFLOP/s",
                                              frac=(alu_ach or 0) / alu_peak),
                    scan_byte_rate=dict(achieved=rate, unit="GB/s",
                                        note="16 B per iSAX word + 64 B per 16-point chunk, counted per work "
                                             "item (query group); L2 serves the groups' repeats"),
                    dram=dram, share_of_step=None)

    if args.form == "plain":
        pr = plain_roof(agg_ins)
        roof = dict(bound="alu", achieved=pr["alu"]["achieved"], peak=alu_peak, unit="TFLOP/s",
                    frac=pr["alu"]["frac"], kernel="k_scan",
                    traffic=(pr["dram"]["achieved"] * agg_ins["scan_ns"] / 1e9 / args.timing_steps * 1e9)
                    if pr["dram"] else None,
                    peak_note="derived: 152 SMs x 128 FP32 lanes x 2 flops x %.0f MHz; "
                              "3 flops per (q-x)^2 point" % pk["sm_max_mhz"],
                    scan_byte_rate=pr["scan_byte_rate"], dram=pr["dram"])
        roof["kernel_share_of_step"] = agg_ins["scan_ns"] / 1e9 / t_ins
        for name, a in plain_runs:
            roof[name + "_k_scan"] = plain_roof(a)
    else:
        a = agg_ins
        tc_s = a["tc_ns"] / 1e9
        flops = 2.0 * n * a["tc_pairs"]
        ach = flops / tc_s / 1e12 if tc_s else None
        peak_t = pk.get("bf16_tflops_sustained") or 1713.1
        tr = traffic_ratio("k_tc_scan", args.form)
        alg = a.get("tc_leaf_bytes", 0) / args.timing_steps
        roof = dict(bound="tensor", achieved=ach, peak=peak_t, unit="TFLOP/s", frac=(ach or 0) / peak_t,
                    traffic=tr["exact"] * alg if tr else None, kernel="k_tc_scan",
                    traffic_note=("DRAM bytes per exact-step launch: %.3f x its algorithmic bytes, the ratio "
                                  "of an ncu capture of %s" % (tr["exact"], tr["capture"])) if tr else
                                 "no DRAM capture of this kernel source",
                    algorithmic_dram_bytes_per_launch=alg,
                    peak_note="of measured sustained bf16 (%s); %s dense rate equals bf16's nominally; "
                              "2n flops per (query, series) pair" % (pk["source"], args.form),
                    frac_of_burst=(ach or 0) / (pk.get("bf16_tflops") or 1920.7),
                    bulk_copy_rate=dict(achieved=a["tc_bytes"] / tc_s / 1e9 if tc_s else None, unit="GB/s",
                                        note="16-bit rows + norms the bulk copies move per query block, "
                                             "served by L2 and DRAM together (not an HBM figure)"),
                    kernel_share_of_step=tc_s / t_ins, timing_steps=args.timing_steps)
        tca_s = a.get("tc_approx_ns", 0) / 1e9
        if tca_s:
            roof["approx_step_launches"] = dict(
                kernel="k_tc_scan", share_of_step=tca_s / t_ins,
                bulk_copy_rate=dict(achieved=a["tc_approx_bytes"] / tca_s / 1e9, unit="GB/s"),
                traffic=tr["approx"] * a.get("tc_approx_bytes", 0) / args.timing_steps
                if tr and tr["approx"] else None,
                note="the same kernel on each query's approximate-search leaves (few queries per "
                     "leaf: bound by the 16-bit rows it streams, not by the MMA)")
        for name, a in plain_runs:
            roof[name + "_k_scan"] = plain_roof(a)

    cpu = None
    if sample is not None:
        cores = len(os.sched_getaffinity(0))
        nqb = max(1, min(16, cores))
        qps, dt, rows, thr, nqs = cpu_oracle_rate(sample, Q_all[:256].cpu().numpy(), N)
        cpu = dict(value=qps, unit="queries/s", cores=thr, kind="oracle",
                   sample="%d queries (blocks of %d) x first %d series (%.1f s of CPU), time scaled to "
                          "%d series" % (nqs, nqb, rows, dt, N))

    lat = sorted(step_ms)
    dtype = {"plain": "f32", "bf16": "bf16", "fp16": "fp16"}[args.form]
    line = dict(
        metric=metric_name(wl),
        value=value, unit="queries/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
        ms_per_step=t_dev / args.steps * 1e3, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype=dtype, data="synthetic",
        config=dict(workload=wl["desc"], N=N, n=n, leaf_capacity=wl["tau"], k=k,
                    queries_per_step=B, queries_total=wl["nq"],
                    form={"plain": "float32 scan", "bf16": "tensor cores, bfloat16 copy",
                          "fp16": "tensor cores, float16 copy"}[args.form]
                         + " + exact float32/binary64 rescore",
                    parallelism="replicas" if ws > 1 else "1 GPU",
                    l2="inputs larger than L2 (%.0f GB collection)" % (N * n * 4 / 1e9)),
        latency_ms=dict(kind="batch completion (closed loop, %d queries per batch; CUDA events between "
                             "consecutive calls on the query stream)" % B,
                        p50=lat[len(lat) // 2], p99=lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                        per_step=[round(x, 3) for x in step_ms]),
        clocks=clocks, e2e=e2e, gpu_launches=agg["kernel_launches"], roofline=roof,
        cpu_baseline=cpu, forms=forms, serving=serving,
        pruning=dict(leaves_candidate_frac=agg["leaves_candidate"] / max(1, agg["leaves_total"]),
                     series_candidate=agg["series_candidate"], sax_pruned=agg["series_sax_pruned"],
                     abandoned=agg["series_abandoned"], full=agg["series_full"],
                     points=agg["points_computed"], tc_pairs=agg["tc_pairs"],
                     tc_candidates=agg["tc_candidates"], tc_approx_pairs=agg.get("tc_approx_pairs", 0),
                     rescored=agg["rescored"],
                     retried=agg["retried_queries"], fallback=agg["fallback_queries"],
                     skip_sequential=agg["skip_sequential"]),
        index=dict(build_s=t_build, gen_s=t_gen, leaves=info["leaves"], depth=info["depth"],
                   max_segments=info["max_segments"]),
    )
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
