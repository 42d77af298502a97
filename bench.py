"""Benchmark of the EVP ternary search hot path on one GB300.

Workload (defaults): a resident database of 10,000,000 l2-normalised
Gaussian-mixture embeddings, d = 768 (1,024 centres, anisotropic scales),
encoded once at x = 512 (packed codes 1.92 GB; float32 originals 30.7 GB
kept for the rerank).  One step = one batch of 1,024 float32 queries through
the whole path: evp_encode -> ternary_knn (shortlist of 100 by Delta) ->
rerank (best 10 by float32 scalar product).  Inputs are larger than L2, so
no flush is needed between steps.

Prints one JSON line.  `--impl reference` times the CPU oracle instead (a
bounded sample of the same workload, scaled to the full database).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "queries/s at 10Mx768 ternary (encode + scan + rerank), recall@10"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--d", type=int, default=768)
    ap.add_argument("--x", type=int, default=0, help="0 = default x (2d/3 rule)")
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--shortlist", type=int, default=100)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--centres", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-recall", action="store_true")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the tensor-core rate probe (roofline then uses 2 x bf16)")
    ap.add_argument("--path", type=int, default=0,
                    help="0 auto, 1 popcount, 2 tensor core, 3 packed tensor core, "
                         "4 int8 queries (asymmetric scan), 5 sparse codes (small x)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched-form and served-form measurements")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-rates", default="100,200,400,800,1200,1600",
                    help="Poisson request rates (requests/s) of the served-form sweep")
    ap.add_argument("--recall-sweep", action="store_true",
                    help="instead of the benchmark: recall of the ternary scan against exact "
                         "float32 cosine kNN for several x (1M x 768 mixture by default)")
    ap.add_argument("--sweep-queries", type=int, default=2000)
    ap.add_argument("--spearman", action="store_true",
                    help="instead of the benchmark: Table 1's Uniform rows (Spearman rho of "
                         "EVP, 1-bit and b1.58 proxy distances) through the library")
    return ap.parse_args()


def make_config(a, x, world):
    """The workload description both arms print (identical dicts)."""
    n, d, B = a.n, a.d, a.batch
    W = (d + 63) // 64
    return {"workload": f"{n}x{d} ternary kNN (Gaussian mixture, {a.centres} centres, "
                        f"anisotropic), x={x}, batch {B} queries/step, shortlist "
                        f"{a.shortlist} by Delta, rerank to k={a.k}",
            "n": n, "d": d, "x": x, "batch": B, "shortlist": a.shortlist, "k": a.k,
            "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 (codes {n * 16 * W / 1e9:.2f} GB, floats "
                  f"{n * d * 4 / 1e9:.1f} GB); no flush"}


def measure_tensor_peak(evp, sampler_cls, local, seconds=1.0):
    """Measured dense tensor-core rate (evp_probe_tensor_rate) for the
    instruction shapes the scans issue, each run back to back for about
    `seconds` with the SM clocks sampled meanwhile."""
    import torch
    out = {}
    shapes = [("f4_pair_m256_n256", 2, True, 256), ("f4_m128_n256", 2, False, 256),
              ("f8_pair_m256_n256", 0, True, 256), ("f8_m128_n256", 0, False, 256),
              ("bf16_m128_n256", 1, False, 256), ("f8_m128_n64", 0, False, 64),
              ("f8_m128_n16", 0, False, 16)]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for name, kind, pair, nn in shapes:
        evp.probe_tensor_rate(kind, pair, nn, 1 << 12)          # warm-up
        sampler = sampler_cls(local)
        sampler.start()
        t_end = time.perf_counter() + (seconds if nn == 256 else 0.25)
        rates, cycles = [], []
        # long launches (tens of ms), so that launch and set-up time is a
        # small part of the elapsed time the rate is taken over
        iters = 1 << 18 if nn == 256 else 1 << 17
        while time.perf_counter() < t_end:
            tf, cyc, _ = evp.probe_tensor_rate(kind, pair, nn, iters)
            rates.append(tf)
            cycles.append(cyc)
        clk = sampler.stop()
        m = 256 if pair else 128
        kk = {0: 32, 1: 16, 2: 64}[kind]
        fpc = 2.0 * m * nn * kk / float(np.median(cycles)) / (2 if pair else 1)
        mhz = clk.get("sm_mhz")
        out[name] = {"tflops": float(np.median(rates)), "cycles_per_mma": float(np.median(cycles)),
                     "flop_per_clk_per_sm": fpc,
                     "tflops_at_sampled_clock": fpc * sms * mhz * 1e6 / 1e12 if mhz else None,
                     "launches": len(rates), "sm_mhz": mhz,
                     "reasons": clk.get("reasons")}
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return j.get("hbm_gbs", 6800.0), j.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# POPC issue rate measured on this GB300 (16 per clock per SM) at the
# maximum SM clock, for the integer-pipe roofline of the popcount scan.
POPC_PER_CLK_PER_SM = 16

# DRAM traffic per launch of the dominant kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, one capture of this bench's own command), keyed by
# (kernel, rows, d, queries per step, scan k).  Each entry carries the
# SHA-256 of the kernel sources it was measured on and is reported only
# while those sources are unchanged; otherwise the traffic is null.
KERNEL_SOURCES = {
    "scan_mma": ["paper_2506_00528_gb300/csrc/scan_mma.cu",
                 "paper_2506_00528_gb300/csrc/evp_internal.cuh"],
    "scan_popc": ["paper_2506_00528_gb300/csrc/scan_popc.cu",
                  "paper_2506_00528_gb300/csrc/evp_internal.cuh"],
    "scan_mma_packed": ["paper_2506_00528_gb300/csrc/scan_mma_packed.cu",
                        "paper_2506_00528_gb300/csrc/evp_internal.cuh"],
}
MEASURED_TRAFFIC = {
    # DRAM bytes of one launch at the 10M-row workload, from a capture of
    # the same command on 1,000,000 rows (the recipe's size rule): reads
    # scaled by the rows (the database stream), writes (per-query lists and
    # histograms, independent of the rows) as captured.
    # profiles/scan_mma_10Mx768_b1024_launches.md
    ("scan_mma", 10_000_000, 768, 1024, 100): {
        "bytes": 386_409_728 * 10 + 3_898_368,
        "sources_sha256": "0ded91804e7e82397f9acc8e74bb217f2f7ef915086e8450a78a0356e3f501a6"},
    # profiles/scan_popc_1Mx768_b1_ncu.md
    ("scan_popc", 10_000_000, 768, 1, 100): {
        "bytes": 192_033_024 * 10 + 3_496_192,
        "sources_sha256": "cdf7029f81db7af20486a0732bd77ca154d54c6067ec22f9d701f7fcae8b85bf"},
    # profiles/scan_mma_packed_10Mx768_b16.md
    ("scan_mma_packed", 10_000_000, 768, 16, 100): {
        "bytes": 194_052_096 * 10 + 9_144_832,
        "sources_sha256": "f6f8798da020b1700b119d945568766194ea2a950212a4bdf4c95d4ea2e665e5"},
}


def kernel_sources_sha(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(kernel: str, n: int, d: int, batch: int, k_scan: int):
    e = MEASURED_TRAFFIC.get((kernel, n, d, batch, k_scan))
    if e is None or e["sources_sha256"] != kernel_sources_sha(kernel):
        return None
    return e["bytes"]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"evp_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_oracle_sample(U_dev, Q_host, x, shortlist, k, n_total, n_rows=200_000, n_q=8):
    """Time the oracle as it stands (single thread) on a bounded sample:
    n_q queries encoded, scanned exhaustively over n_rows database rows,
    and re-ranked; the scan part is scaled to the full database."""
    import concurrent.futures as cf
    import oracle
    import torch
    rows = U_dev[:n_rows].cpu().numpy()
    # encoding the sample database is pre-processing (untimed), spread over threads
    chunks = np.array_split(np.arange(n_rows), os.cpu_count() or 1)
    Vs = np.empty(rows.shape, dtype=np.int8)

    def job(ix):
        if len(ix):
            Vs[ix[0]:ix[-1] + 1] = oracle.encode(rows[ix[0]:ix[-1] + 1], x)

    with cf.ThreadPoolExecutor(len(chunks)) as ex:
        list(ex.map(job, chunks))
    Qs = Q_host[:n_q]
    t0 = time.perf_counter()
    Vq = oracle.encode(Qs, x)
    t1 = time.perf_counter()
    ids, _ = oracle.knn(Vq, Vs, shortlist)
    t2 = time.perf_counter()
    oracle.rerank(Qs, rows, ids, k)
    t3 = time.perf_counter()
    scale = n_total / n_rows
    per_query = ((t1 - t0) + (t2 - t1) * scale + (t3 - t2)) / n_q
    # the same oracle on every host core: one query's exhaustive scan per
    # thread (the C oracle runs without the interpreter lock)
    cores = os.cpu_count() or 1
    Vq_all = oracle.encode(Q_host[:cores], x)
    t4 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda i: oracle.knn(Vq_all[i:i + 1], Vs, shortlist), range(len(Vq_all))))
    t5 = time.perf_counter()
    scan_all = (t5 - t4) * scale / len(Vq_all)       # scan seconds per query, all cores
    per_query_all = ((t1 - t0) + (t3 - t2)) / n_q + scan_all
    # the paper's float baseline ("Euclidean", Tables 4 and 5): exact float32
    # brute force over the same rows, one thread
    n_e = max(1, n_q // 4)
    t6 = time.perf_counter()
    oracle.l2_knn(Qs[:n_e], rows, k)
    t7 = time.perf_counter()
    euclid_per_query = (t7 - t6) * scale / n_e
    del torch
    return 1.0 / per_query, {
        "sample": f"{n_q} queries over the first {n_rows} database rows "
                  f"(scan time scaled x{scale:.0f} to {n_total} rows); encode+knn+rerank",
        "seconds": t3 - t0,
        "all_cores": {"value": 1.0 / per_query_all, "cores": cores,
                      "sample": f"{len(Vq_all)} concurrent query scans over the same rows, "
                                "one per thread; encode and rerank as single-thread"},
        "euclidean_fp32": {"value": 1.0 / euclid_per_query, "cores": 1,
                           "sample": f"{n_e} queries, exact float32 squared-Euclidean brute "
                                     f"force over the first {n_rows} rows (scaled x{scale:.0f}), "
                                     f"top-{k}"}}


def measure_batched(evp, synth, dev, seed_batches=64):
    """Batched form: three resident databases (1M x 384 at x = 128, 4M x 768
    at x = 256, 2M x 1024 at x = 384), 64 kNN batches with sizes
    round(logU[1, 8192]) and k in {10, 100}, each against a database drawn
    at random.  Timed four ways on the same inputs: the plan with its fused
    tensor-core scan (one persistent launch over every fp4-path batch)
    replayed as a CUDA graph, the same plan run eagerly, a plan of separate
    per-batch calls replayed as a graph, and one plain evp_db_knn call per
    batch (automatic path); the results of all four must be identical."""
    import torch
    rng = np.random.default_rng(20250601)
    shapes = [(1_000_000, 384, 128), (4_000_000, 768, 256), (2_000_000, 1024, 384)]
    dbs = []
    for i, (n, d, x) in enumerate(shapes):
        U = synth.mixture_torch(n, d, n_centres=1024, anisotropic=True, stream=40 + i, device=dev)
        T = evp.encode(U, x)
        del U
        dbs.append((evp.Database(T, None, d, x), T, d, x))
    sizes = np.clip(np.rint(np.exp(rng.uniform(0, np.log(8192), seed_batches))), 1, 8192).astype(int)
    ks = rng.choice([10, 100], seed_batches)
    which = rng.integers(0, 3, seed_batches)
    spec = []
    for i in range(seed_batches):
        db, T, d, x = dbs[which[i]]
        Q = synth.mixture_torch(int(sizes[i]), d, n_centres=1024, anisotropic=True,
                                stream=100 + i, device=dev)
        spec.append({"db": db, "Qc": evp.encode(Q, x), "k": int(ks[i])})
    stream = torch.cuda.Stream(dev)
    reps = 3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def time_plan(plan):
        with torch.cuda.stream(stream):
            plan.run(stream=stream)          # capture (graph) + first run
            plan.run(stream=stream)
            e0.record(stream)
            for _ in range(reps):
                plan.run(stream=stream)
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    t0 = time.perf_counter()
    fused = evp.BatchPlan(spec, graph=True, tune=True, fused=True, stream=stream)
    tune_s = time.perf_counter() - t0
    fused_ms = time_plan(fused)
    outs = [tuple(t.clone() for t in fused.outputs(i)) for i in range(len(spec))]
    paths = [fused.path(i) for i in range(len(spec))]
    tiles = sorted({fused.tile(i) for i in range(len(spec)) if fused.tile(i) > 0})
    n_fused = fused.fused
    fused.close()
    eager = evp.BatchPlan(spec, graph=False, tune=True, fused=True, stream=stream)
    eager_ms = time_plan(eager)
    eager.close()
    sep = evp.BatchPlan(spec, graph=True, tune=True, fused=False, stream=stream)
    sep_ms = time_plan(sep)
    same = all(torch.equal(o[0], g[0]) and torch.equal(o[1], g[1])
               for o, g in zip(outs, (sep.outputs(i) for i in range(len(spec)))))
    sep.close()
    # plain: one evp_db_knn call per batch on one stream, automatic path
    plain_out = [None] * len(spec)

    def plain():
        for i, b in enumerate(spec):
            plain_out[i] = b["db"].knn(b["Qc"], b["k"], stream=stream)

    with torch.cuda.stream(stream):
        plain()
        e0.record(stream)
        for _ in range(reps):
            plain()
        e1.record(stream)
    stream.synchronize()
    plain_ms = e0.elapsed_time(e1) / reps
    same = same and all(torch.equal(o[0], p_[0]) and torch.equal(o[1], p_[1])
                        for o, p_ in zip(outs, plain_out))
    total_q = int(sizes.sum())
    for db, *_ in dbs:
        db.close()
    qps = lambda ms: total_q / (ms / 1e3)
    return {"batches": seed_batches, "queries": total_q,
            "fused_graph_qps": qps(fused_ms), "fused_graph_ms": fused_ms,
            "fused_eager_qps": qps(eager_ms), "separate_graph_qps": qps(sep_ms),
            "plain_qps": qps(plain_ms), "plain_ms": plain_ms,
            "fused_batches": n_fused, "fused_tiles_per_item": tiles, "plan_and_tune_s": tune_s,
            "paths": {"popc": paths.count(1), "mma": paths.count(2),
                      "mma_packed": paths.count(3)},
            "identical_results": bool(same),
            "workload": "3 DBs (1Mx384 x128, 4Mx768 x256, 2Mx1024 x384), 64 kNN batches "
                        "logU[1,8192] queries, k in {10,100}; fused = one persistent "
                        "tensor-core launch for every fp4-path batch"}


def _request_stream(rate, seconds, seed):
    rng = np.random.default_rng(seed)
    n_req = max(1, int(seconds * rate))
    arr = np.cumsum(rng.exponential(1.0 / rate, n_req))
    sizes = np.clip(np.rint(np.exp(rng.uniform(0, np.log(1024), n_req))), 1, 1024).astype(int)
    ks = rng.choice([10, 100], n_req)
    offs = rng.integers(0, 4096 - sizes + 1)
    return arr, sizes, ks, offs


def measure_served(evp, synth, db, d, seconds, rates, dev):
    """Served form: for each Poisson rate, the same request stream (sizes
    round(logU[1, 1024]) queries, k in {10, 100}, shortlist 10 k capped at
    1024, reranked to k) run (a) through the continuous-batching server
    (3 slots) and (b) as plain per-request evp_db_search_host calls in
    arrival order on one stream; latency = completion - arrival."""
    import torch
    pool = synth.mixture_torch(4096, d, n_centres=1024, anisotropic=True, stream=77,
                               device=dev).cpu().pin_memory()
    out = []
    srv = evp.Server(db, max_batch_queries=4096, max_k=100, shortlist_factor=10, max_slots=3,
                     mem_budget_bytes=48 << 30)
    for k in (10, 100):                                   # warm-up of each class
        srv.wait(srv.submit(pool[:64], k))
    ids_flat = torch.empty(1024 * 100, dtype=torch.int64).pin_memory()
    sc_flat = torch.empty(1024 * 100, dtype=torch.float32).pin_memory()

    def outs(nq, k):
        return ids_flat[:nq * k].view(nq, k), sc_flat[:nq * k].view(nq, k)

    stream = torch.cuda.Stream(dev)
    ws = torch.empty(db.search_host_workspace_bytes(1024, 1000, 100), dtype=torch.uint8,
                     device=dev)
    for k in (10, 100):
        db.search_host(pool[:64], min(10 * k, 1024), k, *outs(64, k), ws=ws, stream=stream)
    stream.synchronize()
    for rate in rates:
        arr, sizes, ks, offs = _request_stream(rate, seconds, 20250602)
        # (a) continuous batching
        srv.reset_stats()
        t0 = time.perf_counter()
        rids = []
        for i in range(len(arr)):
            now = time.perf_counter() - t0
            if arr[i] > now:
                time.sleep(arr[i] - now)
            rids.append(srv.submit(pool[offs[i]:offs[i] + sizes[i]], int(ks[i])))
        for r in rids:
            srv.wait(r, timeout_s=600)
        wall = time.perf_counter() - t0
        st = srv.stats()
        served = {"qps": int(sizes.sum()) / wall, "p50_ms": st["p50_us"] / 1e3,
                  "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3,
                  "batches": st["batches"], "wall_s": wall}
        # (b) plain: one synchronous search per request, in arrival order
        lat = []
        t0 = time.perf_counter()
        for i in range(len(arr)):
            now = time.perf_counter() - t0
            if arr[i] > now:
                time.sleep(arr[i] - now)
            k = int(ks[i])
            nq = int(sizes[i])
            db.search_host(pool[offs[i]:offs[i] + nq], min(10 * k, 1024), k, *outs(nq, k),
                           ws=ws, stream=stream)
            stream.synchronize()
            lat.append(time.perf_counter() - t0 - arr[i])
        wall_p = time.perf_counter() - t0
        lat = np.array(lat) * 1e3
        plain = {"qps": int(sizes.sum()) / wall_p, "p50_ms": float(np.percentile(lat, 50)),
                 "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                 "wall_s": wall_p}
        out.append({"rate_req_s": rate, "requests": len(arr), "queries": int(sizes.sum()),
                    "offered_qps": int(sizes.sum()) / float(arr[-1]) if len(arr) > 1 else None,
                    "continuous_batching": served, "plain_per_request": plain})
    slots = srv.slots
    srv.close()
    return {"slots": slots, "sweep": out,
            "workload": "10Mx768 resident, Poisson arrivals, sizes logU[1,1024], "
                        "k in {10,100}, shortlist 10k reranked; each rate's stream run "
                        "through the server and as plain per-request calls"}


def main_reference(a):
    """CPU oracle on the same workload, one bounded sample per step."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2506_00528_gb300 import synth
    d = a.d
    x = a.x or (2 * d + 1) // 3
    n_rows = min(a.n, 100_000)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    U = synth.mixture_torch(n_rows, d, n_centres=a.centres, anisotropic=True,
                            stream=synth.STREAM_DB, device=dev)
    Qh = synth.mixture_torch(64, d, n_centres=a.centres, anisotropic=True,
                             stream=synth.STREAM_QUERIES, device=dev).cpu().numpy()
    vals = []
    samp = None
    for i in range(a.warmup + a.steps):
        v, info = cpu_oracle_sample(U, Qh, x, a.shortlist, a.k, a.n, n_rows=n_rows, n_q=2)
        samp = info["sample"]
        if i >= a.warmup:
            vals.append(v)
    value = float(np.median(vals))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1000.0 * a.batch / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8 ternary / f64", "data": "synthetic",
        "config": make_config(a, x, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": 1, "kind": "oracle",
                         "sample": samp},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def exact_topk(Qf, U, k, chunk=1 << 18):
    """Exact float32 top-k by scalar product (cosine on normalised rows)."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    nq = Qf.shape[0]
    best_s = torch.full((nq, k), -float("inf"), device=Qf.device)
    best_i = torch.zeros((nq, k), dtype=torch.int64, device=Qf.device)
    for c0 in range(0, U.shape[0], chunk):
        sc = Qf @ U[c0:c0 + chunk].T
        v, i = torch.topk(sc, min(k, sc.shape[1]), dim=1)
        cat_s = torch.cat([best_s, v], 1)
        cat_i = torch.cat([best_i, i + c0], 1)
        best_s, j = torch.topk(cat_s, k, dim=1)
        best_i = torch.gather(cat_i, 1, j)
    return best_i


def main_recall_sweep(a):
    """Recall of the ternary proxy against exact float32 cosine kNN, per x:
    ternary top-K vs exact top-K (recall@K), and the best k after reranking
    a 10k shortlist vs the exact top-k.  Reported, not pinned."""
    import torch
    from paper_2506_00528_gb300 import build as _build
    from paper_2506_00528_gb300 import evp, synth
    dev = torch.device("cuda", 0)
    _build.build()
    evp.load()
    n = a.n if a.n != 10_000_000 else 1_000_000
    d, nqs = a.d, a.sweep_queries
    U = synth.mixture_torch(n, d, n_centres=a.centres, anisotropic=True,
                            stream=synth.STREAM_DB, device=dev)
    Q = synth.mixture_torch(nqs, d, n_centres=a.centres, anisotropic=True,
                            stream=synth.STREAM_QUERIES, device=dev)
    K, k = 100, 10
    truth_K = exact_topk(Q, U, K).cpu().numpy()
    truth_k = truth_K[:, :k]
    out = {"kind": "recall_sweep", "n": n, "d": d, "queries": nqs, "path": "popcount",
           "data": "synthetic Gaussian mixture, 1024 centres, anisotropic, l2-normalised",
           "recall": {}}
    for x in sorted({64, 256, 384, evp.default_x(d)}):
        T = evp.encode(U, x)
        Tq = evp.encode(Q, x)
        db = evp.Database(T, U, d, x, tensor_copy=False)
        ids_K = torch.empty((nqs, K), dtype=torch.int64, device=dev)
        for q0 in range(0, nqs, 1024):
            ids, _ = db.knn(Tq[q0:q0 + 1024], K, path=1)
            ids_K[q0:q0 + 1024] = ids
        got_K = ids_K.cpu().numpy()
        rr_ids = torch.empty((nqs, k), dtype=torch.int64, device=dev)
        for q0 in range(0, nqs, 1024):
            ids, _ = db.search(Q[q0:q0 + 1024].contiguous(), 10 * k, k)
            rr_ids[q0:q0 + 1024] = ids
        got_rr = rr_ids.cpu().numpy()
        rec = lambda g, t, m: float(np.mean([len(set(a_[:m]) & set(b_[:m])) / m
                                             for a_, b_ in zip(g, t)]))
        out["recall"][str(x)] = {"recall_at_100": rec(got_K, truth_K, K),
                                 "recall_at_10": rec(got_K, truth_K, k),
                                 "rerank_10_of_100": rec(got_rr, truth_k, k)}
        db.close()
        del T, db
        torch.cuda.empty_cache()
    print(json.dumps(out))


def pack_ternary_torch(V):
    """Comparator helper: ternary int tensor [n, d] -> packed codes [n, 2W]
    (v+ words then v- words, bit j of word j // 64).  Used only for the
    b1.58 comparator codes, which the library does not produce."""
    import torch
    n, d = V.shape
    W = (d + 63) // 64
    pad = torch.zeros((n, 64 * W), dtype=torch.int64, device=V.device)
    pad[:, :d] = V.to(torch.int64)
    weights = torch.ones(64, dtype=torch.int64, device=V.device)
    weights[1:] = 2 ** torch.arange(1, 64, device=V.device, dtype=torch.int64)
    weights[63] = -(2 ** 63)
    p = ((pad == 1).to(torch.int64).view(n, W, 64) * weights).sum(-1)
    m = ((pad == -1).to(torch.int64).view(n, W, 64) * weights).sum(-1)
    return torch.cat([p, m], 1).contiguous()


def spearman_study(evp, synth, dev, d, nq=100, ns=1000):
    """Table 1's 'Uniform' rows through the library: uniform points on the
    sphere; proxy distances of all nq x ns pairs from the GPU scan (popcount
    path, exact ||q - s||^2 for any ternary codes) for the {x,d} EVP codes
    (evp_encode at the default x), the 1-bit codes ({d,d} EVP, evp_encode
    at x = d) and the b1.58 codes (comparator, per-vector absmean gamma);
    Spearman rho of each against the true Euclidean distance."""
    import torch
    from scipy.stats import spearmanr
    U = synth.uniform_sphere(nq + ns, d, stream=30 + d)
    Ud = torch.from_numpy(U).to(dev)
    true = np.linalg.norm(U[:nq, None, :].astype(np.float64) - U[None, nq:, :], axis=2)

    def all_pairs(T, x):
        ids, dist = evp.ternary_knn(T[:nq].contiguous(), T[nq:].contiguous(), d, x, ns,
                                    path=evp.PATH_POPC)
        D = torch.empty((nq, ns), dtype=torch.int32, device=dev)
        D.scatter_(1, ids, dist)
        return D.cpu().numpy()

    x = evp.default_x(d)
    st = evp.new_status(dev)
    D_evp = all_pairs(evp.encode(Ud, x, status=st), x)
    D_one = all_pairs(evp.encode(Ud, d, status=st), d)
    gamma = Ud.abs().mean(1, keepdim=True)
    B = torch.clamp(torch.round(Ud / (gamma + 1e-8)), -1, 1)
    D_b158 = all_pairs(pack_ternary_torch(B), d)
    torch.cuda.synchronize()
    evp.check_status(st, "spearman encode")
    t = true.ravel()
    return {"d": d, "x": x, "pairs": nq * ns,
            "rho_evp": float(spearmanr(t, D_evp.ravel()).correlation),
            "rho_1bit": float(spearmanr(t, D_one.ravel()).correlation),
            "rho_b158": float(spearmanr(t, D_b158.ravel()).correlation),
            "D_evp": D_evp, "true": true}


def main_spearman(a):
    """Table 1 ('Uniform-100', 'Uniform-1000') reproduced through the library."""
    import torch
    from paper_2506_00528_gb300 import build as _build
    from paper_2506_00528_gb300 import evp, synth
    _build.build()
    evp.load()
    dev = torch.device("cuda", 0)
    paper = {100: (0.80, 0.70, 0.75), 1000: (0.79, 0.64, 0.71)}
    rows = []
    for d in (100, 1000):
        r = spearman_study(evp, synth, dev, d)
        rows.append({k: v for k, v in r.items() if k not in ("D_evp", "true")} |
                    {"paper_evp_1bit_b158": paper[d]})
    print(json.dumps({"kind": "spearman", "data": "uniform points on the unit sphere "
                      "(the paper's Uniform rows), 100 x 1000 pairs per d",
                      "rows": rows}))


def main():
    a = parse()
    if a.spearman:
        return main_spearman(a)
    if a.impl == "reference":
        return main_reference(a)
    if a.recall_sweep:
        return main_recall_sweep(a)

    import torch
    import torch.distributed as dist

    from paper_2506_00528_gb300 import build as _build
    from paper_2506_00528_gb300 import dist as evp_dist
    from paper_2506_00528_gb300 import evp, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.barrier()
    evp.load()

    d, B, n, n_sl, k = a.d, a.batch, a.n, a.shortlist, a.k
    x = a.x or evp.default_x(d)
    W = evp.words(d)
    # ---- resident database (replicas only: every rank holds the same one)
    U = synth.mixture_torch(n, d, n_centres=a.centres, anisotropic=True,
                            stream=synth.STREAM_DB, device=dev)
    st = evp.new_status(dev)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    S = evp.encode(U, x, status=st)
    t1.record()
    torch.cuda.synchronize()
    evp.check_status(st, "database encode")
    db_encode_ms = t0.elapsed_time(t1)
    # ---- query batches: distinct per step (cycled pool of 8)
    pool = 8
    Qall = synth.mixture_torch(pool * B, d, n_centres=a.centres, anisotropic=True,
                               stream=synth.STREAM_QUERIES + 10 * rank, device=dev)
    Qb = [Qall[i * B:(i + 1) * B] for i in range(pool)]
    db = evp.Database(S, U, d, x, tensor_copy=(a.path in (0, 2)))
    Tq = torch.empty((B, 2 * W), dtype=torch.int64, device=dev)
    sl = torch.empty((B, n_sl), dtype=torch.int64, device=dev)
    sd = torch.empty((B, n_sl), dtype=torch.int32, device=dev)
    rid = torch.empty((B, k), dtype=torch.int64, device=dev)
    rsc = torch.empty((B, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    Q8 = torch.empty((B, d), dtype=torch.int8, device=dev)
    if a.path == 0:
        ws = torch.empty(db.search_workspace_bytes(B, n_sl, k), dtype=torch.uint8, device=dev)
    elif a.path == 4:   # int8 queries: the asymmetric tensor-core scan
        ws = torch.empty(int(evp.load().ternary_knn_i8q_workspace(B, n, d, n_sl)),
                         dtype=torch.uint8, device=dev)
    elif a.path == 5:   # sparse database codes
        E = evp.pack_sparse(S, d, x, status=st)
        ws = torch.empty(int(evp.load().ternary_knn_sparse_workspace(B, n, d, x, n_sl)),
                         dtype=torch.uint8, device=dev)
    else:
        ws = torch.empty(int(evp.load().evp_db_knn_workspace(db.handle, B, n_sl, a.path)),
                         dtype=torch.uint8, device=dev)

    def step(Q):
        if a.path == 0:   # one C-ABI call: encode -> scan -> rerank
            db.search(Q, n_sl, k, ids=rid, scores=rsc, ws=ws, status=st, stream=stream)
        elif a.path == 4:  # quantize -> asymmetric scan (masked-addition score) -> rerank
            evp.quantize_i8(Q, out=Q8, status=st, stream=stream)
            evp.ternary_knn_i8q(Q8, S, d, x, n_sl, ids=sl, score=sd, ws=ws, status=st,
                                stream=stream)
            evp.rerank(Q, U, sl, k, ids=rid, scores=rsc, status=st, stream=stream)
        elif a.path == 5:  # encode -> scan of the sparse codes -> rerank
            evp.encode(Q, x, out=Tq, status=st, stream=stream)
            evp.ternary_knn_sparse(Tq, E, d, x, n_sl, ids=sl, dist=sd, ws=ws, status=st,
                                   stream=stream)
            evp.rerank(Q, U, sl, k, ids=rid, scores=rsc, status=st, stream=stream)
        else:             # the same three steps with the scan path forced
            evp.encode(Q, x, out=Tq, status=st, stream=stream)
            db.knn(Tq, n_sl, ids=sl, dist=sd, ws=ws, status=st, stream=stream, path=a.path)
            evp.rerank(Q, U, sl, k, ids=rid, scores=rsc, status=st, stream=stream)

    for i in range(a.warmup):
        step(Qb[i % pool])
    torch.cuda.synchronize()
    evp.check_status(st, "warmup")

    # ---- device-resident timing (the library's kernel timing is off here)
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(a.steps):
        step(Qb[i % pool])
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    evp.check_status(st, "timed steps")
    # replicas: every rank searched its own B queries per step; the job's
    # throughput is all ranks' queries over the slowest rank's time
    total_q, ms = evp_dist.aggregate(B * a.steps, ms, device=dev)
    ms_per_step = ms / a.steps
    value = total_q / (ms / 1000.0)

    # ---- per-kernel durations: the same steps again, with the library's
    # CUDA events around each of its launches (on the launching stream)
    evp.timing_reset()
    evp.timing_enable(True)
    for i in range(a.steps):
        step(Qb[i % pool])
    torch.cuda.synchronize()
    evp.timing_enable(False)
    per_kernel = {name: evp.timing_read(name) for name in
                  ("encode", "quantize", "scan_init", "scan_popc", "unpack_fp4", "scan_mma",
                   "scan_mma_packed", "scan_i8q", "scan_sparse", "final_merge", "scan_repair",
                   "rerank")}
    evp.check_status(st, "timed kernels")

    # ---- end to end through the API with host buffers (pinned)
    Qh = [q.cpu().pin_memory() for q in Qb]
    ids_h = torch.empty((B, k), dtype=torch.int64).pin_memory()
    sc_h = torch.empty((B, k), dtype=torch.float32).pin_memory()
    ws_h = torch.empty(db.search_host_workspace_bytes(B, n_sl, k), dtype=torch.uint8, device=dev)
    Qd = torch.empty((B, d), dtype=torch.float32, device=dev)

    def step_host(i):
        if a.path == 0:   # evp_db_search_host: H2D, encode, scan, rerank, D2H
            db.search_host(Qh[i % pool], n_sl, k, ids_h, sc_h, ws=ws_h, status=st, stream=stream)
        else:
            Qd.copy_(Qh[i % pool], non_blocking=True)
            step(Qd)
            ids_h.copy_(rid, non_blocking=True)
            sc_h.copy_(rsc, non_blocking=True)

    for i in range(a.warmup):
        step_host(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for i in range(a.steps):
        step_host(i)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_q, e2e_ms = evp_dist.aggregate(B * a.steps, e2e_ms, device=dev)
    e2e_value = e2e_q / (e2e_ms / 1000.0)

    # ---- measured tensor-core peak (the probe), then the roofline of the
    # dominant kernel
    hbm_peak, bf16_peak, peak_src = load_peaks()
    tpeak = None if a.no_probe else measure_tensor_peak(evp, ClockSampler, local)
    fp8_2x_bf16 = 2.0 * bf16_peak          # nominal fp8 : bf16 dense ratio 2 : 1
    fp4_4x_bf16 = 4.0 * bf16_peak          # block-scaled fp4 (mxf4) : bf16, 4 : 1 per clock (probe)
    if tpeak:
        fp8_peak = max(tpeak["f8_pair_m256_n256"]["tflops"], tpeak["f8_m128_n256"]["tflops"])
        fp4_peak = max(tpeak["f4_pair_m256_n256"]["tflops"], tpeak["f4_m128_n256"]["tflops"])
        fp8_src = (f"fp8 dense measured by evp_probe_tensor_rate on every SM "
                   f"({fp8_peak:.0f} TFLOP/s at {tpeak['f8_pair_m256_n256']['sm_mhz']} MHz); "
                   f"2 x measured bf16 = {fp8_2x_bf16:.0f} beside it; HBM {hbm_peak} GB/s "
                   f"({peak_src})")
        fp4_src = (f"fp4 (kind::mxf4) dense measured by evp_probe_tensor_rate on every SM "
                   f"({fp4_peak:.0f} TFLOP/s at {tpeak['f4_pair_m256_n256']['sm_mhz']} MHz); "
                   f"4 x measured bf16 = {fp4_4x_bf16:.0f} beside it; HBM {hbm_peak} GB/s "
                   f"({peak_src})")
    else:
        fp8_peak = fp8_2x_bf16
        fp4_peak = fp4_4x_bf16
        fp8_src = f"fp8 dense = 2 x bf16 {bf16_peak} TFLOP/s ({peak_src}); HBM {hbm_peak} GB/s"
        fp4_src = (f"fp4 (kind::mxf4) dense = 4 x bf16 {bf16_peak} TFLOP/s ({peak_src}); "
                   f"HBM {hbm_peak} GB/s")
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    n_mma, mma_ms = per_kernel["scan_mma"]
    n_scan, scan_ms = per_kernel["scan_popc"]
    n_pk, pk_ms = per_kernel["scan_mma_packed"]
    n_iq, iq_ms = per_kernel["scan_i8q"]
    n_sp, sp_ms = per_kernel["scan_sparse"]
    if iq_ms > 0 or sp_ms > 0:
        # asymmetric scan: one launch per <= 32 int8 queries reads the packed
        # codes (16 W bytes per row); sparse scan: one launch per <= 4
        # queries reads the sparse codes (2 x bytes per row)
        name, cnt, tot = ("scan_i8q", n_iq, iq_ms) if iq_ms > 0 else ("scan_sparse", n_sp, sp_ms)
        avg = tot / max(1, cnt)
        per_row = 16 * W if iq_ms > 0 else 2 * x
        gbs = float(n) * per_row / (avg / 1e3) / 1e9
        roofline = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                    "unit": "GB/s", "frac": gbs / hbm_peak, "traffic": None,
                    "peak_source": f"HBM {hbm_peak} GB/s ({peak_src})", "launches": cnt,
                    "avg_ms": avg, "bytes_per_row_per_launch": per_row,
                    "queries_per_launch": 32 if iq_ms > 0 else 4}
        if iq_ms > 0 and tpeak:
            # two MMAs per K step (the query's hi and lo parts) per 128-row tile
            cyc = tpeak["f8_m128_n64" if B > 16 else "f8_m128_n16"]["cycles_per_mma"]
            mmas = float((n + 127) // 128) * 4 * W
            mhz = clocks.get("sm_mhz") or 2070.0
            roofline["mma_instruction_floor_ms"] = mmas * cyc / sm_count / (mhz * 1e6) * 1e3
            roofline["frac_of_mma_instruction_floor"] = roofline["mma_instruction_floor_ms"] / avg
        dtype = ("int8 query x e4m3 split (16 hi + lo) -> f32 tensor-core scan (exact)"
                 if iq_ms > 0 else "uint16 sparse codes, byte-packed table lookups -> int32 Delta")
    elif pk_ms > max(mma_ms, scan_ms):
        # packed tensor-core scan: one launch per <= 64 queries reads the
        # packed codes (16 W bytes per row) once; 2 d flops per (query, row).
        # Its instruction shape (M = 128, N <= 64) has a fixed cost per MMA,
        # so its tensor ceiling is the probe's rate at that N.
        avg = pk_ms / max(1, n_pk)
        passes_per_step = (B + 63) // 64
        qn = 16 if B <= 16 else 32 if B <= 32 else 64
        bytes_per_launch = float(n) * 16 * W
        flops = 2.0 * d * n * (B / passes_per_step)
        gbs = bytes_per_launch / (avg / 1e3) / 1e9
        tflops = flops / (avg / 1e3) / 1e12
        tensor_frac, hbm_frac = tflops / fp8_peak, gbs / hbm_peak
        bound = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                 "frac": hbm_frac}
        if tensor_frac >= hbm_frac:
            bound = {"bound": "tensor", "achieved": tflops, "peak": fp8_peak,
                     "unit": "TFLOP/s", "frac": tensor_frac}
        roofline = {
            "kernel": "scan_mma_packed", **bound,
            "traffic": measured_traffic("scan_mma_packed", n, d, B, a.shortlist),
            "tensor_frac": tensor_frac, "hbm_frac": hbm_frac, "packed_gbs": gbs,
            "peak_source": fp8_src, "launches": n_pk, "avg_ms": avg,
        }
        if tpeak:
            # MMA instructions per launch over the probe's instruction rate at this N
            key = "f8_m128_n64" if qn == 64 else "f8_m128_n16"
            cyc = tpeak[key]["cycles_per_mma"]
            mmas = float((n + 127) // 128) * W           # 128-row tiles x K steps (64 elements, e2m1)
            mhz = clocks.get("sm_mhz") or 2070.0
            floor_ms = mmas * cyc / sm_count / (mhz * 1e6) * 1e3
            roofline["mma_instruction_floor_ms"] = floor_ms
            roofline["frac_of_mma_instruction_floor"] = floor_ms / avg
        dtype = "e4m3 x e4m3 -> f32 tensor-core scan (exact on -1/0/+1), f32 encode/rerank"
    elif mma_ms >= scan_ms:
        # tensor-core scan: algorithmic flops = 2 d per (query, row) pair; it
        # reads the database's e2m1 copy (Kp bytes per row, two elements a
        # byte) once per launch, which binds instead for small batches
        avg = mma_ms / max(1, n_mma)
        flops = 2.0 * d * B * n * (a.steps / max(1, n_mma))
        kp = (d + 255) // 256 * 128
        fp4_bytes = float(n) * kp
        tflops = flops / (avg / 1e3) / 1e12
        gbs = fp4_bytes / (avg / 1e3) / 1e9
        tensor_frac, hbm_frac = tflops / fp4_peak, gbs / hbm_peak
        if tensor_frac >= hbm_frac:
            bound = {"bound": "tensor", "achieved": tflops, "peak": fp4_peak, "unit": "TFLOP/s",
                     "frac": tensor_frac}
        else:
            bound = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": hbm_frac}
        roofline = {
            "kernel": "scan_mma", **bound,
            "traffic": measured_traffic("scan_mma", n, d, B, a.shortlist),
            "tensor_frac": tensor_frac, "hbm_frac": hbm_frac, "fp4_gbs": gbs,
            "peak_4x_bf16": fp4_4x_bf16, "frac_vs_4x_bf16": tflops / fp4_4x_bf16,
            "frac_vs_fp8_peak": tflops / fp8_peak,
            "peak_source": fp4_src, "launches": n_mma, "avg_ms": avg,
        }
        dtype = "e2m1 x e2m1 -> f32 tensor-core scan (kind::mxf4, unit scales; exact on -1/0/+1), f32 encode/rerank"
    else:
        # popcount scan: one pass over the codes per <= 16 queries; per
        # (query, row) pair 4W 32-bit popcounts
        avg = scan_ms / max(1, n_scan)
        passes_per_step = (B + 15) // 16
        pairs_per_launch = n * (B / passes_per_step)
        popc_per_launch = pairs_per_launch * 4 * W
        bytes_per_launch = n * 16 * W
        popc_peak = POPC_PER_CLK_PER_SM * sm_count * 2070e6
        hbm_bound = B <= 3
        roofline = {
            "kernel": "scan_popc",
            "bound": "hbm" if hbm_bound else "alu",
            "achieved": (bytes_per_launch / (avg / 1e3) / 1e9) if hbm_bound
            else popc_per_launch / (avg / 1e3) / 1e12,
            "peak": hbm_peak if hbm_bound else popc_peak / 1e12,
            "unit": "GB/s" if hbm_bound else "Tpopc/s",
            "frac": (bytes_per_launch / (avg / 1e3) / 1e9 / hbm_peak) if hbm_bound
            else (popc_per_launch / (avg / 1e3)) / popc_peak,
            "traffic": measured_traffic("scan_popc", n, d, B, a.shortlist),
            "hbm_achieved_gbs": bytes_per_launch / (avg / 1e3) / 1e9,
            "popc_achieved_tops": popc_per_launch / (avg / 1e3) / 1e12,
            "peak_source": f"POPC 16/clk/SM (probe) x {sm_count} SMs x 2070 MHz; HBM {peak_src}",
            "launches": n_scan, "avg_ms": avg,
        }
        dtype = "u64 bitplanes, popcount -> int32 Delta; f32 encode/rerank"
    kernels = {nm: {"launches": c, "total_ms": round(t, 3)} for nm, (c, t) in per_kernel.items()}

    # ---- recall@10 against exact float32 cosine kNN, over the whole batch,
    # for the bench's x and for the other x of the paper's table
    recall = None
    if not a.no_recall:
        Qr = Qb[0]
        truth = exact_topk(Qr, U, k).cpu().numpy()
        rec = lambda g, t: float(np.mean([len(set(a_[:k]) & set(b_[:k])) / k
                                          for a_, b_ in zip(g, t)]))
        step(Qb[0])
        torch.cuda.synchronize()
        got_rr = rid.cpu().numpy()
        tern_ids, _ = db.knn(evp.encode(Qr, x), k)
        recall = {"queries": B, "x": x, "rerank_10_at_100": rec(got_rr, truth),
                  "ternary_10_at_10": rec(tern_ids.cpu().numpy(), truth), "per_x": {}}
        if a.path == 4:
            # the asymmetric ranking itself (int8 queries against the codes)
            a_ids, _ = evp.ternary_knn_i8q(evp.quantize_i8(Qr), S, d, x, k)
            recall["asymmetric_10_at_10"] = rec(a_ids.cpu().numpy(), truth)
        for xx in (64, 256, 384, x):
            Tx = evp.encode(U, xx)
            dbx = evp.Database(Tx, U, d, xx)
            r_ids, _ = dbx.search(Qr, n_sl, k)
            t_ids, _ = dbx.knn(evp.encode(Qr, xx), k)
            recall["per_x"][str(xx)] = {"rerank_10_at_100": rec(r_ids.cpu().numpy(), truth),
                                        "ternary_10_at_10": rec(t_ids.cpu().numpy(), truth)}
            dbx.close()
            del Tx, dbx
            torch.cuda.empty_cache()

    # ---- batched and served forms (rank 0, N = 1)
    forms = None
    if not a.no_forms and world == 1:
        rates = [float(r) for r in a.serve_rates.split(",") if r]
        served = measure_served(evp, synth, db, d, a.serve_seconds, rates, dev)
        batched = measure_batched(evp, synth, dev)
        forms = {"batched": batched, "served": served}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1)
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        v, info = cpu_oracle_sample(U, Qall[:64].cpu().numpy(), x, n_sl, k, n)
        cpu = {"value": v, "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": info["sample"], "all_cores": info["all_cores"],
               "euclidean_fp32": info["euclidean_fp32"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic",
            "config": make_config(a, x, world),
            "scanned_gbs_logical": B * n * 16 * W / (ms_per_step / 1e3) / 1e9,
            "db_encode": {"rows": n, "ms": db_encode_ms,
                          "gbs": n * (4 * d + 16 * W) / (db_encode_ms / 1e3) / 1e9},
            "roofline": roofline,
            "tensor_peak_probe": tpeak,
            "kernels": kernels,
            "recall_at_10": recall,
            "forms": forms,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "queries/s",
                    "h2d_bytes_per_step": B * d * 4, "d2h_bytes_per_step": B * k * 12},
            "gpu_launches": sum(c for c, _ in per_kernel.values()),
            "clocks": clocks,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
