#!/usr/bin/env python3
"""DPC points/sec on one GB300: density + dependent points (+ clusters).

Headline workload: n = 1,280,000 unit-norm rows of d = 1024 (1,000 vMF-like
clusters, concentration log-uniform in [20, 200], log-normal sizes; inner
product), k = 16, product center with 1,000 clusters, on the brute-force index
(Sec. 5.1: exact k-NN; tensor-core screen, exact FP32 decision). On this data
the Vamana graph (R = 64) stays far below the 0.95 k-NN recall the metric is
quoted at (0.64 at beam 200, 0.69 at beam 1,600), so the exact index is the
configuration that meets it; the graph path is reported beside it.

A step is one pass of the path over the whole point set: k-NN + density,
dependent points, the cluster cut. The same JSON line carries, under
"variants", report lines measured in the same run:
  * the 1.28M x 1024 set on a Vamana graph (R 64, beam 200) with FP32, BF16
    and FP8-e4m3 traversal and exact FP32 re-rank, recall and ARI judged
    against the exact index at full n;
  * n = 1,000,000 x d = 128 uint8 (100 Zipf-weighted Gaussians + 5% noise) on
    its Vamana graph (R 64, beam 128, k 10), on an NN-Descent graph, on an
    HCNNG graph (all searched with the same beam) and on the exact index.
Graph builds are timed separately (build_s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload vmf1024|vmf1024-graph|u8-1m|batched64|sphere384]
                  [--quick] [--graph-line-only | --exact-line-only] [--n N]

Prints one JSON line (rank 0). For N > 1 (torchrun) every rank runs its own
replica of the workload on its GPU; value = all points processed / the max
over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DPC points/sec (density + dependent-point search) at >=0.95 recall; % HBM peak"
UNIT = "points/s"

VMF = dict(n=1_280_000, d=1024, components=1000, k=16, n_clusters=1000, R=64, L=200, L_build=400, alpha=1.2,
           build_passes=2, n_start=10485)
VMF_NAME = ("vmf-like unit-norm n=1,280,000 d=1024 inner product (1,000 clusters, kappa log-uniform [20,200], "
            "log-normal sizes); kth density k=16; product center 1000")
U8 = dict(n=1_000_000, d=128, components=100, R=64, L=128, alpha=1.2, k=10, n_clusters=100, L_build=256,
          n_start=8192, build_passes=2)
U8_NAME = ("u8-gaussian-mixture n=1,000,000 d=128 (100 components, Zipf 1.1 weights, sigma U[5,20], "
           "5% uniform noise); kth density k=10; product center 100")
# NN-Descent graph of the uint8 rows (report line): K-lists, 3 repeats and alpha 1.1 as in the paper's
# comparison of graph indices; rounds stop earlier when no list changes
NND = dict(K=32, repeats=3, rounds=12, alpha=1.1)
# HCNNG graph of the uint8 rows (report line): leaves of up to 200 points (the kernel's limit) and
# spanning forests of degree <= 3 need more repeats than the paper's 3 on these rows (k-NN recall at
# beam 128: 0.30 / 0.55 / 0.72 / 0.85 with 3 / 8 / 16 / 32 repeats); 32 are used
HC = dict(repeats=32, leaf=200, mst_deg=3, alpha=1.1)
CPU_SAMPLE = 16       # points per oracle timing sample (brute-force index on the full rows)
CPU_SAMPLE_GRAPH = 256  # points per oracle timing sample (beam search on the same graph)
RECALL_QUERIES = 200  # FP64 exact k-NN of sampled points (CPU)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=0, help="points (profiling runs use fewer; 0 = the workload's)")
    ap.add_argument("--quick", action="store_true",
                    help="headline only: no variants, recall, e2e or CPU baseline")
    ap.add_argument("--variant-steps", type=int, default=2, help="timed steps of each report line")
    ap.add_argument("--graph-line-only", action="store_true",
                    help="u8-1m / vmf1024-graph: the Vamana FP32 (or uint8) graph line alone, without CPU baseline, "
                         "e2e or recall (for short profiling runs)")
    ap.add_argument("--exact-line-only", action="store_true",
                    help="u8-1m: the exact-index line alone, without CPU baseline or recall (profiling runs)")
    ap.add_argument("--workload", default="vmf1024",
                    choices=["vmf1024", "vmf1024-graph", "u8-1m", "batched64", "sphere384"],
                    help="vmf1024: the benchmark line (with its variants); vmf1024-graph / u8-1m: report lines alone")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"pecann_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers

def max_over_ranks(elapsed_s: float, dist=None, device=None) -> float:
    """The slowest rank's timed region (every rank gets it)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return elapsed_s
    import torch

    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(points_per_rank: int, steps: int, world: int, elapsed_s: float) -> float:
    """Whole-job points/s of `world` replicas that each processed
    points_per_rank points `steps` times within the slowest rank's time."""
    return world * points_per_rank * steps / elapsed_s


# the sources each profiled kernel is built from: a profile's counters stand
# for the kernel only while these files are unchanged
KERNEL_SOURCES = {
    "k_bf_screen": ["bf_screen.cu", "tcgen05.cuh", "common.cuh"],
    "k_search": ["search.cu", "search_kernel.cuh", "search_common.cuh", "search_u8.cu", "search_f32.cu",
                 "search_f32ip.cu", "search_bf16.cu", "search_fp8.cu", "dispatch.cuh", "common.cuh", "internal.h"],
}


def source_sha(kernel: str | None = None) -> str:
    """Digest of the named kernel's sources (all of csrc/ when None)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2312_03940_gb300", "csrc")
    files = KERNEL_SOURCES.get(kernel) if kernel else None
    for f in sorted(files if files else os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch recorded by the ncu summary under profiles/, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_sha") != source_sha(vals.get("kernel_sources")):
        return None
    try:
        return float(vals["traffic_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- workloads

def vmf_data(n):
    from paper_2312_03940_gb300 import synth

    return synth.vmf_like(n=n, d=VMF["d"], components=VMF["components"])


def u8_data(n):
    from paper_2312_03940_gb300 import synth

    return synth.u8_mixture(n=n, d=U8["d"], components=U8["components"])


def cpu_knn_rate(X, metric, G, L, k, m, threads, steps=1, seed=11):
    """The oracle as it stands, timed on the host cores: k-NN + density of m
    sampled points of the same rows (G None: the brute-force index; else
    Algorithm 1 on the same graph). Returns (points/s, seconds, sample text)."""
    import oracle
    from paper_2312_03940_gb300 import synth

    P = oracle.Points(X, metric=metric)
    dt = 0.0
    for s in range(steps):
        rows = synth.sample_ids(len(X), m, seed=seed + s)
        t0 = time.perf_counter()
        oracle.knn_density_rows(P, G, rows, L=L, k=k, threads=threads)
        dt += time.perf_counter() - t0
    return m * steps / dt, dt


def exact_recall(X, metric, knn_dist, k, m=RECALL_QUERIES, seed=12):
    """Tie-aware k-NN recall of sampled points against the FP64 exact k-NN."""
    from oracle import exact
    from paper_2312_03940_gb300 import synth

    qs = synth.sample_ids(len(X), m, seed=seed)
    _, ex = exact.exact_knn_queries(X, qs, k, metric=exact.IP if metric == 1 else exact.L2)
    return exact.knn_recall(knn_dist[qs], ex)


def full_recall(got_dist, exact_dist):
    """Tie-aware recall over every point, against exact k-NN distances."""
    kth = exact_dist[:, -1:]
    return float((got_dist <= kth * (1.0 + 1e-5) + 1e-30).mean())


def timed(step, warmup, steps, stream):
    """W untimed steps, then K steps between CUDA events on `stream`; also the
    per-step density-call events that step() records. Returns seconds."""
    import torch

    for _ in range(warmup):
        step(None)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dens = []
    e0.record(stream)
    for _ in range(steps):
        step(dens)
    e1.record(stream)
    torch.cuda.synchronize()
    dens_ms = [a.elapsed_time(b) for a, b in dens]
    return e0.elapsed_time(e1) / 1e3, (float(np.mean(dens_ms)) if dens_ms else None)


class Path:
    """One DPC configuration on one dataset: the calls of a step, reusing
    outputs and workspace."""

    def __init__(self, ds, G, p, dev):
        import torch

        from paper_2312_03940_gb300 import pecann as pc

        self.pc, self.ds, self.G, self.p = pc, ds, G, p
        n = ds.n
        self.ws = pc.workspace(ds, p)
        self.cws = torch.empty(8 * n + (1 << 20), dtype=torch.uint8, device=dev)
        self.dens = dict(knn_ids=torch.empty((n, p.k), dtype=torch.int32, device=dev),
                         knn_dist=torch.empty((n, p.k), dtype=torch.float32, device=dev),
                         density=torch.empty(n, dtype=torch.float32, device=dev),
                         rank_key=torch.empty(n, dtype=torch.float32, device=dev))
        self.dep = dict(dep=torch.empty(n, dtype=torch.int32, device=dev),
                        dep_dist=torch.empty(n, dtype=torch.float32, device=dev))
        self.labels = torch.empty(n, dtype=torch.int32, device=dev)
        self.stats = None

    def step(self, dens_events=None, ds=None, G=None):
        import torch

        pc = self.pc
        ds = ds or self.ds
        G = self.G if G is None else G
        if dens_events is not None:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
        torch.cuda.nvtx.range_push("pecann_density")
        pc.pecann_density(ds, G, self.p, ws=self.ws, out=self.dens)
        torch.cuda.nvtx.range_pop()
        if dens_events is not None:
            b.record()
            dens_events.append((a, b))
        r = pc.pecann_dependent_points(ds, G, self.p, self.dens["rank_key"], self.dens["knn_ids"],
                                       self.dens["knn_dist"], ws=self.ws, out=self.dep)
        self.stats = r["stats"]
        pc.pecann_cluster(self.dens["density"], self.dep["dep"], self.dep["dep_dist"], self.p, ws=self.cws,
                          count=False, labels=self.labels)

    def screen_counts(self):
        """Brute-force index: points of the last call that took the collect
        pass and that the exact SIMT kernels took."""
        return [int(x) for x in self.ws[24:32].cpu().view(__import__("torch").int32).tolist()]


def e2e_rate(path, X_host, G_host, steps):
    """The same metric end to end through the public calls: every step copies
    the rows (and graph) in from pinned host memory and reads rho, dependent
    points, their distances and the labels back."""
    import torch

    from paper_2312_03940_gb300 import pecann as pc

    dev = path.ds.X.device
    Xh = torch.from_numpy(X_host).pin_memory()
    Xd = torch.empty_like(path.ds.X)
    ds = pc.Dataset(Xd, metric=path.ds.metric)
    Gh = G_host.pin_memory() if G_host is not None else None
    Gd = torch.empty_like(path.G) if G_host is not None else None
    n = path.ds.n
    outs = [torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
            torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        Xd.copy_(Xh, non_blocking=True)
        if Gd is not None:
            Gd.copy_(Gh, non_blocking=True)
        path.step(None, ds=ds, G=Gd)
        for h, d in zip(outs, [path.dens["density"], path.dep["dep"], path.dep["dep_dist"], path.labels]):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    h2d = int(Xh.numel() * Xh.element_size() + (Gh.numel() * 4 if Gh is not None else 0))
    return {"value": n / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(16 * n)}


_COUNTS = {}


def graph_roofline(X, metric, Gh, p, row_bytes, dens_s, n, kernel, peak_key="hbm_gbs", traffic_tag=None):
    """Algorithmic bytes of the k-NN beam search per launch: E_q out-lists of
    4R bytes, (C_q + 1) rows, 8k bytes of output and 8 bytes of density per
    query, with E_q and C_q counted by the oracle on 1,000 sampled queries of
    the same graph (its trajectory is the GPU's FP32 trajectory)."""
    import oracle
    from paper_2312_03940_gb300 import synth

    key = (id(Gh), p.L_search)
    if key not in _COUNTS:
        P = oracle.Points(X, metric=metric)
        _COUNTS[key] = oracle.search_counts(P, Gh, synth.sample_ids(n, 1000, seed=99), L=p.L_search)
    e_q, c_q = _COUNTS[key]
    bytes_q = e_q.mean() * 4 * p.R + (c_q.mean() + 1) * row_bytes + 8 * p.k + 8
    alg = bytes_q * n
    pk, src = peaks()
    ach = alg / dens_s / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": pk[peak_key], "peak_source": src,
            "unit": "GB/s", "frac": ach / pk[peak_key], "traffic": profiled_traffic(traffic_tag) if traffic_tag else None,
            "algorithmic_bytes_per_launch": alg, "E_q": float(e_q.mean()), "C_q": float(c_q.mean())}


def screen_roofline(n, d, collect_rows, dens_s, traffic_tag=None):
    """Algorithmic tensor FLOPs of the brute-force screen per density call:
    2 n^2 d for the keep pass plus 2 m n d for the m points of the collect
    pass, over the whole call (screen, collect, exact re-rank)."""
    pk, src = peaks()
    flops = 2.0 * n * n * d + 2.0 * collect_rows * n * d
    ach = flops / dens_s / 1e12
    peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    return {"kernel": "k_bf_screen (BF16 tcgen05 screen of the k-NN pass, whole density call)", "bound": "tensor",
            "achieved": ach, "peak": peak, "peak_source": src + " (bf16, sustained)", "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": profiled_traffic(traffic_tag) if traffic_tag else None,
            "algorithmic_flops_per_launch": flops, "collect_rows": int(collect_rows)}


# ---------------------------------------------------------------- reference arm (the CPU oracle)

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    threads = oracle.default_threads()
    n = args.n or VMF["n"]
    X, _ = vmf_data(n)
    for _ in range(args.warmup):
        cpu_knn_rate(X, 1, None, 0, VMF["k"], CPU_SAMPLE, threads, seed=500)
    rate, dt = cpu_knn_rate(X, 1, None, 0, VMF["k"], CPU_SAMPLE, threads, steps=args.steps)
    sample = (f"oracle brute-force index (exact k-NN + kth density, canonical FP32) of {CPU_SAMPLE} sampled points "
              f"per step over all {n:,} rows of the same workload, {args.steps} steps; the dependent step is not in "
              f"the sample (so the CPU rate is an upper bound)")
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1000 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": VMF_NAME if n == VMF["n"] else VMF_NAME.replace("1,280,000", f"{n:,}"),
                      "index": "brute force (exact)", "oracle_points_per_step": CPU_SAMPLE},
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch

    from paper_2312_03940_gb300 import build as pbuild
    from paper_2312_03940_gb300 import pecann as pc
    from paper_2312_03940_gb300 import synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0:
        pbuild.build()
    if dist:
        dist.barrier()
    pc.load_library()
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()

    # ---- the headline: 1.28M x 1024 on the brute-force index
    n = args.n or VMF["n"]
    X, gt = vmf_data(n)
    Xd = torch.from_numpy(X).to(dev)
    ds = pc.Dataset(Xd, metric=pc.IP)
    p = pc.params(k=VMF["k"], R=VMF["R"], L_search=VMF["L"], L_dep=VMF["L"], center=pc.CENTER_PRODUCT,
                  n_clusters=VMF["n_clusters"], index=pc.INDEX_BRUTE_FORCE)
    path = Path(ds, None, p, dev)
    path.step(None)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = pc.pecann_kernel_launches()
    elapsed, dens_ms = timed(path.step, args.warmup, args.steps, stream)
    barrier()
    launches = pc.pecann_kernel_launches() - l0
    clk = clocks.stop()
    elapsed = max_over_ranks(elapsed, dist, dev)
    counts = path.screen_counts()  # of the last dependent call
    path.pc.pecann_density(ds, None, p, ws=path.ws, out=path.dens)
    knn_counts = path.screen_counts()
    torch.cuda.synchronize()
    name = VMF_NAME if n == VMF["n"] else VMF_NAME.replace("1,280,000", f"{n:,}")
    result = {"metric": METRIC, "value": replica_throughput(n, args.steps, world, elapsed), "unit": UNIT,
              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": elapsed * 1000 / args.steps, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": {"workload": name, "index": "brute force (exact; BF16 tcgen05 screen, FP32 canonical decision)",
                         "n": n, "d": VMF["d"], "k": VMF["k"], "metric": "inner product",
                         "parallelism": "replicas" if world > 1 else "single-gpu",
                         "l2": "inputs (5.2 GB FP32 rows) exceed the 129 MB L2; no flush between steps"},
              "gpu_launches": int(launches), "clocks": clk, "density_ms": dens_ms,
              "unfinished_after_round0": int(path.stats[1]), "screen_collect_rows_knn": knn_counts[0],
              "screen_simt_rows_knn": knn_counts[1], "screen_collect_rows_dep": counts[0],
              "screen_simt_rows_dep": counts[1],
              "roofline": screen_roofline(n, VMF["d"], knn_counts[0], dens_ms / 1e3, traffic_tag="k_bf_screen_vmf1024")}
    if rank == 0 and not args.quick:
        import oracle
        from oracle import exact

        oracle.build()
        threads = oracle.default_threads()
        knn_dist = path.dens["knn_dist"].cpu().numpy()
        exact_labels = path.labels.cpu().numpy()
        result["recall"] = exact_recall(X, 1, knn_dist, VMF["k"])
        result["recall_queries"] = RECALL_QUERIES
        result["ari_vs_generator"] = exact.ari(exact_labels, gt)
        result["e2e"] = e2e_rate(path, X, None, max(2, min(args.steps, 3)))
        rate, dt = cpu_knn_rate(X, 1, None, 0, VMF["k"], CPU_SAMPLE, threads)
        result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                  "sample": (f"oracle brute-force index (exact k-NN + kth density) of {CPU_SAMPLE} "
                                             f"sampled points over all {n:,} rows of the same workload; the "
                                             f"dependent step is not in the sample (an upper bound)")}
        # the report lines run on one GPU only: a multi-GPU run measures the
        # benchmark line's replicas, whose ranks would otherwise wait meanwhile
        if world == 1:
            # ---- variants: the same rows on a Vamana graph, FP32 / BF16 / FP8 traversal
            result["variants"] = vmf_graph_variants(args, X, Xd, knn_dist, exact_labels, dev, stream, threads)
            del path
            torch.cuda.empty_cache()
            # ---- the uint8 workload on its graph and on the exact index
            del Xd, ds
            torch.cuda.empty_cache()
            result["variants"] += u8_variants(args, dev, stream, threads)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def vmf_graph_variants(args, X, Xd, exact_dist, exact_labels, dev, stream, threads):
    import torch

    from oracle import exact
    from paper_2312_03940_gb300 import pecann as pc
    from paper_2312_03940_gb300 import synth

    n = len(X)
    p = pc.params(k=VMF["k"], R=VMF["R"], L_build=VMF["L_build"], L_search=VMF["L"], L_dep=VMF["L"],
                  alpha=VMF["alpha"], build_passes=VMF["build_passes"], n_start=min(n, VMF["n_start"] * n // VMF["n"]),
                  center=pc.CENTER_PRODUCT, n_clusters=VMF["n_clusters"])
    ds32 = pc.Dataset(Xd, metric=pc.IP)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G, _ = pc.pecann_build_graph(ds32, p, order=torch.from_numpy(synth.insertion_order(n)).to(dev))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Gh = G.cpu().numpy()
    Xb = Xd.to(torch.bfloat16).contiguous()
    scale = (Xd.abs().amax(0) / 448.0).clamp_min(torch.finfo(torch.float32).tiny).contiguous()
    Xf8 = (Xd / scale).to(torch.float8_e4m3fn).contiguous()
    kinds = [("fp32", ds32, 4), ("bf16", pc.Dataset(Xb, metric=pc.IP, data_f32=Xd), 2),
             ("fp8-e4m3", pc.Dataset(Xf8, metric=pc.IP, dim_scale=scale, data_f32=Xd), 1)]
    out = []
    base_name = VMF_NAME if n == VMF["n"] else VMF_NAME.replace("1,280,000", f"{n:,}")
    if args.graph_line_only:
        path = Path(ds32, G, p, dev)
        el, dms = timed(path.step, 1, args.variant_steps, stream)
        return [{"metric": METRIC, "value": n / (el / args.variant_steps), "unit": UNIT, "dtype": "fp32",
                 "ms_per_step": el * 1000 / args.variant_steps, "density_ms": dms, "build_s": build_s}]
    rate_cpu, _ = cpu_knn_rate(X, 1, Gh, VMF["L"], VMF["k"], CPU_SAMPLE_GRAPH, threads)
    for tag, ds, s in kinds:
        path = Path(ds, G, p, dev)
        el, dms = timed(path.step, 1, args.variant_steps, stream)
        got = path.dens["knn_dist"].cpu().numpy()
        line = {"metric": METRIC, "value": n / (el / args.variant_steps), "unit": UNIT, "dtype": tag,
                "ms_per_step": el * 1000 / args.variant_steps, "steps": args.variant_steps, "warmup": 1,
                "config": {"workload": base_name, "index": f"Vamana graph R={VMF['R']} beam {VMF['L']} "
                                                          f"(build: {VMF['build_passes']} passes, beam {VMF['L_build']}, "
                                                          f"{p.n_start} start points)",
                           "traversal": tag + ("" if tag == "fp32" else " rows, exact FP32 re-rank")},
                "density_ms": dms, "build_s": build_s, "dep_rounds": int(path.stats[0]),
                "unfinished_after_round0": int(path.stats[1]), "brute_force_tail": int(path.stats[63]),
                "recall_full_n_vs_exact_index": full_recall(got, exact_dist),
                "ari_vs_exact_index": exact.ari(path.labels.cpu().numpy(), exact_labels),
                "below_recall_bar": True,
                "roofline": graph_roofline(X, 1, Gh, p, VMF["d"] * s, dms / 1e3, n,
                                           f"k_search ({tag} rows, k-NN + density pass)",
                                           traffic_tag=f"k_search_vmf1024_{tag}"),
                "cpu_baseline": {"value": rate_cpu, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": (f"oracle beam search (Algorithm 1, FP32) k-NN + kth density of "
                                            f"{CPU_SAMPLE_GRAPH} sampled points on the same graph")}}
        out.append(line)
        del path
        torch.cuda.empty_cache()
    return out


def u8_variants(args, dev, stream, threads):
    import torch

    from oracle import exact
    from paper_2312_03940_gb300 import pecann as pc
    from paper_2312_03940_gb300 import synth

    n = U8["n"] if not args.n else min(args.n, U8["n"])
    X, gt = u8_data(n)
    Xd = torch.from_numpy(X).to(dev)
    ds = pc.Dataset(Xd)
    if args.exact_line_only:
        pb = pc.params(k=U8["k"], center=pc.CENTER_PRODUCT, n_clusters=U8["n_clusters"], index=pc.INDEX_BRUTE_FORCE)
        path = Path(ds, None, pb, dev)
        el, dms = timed(path.step, 1, args.variant_steps, stream)
        return [{"metric": METRIC, "value": n / (el / args.variant_steps), "unit": UNIT, "dtype": "u8",
                 "ms_per_step": el * 1000 / args.variant_steps, "density_ms": dms, "index": "brute force"}]
    p = pc.params(k=U8["k"], R=U8["R"], L_build=U8["L_build"], L_search=U8["L"], L_dep=U8["L"], alpha=U8["alpha"],
                  n_start=min(n, U8["n_start"]), build_passes=U8["build_passes"], center=pc.CENTER_PRODUCT,
                  n_clusters=U8["n_clusters"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G, _ = pc.pecann_build_graph(ds, p, order=torch.from_numpy(synth.insertion_order(n)).to(dev))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Gh = G.cpu().numpy()
    name = U8_NAME if n == U8["n"] else U8_NAME.replace("1,000,000", f"{n:,}")
    out = []
    # graph path (beam 128)
    path = Path(ds, G, p, dev)
    steps = max(args.variant_steps, 5)
    el, dms = timed(path.step, 2, steps, stream)
    graph_dist = path.dens["knn_dist"].cpu().numpy()
    graph_labels = path.labels.cpu().numpy()
    if args.graph_line_only:
        return [{"metric": METRIC, "value": n / (el / steps), "unit": UNIT, "dtype": "u8",
                 "ms_per_step": el * 1000 / steps, "density_ms": dms, "build_s": build_s}]
    rate_cpu, _ = cpu_knn_rate(X, 0, Gh, U8["L"], U8["k"], CPU_SAMPLE_GRAPH * 4, threads)
    line = {"metric": METRIC, "value": n / (el / steps), "unit": UNIT, "dtype": "u8",
            "ms_per_step": el * 1000 / steps, "steps": steps, "warmup": 2,
            "config": {"workload": name, "index": f"Vamana graph R={U8['R']} beam {U8['L']} (build: 2 passes, "
                                                  f"beam {U8['L_build']}, {p.n_start} start points)"},
            "density_ms": dms, "build_s": build_s, "dep_rounds": int(path.stats[0]),
            "unfinished_after_round0": int(path.stats[1]), "brute_force_tail": int(path.stats[63]),
            "recall": exact_recall(X, 0, graph_dist, U8["k"], m=2000), "recall_queries": 2000,
            "roofline": graph_roofline(X, 0, Gh, p, U8["d"], dms / 1e3, n, "k_search (k-NN + density pass)",
                                       traffic_tag="k_search_density_c2"),
            "e2e": e2e_rate(path, X, G.cpu(), 3),
            "cpu_baseline": {"value": rate_cpu, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": (f"oracle beam search (Algorithm 1) k-NN + kth density of "
                                        f"{CPU_SAMPLE_GRAPH * 4} sampled points on the same graph")}}
    del path
    # NN-Descent graph on the same rows, searched with the same beam
    init = torch.from_numpy(synth.random_neighbours(n, NND["K"], repeats=NND["repeats"])).to(dev)
    pn = pc.params(R=U8["R"], alpha=NND["alpha"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nnd = pc.pecann_build_nndescent(ds, pn, NND["K"], init, NND["rounds"])
    torch.cuda.synchronize()
    nnd_build_s = time.perf_counter() - t0
    del init
    path = Path(ds, nnd["graph"], p, dev)
    el_n, dms_n = timed(path.step, 2, steps, stream)
    nnd_dist = path.dens["knn_dist"].cpu().numpy()
    nnd_labels = path.labels.cpu().numpy()
    nnd_line = {"metric": METRIC, "value": n / (el_n / steps), "unit": UNIT, "dtype": "u8",
                "ms_per_step": el_n * 1000 / steps, "steps": steps, "warmup": 2,
                "config": {"workload": name,
                           "index": (f"NN-Descent graph K={NND['K']}, {NND['repeats']} repeats, <= {NND['rounds']} "
                                     f"rounds, RobustPrune alpha {NND['alpha']} to R={U8['R']}; beam {U8['L']}")},
                "density_ms": dms_n, "build_s": nnd_build_s,
                "nndescent_changes_per_round": nnd["changes"].tolist(),
                "dep_rounds": int(path.stats[0]), "unfinished_after_round0": int(path.stats[1]),
                "brute_force_tail": int(path.stats[63]),
                "recall": exact_recall(X, 0, nnd_dist, U8["k"], m=2000), "recall_queries": 2000}
    del path, nnd
    torch.cuda.empty_cache()
    # HCNNG graph on the same rows, searched with the same beam
    ph = pc.params(R=U8["R"], alpha=HC["alpha"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hc = pc.pecann_build_hcnng(ds, ph, HC["repeats"], HC["leaf"], HC["mst_deg"])
    torch.cuda.synchronize()
    hc_build_s = time.perf_counter() - t0
    path = Path(ds, hc["graph"], p, dev)
    el_h, dms_h = timed(path.step, 2, steps, stream)
    hc_dist = path.dens["knn_dist"].cpu().numpy()
    hc_labels = path.labels.cpu().numpy()
    hc_line = {"metric": METRIC, "value": n / (el_h / steps), "unit": UNIT, "dtype": "u8",
               "ms_per_step": el_h * 1000 / steps, "steps": steps, "warmup": 2,
               "config": {"workload": name,
                          "index": (f"HCNNG graph, {HC['repeats']} repeats, leaves <= {HC['leaf']}, forest degree "
                                    f"<= {HC['mst_deg']}, RobustPrune alpha {HC['alpha']} to R={U8['R']}; "
                                    f"beam {U8['L']}")},
               "density_ms": dms_h, "build_s": hc_build_s, "hcnng_leaves": hc["leaves"].tolist(),
               "mean_degree": float(hc["degree"].float().mean().item()),
               "dep_rounds": int(path.stats[0]), "unfinished_after_round0": int(path.stats[1]),
               "brute_force_tail": int(path.stats[63]),
               "recall": exact_recall(X, 0, hc_dist, U8["k"], m=2000), "recall_queries": 2000}
    del path, hc
    torch.cuda.empty_cache()
    # exact index on the same rows
    pb = pc.params(k=U8["k"], R=U8["R"], L_search=U8["L"], L_dep=U8["L"], center=pc.CENTER_PRODUCT,
                   n_clusters=U8["n_clusters"], index=pc.INDEX_BRUTE_FORCE)
    path = Path(ds, None, pb, dev)
    el, dms = timed(path.step, 1, args.variant_steps, stream)
    knn_counts = path.screen_counts()
    ex_dist = path.dens["knn_dist"].cpu().numpy()
    line["recall_full_n_vs_exact_index"] = full_recall(graph_dist, ex_dist)
    line["ari_vs_exact_index"] = exact.ari(graph_labels, path.labels.cpu().numpy())
    out.append(line)
    nnd_line["recall_full_n_vs_exact_index"] = full_recall(nnd_dist, ex_dist)
    nnd_line["ari_vs_exact_index"] = exact.ari(nnd_labels, path.labels.cpu().numpy())
    out.append(nnd_line)
    hc_line["recall_full_n_vs_exact_index"] = full_recall(hc_dist, ex_dist)
    hc_line["ari_vs_exact_index"] = exact.ari(hc_labels, path.labels.cpu().numpy())
    out.append(hc_line)
    rate_cpu_bf, _ = cpu_knn_rate(X, 0, None, 0, U8["k"], CPU_SAMPLE * 4, threads)
    out.append({"metric": METRIC, "value": n / (el / args.variant_steps), "unit": UNIT, "dtype": "u8",
                "ms_per_step": el * 1000 / args.variant_steps, "steps": args.variant_steps, "warmup": 1,
                "config": {"workload": name, "index": "brute force (exact; BF16 tcgen05 screen, exact integer decision)"},
                "density_ms": dms, "recall": 1.0, "ari_vs_generator": exact.ari(path.labels.cpu().numpy(), gt),
                "roofline": screen_roofline(n, U8["d"], knn_counts[0], dms / 1e3, traffic_tag="k_bf_screen_u8"),
                "cpu_baseline": {"value": rate_cpu_bf, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": f"oracle brute-force index k-NN + kth density of {CPU_SAMPLE * 4} sampled "
                                           f"points over all {n:,} rows"}})
    return out


def run_vmf_graph_only(args):
    """The 1.28M x 1024 rows on the Vamana graph alone (report lines), recall
    judged against the exact index run once, untimed."""
    import torch

    from paper_2312_03940_gb300 import build as pbuild
    from paper_2312_03940_gb300 import pecann as pc

    pbuild.build()
    pc.load_library()
    import oracle

    oracle.build()
    dev = torch.device("cuda", 0)
    n = args.n or VMF["n"]
    X, _ = vmf_data(n)
    Xd = torch.from_numpy(X).to(dev)
    p = pc.params(k=VMF["k"], L_search=VMF["L"], center=pc.CENTER_PRODUCT, n_clusters=VMF["n_clusters"],
                  index=pc.INDEX_BRUTE_FORCE)
    ex_dist = ex_labels = None
    if not args.graph_line_only:
        ref = Path(pc.Dataset(Xd, metric=pc.IP), None, p, dev)
        ref.step(None)
        ex_dist, ex_labels = ref.dens["knn_dist"].cpu().numpy(), ref.labels.cpu().numpy()
        del ref
        torch.cuda.empty_cache()
    out = vmf_graph_variants(args, X, Xd, ex_dist, ex_labels, dev, torch.cuda.current_stream(),
                             oracle.default_threads())
    print(json.dumps({"workload": "vmf1024-graph", "lines": out}), flush=True)


def run_u8_only(args):
    """The uint8 workload alone on its graph and on the exact index (report)."""
    import torch

    from paper_2312_03940_gb300 import build as pbuild
    from paper_2312_03940_gb300 import pecann as pc

    pbuild.build()
    pc.load_library()
    import oracle

    oracle.build()
    out = u8_variants(args, torch.device("cuda", 0), torch.cuda.current_stream(), oracle.default_threads())
    print(json.dumps({"workload": "u8-1m", "lines": out}), flush=True)


# ---------------------------------------------------------------- extra report workloads

def _timed_steps(step, warmup, steps):
    import torch

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / steps


def run_batched64(args):
    """64 independent FP32 Gaussian mixtures (n log-uniform in [2,000, 200,000],
    d in {96, 128, 256, 384}, 5-500 components), R=32, L=96, k=8: one batched
    pass (captured in a CUDA graph, knobs autotuned) vs the same sets run one
    after another through the single-set calls."""
    import torch

    from oracle import exact
    from paper_2312_03940_gb300 import autotune
    from paper_2312_03940_gb300 import pecann as pc
    from paper_2312_03940_gb300 import synth

    pc.load_library()
    sets = synth.batched_sets()
    comps = [c for _, _, c in sets]
    p = pc.params(k=8, R=32, L_build=192, L_search=96, L_dep=96, alpha=1.2, build_passes=2, n_clusters=10)
    dss, graphs = [], []
    t0 = time.perf_counter()
    for i, (X, _, _) in enumerate(sets):
        ds = pc.Dataset(torch.from_numpy(X).cuda())
        p.n_start = max(16, min(len(X), 8192 * len(X) // 1_000_000))
        G, _ = pc.pecann_build_graph(ds, p, order=torch.from_numpy(synth.insertion_order(len(X), seed=i)).cuda())
        dss.append(ds)
        graphs.append(G)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    batch = pc.Batch(dss, graphs, p, n_clusters=comps)
    tune = autotune.tune_batch(batch, use_cache=False)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch.run(stream=s)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch.run(stream=s)
    t_graph = _timed_steps(graph.replay, args.warmup, args.steps)
    t_plain = _timed_steps(batch.run, args.warmup, args.steps)
    # the same sets one after another through the single-set calls
    singles = []
    for i, (ds, G) in enumerate(zip(dss, graphs)):
        pi = pc.params(k=8, R=32, L_search=96, L_dep=96, n_clusters=comps[i], hash_slots=p.hash_slots,
                       block_warps=p.block_warps)
        ws = pc.workspace(ds, pi)
        singles.append((ds, G, pi, ws))

    def seq():
        for ds, G, pi, ws in singles:
            d = pc.pecann_density(ds, G, pi, ws=ws)
            dp = pc.pecann_dependent_points(ds, G, pi, d["rank_key"], d["knn_ids"], d["knn_dist"], ws=ws)
            pc.pecann_cluster(d["density"], dp["dep"], dp["dep_dist"], pi, count=False)

    t_seq = _timed_steps(seq, 1, max(1, args.steps // 4))
    # recall on 32 sampled points per set
    got = batch.out["knn_dist"].cpu().numpy()
    rec = []
    for i, (X, _, _) in enumerate(sets):
        qs = synth.sample_ids(len(X), 32, seed=i)
        _, ex = exact.exact_knn_queries(X, qs, 8)
        rec.append(exact.knn_recall(got[batch.offsets[i] + qs], ex))
    N = batch.N
    out = {"metric": METRIC, "value": N / t_graph, "unit": UNIT, "workload": "batched64",
           "config": {"workload": "64 FP32 Gaussian mixtures, n log-uniform [2000, 200000], d in {96,128,256,384}, "
                                  "5-500 components; R=32 L=96 k=8; build 2 passes L=192", "points": N},
           "ms_per_step_graph": t_graph * 1e3, "ms_per_step_batched_no_graph": t_plain * 1e3,
           "ms_per_step_sets_one_by_one": t_seq * 1e3, "points_per_s_one_by_one": N / t_seq,
           "autotune": {k2: v for k2, v in tune.items() if k2 != "tried"}, "autotune_tried": tune.get("tried"),
           "recall": float(np.mean(rec)), "build_s": build_s}
    print(json.dumps(out), flush=True)


def run_reduced(args, kind):
    """The 1M x 384 power-law sphere (L2): FP32 vs BF16 traversal with exact
    FP32 re-rank on the same graph, kth and exp-sum densities."""
    import torch

    from oracle import exact
    from paper_2312_03940_gb300 import pecann as pc
    from paper_2312_03940_gb300 import synth

    pc.load_library()
    n = args.n or 1_000_000
    X, gt = synth.powerlaw_sphere(n=n)
    metric, R, L, k, alpha, ncl = pc.L2, 48, 128, 20, 1.1, 10_000
    dens_fns = [("kth", pc.DENS_KTH), ("exp-sum", pc.DENS_EXPSUM)]
    desc = f"unit-norm power-law-spectrum sphere n={n} d=384, 10,000 Pareto(1.5) clusters; R=48 L=128 alpha=1.1 k=20"
    Xd = torch.from_numpy(X).cuda()
    del X
    Xb = Xd.to(torch.bfloat16).contiguous()
    ds32 = pc.Dataset(Xd, metric=metric)
    dsb = pc.Dataset(Xb, metric=metric, data_f32=Xd)
    variants = [("fp32", ds32), ("bf16", dsb)]
    if metric == pc.IP:
        # s_j = max_i |x_ij| / 448 (the largest e4m3 value); codes of x / s
        scale = (Xd.abs().amax(0) / 448.0).clamp_min(torch.finfo(torch.float32).tiny).contiguous()
        variants.append(("fp8", pc.Dataset((Xd / scale).to(torch.float8_e4m3fn).contiguous(), metric=metric,
                                           dim_scale=scale, data_f32=Xd)))
    p = pc.params(k=k, R=R, L_build=2 * L, L_search=L, L_dep=L, alpha=alpha, build_passes=2,
                  n_start=max(16, min(n, 8192 * n // 1_000_000)), n_clusters=ncl)
    t0 = time.perf_counter()
    G, _ = pc.pecann_build_graph(ds32, p, order=torch.from_numpy(synth.insertion_order(n)).cuda())
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Xh = Xd.cpu().numpy()
    qs = synth.sample_ids(n, 1000)
    _, ex = exact.exact_knn_queries(Xh, qs, k, metric=metric)
    res = {}
    for name, fn in dens_fns:
        p.density = fn
        for tag, ds in variants:
            ws = pc.workspace(ds, p)
            out = {}

            def step():
                d = pc.pecann_density(ds, G, p, ws=ws)
                dp = pc.pecann_dependent_points(ds, G, p, d["rank_key"], d["knn_ids"], d["knn_dist"], ws=ws)
                lab, _ = pc.pecann_cluster(d["density"], dp["dep"], dp["dep_dist"], p, count=False)
                out.update(d, labels=lab)

            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t = _timed_steps(step, args.warmup, args.steps)
            e0.record()
            pc.pecann_density(ds, G, p, ws=ws)
            e1.record()
            torch.cuda.synchronize()
            res[f"{name}/{tag}"] = {"points_per_s": n / t, "ms_per_step": t * 1e3,
                                    "density_ms": e0.elapsed_time(e1),
                                    "recall": exact.knn_recall(out["knn_dist"][torch.from_numpy(qs).cuda()].cpu().numpy(),
                                                               ex),
                                    "labels": out["labels"].cpu().numpy()}
        for tag, _ in variants[1:]:
            res[f"{name}/{tag}"]["ari_vs_fp32"] = exact.ari(res[f"{name}/{tag}"]["labels"],
                                                             res[f"{name}/fp32"]["labels"])
    for v in res.values():
        v.pop("labels")
    print(json.dumps({"workload": kind, "config": {"workload": desc, "build_s": build_s}, "results": res}),
          flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched64(args)
    elif args.workload == "sphere384":
        run_reduced(args, "sphere384")
    elif args.workload == "u8-1m":
        run_u8_only(args)
    elif args.workload == "vmf1024-graph":
        run_vmf_graph_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
