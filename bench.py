#!/usr/bin/env python3
"""DPC points/sec on one GB300: density + dependent points (+ clusters).

Workload: n = 1,000,000 x d = 128 uint8 Gaussian mixture (100 components,
Zipf(1.1) weights, per-component sigma in [5, 20], 5% uniform noise points),
Vamana R = 64, L = 128, alpha = 1.2, k = 10, product center with 100
clusters. A step is one pass of the path over the whole point set on the
graph the GPU built beforehand: k-NN + density, dependent points (round 0,
doubling rounds, brute-force tail) and the cluster cut. The graph build is
timed separately and reported as build_s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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

# The k-NN / dependent searches use beam L = 128. The build (outside the
# metric) uses two passes, beam 256 and 8192 random start points: the paper
# leaves these open, and they give >= 0.95 k-NN recall on this data.
WORKLOAD = dict(n=1_000_000, d=128, components=100, R=64, L=128, alpha=1.2, k=10, n_clusters=100,
                L_build=256, n_start=8192, build_passes=2)
WORKLOAD_NAME = ("u8-gaussian-mixture n=1,000,000 d=128 (100 components, Zipf 1.1 weights, sigma U[5,20], "
                 "5% uniform noise); Vamana R=64 L=128 alpha=1.2 (build: 2 passes, L=256, 8192 start points); "
                 "kth density k=10; product center 100")
METRIC = "DPC points/sec (density + dependent-point search) at >=0.95 recall; % HBM peak"
UNIT = "points/s"
SUBSET_N = 10_000  # oracle sample: the same generator at 10k points


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=WORKLOAD["n"], help="points (profiling runs use fewer)")
    ap.add_argument("--quick", action="store_true", help="skip recall, e2e and the CPU baseline")
    ap.add_argument("--subset", type=int, default=SUBSET_N)
    ap.add_argument("--workload", default="u8-1m", choices=["u8-1m", "batched64", "sphere384", "vmf1024"],
                    help="u8-1m: the benchmark line; the others print extra report lines")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


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


def source_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2312_03940_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
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
    if vals.get("source_sha") != source_sha():
        return None
    try:
        return float(vals["traffic_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def oracle_subset_run(n_sub: int, threads: int, steps: int = 1, warmup: int = 0):
    """The CPU oracle's whole path (k-NN + density, dependent points, clusters)
    on an n_sub-point sample drawn from the same generator, on a graph the
    oracle builds itself (untimed). Returns points/s over the timed steps."""
    import oracle
    from paper_2312_03940_gb300 import synth

    X, _ = synth.u8_mixture(n=n_sub, d=WORKLOAD["d"], components=WORKLOAD["components"])
    P = oracle.Points(X)
    # start points in the same proportion to n as on the full workload
    n_start = max(16, WORKLOAD["n_start"] * n_sub // WORKLOAD["n"])
    G = oracle.build_graph(P, R=WORKLOAD["R"], L=WORKLOAD["L_build"], alpha=WORKLOAD["alpha"],
                           perm=synth.insertion_order(n_sub), n_start=n_start, threads=threads,
                           passes=WORKLOAD["build_passes"])

    def one():
        r = oracle.knn_density(P, G, L=WORKLOAD["L"], k=WORKLOAD["k"], threads=threads)
        d = oracle.dependent_points(P, G, r["key"], r["ids"], Ld=WORKLOAD["L"], threshold=300, threads=threads)
        oracle.cluster(r["rho"], d["lam"], d["delta"], center=oracle.CENTER_PRODUCT,
                       n_clusters=WORKLOAD["n_clusters"])

    for _ in range(warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    dt = time.perf_counter() - t0
    return n_sub * steps / dt, dt


# ---------------------------------------------------------------- reference arm (the CPU oracle)

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    threads = oracle.default_threads()
    n_sub = args.subset
    rate, dt = oracle_subset_run(n_sub, threads, steps=args.steps, warmup=args.warmup)
    sample = (f"oracle k-NN+density, dependent points and clusters on a {n_sub}-point sample of the same "
              f"generator (its own graph, built untimed), {args.steps} steps")
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1000 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "oracle_sample_points": n_sub},
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

    def barrier():
        if dist:
            dist.barrier()

    n = args.n
    X, gt = synth.u8_mixture(n=n, d=WORKLOAD["d"], components=WORKLOAD["components"])
    order = synth.insertion_order(n)
    p = pc.params(k=WORKLOAD["k"], R=WORKLOAD["R"], L_build=WORKLOAD["L_build"], L_search=WORKLOAD["L"],
                  L_dep=WORKLOAD["L"], alpha=WORKLOAD["alpha"], n_start=min(n, WORKLOAD["n_start"]),
                  build_passes=WORKLOAD["build_passes"], center=pc.CENTER_PRODUCT,
                  n_clusters=WORKLOAD["n_clusters"])
    Xd = torch.from_numpy(X).to(dev)
    ds = pc.Dataset(Xd)
    ws = pc.workspace(ds, p)
    stream = torch.cuda.current_stream()

    # ---- graph build (not part of the metric)
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    G, _ = pc.pecann_build_graph(ds, p, order=torch.from_numpy(order).to(dev), ws=ws)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - tb0

    dens_out = dict(knn_ids=torch.empty((n, p.k), dtype=torch.int32, device=dev),
                    knn_dist=torch.empty((n, p.k), dtype=torch.float32, device=dev),
                    density=torch.empty(n, dtype=torch.float32, device=dev),
                    rank_key=torch.empty(n, dtype=torch.float32, device=dev))
    dep_out = dict(dep=torch.empty(n, dtype=torch.int32, device=dev),
                   dep_dist=torch.empty(n, dtype=torch.float32, device=dev))
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    cws = torch.empty(8 * n + (1 << 20), dtype=torch.uint8, device=dev)
    def step():
        pc.pecann_density(ds, G, p, ws=ws, out=dens_out)
        pc.pecann_dependent_points(ds, G, p, dens_out["rank_key"], dens_out["knn_ids"], dens_out["knn_dist"],
                                   ws=ws, out=dep_out)
        pc.pecann_cluster(dens_out["density"], dep_out["dep"], dep_out["dep_dist"], p, ws=cws, count=False,
                          labels=labels)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    timed_density = []
    barrier()
    torch.cuda.synchronize()
    l0 = pc.pecann_kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("pecann_step")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pc.pecann_density(ds, G, p, ws=ws, out=dens_out)
        e1.record(stream)
        pc.pecann_dependent_points(ds, G, p, dens_out["rank_key"], dens_out["knn_ids"], dens_out["knn_dist"],
                                   ws=ws, out=dep_out)
        pc.pecann_cluster(dens_out["density"], dep_out["dep"], dep_out["dep_dist"], p, ws=cws, count=False,
                          labels=labels)
        timed_density.append((e0, e1))
        torch.cuda.nvtx.range_pop()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = pc.pecann_kernel_launches() - l0
    clk = clocks.stop()
    elapsed = max_over_ranks(t0.elapsed_time(t1) / 1000.0, dist, dev)
    dens_avg_s = float(np.mean([a.elapsed_time(b) for a, b in timed_density])) / 1000.0
    value = replica_throughput(n, args.steps, world, elapsed)
    stats = pc.pecann_dependent_points(ds, G, p, dens_out["rank_key"], dens_out["knn_ids"], dens_out["knn_dist"],
                                       ws=ws, out=dep_out)["stats"]
    torch.cuda.synchronize()

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": elapsed * 1000 / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
              "config": {"workload": WORKLOAD_NAME if n == WORKLOAD["n"] else WORKLOAD_NAME.replace(
                  "1,000,000", f"{n:,}"), "n": n, "d": WORKLOAD["d"], "R": p.R, "L": p.L_search, "k": p.k,
                  "alpha": WORKLOAD["alpha"], "dep_threshold": p.dep_threshold, "L_build": p.L_build,
                  "n_start": p.n_start, "build_passes": p.build_passes,
                  "parallelism": "replicas" if world > 1 else "single-gpu",
                  "l2": "inputs (128 MB rows + 256 MB graph) exceed the 129 MB L2; no flush between steps"},
              "gpu_launches": int(launches), "clocks": clk, "build_s": build_s,
              "dep_rounds": int(stats[0]), "unfinished_after_round0": int(stats[1]),
              "brute_force_tail": int(stats[63]), "density_ms": dens_avg_s * 1000}

    if rank == 0 and not args.quick:
        import oracle
        from oracle import exact

        oracle.build()
        # ---- sampled exact k-NN recall (FP64 brute force on 2000 queries)
        qs = synth.sample_ids(n, 2000)
        _, ex_d = exact.exact_knn_queries(X, qs, p.k)
        got = dens_out["knn_dist"][torch.from_numpy(qs).to(dev)].cpu().numpy()
        result["recall"] = exact.knn_recall(got, ex_d)
        result["ari_vs_generator"] = exact.ari(labels.cpu().numpy(), gt)
        # ---- roofline of the dominant kernel (the k-NN beam search of the density pass)
        Gh = G.cpu().numpy()
        P = oracle.Points(X)
        e_q, c_q = oracle.search_counts(P, Gh, synth.sample_ids(n, 2000, seed=99), L=p.L_search)
        row = WORKLOAD["d"] * 1
        bytes_q = e_q.mean() * 4 * p.R + (c_q.mean() + 1) * row + 8 * p.k + 8
        alg_bytes = bytes_q * n
        pk, src = peaks()
        achieved = alg_bytes / dens_avg_s / 1e9
        result["roofline"] = {"kernel": "k_search (k-NN + density pass)", "bound": "hbm", "achieved": achieved,
                              "peak": pk["hbm_gbs"], "peak_source": src, "unit": "GB/s",
                              "frac": achieved / pk["hbm_gbs"], "traffic": profiled_traffic("k_search_density_c2"),
                              "algorithmic_bytes_per_launch": alg_bytes, "E_q": float(e_q.mean()),
                              "C_q": float(c_q.mean())}
        # ---- end to end through the public API from pinned host buffers
        Xh = torch.from_numpy(X).pin_memory()
        Gh_t = G.cpu().pin_memory()
        rho_h = torch.empty(n, dtype=torch.float32).pin_memory()
        dep_h = torch.empty(n, dtype=torch.int32).pin_memory()
        dd_h = torch.empty(n, dtype=torch.float32).pin_memory()
        lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
        Xd2 = torch.empty_like(Xd)
        Gd2 = torch.empty_like(G)
        ds2 = pc.Dataset(Xd2)
        k_e2e = max(3, min(args.steps, 5))
        torch.cuda.synchronize()
        s0 = time.perf_counter()
        for _ in range(k_e2e):
            Xd2.copy_(Xh, non_blocking=True)
            Gd2.copy_(Gh_t, non_blocking=True)
            pc.pecann_density(ds2, Gd2, p, ws=ws, out=dens_out)
            pc.pecann_dependent_points(ds2, Gd2, p, dens_out["rank_key"], dens_out["knn_ids"],
                                       dens_out["knn_dist"], ws=ws, out=dep_out)
            pc.pecann_cluster(dens_out["density"], dep_out["dep"], dep_out["dep_dist"], p, ws=cws, count=False,
                              labels=labels)
            rho_h.copy_(dens_out["density"], non_blocking=True)
            dep_h.copy_(dep_out["dep"], non_blocking=True)
            dd_h.copy_(dep_out["dep_dist"], non_blocking=True)
            lab_h.copy_(labels, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - s0) / k_e2e
        result["e2e"] = {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes + Gh.nbytes),
                         "d2h_bytes_per_step": int(16 * n)}
        # ---- CPU baseline: the oracle as it stands on a bounded sample
        threads = oracle.default_threads()
        rate, _ = oracle_subset_run(args.subset, threads)
        result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                  "sample": (f"oracle k-NN+density, dependent points and clusters on a "
                                             f"{args.subset}-point sample of the same generator, on its own "
                                             f"graph (built untimed); one step")}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


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
    """FP32 traversal vs BF16 (and, for inner product, FP8 e4m3 with per-dimension
    scales) traversal with exact FP32 re-rank, on the same graph."""
    import torch

    from oracle import exact
    from paper_2312_03940_gb300 import pecann as pc
    from paper_2312_03940_gb300 import synth

    pc.load_library()
    if kind == "sphere384":
        n = args.n if args.n != WORKLOAD["n"] else 1_000_000
        X, gt = synth.powerlaw_sphere(n=n)
        metric, R, L, k, alpha, ncl = pc.L2, 48, 128, 20, 1.1, 10_000
        dens_fns = [("kth", pc.DENS_KTH), ("exp-sum", pc.DENS_EXPSUM)]
        desc = f"unit-norm power-law-spectrum sphere n={n} d=384, 10,000 Pareto(1.5) clusters; R=48 L=128 alpha=1.1 k=20"
    else:
        n = args.n if args.n != WORKLOAD["n"] else 1_280_000
        X, gt = synth.vmf_like(n=n)
        metric, R, L, k, alpha, ncl = pc.IP, 64, 200, 16, 1.2, 1000
        dens_fns = [("kth", pc.DENS_KTH)]
        desc = f"unit-norm vMF-like n={n} d=1024 inner product, 1,000 clusters; R=64 L=200 k=16"
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
    elif args.workload in ("sphere384", "vmf1024"):
        run_reduced(args, args.workload)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
