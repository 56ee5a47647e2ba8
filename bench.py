#!/usr/bin/env python
"""Benchmark of the GB300 connectivity path.

Headline (one JSON line on stdout): static connectivity throughput in
Gedges/s (directed CSR entries m per second) on an R-MAT graph of scale 26,
edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), symmetrised, uint64
offsets and uint32 edges, with the default k-out (k=2) + UF-Rem-CAS
combination; its fraction of the HBM roofline (CSR bytes read once over the
measured copy bandwidth); the dominant kernel's roofline; the end-to-end rate
through the host-buffer entry point; the oracle's rate on a bounded sample of
the same graph on the host cores; and the incremental rates (updates/s and
p50/p99 batch latency) on an R-MAT scale-24 base graph.

A step is one cc_static call over the resident graph.  Inputs (7.7 GB CSR,
268 MB labels) exceed the 126 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank labels its own replica of the graph (the
path has no exchange step at one graph per GPU): weak scaling, no collective
on the data path; rank 0 prints the line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "static CC Gedges/s & % HBM peak at RMAT-26; incremental updates/s & p99"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scale", type=int, default=26)
    p.add_argument("--edge-factor", type=int, default=16)
    p.add_argument("--sample", default="kout")
    p.add_argument("--finish", default="uf_rem_cas")
    p.add_argument("--find", default="naive")
    p.add_argument("--splice", default="split_one")
    p.add_argument("--freq-samples", type=int, default=0)
    p.add_argument("--incr-scale", type=int, default=24)
    p.add_argument("--incr-finish", default="uf_rem_cas",
                   help="finish of the incremental handle: a union-find kind (batches of unions) or sv / lt_prf "
                        "(type-2 batches: rounds on the resident forest)")
    p.add_argument("--incr-batches", type=int, default=1000)
    p.add_argument("--incr-qfrac", default="0.1,0.5,0.9",
                   help="comma-separated query fractions of the served workload (one run each)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forest", action="store_true")
    p.add_argument("--no-amsf", action="store_true")
    p.add_argument("--amsf-eps", type=float, default=0.25)
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--configs", default="1,2a,2b,2c,3,4,5",
                   help="which workloads to measure besides the headline: 1 (R-MAT 16, u32 offsets, no sampling "
                        "+ UF-Rem-CAS), 2a (every sampling x finish combination on the headline graph), 2b (16384^2 "
                        "grid, edge drop 0.3), 2c (Erdos-Renyi 2^25, degree 1.2), 3 (10,000 packed graphs), 4 (the "
                        "learned selector), 5 (the served incremental workload); 'none' for the headline only")
    p.add_argument("--minlabel", action="store_true",
                   help="also time the sixteen Liu-Tarjan variants, Stergiou and label propagation (none / k-out)")
    p.add_argument("--batched-graphs", type=int, default=10000)
    p.add_argument("--batched-schedule", default="",
                   help="threads,smem_max_vertices,mode: time this schedule instead of autotuning")
    p.add_argument("--sel-train", type=int, default=2000)
    p.add_argument("--sel-test", type=int, default=200)
    p.add_argument("--sel-scale-lo", type=int, default=14)
    p.add_argument("--sel-scale-hi", type=int, default=22)
    p.add_argument("--cpu-seconds", type=float, default=20.0)
    return p.parse_args()


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (timing is reported for the whole job)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def kernel_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu capture
    (profiles/traffic.json), or None when the kernels' sources (the files
    it lists, hashed together) have changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f)
        ent = tj["kernels"].get(kernel)
        h = hashlib.sha256()
        for src in tj["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if ent is None or h.hexdigest() != tj["sources_sha256"]:
            return None
        return int(ent["bytes_per_launch"])
    except Exception:
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return None
        rows = []
        try:
            with open(self.file.name) as f:
                for ln in f:
                    parts = [x.strip() for x in ln.split(",")]
                    if len(parts) >= 8:
                        rows.append(parts)
            os.unlink(self.file.name)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- workloads
def make_graph(scale, ef, device):
    import synth
    return synth.rmat(scale, ef, seed=1, device=device)


SECTOR = 32   # bytes: the DRAM access granule of a random 4-byte read


def algorithmic_bytes(kernel, n, m, m_finish, n_nz, k, off_bytes):
    """Compulsory bytes of one launch of `kernel`.  Streams (offsets, labels,
    edge ranges) count at word granularity: offsets `off_bytes` per vertex,
    edges, parent and label words 4 B.  A random read into the edge array
    (8.4 GB, no reuse) counts as the 32-byte sector it must bring in (the
    per-vertex figure of the sampled variants: about k sectors per vertex
    for k picked edges); random parent reads count 4 B, as the parent array
    is hot in L2.  n_nz: vertices with at least one edge; m_finish: edges
    out of vertices whose sampled label is not L_max."""
    ob = off_bytes
    table = {
        "k_iota": 4 * n,                                            # write P
        # offsets; the first edge and (k = 2) the random pick of each
        # non-isolated vertex, one random sector each; write P and the
        # stashed pick
        "k_kout_hook_first": ob * (n + 1) + min(k, 2) * SECTOR * n_nz + 8 * n,
        # stashed pick and own parent (streams), the picked vertex's parent
        "k_kout_apply_pick": 8 * n + 4 * n_nz,
        # offsets, own parent, (k-1) picked edges (random sectors) and their
        # parents
        "k_kout_rest": ob * (n + 1) + n_nz * (k - 1) * (SECTOR + 4) + 4 * n,
        "k_compress_mid": 8 * n,                                    # read + write P
        "k_compress_count": 8 * n + n // 8,                         # read + write P, the degree bitmap
        "k_compress": 8 * n,
        "k_final_shortcut": 8 * n,
        "k_count_labels": 4 * n,
        "k_argmax_counts": 4 * n,
        "k_cand_bin": 4 * n + ob * (n + 1),                         # labels + offsets
        "k_light_list": 4 * m_finish * 2,                           # edges + parent of each neighbour
        "k_chunks": 4 * m_finish * 2,
        # offsets, own parent, every edge, parent of each lower neighbour
        "k_range_bin": ob * (n + 1) + 4 * n + 4 * m + 4 * (m // 2),
    }
    return table.get(kernel)


def run_ours(args):
    import torch
    import paper_2008_03909_gb300 as cc
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    t0 = time.time()
    g = make_graph(args.scale, args.edge_factor, dev)
    n, m = g.n, g.m
    gen_s = time.time() - t0
    deg = g.offsets[1:] - g.offsets[:-1]
    n_nz = int((deg > 0).sum().item())
    del deg
    torch.cuda.empty_cache()
    off, edg = g.offsets, g.edges
    so = cc.sample_opt(args.sample, k=2, bfs_tries=3, ldd_beta=0.2, seed=1, freq_samples=args.freq_samples)
    fo = cc.finish_opt(args.finish, args.find, args.splice)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    # one checked run: stats + invariants that hold at any size
    lab, st = cc.cc_static(off, edg, so, fo, labels, stats=True)
    ok, ncomp = check_labels(off, edg, lab)
    torch.cuda.empty_cache()

    for _ in range(args.warmup):
        cc.cc_static(off, edg, so, fo, labels)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = cc.launch_count()
    cc.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            cc.cc_static(off, edg, so, fo, labels)
        e1.record(stream)
        torch.cuda.synchronize()
    prof = cc.profile_read()
    cc.profile_enable(False)
    launches = cc.launch_count() - launches0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    if dist:
        dist.barrier()
    value = job_rate(m, world, ms) / 1e9
    peak, peak_kind = peaks()
    off_bytes = 8 if off.dtype == torch.int64 else 4
    b_csr = off_bytes * (n + 1) + 4 * m
    hbm_frac = (b_csr / (peak * 1e9)) / (ms * 1e-3)

    # dominant kernel roofline (per-launch averages from the timed region)
    kernels = {k: {"launches": v[0], "ms_total": round(v[1], 4), "ms_avg": v[1] / max(v[0], 1),
                   "share": v[1] / max(sum(x[1] for x in prof.values()), 1e-9)} for k, v in prof.items()}
    dom = max(kernels, key=lambda k: kernels[k]["ms_total"]) if kernels else None
    roof = None
    if dom:
        ab = algorithmic_bytes(dom, n, m, st["edges_finish"], n_nz, 2, off_bytes)
        if ab is not None:
            per_launch_ms = kernels[dom]["ms_avg"]
            ach = ab / (per_launch_ms * 1e-3) / 1e9
            roof = {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(ach / peak, 4), "traffic": kernel_traffic(dom), "peak_kind": peak_kind,
                    "algorithmic_bytes": ab, "ms_avg": round(per_launch_ms, 5)}

    # MapEdges / GatherEdges (Table 8): this GPU's floors for reading the
    # graph and for one indirect read per edge
    probes = {}
    xs = torch.arange(n, dtype=torch.int32, device=dev)
    pout = torch.empty(n, dtype=torch.int32, device=dev)
    for name, fn in (("map_edges", lambda: cc.cc_map_edges(off, edg, pout)),
                     ("gather_edges", lambda: cc.cc_gather_edges(off, edg, xs, pout))):
        fn()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record()
        for _ in range(3):
            fn()
        p1.record()
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1) / 3
        probes[name] = {"ms": round(pms, 4), "gedges_s": round(m / (pms * 1e-3) / 1e9, 2),
                        "csr_gbs": round((off_bytes * (n + 1) + 4 * m) / (pms * 1e-3) / 1e9, 1)}
    del xs, pout
    # random-sector reads of the edge array (larger than L2), one per k-out
    # pick: the rate the sampling kernel's random edge reads can reach
    rs = 2 * n_nz
    cc.cc_random_sectors(edg, rs, seed=3)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for _ in range(3):
        cc.cc_random_sectors(edg, rs, seed=3)
    p1.record()
    torch.cuda.synchronize()
    pms = p0.elapsed_time(p1) / 3
    probes["random_sectors"] = {"ms": round(pms, 4), "reads": rs, "sector_gbs": round(32 * rs / (pms * 1e-3) / 1e9, 1)}
    if roof is not None:
        roof["random_sector_gbs"] = probes["random_sectors"]["sector_gbs"]

    # spanning forest with the same sampling and finish (the edges that
    # hooked roots are recorded as they are linked)
    forest = None
    if not args.no_forest:
        fbuf = torch.empty(2 * n, dtype=torch.int32, device=dev)
        pairs, _ = cc.cc_spanning_forest(off, edg, so, fo, forest_out=fbuf)
        fcount = pairs.shape[0]
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(3):
            cc.cc_spanning_forest(off, edg, so, fo, forest_out=fbuf)
        f1.record()
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / 3
        forest = {"ms": round(fms, 4), "gedges_s": round(m / (fms * 1e-3) / 1e9, 2), "edges": fcount,
                  "size_ok": fcount == n - ncomp, "overhead_vs_cc": round(fms / ms - 1.0, 4),
                  "note": "synchronous call (returns the count), timed on the host thread's stream"}
        del fbuf, pairs

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gedges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale}_ef{args.edge_factor}", "n": n, "m": m,
                   "rmat": [0.57, 0.19, 0.19, 0.05], "seed": 1, "offsets": "u64" if off_bytes == 8 else "u32",
                   "sample": args.sample, "finish": f"{args.finish}+{args.find}+{args.splice}",
                   "freq_samples": args.freq_samples, "l2": "inputs exceed L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "hbm_roof_frac": round(hbm_frac, 4), "hbm_roof_peak_gbs": peak,
        "roofline": roof, "kernels": kernels, "gpu_launches": launches, "edge_primitives": probes,
        "spanning_forest": forest,
        "check": {"invariants_ok": ok, "components": ncomp, "lmax": st["lmax"], "edges_finish": st["edges_finish"],
                  "n_nonisolated": n_nz},
        "gen_s": round(gen_s, 2),
    }
    clocks = clk.summary()
    out["clocks"] = clocks

    # end to end through the host-buffer entry point (pinned host CSR)
    if not args.no_e2e:
        h_off = off.cpu().pin_memory()
        h_edg = edg.cpu().pin_memory()
        h_lab = torch.empty(n, dtype=torch.int32).pin_memory()
        cc.cc_static_host(h_off, h_edg, so, fo, h_lab)
        k2 = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t1 = time.perf_counter()
        for _ in range(k2):
            cc.cc_static_host(h_off, h_edg, so, fo, h_lab)
        e2e_s = max_over_ranks((time.perf_counter() - t1) / k2, dist, dev)
        same = bool(torch.equal(h_lab, lab.cpu()))
        out["e2e"] = {"value": round(world * m / e2e_s / 1e9, 3), "unit": "Gedges/s",
                      "h2d_bytes_per_step": b_csr, "d2h_bytes_per_step": 4 * n, "ms_per_step": round(e2e_s * 1e3, 3),
                      "labels_equal_device_path": same,
                      "h2d": ("k-out reads the pinned CSR in place (offsets and about two 32-byte sectors per vertex "
                              "cross the host link); h2d_bytes_per_step counts the whole host-resident input"
                              if args.sample == "kout" else "the CSR is copied to the device each call")}
        del h_off, h_edg, h_lab

    # the oracle on the host cores, on the headline graph (rank 0, one GPU)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(off, edg, args.cpu_seconds)

    # the other workloads, one GPU each: measured by a single-rank run only
    # (under torchrun every rank holds its GPU for the headline alone)
    want = set() if args.configs.strip() in ("", "none") or world > 1 else \
        {c.strip() for c in args.configs.split(",")}
    configs = {}
    if "1" in want:
        configs["1_rmat16_ef8_u32_none_uf_rem_cas"] = bench_config1(cc, synth, dev)
    if "2a" in want:
        configs["2a_rmat26_ef16_combinations"] = bench_combos(args, cc, off, edg, labels, lab, m)
    if args.minlabel:
        out["minlabel"] = bench_minlabel(cc, off, edg, labels, lab, m)
    if not args.no_amsf and world == 1:
        out["amsf"] = bench_amsf(args, cc, synth, g, dev, ncomp)
    if "2b" in want or "2c" in want:
        # free the headline graph first: the grid's CSR takes about 6 GB
        del g, off, edg, labels, lab
        torch.cuda.empty_cache()
        configs.update(bench_matrix(args, cc, synth, dev, grid="2b" in want, er="2c" in want))
    if "3" in want:
        configs["3_batched_10000_graphs"] = bench_batched(args, cc, synth, dev)
    if "4" in want:
        configs["4_selector"] = bench_selector(args, cc, synth, dev)
    if "5" in want:
        configs["5_incremental_rmat24"] = {f"q{q}": bench_incremental(args, cc, synth, dev, float(q))
                                           for q in args.incr_qfrac.split(",")}
    out["configs"] = configs
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out if rank == 0 else None


def bench_config1(cc, synth, dev, reps=50):
    """The small workload: R-MAT scale 16, edge factor 8, uint32 offsets, no
    sampling + UF-Rem-CAS.  Its CSR (4.7 MB) fits in L2, so L2 is flushed
    (a 256 MB write) before every timed call; each call is timed alone with
    CUDA events and the median is reported.  Launch- and latency-bound: the
    line also carries the launches per call."""
    import torch
    g = synth.rmat(16, 8, seed=1, device=dev)
    off, edg, n, m = g.offsets.to(torch.int32), g.edges, g.n, g.m
    so, fo = cc.sample_opt("none"), cc.finish_opt("uf_rem_cas")
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    cc.cc_static(off, edg, so, fo, labels)
    ok, ncomp = check_labels(off, edg, labels)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)
    times = []
    l0 = cc.launch_count()
    for _ in range(reps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cc.cc_static(off, edg, so, fo, labels)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = (cc.launch_count() - l0) / reps
    # warm (L2-resident) back-to-back calls, for comparison
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        cc.cc_static(off, edg, so, fo, labels)
    e1.record()
    torch.cuda.synchronize()
    warm = e0.elapsed_time(e1) / reps
    ms = statistics.median(times)
    peak, _ = peaks()
    b_csr = 4 * (n + 1) + 4 * m
    del flush
    return {"n": n, "m": m, "offsets": "u32", "sample": "none", "finish": "uf_rem_cas+naive+split_one",
            "ms": round(ms, 4), "gedges_s": round(m / (ms * 1e-3) / 1e9, 3),
            "ms_warm_back_to_back": round(warm, 4), "launches_per_call": launches,
            "b_csr_bytes": b_csr, "hbm_roof_frac": round(b_csr / (peak * 1e9) / (ms * 1e-3), 4),
            "bound": "launch and latency: the CSR is 4.7 MB, the parents 0.26 MB",
            "l2": "flushed before each timed call (256 MB write)", "components": ncomp, "invariants_ok": ok}


def bench_combos(args, cc, off, edg, labels, ref, m):
    import torch
    res = {}
    for s in ("none", "kout", "bfs", "ldd"):
        for f in ("uf_rem_cas", "uf_async", "sv", "lt_prf"):
            so = cc.sample_opt(s)
            fo = cc.finish_opt(f, "naive" if f != "uf_async" else "split")
            cc.cc_static(off, edg, so, fo, labels)
            same = bool(torch.equal(labels, ref))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            e0.record()
            for _ in range(reps):
                cc.cc_static(off, edg, so, fo, labels)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[f"{s}+{f}"] = {"ms": round(ms, 3), "gedges_s": round(m / (ms * 1e-3) / 1e9, 2), "exact": same}
    return res


def bench_minlabel(cc, off, edg, labels, ref, m):
    """The min-label finishes that need not be monotone (Appendix D's sixteen
    Liu-Tarjan variants, Stergiou et al., label propagation), without
    sampling and after k-out: time per call, rounds, labels equal to the
    headline path's."""
    import torch
    res = {}
    kinds = sorted(cc.LT_VARIANTS) + ["stergiou", "label_prop"]
    for s in ("none", "kout"):
        for f in kinds:
            so, fo = cc.sample_opt(s), cc.finish_opt(f)
            _, st = cc.cc_static(off, edg, so, fo, labels, stats=True)
            same = bool(torch.equal(labels, ref))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 2
            e0.record()
            for _ in range(reps):
                cc.cc_static(off, edg, so, fo, labels)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[f"{s}+{f}"] = {"ms": round(ms, 3), "gedges_s": round(m / (ms * 1e-3) / 1e9, 2),
                               "rounds": int(st["rounds"]), "exact": same}
    return res


def bench_amsf(args, cc, synth, g, dev, ncomp):
    """Approximate MSF (Section 5.1) on the benchmark graph with exponential
    weights (mean 1, the paper's weighted inputs), eps from --amsf-eps: each
    mode once after one untimed call, with the forest size checked."""
    import torch
    w = synth.edge_weights(g, 1).to(dev)
    buf = torch.empty(2 * g.n, dtype=torch.int32, device=dev)
    res = {"eps": args.amsf_eps, "weights": "exponential, mean 1"}
    for mode in ("nf_s", "coo", "nf"):
        pairs, wt, _ = cc.cc_amsf(g.offsets, g.edges, w, args.amsf_eps, mode, forest_out=buf)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pairs, wt, _ = cc.cc_amsf(g.offsets, g.edges, w, args.amsf_eps, mode, forest_out=buf)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[mode] = {"ms": round(ms, 3), "gedges_s": round(g.m / (ms * 1e-3) / 1e9, 2), "forest_edges": pairs.shape[0],
                     "size_ok": pairs.shape[0] == g.n - ncomp, "weight": round(wt, 3)}
    del w, buf
    torch.cuda.empty_cache()
    return res


def check_labels(off, edg, lab):
    """Properties of a min-id labelling that hold at any size: both ends of
    every edge share a label, label[v] <= v, labels are fixed points.
    Returns (ok, number of components)."""
    import torch
    n = lab.numel()
    dev = lab.device
    src = torch.repeat_interleave(torch.arange(n, device=dev, dtype=torch.int32), off[1:] - off[:-1])
    ok = bool((lab[src.long()] == lab[edg.long()]).all().item()) if edg.numel() else True
    del src
    ar = torch.arange(n, device=dev, dtype=torch.int32)
    ok = ok and bool((lab <= ar).all().item()) and bool((lab[lab.long()] == lab).all().item())
    return ok, int((lab == ar).sum().item())


def bench_matrix(args, cc, synth, dev, grid=True, er=True):
    """Every sampling x finish combination on the high-diameter grid and on
    the near-percolation Erdos-Renyi graph: ms per call (one untimed call,
    then the mean of `reps`), Gedges/s, and whether the labels equal the
    no-sampling union-find labels (which are checked by the invariants)."""
    import torch
    res = {}
    todo = []
    if grid:
        todo.append(("2b_grid16384x16384_p0.3", lambda: synth.grid2d(16384, 16384, 0.3, seed=1, device=dev)))
    if er:
        todo.append(("2c_er_n2^25_d1.2", lambda: synth.erdos_renyi(1 << 25, 1.2, seed=1, device=dev)))
    for name, make in todo:
        t0 = time.time()
        g = make()
        gen_s = time.time() - t0
        torch.cuda.empty_cache()
        off, edg, n, m = g.offsets, g.edges, g.n, g.m
        labels = torch.empty(n, dtype=torch.int32, device=dev)
        base = cc.cc_static(off, edg, cc.sample_opt("none"), cc.finish_opt("uf_rem_cas"), labels).clone()
        ok, ncomp = check_labels(off, edg, base)
        rows = {}
        for s in ("none", "kout", "bfs", "ldd"):
            for f in ("uf_rem_cas", "uf_async", "sv", "lt_prf"):
                so = cc.sample_opt(s)
                fo = cc.finish_opt(f, "naive" if f != "uf_async" else "split")
                cc.cc_static(off, edg, so, fo, labels)
                same = bool(torch.equal(labels, base))
                reps = 2
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    cc.cc_static(off, edg, so, fo, labels)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                rows[f"{s}+{f}"] = {"ms": round(ms, 3), "gedges_s": round(m / (ms * 1e-3) / 1e9, 2), "exact": same}
        best = min(rows, key=lambda k: rows[k]["ms"])
        res[name] = {"n": n, "m": m, "offsets": "u64", "components": ncomp, "invariants_ok": ok,
                     "gen_s": round(gen_s, 1), "best": best, "combos": rows}
        del g, off, edg, labels, base
        torch.cuda.empty_cache()
    return res


def bench_selector(args, cc, synth, dev):
    """Learned selector on seeded graphs (R-MAT, grids, G(n, M), cliques):
    features and every class's time, training on the first part with the
    library's MLP kernels, and the held-out part scored.  Class times are
    realized: each class as the selected path runs it (features and the
    default's k-out sample included, the sample reused by k-out classes),
    so regret includes the cost of choosing.  The selected path itself
    (features, choice, run in one call) is then timed on every held-out
    graph and compared with plain k-out + UF-Rem-CAS calls.  Regret against
    the plain class times (the twelve combinations as cc_static runs them)
    is reported too, and the paper's decision tree (Section 4.7), whose
    no-sampling branch is timed as plain no-sampling + UF-Rem-CAS."""
    import torch
    from paper_2008_03909_gb300 import selector
    N = args.sel_train + args.sel_test
    X = torch.empty(N, 16, dtype=torch.float32)
    TR = torch.empty(N, 12, dtype=torch.float32)
    TP = torch.empty(N, 12, dtype=torch.float32)
    TN = torch.empty(N, dtype=torch.float32)
    t0 = time.time()
    feat_ms = []
    for i in range(N):
        g = synth.selector_graph(i, seed=7, scale_lo=args.sel_scale_lo, scale_hi=args.sel_scale_hi, device=dev)
        lab = torch.empty(g.n, dtype=torch.int32, device=dev)
        feat_ms.append(selector._timed(lambda: cc.cc_features(g.offsets, g.edges), 2))
        X[i] = cc.cc_features(g.offsets, g.edges).cpu()
        TR[i] = selector.time_classes(g.offsets, g.edges, reps=2, labels=lab, realized=True)
        if i >= args.sel_train:   # scoring only
            TP[i] = selector.time_classes(g.offsets, g.edges, reps=2, labels=lab, realized=False)
            TN[i] = selector._timed(lambda: cc.cc_static(g.offsets, g.edges, cc.sample_opt("none"),
                                                         cc.finish_opt("uf_rem_cas"), lab), 2)
        del g, lab
    collect_s = time.time() - t0
    sel = selector.Selector(device=dev, seed=1)
    t1 = time.time()
    hist = sel.fit(X[: args.sel_train].to(dev), TR[: args.sel_train].to(dev), epochs=800, lr=3e-3)
    train_s = time.time() - t1
    Xt, Tr, Tp, Tn = X[args.sel_train:], TR[args.sel_train:], TP[args.sel_train:], TN[args.sel_train:]
    pick = sel.predict(Xt.to(dev)).cpu()
    # the selected path end to end on each held-out graph, and plain default
    sel_ms, def_ms, exact, ran = [], [], True, []
    so0, fo0 = selector.class_opts(selector.DEFAULT)
    for j, i in enumerate(range(args.sel_train, N)):
        g = synth.selector_graph(i, seed=7, scale_lo=args.sel_scale_lo, scale_hi=args.sel_scale_hi, device=dev)
        lab = torch.empty(g.n, dtype=torch.int32, device=dev)
        ref = torch.empty(g.n, dtype=torch.int32, device=dev)
        cc.cc_static(g.offsets, g.edges, so0, fo0, ref)
        _, c = sel.run(g.offsets, g.edges, lab)
        torch.cuda.synchronize()
        exact = exact and bool(torch.equal(lab, ref))
        ran.append(c)
        sel_ms.append(selector._timed(lambda: sel.run(g.offsets, g.edges, lab), 3))
        def_ms.append(selector._timed(lambda: cc.cc_static(g.offsets, g.edges, so0, fo0, lab), 3))
        del g, lab, ref
    dflt = torch.full((args.sel_test,), selector.DEFAULT, dtype=torch.int32)

    def score(T, ch):
        r = selector.regret(T, ch)
        return {"mean_regret": round(float(r.mean()), 4), "median_regret": round(float(r.median()), 4),
                "p90_regret": round(float(r.quantile(0.9)), 4),
                "total_ms": round(float(T.gather(1, ch.long()[:, None]).sum()), 3)}

    tree = [selector.paper_decision_tree(x) for x in Xt]
    tree_ms = sum(float(Tn[j]) if s == "none" else float(Tp[j, selector.CLASSES.index((s, f))])
                  for j, (s, f) in enumerate(tree))
    res = {"train_graphs": args.sel_train, "heldout_graphs": args.sel_test,
           "scales": [args.sel_scale_lo, args.sel_scale_hi],
           "classes": [f"{s}+{f}" for s, f in selector.CLASSES],
           "selected_path": {"total_ms": round(sum(sel_ms), 3), "labels_exact": exact,
                             "classes_run": torch.bincount(torch.tensor(ran), minlength=12).tolist(),
                             "note": "cc_select_static with the trained network: features, choice and run"},
           "default_plain": {"total_ms": round(sum(def_ms), 3), "note": "cc_static k-out + UF-Rem-CAS"},
           "selected_vs_default_time": round(sum(def_ms) / max(sum(sel_ms), 1e-9), 4),
           "realized": {"mlp": score(Tr, pick), "always_default": score(Tr, dflt),
                        "best_total_ms": round(float(Tr.min(dim=1).values.sum()), 3)},
           "plain": {"mlp": score(Tp, pick), "always_default": score(Tp, dflt),
                     "best_total_ms": round(float(Tp.min(dim=1).values.sum()), 3)},
           "paper_decision_tree": {"total_ms": round(tree_ms, 3),
                                   "picks": {k: sum(1 for t in tree if t == k) for k in set(tree)}},
           "train_loss": [round(hist[0], 4), round(hist[-1], 4)],
           "collect_s": round(collect_s, 1), "train_s": round(train_s, 2),
           "features_ms_median": round(float(torch.tensor(feat_ms).median()), 4)}
    res["paper_decision_tree"]["picks"] = {f"{a}+{b}": v for (a, b), v in res["paper_decision_tree"]["picks"].items()}
    return res


def bench_batched(args, cc, synth, dev):
    """The batched workload (10,000 graphs, uint32 packed CSR): one
    autotuned persistent launch vs one cc_static call per graph (no
    sampling, union-find finish), same labels.  The batch's CSR (about 1.8
    GB) exceeds L2.  The launch's roofline counts its compulsory bytes: the
    offsets 4(V+1), the edges 4M and the labels written 4V (parents live in
    shared memory), over the kernel's own time."""
    import torch
    t0 = time.time()
    gs = synth.batch_config3(args.batched_graphs, seed=1)
    gv, off, edg = synth.pack(gs)
    gen_s = time.time() - t0
    V, M = off.numel() - 1, edg.numel()
    if M < 2**32:
        off = off.to(torch.int32)
    gv, off, edg = gv.to(dev), off.to(dev), edg.to(dev)
    ob = 4 if off.dtype == torch.int32 else 8
    if args.batched_schedule:
        t, sm, md = (int(x) for x in args.batched_schedule.split(","))
        best = cc.batch_opt(t, sm, md)
        lab = cc.cc_batched(gv, off, edg, best)
    else:
        lab, best, tune_ms = cc.cc_batched_autotune(gv, off, edg)
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        cc.cc_batched(gv, off, edg, best, lab)
    e1.record()
    torch.cuda.synchronize()
    ms_batched = e0.elapsed_time(e1) / reps
    # the kernel alone, from the library's per-launch events
    cc.profile_enable(True)
    for _ in range(reps):
        cc.cc_batched(gv, off, edg, best, lab)
    torch.cuda.synchronize()
    prof = cc.profile_read()
    cc.profile_enable(False)
    kl, kms = prof.get("k_batched", (reps, ms_batched * reps))
    k_ms = kms / max(kl, 1)
    peak, peak_kind = peaks()
    ab = ob * (V + 1) + 4 * M + 4 * V
    ach = ab / (k_ms * 1e-3) / 1e9
    # one plain launch per graph, on the same packed arrays
    ref = torch.empty_like(lab)
    gvh = gv.cpu().tolist()
    so, fo = cc.sample_opt("none"), cc.finish_opt("uf_rem_cas")
    torch.cuda.synchronize()
    e0.record()
    for i in range(len(gs)):
        b, e = gvh[i], gvh[i + 1]
        if e > b:
            cc.cc_static(off[b:e + 1], edg, so, fo, ref[b:e])
    e1.record()
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    return {"graphs": len(gs), "vertices": V, "edges": M, "offsets": "u32" if ob == 4 else "u64",
            "gen_s": round(gen_s, 1),
            "schedule": {"threads": best.threads, "smem_max_vertices": best.smem_max_vertices,
                         "vertex_mode": best.vertex_mode},
            "ms_batched": round(ms_batched, 4), "edges_per_s_batched": round(M / (ms_batched * 1e-3), 1),
            "roofline": {"kernel": "k_batched", "bound": "hbm", "algorithmic_bytes": ab, "ms_avg": round(k_ms, 5),
                         "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                         "peak_kind": peak_kind},
            "ms_per_graph_launches": round(ms_plain, 3), "edges_per_s_per_graph_launches": round(M / (ms_plain * 1e-3), 1),
            "speedup": round(ms_plain / ms_batched, 2), "labels_equal": bool(torch.equal(lab, ref))}


def bench_incremental(args, cc, synth, dev, qf):
    """The served workload at query fraction qf: an R-MAT scale-24 edge
    factor 16 base in a resident union-find, then the batches (log-uniform
    in [1e3, 1e7] operations, inserts R-MAT distributed, queries uniform)
    staged in pinned host memory.  Times the plain loop (one insert and one
    query launch per batch, host -> device -> answers -> host, synchronous)
    and the continuous-batching request loop, back to back and paced at the
    plain loop's batch rate; every batch's answers of the request loop are
    compared with the plain loop's."""
    import torch
    base = synth.rmat(args.incr_scale, 16, seed=2, device=dev)
    n = base.n
    inc = cc.Incremental(n, base.offsets, base.edges, finish=cc.finish_opt(args.incr_finish))
    del base
    torch.cuda.empty_cache()
    sizes = synth.log_uniform_sizes(args.incr_batches, 1e3, 1e7, seed=3, stream=50)
    # stage every batch in pinned host memory (inserts R-MAT distributed,
    # queries uniform), then time host -> device -> answers -> host
    batches = []
    for b, sz in enumerate(sizes):
        nq = int(round(sz * qf))
        ni = sz - nq
        ins = synth.rmat_pairs(args.incr_scale, ni, seed=100 + b, stream=60, device=dev).reshape(-1)
        qs = synth.random_pairs(n, nq, seed=100 + b, stream=70, device=dev).reshape(-1)
        batches.append((ins.cpu().pin_memory(), qs.cpu().pin_memory(), ni, nq))
    max_i = max(b[2] for b in batches) * 2 + 2
    max_q = max(b[3] for b in batches) * 2 + 2
    d_ins = torch.empty(max_i, dtype=torch.int32, device=dev)
    d_qs = torch.empty(max_q, dtype=torch.int32, device=dev)
    d_ans = torch.empty(max_q // 2, dtype=torch.uint8, device=dev)
    plain_ans = [torch.empty(max(1, nq), dtype=torch.uint8).pin_memory() for (_, _, _, nq) in batches]
    stream = torch.cuda.current_stream()
    lat_dev, lat_e2e = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in batches]
    total_ins = total_q = 0
    torch.cuda.synchronize()
    t_all = time.perf_counter()
    for (hi, hq, ni, nq), (a, b), h_ans in zip(batches, ev, plain_ans):
        t1 = time.perf_counter()
        d_ins[: 2 * ni].copy_(hi, non_blocking=True)
        d_qs[: 2 * nq].copy_(hq, non_blocking=True)
        a.record(stream)
        inc.insert(d_ins[: 2 * ni])
        inc.query(d_qs[: 2 * nq], out=d_ans[:nq])
        b.record(stream)
        h_ans[:nq].copy_(d_ans[:nq], non_blocking=True)
        stream.synchronize()
        lat_e2e.append((time.perf_counter() - t1) * 1e3)
        total_ins += ni
        total_q += nq
    wall = time.perf_counter() - t_all
    for a, b in ev:
        lat_dev.append(a.elapsed_time(b))
    dev_s = sum(lat_dev) / 1e3
    inc.close()

    def pct(xs, p):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(math.ceil(p / 100 * len(xs))) - 1)]

    # the same batches through the continuous-batching request loop, twice:
    # back to back (maximum throughput) and paced at the plain loop's batch
    # rate (latency at the load the plain loop sustains)
    answers = [torch.empty(max(1, nq), dtype=torch.uint8).pin_memory() for (_, _, _, nq) in batches]

    def served(interval_s, stage=False):
        base = synth.rmat(args.incr_scale, 16, seed=2, device=dev)
        inc2 = cc.Incremental(n, base.offsets, base.edges, finish=cc.finish_opt(args.incr_finish))
        del base
        torch.cuda.empty_cache()
        srv = cc.Server(inc2, slots=4, slot_pairs=1 << 22, stage=stage)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = []
        for i, (hi, hq, ni, nq) in enumerate(batches):
            if interval_s:
                while time.perf_counter() < t0 + i * interval_s:
                    pass
            tickets.append(srv.submit(hi, hq, answers[i]))
        lats = []
        for t in tickets:
            _, l = srv.wait(t)
            lats.append(l)
        w = time.perf_counter() - t0
        # every batch's answers equal the plain loop's
        same = all(torch.equal(answers[i][:nq], plain_ans[i][:nq]) for i, (_, _, _, nq) in enumerate(batches))
        srv.close()
        inc2.close()
        return w, lats, same

    served(0.0)   # warm-up: the first request loop of a process pays one-time costs
    wall_srv, lat_srv, same_all = served(0.0)
    wall_pace, lat_pace, same_pace = served(wall / len(batches))
    wall_st, lat_st, same_st = served(0.0, stage=True)
    return {"base": f"rmat{args.incr_scale}_ef16", "n": n, "finish": args.incr_finish, "batches": len(batches),
            "query_fraction": qf,
            "inserts": total_ins, "queries": total_q,
            "updates_per_s_device": round(total_ins / dev_s, 1), "ops_per_s_device": round((total_ins + total_q) / dev_s, 1),
            "updates_per_s_e2e": round(total_ins / wall, 1), "ops_per_s_e2e": round((total_ins + total_q) / wall, 1),
            "p50_ms_device": round(pct(lat_dev, 50), 4), "p99_ms_device": round(pct(lat_dev, 99), 4),
            "p50_ms_e2e": round(pct(lat_e2e, 50), 4), "p99_ms_e2e": round(pct(lat_e2e, 99), 4),
            "batch_sizes": "log-uniform in [1e3, 1e7], seeded",
            "served": {"updates_per_s": round(total_ins / wall_srv, 1),
                       "ops_per_s": round((total_ins + total_q) / wall_srv, 1),
                       "p50_ms": round(pct(lat_srv, 50), 4), "p99_ms": round(pct(lat_srv, 99), 4),
                       "wall_s": round(wall_srv, 4), "plain_wall_s": round(wall, 4),
                       "speedup_vs_plain": round(wall / wall_srv, 3),
                       "answers_equal_plain_every_batch": same_all and same_pace and same_st,
                       "transfer": "kernels read the pinned requests in place over the host link",
                       "staged": {"ops_per_s": round((total_ins + total_q) / wall_st, 1),
                                  "p50_ms": round(pct(lat_st, 50), 4), "p99_ms": round(pct(lat_st, 99), 4),
                                  "wall_s": round(wall_st, 4),
                                  "note": "every request copied through 4 device slots of 2^22 pairs by the copy "
                                          "engines (CC_SERVER_STAGE)"},
                       "latency": "submit to answers in host memory, all batches submitted back to back",
                       "paced": {"interval_ms": round(1e3 * wall / len(batches), 4),
                                 "p50_ms": round(pct(lat_pace, 50), 4), "p99_ms": round(pct(lat_pace, 99), 4),
                                 "wall_s": round(wall_pace, 4)}}}


def cpu_baseline(off, edg, seconds):
    """The oracle's sequential union-find (O1) over the whole graph on one
    host core (about 20 s at R-MAT scale 26), in Gedges/s; when a whole-graph
    run would take far longer than `seconds` (estimated on a prefix), the
    run covers a prefix of the vertices sized for `seconds` instead."""
    import numpy as np
    import oracle
    offs = off.cpu().numpy().astype(np.uint64)
    n = offs.shape[0] - 1
    m = int(offs[-1])
    # estimate the rate on a small prefix
    u_end = min(n, int(np.searchsorted(offs, 20_000_000)))
    e_end = int(offs[u_end])
    edges = edg[:e_end].cpu().numpy().view(np.uint32)
    t0 = time.perf_counter()
    _, cnt = _prefix(oracle, offs, edges, u_end, np.arange(n, dtype=np.uint32))
    rate = cnt / max(time.perf_counter() - t0, 1e-9)
    if m <= rate * seconds * 2.5:
        u_end, e_end = n, m
    else:
        u_end = min(n, int(np.searchsorted(offs, int(rate * seconds))))
        e_end = int(offs[u_end])
    edges = edg[:e_end].cpu().numpy().view(np.uint32)
    P = np.arange(n, dtype=np.uint32)
    t0 = time.perf_counter()
    _, cnt = _prefix(oracle, offs, edges, u_end, P)
    dt = time.perf_counter() - t0
    what = ("the whole graph" if u_end == n else f"the edges of vertices [0, {u_end})")
    return {"value": round(cnt / dt / 1e9, 5), "unit": "Gedges/s", "cores": 1, "kind": "oracle",
            "sample": f"O1 sequential union-find over {what} ({cnt} of {m} directed edges) of the same graph, "
                      f"{dt:.1f} s",
            "seconds": round(dt, 2), "host_cores": len(os.sched_getaffinity(0))}


def _prefix(oracle, offs, edges, u_end, P):
    """uf_prefix on a CSR whose edge array holds only the prefix's edges."""
    import ctypes
    import numpy as np
    L = oracle.lib()
    Ip = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    Ap = edges.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    cnt = L.oracle_uf_prefix(offs.shape[0] - 1, Ip, Ap, u_end, P.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return P, int(cnt)


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample (O1
    over a prefix of the same graph's vertices) on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import numpy as np
    import torch
    import oracle
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    g = make_graph(args.scale, args.edge_factor, dev)
    offs = g.offsets.cpu().numpy().astype(np.uint64)
    n = g.n
    per_step = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    target = 5_000_000
    u_end = min(n, int(np.searchsorted(offs, target)))
    edges = g.edges[: int(offs[u_end])].cpu().numpy().view(np.uint32)
    t0 = time.perf_counter()
    _, cnt = _prefix(oracle, offs, edges, u_end, np.arange(n, dtype=np.uint32))
    rate = cnt / max(time.perf_counter() - t0, 1e-9)
    want = min(int(offs[-1]), int(rate * per_step))
    u_end = min(n, int(np.searchsorted(offs, want)))
    e_end = int(offs[u_end])
    edges = g.edges[:e_end].cpu().numpy().view(np.uint32)
    for _ in range(args.warmup):
        _prefix(oracle, offs, edges, u_end, np.arange(n, dtype=np.uint32))
    times = []
    for _ in range(args.steps):
        P = np.arange(n, dtype=np.uint32)
        t0 = time.perf_counter()
        _, cnt = _prefix(oracle, offs, edges, u_end, P)
        times.append(time.perf_counter() - t0)
    dt = sum(times) / len(times)
    value = cnt / dt / 1e9
    sample = f"O1 over the edges of vertices [0, {u_end}) ({cnt} directed edges) of rmat{args.scale}_ef{args.edge_factor}"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "Gedges/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}_ef{args.edge_factor}", "n": n, "m": int(offs[-1]),
                       "sample": "none", "finish": "O1 sequential union-find (the oracle)"},
            "cpu_baseline": {"value": round(value, 5), "unit": "Gedges/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "Gedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
