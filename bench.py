"""Benchmark: CFL-reachability solve throughput on one GB300 (pairs/s).

One step is one pass of the whole hot path on the alias-analysis workload
(Fig. "wcnf:fica" grammar, 200 000-vertex program-shaped graph with 400 000
'a' and 150 000 'd' edges plus their reverses):
  terminal initialisation from the device-resident edges (cflr_reset),
  the semi-naive closure loop to its fixpoint (cflr_solve),
  and the extraction of every named non-terminal's sorted pairs into
  device buffers, one after another (cflr_get_pairs_device_many).
value = pairs of all named non-terminals / step time (CUDA events on the
solve stream, L2 flushed between steps).  e2e repeats the step through the
host-buffer API: grammar text and host edges in, host pair arrays out.
After the timed steps the extracted pairs of every named non-terminal are
fingerprinted and compared with the oracle's stored fingerprints.

The default line also carries the other workloads, each with its own step
time: the 64-field points-to solve (500 000 vertices), the field-sensitive
alias solve (142 fields, 41 652 vertices) and the context-sensitive
value-flow solve (512 call sites, 100 000 vertices), the 256 batched Dyck-3
instances (one batched CUDA-graph solve against each instance alone in the
per-production form) and a short served Poisson stream of alias solves.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cflr|reference]
                  [--workload all|fica|fsjpt|dyck3_batch|serving]

Under torchrun (N > 1) every rank solves its own replica (different seed):
the single-instance fixpoint has no exchange step that would let it shard,
so multi-GPU runs are independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2401_11029_gb300 import gen  # noqa: E402

METRIC = "CFL-r solve throughput (pairs of all non-terminals / solve time)"
UNIT = "pairs/s"
WORKLOAD = {"workload": "fica_like alias analysis (Fig. wcnf:fica)", "n_vertices": 200_000,
            "a_edges": 400_000, "d_edges": 150_000, "reverse_edges": True, "seed": 2}
FSJPT = {"workload": "fsjpt_like field-sensitive points-to (Fig. wcnf:fsjpt, 64 fields)",
         "n_vertices": 500_000, "forward_edges": 2_000_000, "reverse_edges": True, "seed": 3,
         "productions": 514}
SAMPLE_N = 20_000     # oracle sample: same generator and ratios, 1/10 of the vertices
TUNING_CACHE = os.path.join(ROOT, "paper_2401_11029_gb300", "tuning", "gb300.txt")
GOLDEN = os.path.join(ROOT, "tests", "golden")


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback"}


def workload_graph(seed: int, n: int = None, kind: str = "fica"):
    if kind == "fsjpt":
        n = n or FSJPT["n_vertices"]
        return gen.fsjpt_like(n=n, n_edges=FSJPT["forward_edges"] * n // FSJPT["n_vertices"],
                              seed=seed)
    n = n or WORKLOAD["n_vertices"]
    scale = n / WORKLOAD["n_vertices"]
    return gen.fica_like(n=n, n_a=int(WORKLOAD["a_edges"] * scale),
                         n_d=int(WORKLOAD["d_edges"] * scale), seed=seed)


def grammar_of(kind: str) -> str:
    return gen.grammar_text("fsjpt" if kind == "fsjpt" else "fica")


def golden_of(name: str, g) -> dict | None:
    """The oracle's stored fingerprints of workload `name`, when they exist
    and were made from this very edge list."""
    path = os.path.join(GOLDEN, name + ".json")
    try:
        with open(path) as f:
            gold = json.load(f)
    except OSError:
        return None
    if g is not None and gold.get("edge_digest") != g.edge_digest():
        return None
    return gold


def golden_name(kind: str, n: int) -> str:
    return {"fica": f"fica_like_{n // 1000}k", "fsjpt": f"fsjpt_like_{n // 1000}k"}[kind]


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profile(kernel: str, workload: str = "fica_like"):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if
    the kernel source has not changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernels_cu_sha256:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if not m or not t:
        return None
    src = open(os.path.join(ROOT, "paper_2401_11029_gb300", "csrc", "kernels.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest() != m.group(1):
        return None
    return int(t.group(1))


def oracle_sample_graph(kind: str = "fica"):
    return workload_graph(WORKLOAD["seed"] if kind == "fica" else FSJPT["seed"], SAMPLE_N, kind)


def cpu_oracle_sample(kind: str = "fica") -> dict:
    """The oracle, as it stands, on a bounded sample of the workload: the same
    generator and ratios at SAMPLE_N vertices."""
    import oracle
    g = oracle_sample_graph(kind)
    text = grammar_of(kind)
    res = oracle.solve(text, g)
    pairs = res.total()
    name = "fsjpt_like" if kind == "fsjpt" else "fica_like"
    out = {"value": pairs / res.seconds, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{name} n={SAMPLE_N} (same generator and ratios as the workload, "
                     f"{g.n_edges} edges, {pairs} pairs), one worklist solve, "
                     f"{res.seconds:.1f} s on 1 host core", "seconds": res.seconds,
           "sample_edges": g.n_edges, "sample_pairs": pairs}
    full = golden_of(golden_name(kind, (WORKLOAD if kind == "fica" else FSJPT)["n_vertices"]),
                     None)
    if full and full.get("oracle_seconds"):
        # context only: the same oracle at the full size, recorded when the
        # stored fingerprints were written (one core of the x86 build host)
        out["full_size_oracle"] = {
            "value": full["total_pairs"] / full["oracle_seconds"], "unit": UNIT,
            "seconds": full["oracle_seconds"], "pairs": full["total_pairs"],
            "where": "1 core of the x86-64 build host, recorded with tests/golden/"
                     f"{full['workload']}.json"}
    return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local, dist


def aggregate(dist, device, ms: float, pairs: int, e2e_s: float):
    """Whole-job figures over the ranks: the slowest rank's step time and
    end-to-end time, and the pairs of all ranks (each rank solves its own
    replica, so the work adds up)."""
    if dist is None:
        return ms, float(pairs), e2e_s
    import torch
    t = torch.tensor([ms, float(pairs), e2e_s], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1]), float(mx[2])


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores, on a
    bounded sample of the headline workload (rank 0 only)."""
    world, rank, local, dist = dist_setup()
    if rank != 0:
        return
    vals, secs = [], []
    info = None
    for _ in range(args.warmup):
        cpu_oracle_sample()
    for _ in range(args.steps):
        info = cpu_oracle_sample()
        vals.append(info["value"])
        secs.append(info.pop("seconds"))
    v = statistics.mean(vals)
    info["value"] = v
    scale = SAMPLE_N / WORKLOAD["n_vertices"]
    # the configuration actually solved: the sample, not the full workload
    config = dict(WORKLOAD, n_vertices=SAMPLE_N, a_edges=int(WORKLOAD["a_edges"] * scale),
                  d_edges=int(WORKLOAD["d_edges"] * scale), edges=info["sample_edges"],
                  pairs=info["sample_pairs"],
                  sample_of=f"fica_like at {WORKLOAD['n_vertices']} vertices (same generator "
                            "and ratios, 1/10 of the vertices)",
                  parallelism=f"replicas{args.gpus}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # one step is one oracle solve of the bounded sample
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": config, "cpu_baseline": info,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the timed launch configuration (shared with the full-size parity tests)
# ---------------------------------------------------------------------------

def label_array(ctx, g) -> np.ndarray:
    """Terminal id of every edge (0xFFFFFFFF for labels the grammar lacks)."""
    from paper_2401_11029_gb300 import cflr
    term = {}
    for name in g.labels:
        try:
            i, is_t = cflr.cflr_symbol_id(ctx, name)
            term[name] = i if is_t else 0xFFFFFFFF
        except cflr.CflrError:
            term[name] = 0xFFFFFFFF
    return np.asarray([term[x] for x in g.labels], np.uint32)[g.lab]


def timed_context(g, text, device: int, stream, autotune: bool = True, **cfg):
    """The context the bench times: the device-driven loop (one CUDA graph per
    solve) with the product schedule cflr_autotune picks from the tuning
    cache.  Returns (ctx, tuning)."""
    from paper_2401_11029_gb300 import cflr
    ctx = cflr.cflr_create(device=device, stream=stream, form=cflr.CFLR_FORM_GRAPH,
                           autotune_cache=TUNING_CACHE.encode(), **cfg)
    cflr.cflr_load_grammar(ctx, text)
    cflr.cflr_load_graph(ctx, g.n, g.src, label_array(ctx, g), g.dst)
    tuning = cflr.cflr_autotune(ctx) if autotune else cflr.cflr_get_tuning(ctx)
    return ctx, tuning


def device_step(ctx, n_named: int, out=None, last: dict | None = None) -> int:
    """One step: reset, solve, and extract every named non-terminal's pairs
    into the device buffers `out` (src, dst); returns the pair count."""
    from paper_2401_11029_gb300 import cflr
    cflr.cflr_reset(ctx)
    st = cflr.cflr_solve(ctx)
    if last is not None:
        last.update(st)
    ids = np.arange(n_named, dtype=np.uint32)
    if out is None:
        return int(cflr.cflr_get_pairs_many(ctx, ids, count_only=True)[-1])
    off = cflr.cflr_get_pairs_device_many(ctx, ids, out[0].data_ptr(), out[1].data_ptr(),
                                          min(out[0].numel(), out[1].numel()))
    return int(off[-1])


def device_fingerprints(ctx, names, out) -> dict:
    """Fingerprint of each named non-terminal's pairs as the device extraction
    writes them, all in one call (out: device buffers that hold them all)."""
    from paper_2401_11029_gb300 import cflr
    ids = [cflr.cflr_symbol_id(ctx, name)[0] for name in names]
    off = cflr.cflr_get_pairs_device_many(ctx, ids, out[0].data_ptr(), out[1].data_ptr(),
                                          min(out[0].numel(), out[1].numel()))
    total = int(off[-1])
    s_all = out[0][:total].cpu().numpy().view(np.uint32)
    d_all = out[1][:total].cpu().numpy().view(np.uint32)
    fps = {}
    for i, name in enumerate(names):
        a, b = int(off[i]), int(off[i + 1])
        keys = gen.pair_keys(s_all[a:b], d_all[a:b])
        if keys.size > 1 and not np.all(keys[1:] > keys[:-1]):
            fps[name] = "unsorted"
        else:
            fps[name] = gen.pair_fingerprint(keys)
    return fps


def parity_record(ctx, gold: dict | None, out) -> dict:
    if not gold:
        return {"checked": False, "why": "no stored oracle fingerprints for this graph"}
    fps = device_fingerprints(ctx, list(gold["pairs"]), out)
    bad = [x for x, fp in gold["pairs"].items() if fps.get(x) != fp]
    return {"checked": True, "match": not bad, "mismatched": bad[:8],
            "nonterminals": len(gold["pairs"]),
            "against": f"oracle fingerprints tests/golden/{gold['workload']}.json"}


def kernel_rows(before: dict, after: dict) -> list:
    rows = []
    for name, a in after.items():
        b = before.get(name, {"launches": 0, "ms": 0.0, "alg_bytes": 0})
        rows.append((a["ms"] - b["ms"], a["launches"] - b["launches"],
                     a["alg_bytes"] - b["alg_bytes"], name))
    rows.sort(reverse=True)
    return rows


def roofline_of(rows: list, workload: str) -> dict:
    kms, kl, kb, kname = rows[0]
    pk = peaks()
    achieved = (kb / 1e9) / (kms / 1e3) if kms > 0 else 0.0
    return {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic_from_profile(kname, workload),
            "kernel": kname, "launches": kl, "avg_launch_ms": kms / max(kl, 1),
            "peak_src": pk["src"]}


def profiled_kernels(g, text, tuning, device, stream, n_named, out, flush, steps, warmup,
                     expect):
    """Per-kernel event times of the same steps: a context with the same
    schedule whose iterations are launched one by one from the host with
    CUDA events around every kernel (events cannot sit inside the graph's
    loop body)."""
    from paper_2401_11029_gb300 import cflr
    pctx = cflr.cflr_create(device=device, stream=stream, form=cflr.CFLR_FORM_BATCHED, profile=1)
    cflr.cflr_load_grammar(pctx, text)
    cflr.cflr_set_tuning(pctx, tuning["probe_ratio"], tuning["bin_limit"], tuning["ctas_per_sm"])
    cflr.cflr_load_graph(pctx, g.n, g.src, label_array(pctx, g), g.dst)
    for _ in range(warmup):
        device_step(pctx, n_named, out)
    before = {k["name"]: k for k in cflr.cflr_kernel_stats(pctx)}
    for _ in range(steps):
        flush.fill_(1)
        assert device_step(pctx, n_named, out) == expect
    import torch
    torch.cuda.synchronize()
    after = {k["name"]: k for k in cflr.cflr_kernel_stats(pctx)}
    cflr.cflr_destroy(pctx)
    return kernel_rows(before, after)


def timed_steps(ctx, n_named, out, flush, stream, steps, fill=1, expect=None, last=None):
    import torch
    step_ms = []
    for _ in range(steps):
        flush.fill_(fill)                          # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p = device_step(ctx, n_named, out, last)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        if expect is not None:
            assert p == expect, "pair count changed between steps"
    return step_ms


def run_cflr(args, kind: str = "fica", extras: bool = False):
    import torch
    from paper_2401_11029_gb300 import cflr

    world, rank, local, dist = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl = FSJPT if kind == "fsjpt" else WORKLOAD
    seed = wl["seed"] + 1000 * rank
    g = workload_graph(seed, args.vertices, kind)
    text = grammar_of(kind)

    ctx, tuning = timed_context(g, text, local, stream.cuda_stream,
                                autotune=not args.no_autotune)
    n_nt, n_named, _ = cflr.cflr_grammar_sizes(ctx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    last = {}
    pairs = device_step(ctx, n_named, None, last)
    out = (torch.empty(max(pairs, 1), dtype=torch.int32, device=dev),
           torch.empty(max(pairs, 1), dtype=torch.int32, device=dev))
    for _ in range(max(0, args.warmup - 1)):
        device_step(ctx, n_named, out)

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms = timed_steps(ctx, n_named, out, flush, stream, args.steps, rank + 1, pairs, last)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    solve_stats = dict(last)
    # the result of the timed configuration against the oracle's fingerprints
    gold = golden_of(golden_name(kind, g.n), g) if rank == 0 else None
    parity = parity_record(ctx, gold, out) if rank == 0 else None

    rows = profiled_kernels(g, text, tuning, local, stream.cuda_stream, n_named, out, flush,
                            args.steps, args.warmup, pairs)

    # end-to-end through the host-buffer API
    h_src = torch.from_numpy(g.src.astype(np.uint32).view(np.int32)).pin_memory()
    h_dst = torch.from_numpy(g.dst.astype(np.uint32).view(np.int32)).pin_memory()
    h_out_s = torch.empty(max(pairs, 1), dtype=torch.int32).pin_memory()
    h_out_d = torch.empty(max(pairs, 1), dtype=torch.int32).pin_memory()
    h_out = (h_out_s.numpy().view(np.uint32), h_out_d.numpy().view(np.uint32))
    ids = np.arange(n_named, dtype=np.uint32)
    lab_ids = label_array(ctx, g)
    h_lab = torch.from_numpy(lab_ids.view(np.int32)).pin_memory()
    lib = cflr.load_library()
    import ctypes
    e2e_s = []
    phases = {"create_grammar": [], "load_graph": [], "solve": [], "pairs_to_host": []}
    for k in range(args.steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        c2 = cflr.cflr_create(device=local, stream=stream.cuda_stream,
                              form=cflr.CFLR_FORM_GRAPH, autotune_cache=TUNING_CACHE.encode())
        cflr.cflr_load_grammar(c2, text)
        t1 = time.perf_counter()
        rc = lib.cflr_load_graph(c2, g.n, g.n_edges, h_src.data_ptr(), h_lab.data_ptr(),
                                 h_dst.data_ptr())
        assert rc == 0
        if not args.no_autotune:
            cflr.cflr_autotune(c2)          # the cached schedule of this workload
        t2 = time.perf_counter()
        st2 = cflr.cflr_solve(c2)
        t3 = time.perf_counter()
        tot = int(cflr.cflr_get_pairs_many(c2, ids, out=h_out)[2][-1])
        torch.cuda.synchronize(dev)
        t4 = time.perf_counter()
        dt = t4 - t0
        cflr.cflr_destroy(c2)
        if k > 0:                                   # first call warms the allocator
            e2e_s.append(dt)
            for key, a, b in (("create_grammar", t0, t1), ("load_graph", t1, t2),
                              ("solve", t2, t3), ("pairs_to_host", t3, t4)):
                phases[key].append(1e3 * (b - a))
            fresh = {k: st2[k] for k in ("regrow_buffers", "regrow_sets", "regrow_pools")}
        assert tot == pairs
    # a bare copy of the same bytes into the same pinned arrays, for context:
    # the host copy bandwidth differs between boxes and runs
    bare = []
    for k in range(4):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h_out_s.copy_(out[0], non_blocking=True)
        h_out_d.copy_(out[1], non_blocking=True)
        torch.cuda.synchronize(dev)
        if k:
            bare.append(1e3 * (time.perf_counter() - t0))

    ms = statistics.mean(step_ms)
    ms_all, pairs_all, e2e_all = aggregate(dist, dev, ms, pairs, statistics.mean(e2e_s))
    # + the read-out of each step: unit counts, a three-kernel scan, the rows,
    # the long rows (one list extraction of every named non-terminal)
    launches = sum(r[1] for r in rows) + args.steps * 6
    if rank != 0:
        cflr.cflr_destroy(ctx)
        return
    line = {
        "metric": METRIC, "value": pairs_all / (ms_all / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": dict(wl, n_vertices=int(g.n), edges=int(g.n_edges), pairs=int(pairs),
                       parallelism=f"replicas{world}",
                       l2="flushed between steps (256 MiB write)"),
        "e2e": {"value": pairs_all / e2e_all, "unit": UNIT,
                "h2d_bytes_per_step": int(12 * g.n_edges),
                "d2h_bytes_per_step": int(8 * pairs),
                "phases_ms": {k: round(statistics.mean(v), 2) for k, v in phases.items()},
                "pairs_to_host_each_ms": [round(v, 2) for v in phases["pairs_to_host"]],
                "bare_d2h_copy_ms": round(statistics.median(bare), 2),
                "fresh_context_regrows": fresh},
        "gpu_launches": int(launches),
        "roofline": roofline_of(rows, "fsjpt_like" if kind == "fsjpt" else "fica_like"),
        "kernels": [{"name": r[3], "ms": round(r[0], 4), "launches": r[1],
                     "gbs": round((r[2] / 1e9) / (r[0] / 1e3), 1) if r[0] > 0 else None}
                    for r in rows if r[1]],
        "clocks": clk,
        "tuning": tuning,
        "parity": parity,
        "solve": {"form": "graph", "iterations": solve_stats["iterations"],
                  "groups_per_bin": solve_stats["groups"],
                  "flops": solve_stats["flops"], "flops_bin3": solve_stats["flops_bin3"],
                  "mask_tiles_bin3": solve_stats["mask_tiles_bin3"],
                  "candidates": solve_stats["candidates"],
                  "peak_device_bytes": solve_stats["peak_device_bytes"],
                  "regrows_last_step": solve_stats["regrows"]},
        "steps_ms": [round(t, 3) for t in step_ms],
        "roofline_note": "kernel times from the same steps replayed with per-kernel CUDA "
                         "events (host-launched iterations) right after the timed region",
    }
    cflr.cflr_destroy(ctx)
    del out, flush
    torch.cuda.empty_cache()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(kind)
        line["cpu_baseline"].pop("seconds")
    if extras and world == 1:
        # the other workloads, each with its own steps (fewer of them)
        sub = argparse.Namespace(**vars(args))
        sub.steps = max(1, min(args.steps, 5))
        sub.warmup = max(3, min(args.warmup, 3))
        sub.vertices = None
        for name in EXTRA:
            line[name] = run_extra(name, sub)
        line["dyck3_batch_256"] = run_dyck3_batch(sub, print_line=False)
        sub.requests = args.extra_requests
        sub.serve_warmup = 1.0
        line["serving"] = run_serving(sub, print_line=False)
    print(json.dumps(line), flush=True)


# The other single-instance workloads of the default line: name -> (config,
# graph, grammar text, stored oracle fingerprints)
EXTRA = {
    "fsjpt_like_500k": (FSJPT, lambda: workload_graph(FSJPT["seed"], None, "fsjpt"),
                        lambda: grammar_of("fsjpt")),
    "fsca_like_41k": ({"workload": "fsca_like field-sensitive alias (Fig. wcnf:fsca, 142 "
                                   "fields; the shape of the imagick graph)",
                       "n_vertices": 41_652, "forward_edges": 55_775, "reverse_edges": True,
                       "seed": 6},
                      lambda: gen.fsca_like(), lambda: gen.grammar_text("fsca", index_hi=141)),
    "cscvf_like_100k": ({"workload": "cscvf_like context-sensitive value flow (Fig. "
                                     "wcnf:cscvf, 512 call sites)",
                         "n_vertices": 100_000, "edges": 168_000, "call_sites": 512,
                         "seed": 7},
                        lambda: gen.cscvf_like(n=100_000, n_edges=168_000, calls=512),
                        lambda: gen.grammar_text("cscvf", index_hi=511)),
}


def run_extra(name, args) -> dict:
    """One of the EXTRA workloads in the timed configuration: step time,
    pairs/s, the roofline of its dominant kernel and parity."""
    import torch
    from paper_2401_11029_gb300 import cflr
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wl, make_graph, make_text = EXTRA[name]
    g = make_graph()
    text = make_text()
    ctx, tuning = timed_context(g, text, 0, stream.cuda_stream)
    n_nt, n_named, _ = cflr.cflr_grammar_sizes(ctx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    last = {}
    pairs = device_step(ctx, n_named, None, last)
    out = (torch.empty(max(pairs, 1), dtype=torch.int32, device=dev),
           torch.empty(max(pairs, 1), dtype=torch.int32, device=dev))
    for _ in range(max(0, args.warmup - 1)):
        device_step(ctx, n_named, out)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize(dev)
    step_ms = timed_steps(ctx, n_named, out, flush, stream, args.steps, 1, pairs, last)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    parity = parity_record(ctx, golden_of(name, g), out)
    rows = profiled_kernels(g, text, tuning, 0, stream.cuda_stream, n_named, out, flush,
                            args.steps, args.warmup, pairs)
    cflr.cflr_destroy(ctx)
    ms = statistics.mean(step_ms)
    return {"metric": METRIC, "value": pairs / (ms / 1e3), "unit": UNIT, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms,
            "config": dict(wl, edges=int(g.n_edges), pairs=int(pairs), nonterminals=n_nt,
                           l2="flushed between steps (256 MiB write)"),
            "roofline": roofline_of(rows, name.rsplit("_", 1)[0]),
            "kernels": [{"name": r[3], "ms": round(r[0], 4), "launches": r[1],
                         "gbs": round((r[2] / 1e9) / (r[0] / 1e3), 1) if r[0] > 0 else None}
                        for r in rows if r[1]][:6],
            "clocks": clk, "tuning": tuning, "parity": parity,
            "solve": {"form": "graph", "iterations": last["iterations"],
                      "groups_per_bin": last["groups"], "regrows_last_step": last["regrows"]},
            "steps_ms": [round(t, 3) for t in step_ms]}


def run_dyck3_batch(args, print_line: bool = True):
    """The batched workload: 256 independent Dyck-3 instances (1k-50k vertices
    each, log-uniform).  Times the solve of all of
    them as one batch (every production of every instance in one launch
    sequence per iteration, the iterations looping inside one CUDA graph)
    against solving each alone in the plain per-production form; both after
    cflr_reset from device-resident edges."""
    import torch
    from paper_2401_11029_gb300 import cflr

    world, rank, local, dist = (1, 0, 0, None) if not print_line else dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    text = gen.grammar_text("dyck3")
    graphs = gen.dyck3_batch(count=args.instances, seed0=4000 + 100000 * rank)

    def make(form):
        out = []
        for g in graphs:
            c = cflr.cflr_create(device=local, stream=stream.cuda_stream, form=form)
            cflr.cflr_load_grammar(c, text)
            cflr.cflr_load_graph(c, g.n, g.src, label_array(c, g), g.dst)
            out.append(c)
        return out

    batched = make(cflr.CFLR_FORM_GRAPH)
    plain = make(cflr.CFLR_FORM_PLAIN)

    def timed(fn, ctxs):
        ts = []
        for k in range(args.warmup + args.steps):
            for c in ctxs:
                cflr.cflr_reset(c)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(ctxs)
            e1.record(stream)
            e1.synchronize()
            if k >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        return statistics.mean(ts)

    clocks = ClockSampler(local)
    clocks.start()
    ms_b = timed(lambda cs: cflr.cflr_solve_batch(cs), batched)
    ms_p = timed(lambda cs: [cflr.cflr_solve(c) for c in cs], plain)
    clk = clocks.stop()
    pairs = 0
    for c in batched:
        n_nt, n_named, _ = cflr.cflr_grammar_sizes(c)
        pairs += sum(cflr.cflr_get_pairs(c, x, count_only=True) for x in range(n_named))
    pairs_p = 0
    for c in plain:
        n_nt, n_named, _ = cflr.cflr_grammar_sizes(c)
        pairs_p += sum(cflr.cflr_get_pairs(c, x, count_only=True) for x in range(n_named))
    assert pairs == pairs_p
    # the batched result against the oracle's per-instance fingerprints
    parity = {"checked": False, "why": "no stored oracle fingerprints for these instances"}
    gold = golden_of("dyck3_batch_256", None) if rank == 0 and args.instances == 256 else None
    if gold:
        bad = []
        for c, g, gi in zip(batched, graphs, gold["instances"]):
            if g.edge_digest() != gi["edge_digest"]:
                bad.append((gi["seed"], "graph"))
                continue
            for x, fp in gi["pairs"].items():
                i, _ = cflr.cflr_symbol_id(c, x)
                s, d = cflr.cflr_get_pairs(c, i)
                if gen.pair_fingerprint(gen.pair_keys(s, d)) != fp:
                    bad.append((gi["seed"], x))
        parity = {"checked": True, "match": not bad, "mismatched": bad[:8],
                  "instances": len(gold["instances"]),
                  "against": "oracle fingerprints tests/golden/dyck3_batch_256.json"}
    for c in batched + plain:
        cflr.cflr_destroy(c)
    line = {"metric": "batched CFL-r solve throughput (pairs / solve time)",
            "value": pairs / (ms_b / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"dyck3 x{args.instances} (seeds 4000..)",
                       "vertices": int(sum(g.n for g in graphs)),
                       "edges": int(sum(g.n_edges for g in graphs)), "pairs": pairs,
                       "step": "cflr_solve_batch of all instances (graph form) after "
                               "cflr_reset; extraction not timed"},
            "plain_form": {"ms_per_step": ms_p, "value": pairs / (ms_p / 1e3),
                           "form": "each instance alone, one launch sequence per "
                                   "production"},
            "batched_over_plain": ms_p / ms_b, "parity": parity, "clocks": clk}
    if print_line and rank == 0:
        print(json.dumps(line), flush=True)
    return line


def _gen_request(args):
    n, seed = args
    return gen.fica_like(n=n, n_a=2 * n, n_d=(3 * n) // 4, seed=seed)


def run_serving(args, print_line: bool = True):
    """The serving workload: a Poisson stream of alias-analysis solves (sizes log-uniform
    in [5k, 300k] vertices) served with continuous batching; p50/p99 latency
    from arrival to result on the host, after a warm-up window."""
    import multiprocessing as mp
    reqs = gen.serving_stream(n_req=args.requests, rate=args.rate, seed=5)
    # graphs are made in spawned workers (a forked worker would inherit the
    # parent's CUDA state)
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        graphs = pool.map(_gen_request, [(r.n, r.seed) for r in reqs], chunksize=4)
    import torch
    from paper_2401_11029_gb300.serve import Server, summarize
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    text = gen.grammar_text("fica")
    # warm the library and the allocator on a small request
    w = Server(text, stream=stream.cuda_stream)
    w.run([(0, 0.0, _gen_request((20_000, 99)))])
    w.close()
    # size hint: pairs per input edge of the alias workload (93M pairs over
    # 1.1M edges at 200k vertices), so fresh requests rarely grow their sets
    srv = Server(text, mem_budget_bytes=args.serve_budget_gb << 30, max_active=args.max_active,
                 stream=stream.cuda_stream, size_hint=args.size_hint)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    done = srv.run([(r.rid, r.arrival_s, g) for r, g in zip(reqs, graphs)])
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    srv_time = dict(srv.time)
    summ = summarize(done, warmup_s=args.serve_warmup)
    # saturated (served below the arrival rate): the same requests again at
    # 80 % of the rate served, to report latency where the server keeps up
    sustained = None
    if summ["req_per_s"] and summ["req_per_s"] < 0.95 * args.rate:
        rate2 = 0.8 * summ["req_per_s"]
        scale = args.rate / rate2
        t1 = time.perf_counter()
        done2 = srv.run([(r.rid, r.arrival_s * scale, g) for r, g in zip(reqs, graphs)])
        wall2 = time.perf_counter() - t1
        s2 = summarize(done2, warmup_s=args.serve_warmup * scale)
        # keeping up: no queue builds, i.e. the last quarter of the requests
        # waits about as long as the first quarter
        lat = [f.latency_s for f in sorted(done2, key=lambda f: f.arrival_s)]
        q = max(1, len(lat) // 4)
        first, last = statistics.median(lat[:q]), statistics.median(lat[-q:])
        sustained = dict(s2, rate_per_s=rate2, wall_s=wall2,
                         first_quarter_median_s=first, last_quarter_median_s=last,
                         keeps_up=bool(last <= 2 * first + 0.25))
    srv.close()
    line = {"metric": "served CFL-r solves: throughput (pairs/s) with p50/p99 latency",
            "value": summ["pairs_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": len(done), "warmup": args.serve_warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals of fica_like solves",
                       "rate_per_s": args.rate, "requests": args.requests,
                       "vertices": "log-uniform [5000, 300000]",
                       "mem_budget_gb": args.serve_budget_gb, "max_active": args.max_active},
            "serving": dict(summ, wall_s=wall, warmup_s=args.serve_warmup, host_time=srv_time,
                            saturated=bool(summ["req_per_s"] and
                                           summ["req_per_s"] < 0.95 * args.rate),
                            # saturated, the rate served is the server's capacity
                            capacity_req_per_s=summ["req_per_s"]),
            "serving_below_capacity": sustained,
            "clocks": clk}
    if print_line:
        print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cflr", choices=["cflr", "reference"])
    ap.add_argument("--workload", default="all",
                    choices=["all", "fica", "fsjpt", "dyck3_batch", "serving"],
                    help="all: the alias workload's line with the other workloads as "
                         "extra keys")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--extra-requests", type=int, default=200,
                    help="requests of the serving run inside the default line")
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--serve-warmup", type=float, default=5.0)
    ap.add_argument("--serve-budget-gb", type=int, default=96)
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--size-hint", type=int, default=90)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--vertices", type=int, default=None,
                    help="scale the workload to this many vertices (same generator and "
                         "ratios; for profiling runs, not for bench lines)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "dyck3_batch":
        run_dyck3_batch(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "fsjpt":
        run_cflr(args, "fsjpt")
    else:
        run_cflr(args, "fica", extras=args.workload == "all" and args.vertices is None)


if __name__ == "__main__":
    main()
