"""Benchmark: CFL-reachability solve throughput on one GB300 (pairs/s).

One step is one pass of the whole hot path on the alias-analysis workload
(Fig. "wcnf:fica" grammar, 200 000-vertex program-shaped graph with 400 000
'a' and 150 000 'd' edges plus their reverses):
  terminal initialisation from the device-resident edges (cflr_reset),
  the semi-naive closure loop to its fixpoint (cflr_solve),
  and the extraction of every non-terminal's sorted pairs into device
  buffers (cflr_get_pairs_device).
value = pairs of all named non-terminals / step time (CUDA events on the
solve stream, L2 flushed between steps).  e2e repeats the step through the
host-buffer API: grammar text and host edges in, host pair arrays out.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cflr|reference]

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
SAMPLE_N = 20_000     # oracle sample: same generator and ratios, 1/10 of the vertices
TUNING_CACHE = os.path.join(ROOT, "paper_2401_11029_gb300", "tuning", "gb300.txt")


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": float(p["hbm_gbs"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback"}


FSJPT = {"workload": "fsjpt_like field-sensitive points-to (Fig. wcnf:fsjpt, 64 fields)",
         "n_vertices": 500_000, "forward_edges": 2_000_000, "reverse_edges": True, "seed": 3,
         "productions": 514}


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


def traffic_from_profile(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if
    the kernel source has not changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_fica_like.md")
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


def cpu_oracle_sample(seed: int, kind: str = "fica") -> dict:
    """The oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    g = workload_graph(seed, SAMPLE_N, kind)
    text = grammar_of(kind)
    res = oracle.solve(text, g)
    pairs = res.total()
    name = "fsjpt_like" if kind == "fsjpt" else "fica_like"
    return {"value": pairs / res.seconds, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{name} n={SAMPLE_N} (same generator and ratios as the workload, "
                      f"{g.n_edges} edges, {pairs} pairs), one worklist solve, "
                      f"{res.seconds:.1f} s on 1 host core", "seconds": res.seconds}


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
    world, rank, local, dist = dist_setup()
    if rank != 0:
        return
    vals, secs = [], []
    info = None
    for _ in range(args.warmup):
        cpu_oracle_sample(WORKLOAD["seed"])
    for _ in range(args.steps):
        info = cpu_oracle_sample(WORKLOAD["seed"])
        vals.append(info["value"])
        secs.append(info.pop("seconds"))
    v = statistics.mean(vals)
    info["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # one step is one oracle solve of the bounded sample
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism=f"replicas{args.gpus}"),
            "cpu_baseline": info,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cflr(args):
    import torch
    from paper_2401_11029_gb300 import cflr

    world, rank, local, dist = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    kind = args.workload
    wl = FSJPT if kind == "fsjpt" else WORKLOAD
    seed = wl["seed"] + 1000 * rank
    g = workload_graph(seed, args.vertices, kind)
    text = grammar_of(kind)

    # timed context: the device-driven loop (one CUDA graph per solve), with
    # the product schedule picked by cflr_autotune (cached per grammar and size)
    ctx = cflr.cflr_create(device=local, stream=stream.cuda_stream, form=cflr.CFLR_FORM_GRAPH,
                           autotune_cache=TUNING_CACHE.encode())
    cflr.cflr_load_grammar(ctx, text)
    n_nt, n_named, _ = cflr.cflr_grammar_sizes(ctx)
    term = {}
    for name in g.labels:
        try:
            i, is_t = cflr.cflr_symbol_id(ctx, name)
            term[name] = i if is_t else 0xFFFFFFFF
        except cflr.CflrError:
            term[name] = 0xFFFFFFFF
    lab = np.asarray([term[x] for x in g.labels], np.uint32)[g.lab]
    # pinned host copies of the inputs for the end-to-end leg
    h_src = torch.from_numpy(g.src.astype(np.uint32).view(np.int32)).pin_memory()
    h_lab = torch.from_numpy(lab.view(np.int32)).pin_memory()
    h_dst = torch.from_numpy(g.dst.astype(np.uint32).view(np.int32)).pin_memory()
    cflr.cflr_load_graph(ctx, g.n, h_src.numpy().view(np.uint32), h_lab.numpy().view(np.uint32),
                         h_dst.numpy().view(np.uint32))
    tuning = cflr.cflr_autotune(ctx) if not args.no_autotune else cflr.cflr_get_tuning(ctx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # profiled context: the same iterations launched one by one from the host
    # with CUDA events around every kernel (events cannot sit inside the
    # graph's loop body); it supplies the per-kernel times of the roofline
    pctx = cflr.cflr_create(device=local, stream=stream.cuda_stream,
                            form=cflr.CFLR_FORM_BATCHED, profile=1)
    cflr.cflr_load_grammar(pctx, text)
    cflr.cflr_set_tuning(pctx, tuning["probe_ratio"], tuning["bin_limit"], tuning["ctas_per_sm"])
    cflr.cflr_load_graph(pctx, g.n, h_src.numpy().view(np.uint32), h_lab.numpy().view(np.uint32),
                         h_dst.numpy().view(np.uint32))

    last = {}

    def device_step(out=None, c=None):
        c = c or ctx
        cflr.cflr_reset(c)
        last.update(cflr.cflr_solve(c))
        total = 0
        for x in range(n_named):
            cnt = cflr.cflr_get_pairs(c, x, count_only=True)
            if cnt and out is not None:
                cflr.cflr_get_pairs_device(c, x, out[0].data_ptr(), out[1].data_ptr(), cnt)
            total += cnt
        return total

    pairs = device_step()
    cap = max(cflr.cflr_get_pairs(ctx, x, count_only=True) for x in range(n_named))
    out = (torch.empty(cap, dtype=torch.int32, device=dev),
           torch.empty(cap, dtype=torch.int32, device=dev))
    for _ in range(max(0, args.warmup - 1)):
        device_step(out)

    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(rank + 1)                      # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p = device_step(out)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        assert p == pairs, "pair count changed between steps"
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    solve_stats = dict(last)

    # per-kernel event times: the same steps on the profiled context
    for _ in range(args.warmup):
        device_step(out, pctx)
    before = {k["name"]: k for k in cflr.cflr_kernel_stats(pctx)}
    for _ in range(args.steps):
        flush.fill_(rank + 1)
        assert device_step(out, pctx) == pairs
    torch.cuda.synchronize(dev)
    after = {k["name"]: k for k in cflr.cflr_kernel_stats(pctx)}
    cflr.cflr_destroy(pctx)

    # end-to-end through the host-buffer API
    h_out_s = torch.empty(cap, dtype=torch.int32).pin_memory()
    h_out_d = torch.empty(cap, dtype=torch.int32).pin_memory()
    e2e_s = []
    for k in range(args.steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        c2 = cflr.cflr_create(device=local, stream=stream.cuda_stream,
                              form=cflr.CFLR_FORM_GRAPH, autotune_cache=TUNING_CACHE.encode())
        cflr.cflr_load_grammar(c2, text)
        cflr.cflr_load_graph(c2, g.n, h_src.numpy().view(np.uint32),
                             h_lab.numpy().view(np.uint32), h_dst.numpy().view(np.uint32))
        if not args.no_autotune:
            cflr.cflr_autotune(c2)          # the cached schedule of this workload
        cflr.cflr_solve(c2)
        tot = 0
        lib = cflr.load_library()
        import ctypes
        for x in range(n_named):
            n_p = ctypes.c_uint64()
            rc = lib.cflr_get_pairs(c2, x, h_out_s.data_ptr(), h_out_d.data_ptr(), cap,
                                    ctypes.byref(n_p))
            assert rc == 0
            tot += n_p.value
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        cflr.cflr_destroy(c2)
        if k > 0:                                   # first call warms the allocator
            e2e_s.append(dt)
        assert tot == pairs

    ms = statistics.mean(step_ms)
    ms_all, pairs_all, e2e_all = aggregate(dist, dev, ms, pairs, statistics.mean(e2e_s))

    # roofline of the dominant kernel over the timed steps
    rows = []
    for name, a in after.items():
        b = before.get(name, {"launches": 0, "ms": 0.0, "alg_bytes": 0})
        rows.append((a["ms"] - b["ms"], a["launches"] - b["launches"],
                     a["alg_bytes"] - b["alg_bytes"], name))
    rows.sort(reverse=True)
    kms, kl, kb, kname = rows[0]
    pk = peaks()
    achieved = (kb / 1e9) / (kms / 1e3) if kms > 0 else 0.0
    traffic = traffic_from_profile(kname)
    launches = sum(r[1] for r in rows) + args.steps * n_named * 6   # + extraction kernels
    if rank != 0:
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
                "d2h_bytes_per_step": int(8 * pairs)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     "traffic": traffic, "kernel": kname,
                     "launches": kl, "avg_launch_ms": kms / max(kl, 1),
                     "peak_src": pk["src"]},
        "kernels": [{"name": r[3], "ms": round(r[0], 4), "launches": r[1],
                     "gbs": round((r[2] / 1e9) / (r[0] / 1e3), 1) if r[0] > 0 else None}
                    for r in rows if r[1]],
        "clocks": clk,
        "tuning": tuning,
        "solve": {"form": "graph", "iterations": solve_stats["iterations"],
                  "groups_per_bin": solve_stats["groups"],
                  "flops": solve_stats["flops"], "candidates": solve_stats["candidates"],
                  "peak_device_bytes": solve_stats["peak_device_bytes"]},
        "roofline_note": "kernel times from the same steps replayed with per-kernel CUDA "
                         "events (host-launched iterations) right after the timed region",
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(wl["seed"], kind)
        line["cpu_baseline"].pop("seconds")
    print(json.dumps(line), flush=True)
    cflr.cflr_destroy(ctx)


def run_dyck3_batch(args):
    """The batched workload: 256 independent Dyck-3 instances (1k-50k vertices
    each, log-uniform).  Times the solve of all of
    them as one batch (every production of every instance in one launch
    sequence per iteration, the iterations looping inside one CUDA graph)
    against solving each alone in the plain per-production form; both after
    cflr_reset from device-resident edges."""
    import torch
    from paper_2401_11029_gb300 import cflr

    world, rank, local, dist = dist_setup()
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
            ids = {}
            for name in g.labels:
                i, _ = cflr.cflr_symbol_id(c, name)
                ids[name] = i
            lab = np.asarray([ids[x] for x in g.labels], np.uint32)[g.lab]
            cflr.cflr_load_graph(c, g.n, g.src, lab, g.dst)
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

    ms_b = timed(lambda cs: cflr.cflr_solve_batch(cs), batched)
    ms_p = timed(lambda cs: [cflr.cflr_solve(c) for c in cs], plain)
    named = None
    pairs = 0
    for c in batched:
        n_nt, n_named, _ = cflr.cflr_grammar_sizes(c)
        pairs += sum(cflr.cflr_get_pairs(c, x, count_only=True) for x in range(n_named))
    pairs_p = 0
    for c in plain:
        n_nt, n_named, _ = cflr.cflr_grammar_sizes(c)
        pairs_p += sum(cflr.cflr_get_pairs(c, x, count_only=True) for x in range(n_named))
    assert pairs == pairs_p
    if rank == 0:
        line = {"metric": "batched CFL-r solve throughput (pairs / solve time)",
                "value": pairs / (ms_b / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic",
                "config": {"workload": f"dyck3 x{args.instances} (seeds 4000..)",
                           "vertices": int(sum(g.n for g in graphs)),
                           "edges": int(sum(g.n_edges for g in graphs)), "pairs": pairs},
                "plain_form": {"ms_per_step": ms_p, "value": pairs / (ms_p / 1e3),
                               "form": "each instance alone, one launch sequence per "
                                       "production"},
                "batched_over_plain": ms_p / ms_b}
        print(json.dumps(line), flush=True)
    for c in batched + plain:
        cflr.cflr_destroy(c)


def _gen_request(args):
    n, seed = args
    return gen.fica_like(n=n, n_a=2 * n, n_d=(3 * n) // 4, seed=seed)


def run_serving(args):
    """The serving workload: a Poisson stream of alias-analysis solves (sizes log-uniform
    in [5k, 300k] vertices) served with continuous batching; p50/p99 latency
    from arrival to result on the host, after a warm-up window."""
    import multiprocessing as mp
    reqs = gen.serving_stream(n_req=args.requests, rate=args.rate, seed=5)
    # graphs are made before the first GPU call, in spawned workers
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        graphs = pool.map(_gen_request, [(r.n, r.seed) for r in reqs], chunksize=4)
    import torch
    from paper_2401_11029_gb300 import cflr
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
    srv.close()
    summ = summarize(done, warmup_s=args.serve_warmup)
    line = {"metric": "served CFL-r solves: throughput (pairs/s) with p50/p99 latency",
            "value": summ["pairs_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": len(done), "warmup": args.serve_warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals of fica_like solves",
                       "rate_per_s": args.rate, "requests": args.requests,
                       "vertices": "log-uniform [5000, 300000]",
                       "mem_budget_gb": args.serve_budget_gb, "max_active": args.max_active},
            "serving": dict(summ, wall_s=wall, warmup_s=args.serve_warmup, host_time=srv_time),
            "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cflr", choices=["cflr", "reference"])
    ap.add_argument("--workload", default="fica",
                    choices=["fica", "fsjpt", "dyck3_batch", "serving"])
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--requests", type=int, default=1000)
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
    else:
        run_cflr(args)


if __name__ == "__main__":
    main()
