"""Continuous-batching CFL-reachability server over the C ABI.

Requests (a graph each, all under one grammar) arrive over time.  The
server keeps every admitted request's matrices resident on the GPU and
advances all of them together: a tick runs closure iterations of
Algorithm 1 for every unfinished request as one batched launch sequence
per iteration (inside one CUDA graph), until some request reaches its
fixpoint or the tick's iteration cap is hit (cflr_solve_batch led by a
context with stop_on_first_converged).  Between ticks the server retires
the finished requests (their pairs are copied out and their device memory
freed) and admits the requests that are loaded.  Loading (a context, the
grammar, the graph's upload and renumbering, the terminal initialisation)
runs on a second host thread, on each context's own stream, while ticks run:
a request is taken for loading once it has arrived and its estimated device
footprint fits the memory budget next to the requests in flight.  A
request's result is the same whether it is solved alone or in the mix: the
batch only interleaves independent fixpoints.

This module only schedules; all CFL-r work runs in libcflr.so.
"""
from __future__ import annotations

import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import cflr


@dataclass
class Finished:
    rid: int
    n: int
    edges: int
    pairs: int
    iterations: int
    arrival_s: float
    admitted_s: float
    done_s: float
    keys: dict = field(default_factory=dict)   # non-terminal -> sorted uint64 keys

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


class Server:
    """Admission by device-memory footprint, resident state, one batched
    closure iteration per tick."""

    # device bytes per input edge and per vertex-nonterminal, measured on the
    # alias-analysis workload (peak bytes / edges of a 200k-vertex solve),
    # used to admit requests before their closure size is known
    BYTES_PER_EDGE = 8192
    BYTES_PER_VERTEX_NT = 40

    def __init__(self, grammar_text: str, mem_budget_bytes: int = 64 << 30,
                 max_active: int = 128, device: int = 0, stream=None,
                 keep_pairs: bool = False, form: int = cflr.CFLR_FORM_GRAPH,
                 tick_iterations: int = 16, size_hint: int = 0):
        self.text = grammar_text
        self.budget = int(mem_budget_bytes)
        self.max_active = max_active
        self.device = device
        self.stream = stream
        self.keep_pairs = keep_pairs
        self.form = form
        self.size_hint = size_hint
        # the leader holds the shared work buffers and the tick's iteration
        # limit; its own (empty) graph is solved at once, so it never does work
        self.leader = cflr.cflr_create(device=device, stream=stream,
                                       max_iterations=tick_iterations,
                                       stop_on_first_converged=1, form=form)
        cflr.cflr_load_grammar(self.leader, grammar_text)
        cflr.cflr_load_graph(self.leader, 1, [], [], [])
        cflr.cflr_solve(self.leader)
        self.n_nt, self.n_named, _ = cflr.cflr_grammar_sizes(self.leader)
        self.term = {}
        self.time = {"admit_s": 0.0, "tick_s": 0.0, "retire_s": 0.0, "ticks": 0, "regrows": 0,
                     "regrow_buffers": 0, "regrow_sets": 0, "regrow_pools": 0}

    def close(self):
        cflr.cflr_destroy(self.leader)
        self.leader = None

    def footprint(self, graph) -> int:
        return (self.BYTES_PER_EDGE * graph.n_edges +
                self.BYTES_PER_VERTEX_NT * graph.n * self.n_nt + (32 << 20))

    def _label_ids(self, ctx, labels):
        out = []
        for name in labels:
            if name not in self.term:
                try:
                    i, is_t = cflr.cflr_symbol_id(ctx, name)
                    self.term[name] = i if is_t else 0xFFFFFFFF
                except cflr.CflrError:
                    self.term[name] = 0xFFFFFFFF
            out.append(self.term[name])
        return np.asarray(out, dtype=np.uint32)

    def _admit(self, graph):
        # a private stream: the load overlaps the tick running on the
        # leader's stream (the load ends synchronised with the host)
        ctx = cflr.cflr_create(device=self.device, form=self.form, size_hint=self.size_hint)
        cflr.cflr_load_grammar(ctx, self.text)
        ids = self._label_ids(ctx, graph.labels)
        cflr.cflr_load_graph(ctx, graph.n, graph.src, ids[graph.lab], graph.dst)
        return ctx

    def _retire(self, ctx, rec) -> dict:
        keys = {}
        total = 0
        for x in range(self.n_named):
            if self.keep_pairs:
                s, d = cflr.cflr_get_pairs(ctx, x)
                keys[x] = (s.astype(np.uint64) << np.uint64(32)) | d.astype(np.uint64)
                total += s.size
            else:
                total += cflr.cflr_get_pairs(ctx, x, count_only=True)
        cflr.cflr_destroy(ctx)
        return total, keys

    def run(self, requests, clock=time.perf_counter) -> list:
        """Serve ``requests``: an iterable of (rid, arrival_s, graph), sorted
        by arrival.  Returns a list of ``Finished``."""
        requests = list(requests)
        ready = queue.Queue()       # loaded requests waiting for the next tick
        cond = threading.Condition()
        inflight = {"used": 0, "n": 0}     # footprint and count being loaded or solved
        failure = []
        t0 = clock()

        def loader():
            try:
                for rid, arr, g in requests:
                    wait = arr - (clock() - t0)
                    if wait > 0:
                        time.sleep(wait)
                    fp = self.footprint(g)
                    with cond:
                        # room: a slot, and the footprint within the budget
                        # (a request alone is always taken)
                        while inflight["n"] and (inflight["n"] >= self.max_active or
                                                 inflight["used"] + fp > self.budget):
                            cond.wait()
                        inflight["used"] += fp
                        inflight["n"] += 1
                    ta = clock()
                    ctx = self._admit(g)
                    self.time["admit_s"] += clock() - ta
                    ready.put([ctx, rid, g, arr, clock() - t0, fp, 0])
            except BaseException as exc:        # handed to the serving thread
                failure.append(exc)
                ready.put(None)

        th = threading.Thread(target=loader, name="cflr-loader", daemon=True)
        th.start()
        active = []          # [ctx, rid, graph, arrival, admitted, footprint, iterations]
        done = []
        try:
            while len(done) < len(requests):
                # admit what is loaded; wait for the loader when idle
                block = not active
                while True:
                    try:
                        item = ready.get(block=block, timeout=0.05 if block else None)
                    except queue.Empty:
                        break
                    if item is None:
                        raise failure[0]
                    item[4] = clock() - t0
                    active.append(item)
                    block = False
                if not active:
                    continue
                tt = clock()
                stats = cflr.cflr_solve_batch([self.leader] + [a[0] for a in active],
                                              allow_limit=True)
                self.time["tick_s"] += clock() - tt
                self.time["ticks"] += 1
                still = []
                for k in ("regrows", "regrow_buffers", "regrow_sets", "regrow_pools"):
                    self.time[k] += stats[0][k]
                for a, st in zip(active, stats[1:]):
                    a[6] = st["iterations"]
                    if st["converged"]:
                        tr = clock()
                        pairs, keys = self._retire(a[0], a)
                        self.time["retire_s"] += clock() - tr
                        with cond:
                            inflight["used"] -= a[5]
                            inflight["n"] -= 1
                            cond.notify()
                        done.append(Finished(rid=a[1], n=a[2].n, edges=a[2].n_edges,
                                             pairs=pairs, iterations=a[6], arrival_s=a[3],
                                             admitted_s=a[4], done_s=clock() - t0, keys=keys))
                    else:
                        still.append(a)
                active = still
        finally:
            th.join(timeout=60)
        return done


def summarize(done: list, warmup_s: float = 0.0) -> dict:
    """Latency percentiles and throughput of the requests that arrived after
    ``warmup_s``."""
    kept = [f for f in done if f.arrival_s >= warmup_s] or done
    lat = np.asarray([f.latency_s for f in kept])
    span = max(f.done_s for f in kept) - min(f.arrival_s for f in kept)
    return {"requests": len(kept), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "req_per_s": len(kept) / span if span > 0 else None,
            "pairs_per_s": sum(f.pairs for f in kept) / span if span > 0 else None}
