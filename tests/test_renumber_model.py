"""The device vertex-order search, step by step, against a plain queue search.

`renumber.cu` finds the breadth-first order of the undirected edges with
level-synchronous passes: components by hooking roots under smaller ones and
pointer jumping, then one search from all roots at once in which an unseen
vertex goes to the smallest key (frontier position, list position) that
reaches it, and final positions come from per-root segment tables.  This test
runs those steps sequentially, with the atomic operations' order shuffled, and
checks that they give exactly the queue order.  It pins the algorithm; the
GPU tests (`test_gpu_renumber.py`) pin the kernels to the same order."""
import random

import numpy as np


def queue_order(n, src, dst):
    adj = [[] for _ in range(n)]
    for s, d in zip(src, dst):
        adj[s].append(d)
        adj[d].append(s)
    seen = [False] * n
    order = []
    for s in range(n):
        if seen[s]:
            continue
        seen[s] = True
        order.append(s)
        h = len(order) - 1
        while h < len(order):
            u = order[h]
            h += 1
            for v in adj[u]:
                if not seen[v]:
                    seen[v] = True
                    order.append(v)
    return order


def device_steps(n, src, dst, rng):
    m = len(src)
    # adjacency: lists of (edge << 32 | neighbour), filled in any order, sorted
    off = [0] * (n + 1)
    for s, d in zip(src, dst):
        off[s + 1] += 1
        off[d + 1] += 1
    for v in range(n):
        off[v + 1] += off[v]
    cur = off[:n]
    adj = [0] * (2 * m)
    es = list(range(m))
    rng.shuffle(es)
    for e in es:
        s, d = src[e], dst[e]
        adj[cur[s]] = (e << 32) | d
        cur[s] += 1
        adj[cur[d]] = (e << 32) | s
        cur[d] += 1
    for v in range(n):
        adj[off[v]:off[v + 1]] = sorted(adj[off[v]:off[v + 1]])
    # components: compress, then hook the larger root under the smaller
    parent = list(range(n))
    for _ in range(128):
        more = False
        for v in rng.sample(range(n), n):
            x = parent[v]
            while parent[x] != x:
                x = parent[x]
            parent[v] = x
        for e in rng.sample(range(m), m):
            ru, rv = parent[src[e]], parent[dst[e]]
            if ru != rv:
                hi, lo = max(ru, rv), min(ru, rv)
                parent[hi] = min(parent[hi], lo)
                more = True
        if not more:
            break
    else:
        raise AssertionError("components did not settle")
    cnt = [0] * n
    for v in range(n):
        cnt[parent[v]] += 1
    comp_off, acc = [0] * n, 0
    for v in range(n):
        comp_off[v] = acc
        acc += cnt[v]
    # level 0: the roots in id order
    unseen = -1
    lvl, key = [unseen] * n, [None] * n
    perm, iperm = [None] * n, [None] * n
    sf, se, pc = [[0] * n, [0] * n], [[0] * n, [0] * n], [[0] * n, [0] * n]
    F = [v for v in range(n) if parent[v] == v]
    for q, v in enumerate(F):
        lvl[v] = 0
        sf[0][v], se[0][v], pc[0][v] = q, q + 1, 0
        iperm[comp_off[v]] = v
        perm[v] = comp_off[v]
    b, level, placed = 0, 0, 0
    while F:
        placed += len(F)
        for q in rng.sample(range(len(F)), len(F)):            # claims
            u = F[q]
            for j in range(off[u], off[u + 1]):
                v = adj[j] & 0xFFFFFFFF
                if lvl[v] == unseen:
                    k = (q << 32) | (j - off[u])
                    key[v] = k if key[v] is None else min(key[v], k)
        won = [sum(1 for j in range(off[u], off[u + 1])
                   if lvl[adj[j] & 0xFFFFFFFF] == unseen
                   and key[adj[j] & 0xFFFFFFFF] == ((q << 32) | (j - off[u])))
               for q, u in enumerate(F)]
        woff = [0] * (len(F) + 1)
        for q in range(len(F)):
            woff[q + 1] = woff[q] + won[q]
        F2 = [None] * woff[-1]
        for q in rng.sample(range(len(F)), len(F)):            # writes
            u = F[q]
            r = parent[u]
            s0, s1 = sf[b][r], se[b][r]
            if q == s0:
                sf[b ^ 1][r], se[b ^ 1][r] = woff[s0], woff[s1]
                pc[b ^ 1][r] = pc[b][r] + (s1 - s0)
            pos0 = comp_off[r] + pc[b][r] + (s1 - s0)
            t = woff[q]
            for j in range(off[u], off[u + 1]):
                v = adj[j] & 0xFFFFFFFF
                if lvl[v] == unseen and key[v] == ((q << 32) | (j - off[u])):
                    F2[t] = v
                    lvl[v] = level + 1
                    iperm[pos0 + t - woff[s0]] = v
                    perm[v] = pos0 + t - woff[s0]
                    t += 1
        F, b, level = F2, b ^ 1, level + 1
    assert placed == n
    assert all(perm[iperm[k]] == k for k in range(n))
    return iperm


def test_random_graphs_self_loops_and_repeated_edges():
    rng = random.Random(5)
    for trial in range(150):
        n = rng.randint(1, 50)
        m = rng.randint(0, 80)
        src = [rng.randrange(n) for _ in range(m)]
        dst = [rng.randrange(n) for _ in range(m)]
        if trial % 3 == 0:
            for _ in range(4):
                v = rng.randrange(n)
                src.append(v)
                dst.append(v)
            src += src[:4]
            dst += dst[:4]
        assert device_steps(n, src, dst, rng) == queue_order(n, src, dst), trial


def test_path_numbered_backwards_and_star():
    rng = random.Random(6)
    n = 600
    src = list(range(n - 1, 0, -1))
    dst = [v - 1 for v in src]
    assert device_steps(n, src, dst, rng) == queue_order(n, src, dst)
    # a hub with edges in a mixed order, plus leaves chained to each other
    src = [0] * 200 + list(range(1, 200))
    dst = list(range(1, 201)) + list(range(2, 201))
    p = np.random.default_rng(7).permutation(len(src))
    src = [src[i] for i in p]
    dst = [dst[i] for i in p]
    assert device_steps(250, src, dst, rng) == queue_order(250, src, dst)
