"""Autotuner for the run-time knobs of libsignedbal (sb_set_tuning).

It times the candidate values on the loaded graph with the library's own
CUDA-event profiler and keeps the fastest per knob:
  bfs_words        64-tree words grown per BFS launch (trees per launch / 64)
  bfs_group        lanes sharing one vertex in the BFS (the words, or twice that)
  score_blocks_sm  blocks per SM of the frustration scorer
  gl_lanes         graphL lanes per row segment (8 -> 32 columns, 16 -> 64, 32 -> 128)
Choices are cached in JSON per (GPU name, graph shape bucket, K, R), so a
later run on the same kind of graph skips the timing.  Results never depend on
the knobs; only speed does.
"""
from __future__ import annotations

import json
import math
import os

import torch

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _bucket(n: int, m: int) -> str:
    return f"n2^{int(math.log2(max(n, 2)))}_m2^{int(math.log2(max(m, 2)))}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time_family(sb, fam: str, fn, reps: int) -> float:
    fn()  # warm-up
    torch.cuda.synchronize()
    sb.profile_read()
    sb.profile(True)
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    sb.profile(False)
    return sb.profile_read()[fam][0] / reps


def tune(sb, K: int = 1024, R: int | None = None, seed: int = 987654321, reps: int = 2, use_cache: bool = True):
    """Picks the knobs for sampling K trees (and graphL with R start points)
    on the graph loaded in `sb`; returns the chosen values (also applied)."""
    key = f"{torch.cuda.get_device_name(sb.device)}|{_bucket(sb.n, sb.m)}|K{K}|R{R}"
    cache = _load() if use_cache else {}
    if key in cache:
        sb.set_tuning(**cache[key])
        return dict(cache[key], cached=True)
    words = max(1, (K + 63) // 64)
    chosen = {}
    # words per BFS launch
    cands = sorted({w for w in (4, 8, 16, 32) if w <= words} | {min(words, 32)})
    t0 = 0

    def sample():
        nonlocal t0
        sb.sample_trees(seed, t0, K)
        t0 += K

    best = None
    for w in cands:
        sb.set_tuning(bfs_words=w)
        t = _time_family(sb, "bfs", sample, reps)
        if best is None or t < best[0]:
            best = (t, w)
    chosen["bfs_words"] = best[1]
    sb.set_tuning(bfs_words=best[1])

    # lanes per vertex group (at least the words of a launch)
    g0 = 1
    while g0 < best[1]:
        g0 <<= 1
    best = None
    for g in sorted({g0, min(32, 2 * g0)}):  # the library widens a group at most twofold
        sb.set_tuning(bfs_group=g)
        t = _time_family(sb, "bfs", sample, reps)
        if best is None or t < best[0]:
            best = (t, g)
    chosen["bfs_group"] = best[1]
    sb.set_tuning(bfs_group=best[1])

    # scorer blocks per SM (the scorer runs once per sampled batch)
    def score():
        sample()
        sb.frustration()

    best = None
    for b in (2, 3, 4, 0):
        sb.set_tuning(score_blocks_sm=b)
        t = _time_family(sb, "score", score, reps)
        if best is None or t < best[0]:
            best = (t, b)
    chosen["score_blocks_sm"] = best[1]
    sb.set_tuning(score_blocks_sm=best[1])

    # graphL segment width
    if R:
        gen = torch.Generator(device="cpu").manual_seed(1)
        g0 = (torch.rand((sb.n, R), generator=gen) * 2 - 1).to(sb.device)
        grad_out = torch.ones(sb._per_graph() * R, device=sb.device)  # G x R in a batch
        best = None
        for lanes in ((8, 16, 32) if R % 4 == 0 else (8,)):
            sb.set_tuning(gl_lanes=lanes)
            t = _time_family(sb, "gl_rows", lambda: sb.graphL_bwd(g0, grad_out), reps)
            if best is None or t < best[0]:
                best = (t, lanes)
        chosen["gl_lanes"] = best[1]
        sb.set_tuning(gl_lanes=best[1])
    if use_cache:
        cache = _load()
        cache[key] = chosen
        _save(cache)
    return dict(chosen, cached=False)
