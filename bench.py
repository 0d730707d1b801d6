#!/usr/bin/env python3
"""graphBpp / graphL benchmark on GB300 (one JSON line on rank 0).

Workload (N=1): the 2^20-vertex R-MAT signed graph (a,b,c,d = 0.57, 0.19,
0.19, 0.05; 2^24 distinct undirected edges; planted two-faction balance with
10% iid sign flips; largest connected component), K = 1024 randomized-BFS
trees per step in one batched launch (16 words of 64 trees).  One step is the
whole graphBpp hot path on one batch: tree sampling + parity labels + state
hash (sb_sample_trees), frustration counts (sb_frustration) and cloud
insertion (sb_cloud).  Ingest is done once, outside the timed region (it is
timed inside the e2e leg).  Metric: edge-evals/s = trees x |E| / s.

Also reported: the plain path (one tree per launch) on the same GPU, graphL
steps/s (R = 256 start points on the same graph), the end-to-end number
through the C ABI with host buffers, the roofline of the dominant kernel and
the CPU oracle on the host cores.

--impl reference times the CPU oracle (plain C, all host cores through a
thread pool) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "graphBpp edge-evals/s (trees x |E| / s), batched"
UNIT = "edge-evals/s"
WORKLOAD = "rmat20_2faction_K1024"
TREES = 1024
SEED = 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale (default 20; 24 for --leg scale24)")
    ap.add_argument("--edges-log2", type=int, default=None, help="log2 of the edge count (default 24; 27)")
    ap.add_argument("--no-extras", action="store_true", help="skip the plain / graphL / e2e / cpu legs")
    ap.add_argument("--leg", default="bpp", choices=["bpp", "graphl", "batch", "scale24", "quality", "kruskal"],
                    help="bpp: the graphBpp line (default); graphl: graphL descent only; batch: uneven batch; "
                         "scale24: R-MAT 2^24 vertices / 2^27 edges, 4096 trees per step; "
                         "quality: graphBpp min S and graphL min F against the planted state; "
                         "kruskal: graphBpp with randomized Kruskal trees instead of BFS trees")
    ap.add_argument("--R", type=int, default=256, help="graphL start points (--leg graphl)")
    ap.add_argument("--gl-steps", type=int, default=500, help="graphL descent steps (--leg graphl)")
    ap.add_argument("--graphs", type=int, default=4096, help="graphs in the uneven batch (--leg batch)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tuning knobs")
    ap.add_argument("--gl-lanes", type=int, default=0, help="graphL lanes per row segment (8 or 32; with --no-tune)")
    args = ap.parse_args()
    big = args.leg == "scale24"
    args.scale = args.scale if args.scale is not None else (24 if big else 20)
    args.edges_log2 = args.edges_log2 if args.edges_log2 is not None else (27 if big else 24)
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    import synth

    n, u, v, s = synth.rmat_two_faction(scale=args.scale, m_target=1 << args.edges_log2)
    return n, u, v, s


def config_dict(args, n_clean, m_clean, world):
    return {
        "workload": WORKLOAD if (args.scale, args.edges_log2) == (20, 24) else f"rmat{args.scale}_e{args.edges_log2}",
        "graph": f"R-MAT scale {args.scale}, 2^{args.edges_log2} undirected edges, two factions + 10% sign noise, LCC",
        "n": n_clean,
        "m": m_clean,
        "trees_per_step": TREES,
        "words_per_launch": TREES // 64,
        "l2": "inputs larger than L2 (CSR 2m x 4 B plus labels and BFS state exceed 129 MB)",
        "parallelism": f"tree ranges sharded over {world} ranks" if world > 1 else "single-gpu",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        import threading

        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.reader = threading.Thread(target=lambda: self.lines.extend(self.proc.stdout), daemon=True)
        self.reader.start()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.reader.join(timeout=5)
        sms, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in list(self.lines):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sms.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


# ------------------------------------------------------------ CPU oracle
def oracle_graph(n, u, v, s):
    import oracle as O

    return O.clean_graph(n, u, v, s)


def oracle_trees(g, t0, count, cores):
    """Samples `count` trees with the oracle on `cores` threads; returns seconds."""
    import oracle as O

    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda i: O.sample(g, SEED, t0 + i, 1, want_labels=False), range(count)))
    return time.perf_counter() - t


def cpu_baseline(g, budget_s=12.0, single_budget_s=3.0):
    cores = os.cpu_count() or 1
    done, el = 0, 0.0
    while el < budget_s:
        el += oracle_trees(g, 10_000_000 + done, cores, cores)
        done += cores
    one, el1 = 0, 0.0
    while el1 < single_budget_s:
        el1 += oracle_trees(g, 20_000_000 + one, 1, 1)
        one += 1
    return {"value": done * g.m / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} trees (BFS tree, labels, count, hash) of the same graph, {cores} threads, {el:.1f} s",
            "single_thread": {"value": one * g.m / el1, "unit": UNIT, "cores": 1,
                              "sample": f"{one} trees on one thread, {el1:.1f} s"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n, u, v, s = workload(args)
    g = oracle_graph(n, u, v, s)
    cores = os.cpu_count() or 1
    per_step = cores
    for i in range(args.warmup):
        oracle_trees(g, i * per_step, per_step, cores)
    el = 0.0
    for i in range(args.steps):
        el += oracle_trees(g, (args.warmup + i) * per_step, per_step, cores)
    value = args.steps * per_step * g.m / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_dict(args, g.n, g.m, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} trees per step ({cores} threads), the same graph"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- ours
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg == "batch":
        import synth

        t = time.perf_counter()  # the process pool starts before any CUDA call
        args.batch_graphs = list(synth.uneven_batch(count=args.graphs, workers=os.cpu_count() or 1))
        args.batch_gen_s = time.perf_counter() - t
    if args.leg == "scale24":
        import synth

        t = time.perf_counter()
        args.scale_graph = synth.rmat_three_faction(scale=args.scale, m_target=1 << args.edges_log2,
                                                    workers=os.cpu_count() or 1)
        args.scale_gen_s = time.perf_counter() - t
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2311_00869_gb300 as P

    if args.leg == "batch":
        return batch_leg(args, P)
    if args.leg == "scale24":
        return scale_leg(args, P)
    if args.leg == "quality":
        return quality_leg(args, P)
    if args.leg == "kruskal":
        return kruskal_leg(args, P)
    n, u, v, s = workload(args)
    stream = torch.cuda.current_stream()
    sb = P.SignedBal(local, stream=stream)
    n1, m1, _ = sb.load_graph(n, u, v, s)
    if args.leg == "graphl":
        tuned = {"default": True}
        if not args.no_tune:
            from paper_2311_00869_gb300 import autotune

            tuned = autotune.tune(sb, K=TREES, R=args.R)
        elif args.gl_lanes:
            sb.set_tuning(gl_lanes=args.gl_lanes)
            tuned = {"gl_lanes": args.gl_lanes}
        res = graphl_leg(P, sb, n1, m1, R=args.R, steps=args.gl_steps, plain_inits=4)
        res["tuning"] = tuned
        line = {"leg": "graphl", "metric": "graphL steps/s", "value": res["graphl_steps_per_s"], "unit": "steps/s",
                "n_gpus": 1, "steps": args.gl_steps, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "config": config_dict(args, n1, m1, 1), "extras": res}
        print(json.dumps(line), flush=True)
        sb.close()
        return 0
    tuned = {"default": True}
    if not args.no_tune:
        try:
            from paper_2311_00869_gb300 import autotune

            tuned = autotune.tune(sb, K=TREES)
        except Exception as e:  # tuning only changes speed
            tuned = {"error": repr(e)}
    steps_total = args.warmup + args.steps
    sb.cloud_reset(max_states=(steps_total + 2) * TREES + 64)
    counts = torch.empty(TREES, dtype=torch.int32, device="cuda")
    hashes = torch.empty(TREES, dtype=torch.int64, device="cuda")

    # trees are independent: rank r takes its own tree ranges (weak scaling)
    def step(i):
        t0 = ((i * world) + rank) * TREES
        sb.sample_trees(SEED, t0, TREES)
        sb.frustration(counts, hashes)
        return sb.cloud_insert()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    sb.profile_read()
    sb.profile(True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    sb.profile(False)
    prof = sb.profile_read()
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = world * TREES * m1 / (ms_step / 1000.0)
    launches = sum(c for _, c in prof.values())

    cl, fr_min = sb.cloud()
    extras = {"fr_min": int(fr_min), "distinct_states": int(cl["S"].shape[0]), "tuning": tuned,
              "bfs_stats": sb.stats(), "trees_per_s": world * TREES / (ms_step / 1000.0)}
    if dist:  # host-side merge of the rank clouds, after the timed region
        from paper_2311_00869_gb300 import shard

        merged = shard.gather_cloud(cl)
        extras["distinct_states_all_ranks"] = int(merged["S"].shape[0])
        extras["fr_min_all_ranks"] = int(merged["S"].min()) if merged["S"].size else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": config_dict(args, n1, m1, world),
        "gpu_launches": launches, "clocks": clk,
        "stages_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]},
    }
    line["roofline"] = roofline(prof, n1, m1, TREES, extras["bfs_stats"], (clk or {}).get("sm_mhz"))
    extras["roofline_score"] = roofline_family("score", prof, n1, m1, TREES)
    if not args.no_extras and rank == 0:
        try:
            extras.update(plain_leg(sb, m1))
        except Exception as e:  # a failing side leg must not hide the main number
            extras["plain_error"] = repr(e)
        try:
            from paper_2311_00869_gb300 import autotune

            extras["graphl_tuning"] = autotune.tune(sb, K=TREES, R=256)
            extras.update(graphl_leg(P, sb, n1, m1))
        except Exception as e:
            extras["graphl_error"] = repr(e)
        try:
            line["e2e"] = e2e_leg(P, sb, n, u, v, s)
        except Exception as e:
            line["e2e"] = {"error": repr(e)}
        try:
            g = oracle_graph(n, u, v, s)
            line["cpu_baseline"] = cpu_baseline(g)
        except Exception as e:
            line["cpu_baseline"] = {"error": repr(e)}
    line["extras"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)
    sb.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _src_digest(paths):
    """sha256 of kernel sources with comments and whitespace removed."""
    import hashlib
    import re

    h = hashlib.sha256()
    for rel in paths:
        txt = open(os.path.join(ROOT, rel)).read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", " ", txt)
        h.update(" ".join(txt.split()).encode())
    return h.hexdigest()


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a
# kernel, from an ncu capture of this bench's own workload (the command is in
# the matching summary under profiles/).  A figure is reported only while the
# kernel sources still match the digest taken when it was captured.
_BPP_SRC = ("paper_2311_00869_gb300/csrc/sb_bpp.cu", "paper_2311_00869_gb300/csrc/sb_internal.cuh")
NCU_TRAFFIC = {
    "bfs": (3531305216 + 1342316288, _BPP_SRC, "6c4d6c063cf4b1545500acebecd4ca1d2d8ff8ca7bef70d0c656dc40ed4bc53e"),
}


def _traffic_bytes():
    out = {}
    for fam, (nbytes, srcs, digest) in NCU_TRAFFIC.items():
        try:
            out[fam] = nbytes if _src_digest(srcs) == digest else None
        except OSError:
            out[fam] = None
    return out


NCU_TRAFFIC_BYTES = _traffic_bytes()
ALU_LANES_PER_SM = 128  # INT32-capable lanes per SM (4 partitions x 32)
NUM_SMS = 152
OPS_PER_HASH = 11  # (u ^ y) + key: 2, the 32-bit finaliser: 8, compare: 1


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def roofline_family(fam, prof, n, m, K, stats=None, sm_mhz=None):
    """Roofline of one kernel family: HBM-bound families against the measured
    copy bandwidth with their algorithmic bytes per launch; the BFS against
    the integer-ALU peak (SMs x INT32 lanes x SM clock) with the parent-key
    hashes the kernel computes per launch (every candidate of every open tree,
    as counted by the kernel)."""
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    ms, launches = prof.get(fam, (0.0, 0))
    if launches == 0 or ms <= 0:
        return None
    avg_s = ms / launches / 1000.0
    if fam == "bfs":
        if not stats or not stats.get("bfs_launches"):
            return None
        hashes = (stats["hashed_candidates"] + stats["hashed_candidates_split_rows"]) / stats["bfs_launches"]
        mhz = 2070.0
        peak = NUM_SMS * ALU_LANES_PER_SM * mhz * 1e6 / 1e9  # Gop/s at the maximum SM clock
        achieved = OPS_PER_HASH * hashes / avg_s / 1e9
        return {"bound": "alu", "kernel": "k_bfs", "achieved": achieved, "peak": peak,
                "peak_source": f"derived: {NUM_SMS} SMs x {ALU_LANES_PER_SM} INT32 lanes x {mhz:.0f} MHz",
                "unit": "Gop/s", "frac": achieved / peak, "traffic": NCU_TRAFFIC_BYTES.get("bfs"),
                "algorithmic_ops_per_launch": OPS_PER_HASH * hashes, "avg_launch_ms": 1000 * avg_s,
                "launches": launches, "sm_mhz_median": sm_mhz}
    W = (K + 63) // 64
    per_launch = {
        # edge stream (8 B per edge) + every label word read once (n x W x 8 B) + counts
        "score": 8 * m + n * W * 8 + 4 * K,
        "hash": n * W * 8 + n * 8 + 8 * K,
        "cloud": n * W * 8 + n * W * 8,
    }.get(fam)
    if per_launch is None:
        return None
    achieved = per_launch / avg_s / 1e9
    return {"bound": "hbm", "kernel": {"score": "k_score", "hash": "k_state_hash", "cloud": "cloud"}[fam],
            "achieved": achieved, "peak": hbm, "peak_source": src, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": NCU_TRAFFIC_BYTES.get(fam), "algorithmic_bytes_per_launch": per_launch,
            "avg_launch_ms": 1000 * avg_s, "launches": launches}


def roofline(prof, n, m, K, stats=None, sm_mhz=None):
    """Roofline object of the dominant kernel family."""
    fam = max(prof, key=lambda k: prof[k][0])
    r = roofline_family(fam, prof, n, m, K, stats, sm_mhz)
    return r if r is not None else {"bound": "hbm", "kernel": fam, "achieved": None, "peak": None, "unit": "GB/s",
                                    "frac": None, "traffic": None}


def plain_leg(sb, m):
    """The same 64 trees, one tree per launch (plain) vs one 64-tree launch."""
    import torch

    sb.cloud_reset(max_states=8192)
    t0 = 50_000_000
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in range(64):
        sb.sample_trees(SEED, t0 + i, 1)
        sb.frustration()
        sb.cloud_insert()
    torch.cuda.synchronize()
    plain = time.perf_counter() - t
    c_plain, _ = sb.cloud()
    sb.cloud_reset(max_states=8192)
    torch.cuda.synchronize()
    t = time.perf_counter()
    sb.sample_trees(SEED, t0, 64)
    counts, _ = sb.frustration()
    sb.cloud_insert()
    torch.cuda.synchronize()
    batched = time.perf_counter() - t
    c_b, fr_b = sb.cloud()
    same = bool(np.array_equal(c_plain["S"], c_b["S"]) and np.array_equal(c_plain["count"], c_b["count"]))
    return {"plain_edge_evals_per_s": 64 * m / plain, "batched64_edge_evals_per_s": 64 * m / batched,
            "plain_vs_batched_same_cloud": same, "plain64_fr_min": int(c_plain["S"].min())}


def graphl_leg(P, sb, n, m, R=256, steps=50, alpha=0.05, plain_inits=0):
    import torch

    import synth

    g0 = torch.from_numpy(synth.gamma0(n, R, seed=0)).cuda()
    out = torch.empty_like(g0)
    sb.graphL_descent(g0, alpha, steps, out=out)  # warm-up: captures the step loop as a CUDA graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sb.profile_read()
    sb.profile(True)
    e0.record()
    _, exps, _, F_final = sb.graphL_descent(g0, alpha, steps, out=out)
    e1.record()
    torch.cuda.synchronize()
    sb.profile(False)
    prof = sb.profile_read()
    ms = e0.elapsed_time(e1)
    F0, _ = sb.graphL_round(g0)
    res = {"graphl_steps_per_s": steps / (ms / 1000.0), "graphl_R": R, "graphl_steps": steps,
           "graphl_init_steps_per_s": R * steps / (ms / 1000.0), "graphl_F_min_start": int(F0.min()),
           "graphl_F_min_final": int(F_final.min()), "graphl_row_kernel_ms_per_step": prof["gl_rows"][0] / steps}
    if plain_inits:
        # untimed: the discrete loss before every 50th step
        _, _, F_trace, _ = sb.graphL_descent(g0, alpha, steps, trace=True, out=out)
        res["graphl_F_min_every_50"] = [int(x) for x in F_trace[::50].min(dim=1).values.cpu()]
        # plain: one start point per launch, the same columns, must reach the same F
        Fb = F_final.cpu()
        same = True
        t_plain = 0.0
        for r in range(plain_inits):
            col = g0[:, r:r + 1].contiguous()
            o1 = torch.empty_like(col)
            sb.graphL_descent(col, alpha, steps, out=o1)
            torch.cuda.synchronize()
            e0.record()
            _, _, _, F1 = sb.graphL_descent(col, alpha, steps, out=o1)
            e1.record()
            torch.cuda.synchronize()
            t_plain += e0.elapsed_time(e1)
            same = same and int(F1[0]) == int(Fb[r])
        res["graphl_plain_init_steps_per_s"] = plain_inits * steps / (t_plain / 1000.0)
        res["graphl_plain_inits"] = plain_inits
        res["graphl_plain_same_F"] = same
    return res


def e2e_leg(P, sb, n, u, v, s, steps=3):
    """Through the C ABI with host buffers: per step the COO goes host -> device
    from pinned memory, is ingested, K trees are sampled, and the counts,
    hashes and cloud come back to host memory."""
    import torch

    pu = torch.from_numpy(u).pin_memory()
    pv = torch.from_numpy(v).pin_memory()
    ps = torch.from_numpy(s).pin_memory()
    hc = torch.empty(TREES, dtype=torch.int32).pin_memory()
    hh = torch.empty(TREES, dtype=torch.int64).pin_memory()
    m1 = 0
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in range(steps):
        _, m1, _ = sb.load_graph(n, pu, pv, ps)
        sb.sample_trees(SEED, 90_000_000 + i * TREES, TREES)
        sb.frustration(hc, hh)
        cl, fr = sb.cloud()
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    h2d = u.nbytes + v.nbytes + s.nbytes
    d2h = hc.numel() * 4 + hh.numel() * 8 + int(cl["S"].shape[0]) * 24
    return {"value": steps * TREES * m1 / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "includes": "H2D of the COO, ingest, sample, count, cloud, D2H"}



def batch_cpu_baseline(graphs, K, count=64):
    """The oracle on `count` graphs of the batch drawn with a fixed seed, K
    trees each, on all host cores; edge-evals/s over that subset."""
    import oracle as O

    cores = os.cpu_count() or 1
    idx = np.random.default_rng(7).choice(len(graphs), size=min(count, len(graphs)), replace=False)
    gs = [O.clean_graph(*graphs[i]) for i in idx]
    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda g: O.sample(g, SEED, 0, K, want_labels=False), gs))
    el = time.perf_counter() - t
    m_sub = sum(g.m for g in gs)
    return {"value": K * m_sub / el, "unit": "edge-evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(gs)} of the graphs (seeded choice, {m_sub} edges), {K} trees each, {el:.1f} s"}


def batch_leg(args, P):
    """Uneven batch: `--graphs` Chung-Lu graphs (vertex counts log-uniform in
    [50, 50000], mean degree 8, exponent 2.5, 5-30% negative), 256 trees per
    graph in one sampling call over the disjoint union, per-graph clouds, and
    32 graphL start points per graph for `--steps` descent steps."""
    import torch

    import synth

    graphs, gen_s = args.batch_graphs, args.batch_gen_s
    sb = P.SignedBal(0)
    nv, mv = sb.load_batch(graphs)
    K, R = 256, 32
    n_tot, m_tot = int(nv.sum()), int(mv.sum())
    tuned = {"default": True}
    if not args.no_tune:
        from paper_2311_00869_gb300 import autotune

        tuned = autotune.tune(sb, K=K, R=R)
    for i in range(args.warmup):
        sb.sample_trees(SEED, i * K, K)
        sb.batch_cloud(want_entries=False)
    torch.cuda.synchronize()
    sb.profile_read()
    sb.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(args.steps):
        sb.sample_trees(SEED, (args.warmup + i) * K, K)
        cl = sb.batch_cloud(want_entries=False)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = sb.profile_read()
    bfs_stats = sb.stats()
    g0 = torch.from_numpy(synth.gamma0(n_tot, R, seed=0)).cuda()
    out = torch.empty_like(g0)
    steps_gl = 100
    sb.graphL_descent(g0, 0.05, steps_gl, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, _, _, F_final = sb.graphL_descent(g0, 0.05, steps_gl, out=out)
    e1.record()
    torch.cuda.synchronize()
    gl_ms = e0.elapsed_time(e1)
    line = {
        "leg": "batch", "metric": "graphBpp edge-evals/s over the uneven batch", "value": K * m_tot / (ms / 1000.0),
        "unit": "edge-evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"uneven_batch_{args.graphs}_chung_lu", "graphs": args.graphs, "n_total": n_tot,
                   "m_total": m_tot, "trees_per_graph": K, "graphl_R": R, "generation_s": gen_s},
        "stages_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]},
        "graphl_steps_per_s": steps_gl / (gl_ms / 1000.0),
        "fr_min_median": float(np.median(cl["fr_min"])),
        "states_median": float(np.median(cl["n_states"])),
        "graphl_F_median": float(np.median(F_final.cpu().numpy())),
        "tuning": tuned,
        "bfs_stats": bfs_stats,
    }
    try:
        line["cpu_baseline"] = batch_cpu_baseline(graphs, K)
    except Exception as e:  # the baseline must not hide the main number
        line["cpu_baseline"] = {"error": repr(e)}
    print(json.dumps(line), flush=True)
    sb.close()
    return 0


def quality_leg(args, P, K_total=4096, R=256, steps=500, alpha=0.05):
    """graphL against graphBpp on the 2^20 two-faction graph: the smallest S
    among the first K trees (K = 64 ... 4096) and distinct states, the
    smallest graphL F among the first r start points (r = 1, 16, 256) after
    every 50 steps, and the frustration of the planted two-faction state."""
    import torch

    import synth

    n, u, v, s, fac = synth.rmat_two_faction(scale=args.scale, m_target=1 << args.edges_log2, with_factions=True)
    sb = P.SignedBal(0)
    n1, m1, vmap = sb.load_graph(n, u, v, s, want_vmap=True)
    if not args.no_tune:
        from paper_2311_00869_gb300 import autotune

        autotune.tune(sb, K=TREES, R=R)
    # planted state on the cleaned graph: edges whose sign disagrees with it
    cu, cv, cneg = (t.cpu().numpy() for t in sb.graph_edges())
    inv = np.empty(n1, np.int64)
    inv[vmap[vmap >= 0]] = np.nonzero(vmap >= 0)[0]
    planted = int(np.count_nonzero((fac[inv[cu]] * fac[inv[cv]] < 0) != (cneg != 0)))
    sb.cloud_reset(max_states=K_total + 64)
    mins, counts_all = {}, []
    t0 = 0
    while t0 < K_total:
        sb.sample_trees(SEED, t0, TREES)
        c, _ = sb.frustration()
        counts_all.append(c.cpu().numpy())
        sb.cloud_insert()
        t0 += TREES
    cs = np.concatenate(counts_all)
    for k in (64, 256, 1024, 4096):
        if k <= K_total:
            mins[str(k)] = int(cs[:k].min())
    cl, fr = sb.cloud()
    g0 = torch.from_numpy(synth.gamma0(n1, R, seed=0)).cuda()
    _, _, F_trace, F_final = sb.graphL_descent(g0, alpha, steps, trace=True)
    Ft = F_trace.cpu().numpy()
    Ff = F_final.cpu().numpy()
    gl = {}
    for r in (1, 16, 256):
        if r <= R:
            gl[str(r)] = [int(Ft[st, :r].min()) for st in range(0, steps, 50)] + [int(Ff[:r].min())]
    line = {"leg": "quality", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n1, "m": m1, "graphl_R": R, "graphl_steps": steps,
                       "graphl_alpha": alpha},
            "planted_state_frustration": planted,
            "graphbpp_min_S_after_K_trees": mins, "graphbpp_distinct_states": int(cl["S"].shape[0]),
            "graphl_min_F_every_50_steps_then_final_by_start_points": gl}
    print(json.dumps(line), flush=True)
    sb.close()
    return 0


def kruskal_leg(args, P):
    """graphBpp with the randomized Kruskal sampler on the 2^20 graph: K = 1024
    trees per step (sample, count, hash, cloud), timed like the main line; the
    BFS sampler's step on the same graph beside it, the smallest S and the
    distinct states of both samplers over the same trees, and the oracle's
    Kruskal trees on the host cores."""
    import torch

    n, u, v, s = workload(args)
    stream = torch.cuda.current_stream()
    sb = P.SignedBal(0, stream=stream)
    n1, m1, _ = sb.load_graph(n, u, v, s)
    K = TREES
    steps_total = args.warmup + args.steps

    def run(sample):
        sb.cloud_reset(max_states=(steps_total + 2) * K + 64)
        for i in range(args.warmup):
            sample(SEED, i * K, K)
            sb.frustration()
            sb.cloud_insert()
        torch.cuda.synchronize()
        sb.profile_read()
        sb.profile(True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(args.steps):
            sample(SEED, (args.warmup + i) * K, K)
            sb.frustration()
            sb.cloud_insert()
        ev1.record(stream)
        torch.cuda.synchronize()
        sb.profile(False)
        prof = sb.profile_read()
        ms = ev0.elapsed_time(ev1) / args.steps
        cl, frmin = sb.cloud()
        return {"ms_per_step": ms, "edge_evals_per_s": K * m1 / (ms / 1000.0),
                "stages_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]},
                "gpu_launches_per_step": sum(c for _, c in prof.values()) / args.steps,
                "fr_min": int(frmin), "distinct_states": int(cl["S"].shape[0]), "trees": steps_total * K}

    kr = run(sb.sample_trees_kruskal)
    bfs = run(sb.sample_trees)
    line = {"leg": "kruskal", "metric": METRIC + " (Kruskal sampler)", "value": kr["edge_evals_per_s"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": kr["ms_per_step"],
            "higher_is_better": True, "dtype": "u64", "data": "synthetic",
            "config": config_dict(args, n1, m1, 1), "kruskal": kr, "bfs_same_trees": bfs}
    if not args.no_extras:
        import oracle as O

        g = oracle_graph(n, u, v, s)
        cores = os.cpu_count() or 1
        t = time.perf_counter()
        with ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(lambda i: O.mst_sample(g, SEED, 30_000_000 + i, 1, want_labels=False), range(cores)))
        el = time.perf_counter() - t
        line["cpu_baseline"] = {"value": cores * g.m / el, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{cores} Kruskal trees (sort, union-find, labels, count, hash), "
                                          f"{cores} threads, {el:.1f} s"}
    print(json.dumps(line), flush=True)
    sb.close()
    return 0


def scale_cpu_baseline(sb, n, u, v, s, K, each=8):
    """The oracle on trees [0, each) and [K - each, K) of the paper-scale
    graph on all host cores (the rate is extrapolated to all K trees), and a
    bit-for-bit check of those trees' counts and hashes against the GPU."""
    import oracle as O

    cores = os.cpu_count() or 1
    t = time.perf_counter()
    g = O.clean_graph(n, u, v, s)
    clean_s = time.perf_counter() - t
    trees = list(range(each)) + list(range(K - each, K))
    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        refs = list(ex.map(lambda tt: O.sample(g, SEED, tt, 1, want_labels=False), trees))
    el = time.perf_counter() - t
    sb.sample_trees(SEED, 0, K)
    counts, hashes = sb.frustration()
    counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
    same = all(counts[tt] == r["counts"][0] and hashes[tt] == r["hashes"][0] for tt, r in zip(trees, refs))
    return {"value": len(trees) * g.m / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"trees [0,{each}) and [{K - each},{K}) on {cores} threads, {el:.1f} s "
                      f"(rate extrapolated to {K} trees); cleaning the graph took {clean_s:.1f} s",
            "bit_exact_on_sample": bool(same)}


def scale_leg(args, P):
    """Paper-scale graphBpp: R-MAT with 2^24 vertex ids and 2^27 distinct
    undirected edges, three planted factions (94.8 / 2.6 / 2.6 %, inter-faction
    edges negative) with 15 % sign noise; each step grows 4096 trees (64
    words), scores them and adds them to the cloud."""
    import torch

    n, u, v, s = args.scale_graph
    sb = P.SignedBal(0)
    t = time.perf_counter()
    n1, m1, _ = sb.load_graph(n, u, v, s)
    torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t
    K = 4096
    tuned = {"default": True}
    if not args.no_tune:
        from paper_2311_00869_gb300 import autotune

        tuned = autotune.tune(sb, K=K)
    sb.cloud_reset(max_states=(args.warmup + args.steps) * K + 64)
    counts = torch.empty(K, dtype=torch.int32, device="cuda")
    hashes = torch.empty(K, dtype=torch.int64, device="cuda")

    def step(i):
        sb.sample_trees(SEED, i * K, K)
        sb.frustration(counts, hashes)
        return sb.cloud_insert()

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    sb.profile_read()
    sb.profile(True)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sb.profile(False)
    prof = sb.profile_read()
    ms = ev0.elapsed_time(ev1) / args.steps
    stats = sb.stats()
    cl, fr_min = sb.cloud()
    line = {
        "leg": "scale24", "metric": "graphBpp edge-evals/s (trees x |E| / s), batched", "value": K * m1 / (ms / 1e3),
        "unit": "edge-evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"rmat{args.scale}_3faction_K4096", "n": n1, "m": m1, "trees_per_step": K,
                   "graph": f"R-MAT scale {args.scale}, 2^{args.edges_log2} undirected edges, three factions + "
                            "15% sign noise, LCC",
                   "generation_s": args.scale_gen_s, "ingest_s": ingest_s},
        "gpu_launches": sum(c for _, c in prof.values()), "clocks": clk,
        "stages_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]},
        "roofline": roofline(prof, n1, m1, K, stats, (clk or {}).get("sm_mhz")),
        "roofline_score": roofline_family("score", prof, n1, m1, K),
        "extras": {"fr_min": int(fr_min), "distinct_states": int(cl["S"].shape[0]), "bfs_stats": stats, "tuning": tuned,
                   "negative_fraction": float((s < 0).mean())},
    }
    if not args.no_extras:
        try:
            line["cpu_baseline"] = scale_cpu_baseline(sb, n, u, v, s, K)
        except Exception as e:  # the baseline must not hide the main number
            line["cpu_baseline"] = {"error": repr(e)}
    print(json.dumps(line), flush=True)
    sb.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
