#!/usr/bin/env python3
"""graphBpp / graphL benchmark on GB300 (one JSON line on rank 0).

Workload (N=1): the paper-scale R-MAT signed graph with 2^24 vertex ids and
2^27 distinct undirected edges (a,b,c,d = 0.57, 0.19, 0.19, 0.05; three
planted factions 94.8 / 2.6 / 2.6 %, inter-faction edges negative, 15 % iid
sign flips; largest connected component), K = 4096 randomized-BFS trees per
step (64 words of 64 trees).  One step is the whole graphBpp hot path on one
batch: tree sampling + parity labels + state hash (sb_sample_trees),
frustration counts (sb_frustration) and cloud insertion (sb_cloud).  Ingest is
done once, outside the timed region (it is timed inside the e2e leg).
Metric: edge-evals/s = trees x |E| / s.  The inputs (CSR 1.07 GB, labels
3.8 GB) are far larger than L2, so no flush is needed between steps.

Also reported: the 2^20-vertex workload (1024 trees per step), the plain path
(one tree per launch) against one batched launch at the same cloud on the
1,000-vertex Erdos-Renyi graph and on the 2^20 graph, graphL steps/s (R = 256
start points, 500 steps, against one start point per launch at the same F),
the end-to-end number through the C ABI with host buffers, the roofline of
the dominant kernel against a measured ceiling and the CPU oracle on the host
cores.

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
SEED = 0
# name -> (R-MAT scale, log2 of the edges, planted factions, trees per step)
WORKLOADS = {
    "rmat24": (24, 27, 3, 4096),
    "rmat20": (20, 24, 2, 1024),
}
WORKLOAD_NAMES = {"rmat24": "rmat24_3faction_K4096", "rmat20": "rmat20_2faction_K1024"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS),
                    help="rmat24: 2^24 vertex ids, 2^27 edges, three factions, 4096 trees per step (default); "
                         "rmat20: 2^20 vertex ids, 2^24 edges, two factions, 1024 trees per step")
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale (overrides the workload's)")
    ap.add_argument("--edges-log2", type=int, default=None, help="log2 of the edge count (overrides the workload's)")
    ap.add_argument("--trees", type=int, default=None, help="trees per step (overrides the workload's)")
    ap.add_argument("--no-extras", action="store_true", help="skip the side legs, e2e and the CPU baseline")
    ap.add_argument("--leg", default="bpp", choices=["bpp", "graphl", "batch", "quality", "kruskal"],
                    help="bpp: the graphBpp line (default); graphl: graphL descent only; batch: uneven batch; "
                         "quality: graphBpp min S and graphL min F against the planted state; "
                         "kruskal: graphBpp with randomized Kruskal trees instead of BFS trees")
    ap.add_argument("--R", type=int, default=256, help="graphL start points (--leg graphl)")
    ap.add_argument("--gl-steps", type=int, default=500, help="graphL descent steps (--leg graphl)")
    ap.add_argument("--graphs", type=int, default=4096, help="graphs in the uneven batch (--leg batch)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tuning knobs")
    ap.add_argument("--gl-lanes", type=int, default=0, help="graphL lanes per row segment (8, 16 or 32; with --no-tune)")
    ap.add_argument("--bfs-words", type=int, default=0, help="64-tree words per BFS launch (with --no-tune)")
    ap.add_argument("--bfs-group", type=int, default=0, help="lanes per BFS vertex group (with --no-tune)")
    args = ap.parse_args()
    if args.leg in ("graphl", "quality", "kruskal") and args.workload == "rmat24" and args.scale is None:
        args.workload = "rmat20"  # these legs run on the 2^20 two-faction graph
    sc, el, fac, K = WORKLOADS[args.workload]
    args.custom = args.scale is not None or args.edges_log2 is not None
    args.scale = args.scale if args.scale is not None else sc
    args.edges_log2 = args.edges_log2 if args.edges_log2 is not None else el
    args.factions = fac
    args.K = args.trees if args.trees is not None else K
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def gen_graph(scale, edges_log2, factions, workers=0):
    """(n, src, dst, sign) of the R-MAT workload (drawn before any CUDA call:
    the three-faction draw may use a spawned process pool)."""
    import synth

    if factions == 3:
        return synth.rmat_three_faction(scale=scale, m_target=1 << edges_log2, workers=workers)
    return synth.rmat_two_faction(scale=scale, m_target=1 << edges_log2)


def workload_name(args):
    if args.custom:
        return f"rmat{args.scale}_e{args.edges_log2}"
    return WORKLOAD_NAMES[args.workload]


def graph_text(scale, edges_log2, factions):
    noise = "three factions (94.8 / 2.6 / 2.6 %, inter-faction negative) + 15% sign noise" if factions == 3 \
        else "two factions + 10% sign noise"
    return f"R-MAT scale {scale}, 2^{edges_log2} undirected edges, {noise}, LCC"


def config_dict(args, n_clean, m_clean, world):
    return {
        "workload": workload_name(args),
        "graph": graph_text(args.scale, args.edges_log2, args.factions),
        "n": n_clean,
        "m": m_clean,
        "trees_per_step": args.K,
        "words_per_step": (args.K + 63) // 64,
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


def oracle_trees(g, t0, count, cores, want=False):
    """Samples trees [t0, t0 + count) with the oracle, one tree per task on
    `cores` threads; returns (seconds, per-tree results if want)."""
    import oracle as O

    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        res = list(ex.map(lambda i: O.sample(g, SEED, t0 + i, 1, want_labels=False), range(count)))
    return time.perf_counter() - t, (res if want else None)


def cpu_baseline(sb, g, t0=10_000_000, budget_s=10.0):
    """The oracle on the host cores: rounds of one tree per core (BFS tree,
    labels, count, hash) until `budget_s` has passed; the trees of the first
    round are also checked bit for bit against the GPU's."""
    cores = os.cpu_count() or 1
    done, el, first = 0, 0.0, None
    while el < budget_s:
        dt, res = oracle_trees(g, t0 + done, cores, cores, want=first is None)
        if first is None:
            first = res
        el += dt
        done += cores
    sb.sample_trees(SEED, t0, cores)
    counts, hashes = sb.frustration()
    counts, hashes = counts.cpu().numpy(), hashes.cpu().numpy().view(np.uint64)
    same = all(int(counts[i]) == int(r["counts"][0]) and int(hashes[i]) == int(r["hashes"][0])
               for i, r in enumerate(first))
    return {"value": done * g.m / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} trees (BFS tree, labels, count, hash) of the same graph, one per thread on "
                      f"{cores} threads, {el:.1f} s",
            "bit_exact_on_first_round": bool(same)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n, u, v, s = gen_graph(args.scale, args.edges_log2, args.factions, workers=os.cpu_count() or 1)
    g = oracle_graph(n, u, v, s)
    cores = os.cpu_count() or 1
    per_step = cores
    for i in range(args.warmup):
        oracle_trees(g, i * per_step, per_step, cores)
    el = 0.0
    for i in range(args.steps):
        el += oracle_trees(g, (args.warmup + i) * per_step, per_step, cores)[0]
    value = args.steps * per_step * g.m / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": config_dict(args, g.n, g.m, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} trees per step, one per thread on {cores} threads, the same graph "
                                   f"(the workload's {args.K} trees per step are not all run)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- ours
def bpp_timed(sb, K, steps, warmup, stream, world=1, rank=0, dist=None, clocks=None):
    """`warmup` untimed then `steps` timed graphBpp steps of K trees (sample,
    count, hash, cloud), bracketed by CUDA events on the library's stream."""
    import torch

    sb.cloud_reset(max_states=(warmup + steps + 2) * K + 64)
    counts = torch.empty(K, dtype=torch.int32, device="cuda")
    hashes = torch.empty(K, dtype=torch.int64, device="cuda")

    # trees are independent: rank r takes its own tree ranges (weak scaling)
    def step(i):
        t0 = ((i * world) + rank) * K
        sb.sample_trees(SEED, t0, K)
        sb.frustration(counts, hashes)
        return sb.cloud_insert()

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    sb.profile_read()
    sb.profile(True)
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(steps):
        step(warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    sb.profile(False)
    prof = sb.profile_read()
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    cl, fr_min = sb.cloud()
    return {"ms_step": ms / steps, "prof": prof, "stats": sb.stats(), "clk": clk, "cloud": cl, "fr_min": fr_min}


def stages(prof, steps):
    return {k: round(v[0] / steps, 4) for k, v in prof.items() if v[1]}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    workers = os.cpu_count() or 1
    if args.leg == "batch":
        import synth

        t = time.perf_counter()  # the process pool starts before any CUDA call
        args.batch_graphs = list(synth.uneven_batch(count=args.graphs, workers=workers))
        args.batch_gen_s = time.perf_counter() - t
    elif args.leg != "quality":  # the quality leg draws its graph with the planted factions
        t = time.perf_counter()
        args.graph = gen_graph(args.scale, args.edges_log2, args.factions, workers=workers)
        args.gen_s = time.perf_counter() - t
    side = args.leg == "bpp" and not args.no_extras and rank == 0 and args.workload == "rmat24" and not args.custom
    if side:  # the 2^20-vertex graph of the side legs (graphL runs on it)
        args.side_graph = gen_graph(20, 24, 2)
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2311_00869_gb300 as P

    if args.leg == "batch":
        return batch_leg(args, P)
    if args.leg == "quality":
        return quality_leg(args, P)
    if args.leg == "kruskal":
        return kruskal_leg(args, P)
    n, u, v, s = args.graph
    stream = torch.cuda.current_stream()
    sb = P.SignedBal(local, stream=stream)
    t = time.perf_counter()
    n1, m1, _ = sb.load_graph(n, u, v, s)
    torch.cuda.synchronize()
    ingest_s = time.perf_counter() - t
    if args.leg == "graphl":
        tuned = {"default": True}
        if not args.no_tune:
            from paper_2311_00869_gb300 import autotune

            tuned = autotune.tune(sb, K=1024, R=args.R)
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
    K = args.K
    tuned = {"default": True}
    if args.no_tune and (args.bfs_words or args.bfs_group):
        knobs = {k: v for k, v in (("bfs_words", args.bfs_words), ("bfs_group", args.bfs_group)) if v}
        sb.set_tuning(**knobs)
        tuned = dict(knobs, default=False)
    if not args.no_tune:
        try:
            from paper_2311_00869_gb300 import autotune

            tuned = autotune.tune(sb, K=K)
        except Exception as e:  # tuning only changes speed
            tuned = {"error": repr(e)}
    peak_hps = None
    try:
        peak_hps = sb.hash_peak(1.0)  # measured ceiling of the BFS hash mix
    except Exception:
        pass
    r = bpp_timed(sb, K, args.steps, args.warmup, stream, world, rank, dist, ClockSampler(local))
    ms_step, prof = r["ms_step"], r["prof"]
    value = world * K * m1 / (ms_step / 1000.0)
    launches = sum(c for _, c in prof.values())
    cl = r["cloud"]
    extras = {"fr_min": int(r["fr_min"]), "distinct_states": int(cl["S"].shape[0]), "tuning": tuned,
              "bfs_stats": r["stats"], "trees_per_s": world * K / (ms_step / 1000.0),
              "generation_s": round(args.gen_s, 1), "ingest_s": round(ingest_s, 3)}
    if args.factions == 3:
        extras["negative_fraction"] = float((s < 0).mean())
    if dist:  # host-side merge of the rank clouds, after the timed region
        from paper_2311_00869_gb300 import shard

        merged = shard.gather_cloud(cl)
        extras["distinct_states_all_ranks"] = int(merged["S"].shape[0])
        extras["fr_min_all_ranks"] = int(merged["S"].min()) if merged["S"].size else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": config_dict(args, n1, m1, world),
        "gpu_launches": launches, "clocks": r["clk"], "stages_ms_per_step": stages(prof, args.steps),
    }
    line["roofline"] = roofline(prof, n1, m1, K, r["stats"], peak_hps, workload_name(args), bfs_shape(sb))
    extras["roofline_score"] = roofline_family("score", prof, n1, m1, K)
    extras["roofline_hash"] = roofline_family("hash", prof, n1, m1, K)
    if not args.no_extras and rank == 0:
        try:
            line["e2e"] = e2e_leg(P, sb, n, u, v, s, K)
        except Exception as e:
            line["e2e"] = {"error": repr(e)}
        g = None
        try:
            g = oracle_graph(n, u, v, s)
            line["cpu_baseline"] = cpu_baseline(sb, g)
        except Exception as e:
            line["cpu_baseline"] = {"error": repr(e)}
        del g
    sb.close()
    torch.cuda.empty_cache()
    if side:
        try:
            extras["rmat20_2faction_K1024"] = side_legs(P, args, stream, peak_hps)
        except Exception as e:  # a failing side leg must not hide the main number
            extras["rmat20_error"] = repr(e)
        try:
            extras["plain_er1000_K64"] = plain_leg_er(P, stream)
        except Exception as e:
            extras["plain_er1000_error"] = repr(e)
    line["extras"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def side_legs(P, args, stream, peak_hps, K=1024, steps=10, warmup=3):
    """The 2^20-vertex two-faction graph: its graphBpp line (1024 trees per
    step), plain against batched on 64 of its trees, and graphL with R = 256
    start points for 500 steps against one start point per launch."""
    n, u, v, s = args.side_graph
    sb = P.SignedBal(0, stream=stream)
    try:
        n1, m1, _ = sb.load_graph(n, u, v, s)
        from paper_2311_00869_gb300 import autotune

        tuned = autotune.tune(sb, K=K)
        r = bpp_timed(sb, K, steps, warmup, stream)
        out = {"n": n1, "m": m1, "trees_per_step": K, "steps": steps, "ms_per_step": r["ms_step"],
               "edge_evals_per_s": K * m1 / (r["ms_step"] / 1000.0), "trees_per_s": K / (r["ms_step"] / 1000.0),
               "stages_ms_per_step": stages(r["prof"], steps), "bfs_stats": r["stats"], "tuning": tuned,
               "roofline": roofline_family("bfs", r["prof"], n1, m1, K, r["stats"], peak_hps,
                                           traffic_bytes("bfs", WORKLOAD_NAMES["rmat20"], bfs_shape(sb))),
               "roofline_score": roofline_family("score", r["prof"], n1, m1, K),
               "fr_min": int(r["fr_min"])}
        out["plain_vs_batched"] = plain_leg(sb, m1)
        out["graphl_tuning"] = autotune.tune(sb, K=K, R=256)
        out["graphl"] = graphl_leg(P, sb, n1, m1, R=256, steps=500, plain_inits=4)
    finally:
        sb.close()
    return out


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
# the matching summary under profiles/), keyed by (family, workload, 64-tree
# words per BFS launch, lanes per BFS vertex group).  A figure is reported
# only for the launch shape it was taken on, and only while the kernel
# sources still match the digest taken when it was captured.
_BPP_SRC = ("paper_2311_00869_gb300/csrc/sb_bpp.cu", "paper_2311_00869_gb300/csrc/sb_internal.cuh")
NCU_TRAFFIC = {
    # profiles/k_bfs_rmat24_K4096.md and profiles/k_bfs_rmat20_K1024.md (one-pass captures of
    # the benchmark workloads; ncu prints GB to 10 MB)
    ("bfs", "rmat24_3faction_K4096", 32, 32): (233_050_000_000 + 29_910_000_000, _BPP_SRC,
                                               "d19a2ec8d19cd60565472ba7e5162344415b710f779e88ab2453464d4156c557"),
    ("bfs", "rmat24_3faction_K4096", 16, 16): (92_790_000_000 + 14_120_000_000, _BPP_SRC,
                                               "d19a2ec8d19cd60565472ba7e5162344415b710f779e88ab2453464d4156c557"),
    ("bfs", "rmat20_2faction_K1024", 16, 16): (3_120_000_000 + 1_250_000_000, _BPP_SRC,
                                               "d19a2ec8d19cd60565472ba7e5162344415b710f779e88ab2453464d4156c557"),
}


def bfs_shape(sb):
    """(words per BFS launch, lanes per vertex group) the library will use."""
    t = sb.get_tuning()
    words = t["bfs_words"] or 32
    gw = 1
    while gw < words:
        gw <<= 1
    g = t["bfs_group"]
    return words, (g if gw < g <= 2 * gw else gw)


def traffic_bytes(fam, workload, shape):
    e = NCU_TRAFFIC.get((fam, workload) + tuple(shape))
    if e is None:
        return None
    nbytes, srcs, digest = e
    try:
        return nbytes if _src_digest(srcs) == digest else None
    except OSError:
        return None


OPS_PER_HASH = 10  # per hashed candidate: + tree salt (1), the 32-bit finaliser (8), running minimum (1)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _derived_alu_peak():
    """SMs x 128 INT32 lanes x the largest SM clock, in Gop/s (an upper bound:
    the finaliser's two multiplies do not issue at that rate)."""
    try:
        import torch

        sms = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        sms = 152
    mhz = float(_peaks().get("sm_max_mhz", 2070.0))
    return sms * 128 * mhz * 1e6 / 1e9, f"derived: {sms} SMs x 128 INT32 lanes x {mhz:.0f} MHz"


def roofline_family(fam, prof, n, m, K, stats=None, peak_hps=None, traffic=None):
    """Roofline of one kernel family: HBM-bound families against the measured
    copy bandwidth with their algorithmic bytes per launch; the BFS against
    the measured rate of its own hash mix (sb_hash_peak: the add, finaliser
    and minimum of one hashed candidate, on independent chains over the whole
    GPU), with the candidates the kernel hashes per launch (every candidate
    of every open tree, as counted by the kernel)."""
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
        achieved = OPS_PER_HASH * hashes / avg_s / 1e9
        derived, dsrc = _derived_alu_peak()
        if peak_hps:
            peak = OPS_PER_HASH * peak_hps / 1e9
            psrc = ("measured: sb_hash_peak, the BFS's per-candidate hash mix (salt add, fmix32, min) on 8 "
                    "independent chains per thread over a full grid, 1 s, CUDA events")
        else:
            peak, psrc = derived, dsrc
        return {"bound": "alu", "kernel": "k_bfs", "achieved": achieved, "peak": peak, "peak_source": psrc,
                "unit": "Gop/s", "frac": achieved / peak, "traffic": traffic,
                "ops_per_hash": OPS_PER_HASH, "hashes_per_launch": hashes,
                "algorithmic_ops_per_launch": OPS_PER_HASH * hashes, "avg_launch_ms": 1000 * avg_s,
                "launches": launches, "derived_peak": derived, "derived_peak_source": dsrc}
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
    return {"bound": "hbm", "kernel": {"score": "k_score", "hash": "k_state_hash_tab", "cloud": "cloud"}[fam],
            "achieved": achieved, "peak": hbm, "peak_source": src, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "algorithmic_bytes_per_launch": per_launch,
            "avg_launch_ms": 1000 * avg_s, "launches": launches}


def roofline(prof, n, m, K, stats=None, peak_hps=None, workload=None, shape=None):
    """Roofline object of the dominant kernel family."""
    fam = max(prof, key=lambda k: prof[k][0])
    r = roofline_family(fam, prof, n, m, K, stats, peak_hps, traffic_bytes(fam, workload, shape or ()))
    return r if r is not None else {"bound": "hbm", "kernel": fam, "achieved": None, "peak": None, "unit": "GB/s",
                                    "frac": None, "traffic": None}


def _same_cloud(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("hash", "S", "count", "first_tree"))


def plain_leg(sb, m, trees=64, reps=3, t0=50_000_000):
    """The same `trees` trees, one tree per launch (plain: sample, count, cloud
    per tree) against one batched launch; each arm warmed up once, then timed
    `reps` times with CUDA events; the two clouds must be equal (hash, S,
    count, first tree)."""
    import torch

    def plain():
        sb.cloud_reset(max_states=trees + 64)
        for i in range(trees):
            sb.sample_trees(SEED, t0 + i, 1)
            sb.frustration()
            sb.cloud_insert()

    def batched():
        sb.cloud_reset(max_states=trees + 64)
        sb.sample_trees(SEED, t0, trees)
        sb.frustration()
        sb.cloud_insert()

    out = {}
    for name, fn in (("plain", plain), ("batched", batched)):
        fn()  # warm-up (buffers sized for this arm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name] = (e0.elapsed_time(e1) / reps, sb.cloud()[0])
    return {"trees": trees, "plain_ms": out["plain"][0], "batched_ms": out["batched"][0],
            "plain_edge_evals_per_s": trees * m / (out["plain"][0] / 1000.0),
            "batched_edge_evals_per_s": trees * m / (out["batched"][0] / 1000.0),
            "same_cloud": bool(_same_cloud(out["plain"][1], out["batched"][1])),
            "fr_min": int(out["batched"][1]["S"].min())}


def plain_leg_er(P, stream):
    """The small plain workload: Erdos-Renyi n = 1,000, m = 5,000, 20 %
    negative, K = 64 trees from seed 0, one tree per launch, against the same
    64 trees in one launch."""
    import synth

    n, u, v, s = synth.er_graph()
    sb = P.SignedBal(0, stream=stream)
    try:
        n1, m1, _ = sb.load_graph(n, u, v, s)
        res = plain_leg(sb, m1, trees=64, reps=5, t0=0)
        res.update({"n": n1, "m": m1})
    finally:
        sb.close()
    return res


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


def e2e_leg(P, sb, n, u, v, s, K, steps=3):
    """Through the C ABI with host buffers: per step the COO goes host -> device
    from pinned memory, is ingested, K trees are sampled, and the counts,
    hashes and cloud come back to host memory."""
    import torch

    pu = torch.from_numpy(u).pin_memory()
    pv = torch.from_numpy(v).pin_memory()
    ps = torch.from_numpy(s).pin_memory()
    hc = torch.empty(K, dtype=torch.int32).pin_memory()
    hh = torch.empty(K, dtype=torch.int64).pin_memory()
    m1 = 0
    n_states = 0
    sb.cloud_reset(max_states=K + 64)  # room for one step's trees (the timed line kept every step's)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in range(steps):
        _, m1, _ = sb.load_graph(n, pu, pv, ps)
        sb.sample_trees(SEED, 90_000_000 + i * K, K)
        sb.frustration(hc, hh)
        cl, fr = sb.cloud()
        n_states = int(cl["S"].shape[0])
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    h2d = u.nbytes + v.nbytes + s.nbytes
    d2h = hc.numel() * 4 + hh.numel() * 8 + n_states * 24
    return {"value": steps * K * m1 / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps,
            "includes": "H2D of the COO, ingest, sample, count, cloud, D2H"}


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
    32 graphL start points per graph for `--steps` descent steps.  The steps
    are timed three ways: one call per stage with its host synchronisation,
    sb_batch_steps with the kernels enqueued directly, and sb_batch_steps
    replaying one captured CUDA graph per step."""
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
    # the same steps with no host synchronisation: kernels enqueued directly,
    # and one step captured as a CUDA graph and replayed
    steps_ms = {}
    fr_steps = {}
    for use_graph in (False, True):
        sb.batch_steps(SEED, 0, K, 2, use_graph=use_graph)  # warm-up (and capture)
        sb.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fr, _ = sb.batch_steps(SEED, args.warmup * K, K, args.steps, use_graph=use_graph)
        e1.record()
        sb.sync()
        steps_ms["graph" if use_graph else "direct"] = e0.elapsed_time(e1) / args.steps
        fr_steps[use_graph] = fr.cpu().numpy()
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
        "steps_no_sync_ms": steps_ms,
        "steps_no_sync_edge_evals_per_s": {k: K * m_tot / (v / 1000.0) for k, v in steps_ms.items()},
        "steps_graph_equals_direct": bool(np.array_equal(fr_steps[False], fr_steps[True])),
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

        autotune.tune(sb, K=args.K, R=R)
    # planted state on the cleaned graph: edges whose sign disagrees with it
    cu, cv, cneg = (t.cpu().numpy() for t in sb.graph_edges())
    inv = np.empty(n1, np.int64)
    inv[vmap[vmap >= 0]] = np.nonzero(vmap >= 0)[0]
    planted = int(np.count_nonzero((fac[inv[cu]] * fac[inv[cv]] < 0) != (cneg != 0)))
    sb.cloud_reset(max_states=K_total + 64)
    mins, counts_all = {}, []
    t0 = 0
    while t0 < K_total:
        sb.sample_trees(SEED, t0, args.K)
        c, _ = sb.frustration()
        counts_all.append(c.cpu().numpy())
        sb.cloud_insert()
        t0 += args.K
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
            "config": {"workload": workload_name(args), "n": n1, "m": m1, "graphl_R": R, "graphl_steps": steps,
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

    n, u, v, s = args.graph
    stream = torch.cuda.current_stream()
    sb = P.SignedBal(0, stream=stream)
    n1, m1, _ = sb.load_graph(n, u, v, s)
    K = args.K
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


if __name__ == "__main__":
    sys.exit(main())
