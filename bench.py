"""Benchmark: exact all-k global clique counts, edges/s, on one GB300.

Workload (default): Chung-Lu power-law graph, n = 1M, m ~ 10.8M, degree
exponent 2.1, plus 500 planted communities of 20-60 vertices at density 0.9
(synthetic, seeded).  One step = the whole hot path on a graph already in
HBM: degeneracy orientation (k-core peel, DAG CSR, root classes) + the SCT
walk over every root + the exact multi-word combine -> C_k for all k.

Prints one JSON line (see the keys below).  `--impl reference` times the CPU
oracle (root-parallel, every host core) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "cl1m_m10m_b2.1_comm500"
METRIC = "all-k clique-count edges/s (bit-exact)"
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
POPC_PER_CLK_PER_SM = 16     # 32-bit population count issue rate per SM per clock
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) per launch of a kernel, from an ncu capture of the
# kernel as it is now (summarised under profiles/, with the capture's date);
# an entry is removed whenever its kernel changes, so that the bench line
# reports null instead of a stale figure
NCU_DRAM_BYTES = {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sequential", action="store_true", help="skip the one-core oracle run of the CPU baseline")
    ap.add_argument("--no-local", action="store_true", help="skip the per-vertex / per-edge measurement")
    ap.add_argument("--profile", default=None, choices=["lanes", "cta", "local", "peel"],
                    help="run one small case of one kernel family for a profiler and exit (no JSON line)")
    ap.add_argument("--no-cl3m", action="store_true",
                    help="skip the all-k count of the 128M-edge com-orkut-shaped graph (about 100 s)")
    ap.add_argument("--serving-queries", type=int, default=10000,
                    help="queries in the serving stream (10000 by default); 0 skips serving")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self, ready_s: float = 3.0):
        """Start sampling; returns once the first sample is written (or after
        ready_s), so that the region timed next is sampled from its start."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < ready_s and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, device) -> float:
    """The largest of every rank's x (all ranks call this; one rank: x)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of N replicas: the units all ranks processed over
    the slowest rank's time."""
    return world * units_per_rank / seconds_max


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the baseline's context."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def min_words(n: int, alpha: int) -> int:
    """64-bit words that hold every count: each is at most n * 2^alpha."""
    return max(1, (int(n).bit_length() + alpha + 1 + 63) // 64)


def workload_config(name, n, m, alpha, omega):
    """The `config` of both arms: the workload and what it fixes."""
    return {"workload": name, "n": n, "m": m, "alpha": alpha, "omega": omega, "kmax": alpha + 1,
            "W": min_words(n, alpha), "counts": "global C_k, every k",
            "l2": "GPU arm: a 256 MiB write flushes the 129 MB L2 between timed steps"}


def run_reference(args, ws, rank):
    """The CPU oracle as the reference arm: every step counts the whole
    workload with the root-parallel oracle (one thread per host core, the
    paper's parallel scheme); edges/s = m / step time."""
    if rank != 0:
        return
    import oracle
    from paper_2001_06784_gb300 import graphgen
    rp, col = graphgen.workload(args.workload)
    n, m = len(rp) - 1, len(col) // 2
    cores = os.cpu_count() or 1
    _, _, alpha = oracle.orient(rp, col)
    times, C = [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        C = oracle.count(rp, col, kmax=alpha + 1, threads=cores)["C"]
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = m / t
    omega = max(k for k, c in enumerate(C) if c)
    sample = "whole workload every step (root-parallel oracle, one thread per host core)"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1000.0, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32 limbs (exact)", "data": "synthetic",
           "config": workload_config(args.workload, n, m, alpha, omega),
           "cpu_baseline": {"value": value, "unit": "edges/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) of this machine's GPUs, else the
    profiling recipe's fallback, and which it is."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def kernel_rooflines(args, dev, rp_d, col_d, step_policy, kmax, W, n, m):
    """Roofline fraction of every kernel of one step, each timed alone: one
    orient + global count with profiling on and the out-degree classes run
    one after another (policy.serial), CUDA events around each phase on its
    stream.  HBM-bound phases (peel, orientation) count the bytes the method
    must move; walk kernels count their AND+POPC word pairs of pivot
    selection against the measured integer rate.  Returns (list, the
    dominant kernel's entry)."""
    import paper_2001_06784_gb300 as pvt
    hbm, hbm_src = hbm_peak()
    nominal = POPC_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e9  # Gop/s
    try:
        alu = pvt.measure_popc_rate(dev) / 1e9
        alu_src = "measured: AND+POPC+ADD register chains on every SM (pvt_measure_popc_rate)"
    except Exception as exc:  # report the nominal figure, and say so
        alu, alu_src = nominal, f"nominal (measurement failed: {exc})"
    ms = {}
    for _ in range(2):  # the second run is kept (warm library, cold L2 after the flush)
        flush = torch_flush(dev)
        dag = pvt.orient(rp_d, col_d, profile=True)
        so = dag.stats()
        dag.set_policy(**dict(step_policy, serial=True))
        dag.count_global(kmax=kmax, W=W)
        sc = dag.stats()
        ms = dict(sc["ms"])
        ms["peel"], ms["orient"] = so["ms"]["peel"], so["ms"]["orient"]
        dag.free()
        del flush
    out = []
    # peel: the CSR read once (col 4 B per directed entry, row_ptr 8 B per vertex)
    peel_b = 4 * 2 * m + 8 * (n + 1)
    # orientation: CSR read, DAG written (ocol 4 B per edge, orow 8 B per vertex), root classes
    orient_b = 4 * 2 * m + 8 * (n + 1) + 4 * m + 8 * (n + 1) + 4 * n
    for name, b in (("peel", peel_b), ("orient", orient_b)):
        t = ms[name]
        if t > 0:
            a = b / (t / 1000.0) / 1e9
            out.append({"kernel": name, "bound": "hbm", "ms": t, "algorithmic": b, "achieved": a, "peak": hbm,
                        "unit": "GB/s", "frac": a / hbm, "peak_source": hbm_src})
    names = pvt.Dag.PHASES
    for c in range(1, 7):
        t = ms[names[1 + c]]
        wds = sc["class_words"][c]
        if t > 0:
            a = wds / (t / 1000.0) / 1e9
            out.append({"kernel": names[1 + c], "bound": "alu", "ms": t, "algorithmic": wds, "achieved": a,
                        "peak": alu, "unit": "Gop/s", "frac": a / alu, "roots": sc["roots"][c]})
    t = ms["walk_frames"]
    if t > 0:
        a = sc["frame_words"] / (t / 1000.0) / 1e9
        out.append({"kernel": "walk_frames", "bound": "alu", "ms": t, "algorithmic": sc["frame_words"],
                    "achieved": a, "peak": alu, "unit": "Gop/s", "frac": a / alu, "frames": sc["frames"]})
    walks = [k for k in out if k["bound"] == "alu"]
    dom = max(walks, key=lambda k: k["ms"])
    roofline = {"bound": "alu", "achieved": dom["achieved"], "peak": alu, "unit": "Gop/s", "frac": dom["frac"],
                "traffic": NCU_DRAM_BYTES.get(dom["kernel"]), "kernel": dom["kernel"], "kernel_ms": dom["ms"],
                "op": "32-bit AND+POPC word pairs of pivot selection", "peak_source": alu_src,
                "nominal_peak": nominal,
                "nominal_source": f"{POPC_PER_CLK_PER_SM} POPC/clk/SM x {SM_COUNT} SMs x {SM_MAX_MHZ:.0f} MHz",
                "timing": "the kernel alone (classes serialised), CUDA events on its stream"}
    return out, roofline


def torch_flush(dev):
    """A write larger than the 129 MB L2."""
    import torch
    f = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    f.zero_()
    return f


def serving_specs(q, seed=5):
    """Parameters of the query stream, drawn in order from one seeded
    generator: independent ER or Chung-Lu graphs, n log-uniform in
    [100, 50000], average degree U[5, 60], exponent U[2.0, 2.5]; each asks
    global all-k or per-edge counts with probability 1/2."""
    rng = np.random.default_rng(seed)
    spec = []
    for i in range(q):
        n = int(np.exp(rng.uniform(np.log(100), np.log(50000))))
        deg = float(rng.uniform(5, 60))
        kind = "global" if rng.random() < 0.5 else "edge"
        if rng.random() < 0.5:
            spec.append((i, n, "er", min(deg, n - 1), None, kind))
        else:
            m = max(1, min(int(n * deg / 2), n * (n - 1) // 4))
            spec.append((i, n, "cl", m, float(rng.uniform(2.0, 2.5)), kind))
    return spec


def serving_graphs(spec):
    """The graphs of a slice of the stream, generated on host threads (the
    generator runs outside the interpreter lock)."""
    import concurrent.futures as cf
    from paper_2001_06784_gb300 import graphgen

    def make(sp):
        i, n, kind_g, a, beta, kind = sp
        if kind_g == "er":
            rp, col = graphgen.generate(n, er_avg_deg=a, seed=5_000_000 + i)
        else:
            rp, col = graphgen.generate(n, chung_lu=(a, beta), seed=5_000_000 + i)
        return rp, col, kind

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(make, spec))


def serving_stream(q, seed=5):
    """The whole stream of q queries (small q only: every graph stays in
    host memory)."""
    return serving_graphs(serving_specs(q, seed))


def run_local(args, dev, flush):
    """Per-vertex and per-edge tables, all k up to the clique number, on the
    Chung-Lu n=500k, m~8.4M, exponent 2.3 graph with 200 planted cliques:
    orient + count on the resident graph, edges/s, bit-exact identities."""
    import torch
    import paper_2001_06784_gb300 as pvt
    from paper_2001_06784_gb300 import graphgen
    name = "cl500k_m8m_b2.3_clq200"
    rp, col = graphgen.workload(name)
    n, m = len(rp) - 1, len(col) // 2
    rpd = torch.from_numpy(rp).to(dev)
    cd = torch.from_numpy(col.view(np.int32)).to(dev)
    dag = pvt.orient(rpd, cd)
    C = pvt.to_ints(dag.count_global())
    omega = max(k for k, c in enumerate(C) if c)
    W = dag.min_words
    dag.free()
    stream = torch.cuda.current_stream(dev)
    res = {"workload": name, "n": n, "m": m, "kmax": omega, "W": W}
    for kind in ("vertex", "edge"):
        rows = n if kind == "vertex" else m
        out = torch.empty((rows, omega + 1, W), dtype=torch.int64, device=dev)
        times = []
        for i in range(1 + max(1, args.steps)):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dag = pvt.orient(rpd, cd)
            if kind == "vertex":
                dag.count_local_vertex(kmax=omega, W=W, out=out)
            else:
                dag.count_local_edge(kmax=omega, W=W, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if i:
                times.append(e0.elapsed_time(e1))
            dag.free()
        # identity against the global counts: sum of c_k over rows = k * C_k or C(k,2) * C_k
        t = out.cpu().numpy().view(np.uint64)
        lo = (t & np.uint64(0xFFFFFFFF)).sum(axis=0, dtype=np.uint64)
        hi = (t >> np.uint64(32)).sum(axis=0, dtype=np.uint64)
        tot = [sum((int(lo[k, w]) + (int(hi[k, w]) << 32)) << (64 * w) for w in range(W)) for k in range(omega + 1)]
        import math
        want = [(k if kind == "vertex" else math.comb(k, 2)) * C[k] for k in range(omega + 1)]
        ms = float(np.mean(times))
        res[kind] = {"ms_per_step": ms, "edges_per_s": m / (ms / 1000.0), "table_bytes": int(t.nbytes),
                     "sum_identity": tot == want}
        # f_k(b) over the table at the k the paper plots (5, 10, ..., 25)
        dist = {}
        for k in (5, 10, 15, 20, 25):
            if k > omega:
                continue
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vals, cnts = pvt.local_distribution(out, k)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            f_mass = int(cnts.sum().item())
            dist[str(k)] = {"ms": e0.elapsed_time(e1), "distinct": int(len(cnts)), "rows": f_mass}
        res[kind]["distribution"] = dist
        del out, t
    return res


def run_cl3m(args, dev):
    """All-k global counts of the com-orkut-shaped graph (Chung-Lu n = 3M,
    m ~ 128M, exponent 2.0, 2,000 planted communities of 50-120 vertices at
    density 0.8; degeneracy 733): one orient + count_global on the graph
    already in HBM, timed with CUDA events, phases with the classes run one
    after another.  Its tree holds about 1.1e12 nodes, so a count takes on
    the order of 100 s: it is timed once, not K + W times.  Checks: C_1 = n,
    C_2 = m and C_3 = the oracle's triangle enumeration (plain definition,
    no SCT), word for word; every count is exact by construction (the
    device's root-path check ran)."""
    import torch
    import paper_2001_06784_gb300 as pvt
    from paper_2001_06784_gb300 import graphgen
    import oracle
    name = "cl3m_m117m_b2.0_comm2000"
    rp, col = graphgen.workload(name)
    n, m = len(rp) - 1, len(col) // 2
    rpd = torch.from_numpy(rp).to(dev)
    cd = torch.from_numpy(col.view(np.int32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch_flush(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(int(str(dev).split(":")[-1]) if ":" in str(dev) else 0)
    sampler.start()
    e0.record(stream)
    dag = pvt.orient(rpd, cd, profile=True)
    so = dag.stats()
    dag.set_policy(serial=True)
    C = dag.count_global()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    st = dag.stats()
    words = pvt.to_ints(C)
    depths = dag.leaf_depths()
    dag.free()
    del flush
    omega = max(k for k, c in enumerate(words) if c)
    T = oracle.triangles(rp, col, threads=os.cpu_count() or 1)
    ph = dict(st["ms"])
    ph["peel"], ph["orient"] = so["ms"]["peel"], so["ms"]["orient"]
    try:
        alu = pvt.measure_popc_rate(dev) / 1e9
    except Exception:
        alu = POPC_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e9
    names = pvt.Dag.PHASES
    kern = []
    for c in range(1, 7):
        t = ph[names[1 + c]]
        if t > 0:
            a = st["class_words"][c] / (t / 1000.0) / 1e9
            kern.append({"kernel": names[1 + c], "ms": t, "algorithmic": st["class_words"][c], "achieved": a,
                         "unit": "Gop/s", "frac": a / alu, "roots": st["roots"][c]})
    dom = max(kern, key=lambda k: k["ms"])
    return {"workload": name, "n": n, "m": m, "alpha": len(depths) - 2, "omega": omega, "kmax": len(words) - 1,
            "ms": ms, "edges_per_s": m / (ms / 1000.0), "counts": {"C1": words[1], "C2": words[2], "C3": words[3],
                                                                  "C_max": str(max(words))},
            "checks": {"C1_is_n": words[1] == n, "C2_is_m": words[2] == m, "C3_is_oracle_triangles": words[3] == T},
            "sct": {"nodes": st["sct_nodes"], "leaves": st["sct_leaves"], "pivot_words": st["pivot_words"],
                    "leaf_depth_mode": int(np.argmax(depths))},
            "phases_ms": ph, "kernels": kern,
            "roofline": {"bound": "alu", "kernel": dom["kernel"], "achieved": dom["achieved"], "peak": alu,
                         "unit": "Gop/s", "frac": dom["frac"]},
            "clocks": clocks,
            "timing": "one orient + all-k count, CUDA events, classes serialised (policy.serial)"}


def run_graph_replay(args, dev, reps=50):
    """Global counts on a resident small graph (ER n=2000, avg degree 20,
    one 30-clique), called repeatedly: the launch sequence issued directly
    against the replay of its recorded CUDA graph (device time per call,
    CUDA events around each call)."""
    import torch
    import paper_2001_06784_gb300 as pvt
    from paper_2001_06784_gb300 import graphgen
    name = "er2k_d20_clique30"
    rp, col = graphgen.workload(name)
    dag = pvt.orient(torch.from_numpy(rp).to(dev), torch.from_numpy(col.view(np.int32)).to(dev))
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((dag.alpha + 2, dag.min_words), dtype=torch.int64, device=dev)
    res = {"workload": name}
    ref = None
    for form in ("direct", "graph"):
        dag.set_policy(graph=(form == "graph"))
        ms = []
        for i in range(reps + 3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            dag.count_global(out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if i >= 3:
                ms.append((e0.elapsed_time(e1), (time.perf_counter() - t0) * 1000.0))
        got = pvt.to_ints(out)
        ref = got if ref is None else ref
        assert got == ref, "graph replay differs from direct launches"
        res[form] = {"device_ms": float(np.median([a for a, _ in ms])),
                     "host_ms": float(np.median([b for _, b in ms])), "launches": dag.stats()["launches"]}
    dag.free()
    return res


SERVING_CHUNK = 2000  # queries held in host memory at once (about 2 GB of CSR)


def run_serving(args, dev):
    """The query server (continuous batching, large queries on the whole-GPU
    direct path beside the batches) against one launch sequence per graph, on
    the same query stream, in chunks of SERVING_CHUNK queries (the whole
    stream's CSRs do not fit in host memory).  Per chunk: closed-loop
    saturation throughput of each form (one query after another / every
    query submitted at once), then p50/p99 latency with Poisson arrivals at
    0.8 x the plain form's saturation rate (measured on the first chunk).
    Every served result is checked against the plain form's (length, 64-bit
    sum and xor of the words), and the eight smallest queries of the first
    chunk word for word against the oracle."""
    import threading as th
    from concurrent.futures import ThreadPoolExecutor
    import torch
    import paper_2001_06784_gb300 as pvt
    import oracle
    specs = serving_specs(args.serving_queries)
    cfg = dict(mem_budget=64 << 30, max_inflight=4096, max_batch=256, streams=4)

    def digest(a):
        # a 64-bit sum and xor of the result's words (a full hash of the
        # 10-20 MB per-edge tables would cost more than serving them)
        w = np.ascontiguousarray(a).reshape(-1).view(np.uint64)
        return (w.size, int(np.add.reduce(w, dtype=np.uint64)), int(np.bitwise_xor.reduce(w)) if w.size else 0)

    def plain_one(rp, col, kind):
        rpd = torch.from_numpy(rp).to(dev, non_blocking=True)
        cd = torch.from_numpy(col.view(np.int32)).to(dev, non_blocking=True)
        dag = pvt.orient(rpd, cd)
        out = dag.count_global() if kind == "global" else dag.count_local_edge()
        host = out.cpu().numpy().view(np.uint64)
        dag.free()
        return host.reshape((1,) + host.shape) if kind == "global" else host

    lam = None
    edges = 0
    t_sat_plain = t_sat_srv = 0.0
    lat_plain, lat_srv = [], []
    span_plain = span_srv = 0.0
    mismatch = 0
    oracle_ok, n_oracle = True, 0
    for c0 in range(0, len(specs), SERVING_CHUNK):
        qs = serving_graphs(specs[c0:c0 + SERVING_CHUNK])
        edges += sum(len(c) // 2 for _, c, _ in qs)
        if c0 == 0:
            for rp, col, kind in qs[:3]:  # warm-up
                plain_one(rp, col, kind)
            torch.cuda.synchronize(dev)
        # ---- closed loop, plain: one query after another (the checksum of
        # each result is taken with the clock stopped)
        plain_hash = []
        dt = 0.0
        for rp, col, kind in qs:
            t0 = time.perf_counter()
            res = plain_one(rp, col, kind)
            dt += time.perf_counter() - t0
            plain_hash.append(digest(res))
        t_sat_plain += dt
        if lam is None:
            lam = 0.8 * len(qs) / dt
        arrivals = np.cumsum(np.random.default_rng(55 + c0).exponential(1.0 / lam, len(qs)))
        small = sorted(range(len(qs)), key=lambda i: len(qs[i][1]))[:8] if c0 == 0 else []
        kept = {}
        with pvt.Server(**cfg) as sv:
            for rp, col, kind in qs[:3]:  # warm-up
                t = sv.submit(rp, col, kind)
                sv.wait(t)
                sv.result(t)
            # ---- closed loop, served: every query submitted at once (the
            # checksums are taken by helper threads beside the loop)
            with ThreadPoolExecutor(4) as ex:
                t0 = time.perf_counter()
                tickets = [sv.submit(rp, col, kind) for rp, col, kind in qs]
                sums = []
                for i, t in enumerate(tickets):
                    sv.wait(t)
                    words, _ = sv.result(t)
                    sums.append(ex.submit(digest, words))
                    if i in small:
                        kept[i] = words
                t_sat_srv += time.perf_counter() - t0
                mismatch += sum(f.result() != plain_hash[i] for i, f in enumerate(sums))
        for i in small:
            rp, col, kind = qs[i]
            K = kept[i].shape[1] - 1
            ref = oracle.count(rp, col, kmax=K, edge=kind == "edge")
            want = ref["C"] if kind == "global" else oracle.to_int(ref["ce"])
            got = pvt.to_ints(kept[i][0]) if kind == "global" else pvt.to_ints(kept[i])
            oracle_ok = oracle_ok and got == want
            n_oracle += 1
        # ---- open loop, plain: replayed in real time, one query at a time
        t0 = time.perf_counter()
        for (rp, col, kind), ta in zip(qs, arrivals):
            now = time.perf_counter() - t0
            if now < ta:
                time.sleep(ta - now)
            plain_one(rp, col, kind)
            lat_plain.append(time.perf_counter() - t0 - ta)
        span_plain += time.perf_counter() - t0
        # ---- open loop, served: a submitter thread keeps the arrivals,
        # latency measured inside the server (submit -> result ready)
        lat = [None] * len(qs)
        with pvt.Server(**cfg) as sv:
            for rp, col, kind in qs[:3]:  # warm-up
                t = sv.submit(rp, col, kind)
                sv.wait(t)
                sv.result(t)
            tickets = [None] * len(qs)
            t0 = time.perf_counter()

            def submitter():
                for i, ((rp, col, kind), ta) in enumerate(zip(qs, arrivals)):
                    now = time.perf_counter() - t0
                    if now < ta:
                        time.sleep(ta - now)
                    tickets[i] = sv.submit(rp, col, kind)

            thr = th.Thread(target=submitter)
            thr.start()
            for i in range(len(qs)):
                while tickets[i] is None:
                    time.sleep(0.0005)
                sv.wait(tickets[i])
                _, lat[i] = sv.result(tickets[i])
            thr.join()
            span_srv += time.perf_counter() - t0
        lat_srv += lat
        del qs

    def summary(lat, span):
        a = np.asarray(lat) * 1000.0
        return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
                "mean_ms": float(a.mean()), "throughput_qps": len(a) / span, "edges_per_s": edges / span}

    nq = len(specs)
    return {"queries": nq, "chunk": SERVING_CHUNK,
            "stream": "ER or Chung-Lu, n log-uniform 100..50000, avg deg U[5,60], "
                      "global or per-edge (1/2 each), Poisson arrivals, seed 5",
            "edges_total": edges,
            "saturation": {"plain_qps": nq / t_sat_plain, "served_qps": nq / t_sat_srv,
                           "plain_edges_per_s": edges / t_sat_plain, "served_edges_per_s": edges / t_sat_srv,
                           "form": "closed loop: plain one query after another; served all of a chunk at once"},
            "arrival_rate_qps": lam,
            "plain": summary(lat_plain, span_plain), "batched": summary(lat_srv, span_srv),
            "check": {"served_vs_plain_mismatches": int(mismatch), "oracle_sample": n_oracle,
                      "oracle_sample_ok": bool(oracle_ok)}}


def run_profile_case(args, dev):
    """One small case per kernel family, for ncu (`--profile`):
    lanes  orient + global count of the bench graph (the frame phase, k_lanes)
    cta    orient the bench graph, global count k <= 4 with the 129..256
           out-degree class on the block-per-root kernel (k_cta<8>)
    local  per-vertex and per-edge tables of the 500k-vertex graph, k <= 12
           (k_count in MODE_VERTEX / MODE_EDGE)
    peel   orient the bench graph (k_peel, k_peel_tail)"""
    import torch
    import paper_2001_06784_gb300 as pvt
    from paper_2001_06784_gb300 import graphgen
    name = {"lanes": DEFAULT_WORKLOAD, "peel": DEFAULT_WORKLOAD, "cta": DEFAULT_WORKLOAD,
            "local": "cl500k_m8m_b2.3_clq200"}[args.profile]
    rp, col = graphgen.workload(name)
    rpd = torch.from_numpy(rp).to(dev)
    cd = torch.from_numpy(col.view(np.int32)).to(dev)
    dag = pvt.orient(rpd, cd)
    if args.profile == "lanes":
        C = pvt.to_ints(dag.count_global())
        print("profile lanes: omega", max(k for k, c in enumerate(C) if c))
    elif args.profile == "cta":
        dag.set_policy(cta=[0, 0, 0, 0, 1, 0, 0])
        C = pvt.to_ints(dag.count_global(kmax=4))
        print("profile cta: C4", C[4])
    elif args.profile == "local":
        dag.count_local_vertex(kmax=12)
        dag.count_local_edge(kmax=12)
        print("profile local: rows", dag.n, dag.m)
    else:
        print("profile peel: alpha", dag.alpha)
    torch.cuda.synchronize(dev)
    dag.free()


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.profile:
        import torch
        run_profile_case(args, torch.device("cuda", local))
        return

    import torch
    import paper_2001_06784_gb300 as pvt
    from paper_2001_06784_gb300 import graphgen

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    rp_np, col_np = graphgen.workload(args.workload)
    n, m = len(rp_np) - 1, len(col_np) // 2
    rp_h = torch.from_numpy(rp_np).pin_memory()
    col_h = torch.from_numpy(col_np.view(np.int32)).pin_memory()
    rp_d = rp_h.to(dev)
    col_d = col_h.to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # warm-up (also fixes kmax / W for the run)
    dag = None
    for _ in range(max(args.warmup, 1)):
        dag = pvt.orient(rp_d, col_d)
        C = dag.count_global()
        alpha, W = dag.alpha, dag.min_words
        dag.free()
    kmax = alpha + 1
    # launch policy per out-degree class, picked once by the library's
    # autotuner and applied to every step's dag
    dag = pvt.orient(rp_d, col_d)
    policy, tune_ms, Ct = dag.autotune(kmax=kmax, W=W)
    tuned_C = pvt.to_ints(Ct)
    dag.free()
    step_policy = dict(policy, graph=False)

    # ---- device-resident timed steps (L2 flushed between steps)
    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    step_ms, phase_ms, launches, walk = [], [], [], None
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dag = pvt.orient(rp_d, col_d, profile=True)
        so = dag.stats()
        dag.set_policy(**step_policy)
        C = dag.count_global(kmax=kmax, W=W)
        e1.record(stream)
        sc = dag.stats()
        torch.cuda.synchronize(dev)
        step_ms.append(e0.elapsed_time(e1))
        ph = dict(sc["ms"])
        ph["peel"], ph["orient"] = so["ms"]["peel"], so["ms"]["orient"]
        phase_ms.append(ph)
        launches.append(so["launches"] + sc["launches"])
        walk = sc
        dag.free()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    total_s = max_over_ranks(sum(step_ms) / 1000.0, dev)
    ms_per_step = total_s * 1000.0 / args.steps
    value = whole_job_rate(m * args.steps, ws, total_s)
    C_words = C.cpu()
    C_ints = pvt.to_ints(C_words)
    assert tuned_C == C_ints, "autotuner run and timed steps differ"
    omega = max(k for k, c in enumerate(C_ints) if c)

    # ---- the plain form on the same steps: one warp per root, one launch per
    # out-degree class, no work queue (what the persistent form is measured against)
    plain_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dag = pvt.orient(rp_d, col_d)
        dag.set_policy(persistent=False, chunk=1)
        Cp = dag.count_global(kmax=kmax, W=W)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms.append(e0.elapsed_time(e1))
        dag.free()
    assert pvt.to_ints(Cp) == C_ints, "plain and persistent forms differ"
    plain_value = whole_job_rate(m * len(plain_ms), ws, max_over_ranks(sum(plain_ms) / 1000.0, dev))

    # ---- end to end through the public API: pinned host CSR in, counts out
    C_host = torch.empty((kmax + 1, W), dtype=torch.int64).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rp_x = rp_h.to(dev, non_blocking=True)
        col_x = col_h.to(dev, non_blocking=True)
        dag = pvt.orient(rp_x, col_x)
        dag.set_policy(**step_policy)
        Cx = dag.count_global(kmax=kmax, W=W)
        C_host.copy_(Cx, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
        dag.free()
        del rp_x, col_x
    e2e_s = max_over_ranks(sum(e2e_ms) / 1000.0, dev)
    e2e_value = whole_job_rate(m * len(e2e_ms), ws, e2e_s)
    assert pvt.to_ints(C_host) == C_ints, "end-to-end result differs from the device-resident one"

    mean_ph = {k: float(np.mean([p[k] for p in phase_ms])) for k in phase_ms[0]}
    kernels, roofline = kernel_rooflines(args, dev, rp_d, col_d, step_policy, kmax, W, n, m)

    out = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64 words (exact integers)", "data": "synthetic",
           "config": workload_config(args.workload, n, m, alpha, omega),
           "run": {"form": "persistent work queue", "policy": step_policy,
                   "autotune_ms": {c: [round(float(x), 3) for x in tune_ms[i]]
                                   for i, c in enumerate(("chunk4_split", "chunk1_nosplit", "chunk16_split"))},
                   "parallelism": "replicas" if ws > 1 else "single"},
           "roofline": roofline,
           "kernels": kernels,
           "e2e": {"value": e2e_value, "unit": "edges/s", "ms_per_step": e2e_s * 1000.0 / len(e2e_ms),
                   "h2d_bytes_per_step": int(rp_h.numel() * 8 + col_h.numel() * 4),
                   "d2h_bytes_per_step": int(C_host.numel() * 8)},
           "plain": {"value": plain_value, "unit": "edges/s", "ms_per_step": float(np.mean(plain_ms)),
                     "form": "one warp per root, one launch per out-degree class"},
           "gpu_launches": int(np.mean(launches)) * args.steps,
           "clocks": clocks,
           "phases_ms": mean_ph,
           "sct": {"nodes": walk["sct_nodes"], "leaves": walk["sct_leaves"], "pivot_words": walk["pivot_words"],
                   "roots_per_class": walk["roots"], "pivot_words_per_class": walk["class_words"],
                   "frame_words": walk["frame_words"], "frames": walk["frames"]},
           "peel": {"rounds": so["peel_rounds"], "levels": so["peel_levels"]}}

    def section(key, fn):
        """A secondary measurement; its failure is reported in its place
        instead of losing the line.  Progress goes to stderr."""
        t0 = time.perf_counter()
        print(f"bench: {key} ...", file=sys.stderr, flush=True)
        try:
            out[key] = fn()
        except Exception as exc:  # noqa: BLE001 - reported in the JSON line
            out[key] = {"error": f"{type(exc).__name__}: {exc}"}
        print(f"bench: {key} done in {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)

    # ---- launch cost: direct launches vs replay of the recorded CUDA graph
    if rank == 0:
        section("graph_replay", lambda: run_graph_replay(args, dev))

    # ---- local counts (per-vertex, per-edge) on the 500k-vertex graph
    if rank == 0 and not args.no_local:
        section("local", lambda: run_local(args, dev, flush))
    del flush

    # ---- all-k counts of the 128M-edge com-orkut-shaped graph, timed once
    if rank == 0 and not args.no_cl3m:
        section("cl3m_allk", lambda: run_cl3m(args, dev))

    # ---- serving: Poisson stream of independent queries (rank 0 only)
    if rank == 0 and args.serving_queries > 0:
        section("serving", lambda: run_serving(args, dev))

    # ---- CPU baseline: the oracle, whole workload, every host core (the
    # paper's parallel scheme) and one core (its sequential form); also
    # confirms this run's counts bit-exactly
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        ref = oracle.count(rp_np, col_np, kmax=kmax, threads=cores)
        dt = time.perf_counter() - t0
        seq = None
        if not args.no_sequential:
            t0 = time.perf_counter()
            ref1 = oracle.count(rp_np, col_np, kmax=kmax, threads=1)
            dt1 = time.perf_counter() - t0
            seq = {"value": m / dt1, "unit": "edges/s", "cores": 1, "seconds": dt1,
                   "sample": "whole workload, sequential oracle, one run", "parity": ref1["C"] == C_ints}
        out["cpu_baseline"] = {"value": m / dt, "unit": "edges/s", "cores": cores, "cpu": cpu_model(),
                               "kind": "oracle", "sample": "whole workload, root-parallel oracle, one run",
                               "seconds": dt, "sequential": seq}
        out["parity"] = "bit-exact" if ref["C"] == C_ints else "MISMATCH"
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
