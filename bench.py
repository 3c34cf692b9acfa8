"""Benchmark of the sketched |N(u) ∩ N(v)| hot path on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W]
                    [--workload rmat24|rmat24_b50|rmat22|rmat20|variants20|kmv20|er4096|batch4096|serve22|jp22|
                                clique20]
                    [--impl ours|reference]

A step is one pass of the whole sketched path over the synthetic graph of the
workload, starting from the CSR resident in HBM: the upper-edge index, the
sketches of every neighbourhood, and one fused intersection pass per sketch
(per-edge estimate, triangle-count histogram, per-vertex sums, LCC). The
metric is sketched edge intersections per second: one (u, v) estimator
evaluation on one sketch. The exact GPU intersection is the comparison: it is
timed in the same run, outside the step, and gives the estimate's error.

--impl reference times the CPU oracle (oracle/) on a bounded sample of the
same workload on the host cores. Under torchrun (N > 1) every rank runs an
independent replica of the workload (no collective on the data path); the
time is the maximum over ranks and the value the sum of the ranks' work.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import struct
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "sketched edge intersections/s"

# workload -> generator + sketch configuration
WORKLOADS = {
    # R-MAT scale 24, edge factor 32, Bloom at 25% of CSR bytes (b = 2), k-Hash k = 64, exact comparison
    "rmat24": dict(gen=("rmat", 24, 32, 24), budget=0.25, b=2, khash=64, onehash=None, jaccard=False),
    "rmat24_b50": dict(gen=("rmat", 24, 32, 24), budget=0.50, b=2, khash=64, onehash=None, jaccard=False),
    # the same recipe at scale 22 (a quarter of the size): the profiling case for ncu
    "rmat22": dict(gen=("rmat", 22, 32, 22), budget=0.25, b=2, khash=64, onehash=None, jaccard=False),
    # R-MAT scale 20, edge factor 16, Bloom at 25% (b = 2), 1-Hash k = 32, TC + LCC + per-edge Jaccard
    "rmat20": dict(gen=("rmat", 20, 16, 20), budget=0.25, b=2, khash=None, onehash=32, jaccard=True),
    # the estimator variants on R-MAT scale 20 / edge factor 16: Bloom at 25% (b = 2) read by AND, OR and
    # the single-set form, with per-edge Jaccard, overlap and total-neighbour similarities
    "variants20": dict(gen=("rmat", 20, 16, 20), budget=0.25, b=2, khash=None, onehash=None, jaccard=True,
                       similarity=True, bloom_variants=("or", "ss")),
    # Erdos-Renyi n = 4096, average degree 16, Bloom 256 bits b = 2, k-Hash k = 16
    "er4096": dict(gen=("er", 4096, 16.0, 1), bits=256, b=2, khash=16, onehash=None, jaccard=False),
    # KMV (Sec. IX) beside the 1-Hash estimator on the same 1-Hash sketch (k = 32), R-MAT scale 20 / ef 16
    "kmv20": dict(gen=("rmat", 20, 16, 20), budget=0.25, b=2, khash=None, onehash=32, onehash_variants=("kmv",),
                  jaccard=True),
    # 4096 graphs (half Erdos-Renyi, half R-MAT), n log-uniform in [2^8, 2^16], average degree
    # lognormal (median 12, clipped to 4..64); per-graph Bloom length and hash count from the
    # autotuner at 25% of each graph's CSR bytes; one captured batch run against one launch per graph
    "batch4096": dict(batch=4096, budget=0.25, seed=1),
    # serving: resident R-MAT scale 22, edge factor 16, Bloom 512 bits b = 2 and k-Hash k = 32 on the
    # device; pair requests of lognormal size (median 256, sigma 2, clipped to 1..65536), half existing
    # edges and half random pairs, and induced-subgraph triangle counts of BFS balls of 10^U(3,6) edges
    # Jarvis-Patrick clustering on R-MAT scale 22, edge factor 16: Bloom at 25% (b = 2) and k-Hash k = 32,
    # threshold tau = 4 common neighbours; exact clustering as the comparison
    "jp22": dict(jp=True, gen=("rmat", 22, 16, 22), budget=0.25, b=2, khash=32, tau=4.0),
    # 4-clique counting on R-MAT scale 20, edge factor 16: Bloom filters of the oriented neighbourhoods at
    # 256 bits, b = 2; exact 4-clique count as the comparison
    "clique20": dict(clique=True, gen=("rmat", 20, 16, 20), bits=256, b=2),
    "serve22": dict(serve=True, gen=("rmat", 22, 16, 22), bits=512, b=2, khash=32, pair_requests=2000,
                    subgraph_requests=12, subgraph_share=0.02),
}


# ---------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    if ws > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group(backend=backend)


def max_over_ranks(x: float, ws: int, device=None) -> float:
    if ws <= 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        torch.distributed.barrier()


def generate(workload: str, device):
    from paper_2208_11469_gb300 import synth
    if "batch" in WORKLOADS[workload]:
        return generate_batch(workload, device)
    if any(k in WORKLOADS[workload] for k in ("serve", "jp", "clique")):
        kind, scale, ef, seed = WORKLOADS[workload]["gen"]
        return synth.rmat(scale, ef, seed=seed, device=device)
    kind, *a = WORKLOADS[workload]["gen"]
    if kind == "rmat":
        scale, ef, seed = a
        return synth.rmat(scale, ef, seed=seed, device=device)
    n, deg, seed = a
    return synth.erdos_renyi(n, deg, seed=seed, device=device)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        # nvidia-smi numbers GPUs physically; address this device by UUID
        try:
            u = str(torch.cuda.get_device_properties(index).uuid)
            self.index = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def budget_bits(s, n, nnz):
    """Filter length for storage budget s of the CSR bytes (the sizing rule of
    pg_bloom_bits_for_budget, restated for the CPU leg)."""
    words = int(s * (4.0 * (n + 1) + 4.0 * nnz) * 8.0 / (64.0 * n)) if n > 0 else 1
    return 64 * min(16, max(1, words))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# int32 ALU-pipe lane operations per SM per clock (16 lanes in each of the
# four SM sub-partitions), the rate of integer add / logical / shift / min.
ALU_OPS_PER_SM_CLOCK = 64
# ALU-pipe operations per k-Hash hash evaluation in the builders' source: one
# XOR with the seed's pre-image, two shift + XOR pairs and one min (the two
# multiplies run on the multiply-add pipe).
ALU_OPS_PER_HASH = 6


def alu_peak(sm_mhz):
    """Integer ALU-pipe peak of this GPU at the sampled SM clock (ops/s)."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * ALU_OPS_PER_SM_CLOCK * float(sm_mhz) * 1e6, sms


# The sources a pass's DRAM traffic depends on: the pass kernels, the shared
# device code and the edge index (whose list order decides the L2 reuse).
PASS_SOURCES = ("pg_intersect.cu", "pg_internal.cuh", "pg_index.cu")


def code_only(src: str) -> str:
    """C++/CUDA source without its comments, whitespace runs collapsed to one
    space (string and character literals kept as they are), so that the
    fingerprint changes with the code and not with its comments."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_fingerprint() -> str:
    """sha256 over the code of the pass sources (comments removed), in
    PASS_SOURCES order."""
    h = hashlib.sha256()
    for f in PASS_SOURCES:
        src = open(os.path.join(ROOT, "paper_2208_11469_gb300", "csrc", f), encoding="utf-8").read()
        h.update(code_only(src).encode("utf-8"))
    return h.hexdigest()


def profiled_traffic(name: str):
    """DRAM bytes per launch from a committed ncu summary, if the pass
    sources are unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    if not m or not h or source_fingerprint() != h.group(1):
        return None
    return float(m.group(1))


# ------------------------------------------------------------- our path
class Pipeline:
    """Device buffers and the step of one workload."""

    def __init__(self, workload: str, row_ptr, col):
        from paper_2208_11469_gb300 import pg
        self.pg = pg
        cfg = WORKLOADS[workload]
        self.cfg = cfg
        dev = row_ptr.device
        self.g = pg.graph(row_ptr, col, build_index=True)
        g = self.g
        self.n, self.nnz, self.m = g.n, g.nnz, g.m
        bits = cfg.get("bits") or pg.bloom_bits_for_budget(cfg["budget"], g.n, g.nnz)
        self.bits = bits
        self.build_ws = torch.empty(max(pg.build_workspace_bytes(g), 16), dtype=torch.uint8, device=dev)
        self.build_ws_side = torch.empty_like(self.build_ws)  # builds on the side stream
        self.passes = []  # (name, sketch, estimator)
        bf = pg.alloc_sketch(g, pg.SK_BLOOM, bits=bits, b=cfg["b"], seed=1)
        self.passes.append(("bloom", bf, pg.EST_BF_AND))
        # further estimators on the same Bloom sketch (built once per step)
        for nm in cfg.get("bloom_variants", ()):
            self.passes.append(("bloom_" + nm, bf, {"or": pg.EST_BF_OR, "ss": pg.EST_BF_SS, "l": pg.EST_BF_L}[nm]))
        if cfg["khash"]:
            self.passes.append(("khash", pg.alloc_sketch(g, pg.SK_KHASH, k=cfg["khash"], seed=1), pg.EST_KH))
        if cfg["onehash"]:
            oh = pg.alloc_sketch(g, pg.SK_1HASH, k=cfg["onehash"], seed=1)
            self.passes.append(("onehash", oh, pg.EST_1H))
            # further estimators on the same 1-Hash sketch (built once per step)
            for nm in cfg.get("onehash_variants", ()):
                self.passes.append(("onehash_" + nm, oh, {"kmv": pg.EST_1H_KMV}[nm]))
        self.ws = {name: pg.workspace(g, sk, est) for name, sk, est in self.passes}
        self.out = {}
        for name, sk, est in self.passes:
            o = dict(tc=pg.tc_result_buffer(dev), lcc=torch.empty(g.n, dtype=torch.float32, device=dev),
                     tri=torch.empty(g.n, dtype=torch.float64, device=dev))
            if cfg["jaccard"]:
                o["edge_cn"] = torch.empty(self.m, dtype=torch.float32, device=dev)
                o["edge_jac"] = torch.empty(self.m, dtype=torch.float32, device=dev)
            if cfg.get("similarity"):
                o["edge_overlap"] = torch.empty(self.m, dtype=torch.float32, device=dev)
                o["edge_total"] = torch.empty(self.m, dtype=torch.float32, device=dev)
            self.out[name] = o
        self.index_events = None
        self.side = torch.cuda.Stream(device=dev)

    def sketched_per_step(self) -> int:
        return self.m * len(self.passes)

    def sketches(self):
        """The distinct sketches of the step, in build order."""
        out, seen = [], set()
        for _, sk, _ in self.passes:
            if id(sk) not in seen:
                seen.add(id(sk))
                out.append(sk)
        return out

    def step(self, ev=None, builds=True, csr_stream=None, prebuilt=()):
        """One pass of the hot path. ev: optional dict name -> (start, end) events.
        builds=False: the sketches are already built (by upload_build);
        prebuilt: ids of the sketches already built (the others are built here);
        csr_stream: the stream that uploaded the CSR (the side stream then waits
        for it alone, beside the builds' tail on the launching stream).

        The edge index and the sketch builds depend only on the CSR, so they
        run on two streams: the index and then the Bloom builds (bound by memory
        latency and issue) on a side stream, beside the MinHash builds (bound by
        the integer ALU) on the launching stream; each stream has its own build
        workspace. The passes wait for both."""
        pg, g = self.pg, self.g
        s = torch.cuda.current_stream()
        side = self.side if (builds or csr_stream is not None) else s

        def mark(name, i, stream=None):
            if ev is not None:
                ev[name][i].record(stream or s)

        def build(name, sk, stream, ws):
            mark("build_" + name, 0, stream)
            if sk.kind == pg.SK_BLOOM:
                pg.build_bloom(g, sk.bits, sk.b, sk.seed, out=sk, workspace=ws)
            else:
                pg.build_minhash(g, sk.kind, sk.k, sk.seed, out=sk, workspace=ws)
            mark("build_" + name, 1, stream)

        todo, seen = [], set(prebuilt) if builds else {id(sk) for _, sk, _ in self.passes}
        for name, sk, est in self.passes:
            if id(sk) not in seen:
                seen.add(id(sk))
                todo.append((name, sk))
        if side is not s:
            side.wait_stream(s if csr_stream is None else csr_stream)
        with torch.cuda.stream(side):
            mark("index", 0, side)
            pg.build_edge_index_into(g)
            mark("index", 1, side)
            for name, sk in todo:
                if sk.kind == pg.SK_BLOOM:
                    build(name, sk, side, self.build_ws_side)
        for name, sk in todo:
            if sk.kind != pg.SK_BLOOM:
                build(name, sk, s, self.build_ws)
        if side is not s:
            s.wait_stream(side)
        for name, sk, est in self.passes:
            mark("pass_" + name, 0)
            pg.analyze(g, sk, est, ws=self.ws[name], **self.out[name])
            mark("pass_" + name, 1)

    def event_names(self):
        builds, seen = [], set()
        for name, sk, _ in self.passes:
            if id(sk) not in seen:
                seen.add(id(sk))
                builds.append("build_" + name)
        return ["index"] + builds + ["pass_" + p[0] for p in self.passes]

    def results(self):
        return {name: self.pg.read_tc_result(self.out[name]["tc"]) for name, _, _ in self.passes}


def algorithmic_bytes(pipe: Pipeline, name: str) -> float:
    """Algorithmic DRAM bytes of one fused intersection pass:
    per undirected edge the gathered neighbour sketch row (payload bytes) plus
    its CSR entry and the two row offsets of v (degree) for MinHash; per vertex
    its own sketch row, its two row offsets and upper offset, and the outputs
    (T as double, LCC as float)."""
    sk = [p for p in pipe.passes if p[0] == name][0][1]
    est = [p for p in pipe.passes if p[0] == name][0][2]
    payload = sk.bits / 8 if sk.kind == pipe.pg.SK_BLOOM else 4 * sk.k
    per_edge = payload + 4 + (8 if sk.kind != pipe.pg.SK_BLOOM or est == pipe.pg.EST_BF_OR else 0)
    per_vertex = payload + 8 + 4 + 8 + 4
    if pipe.cfg["jaccard"]:
        per_edge += 8
    if pipe.cfg.get("similarity"):
        per_edge += 8
    return pipe.m * per_edge + pipe.n * per_vertex


def time_steps(pipe: Pipeline, steps: int, warmup: int, ws: int):
    for _ in range(warmup):
        pipe.step()
    torch.cuda.synchronize()
    names = pipe.event_names()
    evs = [{nm: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for nm in names}
           for _ in range(steps)]
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    launches0 = pipe.pg.kernel_launches()
    barrier(ws)
    torch.cuda.synchronize()
    marks[0].record()
    for i in range(steps):
        pipe.step(evs[i])
        marks[i + 1].record()
    torch.cuda.synchronize()
    barrier(ws)
    launches = pipe.pg.kernel_launches() - launches0
    total_ms = marks[0].elapsed_time(marks[-1])
    per = {nm: float(np.mean([e[nm][0].elapsed_time(e[nm][1]) for e in evs])) for nm in names}
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(steps)]
    return total_ms / steps, per, launches, step_stats(step_ms)


def step_stats(ms):
    """Median of the per-step times and its 95% non-parametric confidence
    interval (order statistics of a Binomial(K, 1/2) around the median; the
    whole range below 6 steps)."""
    x = np.sort(np.asarray(ms, dtype=np.float64))
    k = x.size
    if k == 0:
        return None
    lo, hi = 0, k - 1
    if k >= 6:
        from math import comb
        # the median lies below x_(lo) (0-based) with probability P(Bin(k, 1/2) <= lo): take the
        # largest lo with that at most 2.5%, and the mirror image above
        cdf, j = 0.0, 0
        while True:
            nxt = cdf + comb(k, j) / 2.0**k
            if nxt > 0.025:
                break
            cdf, j = nxt, j + 1
        lo, hi = j - 1, k - j
    return {"median": float(np.median(x)), "ci95": [float(x[lo]), float(x[hi])], "steps": int(k)}


def time_build_alone(pipe: Pipeline, sk, reps: int = 3) -> float:
    """Mean ms of one MinHash build of sk with nothing else on the GPU (one
    untimed build first)."""
    pg = pipe.pg
    build = lambda: pg.build_minhash(pipe.g, sk.kind, sk.k, sk.seed, out=sk, workspace=pipe.build_ws)
    build()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(reps):
        build()
    end.record()
    torch.cuda.synchronize()
    return start.elapsed_time(end) / reps


def h2d_rate(dev_t, host_t) -> float:
    """GB/s of one copy of host_t (page-locked) into dev_t (same bytes) on the current stream:
    the machine's host-to-device rate, which bounds the end-to-end step."""
    dev_t.copy_(host_t, non_blocking=True)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    dev_t.copy_(host_t, non_blocking=True)
    end.record()
    torch.cuda.synchronize()
    return host_t.numel() * host_t.element_size() / (start.elapsed_time(end) * 1e-3) / 1e9


def e2e_steps(pipe: Pipeline, host_rp, host_col, steps: int):
    """The same step through the public API from pinned host buffers: the CSR
    copy host->device and the results device->host are inside the timing.
    The upload goes through pg_upload_build, which copies the CSR in row
    chunks on a copy stream and builds the MinHash sketches of each chunk
    while the next one is copied; as soon as the last chunk has landed the
    edge index and then the Bloom build run on a side stream (beside the
    remaining MinHash builds), and the passes follow both."""
    pg = pipe.pg
    g = pipe.g
    d2h = []
    for name, _, _ in pipe.passes:
        o = pipe.out[name]
        d2h.append((o["lcc"], torch.empty(o["lcc"].shape, dtype=o["lcc"].dtype, pin_memory=True)))
        d2h.append((o["tc"], torch.empty(o["tc"].shape, dtype=o["tc"].dtype, pin_memory=True)))
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    chunked = [sk for sk in pipe.sketches() if sk.kind != pg.SK_BLOOM]
    copy = torch.cuda.Stream(device=g.device)

    def one():
        pg.upload_build(g, host_rp, host_col, chunked, workspace=pipe.build_ws, copy_stream=copy)
        pipe.step(csr_stream=copy, prebuilt={id(sk) for sk in chunked})
        for dev_t, host_t in d2h:
            host_t.copy_(dev_t, non_blocking=True)

    one()  # untimed: the first upload's one-off costs stay out of the mean
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    start.record()
    for _ in range(steps):
        one()
    end.record()
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3 / steps
    h2d = host_rp.numel() * 4 + host_col.numel() * 4
    d2h_bytes = sum(h.numel() * h.element_size() for _, h in d2h)
    return start.elapsed_time(end) / steps, wall, h2d, d2h_bytes


def tc_deviation_bounds(row_ptr, passes, delta: float = 0.05) -> dict:
    """Thm. 7.1: the deviation t with P(|TC - TC^| >= t) <= delta, per pass.
    Bloom AND (when b * max degree <= 0.499 l log l; the (1 + o(1)) factor
    dropped): t = sqrt(2 m^2 C / (9 delta)), C the MSE bound of Prop. 4.1 at
    the maximum degree; 1-Hash / k-Hash: the smaller t of the two Hoeffding
    forms, (sum d^2) sqrt(ln(2/delta) / (18 k)) and sqrt(4 (max d + 1)
    (sum d^3) ln(2/delta) / (9 k)). passes: (name, kind, l, b, k) tuples;
    None for estimators the theorem does not cover."""
    rp = np.asarray(row_ptr.cpu().numpy() if hasattr(row_ptr, "cpu") else row_ptr, dtype=np.int64)
    d = np.diff(rp).astype(np.float64)
    m = float(d.sum()) / 2.0
    dmax = float(d.max()) if d.size else 0.0
    s2, s3 = float(np.sum(d * d)), float(np.sum(d * d * d))
    lg = math.log(2.0 / delta)
    out = {}
    for name, kind, l, b, k in passes:
        if kind == "bloom_and":
            if b * dmax > 0.499 * l * math.log(l):
                out[name] = {"t": None, "reason": "b * max degree > 0.499 l log l: the bound does not apply"}
                continue
            C = math.exp(dmax * b / (l - 1)) * l / b**2 - l / b**2 - dmax / b
            out[name] = {"t": math.sqrt(2.0 * m * m * max(C, 0.0) / (9.0 * delta))}
        elif kind == "minhash":
            t1 = s2 * math.sqrt(lg / (18.0 * k))
            t2 = math.sqrt(4.0 * (dmax + 1.0) * s3 * lg / (9.0 * k))
            out[name] = {"t": min(t1, t2)}
        else:
            out[name] = None
    return out


def exact_comparison(pipe: Pipeline):
    pg, g = pipe.pg, pipe.g
    ws = pg.workspace(g, None, pg.EST_EXACT)
    tc = pg.tc_result_buffer(g.device)
    pg.triangle_count(g, None, pg.EST_EXACT, ws=ws, out=tc, read=False)  # warm
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pg.triangle_count(g, None, pg.EST_EXACT, ws=ws, out=tc, read=False)
    b.record()
    torch.cuda.synchronize()
    res = pg.read_tc_result(tc)
    del ws
    return a.elapsed_time(b), res


# ------------------------------------------------------- CPU oracle leg
def oracle_passes(cfg, bits):
    """The passes of the workload's step as the oracle's pass descriptors."""
    from oracle import oracle as O
    out = [dict(name="bloom", est=O.EST_BF_AND, l=bits, b=cfg["b"], k=0)]
    for nm in cfg.get("bloom_variants", ()):
        out.append(dict(name="bloom_" + nm, est={"or": O.EST_BF_OR, "ss": O.EST_BF_SS, "l": O.EST_BF_L}[nm],
                        l=bits, b=cfg["b"], k=0))
    if cfg.get("khash"):
        out.append(dict(name="khash", est=O.EST_KH, l=0, b=0, k=cfg["khash"]))
    if cfg.get("onehash"):
        out.append(dict(name="onehash", est=O.EST_1H, l=0, b=0, k=cfg["onehash"]))
        for nm in cfg.get("onehash_variants", ()):
            out.append(dict(name="onehash_" + nm, est={"kmv": O.EST_1H_KMV}[nm], l=0, b=0, k=cfg["onehash"]))
    return out


def host_sub_csr(rp, col_d, rows):
    """The rows `rows` (host int64 ids) of the device CSR as a host sub-CSR
    whose entries keep the graph's neighbour ids (a sketch row depends only on
    its own row, so its sketch equals the whole graph's)."""
    starts = rp[rows]
    lens = rp[rows + 1] - starts
    sub_rp = np.zeros(rows.size + 1, np.int64)
    sub_rp[1:] = np.cumsum(lens)
    idx = np.repeat(starts - sub_rp[:-1], lens) + np.arange(int(sub_rp[-1]), dtype=np.int64)
    sub_col = col_d[torch.from_numpy(idx).to(col_d.device)].cpu().numpy().astype(np.int32)
    return sub_rp.astype(np.int32), sub_col


class OracleLeg:
    """The CPU oracle timed on a bounded sample of the workload, extrapolated
    to the whole graph.

    Every phase of the oracle is per row (sketch builds, Sec. II-D) or per
    edge (counts, estimates, totals and per-vertex sums, Sec. IV and VII), so
    the whole-graph time is
        T = t_build(R sampled rows) * n / R + t_pass(E sampled pairs) * m / E
    with the rows drawn uniformly (an unbiased estimate of the whole build)
    and each pair's endpoints drawn with probability proportional to degree,
    as the endpoints of a uniformly drawn edge are, from a table of copies of
    the sampled rows as large as the whole graph's sketch tables (at most
    TABLE_BYTES per process), so that the pass misses the CPU caches as a
    whole-graph pass does. The serial leg runs the chunks one after another
    on one core; the all-core leg runs one chunk per core, each in its own
    process, and its times are the slowest chunk's."""

    TABLE_BYTES = 768 << 20

    def __init__(self, row_ptr_d, col_d, cfg, bits, seed=0):
        from oracle import oracle as O
        O.build()
        O.lib()
        self.rp = row_ptr_d.cpu().numpy().astype(np.int64)
        self.col_d = col_d
        self.n = self.rp.size - 1
        self.nnz = int(self.rp[-1])
        self.m = self.nnz // 2  # simple symmetric generated graphs
        self.passes = oracle_passes(cfg, bits)
        from oracle import sample_timing as ST
        keys = {ST.sketch_key(p) for p in self.passes}
        # oracle row bytes: Bloom one byte per bit, MinHash k int32
        self.row_bytes = sum(key[1] if key[0] == "bloom" else 4 * key[1] for key in keys)
        self.rng = np.random.default_rng(seed)
        self.order = self.rng.permutation(self.n)
        self.next_row = 0
        self.cores = max(1, os.cpu_count() or 1)
        # calibration chunk: per-row build and per-pair pass costs
        ch = self.chunks(min(self.n, 20000), 20000, 1)[0]
        r = ST.time_chunk(ch["rp"], ch["cl"], self.passes, ch["pairs"], ch["table_rows"], pair_seed=ch["pair_seed"])
        self.c_row = r["build_s"] / max(r["rows"], 1)
        self.c_pair = r["pass_s"] / max(r["pairs"], 1)

    def chunks(self, R, E, parts):
        """parts chunks of R / parts fresh uniformly drawn rows each and
        E / parts pairs each."""
        out = []
        table_rows = int(min(self.n, self.TABLE_BYTES // max(self.row_bytes, 1)))
        for i in range(parts):
            r = max(1, R // parts)
            if self.next_row + r > self.n:
                self.order = self.rng.permutation(self.n)
                self.next_row = 0
            rows = np.sort(self.order[self.next_row:self.next_row + r])
            self.next_row += r
            rp, cl = host_sub_csr(self.rp, self.col_d, rows)
            out.append(dict(rp=rp, cl=cl, rows=rows, pairs=max(1, E // parts), table_rows=table_rows,
                            pair_seed=int(self.rng.integers(1 << 31))))
        return out

    def sized(self, target_s, parts):
        """Chunks sized for about target_s seconds of serial oracle work
        (60% builds, 40% passes)."""
        R = int(min(self.n, max(parts, 0.6 * target_s / max(self.c_row, 1e-12))))
        E = int(min(5_000_000, max(1000 * parts, 0.4 * target_s / max(self.c_pair, 1e-12))))
        return self.chunks(R, E, parts)

    def _rate(self, build_s, pass_s, R, E):
        T = build_s * self.n / R + pass_s * self.m / E
        return len(self.passes) * self.m / T, T

    def serial(self, chunks):
        from oracle import sample_timing as ST
        build = pss = 0.0
        R = E = 0
        for ch in chunks:
            r = ST.time_chunk(ch["rp"], ch["cl"], self.passes, ch["pairs"], ch["table_rows"],
                              pair_seed=ch["pair_seed"])
            build += r["build_s"]
            pss += r["pass_s"]
            R += r["rows"]
            E += r["pairs"]
        rate, T = self._rate(build, pss, R, E)
        return {"value": rate, "cores": 1, "rows": R, "pairs": E, "build_s": build, "pass_s": pss,
                "whole_graph_s": T}

    def parallel(self, chunks):
        """One subprocess per chunk (plain `python -m oracle.sample_timing`,
        no torch, no CUDA), all started together."""
        import tempfile
        with tempfile.TemporaryDirectory() as tmp:
            procs = []
            for i, ch in enumerate(chunks):
                src = os.path.join(tmp, f"c{i}.npz")
                np.savez(src, rp=ch["rp"], cl=ch["cl"], pairs=ch["pairs"], table_rows=ch["table_rows"], seed=1,
                         pair_seed=ch["pair_seed"], passes=json.dumps(self.passes))
                dst = os.path.join(tmp, f"r{i}.json")
                env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
                procs.append((subprocess.Popen([sys.executable, "-m", "oracle.sample_timing", src, dst], cwd=ROOT,
                                               env=env), dst))
            res = []
            for pr, dst in procs:
                if pr.wait() != 0:
                    raise RuntimeError("oracle timing subprocess failed")
                with open(dst) as f:
                    res.append(json.load(f))
        R = sum(r["rows"] for r in res)
        E = sum(r["pairs"] for r in res)
        build = max(r["build_s"] for r in res)
        pss = max(r["pass_s"] for r in res)
        rate, T = self._rate(build, pss, R, E)
        return {"value": rate, "cores": len(chunks), "rows": R, "pairs": E, "build_s": build, "pass_s": pss,
                "whole_graph_s": T}

    def describe(self, leg):
        return (f"{leg['rows']} uniformly drawn rows (sketch builds) and {leg['pairs']} pairs with degree-weighted "
                f"endpoints over tables of copies of those rows as large as the graph's (<= 768 MiB per process) "
                f"({len(self.passes)} passes: counts, estimates, TC sum, per-vertex sums) of the "
                f"n={self.n}, m={self.m} graph; whole-graph time = build * n/rows + pass * m/pairs "
                f"= {leg['whole_graph_s']:.1f} s on {leg['cores']} core(s), oracle C/numpy unchanged, gcc -O3")


def cpu_baseline(pipe_or_none, rp, cl, cfg, bits, serial_s=12.0):
    """Both legs on the same sample: serial (1 core) and all host cores."""
    leg = OracleLeg(rp, cl, cfg, bits, seed=0)
    chunks = leg.sized(serial_s, leg.cores)
    ser = leg.serial(chunks)
    par = leg.parallel(chunks)
    return {"value": par["value"], "unit": "intersections/s", "cores": par["cores"], "kind": "oracle",
            "sample": leg.describe(par), "serial": dict(ser, sample=leg.describe(ser)),
            "all_cores": par, "formula": "passes * m / (t_build * n / rows + t_pass * m / pairs)"}


def parity_sample(pipe, seed=0, vertices=32, max_deg=16, hubs=8):
    """Bit-exact check of the bench graph's own sketches and counts against the
    oracle on a sample, after the timed steps: the sketch rows of `vertices`
    random vertices of degree 2..max_deg, of all their neighbours and of the
    `hubs` highest-degree vertices; the per-pair integer counts of every edge
    at the sampled vertices and of every pair of hubs (pg_edge_counts); and
    T_v and LCC of the sampled vertices from the step's own fused pass (1e-9
    and 1e-5 relative)."""
    from oracle import oracle as O
    pg, g = pipe.pg, pipe.g
    rp = g.row_ptr.cpu().numpy().astype(np.int64)
    d = np.diff(rp)
    rng = np.random.default_rng(seed)
    cand = np.flatnonzero((d >= 2) & (d <= max_deg))
    vs = np.sort(rng.choice(cand, size=min(vertices, cand.size), replace=False))
    top = np.argsort(d)[::-1][:hubs]
    nb_rp, nb_cl = host_sub_csr(rp, g.col, vs)
    rows = np.unique(np.concatenate([vs, nb_cl.astype(np.int64), top]))
    srp, scl = host_sub_csr(rp, g.col, rows)
    loc = {int(v): i for i, v in enumerate(rows)}
    # pairs: (v, u) for every neighbour u of a sampled v, then every pair of hubs
    pu = np.repeat(vs, np.diff(nb_rp))
    pv = nb_cl.astype(np.int64)
    hu, hv = np.triu_indices(top.size, 1)
    pu = np.concatenate([pu, top[hu]])
    pv = np.concatenate([pv, top[hv]])
    lu = np.array([loc[int(x)] for x in pu], np.int32)
    lv = np.array([loc[int(x)] for x in pv], np.int32)
    nv_pairs = int(nb_cl.size)
    pairs_d = torch.from_numpy(np.stack([pu, pv], 1).astype(np.int32)).to(g.device)
    out = {}
    for name, sk, est in pipe.passes:
        kw = dict(l=sk.bits, b=sk.b, k=sk.k)
        rows_t = torch.from_numpy(rows).to(g.device)
        if sk.kind == pg.SK_BLOOM:
            osk = O.bloom_bits(srp, scl, sk.bits, sk.b, sk.seed)
            words = sk.bits // 64
            want = O.bloom_pack(osk, words)
            got = sk.data.view(torch.int64).view(g.n, sk.stride // 8)[rows_t, :words].cpu().numpy().view(np.uint64)
        elif sk.kind == pg.SK_KHASH:
            osk = O.khash(srp, scl, sk.k, sk.seed)
            want = O.khash_values(osk, sk.seed)
            got = sk.data.view(torch.int32).view(g.n, sk.stride // 4)[rows_t, :sk.k].cpu().numpy().view(np.uint32)
        else:
            osk = O.onehash(srp, scl, sk.k, sk.seed)
            want = O.onehash_values(osk, sk.seed)
            got = sk.data.view(torch.int32).view(g.n, sk.stride // 4)[rows_t, :sk.k].cpu().numpy().view(np.uint32)
        row_bad = int(np.count_nonzero(np.any(got != want, axis=1)))
        cnt = O.pair_counts(srp, scl, est, osk, lu, lv, seed=sk.seed)
        gc, _, _ = pg.edge_counts(g, sk, est, pairs_d)
        cnt_bad = int(np.count_nonzero(gc.cpu().numpy() != np.asarray(cnt["count"], np.int32)))
        e = O.pair_estimates(srp, est, cnt, lu, lv, **kw)
        T = np.zeros(vs.size)
        np.add.at(T, np.searchsorted(vs, pu[:nv_pairs]), e[:nv_pairs])
        T *= 0.5
        dv = d[vs].astype(np.float64)
        lcc_want = 2.0 * T / (dv * (dv - 1.0))
        vs_t = torch.from_numpy(vs).to(g.device)
        T_got = pipe.out[name]["tri"][vs_t].cpu().numpy()
        lcc_got = pipe.out[name]["lcc"][vs_t].cpu().numpy().astype(np.float64)
        t_rel = float(np.max(np.abs(T_got - T) / np.maximum(np.abs(T), 1e-300))) if vs.size else 0.0
        l_rel = float(np.max(np.abs(lcc_got - lcc_want) / np.maximum(np.abs(lcc_want), 1e-30))) if vs.size else 0.0
        out[name] = {"rows": int(rows.size), "row_mismatches": row_bad, "pairs": int(pu.size),
                     "count_mismatches": cnt_bad, "vertices": int(vs.size), "T_max_rel": t_rel,
                     "lcc_max_rel": l_rel,
                     "ok": row_bad == 0 and cnt_bad == 0 and t_rel <= 1e-9 and l_rel <= 1e-5}
    return out


# ------------------------------------------------------------ batching
def generate_batch(workload: str, device):
    """The graph mix, its autotuned Bloom parameters, and the graphs ordered
    by (bits, b) and concatenated block-diagonally. Returns (parts, cfg,
    row_ptr, col, voff) with parts and cfg in batch order."""
    from paper_2208_11469_gb300 import pg, synth
    w = WORKLOADS[workload]
    parts = synth.batch_mix(w["batch"], seed=w["seed"], device=device)
    n = np.array([int(rp.numel()) - 1 for rp, _ in parts], dtype=np.int32)
    nnz = np.array([int(cl.numel()) for _, cl in parts], dtype=np.int64)
    cfg = pg.batch_autotune(n, nnz, w["budget"])
    order = sorted(range(len(parts)), key=lambda i: (cfg[i], i))
    parts = [parts[i] for i in order]
    cfg = [cfg[i] for i in order]
    rp, cl, voff = synth.block_diagonal(parts)
    return parts, cfg, rp, cl, voff


def oracle_batch_sample(parts, cfg, target_s=15.0, seed=0):
    """The oracle over whole graphs of the mix, drawn at random until about
    target_s seconds of work: sketches, pass and totals of each graph."""
    from oracle import oracle as O
    gen = np.random.default_rng(seed)
    order = gen.permutation(len(parts))
    edges, secs, graphs = 0, 0.0, 0
    for i in order:
        rp = parts[i][0].cpu().numpy()
        cl = parts[i][1].cpu().numpy()
        t0 = time.perf_counter()
        r = O.analyze(rp, cl, O.EST_BF_AND, l=cfg[i][0], b=cfg[i][1], seed=1)
        secs += time.perf_counter() - t0
        edges += r["m"]
        graphs += 1
        if secs >= target_s:
            break
    desc = (f"{graphs} whole graphs of the mix drawn at random ({edges} upper edges): oracle Bloom sketches, "
            f"AND estimates, triangle count and LCC, serial C/numpy on 1 host core")
    return edges / secs, secs, edges, desc


def run_batch(args, ws, rank, dev):
    from paper_2208_11469_gb300 import pg
    parts, cfg, rp, cl, voff = generate_batch(args.workload, dev)
    G = len(parts)
    g = pg.graph(rp, cl, build_index=False)
    batch = pg.Batch(g, voff, cfg, seed=1, want_tri=False)
    m = int(sum(int((p[0][1:] - p[0][:-1]).sum()) // 2 for p in parts))
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    launches0 = pg.kernel_launches()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            batch.run()
        stream.synchronize()
        launches_w = pg.kernel_launches()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index or 0) as clk:
            barrier(ws)
            torch.cuda.synchronize()
            start.record(stream)
            for _ in range(args.steps):
                batch.run()
            end.record(stream)
            torch.cuda.synchronize()
            barrier(ws)
    graph_launches = pg.kernel_launches() - launches_w
    ms = start.elapsed_time(end) / args.steps
    ms_max = max_over_ranks(ms, ws, dev)
    value = m * ws / (ms_max * 1e-3)
    res = batch.results()
    # kernels inside one captured run: count them on one eager run
    l0 = pg.kernel_launches()
    batch.run(stream=0)
    torch.cuda.synchronize()
    kernels_per_run = pg.kernel_launches() - l0

    # the same work as one launch sequence per graph
    singles = []
    build_ws = torch.empty(max(max(pg.build_workspace_bytes(pg.graph(p[0], p[1], build_index=False))
                                   for p in parts), 16), dtype=torch.uint8, device=dev)
    for (prp, pcl), (bits, b) in zip(parts, cfg):
        gi = pg.graph(prp, pcl, build_index=True)
        sk = pg.alloc_sketch(gi, pg.SK_BLOOM, bits=bits, b=b, seed=1)
        singles.append((gi, sk, pg.workspace(gi, sk, pg.EST_BF_AND), pg.tc_result_buffer(dev),
                        torch.empty(gi.n, dtype=torch.float32, device=dev)))

    def per_graph_step():
        for gi, sk, wsi, tc, lcc in singles:
            pg.build_edge_index_into(gi)
            pg.build_bloom(gi, sk.bits, sk.b, sk.seed, out=sk, workspace=build_ws)
            pg.analyze(gi, sk, pg.EST_BF_AND, ws=wsi, tc=tc, lcc=lcc)

    per_graph_step()
    torch.cuda.synchronize()
    pl0 = pg.kernel_launches()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    a.record()
    per_steps = 2
    for _ in range(per_steps):
        per_graph_step()
    b_.record()
    torch.cuda.synchronize()
    per_ms = a.elapsed_time(b_) / per_steps
    per_wall = (time.perf_counter() - t0) * 1e3 / per_steps
    per_launches = (pg.kernel_launches() - pl0) // per_steps
    mismatch = 0
    for (gi, sk, wsi, tc, lcc), r in zip(singles, res):
        s1 = pg.read_tc_result(tc)
        mismatch += int(s1["count_sum"] != r["count_sum"] or s1["edges"] != r["edges"])
    del singles

    # exact GPU intersection on the union graph: per-vertex triangles -> per-graph counts
    exact = None
    if not args.no_exact:
        gx = pg.graph(rp, cl, build_index=True)
        wsx = pg.workspace(gx, None, pg.EST_EXACT)
        pg.clustering(gx, None, pg.EST_EXACT, ws=wsx)
        torch.cuda.synchronize()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record()
        _, tri, _ = pg.clustering(gx, None, pg.EST_EXACT, ws=wsx)
        eb.record()
        torch.cuda.synchronize()
        seg = torch.repeat_interleave(torch.arange(G, device=dev),
                                      torch.from_numpy(np.diff(voff)).to(dev))
        tc_exact = torch.zeros(G, dtype=torch.float64, device=dev).index_add_(0, seg, tri) / 3.0
        tc_exact = tc_exact.cpu().numpy()
        est = np.array([r["est_tc"] for r in res])
        est_l = np.array([r["est_tc_alt"] for r in res])  # the L estimator on the same histograms
        ok = tc_exact > 0
        rel = np.abs(est[ok] - tc_exact[ok]) / tc_exact[ok]
        rel_l = np.abs(est_l[ok] - tc_exact[ok]) / tc_exact[ok]
        exact = {"ms": ea.elapsed_time(eb), "edges_per_s": m / (ea.elapsed_time(eb) * 1e-3),
                 "tc_rel_error_median": float(np.median(rel)) if rel.size else None,
                 "tc_rel_error_p90": float(np.quantile(rel, 0.9)) if rel.size else None,
                 "tc_rel_error_total": float((est.sum() - tc_exact.sum()) / tc_exact.sum()),
                 "L_estimator": {
                     "tc_rel_error_median": float(np.median(rel_l)) if rel_l.size else None,
                     "tc_rel_error_p90": float(np.quantile(rel_l, 0.9)) if rel_l.size else None,
                     "tc_rel_error_total": float((est_l.sum() - tc_exact.sum()) / tc_exact.sum())}}
        del gx, wsx

    # end to end: the union CSR from pinned host memory, results back to the host
    e2e = None
    if args.e2e_steps > 0:
        host_rp, host_cl = rp.cpu().pin_memory(), cl.cpu().pin_memory()
        h_tc = torch.empty(batch.tc.shape, dtype=torch.uint8, pin_memory=True)
        h_lcc = torch.empty(batch.lcc.shape, dtype=torch.float32, pin_memory=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            for _ in range(args.e2e_steps):
                # pg_batch_run_host: the upload of later graphs overlaps the work on earlier ones
                batch.run_host(host_rp, host_cl)
                h_tc.copy_(batch.tc, non_blocking=True)
                h_lcc.copy_(batch.lcc, non_blocking=True)
            eb.record(stream)
            stream.synchronize()
        e_ms = max_over_ranks(ea.elapsed_time(eb) / args.e2e_steps, ws, dev)
        e2e = {"value": m * ws / (e_ms * 1e-3), "unit": "intersections/s",
               "h2d_bytes_per_step": 4 * (host_rp.numel() + host_cl.numel()),
               "d2h_bytes_per_step": h_tc.numel() + 4 * h_lcc.numel(), "ms_per_step": e_ms}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r, dt, e, desc = oracle_batch_sample(parts, cfg, target_s=15.0)
        cpu = {"value": r, "unit": "intersections/s", "cores": 1, "kind": "oracle", "sample": desc, "seconds": dt}

    # roofline of the captured run as a whole: algorithmic bytes of the builds (CSR read, sketch rows
    # written) and of the pull pass (per CSR entry its id and the neighbour's l/8-byte row; per vertex
    # its own row, row offset, graph id and LCC)
    n_tot, nnz_tot = g.n, g.nnz
    strides = {c: pg.sketch_stride(pg.SK_BLOOM, c[0], 0) for c in set(cfg)}
    sketch_bytes = sum((int(p[0].numel()) - 1) * strides[c] for p, c in zip(parts, cfg))
    pass_bytes = sum(int(cl_.numel()) * (c[0] / 8 + 4) + (int(rp_.numel()) - 1) * (c[0] / 8 + 16)
                     for (rp_, cl_), c in zip(parts, cfg))
    build_bytes = 4 * (n_tot + 1) + 4 * nnz_tot + sketch_bytes
    alg = build_bytes + pass_bytes
    peak, peak_kind = peaks()
    achieved = alg / (ms_max * 1e-3) / 1e9
    buckets = {}
    for c, v in zip(cfg, batch.variants):
        buckets.setdefault(f"{c[0]}b{c[1]}", {"graphs": 0, "groups_per_chunk": v})["graphs"] += 1
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "intersections/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded on-device generator)",
            "config": {"workload": args.workload, "graphs": G, "n": n_tot, "nnz": nnz_tot, "m": m,
                       "budget": WORKLOADS[args.workload]["budget"], "buckets": buckets,
                       "l2": "inputs larger than L2 (union CSR and sketches >> 129 MB), no flush",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "kernel": "pg_batch_run (whole captured run: builds, pull passes, totals)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "algorithmic_bytes": alg, "peak_source": peak_kind},
            "e2e": e2e,
            "gpu_launches": kernels_per_run * args.steps,
            "kernels_per_run": kernels_per_run,
            "cuda_graph_launches": graph_launches,
            "clocks": clk.summary(),
            "per_graph_launches": {"ms_per_step": per_ms, "wall_ms_per_step": per_wall,
                                   "value": m / (per_ms * 1e-3), "kernels_per_step": per_launches,
                                   "speedup_of_batch": per_ms / ms, "integer_mismatches": mismatch},
            "exact_gpu": exact,
            "results": {"est_tc_sum": float(sum(r["est_tc"] for r in res)),
                        "count_sum": int(sum(r["count_sum"] for r in res))},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------ clustering
def run_jp(args, ws, rank, dev):
    """Jarvis-Patrick: one step = edge index, sketch build and the
    clustering pass (counts, keep test, union-find, labels) per sketch."""
    from paper_2208_11469_gb300 import pg
    w = WORKLOADS[args.workload]
    rp, cl = generate(args.workload, dev)
    g = pg.graph(rp, cl, build_index=True)
    bits = pg.bloom_bits_for_budget(w["budget"], g.n, g.nnz)
    bws = torch.empty(max(pg.build_workspace_bytes(g), 16), dtype=torch.uint8, device=dev)
    bf = pg.alloc_sketch(g, pg.SK_BLOOM, bits=bits, b=w["b"], seed=1)
    kh = pg.alloc_sketch(g, pg.SK_KHASH, k=w["khash"], seed=1)
    passes = [("bloom", bf, pg.EST_BF_AND), ("khash", kh, pg.EST_KH)]
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    res = {nm: torch.zeros(32, dtype=torch.uint8, device=dev) for nm, _, _ in passes}
    jws = {nm: torch.empty(max(pg.lib().pg_jarvis_patrick_workspace_bytes(ctypes.byref(g.csr()),
                                                                         ctypes.byref(sk.desc()), est), 16),
                           dtype=torch.uint8, device=dev) for nm, sk, est in passes}
    names = ["index"] + ["build_" + p[0] for p in passes] + ["jp_" + p[0] for p in passes]

    def step(ev=None):
        s = torch.cuda.current_stream()

        def mark(nm, i):
            if ev is not None:
                ev[nm][i].record(s)
        mark("index", 0)
        pg.build_edge_index_into(g)
        mark("index", 1)
        for nm, sk, est in passes:
            mark("build_" + nm, 0)
            if sk.kind == pg.SK_BLOOM:
                pg.build_bloom(g, sk.bits, sk.b, sk.seed, out=sk, workspace=bws)
            else:
                pg.build_minhash(g, sk.kind, sk.k, sk.seed, out=sk, workspace=bws)
            mark("build_" + nm, 1)
        for nm, sk, est in passes:
            mark("jp_" + nm, 0)
            pg.jarvis_patrick(g, sk, est, w["tau"], labels=labels, ws=jws[nm], out=res[nm], read=False)
            mark("jp_" + nm, 1)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [{nm: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for nm in names}
           for _ in range(args.steps)]
    l0 = pg.kernel_launches()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        a.record()
        for i in range(args.steps):
            step(evs[i])
        b_.record()
        torch.cuda.synchronize()
        barrier(ws)
    launches = pg.kernel_launches() - l0
    ms = max_over_ranks(a.elapsed_time(b_) / args.steps, ws, dev)
    per = {nm: float(np.mean([e[nm][0].elapsed_time(e[nm][1]) for e in evs])) for nm in names}
    out = {}
    for nm, _, _ in passes:
        c, k_, e_, _ = struct.unpack("<qqqq", bytes(res[nm].cpu().numpy().tobytes()))
        out[nm] = {"clusters": c, "kept": k_, "edges": e_}
    # the exact clustering
    ex = None
    if not args.no_exact:
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record()
        _, exr = pg.jarvis_patrick(g, None, pg.EST_EXACT, w["tau"], want_labels=False)
        eb.record()
        torch.cuda.synchronize()
        ex = dict(exr, ms=ea.elapsed_time(eb))
        for nm in out:
            out[nm]["relative_cluster_count"] = out[nm]["clusters"] / max(exr["clusters"], 1)
    m = g.m
    peak, peak_kind = peaks()
    dom = max((p[0] for p in passes), key=lambda nm: per["jp_" + nm])
    sk_dom = [p[1] for p in passes if p[0] == dom][0]
    payload = sk_dom.bits / 8 if sk_dom.kind == pg.SK_BLOOM else 4 * sk_dom.k
    # count pass (row of v, v, degrees for MinHash, count out) + union pass (count, u, v, degrees)
    alg = m * (payload + 4 + (8 if sk_dom.kind != pg.SK_BLOOM else 0) + 4) + g.n * (payload + 12) + m * 20 + g.n * 8
    achieved = alg / (per["jp_" + dom] * 1e-3) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(None, rp, cl, dict(w, onehash=None, jaccard=False), bits)
    if rank == 0:
        line = {
            "metric": METRIC + " (Jarvis-Patrick)", "value": m * len(passes) * ws / (ms * 1e-3),
            "unit": "intersections/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded on-device generator)",
            "config": {"workload": args.workload, "n": g.n, "nnz": g.nnz, "m": m, "bloom_bits": bits,
                       "bloom_b": w["b"], "khash_k": w["khash"], "tau": w["tau"],
                       "l2": "inputs larger than L2, no flush", "parallelism": f"replicas x{ws}"},
            "phases_ms": per,
            "roofline": {"bound": "hbm", "kernel": f"pg_jarvis_patrick ({dom}: count pass + union-find)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "algorithmic_bytes": alg, "peak_source": peak_kind},
            "e2e": None, "gpu_launches": launches, "clocks": clk.summary(), "results": out, "exact_gpu": ex,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------- 4-cliques
def run_clique(args, ws, rank, dev):
    """4-clique counting: one step = orientation, Bloom filters of the oriented
    neighbourhoods and the 3-clique enumeration with the triple-AND estimate.
    The unit is one sketched (triple) intersection per 3-clique."""
    from paper_2208_11469_gb300 import pg
    w = WORKLOADS[args.workload]
    rp, cl = generate(args.workload, dev)
    g = pg.graph(rp, cl, build_index=False)
    c = g.csr()
    wsb = torch.empty(pg.lib().pg_clique4_workspace_bytes(ctypes.byref(c), pg.EST_BF_AND, w["bits"]),
                      dtype=torch.uint8, device=dev)
    out = torch.zeros(48, dtype=torch.uint8, device=dev)

    def step():
        pg.clique4_count(g, pg.EST_BF_AND, w["bits"], w["b"], 1, ws=wsb, out=out, read=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = pg.kernel_launches()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        a.record()
        for _ in range(args.steps):
            step()
        b_.record()
        torch.cuda.synchronize()
        barrier(ws)
    launches = pg.kernel_launches() - l0
    ms = max_over_ranks(a.elapsed_time(b_) / args.steps, ws, dev)
    tri, _, cs, _, est, est_alt = struct.unpack("<QQQQdd", bytes(out.cpu().numpy().tobytes()))
    exact = None
    if not args.no_exact:
        wse = torch.empty(pg.lib().pg_clique4_workspace_bytes(ctypes.byref(c), pg.EST_EXACT, 0),
                          dtype=torch.uint8, device=dev)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record()
        r = pg.clique4_count(g, pg.EST_EXACT, ws=wse)
        eb.record()
        torch.cuda.synchronize()
        exact = {"ms": ea.elapsed_time(eb), "count": r["exact"], "triangles": r["triangles"],
                 "rel_error": (est - r["exact"]) / r["exact"] if r["exact"] else None,
                 "rel_error_L": (est_alt - r["exact"]) / r["exact"] if r["exact"] else None}
    peak, peak_kind = peaks()
    # per 3-clique: the filter of w (the filters of u and v are reused by the group); per oriented edge the two
    # list heads and the binary searches are not counted
    alg = tri * (w["bits"] / 8)
    achieved = alg / (ms * 1e-3) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O
        from paper_2208_11469_gb300 import synth
        small = 14
        srp, scl = synth.rmat(small, 16, seed=small)
        t0 = time.perf_counter()
        ro = O.clique4(srp.numpy(), scl.numpy(), O.EST_BF_AND, l=w["bits"], b=w["b"], seed=1)
        dt = time.perf_counter() - t0
        cpu = {"value": ro["triangles"] / dt, "unit": "intersections/s", "cores": 1, "kind": "oracle",
               "sample": f"the same recipe at R-MAT scale {small} ({ro['triangles']} 3-cliques): oracle "
                         f"orientation, oriented Bloom filters and triple-AND counts, serial C on 1 host core",
               "seconds": dt}
    if rank == 0:
        line = {
            "metric": METRIC + " (4-cliques)", "value": tri * ws / (ms * 1e-3), "unit": "intersections/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded on-device generator)",
            "config": {"workload": args.workload, "n": g.n, "nnz": g.nnz, "bloom_bits": w["bits"], "bloom_b": w["b"],
                       "step": "orientation + oriented Bloom filters + 3-clique enumeration with triple-AND counts",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "kernel": "k_clique4 (whole step)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None, "algorithmic_bytes": alg,
                         "peak_source": peak_kind},
            "e2e": None, "gpu_launches": launches, "clocks": clk.summary(),
            "results": {"triangles": tri, "est": est, "est_alt_L": est_alt, "count_sum": cs},
            "exact_gpu": exact, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------- serving
def serve_requests(workload, rp, cl, seed=7):
    """The request set: pair requests (sizes lognormal, half edges and half
    random pairs) and induced-subgraph requests (BFS balls of 10^U(3,6)
    edges), interleaved at random. Host numpy arrays."""
    from paper_2208_11469_gb300 import synth
    w = WORKLOADS[workload]
    rng = np.random.default_rng(seed)
    n = rp.numel() - 1
    sizes = np.clip(np.round(rng.lognormal(np.log(256.0), 2.0, w["pair_requests"])), 1, 65536).astype(np.int64)
    allp = synth.random_pairs(n, int(sizes.sum()), seed, rp, cl, device=rp.device).cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    reqs = [("pairs", allp[offs[i]:offs[i + 1]]) for i in range(sizes.size)]
    rp_h, cl_h = rp.cpu().numpy(), cl.cpu().numpy()
    for i in range(w["subgraph_requests"]):
        j = int(rng.integers(0, cl_h.size))
        v = int(np.searchsorted(rp_h, j, side="right") - 1)
        reqs.append(("sub", synth.bfs_ball(rp_h, cl_h, v, int(10 ** rng.uniform(3, 6)))))
    order = rng.permutation(len(reqs))
    return [reqs[i] for i in order], rp_h, cl_h


def induced_edges(rp_h, cl_h, S):
    mark = np.zeros(rp_h.size - 1, dtype=bool)
    mark[S] = True
    lens = rp_h[S + 1] - rp_h[S]
    idx = np.repeat(rp_h[S] - np.cumsum(np.concatenate([[0], lens[:-1]])), lens) + np.arange(int(lens.sum()))
    return int(mark[cl_h[idx]].sum()) // 2


def serve_burst(sv, reqs, est_pairs, est_sub, pg, pinned=None):
    """Submit every request at once and collect them all: the pair requests
    as one concatenated page-locked array (pg_submit_many, used in place by
    the GPU), the subgraph requests in a second pg_submit_many. Returns
    (seconds, responses in request order, pair outputs in request order)."""
    if pinned is None:
        pinned = serve_pinned(reqs, pg)
    pidx, sidx, offs, buf = pinned
    t0 = time.perf_counter()
    tp, cn, jac = sv.submit_pairs_many(buf, offs, est_pairs, pinned=True)
    ts, _ = sv.submit_many([("sub", reqs[i][1], est_sub) for i in sidx])
    rp_ = sv.poll_many(tp, timeout_us=600_000_000)
    rs_ = sv.poll_many(ts, timeout_us=600_000_000)
    dt = time.perf_counter() - t0
    resp = np.zeros(len(reqs), dtype=rp_.dtype)
    outs = [None] * len(reqs)
    resp[pidx] = rp_
    resp[sidx] = rs_
    for k, i in enumerate(pidx):
        outs[i] = (cn[offs[k]:offs[k + 1]], jac[offs[k]:offs[k + 1]])
    return dt, resp, outs


def serve_pinned(reqs, pg):
    """The pair requests of a request set concatenated in page-locked memory."""
    pidx = [i for i, (k, _) in enumerate(reqs) if k == "pairs"]
    sidx = [i for i, (k, _) in enumerate(reqs) if k != "pairs"]
    sizes = [reqs[i][1].shape[0] for i in pidx]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    buf = pg.pinned_empty((int(offs[-1]), 2), np.int32)
    if pidx:
        buf[...] = np.concatenate([reqs[i][1] for i in pidx])
    return pidx, sidx, offs, buf


def serve_poisson(sv, reqs, rate, duration, est_pairs, est_sub, seed=3):
    """Open-loop Poisson arrivals at `rate` requests/s for `duration` s,
    cycling through the request set; a second thread collects. Returns the
    responses with their kinds."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, int(rate * duration) + 1)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration]
    tickets = []
    lock = threading.Lock()
    done = []

    def collect():
        i = 0
        while True:
            with lock:
                if i >= len(tickets):
                    if finished[0]:
                        break
                    t = None
                else:
                    t = tickets[i]
            if t is None:
                time.sleep(0.0005)
                continue
            kind, tk = t
            done.append((kind, sv.wait(tk, 600.0)))
            i += 1

    finished = [False]
    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for i, at in enumerate(arrivals):
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        kind, x = reqs[i % len(reqs)]
        tk = sv.submit_pairs(x, est_pairs) if kind == "pairs" else sv.submit_subgraph(x, est_sub)
        with lock:
            tickets.append((kind, tk))
    with lock:
        finished[0] = True
    th.join()
    return done, time.perf_counter() - t0


def run_serve(args, ws, rank, dev):
    from paper_2208_11469_gb300 import pg
    w = WORKLOADS[args.workload]
    rp, cl = generate(args.workload, dev)
    g = pg.graph(rp, cl, build_index=True)
    bf = pg.build_bloom(g, w["bits"], w["b"], seed=1)
    kh = pg.build_minhash(g, pg.SK_KHASH, w["khash"], seed=1)
    reqs, rp_h, cl_h = serve_requests(args.workload, rp, cl)
    pairs_total = sum(x.shape[0] for k, x in reqs if k == "pairs")
    sub_edges = {id(x): induced_edges(rp_h, cl_h, x) for k, x in reqs if k == "sub"}
    units = pairs_total + sum(sub_edges.values())
    torch.cuda.synchronize()
    sv = pg.Server(g, [bf, kh], 6 << 30)
    pinned = serve_pinned(reqs, pg)
    for _ in range(args.warmup):
        serve_burst(sv, reqs, pg.EST_BF_AND, pg.EST_BF_AND, pg, pinned)
    st0 = sv.stats()
    times = []
    with ClockSampler(dev.index or 0) as clk:
        for _ in range(args.steps):
            dt, out, _ = serve_burst(sv, reqs, pg.EST_BF_AND, pg.EST_BF_AND, pg, pinned)
            assert (out["status"] == 0).all()
            times.append(dt)
    st1 = sv.stats()
    burst_s = float(np.median(times))
    value = units * ws / burst_s
    kernel_ns = st1["pair_kernel_ns"] - st0["pair_kernel_ns"]
    pairs_timed = st1["pairs"] - st0["pairs"]
    # k_serve_pairs roofline: per pair two 64-byte rows, the pair (8 B), four row offsets (16 B), two outputs
    per_pair = 2 * w["bits"] / 8 + 8 + 16 + 8
    alg = pairs_timed * per_pair
    peak, peak_kind = peaks()
    achieved = alg / (kernel_ns * 1e-9) / 1e9 if kernel_ns else None

    # latency under open-loop Poisson arrivals, one request per pg_submit: at 70% of the burst request
    # rate, capped at what one Python submitting thread sustains
    rate = min(0.7 * len(reqs) / burst_s, 15000.0)
    lat, wall = serve_poisson(sv, reqs, rate, 3.0, pg.EST_BF_AND, pg.EST_BF_AND)
    pl = np.array([r["total_us"] for k, r in lat if k == "pairs"])
    sl = np.array([r["total_us"] for k, r in lat if k == "sub"])
    latency = {"offered_requests_per_s": rate, "achieved_requests_per_s": len(lat) / wall,
               "requests": len(lat), "seconds": wall,
               "pairs_p50_us": float(np.percentile(pl, 50)) if pl.size else None,
               "pairs_p99_us": float(np.percentile(pl, 99)) if pl.size else None,
               "subgraph_p50_us": float(np.percentile(sl, 50)) if sl.size else None,
               "subgraph_p99_us": float(np.percentile(sl, 99)) if sl.size else None}

    # the same requests through the server with the exact intersection
    ex_dt, ex_out, ex_pairs = serve_burst(sv, reqs, pg.EST_EXACT, pg.EST_EXACT, pg, pinned)
    _, est_out, est_pairs = serve_burst(sv, reqs, pg.EST_BF_AND, pg.EST_BF_AND, pg, pinned)
    _, kh_out, kh_pairs = serve_burst(sv, reqs, pg.EST_KH, pg.EST_BF_AND, pg, pinned)
    # accuracy on a seeded 1% sample of the requests (exact answers from the exact GPU path)
    rng = np.random.default_rng(1)
    sample = rng.choice(len(reqs), max(1, len(reqs) // 100), replace=False)
    cn_err, cn_err_kh, tc_rel = [], [], []
    for i in sample:
        if reqs[i][0] == "pairs":
            cn_err.append(float(np.mean(np.abs(est_pairs[i][0] - ex_pairs[i][0]))))
            cn_err_kh.append(float(np.mean(np.abs(kh_pairs[i][0] - ex_pairs[i][0]))))
        elif ex_out[i]["exact_tc"]:
            tc_rel.append(abs(est_out[i]["est_tc"] - ex_out[i]["exact_tc"]) / ex_out[i]["exact_tc"])
    sub_idx = [i for i in range(len(reqs)) if reqs[i][0] == "sub" and ex_out[i]["exact_tc"]]
    tc_rel_all = [float(abs(est_out[i]["est_tc"] - ex_out[i]["exact_tc"]) / ex_out[i]["exact_tc"]) for i in sub_idx]
    exact_mean_cn = float(np.mean([np.mean(ex_pairs[i][0]) for i in sample if reqs[i][0] == "pairs"]))
    sv.close()

    # one request per launch: each pair request alone through pg_jaccard_pairs (same pass kernels)
    per = []
    t0 = time.perf_counter()
    n_single = 0
    for kind, x in reqs:
        if kind != "pairs":
            continue
        ts = time.perf_counter()
        h = torch.from_numpy(x)
        d = h.to(dev, non_blocking=False)
        cn, jac = pg.jaccard_pairs(g, bf, pg.EST_BF_AND, d)
        cn_h, jac_h = cn.cpu(), jac.cpu()
        per.append((time.perf_counter() - ts) * 1e6)
        n_single += 1
    single_s = time.perf_counter() - t0
    per = np.array(per)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(None, rp, cl, dict(w, onehash=None, jaccard=False), w["bits"])

    if rank == 0:
        line = {
            "metric": METRIC + " (served)", "value": value, "unit": "intersections/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": burst_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded on-device generator)",
            "config": {"workload": args.workload, "n": g.n, "nnz": g.nnz, "m": g.m, "bloom_bits": w["bits"],
                       "bloom_b": w["b"], "khash_k": w["khash"], "requests": len(reqs),
                       "pair_requests": w["pair_requests"], "pairs": pairs_total,
                       "subgraph_requests": w["subgraph_requests"], "subgraph_edges": int(sum(sub_edges.values())),
                       "step": "one burst of the whole request set, host submit to host result",
                       "l2": "sketch tables 268 MB + 537 MB > 129 MB L2, no flush",
                       "timing": "host wall clock (requests cross the host boundary); kernel time from CUDA events",
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "kernel": "k_serve_pairs", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak if achieved else None, "traffic": None,
                         "algorithmic_bytes": alg, "peak_source": peak_kind},
            "e2e": {"value": value, "unit": "intersections/s",
                    "h2d_bytes_per_step": int(8 * pairs_total + 4 * sum(x.size for k, x in reqs if k == "sub")),
                    "d2h_bytes_per_step": int(8 * pairs_total + 48 * w["subgraph_requests"]),
                    "note": "pair inputs and outputs are page-locked host buffers the kernel reads and writes in place"},
            "gpu_launches": int(st1["pair_launches"] - st0["pair_launches"]),
            "latency": latency,
            "clocks": clk.summary(),
            "pairs_per_s": pairs_total / burst_s,
            "exact_gpu_served": {"seconds": ex_dt, "intersections_per_s": units / ex_dt},
            "one_request_per_launch": {"pair_requests": n_single, "seconds": single_s,
                                       "pairs_per_s": pairs_total / single_s,
                                       "p50_us": float(np.percentile(per, 50)), "p99_us": float(np.percentile(per, 99))},
            "accuracy_sample": {"requests": int(sample.size), "exact_mean_cn": exact_mean_cn,
                                "pairs_mean_abs_cn_error_bf_and": float(np.mean(cn_err)) if cn_err else None,
                                "pairs_mean_abs_cn_error_khash": float(np.mean(cn_err_kh)) if cn_err_kh else None,
                                "subgraph_tc_rel_error": tc_rel, "subgraph_tc_rel_error_all": tc_rel_all},
            "server": {k: st1[k] for k in ("pair_launches", "pairs", "subgraphs", "arena_peak", "arena_bytes")},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cfg = WORKLOADS[args.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    if "batch" in cfg:
        return run_reference_batch(args, ws, dev)
    rp, cl = generate(args.workload, dev)
    bits = cfg.get("bits") or budget_bits(cfg["budget"], rp.numel() - 1, cl.numel())
    # every step: a fresh sample run on all host cores (one oracle process per core), about 1.5 s of
    # work per core, so that K + W steps stay within a few minutes
    leg = OracleLeg(rp, cl, cfg, bits, seed=1)
    per_step = 1.5 * leg.cores
    for _ in range(args.warmup):
        leg.parallel(leg.sized(per_step, leg.cores))
    rates, secs, last = [], 0.0, None
    for i in range(args.steps):
        chunks = leg.sized(per_step, leg.cores)
        t0 = time.perf_counter()
        last = leg.parallel(chunks)
        secs += time.perf_counter() - t0
        rates.append(last["value"])
    value = float(np.median(rates))
    desc = leg.describe(last) if last else ""
    # the same config keys as our arm's line (the generated graphs are simple and symmetric: m = nnz / 2)
    n = int(rp.numel() - 1)
    m = int(cl.numel()) // 2
    passes = ["bloom"] + ["bloom_" + nm for nm in cfg.get("bloom_variants", ())]
    passes += ["khash"] if cfg["khash"] else []
    passes += (["onehash"] + ["onehash_" + nm for nm in cfg.get("onehash_variants", ())]) if cfg["onehash"] else []
    config = {"workload": args.workload, "n": n, "nnz": int(cl.numel()), "m": m, "bloom_bits": bits,
              "bloom_b": cfg["b"], "khash_k": cfg["khash"], "onehash_k": cfg["onehash"],
              "per_edge_jaccard": cfg["jaccard"], "passes": passes,
              "l2": "a bounded sample on the host cores", "parallelism": "rank 0 only"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "intersections/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": "intersections/s", "cores": leg.cores, "kind": "oracle",
                             "sample": desc,
                             "formula": "passes * m / (t_build * n / rows + t_pass * m / pairs), median over steps"},
            "e2e": {"value": value, "unit": "intersections/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_batch(args, ws, dev):
    parts, cfg, rp_u, cl_u, _ = generate_batch(args.workload, dev)
    per_step = 4.0 * max(1, 60 // max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        oracle_batch_sample(parts, cfg, target_s=min(per_step, 5.0), seed=1)
    rates, secs, desc = [], 0.0, ""
    for i in range(args.steps):
        r, dt, e, desc = oracle_batch_sample(parts, cfg, target_s=per_step, seed=100 + i)
        rates.append(r)
        secs += dt
    value = float(np.median(rates))
    buckets = {}
    for c in cfg:
        buckets.setdefault(f"{c[0]}b{c[1]}", {"graphs": 0})["graphs"] += 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "intersections/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "graphs": len(parts), "n": int(rp_u.numel() - 1),
                       "nnz": int(cl_u.numel()), "m": int(cl_u.numel()) // 2,
                       "budget": WORKLOADS[args.workload]["budget"], "buckets": buckets,
                       "l2": "a bounded sample on the host cores", "parallelism": "rank 0 only"},
            "cpu_baseline": {"value": value, "unit": "intersections/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "intersections/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-exact", action="store_true")
    ap.add_argument("--no-parity-sample", action="store_true")
    ap.add_argument("--source-hash", action="store_true", help="print the pass sources' sha256 and exit")
    args = ap.parse_args()
    if args.source_hash:
        print(source_fingerprint())
        return
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args)
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    init_dist(ws, "nccl")
    from paper_2208_11469_gb300 import build as B
    B.build()
    from paper_2208_11469_gb300 import pg

    dev = torch.device("cuda", local)
    special = [k for k in ("batch", "serve", "jp", "clique") if k in WORKLOADS[args.workload]]
    if special:
        {"batch": run_batch, "serve": run_serve, "jp": run_jp, "clique": run_clique}[special[0]](args, ws, rank, dev)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    rp, cl = generate(args.workload, dev)
    pipe = Pipeline(args.workload, rp, cl)
    torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        ms, per, launches, stats = time_steps(pipe, args.steps, args.warmup, ws)
    ms_max = max_over_ranks(ms, ws, dev)
    units = pipe.sketched_per_step() * ws
    value = units / (ms_max * 1e-3)
    res = pipe.results()

    # roofline of the dominant kernel (the largest intersection pass)
    dom = max((p[0] for p in pipe.passes), key=lambda nm: per["pass_" + nm])
    peak, peak_kind = peaks()
    alg = algorithmic_bytes(pipe, dom)
    achieved = alg / (per["pass_" + dom] * 1e-3) / 1e9
    traffic = profiled_traffic(f"{dom}_pass_{args.workload}.md")
    # every pass against the HBM roofline, and the k-Hash build against the integer ALU roofline
    clocks = clk.summary()
    rooflines = {}
    for nm, sk, _ in pipe.passes:
        a_nm = algorithmic_bytes(pipe, nm)
        g_nm = a_nm / (per["pass_" + nm] * 1e-3) / 1e9
        rooflines["pass_" + nm] = {"bound": "hbm", "achieved": g_nm, "peak": peak, "unit": "GB/s",
                                   "frac": g_nm / peak, "algorithmic_bytes": a_nm, "ms": per["pass_" + nm],
                                   "traffic": profiled_traffic(f"{nm}_pass_{args.workload}.md")}
    for nm, sk, _ in pipe.passes:
        if sk.kind == pg.SK_KHASH and "build_" + nm in per:
            mhz = clocks["sm_mhz"] or 2070.0
            p_alu, sms = alu_peak(mhz)
            hashes = sk.k * pipe.nnz
            # in the step the build shares the GPU with the index and the Bloom build on the
            # side stream, so its roofline is taken from builds timed alone
            alone = time_build_alone(pipe, sk)
            ops = hashes * ALU_OPS_PER_HASH / (alone * 1e-3)
            rooflines["build_" + nm] = {
                "bound": "alu", "kernel": "k_khash_warp + k_khash_hub", "achieved": ops, "peak": p_alu,
                "unit": "int32 ALU ops/s", "frac": ops / p_alu, "hashes_per_s": hashes / (alone * 1e-3),
                "ms": alone, "ms_in_step": per["build_" + nm],
                "timing": "3 builds alone after the timed steps (CUDA events); ms_in_step: the build's phase "
                          "in the step, beside the index and the Bloom build on another stream",
                "peak_derivation": f"{sms} SMs x {ALU_OPS_PER_SM_CLOCK} ALU lane-ops/clock x {mhz:.0f} MHz "
                                   f"(median sampled SM clock); {ALU_OPS_PER_HASH} ALU ops per hash"}

    # end to end from host buffers
    e2e = None
    if args.e2e_steps > 0:
        host_rp = rp.cpu().pin_memory()
        host_col = cl.cpu().pin_memory()
        h2d_gbs = h2d_rate(pipe.g.col, host_col)
        e2e_ms, e2e_wall, h2d, d2h = e2e_steps(pipe, host_rp, host_col, args.e2e_steps)
        e2e_ms = max_over_ranks(e2e_ms, ws, dev)
        e2e = {"value": pipe.sketched_per_step() * ws / (e2e_ms * 1e-3), "unit": "intersections/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
               "wall_ms_per_step": e2e_wall, "h2d_gbs": h2d_gbs,
               "h2d_note": "one copy of the column array from page-locked memory, timed before the e2e steps"}

    exact = None
    if not args.no_exact:
        ex_ms, ex = exact_comparison(pipe)
        rel = {nm: (r["est_tc"] - ex["exact_tc"]) / ex["exact_tc"] if ex["exact_tc"] else None
               for nm, r in res.items()}
        exact = {"ms": ex_ms, "exact_tc": ex["exact_tc"], "edges_per_s": pipe.m / (ex_ms * 1e-3),
                 "tc_rel_error": rel}
        # Thm. 7.1's 95% deviation radius beside the measured error (relative to the exact count)
        try:
            kinds = []
            for nm, sk, est in pipe.passes:
                kind = ("bloom_and" if est == pg.EST_BF_AND else
                        "minhash" if est in (pg.EST_KH, pg.EST_1H) else None)
                kinds.append((nm, kind, sk.bits, sk.b, sk.k))
            bounds = tc_deviation_bounds(rp, kinds)
            exact["thm71_radius_95"] = {
                nm: (None if v is None else dict(v, rel=(v["t"] / ex["exact_tc"]
                                                         if v.get("t") is not None and ex["exact_tc"] else None)))
                for nm, v in bounds.items()}
        except Exception as err:  # a report beside the measurement: never fail the bench line
            exact["thm71_radius_95"] = {"error": repr(err)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pipe, rp, cl, pipe.cfg, pipe.bits)

    parity = None
    if rank == 0 and not args.no_parity_sample:
        parity = parity_sample(pipe)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "intersections/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded on-device generator)",
            "config": {"workload": args.workload, "n": pipe.n, "nnz": pipe.nnz, "m": pipe.m,
                       "bloom_bits": pipe.bits, "bloom_b": pipe.cfg["b"], "khash_k": pipe.cfg["khash"],
                       "onehash_k": pipe.cfg["onehash"], "per_edge_jaccard": pipe.cfg["jaccard"],
                       "passes": [p[0] for p in pipe.passes],
                       "l2": "inputs larger than L2 (CSR and sketch tables >> 129 MB), no flush",
                       "parallelism": f"replicas x{ws}"},
            "phases_ms": per,
            "step_ms": stats,
            "roofline": {"bound": "hbm",
                         "kernel": ("k_onehash" if dict((p[0], p[1]) for p in pipe.passes)[dom].kind == pg.SK_1HASH
                                    else "k_lean") + f" ({dom} pass of pg_analyze)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes": alg, "peak_source": peak_kind},
            "e2e": e2e,
            "rooflines": rooflines,
            "gpu_launches": launches,
            "clocks": clocks,
            "results": res,
            "exact_gpu": exact,
            "cpu_baseline": cpu,
            "parity_sample": parity,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
