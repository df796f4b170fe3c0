#!/usr/bin/env python3
"""Benchmark of the k-mismatch character-class search on the GENOME workload.

Workload (one step): a 3.1 Gbp order-2 Markov text (41 % GC), coded once and
resident in HBM (775 MB), searched for three patterns (m = 32, 128, 1024;
10 % two/three-letter class positions; 100 planted noisy copies each) at
k = 0, 4 and 16: nine (pattern, k) searches, one scan launch each, then the
ordering kernels, all through the C ABI.

metric   window-cells/s = sum over the nine searches of (n - m + 1) * m, per
         second (the paper's nominal count; the early stop of Eq. 4 makes the
         work far smaller than the count).  Text GB/s = 9 * n/4 bytes per
         second is reported beside it.
value    device time of the step (CUDA events on the launching stream), text
         resident; the text (775 MB) is larger than the 129 MB L2, so no
         flush is needed between steps.
e2e      the same metric through the public API with host buffers: every step
         codes the text from pinned host ASCII (pm_encode_text), compiles the
         patterns and searches with host output buffers.
roofline the scan kernel: algorithmic bytes per launch (n/4 text bytes plus
         8 bytes per hit) over its event-timed duration, against the measured
         HBM copy bandwidth.

``--impl reference`` times the oracle (plain C, all host cores) on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GENOME_N = 3_100_000_000
MS = (32, 128, 1024)
KS = (0, 4, 16)
TEXT_SEED = 3
METRIC = "window-cells/s"
VARIANT_NAMES = {1: "pattern-sliced", 2: "window-sliced", 3: "pattern-sliced-64", 4: "all-chunks"}

# DRAM bytes (read + write) of one pattern-sliced (k = 16, m = 128) launch over
# the GENOME text at n = 8e8, from the ncu capture summarised in
# profiles/k_scan_genome_ncu_800M.md; scaled by the window count of a launch.
# Valid only for the kernel source it was captured from: TRAFFIC_SRC_SHA is
# the hash (kernel_source_sha) of the scan kernel's sources at capture time,
# and the line reports no traffic when the sources no longer match.
TRAFFIC_KERNEL = "k_scan<pattern-sliced>"
TRAFFIC_BYTES_8E8 = (200.219136 + 1.242624) * 1e6
TRAFFIC_SRC_SHA = "ca81fa4f46337efd"
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, k = 16 m = 128 launch at "
                  "n = 8e8 (profiles/k_scan_genome_ncu_800M.md), scaled by windows")
KERNEL_SOURCES = ("pm_scan.cu", "pm_scan_impl.cuh", "pm_internal.cuh")


def kernel_source_sha() -> str:
    """SHA-256 (first 16 hex digits) of the scan kernel's source files."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1611_06115_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic(kernel, n):
    """Per-launch DRAM bytes of `kernel` at text length n, or None when no
    capture of the current sources exists."""
    if TRAFFIC_BYTES_8E8 is None or kernel != TRAFFIC_KERNEL or TRAFFIC_SRC_SHA != kernel_source_sha():
        return None
    return TRAFFIC_BYTES_8E8 * (n - 127) / (800_000_000 - 127)


# First-stage ALU-pipe instructions per window of each evaluation (the
# roofline's algorithmic work, counted from the evaluations' definitions):
#   pattern-sliced over 32 positions: 2 funnel shifts + 3 selects = 5;
#   over 64 positions: 10;
#   window-sliced: per listed position and 32 windows one funnel shift plus
#   the counter update (k = 0: half a logic operation, k = 1..3: k+1, k >= 4:
#   11/4 for the binary counters), over the ws_cut(k) positions it tests.
def ws_cut(k: int) -> int:
    return 8 if k == 0 else ((4 + 2 * k) & ~3 if k >= 4 else 4 + 2 * k)


def first_stage_ops(variant: str, k: int, m: int) -> float:
    if variant == "window-sliced":
        per_pos = 1.5 if k == 0 else (1.0 + (k + 1) if k <= 3 else 1.0 + 11.0 / 4.0)
        return min(ws_cut(k), m, 32) * per_pos / 32.0
    if variant == "pattern-sliced-64" and m > 32:
        return 10.0
    if variant == "all-chunks":
        chunks = min((m + 31) // 32, (k + 1 + 21) // 22 + 1)
        return 7.0 * chunks
    return 5.0


def ops_model(variant: str, k: int) -> str:
    if variant == "window-sliced":
        upd = ("half a logic operation" if k == 0 else
               f"{k + 1} logic operations" if k <= 3 else "11/4 logic operations (binary counters)")
        return (f"window-sliced, k = {k}: per listed position and 32 windows 1 funnel shift + {upd}, "
                f"over {ws_cut(k)} positions")
    if variant == "pattern-sliced-64":
        return "10 ALU instructions per window (4 funnel shifts + 6 selects over 64 positions)"
    return "5 ALU instructions per window (2 funnel shifts + 3 selects over 32 positions)"


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=GENOME_N, help="text length per GPU")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-tune", action="store_true",
                    help="batched: built-in options and variant table (no tuning launches)")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="reference arm: target seconds of oracle work for the whole run")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--batched-n", type=int, default=1_000_000_000,
                    help="text length of the BATCHED comparison added to the default line (0: skip)")
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--workload", choices=("genome", "batched", "serving", "large", "profile"),
                    default="genome",
                    help="genome (the default line); batched and serving print their own "
                         "lines; profile runs five single searches for an ncu capture")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: queries per second")
    ap.add_argument("--serve-mode", choices=("one-launch", "launch-per-query"), default="launch-per-query",
                    help="serving: one persistent launch per batch, or one scan launch per query")
    ap.add_argument("--serve-slots", type=int, default=4, help="serving: batches in flight (streams)")
    ap.add_argument("--serve-delivery", choices=("host", "device"), default="host",
                    help="serving: hits delivered to pinned host memory (latency includes the copy) "
                         "or left on the device")
    return ap.parse_args()


# ----------------------------------------------------------------- workload --

def genome_patterns():
    from synth import workloads
    return workloads.genome_patterns(TEXT_SEED + 8, MS)


def build_text(n_local: int, start: int, out: np.ndarray, pats) -> list:
    """Symbols [start, start + n_local) of the GENOME text with planted copies
    of every pattern (copies placed by this rank inside its own range)."""
    import synth
    synth.markov_text(n_local, TEXT_SEED, out=out, start=start)
    rng = np.random.default_rng(TEXT_SEED + 16 + start)
    occ = synth.Occupancy()
    return [synth.plant(out[:n_local], p, 100, 16, rng, occ) for p in pats]


def entries(pats):
    return [(p, k) for p in pats for k in KS]


def cells(n: int, ents) -> int:
    return sum(max(n - len(p) + 1, 0) * len(p) for p, _ in ents)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks --

class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU oracle --

def oracle_sample(n: int, pats, budget_s: float, threads: int):
    """Time the oracle (all host cores) on the first S symbols of the GENOME
    text, S sized so that the run takes about budget_s seconds."""
    import oracle
    import synth
    ents = entries(pats)
    maxm = max(MS)

    def run(S):
        txt = synth.markov_text(S, TEXT_SEED)
        t0 = time.perf_counter()
        for p, k in ents:
            oracle.search(txt, p, k, threads=threads)
        return time.perf_counter() - t0

    S0 = min(n, 4_000_000)
    t0 = run(S0)
    S = int(min(n, max(S0, S0 * budget_s / max(t0, 1e-3))))
    S = max(S, maxm)
    t = run(S) if S != S0 else t0
    return S, t, cells(S, ents) / t


def host_cpu() -> str:
    """Architecture and model of the host cores, from /proc/cpuinfo where it
    names one (x86 'model name'; Arm 'CPU implementer'/'CPU part' codes)."""
    import platform
    desc = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            info = {}
            for line in f:
                k, _, v = line.partition(":")
                info.setdefault(k.strip(), v.strip())
        if info.get("model name"):
            desc += " " + info["model name"]
        elif info.get("CPU part"):
            desc += f" implementer {info.get('CPU implementer', '?')} part {info['CPU part']}"
    except OSError:
        pass
    return desc


def cpu_baseline(n: int, pats, seconds: float) -> dict:
    """The oracle on all host cores (about `seconds` of work) and on one core
    (a quarter of that), on the first symbols of the GENOME text: window-cells/s
    and Gbp/s (symbols searched per second, summed over the searches)."""
    cores = os.cpu_count() or 1
    nsearch = len(entries(pats))
    S, t, v = oracle_sample(n, pats, seconds, cores)
    S1, t1, v1 = oracle_sample(n, pats, seconds / 4, 1)
    return {"value": v, "unit": "window-cells/s", "cores": cores, "kind": "oracle",
            "cpu": host_cpu(), "gbp_per_s": S * nsearch / t / 1e9,
            "sample": f"first {S} symbols of the same text, all {nsearch} (pattern, k) "
                      f"searches, {t:.1f} s",
            "single_thread": {"value": v1, "unit": "window-cells/s",
                              "gbp_per_s": S1 * nsearch / t1 / 1e9,
                              "sample": f"first {S1} symbols, {t1:.1f} s"}}


# ---------------------------------------------------------------- our arm ---

def run_ours(a):
    import torch
    import torch.distributed as dist
    import paper_1611_06115_gb300 as pm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()

    pats = genome_patterns()
    ents = entries(pats)
    maxm = max(len(p) for p in pats)
    n = a.n
    # rank r owns window starts [r n, (r+1) n) of a world*n text: its piece
    # carries the m-1 overlap of Sec. 2.6 (weak scaling, no collective on the
    # data path)
    from paper_1611_06115_gb300.shard import shard_of
    sh = shard_of(world * n, maxm, world, rank)
    n_local = sh.piece_len
    start = sh.start

    host = torch.empty(n_local, dtype=torch.uint8, pin_memory=True)
    host_np = host.numpy()
    t0 = time.perf_counter()
    planted = build_text(n_local, start, host_np, pats)
    gen_s = time.perf_counter() - t0

    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    text = pm.pm_encode_text(host, stream=stream)
    torch.cuda.synchronize()
    encode_s = time.perf_counter() - t0
    cps = [pm.pm_compile_pattern(p) for p in pats]
    cmap = {p: c for p, c in zip(pats, cps)}
    handles = [cmap[p] for p, _ in ents]
    ks = [k for _, k in ents]

    # the evaluation AUTO runs for each k: measured on this GPU (or read from
    # the tuning cache) before anything is timed
    tuned = None
    if a.variant == 0:
        from paper_1611_06115_gb300 import tune
        t0 = time.perf_counter()
        tv = tune.tune_variants(text, kmax=max(ks) + 1)
        tuned = {"cached": tv["cached"], "seconds": time.perf_counter() - t0, "key": tv["key"]}
    auto = pm.pm_get_auto_variants(64)

    def variant_name(k):
        v = a.variant or (auto[k] if k < 64 else pm.PM_VARIANT_ALL_CHUNKS)
        if v == pm.PM_VARIANT_WINDOW_SLICED and k > 8:
            v = pm.PM_VARIANT_PATTERN_SLICED
        if (v == pm.PM_VARIANT_PATTERN_SLICED and k > 31) or (v == pm.PM_VARIANT_PATTERN_SLICED_2 and k > 63):
            v = pm.PM_VARIANT_ALL_CHUNKS
        return VARIANT_NAMES[v]

    # first search (synchronous) learns the output size and checks the planted copies
    r = pm.pm_search_ex(text, handles, ks, variant=a.variant)
    total = r.total
    per = [r.pattern(i) for i in range(len(ents))]
    for i, (p, k) in enumerate(ents):
        found = dict(zip(per[i][0].tolist(), per[i][1].tolist()))
        pl = planted[pats.index(p)]
        bad = [(loc, s) for loc, s in pl if s <= k and found.get(loc) != s]
        if bad:
            raise SystemExit(f"planted copies missed for m={len(p)} k={k}: {bad[:3]}")
    cap = int(total * 1.05) + 1024
    hits_counts = [int(r.offsets[i + 1] - r.offsets[i]) for i in range(len(ents))]
    del r, per

    n_ev = 2 * len(ents)
    ev_sets = []
    for _ in range(a.steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
        for e in evs:
            e.record(stream)
        ev_sets.append(evs)
    torch.cuda.synchronize()

    hits_buf = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    offs_buf = torch.empty(len(ents) + 1, dtype=torch.int64, device=dev)

    def step(evs):
        return pm_search_into(pm, text, handles, ks, hits_buf, offs_buf, cap, evs, stream,
                              a.variant)

    warm = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    for e in warm:
        e.record(stream)
    for _ in range(max(a.warmup, 3)):
        step(warm)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(dev)
    clocks.start()
    time.sleep(0.3)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_start.record(stream)
    for i in range(a.steps):
        step(ev_sets[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t_start.elapsed_time(t_end) / a.steps
    if world > 1:
        dist.barrier()
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    got_total = int(offs_buf[-1].item())
    if got_total != total:
        raise SystemExit(f"timed searches returned {got_total} hits, expected {total}")

    # per-launch scan durations (event pairs on the launching stream)
    dur = np.array([[ev_sets[s][2 * e].elapsed_time(ev_sets[s][2 * e + 1])
                     for e in range(len(ents))] for s in range(a.steps)])
    mean_ms = dur.mean(axis=0)
    n_cells = cells(n_local, ents)
    value = world * cells(n, ents) / (ms / 1e3)
    text_gbs = world * len(ents) * (n / 4) / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    # dominant kernel: the scan-kernel instance with the largest total time
    def instance(k):
        name = variant_name(k)
        return f"k_scan<{name}, k={k}>" if name == "window-sliced" else f"k_scan<{name}>"
    kinds = {}
    for e, (p, k) in enumerate(ents):
        kinds.setdefault(instance(k), []).append(e)
    dom = max(kinds, key=lambda kk: sum(mean_ms[e] for e in kinds[kk]))
    dom_e = kinds[dom]
    # algorithmic bytes of one launch: the packed text once plus 8 bytes per hit
    alg = [(n_local / 4 + 8 * hits_counts[e]) / (mean_ms[e] / 1e3) for e in dom_e]
    achieved = float(np.mean(alg)) / 1e9
    dom_ms = float(np.mean([mean_ms[e] for e in dom_e]))
    # The scan kernels are bound by the integer ALU pipe (ncu: 78-90 % of it
    # busy, DRAM traffic equal to the algorithmic bytes), so the roofline is
    # the ALU one.  Algorithmic work: the pattern-sliced evaluation of Eq. 4
    # over a window's first 32 positions is 5 ALU-pipe instructions (2 funnel
    # shifts that align the text + 3 selects that apply Table 3 to 32 pairs;
    # the popcount runs on the XU pipe, the threshold on the FMA pipe); with
    # k <= 17 that chunk decides almost every window.  Peak: 64 ALU lanes per
    # SM per clock (the unit count; pm_measure_int_pipe measures 63.7 LOP3 per
    # clock per SM) x SMs x the maximum SM clock.
    alu_peak, alu_peak_kind = alu_peak_of(dev)
    dom_var = variant_name(ents[dom_e[0]][1])
    alu_achieved = float(np.mean([first_stage_ops(dom_var, ents[e][1], len(ents[e][0]))
                                  * (n_local - len(ents[e][0]) + 1) / (mean_ms[e] / 1e3) for e in dom_e]))
    lop = None
    try:
        lop = pm.api.pm_measure_int_pipe(0)
    except Exception as ex:  # the roofline is reported without the cross-check
        lop = {"error": str(ex)}

    # ---- e2e through the public API with host buffers ----
    e2e_times = []
    h2d = d2h = 0
    for it in range(a.e2e_steps + 1 if a.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tx = pm.pm_encode_text(host, stream=stream)
        cc = [pm.pm_compile_pattern(p) for p in pats]
        cm = {p: c for p, c in zip(pats, cc)}
        rr = pm.pm_search_ex(tx, [cm[p] for p, _ in ents], ks, capacity=cap, out="host",
                             stream=stream, variant=a.variant)
        tot = rr.total
        if world > 1:
            # Sec. 2.6 across GPUs: each rank keeps the windows it owns, one
            # gather merges the per-rank lists on rank 0 (sorted by location)
            from paper_1611_06115_gb300 import shard as shard_mod
            mine = [shard_mod.owned(sh, *rr.pattern(i)) for i in range(len(ents))]
            got = [None] * world if rank == 0 else None
            dist.gather_object(mine, got, dst=0)
            if rank == 0:
                merged = shard_mod.merge(got)
        dt = time.perf_counter() - t0
        if it > 0:
            e2e_times.append(dt)
        h2d = n_local + sum(16 * ((len(p) + 31) // 32) for p in pats) + 16 * len(ents)
        d2h = 8 * tot + 8 * (len(ents) + 1)
        del tx, rr
    e2e_s = statistics.median(e2e_times) if e2e_times else float("nan")
    if world > 1:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e_value = world * cells(n, ents) / e2e_s if e2e_times else None

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "window-cells/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": max(a.warmup, 3),
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic: seeded order-2 Markov text, 41% GC, planted noisy copies "
                "(stands in for GRCh37 chr2)",
        "config": {
            "workload": "GENOME: n=3.1e9 per GPU, m in {32,128,1024} (10% classes), "
                        "k in {0,4,16}, 100 planted copies per pattern; 9 searches per step",
            "n_per_gpu": n, "patterns_m": list(MS), "ks": list(KS),
            "searches_per_step": len(ents), "launch": "one scan launch per (pattern, k)",
            "l2": "inputs larger than L2 (775 MB packed text vs 129 MB L2); no flush",
            "parallelism": f"text shards with m-1 overlap x{world}",
            "variant": "auto (tuned)" if a.variant == 0 else VARIANT_NAMES[a.variant],
            "variant_per_k": {str(k): variant_name(k) for k in sorted(set(ks))},
        },
        "tuning": tuned,
        "text_gbs": text_gbs,
        "gbp_per_s": world * len(ents) * n / (ms / 1e3) / 1e9,
        "hits_per_step": total,
        "e2e": {"value": e2e_value, "unit": "window-cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "seconds_per_step": e2e_s,
                "what": "pm_encode_text(pinned host ASCII) + pm_compile_pattern + "
                        "pm_search(host outputs), every step" +
                        ("; then each rank's owned hits gathered and merged on rank 0" if world > 1 else "")},
        "gpu_launches": a.steps * (len(ents) + 5),
        "roofline": {"bound": "alu", "achieved": alu_achieved / 1e12, "peak": alu_peak / 1e12,
                     "unit": "Tops/s (integer ALU-pipe instructions)",
                     "frac": alu_achieved / alu_peak,
                     "peak_kind": alu_peak_kind,
                     "model": ops_model(dom_var, ents[dom_e[0]][1]) + "; windows = n - m + 1 per launch",
                     "measured_lop3": lop,
                     "traffic": traffic(dom, n_local),
                     "traffic_source": TRAFFIC_SOURCE if traffic(dom, n_local) else None,
                     "kernel_source_sha": kernel_source_sha(),
                     "traffic_capture_sha": TRAFFIC_SRC_SHA,
                     "algorithmic_bytes": float(np.mean([n_local / 4 + 8 * hits_counts[e] for e in dom_e])),
                     "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_kind": f"{peak_kind} HBM copy GB/s"},
                     "kernel": dom, "kernel_ms": dom_ms,
                     "launches": [f"m={len(ents[e][0])},k={ents[e][1]}" for e in dom_e],
                     "per_launch_ms": {f"m={len(p)},k={k}": float(t)
                                       for (p, k), t in zip(ents, mean_ms)}},
        "clocks": ck,
        "setup_s": {"generate": gen_s, "encode": encode_s,
                    "encode_gbs": n_local / encode_s / 1e9},
    }
    if rank == 0 and world == 1 and a.batched_n > 0:
        # the batched configuration beside the step (not part of the timed step)
        del text, hits_buf, offs_buf
        torch.cuda.empty_cache()
        line["batched"] = batched_compare(a.batched_n, 2, 1, alu_peak)
    if rank == 0 and world == 1 and a.cpu_seconds > 0:
        line["cpu_baseline"] = cpu_baseline(n, pats, a.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def pm_search_into(pm, text, handles, ks, hits, offs, cap, evs, stream, variant):
    """One step: pm_search_ex into preallocated device buffers, asynchronous."""
    import ctypes
    from paper_1611_06115_gb300 import _native as N
    npat = len(handles)
    harr = (ctypes.c_void_p * npat)(*[h.handle for h in handles])
    karr = (ctypes.c_int32 * npat)(*ks)
    earr = (ctypes.c_void_p * len(evs))(*[e.cuda_event for e in evs])
    opts = N.pm_options(variant, 0, ctypes.cast(earr, ctypes.POINTER(ctypes.c_void_p)))
    st = N.lib().pm_search_ex(text.handle, harr, npat, karr, ctypes.c_void_p(hits.data_ptr()), cap,
                              ctypes.c_void_p(offs.data_ptr()), None, ctypes.byref(opts),
                              ctypes.c_void_p(stream.cuda_stream))
    N.check(st, "pm_search_ex")


# ---------------------------------------------------------- reference arm ---

def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import synth
    pats = genome_patterns()
    ents = entries(pats)
    threads = os.cpu_count() or 1
    budget = a.ref_seconds  # seconds for the whole run
    steps_total = a.steps + max(a.warmup, 3)
    S0 = 2_000_000
    txt0 = synth.markov_text(S0, TEXT_SEED)
    t0 = time.perf_counter()
    for p, k in ents:
        oracle.search(txt0, p, k, threads=threads)
    t_probe = time.perf_counter() - t0
    per_step = budget / steps_total
    S = int(max(max(MS), min(a.n, S0 * per_step / max(t_probe, 1e-4))))
    txt = synth.markov_text(S, TEXT_SEED)

    def step():
        for p, k in ents:
            oracle.search(txt, p, k, threads=threads)

    for _ in range(max(a.warmup, 3)):
        step()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step()
    dt = (time.perf_counter() - t0) / a.steps
    v = cells(S, ents) / dt
    line = {
        "impl": "reference",
        "metric": METRIC, "value": v, "unit": "window-cells/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": max(a.warmup, 3), "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic: seeded order-2 Markov text, 41% GC",
        "config": {"workload": "GENOME recipe, bounded sample: first "
                               f"{S} symbols of the 3.1e9 text, m in {{32,128,1024}}, "
                               "k in {0,4,16}; 9 searches per step",
                   "sample_symbols": S},
        "cpu_baseline": {"value": v, "unit": "window-cells/s", "cores": threads, "kind": "oracle",
                         "cpu": host_cpu(), "sample": f"first {S} symbols per step"},
        "e2e": {"value": v, "unit": "window-cells/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_compare(n: int, reps: int, warmup: int, alu_peak: float | None = None, options=None) -> dict:
    """The BATCHED workload (n-symbol Markov text, 4096 patterns, m log-uniform
    in 12..512, k uniform in 0..m/8, one planted copy each): the whole batch
    as one pm_batch run (one persistent launch per category of evaluation
    plus the ordering, in one CUDA graph) against one launch per pattern
    (pm_search_ex), both checked against each other, timed with CUDA events
    over `reps` runs after `warmup`."""
    import torch
    import paper_1611_06115_gb300 as pm
    from synth import workloads
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    w = workloads.batched(n=n, count=4096, out=host.numpy())
    text = pm.pm_encode_text(host)
    cps = [pm.pm_compile_pattern(p) for p in w.patterns]
    ks = [kk[0] for kk in w.ks]
    ref = pm.pm_search(text, cps, ks)
    cap = ref.total + 1024
    for i, pl in enumerate(w.planted):
        l, c = ref.pattern(i)
        found = dict(zip(l.tolist(), c.tolist()))
        assert all(found.get(loc) == s for loc, s in pl), f"planted copy missed, pattern {i}"
    opts = dict(options or {})
    g = pm.GraphedBatch(pm.Batch(text, cps, ks, capacity=cap, **opts))

    def timed(fn):
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(max(warmup, 1)):
            fn()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    t_batch = timed(g.replay)
    out = g.out
    assert out.total == ref.total and np.array_equal(out.numpy()[0], ref.numpy()[0])
    del g, out
    t_per = timed(lambda: pm.pm_search_ex(text, cps, ks, capacity=cap, sync=False))
    n_cells = sum((n - len(p) + 1) * len(p) for p in w.patterns)
    res = {"workload": "BATCHED: n=1e9 Markov text, 4096 patterns, m log-uniform 12..512, "
                       "k uniform 0..m/8, 10% classes", "n": n, "patterns": len(cps),
           "seconds_one_batch": t_batch, "seconds_per_pattern_launches": t_per,
           "batched_over_per_pattern": t_per / t_batch, "hits": ref.total,
           "window_cells_per_s": n_cells / t_batch, "options": opts,
           "launch": "one persistent launch per category of evaluation + ordering, one CUDA graph"}
    if alu_peak:
        # algorithmic first-stage ALU instructions of each pair (first_stage_ops)
        ob = {"ws_below": 9, "ps1_below": 18, "ps2_below": 41}
        ob.update({k: v for k, v in opts.items() if k in ob and v})
        auto = pm.pm_get_auto_variants(64)

        def var_batch(k, m):
            if k < ob["ws_below"]:
                return "window-sliced"
            if k < ob["ps1_below"] or (m <= 32 and k <= 31):
                return "pattern-sliced"
            return "pattern-sliced-64" if k < ob["ps2_below"] else "all-chunks"

        def var_auto(k, m):
            v = VARIANT_NAMES[auto[k]] if k < 64 else "all-chunks"
            return "pattern-sliced" if v == "pattern-sliced-64" and m <= 32 and k <= 31 else v

        ops_b = sum(first_stage_ops(var_batch(k, len(p)), k, len(p)) * (n - len(p) + 1)
                    for p, k in zip(w.patterns, ks))
        ops_p = sum(first_stage_ops(var_auto(k, len(p)), k, len(p)) * (n - len(p) + 1)
                    for p, k in zip(w.patterns, ks))
        res["integer_pipe"] = {
            "bound": "alu", "unit": "Tops/s (integer ALU-pipe instructions)", "peak": alu_peak / 1e12,
            "one_batch": {"achieved": ops_b / t_batch / 1e12, "frac": ops_b / t_batch / alu_peak},
            "per_pattern_launches": {"achieved": ops_p / t_per / 1e12, "frac": ops_p / t_per / alu_peak},
            "model": "per pair, first-stage ALU instructions per window of its evaluation "
                     "(bench.first_stage_ops) x (n - m + 1) windows"}
    return res


def alu_peak_of(dev) -> tuple[float, str]:
    """64 ALU lanes per SM per clock x SMs x the maximum SM clock."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            sm_max_mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        sm_max_mhz = 2070.0
    return (64 * props.multi_processor_count * sm_max_mhz * 1e6,
            f"derived: 64 ALU lanes/clk/SM x {props.multi_processor_count} SMs x {sm_max_mhz:.0f} MHz")


def run_batched(a):
    """BATCHED alone (see batched_compare), with the batch options picked by
    the autotuner (or the defaults with --no-tune)."""
    import torch
    import paper_1611_06115_gb300 as pm
    from synth import workloads
    from paper_1611_06115_gb300 import tune
    n = min(a.n, workloads.BATCHED_N)
    opts, tune_info = {}, None
    if not a.no_tune:
        host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        w = workloads.batched(n=n, count=4096, out=host.numpy())
        text = pm.pm_encode_text(host)
        cps = [pm.pm_compile_pattern(p) for p in w.patterns]
        ks = [kk[0] for kk in w.ks]
        cap = pm.pm_search(text, cps, ks).total + 1024
        t0 = time.perf_counter()
        tv = tune.tune_variants(text, kmax=64)
        tb = tune.tune_batch(text, cps, ks, cap, sample=256)
        opts = tb["options"]
        tune_info = {"seconds": time.perf_counter() - t0, "variants_cached": tv["cached"],
                     "batch_cached": tb["cached"], "batch_key": tb["key"],
                     "candidates_timed": len(tb["log"]), "whole_batch_check": tb.get("checked")}
        del text, host, cps
    peak, _ = alu_peak_of(torch.cuda.current_device())
    res = batched_compare(n, max(1, min(a.steps, 3)), a.warmup, peak, options=opts)
    res.update({"metric": METRIC, "unit": "window-cells/s", "value": res["window_cells_per_s"],
                "tuning": tune_info})
    print(json.dumps(res), flush=True)


def run_serving(a):
    """SERVING: Poisson arrivals (default 2000 queries/s for 10 s), m log-uniform
    in 16..4096, k in 0..8, against the resident GENOME text; continuous
    batching over 4 streams, admission by device memory."""
    import torch
    import paper_1611_06115_gb300 as pm
    from paper_1611_06115_gb300 import serve
    from synth import workloads
    n = a.n
    pats = genome_patterns()
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    build_text(n, 0, host.numpy(), pats)
    text = pm.pm_encode_text(host)
    qs = workloads.serving_queries(rate=a.rate, duration=a.duration)
    queries = [(q.arrival, q.pattern, q.k) for q in qs]
    # the evaluation each k of the mix runs: measured on this GPU (or cached)
    from paper_1611_06115_gb300 import tune
    tv = tune.tune_variants(text, kmax=max(q.k for q in qs) + 1)
    to_host = a.serve_delivery == "host"
    backend = serve.GpuBackend(text, slots=a.serve_slots, batch={} if a.serve_mode == "one-launch" else None,
                               copy_to_host=to_host)
    # the client takes each result as it completes and lets go of it, so the
    # pinned buffers return to the allocator
    def server():
        return serve.Server(backend, n=n, slots=a.serve_slots, max_batch=32, mem_budget=32 << 30,
                            keep_hits=False)
    # warm the kernels, the device pool and the pinned-host pool
    serve.run_trace(server(), queries[:200])
    srv = server()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    stats = serve.run_trace(srv, queries)
    torch.cuda.synchronize()
    ck = clocks.stop()
    n_cells = sum((n - len(r.pattern) + 1) * len(r.pattern) for r in srv.done)
    stats.update({"workload": "SERVING", "mode": a.serve_mode, "slots": a.serve_slots, "n": n,
                  "offered_rate_qps": a.rate,
                  "variant_per_k": {str(k): VARIANT_NAMES[v] for k, v in enumerate(tv["table"])},
                  "arrival_seconds": a.duration, "queries": len(queries),
                  "window_cells_per_s": n_cells / stats["span_s"],
                  "hits": int(sum(max(r.count, 0) for r in srv.done)), "clocks": ck,
                  "admission": "letter frequencies measured on the resident text",
                  "delivery": a.serve_delivery,
                  "note": ("latency = hits in pinned host memory minus arrival" if to_host else
                           "latency = hits on the device minus arrival (no copy to the host)") +
                          "; the client drops each result after delivery; saturation when "
                          "offered load exceeds the sustainable rate"})
    print(json.dumps(stats), flush=True)


def run_large(a):
    """LARGE: the 3.1 Gbp Markov text, patterns m in {1e4, 1e5} with 5 % class
    positions and 10 planted copies each (s uniform in 0..500), k in {0, 100,
    1000}: kernel time per search (CUDA events around the scan launch) and
    the whole pm_search call; every planted copy with s <= k must be found
    with its exact count."""
    import torch
    import paper_1611_06115_gb300 as pm
    from synth import workloads
    n = a.n
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    w = workloads.large(n=n, out=host.numpy())
    text = pm.pm_encode_text(host)
    del host
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for e in ev:
        e.record(st)
    rows = []
    for p, pl in zip(w.patterns, w.planted):
        c = pm.pm_compile_pattern(p)
        for k in w.meta["ks"]:
            best_k, best_call = float("inf"), float("inf")
            for rep in range(max(a.steps, 1) + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = pm.pm_search_ex(text, [c], [k], events=ev)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if rep:
                    best_k = min(best_k, ev[0].elapsed_time(ev[1]) / 1e3)
                    best_call = min(best_call, dt)
            found = dict(zip(*[x.tolist() for x in r.pattern(0)]))
            ok = all(found.get(loc) == s for loc, s in pl if s <= k)
            if not ok:
                raise SystemExit(f"LARGE: planted copy missed for m={len(p)} k={k}")
            cells = (n - len(p) + 1) * len(p)
            rows.append({"m": len(p), "k": k, "kernel_s": best_k, "call_s": best_call,
                         "hits": r.total, "window_cells_per_s": cells / best_k})
    print(json.dumps({"workload": "LARGE", "metric": METRIC, "n": n, "searches": rows,
                      "planted_found": True}), flush=True)


def run_profile(a):
    """Five single searches of the GENOME m = 128 pattern over the first n
    symbols, one per kernel kind, for a small ncu capture:
    (window-sliced, k = 0), (window-sliced, 4), (window-sliced, 8),
    (pattern-sliced, 16), (pattern-sliced over 64 positions, 24)."""
    import torch
    import paper_1611_06115_gb300 as pm
    pats = genome_patterns()
    host = torch.empty(a.n, dtype=torch.uint8, pin_memory=True)
    build_text(a.n, 0, host.numpy(), pats)
    text = pm.pm_encode_text(host)
    c = pm.pm_compile_pattern(pats[1])
    for v, k in ((2, 0), (2, 4), (2, 8), (1, 16), (3, 24)):
        r = pm.pm_search_ex(text, [c], [k], variant=v)
        print(json.dumps({"variant": v, "k": k, "hits": r.total}), flush=True)


if __name__ == "__main__":
    a = args_()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "profile":
        run_profile(a)
    elif a.workload == "large":
        run_large(a)
    elif a.workload == "batched":
        run_batched(a)
    elif a.workload == "serving":
        run_serving(a)
    else:
        run_ours(a)
