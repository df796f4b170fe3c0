"""Autotuner: picks, by measurement on the current GPU, how the search runs.

Every choice below gives bit-identical hits (they are equivalent evaluations
of Eq. 4 with the early stop of Sec. 2.4-2.5); only the time differs, and it
depends on the GPU, on k and on the text's statistics.  Two things are tuned:

* the variant PM_VARIANT_AUTO runs for each k (``tune_variants``): every
  evaluation that is valid at that k is timed on synthetic patterns of a few
  lengths over the resident text, and the fastest is installed with
  pm_set_auto_variants;
* the options of a batched launch (``tune_batch``): the k thresholds between
  its evaluations, the warp tiles per work item (how many tiles a warp walks
  with one row of pairs loaded) and the grid, by coordinate descent from
  the library's defaults, each candidate timed on a sample of the batch.

Results are cached in a JSON file (``PM_TUNE_CACHE``, default
``~/.cache/paper_1611_06115_gb300/tune.json``) keyed by the device (name and
SM count), the text length (log2 bucket) and, for batches, by the batch size,
m and k buckets, so a later run on the same kind of GPU and workload reuses
them without measuring.

The measuring parts take a ``timer`` callable, so the selection logic, the
coordinate descent and the cache can be exercised without a GPU.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable

import numpy as np

from . import _native as N

VARIANT_NAMES = {N.PM_VARIANT_PATTERN_SLICED: "pattern-sliced",
                 N.PM_VARIANT_WINDOW_SLICED: "window-sliced",
                 N.PM_VARIANT_PATTERN_SLICED_2: "pattern-sliced-64",
                 N.PM_VARIANT_ALL_CHUNKS: "all-chunks"}

# the batch options tuned, their candidate values, in descent order
BATCH_SPACE = (
    ("ws_below", (1, 3, 5, 7, 9)),
    ("ps1_below", (12, 15, 18, 21, 24)),
    ("ps2_below", (33, 37, 41, 45, 49)),
    ("tiles", (2, 4, 8, 16, 32, 64)),
    ("grid", (0,)),  # extended at run time with fractions of the resident grid
)
BATCH_DEFAULTS = {"ws_below": 9, "ps1_below": 18, "ps2_below": 41, "tiles": 16, "grid": 0}


def valid_variants(k: int) -> list[int]:
    """The evaluations that exist at this k (include/pm.h, pm_search_ex)."""
    out = []
    if k <= 8:
        out.append(N.PM_VARIANT_WINDOW_SLICED)
    if k <= 31:
        out.append(N.PM_VARIANT_PATTERN_SLICED)
    if k <= 63:
        out.append(N.PM_VARIANT_PATTERN_SLICED_2)
    out.append(N.PM_VARIANT_ALL_CHUNKS)
    return out


# ------------------------------------------------------------------- cache --

def cache_path() -> str:
    return os.environ.get("PM_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1611_06115_gb300", "tune.json")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(data: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _bucket(x: int) -> int:
    return int(math.ceil(math.log2(max(int(x), 1))))


def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}"


def variants_key(device: str, n: int) -> str:
    return f"variants|{device}|n2^{_bucket(n)}"


def batch_key(device: str, n: int, ms, ks) -> str:
    ms = np.asarray(ms)
    ks = np.asarray(ks)
    hist = lambda a, edges: ",".join(str(int(c)) for c in np.histogram(a, bins=edges)[0] * 8 // max(len(a), 1))
    return (f"batch|{device}|n2^{_bucket(n)}|npat2^{_bucket(len(ms))}"
            f"|m{hist(ms, [0, 33, 129, 513, 1 << 30])}|k{hist(ks, [0, 5, 18, 41, 1 << 30])}")


# ------------------------------------------------------------ variant table --

def select_variants(times: dict[int, dict[int, float]]) -> list[int]:
    """The fastest variant per k from times[k][variant] (ms); k = 0 .. K-1
    must all be present."""
    table = []
    for k in range(len(times)):
        t = times[k]
        best = min(sorted(t), key=lambda v: (t[v], v))
        if best not in valid_variants(k):
            raise ValueError(f"variant {best} is not valid at k = {k}")
        table.append(best)
    return table


def probe_pattern(m: int, rng: np.random.Generator, class_fraction: float = 0.1) -> str:
    """A probe pattern: uniform letters, about class_fraction of the positions
    two- or three-letter IUPAC classes."""
    sym = np.array(list("ACGT"))[rng.integers(0, 4, size=m)]
    classes = np.array(list("MRWSYKVHDB"))
    pos = rng.choice(m, size=int(round(class_fraction * m)), replace=False)
    sym[pos] = classes[rng.integers(0, len(classes), size=pos.size)]
    return "".join(sym)


def measure_variants(text, ks, ms=(128, 1024), reps: int = 3, seed: int = 0) -> dict:
    """times[k][variant] = summed min-of-reps kernel ms over one probe
    pattern per length in ms, searched alone over the text with that
    variant."""
    import torch
    from . import api
    rng = np.random.default_rng(seed)
    pats = [api.pm_compile_pattern(probe_pattern(int(m), rng)) for m in ms]
    st = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for e in ev:
        e.record(st)
    times: dict[int, dict[int, float]] = {}
    with torch.cuda.stream(st):
        for k in ks:
            times[k] = {}
            for v in valid_variants(k):
                total = 0.0
                for p in pats:
                    best = float("inf")
                    for r in range(reps + 1):
                        api.pm_search_ex(text, [p], [k], capacity=1 << 22, stream=st, sync=False,
                                         variant=v, events=ev)
                        st.synchronize()
                        if r:
                            best = min(best, ev[0].elapsed_time(ev[1]))
                    total += best
                times[k][v] = total
    return times


def tune_variants(text, kmax: int = 64, ms=(128, 1024), reps: int = 3, cache: str | None = None,
                  retune: bool = False, timer: Callable | None = None, install: bool = True) -> dict:
    """Pick and install the PM_VARIANT_AUTO table for k < kmax (<= 64).

    timer: None to measure on the GPU, else timer(ks) -> times[k][variant].
    Returns {"key", "table", "times", "cached"}.
    """
    from . import api
    kmax = min(int(kmax), 64)
    dev = device_key() if timer is None else "test-device"
    key = variants_key(dev, text.n if hasattr(text, "n") else int(text))
    data = load_cache(cache)
    entry = data.get(key)
    if entry and not retune and len(entry.get("table", [])) >= kmax:
        table = entry["table"][:kmax]
        if install:
            api.pm_set_auto_variants(table)
        return {"key": key, "table": table, "times": entry.get("times"), "cached": True}
    ks = list(range(kmax))
    times = timer(ks) if timer is not None else measure_variants(text, ks, ms, reps)
    table = select_variants({k: times[k] for k in ks})
    data[key] = {"table": table, "times": {str(k): {str(v): t for v, t in times[k].items()} for k in ks}}
    save_cache(data, cache)
    if install:
        api.pm_set_auto_variants(table)
    return {"key": key, "table": table, "times": data[key]["times"], "cached": False}


# ------------------------------------------------------------ batch options --

def coordinate_descent(timer: Callable[[dict], float], space=BATCH_SPACE, start=None,
                       rounds: int = 2) -> tuple[dict, float, list]:
    """Minimise timer(options) one option at a time over its candidate
    values, `rounds` sweeps or until a sweep changes nothing.  Returns (best
    options, its time, every (options, time) measured)."""
    best = dict(start or BATCH_DEFAULTS)
    seen: dict[tuple, float] = {}
    log = []

    def t(o):
        key = tuple(sorted(o.items()))
        if key not in seen:
            seen[key] = float(timer(dict(o)))
            log.append((dict(o), seen[key]))
        return seen[key]

    best_t = t(best)
    for _ in range(rounds):
        changed = False
        for name, values in space:
            for v in values:
                if v == best[name]:
                    continue
                cand = dict(best, **{name: v})
                ct = t(cand)
                if ct < best_t:
                    best, best_t, changed = cand, ct, True
        if not changed:
            break
    return best, best_t, log


def sample_batch(patterns, k, size: int, seed: int = 0):
    """A stratified sample of the batch (by k, then m) of at most `size` pairs."""
    idx = np.lexsort((np.array([len(p) if isinstance(p, str) else p.m for p in patterns]), np.array(k)))
    if len(idx) <= size:
        return list(idx)
    return [int(idx[int(i)]) for i in np.linspace(0, len(idx) - 1, size)]


def tune_batch(text, patterns, k, capacity: int, sample: int = 512, reps: int = 2,
               cache: str | None = None, retune: bool = False, timer: Callable | None = None,
               full_timer: Callable | None = None) -> dict:
    """Options for a pm_batch_create of these pairs: cached, else found by
    coordinate descent over BATCH_SPACE, each candidate timed as one
    batched launch over a stratified sample of at most `sample` pairs.  A
    sample can favour options that do not carry over to the whole batch, so
    the winner is then timed on the whole batch against the defaults and the
    faster of the two is kept.

    patterns: compiled Pattern objects (or, with a timer, anything with an m).
    timer: None to measure on the GPU, else timer(options) -> ms on the
    sample; full_timer likewise on the whole batch (None with a timer: no
    check against the defaults).
    Returns {"key", "options", "ms", "cached", "log", "checked"}.
    """
    ks = [int(x) for x in (k if not np.isscalar(k) else [k] * len(patterns))]
    ms = [p.m if hasattr(p, "m") else len(p) for p in patterns]
    dev = device_key() if timer is None else "test-device"
    n = text.n if hasattr(text, "n") else int(text)
    key = batch_key(dev, n, ms, ks)
    data = load_cache(cache)
    entry = data.get(key)
    if entry and not retune:
        return {"key": key, "options": entry["options"], "ms": entry.get("ms"), "cached": True, "log": [],
                "checked": entry.get("checked")}
    space = list(BATCH_SPACE)
    if timer is None:
        import torch
        from . import api
        idx = sample_batch(patterns, ks, sample)
        sp = [patterns[i] for i in idx]
        sk = [ks[i] for i in idx]
        cap = max(int(capacity * len(idx) / max(len(ks), 1)) * 2, 1 << 20)
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        space[-1] = ("grid", (0, sms, 2 * sms))
        st = torch.cuda.Stream()

        def gpu_time(pats, kk, cp, o):
            b = api.Batch(text, pats, kk, capacity=cp, stream=st, **o)
            out = b.buffers()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = float("inf")
            with torch.cuda.stream(st):
                for r in range(reps + 1):
                    e0.record(st)
                    b.run(out, stream=st)
                    e1.record(st)
                    st.synchronize()
                    if r:
                        best = min(best, e0.elapsed_time(e1))
            b.free()
            return best

        def timer(o):  # noqa: F811 - the GPU timer on the sample
            return gpu_time(sp, sk, cap, o)

        if full_timer is None:
            def full_timer(o):  # on the whole batch
                return gpu_time(patterns, ks, capacity, o)
    opts, t, log = coordinate_descent(timer, space)
    checked = None
    if full_timer is not None and opts != BATCH_DEFAULTS:
        t_best, t_def = float(full_timer(opts)), float(full_timer(dict(BATCH_DEFAULTS)))
        checked = {"tuned_ms": t_best, "default_ms": t_def}
        if t_def <= t_best:
            opts, t = dict(BATCH_DEFAULTS), t_def
    data[key] = {"options": opts, "ms": t, "checked": checked}
    save_cache(data, cache)
    return {"key": key, "options": opts, "ms": t, "cached": False, "log": log, "checked": checked}
