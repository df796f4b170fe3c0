"""Python binding of libpm, with the C ABI's names (include/pm.h).

Marshalling only: every step of the search runs in the library's CUDA
kernels.  PyTorch provides device memory (output tensors), pinned host memory
and streams.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _buffer(data) -> tuple[int, int, object]:
    """(address, length, keep-alive) of a contiguous byte buffer."""
    if isinstance(data, torch.Tensor):
        if data.dtype != torch.uint8 or not data.is_contiguous():
            raise TypeError("text tensor must be contiguous uint8")
        return data.data_ptr(), data.numel(), data
    if isinstance(data, str):
        data = data.encode("ascii")
    if isinstance(data, (bytes, bytearray, memoryview)):
        arr = np.frombuffer(bytes(data), dtype=np.uint8)
    else:
        arr = np.ascontiguousarray(np.asarray(data, dtype=np.uint8))
    return arr.ctypes.data, arr.size, arr


class Text:
    """An encoded, device-resident text (handle owned by the library)."""

    def __init__(self, handle: ctypes.c_void_p, n: int):
        self._h = handle
        self.n = n

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def planes(self) -> tuple[int, int]:
        """(device address, bytes) of the coded bit planes."""
        p, b = ctypes.c_void_p(), ctypes.c_uint64()
        N.check(N.lib().pm_text_device_planes(self._h, ctypes.byref(p), ctypes.byref(b)),
                "pm_text_device_planes")
        return int(p.value or 0), int(b.value)

    def save(self, path: str) -> None:
        """Write the coded text to a file (pm_text_save)."""
        N.check(N.lib().pm_text_save(self._h, os.fsencode(path)), "pm_text_save")

    @classmethod
    def load(cls, path: str, stream=None) -> "Text":
        """Read a coded text written by save() onto the current device
        (pm_text_load)."""
        out = ctypes.c_void_p()
        N.check(N.lib().pm_text_load(os.fsencode(path), _stream(stream), ctypes.byref(out)),
                "pm_text_load")
        return cls(out, int(N.lib().pm_text_length(out)))

    def unknown(self) -> int:
        """Symbols coded as unknown (pm_text_unknown)."""
        return int(N.lib().pm_text_unknown(self._h))

    def letter_counts(self) -> list[int]:
        """How many A, C, G, T the text holds (pm_text_letter_counts)."""
        arr = (ctypes.c_uint64 * 4)()
        N.check(N.lib().pm_text_letter_counts(self._h, arr), "pm_text_letter_counts")
        return list(arr)

    def free(self):
        if self._h is not None and self._h.value:
            N.lib().pm_text_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Pattern:
    """A compiled pattern (host data owned by the library)."""

    def __init__(self, handle: ctypes.c_void_p, iupac: str):
        self._h = handle
        self.iupac = iupac
        self.m = int(N.lib().pm_pattern_length(handle))
        self.unknown = int(N.lib().pm_pattern_unknown(handle))

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def masks(self) -> np.ndarray:
        """(ceil(m/32), 4) uint32 membership words A, C, G, T per 32-position chunk."""
        nch = (self.m + 31) // 32
        buf = np.zeros(4 * nch, dtype=np.uint32)
        N.check(N.lib().pm_pattern_masks(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                         buf.size), "pm_pattern_masks")
        return buf.reshape(nch, 4)

    def free(self):
        if self._h is not None and self._h.value:
            N.lib().pm_pattern_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def pm_encode_text(ascii, stream=None) -> Text:
    """Code a text with Table 1 into device-resident bit planes.

    ``ascii``: bytes, str, numpy uint8 array, or uint8 tensor (host, pinned
    host, or CUDA).  Raises PmError(PM_E_SYMBOL) on a byte outside ACGT/acgt.
    """
    ptr, n, keep = _buffer(ascii)
    out = ctypes.c_void_p()
    N.check(N.lib().pm_encode_text(ctypes.c_void_p(ptr), n, _stream(stream), ctypes.byref(out)),
            "pm_encode_text")
    del keep
    return Text(out, n)


def pm_encode_text_ex(ascii, flags: int = 0, stream=None) -> Text:
    """pm_encode_text with flags (include/pm.h); PM_TEXT_UNKNOWN_AS_N accepts
    bytes outside ACGT as unknown symbols, matched by the class N only."""
    ptr, n, keep = _buffer(ascii)
    out = ctypes.c_void_p()
    N.check(N.lib().pm_encode_text_ex(ctypes.c_void_p(ptr), n, int(flags), _stream(stream),
                                      ctypes.byref(out)), "pm_encode_text_ex")
    del keep
    return Text(out, n)


def pm_compile_pattern(iupac) -> Pattern:
    """Code a pattern with Table 2 (unknown symbols become "-")."""
    b = iupac.encode("ascii") if isinstance(iupac, str) else bytes(iupac)
    out = ctypes.c_void_p()
    N.check(N.lib().pm_compile_pattern(b, len(b), ctypes.byref(out)), "pm_compile_pattern")
    return Pattern(out, b.decode("ascii", errors="replace"))


@dataclass
class SearchResult:
    """hits: (capacity, 2) int32 tensor of (location, mismatches) as uint32 bits;
    offsets: (npat + 1,) int64 tensor; pattern p owns hits[offsets[p]:offsets[p+1]]."""
    hits: torch.Tensor
    offsets: torch.Tensor

    @property
    def total(self) -> int:
        return int(self.offsets[-1].item())

    def numpy(self) -> tuple[np.ndarray, np.ndarray]:
        off = self.offsets.cpu().numpy().astype(np.uint64)
        tot = int(off[-1])
        h = self.hits[:tot].cpu().numpy().view(np.uint32).reshape(-1, 2)
        return h, off

    def pattern(self, p: int) -> tuple[np.ndarray, np.ndarray]:
        """(locations uint32, mismatches uint32) of pattern p."""
        h, off = self.numpy()
        seg = h[int(off[p]):int(off[p + 1])]
        return seg[:, 0].copy(), seg[:, 1].copy()


def _event_handles(events) -> ctypes.Array | None:
    if events is None:
        return None
    arr = (ctypes.c_void_p * len(events))()
    for i, e in enumerate(events):
        arr[i] = e if isinstance(e, int) else e.cuda_event
    return arr


def pm_search_ex(text: Text, patterns, k, capacity: int | None = None, out: str = "device",
                 stream=None, variant: int = N.PM_VARIANT_AUTO, grid: int = 0, events=None,
                 sync: bool = True, batch: dict | None = None) -> SearchResult:
    """Search every pattern (with its k) over the text; see pm_search in include/pm.h.

    capacity None: start from an estimate and grow on PM_E_OVERFLOW.
    out: "device" (CUDA tensors) or "host" (pinned CPU tensors).
    sync False (device output, explicit capacity): asynchronous; read
    ``result.offsets[-1]`` after the stream to learn the total.
    events: None or 2 * len(patterns) torch.cuda.Event objects, already created
    (recorded once), recorded around each pattern's scan kernel.
    batch: None for one scan launch per pattern, else a dict of batch options
    (``Batch.OPTIONS``; {} for the defaults): all pairs in one persistent
    launch with stream-ordered scratch.
    """
    pats = list(patterns)
    npat = len(pats)
    ks = [int(k)] * npat if np.isscalar(k) else [int(x) for x in k]
    if len(ks) != npat:
        raise ValueError("one k per pattern")
    handles = (ctypes.c_void_p * max(npat, 1))(*[p.handle for p in pats])
    karr = (ctypes.c_int32 * max(npat, 1))(*ks)
    ev = _event_handles(events)
    if ev is not None and len(ev) != 2 * npat:
        raise ValueError("events must hold 2 per pattern")
    bopts = None
    if batch is not None:
        unknown = set(batch) - set(Batch.OPTIONS)
        if unknown:
            raise ValueError(f"unknown batch options {sorted(unknown)}")
        bopts = N.pm_batch_options(**{name: int(batch.get(name, 0)) for name in Batch.OPTIONS})
    opts = N.pm_options(variant, grid, ctypes.cast(ev, ctypes.POINTER(ctypes.c_void_p)) if ev else None,
                        ctypes.pointer(bopts) if bopts is not None else None)
    grow = capacity is None
    cap = int(capacity) if capacity is not None else 1 << 20
    if not sync and (out != "device" or grow):
        raise ValueError("asynchronous search needs device output and an explicit capacity")
    dev = torch.cuda.current_device()
    while True:
        if out == "device":
            hits = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev)
            offsets = torch.empty(npat + 1, dtype=torch.int64, device=dev)
        elif out == "host":
            hits = torch.empty((max(cap, 1), 2), dtype=torch.int32, pin_memory=True)
            offsets = torch.empty(npat + 1, dtype=torch.int64, pin_memory=True)
        else:
            raise ValueError("out must be 'device' or 'host'")
        needed = ctypes.c_uint64(0)
        st = N.lib().pm_search_ex(text.handle, handles, npat, karr,
                                  ctypes.c_void_p(hits.data_ptr()), cap,
                                  ctypes.c_void_p(offsets.data_ptr()),
                                  ctypes.byref(needed) if sync else None, ctypes.byref(opts),
                                  _stream(stream))
        if st == N.PM_E_OVERFLOW and grow:
            cap = int(needed.value)
            continue
        N.check(st, "pm_search")
        return SearchResult(hits, offsets)


def pm_search(text: Text, patterns, k, capacity: int | None = None, out: str = "device",
              stream=None) -> SearchResult:
    """pm_search of include/pm.h (default options)."""
    return pm_search_ex(text, patterns, k, capacity=capacity, out=out, stream=stream)


class Batch:
    """A batch of (pattern, k) pairs resident on the device (pm_batch_create).

    ``run`` queues one persistent launch plus the ordering kernels into the
    given device buffers without allocating or waiting, so it can be
    captured in a CUDA graph (see ``GraphedBatch``).
    """

    OPTIONS = ("group", "grid", "tiles", "ws_below", "ps1_below", "ps2_below")

    def __init__(self, text: Text, patterns, k, capacity: int, group: int = 0, grid: int = 0,
                 tiles: int = 0, ws_below: int = 0, ps1_below: int = 0, ps2_below: int = 0,
                 stream=None):
        """Options as pm_batch_options in include/pm.h (0: default)."""
        pats = list(patterns)
        self.npat = len(pats)
        ks = [int(k)] * self.npat if np.isscalar(k) else [int(x) for x in k]
        if len(ks) != self.npat:
            raise ValueError("one k per pattern")
        handles = (ctypes.c_void_p * max(self.npat, 1))(*[p.handle for p in pats])
        karr = (ctypes.c_int32 * max(self.npat, 1))(*ks)
        opts = N.pm_batch_options(group, grid, tiles, ws_below, ps1_below, ps2_below)
        self.options = dict(group=group, grid=grid, tiles=tiles, ws_below=ws_below,
                            ps1_below=ps1_below, ps2_below=ps2_below)
        out = ctypes.c_void_p()
        N.check(N.lib().pm_batch_create(text.handle, handles, self.npat, karr, int(capacity),
                                        ctypes.cast(ctypes.byref(opts), ctypes.c_void_p),
                                        _stream(stream), ctypes.byref(out)), "pm_batch_create")
        self._h = out
        self._text = text  # the text must outlive the batch
        self.capacity = int(capacity)

    def buffers(self, device=None) -> SearchResult:
        dev = torch.cuda.current_device() if device is None else device
        return SearchResult(torch.empty((max(self.capacity, 1), 2), dtype=torch.int32, device=dev),
                            torch.empty(self.npat + 1, dtype=torch.int64, device=dev))

    def run(self, out: SearchResult | None = None, stream=None) -> SearchResult:
        """Queue the batch into ``out`` (device buffers; allocated if None).
        Asynchronous: read ``out.total`` after the stream; a total above the
        capacity means nothing was written."""
        if out is None:
            out = self.buffers()
        N.check(N.lib().pm_batch_run(self._h, ctypes.c_void_p(out.hits.data_ptr()),
                                     ctypes.c_void_p(out.offsets.data_ptr()), _stream(stream)),
                "pm_batch_run")
        return out

    def free(self):
        if self._h is not None and self._h.value:
            N.lib().pm_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class GraphedBatch:
    """A Batch run captured once in a CUDA graph and replayed.

    Replays reuse the same output buffers (``self.out``); each replay
    rewrites them completely.
    """

    def __init__(self, batch: Batch):
        self.batch = batch
        self.out = batch.buffers()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            batch.run(self.out, stream=s)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            batch.run(self.out, stream=torch.cuda.current_stream())

    def replay(self) -> SearchResult:
        self.graph.replay()
        return self.out


INT_OPS = ("LOP3", "SHF", "POPC", "IMAD", "MMA_S8_M16N8K32", "MMA_B1_M16N8K256", "MMA_B1_M16N8K128")


def pm_set_auto_variants(variant_for_k) -> None:
    """Install the PM_VARIANT_AUTO table of the current device for k = 0 ..
    len(variant_for_k) - 1 (see include/pm.h); an empty list restores the
    built-in table."""
    v = [int(x) for x in variant_for_k]
    arr = (ctypes.c_int32 * max(len(v), 1))(*v)
    N.check(N.lib().pm_set_auto_variants(arr, len(v)), "pm_set_auto_variants")


def pm_get_auto_variants(nk: int = 64) -> list[int]:
    """The variants PM_VARIANT_AUTO runs on the current device for k < nk."""
    arr = (ctypes.c_int32 * max(nk, 1))()
    N.check(N.lib().pm_get_auto_variants(arr, nk), "pm_get_auto_variants")
    return list(arr)[:nk]


def pm_check_bounded_wait(limit_ns: int, arrive: bool) -> bool:
    """Run the kernels' bounded barrier wait once (include/pm.h); True when
    it gave up after limit_ns."""
    out = ctypes.c_uint32(0)
    N.check(N.lib().pm_check_bounded_wait(int(limit_ns), 1 if arrive else 0, ctypes.byref(out)),
            "pm_check_bounded_wait")
    return bool(out.value)


def pm_measure_int_pipe(op: int, iters: int = 20000) -> dict:
    """Measured throughput of one integer instruction kind (see include/pm.h)."""
    ops, mhz, per = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    N.check(N.lib().pm_measure_int_pipe(op, iters, ctypes.byref(ops), ctypes.byref(mhz),
                                        ctypes.byref(per)), "pm_measure_int_pipe")
    return {"op": INT_OPS[op], "ops_per_s": ops.value, "sm_mhz": mhz.value,
            "per_clk_per_sm": per.value}
