// pm_search_noalloc: the search without any memory allocation.
//
// Some callers cannot allocate device memory during a search: applications
// whose device memory is fully carved up by their own allocator before the
// search starts, and real-time loops where an allocation (the allocator's
// locks, and the implicit synchronisation it may cause) is not allowed.
// pm_search takes its scratch from the stream-ordered pool and a pinned host
// ring, so it does not suit them.  (The call still issues copies, memsets
// and kernel launches, and waits for the stream when asked for the total,
// so it is not for code that may not call CUDA at all, such as a host
// callback.)  This entry point runs the same scan and
// ordering kernels, but every byte of scratch lives in one fixed array in
// device global memory that the library declares at file scope.  The array
// is part of the module: each GPU that loads libpm keeps it until the
// process exits.  Calls allocate nothing (no cudaMalloc, cudaMallocAsync,
// cudaHostAlloc or free).
//
// Because every call uses the same array, two calls whose work overlaps on
// the GPU (different streams, or different host threads) race and corrupt
// each other's results; serialise them, e.g. by issuing them on one stream.
#include <mutex>
#include <vector>

#include "pm_internal.cuh"

namespace pm {
namespace {

// Limits of this entry point (checked on every call).
constexpr uint32_t kNaMaxPatterns = 64;            // (pattern, k) pairs per call
constexpr uint64_t kNaMaxChunks = 4096;            // sum of ceil(m/32) over distinct patterns
constexpr uint64_t kNaMaxTiles = 1ull << 21;       // warp tiles (4096 or 8192 windows) over the pairs
constexpr uint64_t kNaMaxHits = 1ull << 22;        // capacity
// arena: chunk masks plus each distinct pattern's window-sliced list (<= 8 units)
constexpr uint64_t kNaMaxArena = kNaMaxChunks + 8ull * kNaMaxPatterns;

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffMasks = 0;
constexpr size_t kOffTile0 = kOffMasks + al256(kNaMaxArena * sizeof(uint4));
constexpr size_t kOffCtl = kOffTile0 + al256((kNaMaxPatterns + 1) * sizeof(uint64_t));
constexpr size_t kOffTable = kOffCtl + 256;
constexpr size_t kOffTmp = kOffTable + al256(kNaMaxTiles * sizeof(TileEntry));
constexpr size_t kOffOrder = kOffTmp + al256(kNaMaxHits * sizeof(pm_hit));
// order scratch: per-block partials (+1) and one destination per tile entry
constexpr size_t kOrderBytes = (kNaMaxTiles / 4096 + 2) * 8 + kNaMaxTiles * 8 + 256;
constexpr size_t kScratchBytes = kOffOrder + al256(kOrderBytes);

// The scratch array (about 64 MiB).  Host code must not use its name as an
// address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_mu;
void *g_addr[kMaxDev];

// Once per device, with that device current: look up the array's address.
// The address is kept for the life of the process; after cudaDeviceReset of
// a device it no longer holds, so this entry point is not for processes that
// reset a device and search on it again.
pm_status scratch_address(int dev, char **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e != cudaSuccess ? e : cudaErrorUnknown,
                                                        "cudaGetSymbolAddress(scratch)");
        g_addr[dev] = p;
    }
    *out = (char *)g_addr[dev];
    return PM_OK;
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_search_noalloc(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                            const int32_t *k, pm_hit *hits, uint64_t capacity, uint64_t *offsets,
                            uint64_t *needed, void *stream)
{
    TraceRange trace("pm_search_noalloc");
    if (!text || !offsets || (npat > 0 && (!patterns || !k)) || (capacity > 0 && !hits)) {
        set_error("pm_search_noalloc: NULL argument");
        return PM_E_ARG;
    }
    if (npat > kNaMaxPatterns) {
        set_error("pm_search_noalloc: npat = %u exceeds this entry point's limit of %u", npat,
                  kNaMaxPatterns);
        return PM_E_TOO_LARGE;
    }
    if (capacity > kNaMaxHits) {
        set_error("pm_search_noalloc: capacity %llu exceeds this entry point's limit of %llu hits",
                  (unsigned long long)capacity, (unsigned long long)kNaMaxHits);
        return PM_E_TOO_LARGE;
    }
    for (uint32_t p = 0; p < npat; ++p) {
        if (!patterns[p] || k[p] < 0) {
            set_error("pm_search_noalloc: pattern %u is NULL or has k < 0", p);
            return PM_E_ARG;
        }
    }
    int dev = 0;
    pm_status rc0 = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc0) return rc0;
    if (dev < 0 || dev >= kMaxDev) {
        set_error("pm_search_noalloc: device %d is beyond this entry point's %d devices", dev, kMaxDev);
        return PM_E_ARG;
    }
    if (dev != text->device) {
        set_error("pm_search_noalloc: text lives on device %d, current device is %d", text->device,
                  dev);
        return PM_E_ARG;
    }
    if (!is_device_pointer(offsets) || (capacity > 0 && !is_device_pointer(hits))) {
        set_error("pm_search_noalloc: hits and offsets must be device memory");
        return PM_E_ARG;
    }

    // descriptors; a handle repeated with several k is packed once
    PatDesc desc[kNaMaxPatterns];
    Variant var[kNaMaxPatterns];
    uint64_t tile0[kNaMaxPatterns + 1];
    const pm_pattern *distinct[kNaMaxPatterns];
    uint64_t where[kNaMaxPatterns];
    uint32_t ndistinct = 0;
    uint64_t nmask = 0, entries = 0;
    for (uint32_t p = 0; p < npat; ++p) {
        const pm_pattern *pt = patterns[p];
        uint64_t mo = ~0ull;
        for (uint32_t q = 0; q < ndistinct; ++q)
            if (distinct[q] == pt) mo = where[q];
        if (mo == ~0ull) {
            mo = nmask;
            distinct[ndistinct] = pt;
            where[ndistinct++] = mo;
            nmask += pt->nchunks + wslist_units(pt);
        }
        PatDesc &d = desc[p];
        d.m = pt->m;
        d.nchunks = pt->nchunks;
        d.k = k[p];
        d.n_single = pt->n_single;
        d.n_general = pt->n_general;
        desc_constants(d);
        d.masks = mo;
        d.wslist = mo + pt->nchunks;
        d.nwin = pt->m <= text->n ? text->n - pt->m + 1 : 0;
        const Variant v = auto_variant(d, dev);
        var[p] = v;
        if (v == Variant::kPatternSliced || v == Variant::kPatternSliced2)
            d.c0 = first_stage_chunk(pt, text, v == Variant::kPatternSliced2 ? 2 : 1);
        const uint64_t tw = scan_tile_windows(v, d.k);
        d.tile0 = entries;
        d.ntiles = (d.nwin + tw - 1) / tw;
        entries += d.ntiles;
        tile0[p] = d.tile0;
    }
    tile0[npat] = entries;
    uint64_t chunks = 0;
    for (uint32_t q = 0; q < ndistinct; ++q) chunks += distinct[q]->nchunks;
    if (chunks > kNaMaxChunks || entries > kNaMaxTiles) {
        set_error("pm_search_noalloc: %llu pattern chunks (limit %llu) and %llu tiles (limit %llu)",
                  (unsigned long long)chunks, (unsigned long long)kNaMaxChunks,
                  (unsigned long long)entries, (unsigned long long)kNaMaxTiles);
        return PM_E_TOO_LARGE;
    }

    char *base = nullptr;
    pm_status rc = scratch_address(dev, &base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    uint4 *d_masks = (uint4 *)(base + kOffMasks);
    uint64_t *d_tile0 = (uint64_t *)(base + kOffTile0);
    char *ctl = base + kOffCtl;
    unsigned long long *d_cursor = (unsigned long long *)ctl;
    uint32_t *d_status = (uint32_t *)(ctl + 8);
    TileEntry *d_table = (TileEntry *)(base + kOffTable);
    pm_hit *d_tmp = (pm_hit *)(base + kOffTmp);
    void *d_order = base + kOffOrder;

    // Copies from pageable host memory are staged by the driver: the source
    // may be reused as soon as each call returns.
    for (uint32_t q = 0; !rc && q < ndistinct; ++q) {
        const pm_pattern *pt = distinct[q];
        rc = cuda_status(cudaMemcpyAsync(d_masks + where[q], pt->masks, pt->nchunks * sizeof(uint4),
                                         cudaMemcpyHostToDevice, st),
                         "upload masks");
        const uint64_t nl = wslist_units(pt);
        uint4 list[8] = {};  // one word per position of the first 32
        ordered_wslist(pt, text, (uint32_t *)list);
        if (!rc && nl)
            rc = cuda_status(cudaMemcpyAsync(d_masks + where[q] + pt->nchunks, list,
                                             nl * sizeof(uint4), cudaMemcpyHostToDevice, st),
                             "upload lists");
    }
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(d_tile0, tile0, (npat + 1) * sizeof(uint64_t),
                                         cudaMemcpyHostToDevice, st),
                         "upload tile offsets");
    // the array keeps the previous call's contents: the hit cursor and the
    // status word must start at zero (the tile table is rewritten in full)
    if (!rc) rc = cuda_status(cudaMemsetAsync(ctl, 0, 256, st), "clear control words");
    for (uint32_t p = 0; !rc && p < npat; ++p) {
        const Variant v = var[p];
        rc = cuda_status(launch_scan(v, text->planes, text->unk, desc[p], d_masks, d_table, d_tmp, capacity,
                                     d_cursor, d_status, scan_grid_limit(v, desc[p].k, dev), st),
                         "scan kernel");
    }
    if (!rc)
        rc = cuda_status(launch_order(d_table, entries, d_tile0, npat, d_tmp, hits, capacity, offsets,
                                      d_status, d_order, st),
                         "order kernels");
    if (rc || !needed) return rc;
    uint64_t total = 0;
    rc = cuda_status(cudaMemcpyAsync(&total, offsets + npat, sizeof total, cudaMemcpyDeviceToHost, st),
                     "copy total");
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "stream synchronize");
    if (rc) return rc;
    if (total == PM_TOTAL_ERROR) {
        set_error("pm_search_noalloc: a device wait timed out");
        return PM_E_TIMEOUT;
    }
    *needed = total;
    if (total > capacity) {
        set_error("pm_search_noalloc: %llu hits, capacity %llu", (unsigned long long)total,
                  (unsigned long long)capacity);
        return PM_E_OVERFLOW;
    }
    return PM_OK;
}

}  // extern "C"
