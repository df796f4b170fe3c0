// pm_search: one scan launch per pattern, then the ordering kernels.
//
// Per call, the host builds one descriptor per (pattern, k) pair, packs the
// patterns' chunk masks into one arena (a pattern handle that appears more
// than once is packed once), and uploads arena and per-pattern tile offsets
// through a small ring of pinned host buffers so that the upload is a true
// asynchronous copy.  Scratch comes from the current device's stream-ordered
// pool (cudaMallocAsync) and goes back to it on the same stream.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr int kRing = 4;
constexpr int kMaxDevices = 64;

struct PinnedSlot {
    void *ptr = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
};

std::mutex g_ring_mu;
PinnedSlot g_ring[kMaxDevices][kRing];
int g_ring_next[kMaxDevices];

// A pinned host buffer of at least `bytes`, free of earlier copies.  The
// caller must call release_pinned() after queueing its copy from it.
pm_status acquire_pinned(int dev, size_t bytes, PinnedSlot **out)
{
    std::lock_guard<std::mutex> lk(g_ring_mu);
    PinnedSlot &s = g_ring[dev][g_ring_next[dev]++ % kRing];
    if (s.pending) {
        cudaEventSynchronize(s.done);
        s.pending = false;
    }
    if (!s.done) {
        pm_status rc = cuda_status(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming),
                                   "cudaEventCreate");
        if (rc) return rc;
    }
    if (s.cap < bytes) {
        if (s.ptr) cudaFreeHost(s.ptr);
        s.ptr = nullptr;
        s.cap = 0;
        const size_t want = std::max<size_t>(bytes + bytes / 2, 1 << 16);
        pm_status rc = cuda_status(cudaHostAlloc(&s.ptr, want, cudaHostAllocPortable), "cudaHostAlloc");
        if (rc) return rc;
        s.cap = want;
    }
    *out = &s;
    return PM_OK;
}

void release_pinned(PinnedSlot *s, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_ring_mu);
    if (cudaEventRecord(s->done, st) == cudaSuccess) s->pending = true;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Reads the total (and, for host outputs, the results) back when the caller
// asked for them; shared tail of both search paths.
pm_status finish_search(uint32_t npat, pm_hit *hits, uint64_t capacity, uint64_t *offsets,
                        uint64_t *needed, bool dev_out, const pm_hit *d_hits,
                        const uint64_t *d_offsets, void *const *scratch, int nscratch,
                        pm_status rc, cudaStream_t st)
{
    uint64_t total = 0;
    bool waited = false;
    if (!rc && !dev_out) {
        rc = cuda_status(cudaMemcpyAsync(offsets, d_offsets, (npat + 1) * sizeof(uint64_t),
                                         cudaMemcpyDeviceToHost, st),
                         "copy offsets");
        if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "stream synchronize");
        waited = true;
        total = offsets[npat];
        if (!rc && total != PM_TOTAL_ERROR && total <= capacity && total > 0) {
            rc = cuda_status(cudaMemcpyAsync(hits, d_hits, total * sizeof(pm_hit),
                                             cudaMemcpyDeviceToHost, st),
                             "copy hits");
        }
    } else if (!rc && needed) {
        rc = cuda_status(cudaMemcpyAsync(&total, d_offsets + npat, sizeof total,
                                         cudaMemcpyDeviceToHost, st),
                         "copy total");
        waited = true;
    }
    for (int i = 0; i < nscratch; ++i)
        if (scratch[i]) cudaFreeAsync(scratch[i], st);
    if (waited) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (!rc) rc = cuda_status(e, "stream synchronize");
    }
    if (rc) return rc;
    if (waited) {
        if (total == PM_TOTAL_ERROR) {
            set_error("pm_search: a device wait timed out");
            return PM_E_TIMEOUT;
        }
        if (needed) *needed = total;
        if (total > capacity) {
            set_error("pm_search: %llu hits, capacity %llu", (unsigned long long)total,
                      (unsigned long long)capacity);
            return PM_E_OVERFLOW;
        }
    }
    return PM_OK;
}

// pm_search_ex with options->batch: one persistent launch for all pairs.
pm_status search_ex_batched(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                            const int32_t *k, pm_hit *hits, uint64_t capacity, uint64_t *offsets,
                            uint64_t *needed, bool dev_out, const pm_options &o, cudaStream_t st)
{
    if (o.events) {
        set_error("pm_search: per-pattern events need one launch per pattern (options->batch is set)");
        return PM_E_ARG;
    }
    void *scratch[2] = {nullptr, nullptr};
    pm_hit *d_hits = hits;
    uint64_t *d_offsets = offsets;
    pm_status rc = PM_OK;
    if (!dev_out) {  // host outputs: device buffers first
        const size_t hb = align256((capacity ? capacity : 1) * sizeof(pm_hit));
        rc = cuda_status(cudaMallocAsync(&scratch[1], hb + (npat + 1) * sizeof(uint64_t), st),
                         "cudaMallocAsync outputs");
        if (rc) return rc;
        d_hits = (pm_hit *)scratch[1];
        d_offsets = (uint64_t *)((char *)scratch[1] + hb);
    }
    rc = search_batched(text, patterns, npat, k, capacity, o.batch, d_hits, d_offsets, &scratch[0], st);
    return finish_search(npat, hits, capacity, offsets, needed, dev_out, d_hits, d_offsets, scratch, 2,
                         rc, st);
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_search_ex(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                       const int32_t *k, pm_hit *hits, uint64_t capacity, uint64_t *offsets,
                       uint64_t *needed, const pm_options *opts, void *stream)
{
    TraceRange trace("pm_search");
    if (!text || !offsets || (npat > 0 && (!patterns || !k)) || (capacity > 0 && !hits)) {
        set_error("pm_search: NULL argument");
        return PM_E_ARG;
    }
    if (npat > PM_MAX_BATCH) {
        set_error("pm_search: npat = %u exceeds %u", npat, PM_MAX_BATCH);
        return PM_E_TOO_LARGE;
    }
    for (uint32_t p = 0; p < npat; ++p) {
        if (!patterns[p] || k[p] < 0) {
            set_error("pm_search: pattern %u is NULL or has k < 0", p);
            return PM_E_ARG;
        }
    }
    const pm_options o = opts ? *opts : pm_options{};
    if (o.variant < PM_VARIANT_AUTO || o.variant > PM_VARIANT_ALL_CHUNKS) {
        set_error("pm_search: unknown variant %d", o.variant);
        return PM_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != text->device) {
        set_error("pm_search: text lives on device %d, current device is %d", text->device, dev);
        return PM_E_ARG;
    }
    const bool dev_out = is_device_pointer(offsets);
    if (capacity > 0 && is_device_pointer(hits) != dev_out) {
        set_error("pm_search: hits and offsets must both be host or both be device memory");
        return PM_E_ARG;
    }

    if (capacity > kMaxCapacity) {
        set_error("pm_search: capacity %llu exceeds %llu", (unsigned long long)capacity,
                  (unsigned long long)kMaxCapacity);
        return PM_E_TOO_LARGE;
    }

    if (o.batch && npat > 0) return search_ex_batched(text, patterns, npat, k, hits, capacity, offsets,
                                                     needed, dev_out, o, st);

    // ---- descriptors and the arena (chunk masks, window-sliced lists) ----
    std::vector<PatDesc> desc(npat);
    std::vector<Variant> var(npat);
    struct Placed { uint64_t masks, list; };
    std::unordered_map<const pm_pattern *, Placed> where;
    uint64_t nmask = 0, entries = 0;
    for (uint32_t p = 0; p < npat; ++p) {
        const pm_pattern *pt = patterns[p];
        auto it = where.find(pt);
        if (it == where.end()) {
            Placed pl{nmask, nmask + pt->nchunks};
            it = where.emplace(pt, pl).first;
            nmask += pt->nchunks + wslist_units(pt);
        }
        PatDesc &d = desc[p];
        d.m = pt->m;
        d.nchunks = pt->nchunks;
        d.k = k[p];
        d.n_single = pt->n_single;
        d.n_general = pt->n_general;
        desc_constants(d);
        d.masks = it->second.masks;
        d.wslist = it->second.list;
        d.nwin = pt->m <= text->n ? text->n - pt->m + 1 : 0;
        const Variant v = o.variant == PM_VARIANT_AUTO ? auto_variant(d, dev)
                                                       : resolve_variant(variant_from_public(o.variant), d.k);
        var[p] = v;
        if (v == Variant::kPatternSliced || v == Variant::kPatternSliced2)
            d.c0 = first_stage_chunk(pt, text, v == Variant::kPatternSliced2 ? 2 : 1);
        const uint64_t tw = scan_tile_windows(v, d.k);
        d.tile0 = entries;
        d.ntiles = (d.nwin + tw - 1) / tw;
        entries += d.ntiles;
    }

    // ---- scratch layout ----
    const size_t sz_masks = align256(nmask * sizeof(uint4));
    const size_t sz_tile0 = align256((npat + 1) * sizeof(uint64_t));
    const size_t sz_table = align256(entries * sizeof(TileEntry));
    const size_t sz_tmp = align256(capacity * sizeof(pm_hit));
    const size_t sz_ctl = 256;  // cursor + status
    const size_t sz_order = align256(order_scratch_bytes(entries));
    const size_t sz_out = dev_out ? 0 : align256(capacity * sizeof(pm_hit)) +
                                            align256((npat + 1) * sizeof(uint64_t));
    const size_t total_bytes = sz_masks + sz_tile0 + sz_table + sz_tmp + sz_ctl + sz_order + sz_out;

    char *scratch = nullptr;
    pm_status rc = cuda_status(cudaMallocAsync((void **)&scratch, total_bytes, st), "cudaMallocAsync scratch");
    if (rc) return rc;
    char *cur = scratch;
    auto take = [&](size_t b) { char *r = cur; cur += b; return r; };
    uint4 *d_masks = (uint4 *)take(sz_masks);
    uint64_t *d_tile0 = (uint64_t *)take(sz_tile0);
    TileEntry *d_table = (TileEntry *)take(sz_table);
    pm_hit *d_tmp = (pm_hit *)take(sz_tmp);
    char *ctl = take(sz_ctl);
    unsigned long long *d_cursor = (unsigned long long *)ctl;
    uint32_t *d_status = (uint32_t *)(ctl + 8);
    void *d_order = take(sz_order);
    pm_hit *d_hits = hits;
    uint64_t *d_offsets = offsets;
    if (!dev_out) {
        d_hits = (pm_hit *)take(align256(capacity * sizeof(pm_hit)));
        d_offsets = (uint64_t *)take(align256((npat + 1) * sizeof(uint64_t)));
    }

    // ---- upload masks and tile offsets through pinned memory ----
    const size_t up_bytes = nmask * sizeof(uint4) + (npat + 1) * sizeof(uint64_t);
    PinnedSlot *slot = nullptr;
    rc = acquire_pinned(dev, up_bytes, &slot);
    if (!rc) {
        char *h = (char *)slot->ptr;
        for (const auto &kv : where) {
            const pm_pattern *pt = kv.first;
            std::memcpy(h + kv.second.masks * sizeof(uint4), pt->masks, pt->nchunks * sizeof(uint4));
            uint32_t *wl = (uint32_t *)(h + kv.second.list * sizeof(uint4));
            std::memset(wl, 0, wslist_units(pt) * sizeof(uint4));
            ordered_wslist(pt, text, wl);
        }
        uint64_t *ht0 = (uint64_t *)(h + nmask * sizeof(uint4));
        for (uint32_t p = 0; p < npat; ++p) ht0[p] = desc[p].tile0;
        ht0[npat] = entries;
        rc = cuda_status(cudaMemcpyAsync(d_masks, h, nmask * sizeof(uint4), cudaMemcpyHostToDevice, st),
                         "upload masks");
        if (!rc)
            rc = cuda_status(cudaMemcpyAsync(d_tile0, ht0, (npat + 1) * sizeof(uint64_t),
                                             cudaMemcpyHostToDevice, st),
                             "upload tile offsets");
        release_pinned(slot, st);
    }
    if (!rc) rc = cuda_status(cudaMemsetAsync(ctl, 0, sz_ctl, st), "memset control words");

    // ---- one scan launch per pattern ----
    for (uint32_t p = 0; !rc && p < npat; ++p) {
        const Variant v = var[p];
        const int grid = o.grid > 0 ? o.grid : scan_grid_limit(v, desc[p].k, dev);
        if (o.events) cudaEventRecord((cudaEvent_t)o.events[2 * p], st);
        rc = cuda_status(launch_scan(v, text->planes, text->unk, desc[p], d_masks, d_table, d_tmp, capacity,
                                     d_cursor, d_status, grid, st),
                         "scan kernel");
        if (o.events) cudaEventRecord((cudaEvent_t)o.events[2 * p + 1], st);
    }
    if (!rc)
        rc = cuda_status(launch_order(d_table, entries, d_tile0, npat, d_tmp, d_hits, capacity,
                                      d_offsets, d_status, d_order, st),
                         "order kernels");

    void *const scr[1] = {scratch};
    return finish_search(npat, hits, capacity, offsets, needed, dev_out, d_hits, d_offsets, scr, 1, rc,
                         st);
}

pm_status pm_search(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                    const int32_t *k, pm_hit *hits, uint64_t capacity, uint64_t *offsets,
                    uint64_t *needed, void *stream)
{
    return pm_search_ex(text, patterns, npat, k, hits, capacity, offsets, needed, nullptr, stream);
}

}  // extern "C"
