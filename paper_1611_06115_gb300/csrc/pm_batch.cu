// Batched search: many patterns of uneven m and k in one persistent launch
// over the resident text.
//
// pm_batch_create sorts the (pattern, k) pairs into groups of up to kP pairs
// of one kind: groups whose k is small (window-sliced evaluation, see
// pm_scan.cu) and groups evaluated pattern-sliced.  Work items are (text
// tile, group), tile-major, so that the warps running at any moment share a
// few tiles in L2 and the text is read from device memory about once for
// the whole batch.  A warp takes an item and stages the tile (plus halo) in
// shared memory with one bulk copy, then
//   * pattern-sliced group: for each window, the two funnel shifts that line
//     the text up with positions 0..31 are done once and serve every pattern
//     of the group (whose chunk-0 masks sit in shared memory), so a
//     pattern-window costs three selects, one popcount and a quarter of the
//     byte-packed threshold test;
//   * window-sliced group: each pattern runs the thermometer-counter scan
//     over the tile, reading its position list through the read-only path.
// Every 1024-window group of a tile with hits for a pattern writes them
// contiguously, in window order, through a warp-aggregated atomic and
// appends one segment record; records are radix-sorted by (pattern, tile,
// group) (pm_sort.cu) and the ordering pass (pm_order.cu) lays the hits out
// as per-pattern CSR lists sorted by location.
//
// pm_batch_create allocates everything once; pm_batch_run allocates nothing
// and never waits on the host, so it can be captured in a CUDA graph and
// replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "pm_scan_impl.cuh"

namespace pm {
namespace {
constexpr int kP = 8;  // pairs per group
// group kinds
constexpr uint32_t kKindShort = 0;  // pattern-sliced, k <= 31, shared shifts
constexpr uint32_t kKindWs = 1;     // window-sliced
constexpr uint32_t kKindLong = 2;   // pattern-sliced over all chunks, k > 31
}
}  // namespace pm

struct pm_batch {
    int device;
    uint32_t npat;
    uint32_t ngroups;
    uint32_t nphases;  // one per category of groups
    int ws_max;        // largest k evaluated window-sliced (-1: none)
    int grid;
    int key_bits;
    uint64_t ntiles;
    uint64_t capacity;
    const uint2 *planes;  // the text's planes (not owned)
    void *mem;            // one device allocation holding everything below
    pm::PatDesc *pats;
    uint32_t *order;      // pair indices, grouped
    uint32_t *gkind;      // per group: kind and number of pairs
    uint2 *phases;        // per phase: [first group, end group)
    uint4 *arena;
    pm_hit *tmp;
    pm::SegRecord *recs;
    void *sort_scratch;
    pm::TileEntry *entries;
    void *order_scratch;
    unsigned long long *ctl;  // [0] hit cursor, [1] record cursor, [2] status
    unsigned long long *pat_counts;
};

namespace pm {
namespace {

using namespace scan;

struct BatchArgs {
    const uint2 *planes;
    const PatDesc *pats;
    const uint32_t *order;
    const uint32_t *gkind;
    const uint2 *phases;    // [first group, end group) of each phase
    const uint4 *arena;
    uint32_t npat, ngroups;
    uint64_t ntiles, items;  // items = phases * ntiles, phase-major
    pm_hit *tmp;
    uint64_t cap;
    unsigned long long *cursor;
    SegRecord *recs;
    uint64_t rec_cap;
    unsigned long long *rec_cursor;
    unsigned long long *pat_counts;
    uint32_t *status;
};

// Emit the hits of one 1024-window group (pass bits of every lane) in window
// order through one warp-aggregated atomic, and append its segment record.
__device__ __forceinline__ void emit_group(uint32_t pass, uint64_t blk, uint32_t p, uint64_t key,
                                           uint32_t nchunks, uint32_t k,
                                           const uint4 *__restrict__ M, const BatchArgs &ba)
{
    const int lane = threadIdx.x & 31;
    const uint32_t nh = __popc(pass);
    uint32_t incl = nh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    unsigned long long base = 0;
    if (lane == 0) {
        base = atomicAdd(ba.cursor, (unsigned long long)total);
        atomicAdd(ba.pat_counts + p, (unsigned long long)total);
        const unsigned long long r = atomicAdd(ba.rec_cursor, 1ull);
        if (r < ba.rec_cap) ba.recs[r] = SegRecord{key, (uint32_t)base, total};
    }
    base = __shfl_sync(kFull, base, 0);
    unsigned long long q = base + incl - nh;
    uint32_t hm = pass;
    while (hm) {
        const uint32_t w = __ffs(hm) - 1;
        hm &= hm - 1;
        if (q < ba.cap) {
            const uint32_t c = window_count_from(ba.planes, blk, w, M, 0, nchunks, 0u, k);
            ba.tmp[q] = pm_hit{(uint32_t)(blk * 32ull + w), c};
        }
        ++q;
    }
}

// WSMAX: the largest k of the batch's window-sliced pairs (0..6).
template <int WSMAX>
__global__ void __launch_bounds__(kScanThreads, 3) k_scan_batched(const BatchArgs ba)
{
    __shared__ __align__(128) uint2 sbuf[kScanWarps][2][kStageBlocks];
    __shared__ __align__(8) uint64_t sbar[kScanWarps][2];
    __shared__ uint4 sM0[kScanWarps][kP];
    __shared__ uint4 sP[kScanWarps][kP];  // pattern-sliced group: {pair, k, k in every byte, 0}

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        dev::mbar_init(&sbar[warp][0], 1);
        dev::mbar_init(&sbar[warp][1], 1);
        dev::fence_mbar_init();
    }
    __syncwarp();

    const uint64_t stride = (uint64_t)gridDim.x * kScanWarps;
    const uint64_t first = (uint64_t)blockIdx.x * kScanWarps + warp;
    if (lane == 0) {
        if (first < ba.items)
            issue_tile(ba.planes, first % ba.ntiles, &sbuf[warp][0][0], &sbar[warp][0]);
        if (first + stride < ba.items)
            issue_tile(ba.planes, (first + stride) % ba.ntiles, &sbuf[warp][1][0], &sbar[warp][1]);
    }

    uint32_t it = 0;
    for (uint64_t item = first; item < ba.items; item += stride, ++it) {
        const int s = it & 1;
        const bool ok = dev::mbar_wait_bounded(&sbar[warp][s], (it >> 1) & 1u, kWaitLimitNs);
        if (__any_sync(kFull, !ok)) {
            if (lane == 0) {
                atomicOr(ba.status, kDevTimeout);
                dev::mbar_wait_bounded(&sbar[warp][s], (it >> 1) & 1u, kWaitLimitNs);
                if (item + stride < ba.items)
                    dev::mbar_wait_bounded(&sbar[warp][s ^ 1], ((it + 1) >> 1) & 1u, kWaitLimitNs);
            }
            return;
        }
        // items run phase-major: all warps work on one kind of group at a time
        const uint64_t tile = item % ba.ntiles;
        const uint2 ph = __ldg(ba.phases + item / ba.ntiles);
        const uint32_t g_begin = ph.x, g_end = ph.y;
        uint2 a[G], b[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            a[g] = sbuf[warp][s][32 * g + lane];
            b[g] = sbuf[warp][s][32 * g + lane + 1];
        }
        __syncwarp();
        if (lane == 0 && item + 2 * stride < ba.items) {
            dev::fence_proxy_async_smem();
            issue_tile(ba.planes, (item + 2 * stride) % ba.ntiles, &sbuf[warp][s][0], &sbar[warp][s]);
        }
        for (uint32_t grp = g_begin; grp < g_end; ++grp) {
        const uint32_t pfirst = grp * kP;
        const uint32_t gk = __ldg(ba.gkind + grp);
        const uint32_t kind = gk & 3u, cnt = gk >> 2;

        if (kind == kKindLong) {
            // ---- k > 31: every chunk counted, one pattern at a time ----
            for (uint32_t i = 0; i < cnt; ++i) {
                const uint32_t p = __ldg(ba.order + pfirst + i);
                const PatDesc d = ba.pats[p];
                const uint4 *M = ba.arena + d.masks;
#pragma unroll 1
                for (int g = 0; g < G; ++g) {
                    const uint64_t blk = tile * (32ull * G) + 32ull * g + (uint64_t)lane;
                    const uint32_t valid = valid_mask(blk, d.nwin);
                    const uint32_t pass = pass_multi_chunk(ba.planes, blk, M, d.nchunks, (uint32_t)d.k,
                                                           valid, a[g], b[g]);
                    if (__any_sync(kFull, pass != 0u))
                        emit_group(pass, blk, p, ((unsigned long long)p * ba.ntiles + tile) * G + g,
                                   d.nchunks, (uint32_t)d.k, M, ba);
                }
            }
        } else if (kind == kKindShort) {
            // ---- pattern-sliced group: shared shifts, masks from shared memory ----
            // Bytes hold 4 * (matches + k): bit 7 of a byte is set exactly when
            // matches + k >= 32, i.e. the window has at most k mismatches.
            const uint32_t two = ba.pats[ba.order[pfirst]].two;
            const uint32_t m1 = two << 1, m8 = m1 << 8, m16 = m1 << 16, m24 = m1 << 24;
            if (lane < (int)cnt) {
                const uint32_t pi = __ldg(ba.order + pfirst + lane);
                const PatDesc &dl = ba.pats[pi];
                const uint32_t kl = (uint32_t)dl.k;
                sM0[warp][lane] = __ldg(ba.arena + dl.masks);
                sP[warp][lane] = make_uint4(pi, kl, (kl < 32u ? kl : 0u) * (m24 | m16 | m8 | m1), 0u);
            }
            __syncwarp();
#pragma unroll 1
            for (int g = 0; g < G; ++g) {
                const uint64_t blk = tile * (32ull * G) + 32ull * g + (uint64_t)lane;
                uint32_t acc[kP];
#pragma unroll
                for (int p = 0; p < kP; ++p) acc[p] = 0u;
#pragma unroll
                for (uint32_t j = 0; j < 8; ++j) {
                    uint32_t lo[4], hi[4];
#pragma unroll
                    for (uint32_t q = 0; q < 4; ++q) {
                        lo[q] = __funnelshift_r(a[g].x, b[g].x, 4 * j + q);
                        hi[q] = __funnelshift_r(a[g].y, b[g].y, 4 * j + q);
                    }
#pragma unroll
                    for (int p = 0; p < kP; ++p) {
                        if (p < (int)cnt) {
                            const uint4 M0 = sM0[warp][p];
                            uint32_t gm[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) gm[q] = __popc(class_match(lo[q], hi[q], M0));
                            uint32_t v = mad_lo(gm[3], m24, sP[warp][p].z);
                            v = mad_lo(gm[2], m16, v);
                            v = mad_lo(gm[1], m8, v);
                            v = mad_lo(gm[0], m1, v);
                            // window 4j + q goes to bit 8q + j
                            acc[p] |= (v >> (7 - j)) & (0x01010101u << j);
                        }
                    }
                }
#pragma unroll
                for (int p = 0; p < kP; ++p) {
                    if (p < (int)cnt) {
                        const uint32_t pi = sP[warp][p].x, kp = sP[warp][p].y;
                        const PatDesc &d = ba.pats[pi];
                        const uint32_t valid = valid_mask(blk, d.nwin);
                        const uint4 *M = ba.arena + d.masks;
                        uint32_t pass = acc[p] ? untranspose(acc[p]) & valid : 0u;
                        if (d.nchunks > 1) pass = settle_lane(pass, blk, M, d.nchunks, kp, ba.planes);
                        if (__any_sync(kFull, pass != 0u))
                            emit_group(pass, blk, pi, ((unsigned long long)pi * ba.ntiles + tile) * G + g,
                                       d.nchunks, kp, M, ba);
                    }
                }
            }
        } else {
            // ---- window-sliced group: one pattern at a time over all groups ----
            for (uint32_t i = 0; i < cnt; ++i) {
                const uint32_t p = __ldg(ba.order + pfirst + i);
                const PatDesc d = ba.pats[p];
                uint64_t blk[G];
                uint32_t valid[G], pass[G];
                uint32_t anyv = 0;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    blk[g] = tile * (32ull * G) + 32ull * g + (uint64_t)lane;
                    valid[g] = valid_mask(blk[g], d.nwin);
                    anyv |= valid[g];
                }
                if (!__any_sync(kFull, anyv != 0u)) continue;
                const uint4 *list = ba.arena + d.wslist;
                // only the thresholds this batch uses are compiled in (instruction cache)
                if (d.k == 0) alive_window_sliced<0, true>(a, b, list, d.n_single, d.n_general, valid, pass);
                else if (WSMAX >= 1 && d.k == 1) alive_window_sliced<(WSMAX >= 1 ? 1 : 0), true>(a, b, list, d.n_single, d.n_general, valid, pass);
                else if (WSMAX >= 2 && d.k == 2) alive_window_sliced<(WSMAX >= 2 ? 2 : 0), true>(a, b, list, d.n_single, d.n_general, valid, pass);
                else if (WSMAX >= 3 && d.k == 3) alive_window_sliced<(WSMAX >= 3 ? 3 : 0), true>(a, b, list, d.n_single, d.n_general, valid, pass);
                else if (WSMAX >= 4 && d.k == 4) alive_window_sliced<(WSMAX >= 4 ? 4 : 0), true>(a, b, list, d.n_single, d.n_general, valid, pass);
                else if (WSMAX >= 5 && d.k == 5) alive_window_sliced<(WSMAX >= 5 ? 5 : 0), true>(a, b, list, d.n_single, d.n_general, valid, pass);
                else alive_window_sliced<(WSMAX >= 6 ? 6 : 0), true>(a, b, list, d.n_single, d.n_general, valid, pass);
                const uint4 *M = ba.arena + d.masks;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const uint32_t ps = d.nchunks > 1
                        ? settle_lane(pass[g], blk[g], M, d.nchunks, (uint32_t)d.k, ba.planes)
                        : pass[g];
                    if (__any_sync(kFull, ps != 0u))
                        emit_group(ps, blk[g], p, ((unsigned long long)p * ba.ntiles + tile) * G + g,
                                   d.nchunks, (uint32_t)d.k, M, ba);
                }
            }
        }
        }  // groups of the item
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

const void *batched_kernel(int ws_max)
{
    switch (ws_max < 0 ? 0 : ws_max) {
    case 0: return (const void *)&k_scan_batched<0>;
    case 1: return (const void *)&k_scan_batched<1>;
    case 2: return (const void *)&k_scan_batched<2>;
    case 3: return (const void *)&k_scan_batched<3>;
    case 4: return (const void *)&k_scan_batched<4>;
    case 5: return (const void *)&k_scan_batched<5>;
    default: return (const void *)&k_scan_batched<6>;
    }
}

int batched_grid(int device, int ws_max)
{
    static int cache[64][8] = {};
    if (device < 0 || device >= 64) return 0;
    const int slot = ws_max < 0 ? 0 : (ws_max > 6 ? 6 : ws_max);
    if (cache[device][slot]) return cache[device][slot];
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel(slot), kScanThreads, 0);
    cache[device][slot] = sms * (per_sm < 1 ? 1 : per_sm);
    return cache[device][slot];
}

}  // namespace
}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_batch_create(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                          const int32_t *k, uint64_t capacity, const pm_batch_options *opts,
                          void *stream, pm_batch **out)
{
    if (!text || !out || (npat > 0 && (!patterns || !k))) {
        set_error("pm_batch_create: NULL argument");
        return PM_E_ARG;
    }
    *out = nullptr;
    if (npat == 0 || npat > PM_MAX_BATCH || capacity > kMaxCapacity) {
        set_error("pm_batch_create: npat = %u (1..%u), capacity %llu (<= %llu)", npat, PM_MAX_BATCH,
                  (unsigned long long)capacity, (unsigned long long)kMaxCapacity);
        return npat == 0 ? PM_E_ARG : PM_E_TOO_LARGE;
    }
    for (uint32_t p = 0; p < npat; ++p) {
        if (!patterns[p] || k[p] < 0) {
            set_error("pm_batch_create: pattern %u is NULL or has k < 0", p);
            return PM_E_ARG;
        }
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != text->device) {
        set_error("pm_batch_create: text lives on device %d, current device is %d", text->device, dev);
        return PM_E_ARG;
    }
    const pm_batch_options o = opts ? *opts : pm_batch_options{};
    cudaStream_t st = (cudaStream_t)stream;
    // in a batch the pattern-sliced groups share their text shifts, which
    // makes them cheaper than window-sliced evaluation from k = 3 on
    const int ws_max = o.ws_max_k > 0 ? std::min(o.ws_max_k, kWsMaxK) : (o.ws_max_k < 0 ? -1 : 2);

    // descriptors and arena (host side first)
    std::vector<PatDesc> desc(npat);
    std::unordered_map<const pm_pattern *, std::pair<uint64_t, uint64_t>> where;
    std::vector<uint4> arena;
    uint32_t min_m = UINT32_MAX;
    for (uint32_t p = 0; p < npat; ++p) {
        const pm_pattern *pt = patterns[p];
        auto it = where.find(pt);
        if (it == where.end()) {
            const uint64_t mo = arena.size();
            arena.insert(arena.end(), pt->masks, pt->masks + pt->nchunks);
            const uint64_t lo = arena.size();
            arena.insert(arena.end(), pt->wslist, pt->wslist + pt->n_single + 2 * pt->n_general);
            it = where.emplace(pt, std::make_pair(mo, lo)).first;
        }
        PatDesc &d = desc[p];
        d.m = pt->m;
        d.nchunks = pt->nchunks;
        d.k = k[p];
        d.n_single = pt->n_single;
        d.n_general = pt->n_general;
        desc_constants(d);
        d.masks = it->second.first;
        d.wslist = it->second.second;
        d.nwin = pt->m <= text->n ? text->n - pt->m + 1 : 0;
        d.tile0 = 0;
        d.ntiles = (d.nwin + kTileWindows - 1) / kTileWindows;
        d.variant = (uint32_t)(d.k <= ws_max ? Variant::kWindowSliced : Variant::kPatternSliced);
        min_m = std::min(min_m, pt->m);
    }
    if (arena.empty()) arena.push_back(make_uint4(0, 0, 0, 0));

    // Categories, each one phase of the launch (all warps run one kind of
    // evaluation at a time): window-sliced pairs with k = 0, 1, ..., then
    // pattern-sliced pairs with k <= 31, then those with k > 31.  Within a
    // category pairs are ordered by m and cut into groups of kP.
    std::vector<std::vector<uint32_t>> cats(kWsMaxK + 3);
    for (uint32_t p = 0; p < npat; ++p) {
        const int32_t kp = desc[p].k;
        size_t c;
        if (desc[p].variant == (uint32_t)Variant::kWindowSliced) c = (size_t)kp;
        else c = kp <= 31 ? kWsMaxK + 1 : kWsMaxK + 2;
        cats[c].push_back(p);
    }
    std::vector<uint32_t> order, gkind;
    std::vector<uint2> phases;
    // gkind: bits 0-1 the kind, bits 2.. the number of real pairs (the last
    // group of a category is padded to kP slots; padding is never evaluated)
    for (size_t c = 0; c < cats.size(); ++c) {
        std::vector<uint32_t> &v = cats[c];
        if (v.empty()) continue;
        std::stable_sort(v.begin(), v.end(), [&](uint32_t x, uint32_t y) { return desc[x].m < desc[y].m; });
        const uint32_t kind = c <= (size_t)kWsMaxK ? kKindWs : (c == (size_t)kWsMaxK + 1 ? kKindShort : kKindLong);
        const uint32_t g0 = (uint32_t)gkind.size();
        for (size_t i = 0; i < v.size(); i += kP) {
            const uint32_t count = (uint32_t)std::min<size_t>(kP, v.size() - i);
            for (size_t j = i; j < i + kP; ++j) order.push_back(j < v.size() ? v[j] : v[i]);
            gkind.push_back(kind | (count << 2));
        }
        phases.push_back(make_uint2(g0, (uint32_t)gkind.size()));
    }
    const uint32_t ngroups = (uint32_t)gkind.size();

    pm_batch *b = new (std::nothrow) pm_batch{};
    if (!b) return PM_E_NOMEM;
    b->device = dev;
    b->npat = npat;
    b->ngroups = ngroups;
    b->ws_max = ws_max;
    b->grid = o.grid > 0 ? o.grid : batched_grid(dev, ws_max);
    b->ntiles = min_m <= text->n ? (text->n - min_m + 1 + kTileWindows - 1) / kTileWindows : 0;
    b->nphases = (uint32_t)phases.size();
    b->capacity = capacity;
    b->planes = text->planes;
    const unsigned long long max_key = (unsigned long long)npat * (b->ntiles ? b->ntiles : 1) * G;
    b->key_bits = 0;
    while (b->key_bits < 64 && (max_key >> b->key_bits) != 0) ++b->key_bits;

    const uint64_t cap_e = capacity ? capacity : 1;
    const size_t sz_pats = align256(npat * sizeof(PatDesc));
    const size_t sz_order = align256(order.size() * sizeof(uint32_t));
    const size_t sz_gkind = align256(gkind.size() * sizeof(uint32_t));
    const size_t sz_phases = align256(std::max<size_t>(phases.size(), 1) * sizeof(uint2));
    const size_t sz_arena = align256(arena.size() * sizeof(uint4));
    const size_t sz_tmp = align256(cap_e * sizeof(pm_hit));
    const size_t sz_recs = align256(cap_e * sizeof(SegRecord));
    const size_t sz_sort = align256(sort_scratch_bytes(cap_e));
    const size_t sz_entries = align256(cap_e * sizeof(TileEntry));
    const size_t sz_ordscr = align256(order_scratch_bytes(cap_e));
    const size_t sz_ctl = 256;
    const size_t sz_counts = align256(npat * sizeof(unsigned long long));
    const size_t total = sz_pats + sz_order + sz_gkind + sz_phases + sz_arena + sz_tmp + sz_recs +
                         sz_sort + sz_entries + sz_ordscr + sz_ctl + sz_counts;
    pm_status rc = cuda_status(cudaMalloc(&b->mem, total), "cudaMalloc batch");
    if (rc) {
        delete b;
        return rc;
    }
    char *c = (char *)b->mem;
    auto take = [&](size_t n) { char *r = c; c += n; return (void *)r; };
    b->pats = (PatDesc *)take(sz_pats);
    b->order = (uint32_t *)take(sz_order);
    b->gkind = (uint32_t *)take(sz_gkind);
    b->phases = (uint2 *)take(sz_phases);
    b->arena = (uint4 *)take(sz_arena);
    b->tmp = (pm_hit *)take(sz_tmp);
    b->recs = (SegRecord *)take(sz_recs);
    b->sort_scratch = take(sz_sort);
    b->entries = (TileEntry *)take(sz_entries);
    b->order_scratch = take(sz_ordscr);
    b->ctl = (unsigned long long *)take(sz_ctl);
    b->pat_counts = (unsigned long long *)take(sz_counts);
    rc = cuda_status(cudaMemcpyAsync(b->pats, desc.data(), npat * sizeof(PatDesc),
                                     cudaMemcpyHostToDevice, st), "upload descriptors");
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(b->order, order.data(), order.size() * sizeof(uint32_t),
                                         cudaMemcpyHostToDevice, st), "upload groups");
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(b->gkind, gkind.data(), gkind.size() * sizeof(uint32_t),
                                         cudaMemcpyHostToDevice, st), "upload group kinds");
    if (!rc && !phases.empty())
        rc = cuda_status(cudaMemcpyAsync(b->phases, phases.data(), phases.size() * sizeof(uint2),
                                         cudaMemcpyHostToDevice, st), "upload phases");
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(b->arena, arena.data(), arena.size() * sizeof(uint4),
                                         cudaMemcpyHostToDevice, st), "upload arena");
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "stream synchronize");
    if (rc) {
        cudaFree(b->mem);
        delete b;
        return rc;
    }
    *out = b;
    return PM_OK;
}

pm_status pm_batch_run(pm_batch *b, pm_hit *hits, uint64_t *offsets, void *stream)
{
    if (!b || !offsets || (b->capacity > 0 && !hits)) {
        set_error("pm_batch_run: NULL argument");
        return PM_E_ARG;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) {
        set_error("pm_batch_run: batch lives on device %d, current device is %d", b->device, dev);
        return PM_E_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *cursor = b->ctl, *rec_cursor = b->ctl + 1;
    uint32_t *status = (uint32_t *)(b->ctl + 2);
    pm_status rc = cuda_status(cudaMemsetAsync(b->ctl, 0, 256, st), "clear control words");
    if (!rc)
        rc = cuda_status(cudaMemsetAsync(b->pat_counts, 0, b->npat * sizeof(unsigned long long), st),
                         "clear counts");
    if (rc) return rc;
    const uint64_t items = b->ntiles * b->nphases;
    if (items > 0) {
        BatchArgs ba{b->planes, b->pats, b->order, b->gkind, b->phases, b->arena, b->npat,
                     b->ngroups, b->ntiles, items, b->tmp, b->capacity, cursor, b->recs,
                     b->capacity, rec_cursor, b->pat_counts, status};
        uint64_t grid = (items + kScanWarps - 1) / kScanWarps;
        if (grid > (uint64_t)b->grid) grid = (uint64_t)b->grid;
        void *args[] = {(void *)&ba};
        rc = cuda_status(cudaLaunchKernel(batched_kernel(b->ws_max), dim3((unsigned)grid),
                                          dim3(kScanThreads), args, 0, st),
                         "batched scan kernel");
    }
    SegRecord *sorted = b->recs;
    const uint64_t n_max = b->capacity;
    if (!rc)
        rc = cuda_status(launch_sort_records(b->recs, n_max, rec_cursor, b->key_bits, b->sort_scratch,
                                             st, &sorted),
                         "sort records");
    if (!rc)
        rc = cuda_status(launch_records_to_entries(sorted, n_max, rec_cursor, b->entries, st),
                         "record entries");
    if (!rc)
        rc = cuda_status(launch_order_records(b->entries, n_max, rec_cursor, b->pat_counts, b->npat,
                                              cursor, b->tmp, hits, b->capacity, offsets, status,
                                              b->order_scratch, st),
                         "order kernels");
    return rc;
}

uint64_t pm_batch_capacity(const pm_batch *b) { return b ? b->capacity : 0; }

void pm_batch_free(pm_batch *b)
{
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaFree(b->mem);
    if (cur != b->device) cudaSetDevice(cur);
    delete b;
}

}  // extern "C"
