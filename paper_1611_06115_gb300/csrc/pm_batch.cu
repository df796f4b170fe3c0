// Batched search: many patterns of uneven m and k in one persistent launch
// over the resident text.
//
// The planner sorts the (pattern, k) pairs into categories by evaluation
// (window-sliced per k, pattern-sliced over 32 positions, over 64 positions,
// every chunk; thresholds are options), orders each category by m and cuts
// it into groups of kP pairs and rows of groups.  A work item is a row
// crossed with a run of warp tiles; rows are outermost, so all warps run one
// kind of evaluation at a time and the text is read from device memory
// about once per row.  A warp stages its tiles (plus halo) in shared memory
// by bulk copies two tiles ahead, then per group of the row
//   * pattern-sliced group: for each window, the funnel shifts that line the
//     text up with the first 32 (or 64) positions are done once and serve
//     every pair of the group (whose masks sit in shared memory), so a
//     pair-window costs three (or six) selects, one (or two) popcounts and a
//     quarter of the byte-packed threshold test;
//   * window-sliced group: each pair runs the thermometer-counter scan over
//     the tile, reading its position list through the read-only path;
//   * every-chunk group: each pair keeps 32 running counts per lane.
// Every 1024-window group of a tile with hits for a pair writes them
// contiguously, in window order, through a warp-aggregated atomic and
// appends one segment record; records are radix-sorted by (pair, tile,
// group) (pm_sort.cu) and the ordering pass (pm_order.cu) lays the hits out
// as per-pair CSR lists sorted by location.
//
// pm_batch_create allocates everything once; pm_batch_run allocates nothing
// and never waits on the host, so it can be captured in a CUDA graph and
// replayed.  pm_search_ex with batch options runs the same plan with
// stream-ordered scratch.
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
constexpr uint32_t kKindShort = 0;   // pattern-sliced over positions 0..31, shared shifts (k <= 31)
constexpr uint32_t kKindWs = 1;      // window-sliced (k <= kWsMaxK)
constexpr uint32_t kKindLong = 2;    // pattern-sliced over all chunks (any k)
constexpr uint32_t kKindShort2 = 3;  // pattern-sliced over positions 0..63, shared shifts (k <= 63)
// Warp tiles per work item.  The last run of tiles of an item may reach past
// the text by up to this many tiles minus one; the text's zero padding must
// hold their copies (each tile copies 32*G + 2 blocks).
constexpr int kMaxTilesPerItem = 4;
static_assert((kMaxTilesPerItem + 1) * 32 * kGroups + 2 <= kPadBlocks,
              "the text padding covers the last run of tiles");
}
}  // namespace pm

struct pm_batch {
    int device;
    uint32_t npat;
    uint32_t ngroups;
    uint32_t nphases;  // work-item rows: pieces of the categories of groups
    int ws_max;        // largest k evaluated window-sliced (-1: none)
    int grid;
    int key_bits;
    uint32_t tiles;    // warp tiles per work item
    uint64_t ntiles;   // warp tiles of the longest window range
    uint64_t runs;     // runs of `tiles` tiles covering them
    uint64_t capacity;
    const uint2 *planes;  // the text's planes (not owned)
    const uint32_t *unk;  // the text's unknown-symbol bits or NULL (not owned)
    void *mem;            // one device allocation holding everything below
    pm::PatDesc *pats;
    uint32_t *order;      // pair indices, grouped
    uint32_t *gkind;      // per group: kind and number of pairs
    uint2 *phases;        // per row: [first group, end group)
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
    const uint32_t *unk;
    const PatDesc *pats;
    const uint32_t *order;
    const uint32_t *gkind;
    const uint2 *phases;    // [first group, end group) of each row
    const uint4 *arena;
    uint32_t npat, ngroups;
    uint32_t tiles;         // warp tiles per item
    uint64_t ntiles, runs;  // items = rows * runs, row-major
    uint64_t items;
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
    if (ba.unk) pass = recount_unknown(pass, ba.planes, ba.unk, blk, M, nchunks, k);
    const uint32_t nh = __popc(pass);
    uint32_t incl = nh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;  // every candidate dropped by the recount (warp-uniform)
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
            const uint32_t c = window_count_exact(ba.planes, ba.unk, blk, w, M, nchunks, k);
            ba.tmp[q] = pm_hit{(uint32_t)(blk * 32ull + w), c};
        }
        ++q;
    }
}

// A pattern-sliced group over the first C chunks (C = 1: k <= 31, C = 2:
// k <= 63): for each window the funnel shifts that line the text up with
// the chunks are done once and serve all kP pairs of the group, whose masks
// sit in shared memory.  Bytes of the multiply-add results hold
// (4/C) * (matches + k) <= (4/C) * (64C - 1) < 256, so bit 7 of a byte is set
// exactly when matches + k >= 32C, i.e. when the window has at most k
// mismatches in those positions.  Windows that pass and whose pattern is
// longer are then counted exactly (settle_staged).
// kAll: all kP slots hold pairs (every group but the last of a category);
// otherwise the empty slots are skipped.
template <int C, bool kAll>
__device__ __forceinline__ void short_group(const uint2 *stage, uint64_t tile, uint32_t pfirst,
                                            uint32_t cnt, uint4 *sM0, uint4 *sM1, uint4 *sP,
                                            const BatchArgs &ba)
{
    const int lane = threadIdx.x & 31;
    const uint32_t two = ba.pats[ba.order[pfirst]].two;
    const uint32_t m1 = C == 1 ? two << 1 : two, m8 = m1 << 8, m16 = m1 << 16, m24 = m1 << 24;
    if (lane < kP) {
        // slots past cnt repeat a real pair (never evaluated)
        const uint32_t pi = __ldg(ba.order + pfirst + lane);
        const PatDesc &dl = ba.pats[pi];
        const uint32_t kl = (uint32_t)dl.k;
        sM0[lane] = __ldg(ba.arena + dl.masks);
        if (C == 2)
            sM1[lane] = dl.nchunks > 1 ? __ldg(ba.arena + dl.masks + 1) : make_uint4(kFull, kFull, kFull, kFull);
        sP[lane] = make_uint4(pi, kl, kl * (m24 | m16 | m8 | m1), 0u);
    }
    __syncwarp();
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
        const uint64_t blk = tile * (32ull * G) + 32ull * g + (uint64_t)lane;
        const uint2 ta = stage[32 * g + lane], tb = stage[32 * g + lane + 1];
        const uint2 c = C == 2 ? stage[32 * g + lane + 2] : make_uint2(0u, 0u);
        uint32_t acc[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) acc[p] = 0u;
        // one step at a time: with the steps unrolled the kernel spills at
        // every WSMAX and is larger (instruction fetch was its largest
        // stall); one step at a time measured 1.7 % faster over 4096 pairs
#pragma unroll 1
        for (uint32_t j = 0; j < 8; ++j) {
            uint32_t lo[4], hi[4], lo1[4], hi1[4];
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q) {
                lo[q] = __funnelshift_r(ta.x, tb.x, 8 * q + j);
                hi[q] = __funnelshift_r(ta.y, tb.y, 8 * q + j);
                if (C == 2) {
                    lo1[q] = __funnelshift_r(tb.x, c.x, 8 * q + j);
                    hi1[q] = __funnelshift_r(tb.y, c.y, 8 * q + j);
                }
            }
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                if (!kAll && p >= (int)cnt) break;  // warp-uniform
                const uint4 M0 = sM0[p];
                uint32_t gm[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) gm[q] = __popc(class_match(lo[q], hi[q], M0));
                if (C == 2) {
                    const uint4 M1 = sM1[p];
#pragma unroll
                    for (int q = 0; q < 4; ++q) gm[q] += __popc(class_match(lo1[q], hi1[q], M1));
                }
                uint32_t v = mad_lo(gm[3], m24, sP[p].z);
                v = mad_lo(gm[2], m16, v);
                v = mad_lo(gm[1], m8, v);
                v = mad_lo(gm[0], m1, v);
                // window 8q + j: bit 7 of byte q goes to bit 8q + j
                acc[p] |= (v >> (7 - j)) & (0x01010101u << j);
            }
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            if (p < (int)cnt) {
                const uint32_t pi = sP[p].x, kp = sP[p].y;
                const PatDesc &d = ba.pats[pi];
                const uint32_t valid = valid_mask(blk, d.nwin);
                const uint4 *M = ba.arena + d.masks;
                uint32_t pass = acc[p] & valid;
                if (d.nchunks > (uint32_t)C)
                    pass = settle_staged(pass, blk, ta, tb, stage + 32 * g + lane + 2, M, 0u, d.nchunks,
                                         kp, ba.planes);
                if (__any_sync(kFull, pass != 0u))
                    emit_group(pass, blk, pi, ((unsigned long long)pi * ba.ntiles + tile) * G + g,
                               d.nchunks, kp, M, ba);
            }
        }
    }
    __syncwarp();  // the group's shared slots are rewritten by the next group
}

// WSMAX: the largest k of the batch's window-sliced pairs (0..6).
//
// Each warp walks its own sequence of staged tiles: position s of the
// sequence is tile s % T of work item first + (s / T) * stride, where an item
// is a run of T warp tiles crossed with a row of groups (items row-major:
// all warps work on one kind of group at a time).  The sequence is staged
// two positions ahead into a two-stage ring; a stage is refilled once the
// warp is done with its tile.
template <int WSMAX>
__global__ void __launch_bounds__(kScanThreads, 3) k_scan_batched(const BatchArgs ba)
{
    __shared__ __align__(128) uint2 sbuf[kScanWarps][2][kStageBlocks];
    __shared__ __align__(8) uint64_t sbar[kScanWarps][2];
    __shared__ uint4 sM0[kScanWarps][kP];
    __shared__ uint4 sM1[kScanWarps][kP];
    __shared__ uint4 sP[kScanWarps][kP];  // pattern-sliced group: {pair, k, k in every byte, 0}

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        dev::mbar_init(&sbar[warp][0], 1);
        dev::mbar_init(&sbar[warp][1], 1);
        dev::fence_mbar_init();
    }
    __syncwarp();

    // runs < 2^21 (a text has fewer than 2^32 symbols) and the grid is
    // resident, so 32-bit positions suffice
    const uint32_t stride = gridDim.x * kScanWarps;
    const uint32_t T = ba.tiles;
    const uint32_t runs = (uint32_t)ba.runs;
    const uint32_t nrows = (uint32_t)(ba.items / ba.runs);
    // Sequence positions as (row, run, tile within the run of T): work item
    // row * runs + run.  Moving on by `stride` items needs no division (this
    // runs once per tile; a 64-bit division would cost more than a cheap
    // tile's evaluation).
    struct Pos {
        uint32_t row, u, run;
    };
    auto advance = [&](Pos &q) {
        if (++q.u == T) {
            q.u = 0;
            q.run += stride;
            while (q.run >= runs && q.row < nrows) {
                q.run -= runs;
                ++q.row;
            }
        }
    };
    auto tile_of = [&](const Pos &q) { return (uint64_t)q.run * T + q.u; };
    const uint32_t first = blockIdx.x * kScanWarps + warp;
    Pos cp{first / runs, 0u, first % runs};  // consumed
    if (cp.row > nrows) cp.row = nrows;
    Pos pp = cp;                                                  // next to stage
#pragma unroll
    for (int st = 0; st < 2; ++st) {
        if (lane == 0 && pp.row < nrows) issue_tile(ba.planes, tile_of(pp), &sbuf[warp][st][0], &sbar[warp][st]);
        advance(pp);
    }

    for (uint64_t s = 0; cp.row < nrows; ++s, advance(cp)) {
        const int st = (int)(s & 1);
        const uint32_t par = (uint32_t)(s >> 1) & 1u;
        const uint64_t tile = tile_of(cp);
        const bool ok = dev::mbar_wait_bounded(&sbar[warp][st], par, kWaitLimitNs);
        if (__any_sync(kFull, !ok)) {
            if (lane == 0) {
                atomicOr(ba.status, kDevTimeout);
                // let the copies this warp still has in flight land before it leaves
                dev::mbar_wait_bounded(&sbar[warp][st], par, kWaitLimitNs);
                Pos nq = cp;
                advance(nq);
                if (nq.row < nrows)
                    dev::mbar_wait_bounded(&sbar[warp][st ^ 1], (uint32_t)((s + 1) >> 1) & 1u, kWaitLimitNs);
            }
            return;
        }
        const uint2 *stage = &sbuf[warp][st][0];
        const uint2 ph = __ldg(ba.phases + cp.row);
        const uint32_t kind0 = __ldg(ba.gkind + ph.x) & 3u;  // a row holds one kind
        if (kind0 == kKindWs) {
            // The window-sliced evaluation needs only the lane's two blocks per
            // group: take them into registers and refill the stage now, two
            // tiles ahead (its items are short; a refill after the item would
            // leave the next copy too little time to land).
            uint2 a[G], b[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                a[g] = stage[32 * g + lane];
                b[g] = stage[32 * g + lane + 1];
            }
            __syncwarp();
            if (lane == 0 && pp.row < nrows) {
                dev::fence_proxy_async_smem();
                issue_tile(ba.planes, tile_of(pp), &sbuf[warp][st][0], &sbar[warp][st]);
            }
            advance(pp);
            for (uint32_t grp = ph.x; grp < ph.y; ++grp) {
                const uint32_t pfirst = grp * kP;
                const uint32_t cnt = __ldg(ba.gkind + grp) >> 2;
                {
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
                        bool cut;
                        // only the thresholds this batch uses are compiled in (instruction cache)
                        if (d.k == 0) cut = alive_window_sliced<0, true>(a, b, list, d.n_single, d.n_general, ws_cut(0), valid, pass);
                        else if (WSMAX >= 1 && d.k == 1) cut = alive_window_sliced<(WSMAX >= 1 ? 1 : 0), true>(a, b, list, d.n_single, d.n_general, ws_cut((WSMAX >= 1 ? 1 : 0)), valid, pass);
                        else if (WSMAX >= 2 && d.k == 2) cut = alive_window_sliced<(WSMAX >= 2 ? 2 : 0), true>(a, b, list, d.n_single, d.n_general, ws_cut((WSMAX >= 2 ? 2 : 0)), valid, pass);
                        else if (WSMAX >= 3 && d.k == 3) cut = alive_window_sliced<(WSMAX >= 3 ? 3 : 0), true>(a, b, list, d.n_single, d.n_general, ws_cut((WSMAX >= 3 ? 3 : 0)), valid, pass);
                        else if (WSMAX >= 4 && d.k == 4) cut = alive_window_sliced<(WSMAX >= 4 ? 4 : 0), true>(a, b, list, d.n_single, d.n_general, ws_cut((WSMAX >= 4 ? 4 : 0)), valid, pass);
                        else if (WSMAX >= 5 && d.k == 5) cut = alive_window_sliced<(WSMAX >= 5 ? 5 : 0), true>(a, b, list, d.n_single, d.n_general, ws_cut((WSMAX >= 5 ? 5 : 0)), valid, pass);
                        else cut = alive_window_sliced<(WSMAX >= 6 ? 6 : 0), true>(a, b, list, d.n_single, d.n_general, ws_cut((WSMAX >= 6 ? 6 : 0)), valid, pass);
                        const uint4 *M = ba.arena + d.masks;
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            const uint32_t ps = (cut || d.nchunks > 1)
                                ? settle_from_regs(pass[g], blk[g], a[g], b[g], M, d.nchunks, (uint32_t)d.k,
                                                   ba.planes)
                                : pass[g];
                            if (__any_sync(kFull, ps != 0u))
                                emit_group(ps, blk[g], p, ((unsigned long long)p * ba.ntiles + tile) * G + g,
                                           d.nchunks, (uint32_t)d.k, M, ba);
                        }
                    }
                }
            }
        } else {
            // pattern-sliced groups read the staged tile while they settle the
            // windows that survive their first chunks (and the every-chunk
            // groups read it per group): refill after the item
            for (uint32_t grp = ph.x; grp < ph.y; ++grp) {
                const uint32_t pfirst = grp * kP;
                const uint32_t cnt = __ldg(ba.gkind + grp) >> 2;
                if (kind0 == kKindLong) {
                    // ---- every chunk counted, one pattern at a time ----
                    for (uint32_t i = 0; i < cnt; ++i) {
                        const uint32_t p = __ldg(ba.order + pfirst + i);
                        const PatDesc d = ba.pats[p];
                        const uint4 *M = ba.arena + d.masks;
#pragma unroll 1
                        for (int g = 0; g < G; ++g) {
                            const uint64_t blk = tile * (32ull * G) + 32ull * g + (uint64_t)lane;
                            const uint32_t valid = valid_mask(blk, d.nwin);
                            const uint32_t pass = pass_multi_chunk(ba.planes, blk, M, d.nchunks, (uint32_t)d.k,
                                                                   valid, stage[32 * g + lane],
                                                                   stage[32 * g + lane + 1]);
                            if (__any_sync(kFull, pass != 0u))
                                emit_group(pass, blk, p, ((unsigned long long)p * ba.ntiles + tile) * G + g,
                                           d.nchunks, (uint32_t)d.k, M, ba);
                        }
                    }
                } else if (kind0 == kKindShort) {
                    if (cnt == kP) short_group<1, true>(stage, tile, pfirst, cnt, sM0[warp], sM1[warp], sP[warp], ba);
                    else short_group<1, false>(stage, tile, pfirst, cnt, sM0[warp], sM1[warp], sP[warp], ba);
                } else {
                    if (cnt == kP) short_group<2, true>(stage, tile, pfirst, cnt, sM0[warp], sM1[warp], sP[warp], ba);
                    else short_group<2, false>(stage, tile, pfirst, cnt, sM0[warp], sM1[warp], sP[warp], ba);
                }
            }
            __syncwarp();
            if (lane == 0 && pp.row < nrows) {
                dev::fence_proxy_async_smem();
                issue_tile(ba.planes, tile_of(pp), &sbuf[warp][st][0], &sbar[warp][st]);
            }
            advance(pp);
        }
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
    static std::atomic<int> cache[64][8];  // 0 = not yet computed
    if (device < 0 || device >= 64) return 0;
    const int slot = ws_max < 0 ? 0 : (ws_max > 6 ? 6 : ws_max);
    if (const int g = cache[device][slot].load(std::memory_order_relaxed)) return g;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel(slot), kScanThreads, 0);
    const int g = sms * (per_sm < 1 ? 1 : per_sm);
    cache[device][slot].store(g, std::memory_order_relaxed);
    return g;
}

}  // namespace
}  // namespace pm

namespace pm {
namespace {

// Everything pm_batch_create works out on the host before touching the device.
struct BatchPlan {
    std::vector<PatDesc> desc;
    std::vector<uint4> arena;
    std::vector<uint32_t> order, gkind;
    std::vector<uint2> phases;
    int ws_max = -1;
    int grid = 0;
    uint32_t tiles = 1;
    uint64_t ntiles = 0, runs = 0;
    int key_bits = 0;
};

pm_status check_pairs(const char *who, const pm_text *text, const pm_pattern *const *patterns,
                      uint32_t npat, const int32_t *k, uint64_t capacity, int *dev)
{
    if (npat == 0 || npat > PM_MAX_BATCH || capacity > kMaxCapacity) {
        set_error("%s: npat = %u (1..%u), capacity %llu (<= %llu)", who, npat, PM_MAX_BATCH,
                  (unsigned long long)capacity, (unsigned long long)kMaxCapacity);
        return npat == 0 ? PM_E_ARG : PM_E_TOO_LARGE;
    }
    for (uint32_t p = 0; p < npat; ++p) {
        if (!patterns[p] || k[p] < 0) {
            set_error("%s: pattern %u is NULL or has k < 0", who, p);
            return PM_E_ARG;
        }
    }
    cudaGetDevice(dev);
    if (*dev != text->device) {
        set_error("%s: text lives on device %d, current device is %d", who, text->device, *dev);
        return PM_E_ARG;
    }
    return PM_OK;
}

pm_status plan_batch(const char *who, const pm_text *text, const pm_pattern *const *patterns,
                     uint32_t npat, const int32_t *k, const pm_batch_options *opts, int dev,
                     BatchPlan &pl)
{
    const pm_batch_options o = opts ? *opts : pm_batch_options{};
    auto below_ok = [](int32_t v, int32_t hi) { return v >= -1 && v <= hi; };
    if (o.group < 0 || o.grid < 0 || o.tiles < 0 || o.tiles > kMaxTilesPerItem ||
        !below_ok(o.ws_below, kWsMaxK + 1) || !below_ok(o.ps1_below, 32) || !below_ok(o.ps2_below, 64)) {
        set_error("%s: options out of range (group %d, grid %d, tiles %d, ws_below %d, "
                  "ps1_below %d, ps2_below %d)", who, o.group, o.grid, o.tiles, o.ws_below, o.ps1_below,
                  o.ps2_below);
        return PM_E_ARG;
    }
    // Defaults, measured on GB300 (3.1 Gbp text, 64 pairs of m 32..1024):
    // the window-sliced counter while few positions decide a window (k <= 4),
    // then pattern-sliced groups with shared shifts over one chunk while the
    // windows that survive 32 positions are rare (k <= 17), over two chunks
    // while those surviving 64 are (k <= 40).
    auto below = [](int32_t v, int32_t dflt) { return v == 0 ? dflt : (v < 0 ? 0 : v); };
    const int ws_max = below(o.ws_below, 5) - 1;  // -1: none
    const int ps1_max = below(o.ps1_below, 18) - 1;
    const int ps2_max = below(o.ps2_below, 41) - 1;
    const uint32_t tiles = o.tiles > 0 ? (uint32_t)o.tiles : 1u;
    // rows of 2 groups by default: measured faster than whole categories for
    // the pattern-sliced kinds (k = 16..31: 4-20 %), equal for the others
    const uint32_t groups_per_row = o.group > 0 ? (uint32_t)((o.group + kP - 1) / kP) : 2u;

    // descriptors and arena
    std::vector<PatDesc> &desc = pl.desc;
    desc.assign(npat, PatDesc{});
    std::unordered_map<const pm_pattern *, std::pair<uint64_t, uint64_t>> where;
    std::vector<uint4> &arena = pl.arena;
    uint32_t min_m = UINT32_MAX;
    for (uint32_t p = 0; p < npat; ++p) {
        const pm_pattern *pt = patterns[p];
        auto it = where.find(pt);
        if (it == where.end()) {
            const uint64_t mo = arena.size();
            arena.insert(arena.end(), pt->masks, pt->masks + pt->nchunks);
            const uint64_t lo = arena.size();
            uint4 list[64];  // at most 2 entries per position of the first 32
            ordered_wslist(pt, text, list);
            arena.insert(arena.end(), list, list + pt->n_single + 2 * pt->n_general);
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
        // (a pattern of one chunk is decided exactly by its first 32 positions)
        d.variant = (uint32_t)(d.k <= ws_max                                     ? Variant::kWindowSliced
                               : d.k <= ps1_max || (d.nchunks == 1 && d.k <= 31) ? Variant::kPatternSliced
                               : d.k <= ps2_max                                  ? Variant::kPatternSliced2
                                                                                 : Variant::kAllChunks);
        min_m = std::min(min_m, pt->m);
    }
    if (arena.empty()) arena.push_back(make_uint4(0, 0, 0, 0));

    // Categories: window-sliced pairs with k = 0, 1, ..., then pattern-sliced
    // pairs over one chunk, over two chunks, and over all chunks.  Within a
    // category pairs are ordered by m and cut into groups of kP; the groups
    // of a category are cut into rows of groups_per_row.  A work item is a
    // row crossed with a run of `tiles` warp tiles, rows outermost, so all
    // warps run one kind of evaluation at a time.
    std::vector<std::vector<uint32_t>> cats(kWsMaxK + 4);
    for (uint32_t p = 0; p < npat; ++p) {
        const int32_t kp = desc[p].k;
        const Variant v = (Variant)desc[p].variant;
        const size_t c = v == Variant::kWindowSliced    ? (size_t)kp
                         : v == Variant::kPatternSliced  ? kWsMaxK + 1
                         : v == Variant::kPatternSliced2 ? kWsMaxK + 2
                                                         : kWsMaxK + 3;
        cats[c].push_back(p);
    }
    // gkind: bits 0-1 the kind, bits 2.. the number of real pairs (the last
    // group of a category is padded to kP slots with repeats of its first
    // pair; padding is never emitted)
    for (size_t c = 0; c < cats.size(); ++c) {
        std::vector<uint32_t> &v = cats[c];
        if (v.empty()) continue;
        std::stable_sort(v.begin(), v.end(), [&](uint32_t x, uint32_t y) { return desc[x].m < desc[y].m; });
        const uint32_t kind = c <= (size_t)kWsMaxK       ? kKindWs
                              : c == (size_t)kWsMaxK + 1 ? kKindShort
                              : c == (size_t)kWsMaxK + 2 ? kKindShort2
                                                         : kKindLong;
        const uint32_t g0 = (uint32_t)pl.gkind.size();
        for (size_t i = 0; i < v.size(); i += kP) {
            const uint32_t count = (uint32_t)std::min<size_t>(kP, v.size() - i);
            for (size_t j = i; j < i + kP; ++j) pl.order.push_back(j < v.size() ? v[j] : v[i]);
            pl.gkind.push_back(kind | (count << 2));
        }
        const uint32_t g1 = (uint32_t)pl.gkind.size();
        for (uint32_t r = g0; r < g1; r += std::min(groups_per_row, g1 - r))
            pl.phases.push_back(make_uint2(r, r + std::min(groups_per_row, g1 - r)));
    }
    pl.ws_max = ws_max;
    pl.grid = o.grid > 0 ? o.grid : batched_grid(dev, ws_max);
    pl.tiles = tiles;
    pl.ntiles = min_m <= text->n ? (text->n - min_m + 1 + kTileWindows - 1) / kTileWindows : 0;
    pl.runs = (pl.ntiles + tiles - 1) / tiles;
    const unsigned long long max_key = (unsigned long long)npat * (pl.ntiles ? pl.ntiles : 1) * G;
    pl.key_bits = 0;
    while (pl.key_bits < 64 && (max_key >> pl.key_bits) != 0) ++pl.key_bits;
    return PM_OK;
}

// Lay the batch's device data out from `base` (nullptr: only size it).
// Returns the bytes needed.
size_t carve_batch(const BatchPlan &pl, uint32_t npat, uint64_t capacity, pm_batch *b, char *base)
{
    const uint64_t cap_e = capacity ? capacity : 1;
    const size_t sz[] = {
        align256(npat * sizeof(PatDesc)),
        align256(pl.order.size() * sizeof(uint32_t)),
        align256(pl.gkind.size() * sizeof(uint32_t)),
        align256(std::max<size_t>(pl.phases.size(), 1) * sizeof(uint2)),
        align256(pl.arena.size() * sizeof(uint4)),
        align256(cap_e * sizeof(pm_hit)),
        align256(cap_e * sizeof(SegRecord)),
        align256(sort_scratch_bytes(cap_e)),
        align256(cap_e * sizeof(TileEntry)),
        align256(order_scratch_bytes(cap_e)),
        256,
        align256(npat * sizeof(unsigned long long)),
    };
    size_t total = 0;
    for (size_t x : sz) total += x;
    if (!base) return total;
    char *c = base;
    auto take = [&](size_t i) { char *r = c; c += sz[i]; return (void *)r; };
    b->pats = (PatDesc *)take(0);
    b->order = (uint32_t *)take(1);
    b->gkind = (uint32_t *)take(2);
    b->phases = (uint2 *)take(3);
    b->arena = (uint4 *)take(4);
    b->tmp = (pm_hit *)take(5);
    b->recs = (SegRecord *)take(6);
    b->sort_scratch = take(7);
    b->entries = (TileEntry *)take(8);
    b->order_scratch = take(9);
    b->ctl = (unsigned long long *)take(10);
    b->pat_counts = (unsigned long long *)take(11);
    return total;
}

void fill_batch(const BatchPlan &pl, const pm_text *text, uint32_t npat, uint64_t capacity, int dev,
                pm_batch *b)
{
    b->device = dev;
    b->npat = npat;
    b->ngroups = (uint32_t)pl.gkind.size();
    b->ws_max = pl.ws_max;
    b->grid = pl.grid;
    b->ntiles = pl.ntiles;
    b->tiles = pl.tiles;
    b->runs = pl.runs;
    b->nphases = (uint32_t)pl.phases.size();
    b->capacity = capacity;
    b->planes = text->planes;
    b->unk = text->unk;
    b->key_bits = pl.key_bits;
}

// Copies from pageable host memory are staged by the driver: the plan may be
// destroyed as soon as these calls return.
pm_status upload_batch(const BatchPlan &pl, pm_batch *b, cudaStream_t st)
{
    pm_status rc = cuda_status(cudaMemcpyAsync(b->pats, pl.desc.data(), b->npat * sizeof(PatDesc),
                                               cudaMemcpyHostToDevice, st), "upload descriptors");
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(b->order, pl.order.data(), pl.order.size() * sizeof(uint32_t),
                                         cudaMemcpyHostToDevice, st), "upload groups");
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(b->gkind, pl.gkind.data(), pl.gkind.size() * sizeof(uint32_t),
                                         cudaMemcpyHostToDevice, st), "upload group kinds");
    if (!rc && !pl.phases.empty())
        rc = cuda_status(cudaMemcpyAsync(b->phases, pl.phases.data(), pl.phases.size() * sizeof(uint2),
                                         cudaMemcpyHostToDevice, st), "upload rows");
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(b->arena, pl.arena.data(), pl.arena.size() * sizeof(uint4),
                                         cudaMemcpyHostToDevice, st), "upload arena");
    return rc;
}

// The persistent launch plus the ordering kernels into device buffers.
pm_status run_batch(const pm_batch *b, pm_hit *hits, uint64_t *offsets, cudaStream_t st)
{
    unsigned long long *cursor = b->ctl, *rec_cursor = b->ctl + 1;
    uint32_t *status = (uint32_t *)(b->ctl + 2);
    pm_status rc = cuda_status(cudaMemsetAsync(b->ctl, 0, 256, st), "clear control words");
    if (!rc)
        rc = cuda_status(cudaMemsetAsync(b->pat_counts, 0, b->npat * sizeof(unsigned long long), st),
                         "clear counts");
    if (rc) return rc;
    const uint64_t items = b->runs * b->nphases;
    if (items > 0) {
        BatchArgs ba{b->planes, b->unk, b->pats,  b->order,  b->gkind, b->phases,  b->arena,
                     b->npat,   b->ngroups, b->tiles, b->ntiles, b->runs, items,
                     b->tmp,    b->capacity, cursor,  b->recs,  b->capacity, rec_cursor,
                     b->pat_counts, status};
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

}  // namespace

pm_status search_batched(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                         const int32_t *k, uint64_t capacity, const pm_batch_options *opts,
                         pm_hit *d_hits, uint64_t *d_offsets, void **scratch, cudaStream_t st)
{
    *scratch = nullptr;
    int dev = 0;
    pm_status rc = check_pairs("pm_search (batched)", text, patterns, npat, k, capacity, &dev);
    if (rc) return rc;
    BatchPlan pl;
    rc = plan_batch("pm_search (batched)", text, patterns, npat, k, opts, dev, pl);
    if (rc) return rc;
    pm_batch b{};
    fill_batch(pl, text, npat, capacity, dev, &b);
    const size_t total = carve_batch(pl, npat, capacity, &b, nullptr);
    rc = cuda_status(cudaMallocAsync(scratch, total, st), "cudaMallocAsync batch scratch");
    if (rc) return rc;
    carve_batch(pl, npat, capacity, &b, (char *)*scratch);
    rc = upload_batch(pl, &b, st);
    if (!rc) rc = run_batch(&b, d_hits, d_offsets, st);
    return rc;
}

}  // namespace pm

using namespace pm;

extern "C" {

pm_status pm_batch_create(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                          const int32_t *k, uint64_t capacity, const pm_batch_options *opts,
                          void *stream, pm_batch **out)
{
    TraceRange trace("pm_batch_create");
    if (!text || !out || (npat > 0 && (!patterns || !k))) {
        set_error("pm_batch_create: NULL argument");
        return PM_E_ARG;
    }
    *out = nullptr;
    int dev = 0;
    pm_status rc = check_pairs("pm_batch_create", text, patterns, npat, k, capacity, &dev);
    if (rc) return rc;
    BatchPlan pl;
    rc = plan_batch("pm_batch_create", text, patterns, npat, k, opts, dev, pl);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    pm_batch *b = new (std::nothrow) pm_batch{};
    if (!b) return PM_E_NOMEM;
    fill_batch(pl, text, npat, capacity, dev, b);
    const size_t total = carve_batch(pl, npat, capacity, b, nullptr);
    rc = cuda_status(cudaMalloc(&b->mem, total), "cudaMalloc batch");
    if (rc) {
        delete b;
        return rc;
    }
    carve_batch(pl, npat, capacity, b, (char *)b->mem);
    rc = upload_batch(pl, b, st);
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
    TraceRange trace("pm_batch_run");
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
    return run_batch(b, hits, offsets, (cudaStream_t)stream);
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
