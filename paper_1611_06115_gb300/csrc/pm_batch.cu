// Batched search: many patterns of uneven m and k in one persistent launch
// per category of evaluation over the resident text.
//
// The planner sorts the (pattern, k) pairs into categories by evaluation
// (window-sliced for each k, pattern-sliced over 32 positions, over 64
// positions, every chunk; thresholds are options), orders each category by m
// and cuts it into rows of up to kP pairs.  Each category present gets its
// own launch, so every kernel carries only its own evaluation.  A work item
// is a row crossed with a run of warp tiles, items numbered run-major: the
// warps at work at any time cover a few runs of tiles with every row, so a
// tile comes from device memory once per launch and from L2 for the other
// rows.  A warp stages its tiles (plus halo) in shared memory by its lanes'
// own asynchronous copies kStages tiles ahead, loads its item's row into
// shared memory once, then per tile
//   * pattern-sliced row: for each window, the funnel shifts that line the
//     text up with the first 32 (or 64) positions are done once and serve
//     every pair of the row (whose masks sit in shared memory), so a
//     pair-window costs three (or six) selects, one (or two) popcounts and a
//     quarter of the byte-packed threshold test;
//   * window-sliced row: each pair runs the letter-plane scan over the tile
//     from its compact position list in shared memory;
//   * every-chunk row: each pair keeps 32 running counts per lane.
// The candidates of a pair in a tile (or a 1024-window group of it) are
// settled by the whole warp from a shared-memory queue; their hits are
// written contiguously, in window order, behind one warp-aggregated atomic,
// and one segment record describes them; records are radix-sorted by
// (pair, tile, group) (pm_sort.cu) and the ordering pass (pm_order.cu) lays
// the hits out as per-pair CSR lists sorted by location.
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
constexpr uint32_t kSpassWords = kP * scan::G * 32;  // pass words of one pattern-sliced row and tile
// 32-window groups per lane in a warp tile of category cat: eight for the
// window-sliced launches (the per-tile work spread over 8192 windows, as in
// the per-pattern kernels), four for the others
constexpr int cat_groups(int cat) { return cat <= kWsMaxK ? 8 : scan::G; }
// group kinds
constexpr uint32_t kKindShort = 0;   // pattern-sliced over positions 0..31, shared shifts (k <= 31)
constexpr uint32_t kKindWs = 1;      // window-sliced (k <= kWsMaxK)
constexpr uint32_t kKindLong = 2;    // pattern-sliced over all chunks (any k)
constexpr uint32_t kKindShort2 = 3;  // pattern-sliced over positions 0..63, shared shifts (k <= 63)
// categories of pairs (one launch each): window-sliced with k = 0..kWsMaxK,
// then these
constexpr int kCatPs1 = kWsMaxK + 1;
constexpr int kCatPs2 = kWsMaxK + 2;
constexpr int kCatLong = kWsMaxK + 3;
constexpr int kCats = kWsMaxK + 4;
// Warp tiles per work item (the last run of tiles may reach past the text;
// those tiles are neither copied nor evaluated).
constexpr int kMaxTilesPerItem = 64;
constexpr uint32_t kDefaultTilesPerItem = 16;
}
}  // namespace pm

struct pm_batch {
    int device;
    uint32_t npat;
    uint32_t ngroups;
    uint32_t nphases;  // work-item rows: pieces of the categories of groups
    uint32_t cat_rows[pm::kWsMaxK + 4][2];  // per category: its rows [first, end)
    int grid;          // CTAs per launch (0: as many as each category's kernel keeps resident)
    int key_bits;
    uint32_t tiles;    // warp tiles per work item
    uint64_t ntiles;   // 4096-window tiles of the longest window range
    uint64_t runs;     // runs of `tiles` such tiles covering them
    uint64_t maxwin;   // that window range (windows of the shortest pattern)
    uint64_t key_stride;  // record keys per pair (record_key)
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
    uint64_t ntiles, runs;  // this launch's tiles; items = rows * runs, run-major
    uint64_t key_stride;    // record keys of pair p: p * key_stride + its group index
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

// The sort key of the record of pair p that starts at group `group` of the
// text (tile * groups per tile + group within the tile): pairs in order,
// then the text's groups in order, whatever the tile width of the pair's
// category.
__device__ __forceinline__ unsigned long long record_key(const BatchArgs &ba, uint32_t p, uint64_t group)
{
    return (unsigned long long)p * ba.key_stride + group;
}

// Append one segment record: `count` hits of pair p at tmp[base ..], in
// window order, for the (pair, tile, group) of `key`.  One lane calls it.
__device__ __forceinline__ void put_record(const BatchArgs &ba, uint32_t p, unsigned long long key,
                                           unsigned long long base, uint32_t count)
{
    atomicAdd(ba.pat_counts + p, (unsigned long long)count);
    const unsigned long long r = atomicAdd(ba.rec_cursor, 1ull);
    if (r < ba.rec_cap) ba.recs[r] = SegRecord{key, (uint32_t)base, count};
}

// Emit the hits of one 1024-window group (pass bits of every lane) in window
// order through one warp-aggregated atomic, and append its segment record
// (each lane counting its own hits: the path for dense hits).
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
        put_record(ba, p, key, base, total);
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

// What a work item keeps in shared memory of each pair of its row.
struct RowPair {
    uint32_t p;        // pair index
    uint32_t k;
    uint32_t nchunks;
    uint32_t masks;    // chunk 0 in the arena (uint4 units)
    uint32_t lists;    // n_single | n_general << 8 (window-sliced list)
    uint32_t ntiles;   // warp tiles holding windows of the pair
    uint32_t nfull;    // warp tiles whose windows are all valid for the pair
    uint32_t pad;
    uint64_t nwin;
};

// Window-valid mask of the 32 windows of pair r that start in block blk of
// warp tile `tile`.
__device__ __forceinline__ uint32_t pair_valid(const RowPair &r, uint64_t tile, uint64_t blk)
{
    return tile < r.nfull ? kFull : valid_mask(blk, r.nwin);
}

// The candidates of pair rp in NG groups (g0 .. g0+NG-1) of one staged warp
// tile of GB groups per lane, settled by the whole warp from its
// shared-memory queue q as in settle_emit_queued (see pm_scan_impl.cuh),
// the hits written once and described by one segment record whose key is
// that of group g0.  Returns false, having done nothing, when there are more
// than kQueueCap candidates or k is too large for a count to share 32 bits
// with its window.  Call with the whole warp.
template <int NG, int GB>
__device__ __forceinline__ bool settle_emit_record(const uint32_t (&cand)[NG], uint32_t g0, uint64_t tile,
                                                   const uint2 *stage, uint32_t *q, const RowPair &rp,
                                                   const BatchArgs &ba)
{
    static_assert(NG == 1 || NG == 4 || NG == 8, "one group or four or eight");
    static_assert((GB == 4 || GB == 8) && NG <= GB, "tiles of four or eight groups");
    constexpr int NW = (NG + 3) / 4;                     // words of packed group counts
    constexpr uint32_t kWinBits = GB == 4 ? 12u : 13u;  // window within the tile
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t k = rp.k;
    const uint4 *__restrict__ M = ba.arena + rp.masks;
    // byte j of word i: this lane's candidates in group g0 + 4i + j
    uint32_t packed[NW];
    uint32_t mine = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        packed[i] = 0;
#pragma unroll
        for (int j = 0; j < 4 && 4 * i + j < NG; ++j) packed[i] |= (uint32_t)__popc(cand[4 * i + j]) << (8 * j);
        mine += (packed[i] * 0x01010101u) >> 24;
    }
    const uint32_t total = __reduce_add_sync(kFull, mine);
    if (total > kQueueCap || k >= (1u << (32u - kWinBits))) return false;
    uint32_t pos[NW];
    uint32_t before = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        uint32_t incl = packed[i];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += v;
        }
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        pos[i] = before * 0x01010101u + tot * 0x01010100u + (incl - packed[i]);  // bytes never carry
        before += (tot * 0x01010101u) >> 24;
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        uint32_t at = (pos[i / 4] >> (8 * (i % 4))) & 0xffu;
        uint32_t m = cand[i];
        while (m) {
            const uint32_t w = __ffs(m) - 1;
            m &= m - 1;
            q[at++] = ((g0 + (uint32_t)i) << 10) | (lane << 5) | w;  // window within the tile
        }
    }
    __syncwarp();
    uint32_t hits = 0;
    for (uint32_t i0 = 0; i0 < total; i0 += 32) {
        const uint32_t i = i0 + lane;
        uint32_t rec = 0;
        bool hit = false;
        if (i < total) {
            const uint32_t e = q[i];
            const uint32_t gl = e >> 5;  // block within the tile
            const uint32_t c = candidate_count(stage + gl, tile * (32ull * GB) + gl, e & 31u, M, 0u, rp.nchunks,
                                               k, ba.planes, ba.unk);
            hit = c <= k;
            rec = e | (c << kWinBits);
        }
        const uint32_t hb = __ballot_sync(kFull, hit);
        __syncwarp();  // every entry of this round is read before any is overwritten
        if (hit) q[hits + __popc(hb & ((1u << lane) - 1u))] = rec;
        hits += __popc(hb);
    }
    if (hits) {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) {
            base = atomicAdd(ba.cursor, (unsigned long long)hits);
            put_record(ba, rp.p, record_key(ba, rp.p, tile * GB + g0), base, hits);
        }
        base = __shfl_sync(kFull, base, 0);
        const uint64_t w0 = tile * (1024ull * GB);
        for (uint32_t i = lane; i < hits; i += 32) {
            const uint32_t r = q[i];
            if (base + i < ba.cap)
                ba.tmp[base + i] = pm_hit{(uint32_t)(w0 + (r & ((1u << kWinBits) - 1u))), r >> kWinBits};
        }
    }
    __syncwarp();  // the queue is rewritten next
    return true;
}

// One pattern-sliced group over the first C chunks (C = 1: k <= 31, C = 2:
// k <= 63) on one staged tile: for each window the funnel shifts that line
// the text up with the chunks are done once and serve all kP slots of the
// group, whose masks sit in shared memory (sM0, sM1; sP {k in every byte};
// loaded once per work item; a slot without a pair has empty masks and
// k = 0, so none of its windows ever passes).  Bytes of the multiply-add
// results hold (4/C) * (matches + k) <= (4/C) * (64C - 1) < 256, so bit 7 of
// a byte is set exactly when matches + k >= 32C, i.e. when the window has at
// most k mismatches in those positions.  The pass words of every slot and
// group go to shared memory (spass); once the tile is done, one loop over the
// pairs (not unrolled, so the kernel carries that code once) settles each
// pair's candidates of the whole tile together with the whole warp
// (settle_emit_record; each lane its own when there are too many).  A
// 1024-window group holds about two candidates of a pair on the 4096-pattern
// workload, so settling per group cost as much as the evaluation.
template <int C>
__device__ __forceinline__ void short_group(const uint2 *stage, uint64_t tile, uint32_t cnt, const RowPair *rp,
                                            const uint4 *sM0, const uint4 *sM1, const uint4 *sP, uint32_t *q,
                                            uint32_t *spass, uint32_t two, const BatchArgs &ba)
{
    const int lane = threadIdx.x & 31;
    const uint32_t m1 = C == 1 ? two << 1 : two, m8 = m1 << 8, m16 = m1 << 16, m24 = m1 << 24;
    uint32_t anyp = 0;
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
        const uint2 ta = stage[32 * g + lane], tb = stage[32 * g + lane + 1];
        const uint2 c = C == 2 ? stage[32 * g + lane + 2] : make_uint2(0u, 0u);
        uint32_t acc[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) acc[p] = 0u;
        // one step at a time: with the steps unrolled the kernel spills and
        // is larger (instruction fetch was its largest stall)
#pragma unroll 1
        for (uint32_t j = 0; j < 8; ++j) {
            uint32_t lo[4], hi[4], lo1[4], hi1[4];
#pragma unroll
            for (uint32_t qq = 0; qq < 4; ++qq) {
                lo[qq] = __funnelshift_r(ta.x, tb.x, 8 * qq + j);
                hi[qq] = __funnelshift_r(ta.y, tb.y, 8 * qq + j);
                if (C == 2) {
                    lo1[qq] = __funnelshift_r(tb.x, c.x, 8 * qq + j);
                    hi1[qq] = __funnelshift_r(tb.y, c.y, 8 * qq + j);
                }
            }
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                const uint4 M0 = sM0[p];
                uint32_t gm[4];
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) gm[qq] = __popc(class_match(lo[qq], hi[qq], M0));
                if (C == 2) {
                    const uint4 M1 = sM1[p];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) gm[qq] += __popc(class_match(lo1[qq], hi1[qq], M1));
                }
                uint32_t v = mad_lo(gm[3], m24, sP[p].x);
                v = mad_lo(gm[2], m16, v);
                v = mad_lo(gm[1], m8, v);
                v = mad_lo(gm[0], m1, v);
                // window 8q + j: bit 7 of byte q goes to bit 8q + j
                acc[p] |= (v >> (7 - j)) & (0x01010101u << j);
            }
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            spass[(p * G + g) * 32 + lane] = acc[p];
            anyp |= acc[p];
        }
    }
    if (!__any_sync(kFull, anyp != 0u)) return;  // warp-uniform; the common case
    __syncwarp();
    uint64_t blk[G];
#pragma unroll
    for (int g = 0; g < G; ++g) blk[g] = tile * (32ull * G) + 32ull * g + (uint64_t)lane;
#pragma unroll 1
    for (uint32_t p = 0; p < cnt; ++p) {
        const RowPair &r = rp[p];
        if (tile >= r.ntiles) continue;
        uint32_t pass[G], anyr = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            pass[g] = spass[(p * G + g) * 32 + lane] & pair_valid(r, tile, blk[g]);
            anyr |= pass[g];
        }
        if (!__any_sync(kFull, anyr != 0u) || settle_emit_record<G, G>(pass, 0u, tile, stage, q, r, ba)) continue;
        const uint4 *M = ba.arena + r.masks;
#pragma unroll 1
        for (int g = 0; g < G; ++g) {
            uint32_t ps = pass[0];  // pass[g] by selects (a run-time index would move pass to local memory)
#pragma unroll
            for (int i = 1; i < G; ++i) ps = g == i ? pass[i] : ps;
            if (r.nchunks > (uint32_t)C)
                ps = settle_staged(ps, blk[0] + 32ull * g, stage[32 * g + lane], stage[32 * g + lane + 1],
                                   stage + 32 * g + lane + 2, M, 0u, r.nchunks, r.k, ba.planes);
            if (__any_sync(kFull, ps != 0u))
                emit_group(ps, blk[0] + 32ull * g, r.p, record_key(ba, r.p, tile * G + g),
                           r.nchunks, r.k, M, ba);
        }
    }
    __syncwarp();  // spass is rewritten by the next tile
}

// Window-sliced pair rp over one staged tile of GB groups per lane (a, b:
// the lane's blocks; list: the pair's compact list in shared memory): the
// scan of alive_window_sliced over all groups at once, the candidates
// settled by the warp together.
template <int K, int GB>
__device__ __forceinline__ void ws_pair(const uint2 (&a)[GB], const uint2 (&b)[GB], const uint2 *stage,
                                        uint64_t tile, const RowPair &rp, const uint32_t *list, uint32_t *q,
                                        const BatchArgs &ba)
{
    const int lane = threadIdx.x & 31;
    uint32_t valid[GB], pass[GB];
    uint64_t blk[GB];
#pragma unroll
    for (int g = 0; g < GB; ++g) {
        blk[g] = tile * (32ull * GB) + 32ull * g + (uint64_t)lane;
        valid[g] = pair_valid(rp, tile, blk[g]);
    }
    const bool cut =
        alive_window_sliced<K>(a, b, list, rp.lists & 0xffu, rp.lists >> 8, ws_cut(K), valid, pass);
    uint32_t anyp = 0;
#pragma unroll
    for (int g = 0; g < GB; ++g) anyp |= pass[g];
    if (__any_sync(kFull, anyp != 0u) && !settle_emit_record<GB, GB>(pass, 0u, tile, stage, q, rp, ba)) {
        const uint4 *M = ba.arena + rp.masks;
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const uint32_t ps = (cut || rp.nchunks > 1)
                                    ? settle_from_regs(pass[g], blk[g], a[g], b[g], M, rp.nchunks, rp.k, ba.planes)
                                    : pass[g];
            if (__any_sync(kFull, ps != 0u))
                emit_group(ps, blk[g], rp.p, record_key(ba, rp.p, tile * GB + g), rp.nchunks,
                           rp.k, M, ba);
        }
    }
}

// CAT: the category of every row of the launch (one launch per category
// present, so that each kernel carries only its own evaluation: one kernel
// holding every kind stalled on instruction fetch): 0..kWsMaxK
// window-sliced pairs with k = CAT, then kCatPs1, kCatPs2, kCatLong.
//
// A row is one group of up to kP pairs; a work item is a run of T warp
// tiles crossed with a row, items numbered run-major (item = run * rows +
// row), so the warps at work at any time cover a few runs of tiles with
// every row: each text tile is read from device memory once and then from
// L2.  A warp loads its item's row (the pairs' descriptors and masks or
// position lists) into shared memory once, then walks the item's tiles;
// the tiles of its whole sequence of items are staged kStages ahead by the
// lanes' own asynchronous copies, and a stage is refilled once the warp is
// done with its tile.
//
// Window-sliced launches run tiles of eight groups per lane (8192 windows),
// the others tiles of four (cat_groups).  The window-sliced and every-chunk
// launches run two CTAs per SM (measured faster than three, whose 80
// registers spill), the pattern-sliced ones three.  The stages (and a
// pattern-sliced row's pass words) sit in dynamic shared memory
// (batched_smem).
template <int CAT>
__global__ void __launch_bounds__(kScanThreads, CAT <= kWsMaxK || CAT == kCatLong ? 2 : 3)
    k_scan_batched(const BatchArgs ba)
{
    constexpr bool kWsCat = CAT <= kWsMaxK;
    constexpr int GB = cat_groups(CAT);
    constexpr uint32_t S = kStages;
    constexpr uint32_t kSB = scan_stage_blocks<GB>();
    extern __shared__ __align__(128) uint2 dsmem[];
    uint2 (*sbuf)[S][kSB] = reinterpret_cast<uint2 (*)[S][kSB]>(dsmem);  // [kScanWarps][S][kSB]
    uint32_t *spass = reinterpret_cast<uint32_t *>(dsmem + kScanWarps * S * kSB);  // kSpassWords per warp
    __shared__ uint32_t squeue[kScanWarps][kQueueCap];
    __shared__ RowPair srow[kScanWarps][kP];
    __shared__ uint32_t slist[kScanWarps][kWsCat ? kP : 1][32];
    __shared__ uint4 sM0[kScanWarps][kP];
    __shared__ uint4 sM1[kScanWarps][kP];
    __shared__ uint4 sP[kScanWarps][kP];  // pattern-sliced group: {k in every byte, 0, 0, 0}

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * kScanWarps;
    const uint32_t T = ba.tiles;
    const uint32_t nrows = (uint32_t)(ba.items / ba.runs);
    const uint32_t items = (uint32_t)ba.items;  // runs * rows < 2^31 (the planner widens the runs)
    const uint64_t ntiles = ba.ntiles;
    // the tile of position u of item i (tiles past the text are never copied nor evaluated)
    auto tile_of = [&](uint32_t i, uint32_t u) { return (uint64_t)(i / nrows) * T + u; };

    const uint32_t first = blockIdx.x * kScanWarps + warp;
    uint32_t pi = first, pu = 0;  // next position to stage
#pragma unroll
    for (uint32_t st = 0; st < S; ++st) {
        if (pi < items) {
            const uint64_t t = tile_of(pi, pu);
            if (t < ntiles) copy_tile_async<GB>(ba.planes, t * (32u * GB), &sbuf[warp][st][0], lane);
        }
        cp_async_commit();
        if (++pu == T) {
            pu = 0;
            pi += stride;
        }
    }

    uint32_t st = 0;
    for (uint32_t item = first; item < items; item += stride) {
        // ---- the item's row into shared memory ----
        const uint32_t row = item % nrows;
        const uint2 ph = __ldg(ba.phases + row);  // one group
        const uint32_t grp = ph.x;
        const uint32_t cnt = __ldg(ba.gkind + grp) >> 2;
        __syncwarp();  // the previous item is done with the row's slots
        if constexpr (!kWsCat) {
            if (lane >= (int)cnt && lane < kP) {  // empty slot: no position matches, k = 0
                sM0[warp][lane] = make_uint4(0u, 0u, 0u, 0u);
                sM1[warp][lane] = make_uint4(0u, 0u, 0u, 0u);
                sP[warp][lane] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        if (lane < (int)cnt) {
            const uint32_t p = __ldg(ba.order + grp * kP + lane);
            const PatDesc &d = ba.pats[p];
            RowPair r;
            r.p = p;
            r.k = (uint32_t)d.k;
            r.nchunks = d.nchunks;
            r.masks = (uint32_t)d.masks;
            r.lists = d.n_single | (d.n_general << 8);
            r.ntiles = (uint32_t)d.ntiles;
            r.nfull = (uint32_t)(d.nwin / (1024u * GB));
            r.pad = 0;
            r.nwin = d.nwin;
            srow[warp][lane] = r;
            if constexpr (!kWsCat) {
                const uint32_t two = d.two;
                const uint32_t m1 = CAT == kCatPs1 ? two << 1 : two;
                sM0[warp][lane] = __ldg(ba.arena + d.masks);
                sM1[warp][lane] = d.nchunks > 1 ? __ldg(ba.arena + d.masks + 1) : make_uint4(kFull, kFull, kFull, kFull);
                sP[warp][lane] = make_uint4(r.k * ((m1 << 24) | (m1 << 16) | (m1 << 8) | m1), 0u, 0u, 0u);
            }
        }
        if constexpr (kWsCat) {
            __syncwarp();
            // kP compact lists of at most 32 words
            for (uint32_t i = lane; i < cnt * 32u; i += 32) {
                const RowPair &r = srow[warp][i >> 5];
                const uint32_t len = (r.lists & 0xffu) + (r.lists >> 8);
                const uint32_t w = i & 31u;
                if (w < len) {
                    const uint32_t p = r.p;
                    slist[warp][i >> 5][w] = __ldg((const uint32_t *)(ba.arena + ba.pats[p].wslist) + w);
                }
            }
        }
        __syncwarp();
        const uint32_t two = ba.pats[srow[warp][0].p].two;

        for (uint32_t u = 0; u < T; ++u) {
            cp_async_wait<S - 1>();  // this tile's group has landed
            __syncwarp();
            const uint64_t tile = tile_of(item, u);
            const uint2 *stage = &sbuf[warp][st][0];
            if (tile < ntiles) {
                if constexpr (kWsCat) {
                    uint2 a[GB], b[GB];
#pragma unroll
                    for (int g = 0; g < GB; ++g) {
                        a[g] = stage[32 * g + lane];
                        b[g] = stage[32 * g + lane + 1];
                    }
                    for (uint32_t i = 0; i < cnt; ++i) {
                        const RowPair &r = srow[warp][i];
                        if (tile >= r.ntiles) continue;  // this pair's windows end before the tile
                        ws_pair<CAT, GB>(a, b, stage, tile, r, slist[warp][i], squeue[warp], ba);
                    }
                } else if constexpr (CAT == kCatLong) {
                    for (uint32_t i = 0; i < cnt; ++i) {
                        const RowPair &r = srow[warp][i];
                        if (tile >= r.ntiles) continue;
                        const uint4 *M = ba.arena + r.masks;
#pragma unroll 1
                        for (int g = 0; g < G; ++g) {
                            const uint64_t blk = tile * (32ull * G) + 32ull * g + (uint64_t)lane;
                            uint32_t pass[1] = {pass_multi_chunk(ba.planes, blk, M, r.nchunks, r.k,
                                                                 pair_valid(r, tile, blk), stage[32 * g + lane],
                                                                 stage[32 * g + lane + 1])};
                            if (__any_sync(kFull, pass[0] != 0u) &&
                                !settle_emit_record<1, G>(pass, (uint32_t)g, tile, stage, squeue[warp], r, ba))
                                emit_group(pass[0], blk, r.p, record_key(ba, r.p, tile * G + g),
                                           r.nchunks, r.k, M, ba);
                        }
                    }
                } else {
                    constexpr int C = CAT == kCatPs1 ? 1 : 2;
                    short_group<C>(stage, tile, cnt, srow[warp], sM0[warp], sM1[warp], sP[warp], squeue[warp],
                                   spass + warp * kSpassWords, two, ba);
                }
            }
            // refill this stage with the position S ahead
            __syncwarp();
            if (pi < items) {
                const uint64_t t = tile_of(pi, pu);
                if (t < ntiles) copy_tile_async<GB>(ba.planes, t * (32u * GB), &sbuf[warp][st][0], lane);
            }
            cp_async_commit();
            if (++pu == T) {
                pu = 0;
                pi += stride;
            }
            if (++st == S) st = 0;
        }
    }
    cp_async_wait<0>();  // nothing in flight when the warp leaves
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int CAT>
const void *batched_ptr()
{
    return (const void *)&k_scan_batched<CAT>;
}

const void *batched_kernel(int cat)
{
    switch (cat) {
    case 0: return batched_ptr<0>();
    case 1: return batched_ptr<1>();
    case 2: return batched_ptr<2>();
    case 3: return batched_ptr<3>();
    case 4: return batched_ptr<4>();
    case 5: return batched_ptr<5>();
    case 6: return batched_ptr<6>();
    case 7: return batched_ptr<7>();
    case 8: return batched_ptr<8>();
    case kCatPs1: return batched_ptr<kCatPs1>();
    case kCatPs2: return batched_ptr<kCatPs2>();
    default: return batched_ptr<kCatLong>();
    }
}
static_assert(kWsMaxK == 8, "one window-sliced launch per k = 0 .. 8");

// Dynamic shared memory of a launch of category cat: the stages of its
// warps and, for a pattern-sliced row, its pass words (with the static
// arrays past the 48 KB that static shared memory may hold).
size_t batched_smem(int cat)
{
    const size_t stages = (size_t)kScanWarps * kStages * (32u * cat_groups(cat) + 4u) * sizeof(uint2);
    return stages + (cat == kCatPs1 || cat == kCatPs2 ? (size_t)kScanWarps * kSpassWords * sizeof(uint32_t) : 0);
}

// Sets the kernel of category cat up on the current device (its dynamic
// shared memory limit) and returns how many CTAs a launch keeps resident
// (0 on failure, with the error left for cudaGetLastError).
int batched_grid(int device, int cat)
{
    static std::atomic<int> cache[64][kCats];  // 0 = not yet set up
    if (device < 0 || device >= 64 || cat < 0 || cat >= kCats) return 0;
    if (const int g = cache[device][cat].load(std::memory_order_relaxed)) return g;
    int sms = 0, per_sm = 0;
    const size_t smem = batched_smem(cat);
    if (smem && cudaFuncSetAttribute(batched_kernel(cat), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel(cat), kScanThreads, smem) !=
            cudaSuccess)
        return 0;
    const int g = sms * (per_sm < 1 ? 1 : per_sm);
    cache[device][cat].store(g, std::memory_order_relaxed);
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
    uint32_t cat_rows[kCats][2] = {};
    int grid = 0;
    uint32_t tiles = 1;
    uint64_t ntiles = 0, runs = 0;  // in 4096-window tiles
    uint64_t maxwin = 0;            // windows of the shortest pattern
    uint64_t key_stride = 0;        // record keys per pair
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
    // the window-sliced counters while few positions decide a window (k <= 8),
    // then pattern-sliced groups with shared shifts over one chunk while the
    // windows that survive 32 positions are rare (k <= 17), over two chunks
    // while those surviving 64 are (k <= 40).
    auto below = [](int32_t v, int32_t dflt) { return v == 0 ? dflt : (v < 0 ? 0 : v); };
    const int ws_max = below(o.ws_below, 9) - 1;  // -1: none
    const int ps1_max = below(o.ps1_below, 18) - 1;
    const int ps2_max = below(o.ps2_below, 41) - 1;
    uint32_t tiles = o.tiles > 0 ? (uint32_t)o.tiles : kDefaultTilesPerItem;
    // a row is one group of kP pairs (o.group is accepted and not used)
    const uint32_t groups_per_row = 1u;

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
            uint4 list[8] = {};  // one word per position of the first 32
            ordered_wslist(pt, text, (uint32_t *)list);
            arena.insert(arena.end(), list, list + wslist_units(pt));
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

    // Categories: window-sliced pairs with k = 0, 1, ..., 8, then pattern-sliced
    // pairs over one chunk, over two chunks, and over all chunks.  Within a
    // category pairs are ordered by m and cut into groups of kP, one row
    // each.  A work item is a row crossed with a run of `tiles` warp tiles;
    // each category runs as its own launch, items numbered run-major.
    std::vector<std::vector<uint32_t>> cats(kCats);
    for (uint32_t p = 0; p < npat; ++p) {
        const int32_t kp = desc[p].k;
        const Variant v = (Variant)desc[p].variant;
        const size_t c = v == Variant::kWindowSliced    ? (size_t)kp
                         : v == Variant::kPatternSliced  ? kCatPs1
                         : v == Variant::kPatternSliced2 ? kCatPs2
                                                         : kCatLong;
        cats[c].push_back(p);
        const uint64_t tw = 1024ull * (uint64_t)cat_groups((int)c);  // the category's tile
        desc[p].ntiles = (desc[p].nwin + tw - 1) / tw;
    }
    // gkind: bits 0-1 the kind, bits 2.. the number of real pairs (the last
    // group of a category is padded to kP slots with repeats of its first
    // pair; padding is never emitted)
    for (size_t c = 0; c < cats.size(); ++c) {
        std::vector<uint32_t> &v = cats[c];
        if (v.empty()) continue;
        std::stable_sort(v.begin(), v.end(), [&](uint32_t x, uint32_t y) { return desc[x].m < desc[y].m; });
        const uint32_t kind = c <= (size_t)kWsMaxK     ? kKindWs
                              : c == (size_t)kCatPs1 ? kKindShort
                              : c == (size_t)kCatPs2 ? kKindShort2
                                                         : kKindLong;
        const uint32_t g0 = (uint32_t)pl.gkind.size();
        for (size_t i = 0; i < v.size(); i += kP) {
            const uint32_t count = (uint32_t)std::min<size_t>(kP, v.size() - i);
            for (size_t j = i; j < i + kP; ++j) pl.order.push_back(j < v.size() ? v[j] : v[i]);
            pl.gkind.push_back(kind | (count << 2));
        }
        const uint32_t g1 = (uint32_t)pl.gkind.size();
        pl.cat_rows[c][0] = (uint32_t)pl.phases.size();
        for (uint32_t r = g0; r < g1; r += std::min(groups_per_row, g1 - r))
            pl.phases.push_back(make_uint2(r, r + std::min(groups_per_row, g1 - r)));
        pl.cat_rows[c][1] = (uint32_t)pl.phases.size();
    }
    pl.grid = o.grid > 0 ? o.grid : 0;
    pl.maxwin = min_m <= text->n ? text->n - min_m + 1 : 0;
    pl.ntiles = (pl.maxwin + kTileWindows - 1) / kTileWindows;  // in the smallest tiles
    // item numbers (runs * rows of a category) stay below 2^31
    const uint64_t rows = std::max<uint64_t>(pl.phases.size(), 1);
    while ((pl.ntiles + tiles - 1) / tiles * rows >= (1ull << 31)) tiles *= 2;
    pl.tiles = tiles;
    pl.runs = (pl.ntiles + tiles - 1) / tiles;
    // keys: pair * key_stride + group of the text (record_key); the stride
    // covers the groups of both tile widths
    pl.key_stride = std::max<uint64_t>(std::max<uint64_t>(pl.ntiles, 1) * (uint64_t)G,
                                       ((pl.maxwin + 8191) / 8192) * 8ull);
    const unsigned long long max_key = (unsigned long long)npat * pl.key_stride;
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
    std::memcpy(b->cat_rows, pl.cat_rows, sizeof b->cat_rows);
    b->grid = pl.grid;
    b->ntiles = pl.ntiles;
    b->tiles = pl.tiles;
    b->runs = pl.runs;
    b->maxwin = pl.maxwin;
    b->key_stride = pl.key_stride;
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
    // one persistent launch per category present, back to back on the stream
    for (int cat = 0; !rc && cat < kCats; ++cat) {
        const uint32_t r0 = b->cat_rows[cat][0], r1 = b->cat_rows[cat][1];
        // the category's tiles (eight or four groups per lane) and runs of them
        const uint64_t tw = 1024ull * (uint64_t)cat_groups(cat);
        const uint64_t ntiles = (b->maxwin + tw - 1) / tw, runs = (ntiles + b->tiles - 1) / b->tiles;
        const uint64_t items = runs * (uint64_t)(r1 - r0);
        if (items == 0) continue;
        BatchArgs ba{b->planes, b->unk, b->pats,  b->order,  b->gkind, b->phases + r0, b->arena,
                     b->npat,   b->ngroups, b->tiles, ntiles, runs, b->key_stride, items,
                     b->tmp,    b->capacity, cursor,  b->recs,  b->capacity, rec_cursor,
                     b->pat_counts, status};
        uint64_t grid = (items + kScanWarps - 1) / kScanWarps;
        const int resident = batched_grid(b->device, cat);
        if (resident == 0) {
            rc = cuda_status(cudaGetLastError(), "batched kernel set-up");
            if (!rc) rc = cuda_status(cudaErrorInvalidValue, "batched kernel set-up");
            break;
        }
        const int lim = b->grid > 0 ? b->grid : resident;
        if (grid > (uint64_t)lim) grid = (uint64_t)lim;
        void *args[] = {(void *)&ba};
        rc = cuda_status(cudaLaunchKernel(batched_kernel(cat), dim3((unsigned)grid), dim3(kScanThreads), args,
                                          batched_smem(cat), st),
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
    // the kernels' set-up on this device happens here, before any launch
    // (and before a stream capture of pm_batch_run)
    for (int cat = 0; cat < kCats; ++cat)
        if (pl.cat_rows[cat][1] > pl.cat_rows[cat][0] && batched_grid(dev, cat) == 0) {
            rc = cuda_status(cudaGetLastError(), "batched kernel set-up");
            return rc ? rc : cuda_status(cudaErrorInvalidValue, "batched kernel set-up");
        }
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
