// Internal declarations of libpm (not part of the public ABI).
//
// Device layout of a coded text (Sec. 2.1, Table 1): symbol s has the 2-bit
// code A=00 C=01 G=10 T=11.  Symbols are grouped in blocks of 32; block b is
// one uint2 {lo, hi} whose bit w holds the low / high code bit of symbol
// 32*b + w.  The planes end with kPadBlocks zero blocks (symbol "A") so that
// every tile copy and every window read stays inside the allocation; windows
// that would use padding are never reported.
//
// Device layout of a compiled pattern (Sec. 2.2, Table 2): chunk c covers
// positions 32c .. 32c+31 and is one uint4 {A, C, G, T} of membership masks:
// bit b of the A word is set iff text letter A lies in the class of position
// 32c+b (Table 3 holds 0 for that pair).  Positions past m have all four bits
// set, so they never count as a mismatch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "pm.h"

struct pm_text {
    uint64_t n;          // symbols
    uint64_t nblocks;    // allocated blocks, padding included
    uint2 *planes;       // device
    uint32_t *unk;       // device, one bit per symbol outside Table 1 (block layout of the
                         //   planes, zero padded); NULL when the text has none
    int device;
    uint64_t count[4];   // how many A, C, G, T the text holds (Table 1 order)
    uint64_t n_unknown;  // symbols outside Table 1 (coded as some letter in the planes)
};

struct pm_pattern {
    uint32_t m;
    uint32_t nchunks;
    uint32_t unknown;  // symbols coded "-" because Table 2 does not list them
    uint4 *masks;      // host, nchunks entries
    // The first min(m, 32) positions as a list for the window-sliced scan:
    // n_single entries {shift j, letter code, 0, 0} for one-letter classes
    // (Table 1 codes A=0 C=1 G=2 T=3), then n_general pairs {j, 0, 0, 0},
    // {A, C, G, T} (membership broadcast) for the other classes; N (every
    // letter) is left out because it never mismatches.
    uint32_t n_single;
    uint32_t n_general;
    uint4 *wslist;     // host, n_single + 2 * n_general entries
};

namespace pm {

// A named range on the host timeline for profilers (NVTX; costs nothing when
// no tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// The window-sliced list of p (see pm_pattern) reordered for text t so that
// windows die as early as possible (the early stop of Sec. 2.4 then ends the
// scan sooner; the sum of Eq. 4 does not depend on the order): one-letter
// entries by increasing frequency of their letter in t (ties by letter, so
// that each letter's entries form one run), then the class entries by
// increasing frequency of their letters.  Stable.  `out` receives the list
// in the kernels' compact form, one 32-bit word per listed position
// (n_single + n_general words, at most 32):
//   one-letter entry  bits 0-4 the position j, bits 5-6 the letter's Table 1
//                     code, bits 8-13 the index one past the end of its run;
//   class entry       bits 0-4 the position j, bits 16-19 the class's
//                     membership (A, C, G, T), bit 31 set.
inline void ordered_wslist(const pm_pattern *p, const pm_text *t, uint32_t *out)
{
    const uint32_t ns = p->n_single, ng = p->n_general;
    uint32_t idx[64];
    uint64_t key[64];
    for (uint32_t i = 0; i < ns; ++i) {
        const uint4 e = p->wslist[i];
        idx[i] = i;
        key[i] = (t->count[e.y & 3u] << 2) | (e.y & 3u);  // counts < 2^32
    }
    for (uint32_t i = 0; i < ng; ++i) {
        const uint4 mem = p->wslist[ns + 2 * i + 1];
        idx[ns + i] = i;
        key[ns + i] = (mem.x ? t->count[0] : 0) + (mem.y ? t->count[1] : 0) +
                      (mem.z ? t->count[2] : 0) + (mem.w ? t->count[3] : 0);
    }
    // insertion sorts (at most 32 entries each), stable
    auto sort_range = [&](uint32_t lo, uint32_t hi) {
        for (uint32_t i = lo + 1; i < hi; ++i)
            for (uint32_t j = i; j > lo && key[j] < key[j - 1]; --j) {
                std::swap(key[j], key[j - 1]);
                std::swap(idx[j], idx[j - 1]);
            }
    };
    sort_range(0, ns);
    sort_range(ns, ns + ng);
    uint32_t code[32];
    for (uint32_t i = 0; i < ns; ++i) {
        const uint4 e = p->wslist[idx[i]];
        code[i] = e.y & 3u;
        out[i] = (e.x & 31u) | (code[i] << 5);
    }
    uint32_t end = ns;
    for (uint32_t i = ns; i-- > 0;) {
        if (i + 1 < ns && code[i + 1] != code[i]) end = i + 1;
        out[i] |= end << 8;
    }
    for (uint32_t i = 0; i < ng; ++i) {
        const uint32_t j = p->wslist[ns + 2 * idx[ns + i]].x;
        const uint4 mem = p->wslist[ns + 2 * idx[ns + i] + 1];
        out[ns + i] = (j & 31u) | ((mem.x & 1u) << 16) | ((mem.y & 1u) << 17) | ((mem.z & 1u) << 18) |
                      ((mem.w & 1u) << 19) | (1u << 31);
    }
}

// uint4 units the compact list of p takes in an arena (four words each).
inline uint32_t wslist_units(const pm_pattern *p) { return (p->n_single + p->n_general + 3) / 4; }

constexpr int kScanThreads = 256;                        // threads per scan CTA
constexpr int kScanWarps = kScanThreads / 32;
constexpr int kGroups = 4;                               // 32-window groups per lane per tile
constexpr uint64_t kTileWindows = 32ull * 32 * kGroups;  // one warp tile: 4096 windows
constexpr uint32_t kStages = 3;                          // tiles a scan warp keeps staged or in flight
constexpr uint64_t kPadBlocks = 1024;                    // zero blocks after the text
constexpr int kWsMaxK = 8;                               // window-sliced scan handles k <= 8
constexpr uint64_t kMaxCapacity = 0xffffffffull;         // hits addressable by a tile entry

// One (pattern, k) of a search, as the kernels see it.
struct PatDesc {
    uint32_t m;          // pattern length
    uint32_t nchunks;    // ceil(m / 32)
    int32_t k;           // allowed mismatches (>= 0)
    uint32_t n_single;   // window-sliced list: one-letter entries
    uint32_t n_general;  // window-sliced list: other-class entry pairs
    uint32_t two;        // the constant 2, given at run time so that the multiply-adds
                         //   built on it stay multiply-adds (FMA pipe)
    uint32_t variant;    // Variant chosen for this pattern (batched kernel)
    uint32_t c0;         // pattern-sliced scan kernels: the chunk their first stage tests
                         //   (first_stage_chunk); 0 everywhere else
    uint64_t masks;      // chunk 0 in the arena (uint4 units)
    uint64_t wslist;     // window-sliced list (compact words, see ordered_wslist) in the arena
                         //   (offset in uint4 units)
    uint64_t nwin;       // windows: n - m + 1, or 0 when m > n
    uint64_t tile0;      // first tile-table entry of this pattern
    uint64_t ntiles;     // warp tiles: ceil(nwin / windows per tile of the kernel that runs)
};

// Hits of one (pattern, warp tile): how many, and where the scan kernel put
// them in the scratch hit buffer.  Within a tile they are in window order.
struct TileEntry {
    uint32_t count;
    uint32_t src;
};

// Device status bits written by kernels.
constexpr uint32_t kDevTimeout = 1u;

// Scan-kernel variants.
enum class Variant : int {
    kPatternSliced = 0,   // per window, positions 0..31 in one word, popc; then settle (k <= 31)
    kWindowSliced = 1,    // per position, 32 windows per word, bit-sliced counters (k <= 8)
    kPatternSliced2 = 2,  // as kPatternSliced over positions 0..63 (k <= 63)
    kAllChunks = 3,       // per window, running counts over every chunk (any k)
};

// The variant that runs when v is asked for at this k: window-sliced beyond
// kWsMaxK becomes pattern-sliced, and a pattern-sliced form beyond its k
// becomes kAllChunks.
Variant resolve_variant(Variant v, int32_t k);

// pm_search_ex's one-launch path (pm_batch.cu): plans the pairs as
// pm_batch_create does, takes all scratch from the stream-ordered pool
// (*scratch, to be freed on the stream by the caller, also on error) and
// queues the batched launch and ordering into the device outputs.
pm_status search_batched(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                         const int32_t *k, uint64_t capacity, const pm_batch_options *opts,
                         pm_hit *d_hits, uint64_t *d_offsets, void **scratch, cudaStream_t st);

// Launch one scan kernel for one pattern (pm_scan.cu).
cudaError_t launch_scan(Variant v, const uint2 *planes, const uint32_t *unk, const PatDesc &d,
                        const uint4 *arena, TileEntry *table, pm_hit *tmp, uint64_t cap,
                        unsigned long long *cursor, uint32_t *status, int grid, cudaStream_t stream);

// Number of resident scan CTAs the device runs at once (pm_scan.cu).
int scan_grid_limit(Variant v, int32_t k, int device);

// The variant chosen when the caller leaves it open (the device's table, see
// pm_set_auto_variants; already resolved for d.k).
Variant auto_variant(const PatDesc &d, int device);

// 32-window groups per lane in a warp tile of the per-pattern scan kernel of
// variant v (resolved) at this k: 8 for the window-sliced kernels, whose
// evaluation per tile is short enough that the per-tile work (copies, list
// reads, checks, the tile's entry) weighs (GB300, 3.1 Gbp, against 4: k = 1
// 0.31 -> 0.27 ms, k = 2 0.47 -> 0.41 ms, k = 4 0.64 -> 0.61 ms, k = 8
// 0.84 -> 0.82 ms; from k = 3 on with half the resident warps, so that the
// counters of eight groups stay in registers), else 4.  A tile covers
// 1024 * scan_groups windows.
inline int scan_groups(Variant v, int32_t) { return v == Variant::kWindowSliced ? 8 : 4; }
inline uint64_t scan_tile_windows(Variant v, int32_t k) { return 1024ull * (uint64_t)scan_groups(v, k); }

// PM_VARIANT_* (not AUTO) <-> Variant.
inline Variant variant_from_public(int32_t v)
{
    switch (v) {
    case PM_VARIANT_WINDOW_SLICED: return Variant::kWindowSliced;
    case PM_VARIANT_PATTERN_SLICED_2: return Variant::kPatternSliced2;
    case PM_VARIANT_ALL_CHUNKS: return Variant::kAllChunks;
    default: return Variant::kPatternSliced;
    }
}
inline int32_t variant_to_public(Variant v)
{
    switch (v) {
    case Variant::kWindowSliced: return PM_VARIANT_WINDOW_SLICED;
    case Variant::kPatternSliced2: return PM_VARIANT_PATTERN_SLICED_2;
    case Variant::kAllChunks: return PM_VARIANT_ALL_CHUNKS;
    default: return PM_VARIANT_PATTERN_SLICED;
    }
}

// The AUTO table: one variant per k < kAutoK for each device (pm_scan.cu).
constexpr int kAutoK = 64;
constexpr int kMaxAutoDevices = 64;
pm_status set_auto_variants(int device, const Variant *table, uint32_t nk);  // nk = 0: defaults
void get_auto_variants(int device, Variant *table);                          // kAutoK entries

// Fill the run-time constants of a descriptor.
inline void desc_constants(PatDesc &d)
{
    d.two = 2u;
    d.variant = 0u;
    d.c0 = 0u;
}

// The chunk a pattern-sliced scan tests first: Eq. 4's sum does not depend on
// the order of its terms, so the first stage may take any 32 (or, C = 2, 64)
// consecutive positions, and the fewer windows pass it the fewer need
// settling.  Chosen among the full chunks (C consecutive ones) as the one
// with the fewest expected matches under the text's letter frequencies
// (each position contributes the share of the text held by its class's
// letters); chunk 0 unless another one expects at least a tenth of a match
// less.  The settling counts chunks c0 and c0+1 from the staged tile first,
// so the others are read only for the rare windows that survive both.
inline uint32_t first_stage_chunk(const pm_pattern *p, const pm_text *t, int C)
{
    const uint32_t full = p->m / 32;
    if (full < (uint32_t)C + 1) return 0u;
    const double tot = (double)(t->count[0] + t->count[1] + t->count[2] + t->count[3]);
    if (tot <= 0) return 0u;
    double f[4];
    for (int a = 0; a < 4; ++a) f[a] = (double)t->count[a] / tot;
    auto expect = [&](uint32_t c) {
        const uint4 w = p->masks[c];
        return f[0] * __builtin_popcount(w.x) + f[1] * __builtin_popcount(w.y) +
               f[2] * __builtin_popcount(w.z) + f[3] * __builtin_popcount(w.w);
    };
    double best = 0.0, e0 = 0.0;
    uint32_t arg = 0;
    for (uint32_t c = 0; c + (uint32_t)C <= full; ++c) {
        double e = expect(c);
        if (C == 2) e += expect(c + 1);
        if (c == 0) e0 = best = e;
        else if (e < best) {
            best = e;
            arg = c;
        }
    }
    return best <= e0 - 0.1 ? arg : 0u;
}

// A (pattern, tile) segment of hits left by the batched scan: key =
// pattern * ntiles + tile, the hits in window order at tmp[src .. src+count).
struct SegRecord {
    unsigned long long key;
    uint32_t src;
    uint32_t count;
};

// Radix sort of segment records by key (pm_sort.cu).  The live count is
// *n_dev (at most n_max); key_bits bounds the keys.  *sorted receives the
// buffer that holds the result (recs or the scratch copy).
size_t sort_scratch_bytes(uint64_t n_max);
cudaError_t launch_sort_records(SegRecord *recs, uint64_t n_max, const unsigned long long *n_dev,
                                int key_bits, void *scratch, cudaStream_t stream,
                                SegRecord **sorted);
cudaError_t launch_records_to_entries(const SegRecord *recs, uint64_t n_max,
                                      const unsigned long long *n_dev, TileEntry *entries,
                                      cudaStream_t stream);

// Ordering: exclusive scan of table counts, per-pattern CSR offsets, and the
// gather of hits into their final places (pm_order.cu).  Needs
// order_scratch_bytes(entries) bytes of scratch.
size_t order_scratch_bytes(uint64_t entries);
cudaError_t launch_order(const TileEntry *table, uint64_t entries, const uint64_t *pat_tile0,
                         uint32_t npat, const pm_hit *tmp, pm_hit *hits, uint64_t cap,
                         uint64_t *offsets, const uint32_t *status, void *scratch,
                         cudaStream_t stream);

// The same for segment records already sorted by (pattern, tile), whose
// number lives in device memory (*n_dev, at most n_max): CSR offsets from
// per-pattern counts, hits gathered unless hits_found exceeds cap.
cudaError_t launch_order_records(const TileEntry *entries, uint64_t n_max,
                                 const unsigned long long *n_dev,
                                 const unsigned long long *pat_counts, uint32_t npat,
                                 const unsigned long long *hits_found, const pm_hit *tmp,
                                 pm_hit *hits, uint64_t cap, uint64_t *offsets,
                                 const uint32_t *status, void *scratch, cudaStream_t stream);

// Text coding kernel (pm_text.cu).
cudaError_t launch_pack(const char *ascii, uint64_t n_chunk, uint64_t first_symbol,
                        uint2 *planes, uint32_t *unk, unsigned long long *bad, cudaStream_t stream);

// Thread-local detailed error message.
void set_error(const char *fmt, ...);
pm_status cuda_status(cudaError_t e, const char *what);

// Classify a pointer: true if the device can use it in place.
bool is_device_pointer(const void *p);

}  // namespace pm

// ---------------------------------------------------------------- device ----
#ifdef __CUDACC__
namespace pm {
namespace dev {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete, giving up after
// limit_ns nanoseconds of wall time.  Returns false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}

// Bitwise select: bits of a where c is 1, bits of b where c is 0.
__device__ __forceinline__ uint32_t sel(uint32_t c, uint32_t a, uint32_t b)
{
    return (c & a) | (~c & b);
}

// Table 3 evaluated on 32 (pattern position, text symbol) pairs at once.
// (lo, hi) are the text code bits, M the membership masks {A, C, G, T} of
// the 32 positions; returns 1 where the pair matches (L = 0).
__device__ __forceinline__ uint32_t class_match(uint32_t lo, uint32_t hi, uint4 M)
{
    return sel(hi, sel(lo, M.w, M.z), sel(lo, M.y, M.x));
}

}  // namespace dev
}  // namespace pm
#endif
