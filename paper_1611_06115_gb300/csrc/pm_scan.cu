// Scan kernels: Eq. 4 with the early stop of Sec. 2.4-2.5 over warp tiles of
// the text (Sec. 2.6).
//
// Work unit: a warp tile of kGroups x 32 consecutive 32-symbol blocks.  Lane l
// owns the 32 windows that start in block 32g + l of the tile, for each group
// g.  Windows need at most m-1 symbols beyond their tile (the overlap of
// Sec. 2.6): the tile and a 2-block halo arrive in shared memory by 16-byte
// asynchronous copies (cp.async) that the warp's lanes issue kStages tiles
// ahead into a ring of stages; deeper blocks, read only by the rare windows
// still alive after 64 positions, come through L1/L2.  (One bulk copy per
// warp tile, the tile's 1040 bytes through the TMA unit, streamed the text
// at 2.7 TB/s on GB300 whatever the depth of the ring; the lanes' own copies
// stream it at 5.7 TB/s.)  Warps never wait for each other: each persistent
// warp walks its own tiles, and a tile's hits are emitted by a
// warp-aggregated atomic.
//
// Four evaluations, all exact, chosen per k (a measured table per device):
//
//  * pattern-sliced over 32 positions (k <= 31): per window, one 32-bit word
//    holds the text symbols under positions 0..31 (two funnel shifts of the
//    bit planes); three bitwise selects apply Table 3 to all 32 pairs;
//    __popc counts the matches g.  Four windows' g are packed into the bytes
//    of one word by multiply-adds (FMA pipe) together with k in every byte;
//    bit 5 of a byte is then set exactly when g + k >= 32, i.e. when the
//    window has at most k mismatches, and two ALU steps move those four bits
//    into the lane's pass mask (the word packs windows j, 8+j, 16+j, 24+j,
//    so each bit lands on its window's own position).  Windows that pass
//    with m > 32 are settled.  The first stage may test any full chunk of
//    the pattern (Eq. 4's sum does not depend on the order of its terms):
//    the host picks the one with the fewest expected matches for the text.
//  * pattern-sliced over 64 positions (k <= 63): the same byte test over two
//    chunks (bit 6), then the same settling.
//  * every chunk (any k): 32 running counts per lane, chunk after chunk,
//    until every window of the warp is past k.
//  * window-sliced (k <= 8): per pattern position j, one word holds the 32
//    windows' symbols at offset j.  The positions come from a list built by
//    pm_compile_pattern and ordered for the text (rarest letters first,
//    one-letter positions grouped into runs by letter); for a run the
//    letter's plane (bit set where the text holds that letter) is built once
//    from the lane's blocks, so a position's match word for 32 windows is one
//    funnel shift; other classes take three selects.  Mismatches are counted
//    for 32 windows at once, by a thermometer of k+1 words (k <= 3: level i
//    set once a window has more than i mismatches) or by six bit-sliced
//    binary counter words that take four positions per carry-save step (k >=
//    4, k <= 8).  The warp stops once every window of its tile is past k (k = 0, the
//    early stop of Sec. 2.4; for larger k a 4096-window tile practically
//    never dies whole that early) or after a fixed number of list entries;
//    the windows still alive are then counted exactly.
//
// Windows that need exact counts (survivors of a first stage, and every hit)
// are settled by the whole warp together from a queue in shared memory, and
// a tile's hits are written once, in window order, behind one atomic.
//
// A hit's count is always exact (recounted over every position when the
// evaluation stopped early for it).
#include <cstring>
#include <mutex>

#include "pm_scan_impl.cuh"

namespace pm {
namespace {

using namespace scan;

// VARIANT: -1 pattern-sliced over positions 0..31 (k <= 31), -3 over
// positions 0..63 (k <= 63), -2 pattern-sliced over all chunks (any k); K in
// 0..kWsMaxK window-sliced with threshold K, a thermometer counter of K+1
// words per group below kWsBinaryFrom, five binary counter words from there
// on.  The -2
// kernel keeps 32 running counts per lane in registers, so it takes twice
// the registers at half the resident warps.  The window-sliced kernels run
// eight groups per lane (tiles of 8192 windows, scan_groups): three CTAs per
// SM for K <= 2, two from K = 3 on (the counters of eight groups take up to
// 128 registers).
//
// Each warp stages its tiles kStages strides ahead, one commit group of
// asynchronous copies per tile (an empty group once the tiles run out, so
// that group i always belongs to the warp's i-th tile); a stage is refilled
// once its tile is done (settling and hit counts read the staged tile).
// Tile indices fit in 32 bits: a text has fewer than 2^32 symbols.
template <int VARIANT, int G>
__global__ void __launch_bounds__(kScanThreads, VARIANT == -2 || (G == 8 && VARIANT >= 3) ? 2 : (G == 8 ? 3 : 4))
    k_scan(const uint2 *__restrict__ planes, const PatDesc d, const uint4 *__restrict__ arena,
           TileEntry *__restrict__ table, pm_hit *__restrict__ tmp, uint64_t cap,
           unsigned long long *__restrict__ cursor, uint32_t *__restrict__ status,
           const uint32_t *__restrict__ unk)
{
    constexpr bool kWS = VARIANT >= 0;
    constexpr uint32_t S = kStages;

    __shared__ __align__(128) uint2 sbuf[kScanWarps][S][scan_stage_blocks<G>()];
    __shared__ uint32_t slist[kWS ? 32 : 1];
    __shared__ uint32_t squeue[kScanWarps][kQueueCap];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint4 *__restrict__ M = arena + d.masks;
    const uint4 M0 = __ldg(M + d.c0);
    // stages start at the even block at or below block tile*32G + c0 (16-byte copies)
    const uint32_t c0e = d.c0 & ~1u, sh = d.c0 & 1u;
    const PsConst pc = ps_const(d.two, (uint32_t)d.k);

    if (kWS) {
        const uint32_t len = d.n_single + d.n_general;  // at most 32 words
        const uint32_t *wl = (const uint32_t *)(arena + d.wslist);
        for (uint32_t i = threadIdx.x; i < len; i += kScanThreads) slist[i] = __ldg(wl + i);
        __syncthreads();  // the only CTA-wide barrier: the list is shared by all warps
    }
    const uint32_t ntiles = (uint32_t)d.ntiles;
    const uint32_t nfull = (uint32_t)(d.nwin / (1024u * G));  // tiles whose windows are all valid
    const uint32_t stride = gridDim.x * kScanWarps;
    const uint32_t first = blockIdx.x * kScanWarps + warp;
#pragma unroll
    for (uint32_t st = 0; st < S; ++st) {
        if (first + st * stride < ntiles)
            copy_tile_async<G>(planes, (uint64_t)(first + st * stride) * (32u * G) + c0e, &sbuf[warp][st][0],
                               lane);
        cp_async_commit();
    }

    uint32_t s = 0;
    for (uint32_t tile = first; tile < ntiles; tile += stride) {
        cp_async_wait<S - 1>();  // this tile's group has landed (later ones may be pending)
        __syncwarp();            // ... for every lane's pieces
        const uint2 *stage = &sbuf[warp][s][sh];  // block tile*32G + c0
        uint2 a[G], b[G];
        uint32_t valid[G], pass[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            a[g] = stage[32 * g + lane];
            b[g] = stage[32 * g + lane + 1];
        }
        if (tile < nfull) {
#pragma unroll
            for (int g = 0; g < G; ++g) valid[g] = kFull;
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g) valid[g] = valid_mask((uint64_t)tile * (32u * G) + 32u * g + lane, d.nwin);
        }
        const bool need = tile_first_stage<VARIANT, G>(a, b, tile, valid, d, M, M0, slist, pc, planes, stage, pass);

        // ---- exact counts and hits of this warp tile, in window order ----
        uint32_t anyp = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) anyp |= pass[g];
        TileEntry *entry = table + d.tile0 + tile;
        if (__any_sync(kFull, anyp != 0u)) {
            if (!settle_emit_queued<G>(pass, tile, stage, squeue[warp], d, M, planes, unk, tmp, cap, cursor,
                                       entry)) {
                // more candidates than the queue holds (dense hits): each lane its own
                uint64_t blk[G];
#pragma unroll
                for (int g = 0; g < G; ++g) blk[g] = (uint64_t)tile * (32u * G) + 32u * g + lane;
                settle_dense<VARIANT, G>(need, a, b, blk, d, M, planes, stage, pass);
                anyp = 0;
#pragma unroll
                for (int g = 0; g < G; ++g) anyp |= pass[g];
                if (__any_sync(kFull, anyp != 0u)) {
                    uint32_t total;
                    unsigned long long base;
                    emit_tile_hits<true, G>(pass, blk, a, b, stage, d, M, planes, unk, tmp, cap, cursor, total,
                                            base);
                    if (lane == 0) *entry = TileEntry{total, (uint32_t)base};
                } else if (lane == 0) {
                    *entry = TileEntry{0u, 0u};
                }
            }
        } else if (lane == 0) {
            *entry = TileEntry{0u, 0u};
        }
        // refill this stage with the tile S strides ahead
        __syncwarp();  // every lane is done reading the stage
        if (tile + S * stride < ntiles)
            copy_tile_async<G>(planes, (uint64_t)(tile + S * stride) * (32u * G) + c0e, &sbuf[warp][s][0], lane);
        cp_async_commit();
        if (++s == S) s = 0;
    }
    cp_async_wait<0>();  // nothing in flight when the warp leaves
}

template <int VARIANT, int G>
const void *kernel_ptr()
{
    return (const void *)&k_scan<VARIANT, G>;
}

// v already resolved for k; the tile width as scan_groups(v, k)
const void *select_kernel(Variant v, int32_t k)
{
    switch (v) {
    case Variant::kWindowSliced:
        switch (k) {
        case 0: return kernel_ptr<0, 8>();
        case 1: return kernel_ptr<1, 8>();
        case 2: return kernel_ptr<2, 8>();
        case 3: return kernel_ptr<3, 8>();
        case 4: return kernel_ptr<4, 8>();
        case 5: return kernel_ptr<5, 8>();
        case 6: return kernel_ptr<6, 8>();
        case 7: return kernel_ptr<7, 8>();
        default: return kernel_ptr<8, 8>();
        }
    case Variant::kPatternSliced: return kernel_ptr<-1, 4>();
    case Variant::kPatternSliced2: return kernel_ptr<-3, 4>();
    default: return kernel_ptr<-2, 4>();
    }
}

// Per device, the variant PM_VARIANT_AUTO uses for k < kAutoK (-1: the
// built-in choice); larger k always run kAllChunks.
std::mutex g_auto_mu;
int8_t g_auto[kMaxAutoDevices][kAutoK];
bool g_auto_init = false;

Variant default_variant(int32_t k)
{
    // measured on GB300 over a 3.1 Gbp text (m = 128 .. 10^4): the
    // window-sliced counter wins while few positions decide a window, one
    // pattern-sliced chunk while the windows that survive it are rare, two
    // chunks while those surviving 64 positions are rare
    if (k <= 8) return Variant::kWindowSliced;
    if (k <= 17) return Variant::kPatternSliced;
    if (k <= 40) return Variant::kPatternSliced2;
    return Variant::kAllChunks;
}

}  // namespace

Variant resolve_variant(Variant v, int32_t k)
{
    switch (v) {
    case Variant::kWindowSliced:
        return k >= 0 && k <= kWsMaxK ? v : resolve_variant(Variant::kPatternSliced, k);
    case Variant::kPatternSliced: return k <= 31 ? v : Variant::kAllChunks;
    case Variant::kPatternSliced2: return k <= 63 ? v : Variant::kAllChunks;
    default: return Variant::kAllChunks;
    }
}

Variant auto_variant(const PatDesc &d, int device)
{
    if (d.k < 0 || d.k >= kAutoK) return Variant::kAllChunks;
    int v = -1;
    if (device >= 0 && device < kMaxAutoDevices) {
        std::lock_guard<std::mutex> lk(g_auto_mu);
        if (g_auto_init) v = g_auto[device][d.k];
    }
    Variant r = resolve_variant(v < 0 ? default_variant(d.k) : (Variant)v, d.k);
    // a pattern of one chunk is decided exactly by its first 32 positions
    if (r == Variant::kPatternSliced2 && d.nchunks == 1 && d.k <= 31) r = Variant::kPatternSliced;
    return r;
}

pm_status set_auto_variants(int device, const Variant *table, uint32_t nk)
{
    if (device < 0 || device >= kMaxAutoDevices) return PM_E_ARG;
    std::lock_guard<std::mutex> lk(g_auto_mu);
    if (!g_auto_init) {
        std::memset(g_auto, -1, sizeof(g_auto));
        g_auto_init = true;
    }
    for (int k = 0; k < kAutoK; ++k)
        g_auto[device][k] = (uint32_t)k < nk ? (int8_t)table[k] : (int8_t)-1;
    return PM_OK;
}

void get_auto_variants(int device, Variant *table)
{
    for (int k = 0; k < kAutoK; ++k) {
        PatDesc d{};
        d.k = k;
        table[k] = auto_variant(d, device);
    }
}

int scan_grid_limit(Variant v, int32_t k, int device)
{
    static std::atomic<int> cache[64][kWsMaxK + 4];  // 0 = not yet computed
    if (device < 0 || device >= 64) return 0;
    v = resolve_variant(v, k);
    const int slot = v == Variant::kWindowSliced     ? k
                     : v == Variant::kPatternSliced  ? kWsMaxK + 1
                     : v == Variant::kPatternSliced2 ? kWsMaxK + 2
                                                     : kWsMaxK + 3;
    if (const int g = cache[device][slot].load(std::memory_order_relaxed)) return g;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel(v, k), kScanThreads, 0);
    if (per_sm < 1) per_sm = 1;
    cache[device][slot].store(sms * per_sm, std::memory_order_relaxed);
    return sms * per_sm;
}

cudaError_t launch_scan(Variant v, const uint2 *planes, const uint32_t *unk, const PatDesc &d,
                        const uint4 *arena, TileEntry *table, pm_hit *tmp, uint64_t cap,
                        unsigned long long *cursor, uint32_t *status, int grid, cudaStream_t stream)
{
    if (d.ntiles == 0) return cudaSuccess;
    const uint64_t ctas_needed = (d.ntiles + kScanWarps - 1) / kScanWarps;
    if ((uint64_t)grid > ctas_needed) grid = (int)ctas_needed;
    if (grid < 1) grid = 1;
    const void *fn = select_kernel(resolve_variant(v, d.k), d.k);
    PatDesc dd = d;
    void *args[] = {(void *)&planes, (void *)&dd,     (void *)&arena,  (void *)&table, (void *)&tmp,
                    (void *)&cap,    (void *)&cursor, (void *)&status, (void *)&unk};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kScanThreads), args, 0, stream);
}

}  // namespace pm

extern "C" {

pm_status pm_set_auto_variants(const int32_t *variant_for_k, uint32_t nk)
{
    if (nk > (uint32_t)pm::kAutoK || (nk > 0 && !variant_for_k)) {
        pm::set_error("pm_set_auto_variants: nk = %u (0..%d) or NULL table", nk, pm::kAutoK);
        return PM_E_ARG;
    }
    pm::Variant t[pm::kAutoK];
    for (uint32_t k = 0; k < nk; ++k) {
        const int32_t v = variant_for_k[k];
        if (v < PM_VARIANT_PATTERN_SLICED || v > PM_VARIANT_ALL_CHUNKS ||
            pm::resolve_variant(pm::variant_from_public(v), (int32_t)k) != pm::variant_from_public(v)) {
            pm::set_error("pm_set_auto_variants: variant %d is not valid for k = %u", v, k);
            return PM_E_ARG;
        }
        t[k] = pm::variant_from_public(v);
    }
    int dev = 0;
    pm_status rc = pm::cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    return pm::set_auto_variants(dev, t, nk);
}

pm_status pm_get_auto_variants(int32_t *out, uint32_t nk)
{
    if (nk > (uint32_t)pm::kAutoK || (nk > 0 && !out)) {
        pm::set_error("pm_get_auto_variants: nk = %u (0..%d) or NULL output", nk, pm::kAutoK);
        return PM_E_ARG;
    }
    int dev = 0;
    pm_status rc = pm::cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    pm::Variant t[pm::kAutoK];
    pm::get_auto_variants(dev, t);
    for (uint32_t k = 0; k < nk; ++k) out[k] = pm::variant_to_public(t[k]);
    return PM_OK;
}

}  // extern "C"
