// Scan kernels: Eq. 4 with the early stop of Sec. 2.4-2.5 over warp tiles of
// the text (Sec. 2.6).
//
// Work unit: a warp tile of kGroups x 32 consecutive 32-symbol blocks.  Lane l
// owns the 32 windows that start in block 32g + l of the tile, for each group
// g.  Windows need at most m-1 symbols beyond their tile (the overlap of
// Sec. 2.6): the tile and a 2-block halo arrive in shared memory by one bulk
// (TMA) copy, issued by the warp itself two tiles ahead into a two-stage
// ring with one mbarrier per stage; deeper blocks, read only by the rare
// windows still alive after 32 positions, come through L1/L2.  Warps never
// wait for each other: each persistent warp walks its own tiles, and a
// tile's hits are emitted by a warp-aggregated atomic.
//
// The first 32 positions are evaluated in one of two ways.
//
//  * pattern-sliced (any k): per window, one 32-bit word holds the text
//    symbols under positions 0..31 (two funnel shifts of the bit planes);
//    three bitwise selects apply Table 3 to all 32 pairs; __popc counts the
//    matches g.  Four windows' g are packed into the bytes of one word by
//    multiply-adds (FMA pipe) together with k in every byte; bit 5 of a byte
//    is then set exactly when g + k >= 32, i.e. when the window has at most
//    k mismatches, and two ALU steps move those four bits into the lane's
//    pass mask (in a transposed bit order, undone only when a window passes).
//  * window-sliced (k <= 6): per pattern position j, one word holds the 32
//    windows' symbols at offset j; a one-letter class gives the mismatch word
//    in two XOR/OR steps, other classes in three selects, N in none; a
//    thermometer counter of k+1 words (level i set once a window has more
//    than i mismatches) adds 32 windows' mismatches at once.  The positions
//    come from a list built by pm_compile_pattern; each list entry read
//    from shared memory serves all groups, and the warp stops as soon as
//    every window of the tile is past k (the early stop of Sec. 2.4).
//
// Windows still at or below k after those 32 positions are counted again one
// at a time, 32 positions per step, from position 0 until their sum exceeds k
// or the pattern ends; that count is exact and is what a hit reports.
#include "pm_internal.cuh"

namespace pm {
namespace {

using dev::class_match;

constexpr uint32_t kFull = 0xffffffffu;
constexpr int G = kGroups;

// Mismatch count of window 32*blk + w over chunks c0.., starting from
// `count`, stopping once it exceeds `limit` (then some value > limit).
__device__ __forceinline__ uint32_t window_count_from(const uint2 *__restrict__ planes,
                                                      uint64_t blk, uint32_t w,
                                                      const uint4 *__restrict__ M,
                                                      uint32_t c0, uint32_t nchunks,
                                                      uint32_t count, uint32_t limit)
{
    uint2 a = __ldg(planes + blk + c0);
    for (uint32_t c = c0; c < nchunks; ++c) {
        const uint2 b = __ldg(planes + blk + c + 1);
        const uint32_t lo = __funnelshift_r(a.x, b.x, w);
        const uint32_t hi = __funnelshift_r(a.y, b.y, w);
        count += __popc(~class_match(lo, hi, __ldg(M + c)));
        if (count > limit) break;
        a = b;
    }
    return count;
}

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// The pass masks below use a transposed bit order: window 4j + b of the lane
// sits at bit 8b + j.  This restores the natural order (window w at bit w).
__device__ __forceinline__ uint32_t untranspose(uint32_t t)
{
    uint32_t r = 0;
    while (t) {
        const uint32_t p = __ffs(t) - 1;
        t &= t - 1;
        r |= 1u << (4 * (p & 7) + (p >> 3));
    }
    return r;
}

// Pattern-sliced first chunk for one lane's 32 windows; transposed pass mask
// of the windows with at most k mismatches in positions 0..31 (k <= 31).
// k4 = k in every byte; one, m8, m16, m24 = 1, 2^8, 2^16, 2^24.
__device__ __forceinline__ uint32_t pass_pattern_sliced(uint2 a, uint2 b, uint4 M0, uint32_t k4,
                                                        uint32_t one, uint32_t m8, uint32_t m16,
                                                        uint32_t m24)
{
    uint32_t pass = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int w = 4 * j + q;
            const uint32_t lo = __funnelshift_r(a.x, b.x, w);
            const uint32_t hi = __funnelshift_r(a.y, b.y, w);
            g[q] = __popc(class_match(lo, hi, M0));
        }
        uint32_t v = mad_lo(g[3], m24, k4);
        v = mad_lo(g[2], m16, v);
        v = mad_lo(g[1], m8, v);
        v = mad_lo(g[0], one, v);
        // bit 5 of byte q: g[q] + k >= 32; move bits 5, 13, 21, 29 to 8q + j
        const uint32_t s = j <= 5 ? v >> (5 - j) : v << (j - 5);
        pass |= s & (0x01010101u << j);
    }
    return pass;
}

// Window-sliced first chunk with a thermometer counter of K+1 levels over the
// listed positions, for all groups of the lane at once.  alive[g] receives
// the windows still at or below K.
template <int K>
__device__ __forceinline__ void alive_window_sliced(const uint2 (&a)[G], const uint2 (&b)[G],
                                                    const uint4 *__restrict__ list,
                                                    uint32_t n_single, uint32_t n_general,
                                                    const uint32_t (&valid)[G],
                                                    uint32_t (&alive)[G])
{
    uint32_t L[G][K + 1];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int i = 0; i <= K; ++i) L[g][i] = ~valid[g];  // invalid windows sit at every level
    auto dead_all = [&]() {
        uint32_t d = kFull;
#pragma unroll
        for (int g = 0; g < G; ++g) d &= L[g][K];
        return !__any_sync(kFull, ~d);
    };
    auto add = [&](int g, uint32_t mis) {
#pragma unroll
        for (int i = K; i >= 1; --i) L[g][i] |= L[g][i - 1] & mis;
        L[g][0] |= mis;
    };
    uint32_t e = 0;
    for (; e + 4 <= n_single; e += 4) {
        uint4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = list[e + u];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            uint32_t mis[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t lo = __funnelshift_r(a[g].x, b[g].x, q[u].x);
                const uint32_t hi = __funnelshift_r(a[g].y, b[g].y, q[u].x);
                mis[u] = (lo ^ q[u].y) | (hi ^ q[u].z);
            }
            if constexpr (K == 0) {
                L[g][0] |= (mis[0] | mis[1]) | (mis[2] | mis[3]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) add(g, mis[u]);
            }
        }
        if (dead_all()) {
#pragma unroll
            for (int g = 0; g < G; ++g) alive[g] = 0u;
            return;
        }
    }
    for (; e < n_single; ++e) {
        const uint4 q = list[e];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t lo = __funnelshift_r(a[g].x, b[g].x, q.x);
            const uint32_t hi = __funnelshift_r(a[g].y, b[g].y, q.x);
            add(g, (lo ^ q.y) | (hi ^ q.z));
        }
    }
    for (uint32_t c = 0; c < n_general; ++c) {
        const uint32_t s = list[n_single + 2 * c].x;
        const uint4 M = list[n_single + 2 * c + 1];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t lo = __funnelshift_r(a[g].x, b[g].x, s);
            const uint32_t hi = __funnelshift_r(a[g].y, b[g].y, s);
            add(g, ~class_match(lo, hi, M));
        }
        if ((c & 3) == 3 && dead_all()) {
#pragma unroll
            for (int g = 0; g < G; ++g) alive[g] = 0u;
            return;
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) alive[g] = ~L[g][K];
}

// One warp tile and its halo, global -> shared, completing on bar.
__device__ __forceinline__ void issue_tile(const uint2 *planes, uint64_t tile, uint2 *dst,
                                           uint64_t *bar)
{
    dev::mbar_arrive_expect_tx(bar, kStageBytes);
    dev::bulk_g2s(dst, planes + tile * (32ull * G), kStageBytes, bar);
}

// VARIANT: -1 pattern-sliced; K in 0..kWsMaxK window-sliced with threshold K.
template <int VARIANT>
__global__ void __launch_bounds__(kScanThreads, 4)
    k_scan(const uint2 *__restrict__ planes, const PatDesc d, const uint4 *__restrict__ arena,
           TileEntry *__restrict__ table, pm_hit *__restrict__ tmp, uint64_t cap,
           unsigned long long *__restrict__ cursor, uint32_t *__restrict__ status)
{
    constexpr bool kWS = VARIANT >= 0;
    constexpr int K = kWS ? VARIANT : 0;

    __shared__ __align__(128) uint2 sbuf[kScanWarps][2][kStageBlocks];
    __shared__ __align__(8) uint64_t sbar[kScanWarps][2];
    __shared__ uint4 slist[kWS ? 64 : 1];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t k = (uint32_t)d.k;
    const uint4 *__restrict__ M = arena + d.masks;
    const uint4 M0 = __ldg(M);
    // run-time constants for the multiply-adds of the pattern-sliced test
    const uint32_t one = d.two >> 1, m8 = one << 8, m16 = one << 16, m24 = one << 24;
    const uint32_t k4 = (k < 32u ? k : 0u) * (m24 | m16 | m8 | one);

    if (kWS) {
        const uint32_t len = d.n_single + 2 * d.n_general;
        for (uint32_t i = threadIdx.x; i < len; i += kScanThreads) slist[i] = __ldg(arena + d.wslist + i);
        __syncthreads();  // the only CTA-wide barrier: the list is shared by all warps
    }
    if (lane == 0) {
        dev::mbar_init(&sbar[warp][0], 1);
        dev::mbar_init(&sbar[warp][1], 1);
        dev::fence_mbar_init();
    }
    __syncwarp();

    const uint64_t stride = (uint64_t)gridDim.x * kScanWarps;
    const uint64_t first = (uint64_t)blockIdx.x * kScanWarps + warp;
    if (lane == 0) {
        if (first < d.ntiles) issue_tile(planes, first, &sbuf[warp][0][0], &sbar[warp][0]);
        if (first + stride < d.ntiles)
            issue_tile(planes, first + stride, &sbuf[warp][1][0], &sbar[warp][1]);
    }

    uint32_t it = 0;
    for (uint64_t tile = first; tile < d.ntiles; tile += stride, ++it) {
        const int s = it & 1;
        const bool ok = dev::mbar_wait_bounded(&sbar[warp][s], (it >> 1) & 1u, kWaitLimitNs);
        if (__any_sync(kFull, !ok)) {
            if (lane == 0) {
                atomicOr(status, kDevTimeout);
                // let the copies this warp still has in flight land before it leaves
                dev::mbar_wait_bounded(&sbar[warp][s], (it >> 1) & 1u, kWaitLimitNs);
                if (tile + stride < d.ntiles)
                    dev::mbar_wait_bounded(&sbar[warp][s ^ 1], ((it + 1) >> 1) & 1u, kWaitLimitNs);
            }
            return;
        }
        uint2 a[G], b[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            a[g] = sbuf[warp][s][32 * g + lane];
            b[g] = sbuf[warp][s][32 * g + lane + 1];
        }
        __syncwarp();
        if (lane == 0 && tile + 2 * stride < d.ntiles) {
            dev::fence_proxy_async_smem();
            issue_tile(planes, tile + 2 * stride, &sbuf[warp][s][0], &sbar[warp][s]);
        }

        uint64_t blk[G];
        uint32_t valid[G], pass[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            blk[g] = tile * (32ull * G) + 32ull * g + (uint64_t)lane;  // windows start at 32*blk
            const uint64_t w0 = blk[g] * 32ull;
            valid[g] = w0 >= d.nwin ? 0u
                       : (d.nwin - w0 >= 32 ? kFull : (1u << (uint32_t)(d.nwin - w0)) - 1u);
        }
        if constexpr (kWS) {
            alive_window_sliced<K>(a, b, slist, d.n_single, d.n_general, valid, pass);
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                uint32_t t = 0u;
                if (k > 31u) t = valid[g];
                else if (valid[g]) t = untranspose(pass_pattern_sliced(a[g], b[g], M0, k4, one, m8,
                                                                       m16, m24)) & valid[g];
                pass[g] = t;
            }
        }
        // Both evaluations are exact for m <= 32.  Longer patterns: count every
        // remaining window exactly and drop those past k.
        if (d.nchunks > 1) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                uint32_t sv = pass[g];
                while (sv) {
                    const uint32_t w = __ffs(sv) - 1;
                    sv &= sv - 1;
                    if (window_count_from(planes, blk[g], w, M, 0, d.nchunks, 0u, k) > k)
                        pass[g] &= ~(1u << w);
                }
            }
        }

        // ---- hits of this warp tile, in window order (warp-aggregated atomic) ----
        uint32_t anyp = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) anyp |= pass[g];
        if (__any_sync(kFull, anyp != 0u)) {
            uint32_t incl[G], tot[G];
            uint32_t total = 0;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const uint32_t nh = __popc(pass[g]);
                incl[g] = nh;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(kFull, incl[g], o);
                    if (lane >= o) incl[g] += v;
                }
                tot[g] = __shfl_sync(kFull, incl[g], 31);
                total += tot[g];
            }
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(cursor, (unsigned long long)total);
                table[d.tile0 + tile] = TileEntry{total, (uint32_t)base};
            }
            base = __shfl_sync(kFull, base, 0);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                unsigned long long q = base + incl[g] - __popc(pass[g]);
                uint32_t hm = pass[g];
                while (hm) {
                    const uint32_t w = __ffs(hm) - 1;
                    hm &= hm - 1;
                    if (q < cap) {
                        const uint32_t c = window_count_from(planes, blk[g], w, M, 0, d.nchunks, 0u, k);
                        tmp[q] = pm_hit{(uint32_t)(blk[g] * 32ull + w), c};
                    }
                    ++q;
                }
                base += tot[g];
            }
        } else if (lane == 0) {
            table[d.tile0 + tile] = TileEntry{0u, 0u};
        }
    }
}

template <int VARIANT>
const void *kernel_ptr()
{
    return (const void *)&k_scan<VARIANT>;
}

const void *select_kernel(Variant v, int32_t k)
{
    if (v == Variant::kWindowSliced && k >= 0 && k <= kWsMaxK) {
        switch (k) {
        case 0: return kernel_ptr<0>();
        case 1: return kernel_ptr<1>();
        case 2: return kernel_ptr<2>();
        case 3: return kernel_ptr<3>();
        case 4: return kernel_ptr<4>();
        case 5: return kernel_ptr<5>();
        case 6: return kernel_ptr<6>();
        default: break;
        }
    }
    return kernel_ptr<-1>();
}

}  // namespace

Variant auto_variant(const PatDesc &d)
{
    // window-sliced wins while few positions decide a window (small k)
    return d.k <= 4 ? Variant::kWindowSliced : Variant::kPatternSliced;
}

int scan_grid_limit(Variant v, int32_t k, int device)
{
    static int cache[64][kWsMaxK + 2] = {};
    if (device < 0 || device >= 64) return 0;
    const int slot = (v == Variant::kWindowSliced && k >= 0 && k <= kWsMaxK) ? k : kWsMaxK + 1;
    if (cache[device][slot]) return cache[device][slot];
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel(v, k), kScanThreads, 0);
    if (per_sm < 1) per_sm = 1;
    cache[device][slot] = sms * per_sm;
    return cache[device][slot];
}

cudaError_t launch_scan(Variant v, const uint2 *planes, const PatDesc &d, const uint4 *arena,
                        TileEntry *table, pm_hit *tmp, uint64_t cap, unsigned long long *cursor,
                        uint32_t *status, int grid, cudaStream_t stream)
{
    if (d.ntiles == 0) return cudaSuccess;
    const uint64_t ctas_needed = (d.ntiles + kScanWarps - 1) / kScanWarps;
    if ((uint64_t)grid > ctas_needed) grid = (int)ctas_needed;
    if (grid < 1) grid = 1;
    const void *fn = select_kernel(v, d.k);
    PatDesc dd = d;
    void *args[] = {(void *)&planes, (void *)&dd, (void *)&arena, (void *)&table,
                    (void *)&tmp,    (void *)&cap, (void *)&cursor, (void *)&status};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kScanThreads), args, 0, stream);
}

}  // namespace pm
