// Scan kernels: Eq. 4 with the early stop of Sec. 2.4-2.5 over one tile of
// the text after another (Sec. 2.6).
//
// A tile is kTileBlocks consecutive 32-symbol blocks; thread t of the CTA
// owns the 32 windows that start in block t of the tile.  Every window of a
// tile needs at most m-1 symbols beyond it (the overlap of Sec. 2.6): the
// first two blocks (tile + one halo block) come from shared memory, filled by
// a bulk (TMA) copy that runs one tile ahead; deeper blocks, which only the
// rare windows still alive after 32 positions read, come through L1/L2.
//
// Two ways to evaluate the sum for the first 32 positions:
//
//  * pattern-sliced: for each window, one 32-bit word holds the 32 text
//    symbols under the first 32 pattern positions (two funnel shifts of the
//    bit planes), Table 3 is applied to all 32 pairs with three bitwise
//    selects, and __popc gives the mismatch count;
//  * window-sliced: for each pattern position j, one word holds the 32
//    windows' text symbols at offset j, the class test gives a 32-window
//    mismatch word, and a bit-sliced counter adds it to 32 running sums at
//    once.  The counter starts at 2^B - (k+1), so a carry out of its top bit
//    marks the windows whose sum exceeded k; the thread stops as soon as all
//    of its 32 windows are out (early stop of Sec. 2.4).
//
// Windows still at or below k after 32 positions continue one at a time,
// 32 positions per step, stopping once their sum exceeds k.  Hits of a tile
// are written in window order: a CTA-wide prefix sum of per-thread hit
// counts, one atomicAdd per tile to reserve room in the scratch hit buffer,
// and a tile-table entry recording where they went (pm_order.cu puts the
// tiles in order).
#include "pm_internal.cuh"

namespace pm {
namespace {

using dev::class_match;

// Mismatch count of window 32*blk + w from chunk c0 on, starting from
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

// Windows of this thread that pass: bit w for window 32*blk + w.
// Pattern-sliced evaluation of the first chunk.
__device__ __forceinline__ uint32_t survivors_pattern_sliced(uint2 a, uint2 b, uint4 M0, uint32_t k)
{
    uint32_t pass = 0;
#pragma unroll
    for (int w = 0; w < 32; ++w) {
        const uint32_t lo = __funnelshift_r(a.x, b.x, w);
        const uint32_t hi = __funnelshift_r(a.y, b.y, w);
        const uint32_t c = __popc(~class_match(lo, hi, M0));
        pass |= (c <= k ? 1u : 0u) << w;
    }
    return pass;
}

// Window-sliced evaluation of the first chunk with a B-bit counter.
// P[j] holds position j's membership masks broadcast to whole words.
// Returns the windows still at or below k; cnt receives the counter planes.
template <int B>
__device__ __forceinline__ uint32_t survivors_window_sliced(uint2 a, uint2 b,
                                                            const uint4 *__restrict__ P,
                                                            uint32_t k, uint32_t dead,
                                                            uint32_t (&cnt)[B > 0 ? B : 1])
{
    const uint32_t v0 = (1u << B) - (k + 1u);  // B == 0 only for k == 0
#pragma unroll
    for (int i = 0; i < B; ++i) cnt[i] = ((v0 >> i) & 1u) ? 0xffffffffu : 0u;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint4 Pj = P[j];
        const uint32_t lo = __funnelshift_r(a.x, b.x, j);
        const uint32_t hi = __funnelshift_r(a.y, b.y, j);
        uint32_t carry = ~class_match(lo, hi, Pj);
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const uint32_t t = cnt[i] & carry;
            cnt[i] ^= carry;
            carry = t;
        }
        dead |= carry;
        if ((j & 3) == 3 && dead == 0xffffffffu) break;
    }
    return ~dead;
}

template <int B>
__device__ __forceinline__ uint32_t counter_value(const uint32_t (&cnt)[B > 0 ? B : 1], uint32_t w,
                                                  uint32_t k)
{
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < B; ++i) v |= ((cnt[i] >> w) & 1u) << i;
    return v - ((1u << B) - (k + 1u));
}

// VARIANT: -1 pattern-sliced, B >= 0 window-sliced with a B-bit counter.
template <int VARIANT>
__global__ void __launch_bounds__(kScanThreads)
    k_scan(const uint2 *__restrict__ planes, const PatDesc d, const uint4 *__restrict__ masks,
           TileEntry *__restrict__ table, pm_hit *__restrict__ tmp, uint64_t cap,
           unsigned long long *__restrict__ cursor, uint32_t *__restrict__ status)
{
    constexpr bool kWS = VARIANT >= 0;
    constexpr int B = kWS ? VARIANT : 0;
    constexpr int kWarps = kScanThreads / 32;

    __shared__ __align__(128) uint2 sbuf[2][kTileBlocks + kHaloBlocks];
    __shared__ __align__(8) uint64_t sbar[2];
    __shared__ uint4 spos[kWS ? 32 : 1];
    __shared__ uint32_t swarp[kWarps];
    __shared__ unsigned long long sbase;

    const int tid = threadIdx.x;
    const uint32_t k = (uint32_t)d.k;
    const uint4 *__restrict__ M = masks + d.masks;
    const uint4 M0 = __ldg(M);

    if (tid == 0) {
        dev::mbar_init(&sbar[0], 1);
        dev::mbar_init(&sbar[1], 1);
        dev::fence_mbar_init();
    }
    if (kWS && tid < 32) {
        // position tid's membership bits, broadcast over 32 windows
        spos[tid] = make_uint4(0u - ((M0.x >> tid) & 1u), 0u - ((M0.y >> tid) & 1u),
                               0u - ((M0.z >> tid) & 1u), 0u - ((M0.w >> tid) & 1u));
    }
    __syncthreads();

    uint64_t tile = blockIdx.x;
    if (tid == 0 && tile < d.ntiles) {
        dev::mbar_arrive_expect_tx(&sbar[0], kTileBytes);
        dev::bulk_g2s(&sbuf[0][0], planes + tile * kTileBlocks, kTileBytes, &sbar[0]);
    }

    for (uint32_t it = 0; tile < d.ntiles; ++it, tile += gridDim.x) {
        const uint32_t s = it & 1u;
        const uint64_t next = tile + gridDim.x;
        if (tid == 0 && next < d.ntiles) {
            dev::fence_proxy_async_smem();
            dev::mbar_arrive_expect_tx(&sbar[s ^ 1u], kTileBytes);
            dev::bulk_g2s(&sbuf[s ^ 1u][0], planes + next * kTileBlocks, kTileBytes, &sbar[s ^ 1u]);
        }
        const bool ok = dev::mbar_wait_bounded(&sbar[s], (it >> 1) & 1u, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(status, kDevTimeout);
                // let copies still in flight land before the CTA leaves
                dev::mbar_wait_bounded(&sbar[s], (it >> 1) & 1u, kWaitLimitNs);
                if (next < d.ntiles)
                    dev::mbar_wait_bounded(&sbar[s ^ 1u], ((it + 1) >> 1) & 1u, kWaitLimitNs);
            }
            return;
        }

        const uint64_t blk = tile * kTileBlocks + (uint64_t)tid;  // first window = 32*blk
        const uint64_t w0 = blk * 32ull;
        const uint32_t valid = w0 >= d.nwin ? 0u
                               : (d.nwin - w0 >= 32 ? 0xffffffffu
                                                    : (1u << (uint32_t)(d.nwin - w0)) - 1u);
        const uint2 a = sbuf[s][tid];
        const uint2 b = sbuf[s][tid + 1];

        uint32_t pass;
        if constexpr (kWS) {
            uint32_t cnt[B > 0 ? B : 1];
            pass = valid ? survivors_window_sliced<B>(a, b, spos, k, ~valid, cnt) : 0u;
            if (d.nchunks > 1) {
                uint32_t sv = pass;
                while (sv) {
                    const uint32_t w = __ffs(sv) - 1;
                    sv &= sv - 1;
                    const uint32_t c = window_count_from(planes, blk, w, M, 1, d.nchunks,
                                                         counter_value<B>(cnt, w, k), k);
                    if (c > k) pass &= ~(1u << w);
                }
            }
        } else {
            pass = valid ? survivors_pattern_sliced(a, b, M0, k) & valid : 0u;
            if (d.nchunks > 1) {
                uint32_t sv = pass;
                while (sv) {
                    const uint32_t w = __ffs(sv) - 1;
                    sv &= sv - 1;
                    const uint32_t c0 = __popc(~class_match(__funnelshift_r(a.x, b.x, w),
                                                            __funnelshift_r(a.y, b.y, w), M0));
                    const uint32_t c = window_count_from(planes, blk, w, M, 1, d.nchunks, c0, k);
                    if (c > k) pass &= ~(1u << w);
                }
            }
        }

        // ---- hits of this tile, in window order ----
        if (__syncthreads_or(pass != 0u)) {
            const uint32_t nh = __popc(pass);
            uint32_t incl = nh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if ((tid & 31) >= o) incl += v;
            }
            if ((tid & 31) == 31) swarp[tid >> 5] = incl;
            __syncthreads();
            if (tid == 0) {
                uint32_t run = 0;
                for (int q = 0; q < kWarps; ++q) {
                    const uint32_t t = swarp[q];
                    swarp[q] = run;
                    run += t;
                }
                const unsigned long long base = atomicAdd(cursor, (unsigned long long)run);
                table[d.tile0 + tile] = TileEntry{base, run, 0u};
                sbase = base;
            }
            __syncthreads();
            unsigned long long q = sbase + swarp[tid >> 5] + (incl - nh);
            uint32_t hm = pass;
            while (hm) {
                const uint32_t w = __ffs(hm) - 1;
                hm &= hm - 1;
                if (q < cap) {
                    const uint32_t c = window_count_from(planes, blk, w, M, 0, d.nchunks, 0u, k);
                    tmp[q] = pm_hit{(uint32_t)(w0 + w), c};
                }
                ++q;
            }
        } else if (tid == 0) {
            table[d.tile0 + tile] = TileEntry{0ull, 0u, 0u};
        }
        __syncthreads();  // sbuf[s] and swarp are reused
    }
}

template <int VARIANT>
const void *kernel_ptr()
{
    return (const void *)&k_scan<VARIANT>;
}

const void *select_kernel(Variant v, int32_t k)
{
    if (v == Variant::kWindowSliced) {
        switch (ws_bits(k)) {
        case 0: return kernel_ptr<0>();
        case 1: return kernel_ptr<1>();
        case 2: return kernel_ptr<2>();
        case 3: return kernel_ptr<3>();
        case 4: return kernel_ptr<4>();
        case 5: return kernel_ptr<5>();
        default: break;
        }
    }
    return kernel_ptr<-1>();
}

}  // namespace

int ws_bits(int32_t k)
{
    if (k < 0) return -1;
    int b = 0;
    while ((1ll << b) < (long long)k + 1) ++b;
    return b <= 5 ? b : -1;
}

int scan_grid_limit(Variant v, int device)
{
    static int cache[2][64] = {};
    const int vi = (int)v;
    if (device < 0 || device >= 64) return 0;
    if (cache[vi][device]) return cache[vi][device];
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel(v, 0), kScanThreads, 0);
    if (per_sm < 1) per_sm = 1;
    cache[vi][device] = sms * per_sm;
    return cache[vi][device];
}

cudaError_t launch_scan(Variant v, const uint2 *planes, const PatDesc &d, const uint4 *masks,
                        TileEntry *table, pm_hit *tmp, uint64_t cap, unsigned long long *cursor,
                        uint32_t *status, int grid, cudaStream_t stream)
{
    if (d.ntiles == 0) return cudaSuccess;
    if ((uint64_t)grid > d.ntiles) grid = (int)d.ntiles;
    if (v == Variant::kWindowSliced && ws_bits(d.k) < 0) v = Variant::kPatternSliced;
    const void *fn = select_kernel(v, d.k);
    PatDesc dd = d;
    void *args[] = {(void *)&planes, (void *)&dd, (void *)&masks, (void *)&table,
                    (void *)&tmp,    (void *)&cap, (void *)&cursor, (void *)&status};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kScanThreads), args, 0, stream);
}

}  // namespace pm
