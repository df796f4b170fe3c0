// Ordering of hits (output contract: per pattern, sorted by location).
//
// The scan kernels leave each (pattern, tile) segment of hits in window
// order somewhere in a scratch buffer and describe it by an entry {count,
// src}.  Entries are either a dense table running pattern-major, tile-minor
// (per-pattern launches), or segment records sorted by (pattern, tile)
// (batched launch); either way they are already in output order.  An
// exclusive prefix sum over the counts gives each segment its final place,
// per-pattern CSR offsets come from the same sums, and a gather copies the
// segments.  No comparison sort of hits is needed.
//
// The number of entries may live in device memory (n_dev, capped by the
// host-side bound n_max that sizes the grids), so that a batched run needs
// no host round trip.
#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr int kOrdThreads = 256;
constexpr int kOrdItems = 16;
constexpr uint64_t kSeg = (uint64_t)kOrdThreads * kOrdItems;  // entries per block

__device__ __forceinline__ uint64_t entry_count(uint64_t n_max, const unsigned long long *n_dev)
{
    if (!n_dev) return n_max;
    const uint64_t n = *n_dev;
    return n < n_max ? n : n_max;
}

// Exclusive prefix sum over a CTA; returns this thread's prefix and sets
// *total (a __shared__ variable) to the CTA sum.
__device__ __forceinline__ unsigned long long block_exclusive(unsigned long long v,
                                                              unsigned long long *total)
{
    __shared__ unsigned long long sw[kOrdThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int q = 0; q < kOrdThreads / 32; ++q) {
            const unsigned long long t = sw[q];
            sw[q] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    const unsigned long long r = sw[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kOrdThreads)
    k_reduce(const TileEntry *__restrict__ table, uint64_t n_max,
             const unsigned long long *__restrict__ n_dev, unsigned long long *__restrict__ partial)
{
    __shared__ unsigned long long stotal;
    const uint64_t entries = entry_count(n_max, n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * kSeg + (uint64_t)threadIdx.x * kOrdItems;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kOrdItems; ++i)
        if (base + i < entries) s += table[base + i].count;
    block_exclusive(s, &stotal);
    if (threadIdx.x == 0) partial[blockIdx.x] = stotal;
}

// One CTA: exclusive scan of the per-block partials in place; total at [n].
__global__ void __launch_bounds__(kOrdThreads)
    k_scan_partials(unsigned long long *__restrict__ partial, uint64_t n)
{
    __shared__ unsigned long long stotal;
    unsigned long long carry = 0;
    for (uint64_t off = 0; off < n; off += kOrdThreads) {
        const uint64_t i = off + threadIdx.x;
        const unsigned long long v = i < n ? partial[i] : 0ull;
        const unsigned long long e = block_exclusive(v, &stotal);
        if (i < n) partial[i] = carry + e;
        carry += stotal;
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[n] = carry;
}

__global__ void __launch_bounds__(kOrdThreads)
    k_dest(const TileEntry *__restrict__ table, uint64_t n_max,
           const unsigned long long *__restrict__ n_dev,
           const unsigned long long *__restrict__ partial, unsigned long long *__restrict__ dest)
{
    __shared__ unsigned long long stotal;
    const uint64_t entries = entry_count(n_max, n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * kSeg + (uint64_t)threadIdx.x * kOrdItems;
    uint32_t c[kOrdItems];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < kOrdItems; ++i) {
        c[i] = base + i < entries ? table[base + i].count : 0u;
        s += c[i];
    }
    unsigned long long run = partial[blockIdx.x] + block_exclusive(s, &stotal);
#pragma unroll
    for (int i = 0; i < kOrdItems; ++i) {
        if (base + i < entries) dest[base + i] = run;
        run += c[i];
    }
}

__global__ void k_offsets(const uint64_t *__restrict__ pat_tile0, uint32_t npat, uint64_t entries,
                          const unsigned long long *__restrict__ dest,
                          const unsigned long long *__restrict__ total,
                          const uint32_t *__restrict__ status, uint64_t *__restrict__ offsets)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > npat) return;
    if (p == npat) {
        offsets[p] = (*status & kDevTimeout) ? PM_TOTAL_ERROR : (uint64_t)*total;
        return;
    }
    const uint64_t e = pat_tile0[p];
    offsets[p] = e < entries ? (uint64_t)dest[e] : (uint64_t)*total;
}

// One CTA: CSR offsets from per-pattern hit counts (exclusive prefix sum),
// the total at [npat] (PM_TOTAL_ERROR after a device-side failure).
__global__ void __launch_bounds__(kOrdThreads)
    k_offsets_from_counts(const unsigned long long *__restrict__ counts, uint32_t npat,
                          const uint32_t *__restrict__ status, uint64_t *__restrict__ offsets)
{
    __shared__ unsigned long long stotal;
    unsigned long long carry = 0;
    for (uint64_t off = 0; off < npat; off += kOrdThreads) {
        const uint64_t i = off + threadIdx.x;
        const unsigned long long v = i < npat ? counts[i] : 0ull;
        const unsigned long long e = block_exclusive(v, &stotal);
        if (i < npat) offsets[i] = carry + e;
        carry += stotal;
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[npat] = (*status & kDevTimeout) ? PM_TOTAL_ERROR : carry;
}

// One warp per entry: copy its segment to its final place.
__global__ void __launch_bounds__(kOrdThreads)
    k_gather(const TileEntry *__restrict__ table, uint64_t n_max,
             const unsigned long long *__restrict__ n_dev,
             const unsigned long long *__restrict__ dest, const unsigned long long *__restrict__ total,
             const uint32_t *__restrict__ status, const pm_hit *__restrict__ tmp,
             pm_hit *__restrict__ hits, uint64_t cap)
{
    // total: all hits found (nothing is written when they do not fit)
    if (*total > cap || (*status & kDevTimeout)) return;
    const uint64_t entries = entry_count(n_max, n_dev);
    const uint64_t warps = (uint64_t)gridDim.x * (kOrdThreads / 32);
    const int lane = threadIdx.x & 31;
    // each lane reads one entry of a run of 32 (most entries are empty); the
    // warp then copies the non-empty ones one after another, coalesced
    for (uint64_t base = ((uint64_t)blockIdx.x * (kOrdThreads / 32) + (threadIdx.x >> 5)) * 32;
         base < entries; base += warps * 32) {
        const uint64_t e = base + (uint64_t)lane;
        const TileEntry te = e < entries ? table[e] : TileEntry{0u, 0u};
        const unsigned long long d = te.count ? dest[e] : 0ull;
        uint32_t nz = __ballot_sync(0xffffffffu, te.count != 0u);
        while (nz) {
            const int j = __ffs(nz) - 1;
            nz &= nz - 1;
            const uint32_t cnt = __shfl_sync(0xffffffffu, te.count, j);
            const uint64_t src = __shfl_sync(0xffffffffu, te.src, j);
            const unsigned long long dd = __shfl_sync(0xffffffffu, d, j);
            for (uint32_t i = lane; i < cnt; i += 32) hits[dd + i] = tmp[src + i];
        }
    }
}

// prefix sums of the entry counts: dest[e] and the total (partial[nblk])
void launch_dest(const TileEntry *table, uint64_t n_max, const unsigned long long *n_dev,
                 unsigned long long *partial, unsigned long long *dest, cudaStream_t stream)
{
    const uint64_t nblk = (n_max + kSeg - 1) / kSeg;
    if (nblk > 0) k_reduce<<<(unsigned)nblk, kOrdThreads, 0, stream>>>(table, n_max, n_dev, partial);
    k_scan_partials<<<1, kOrdThreads, 0, stream>>>(partial, nblk);
    if (nblk > 0)
        k_dest<<<(unsigned)nblk, kOrdThreads, 0, stream>>>(table, n_max, n_dev, partial, dest);
}

void launch_gather(const TileEntry *table, uint64_t n_max, const unsigned long long *n_dev,
                   const unsigned long long *dest, const unsigned long long *total,
                   const uint32_t *status, const pm_hit *tmp, pm_hit *hits, uint64_t cap,
                   cudaStream_t stream)
{
    if (n_max == 0) return;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n_max + kOrdThreads - 1) / kOrdThreads;  // one run of 32 entries per warp
    uint64_t grid = want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8;
    if (grid < 1) grid = 1;
    k_gather<<<(unsigned)grid, kOrdThreads, 0, stream>>>(table, n_max, n_dev, dest, total, status,
                                                         tmp, hits, cap);
}

}  // namespace

size_t order_scratch_bytes(uint64_t entries)
{
    const uint64_t nblk = (entries + kSeg - 1) / kSeg;
    // partials (+1 for the total) and per-entry destinations
    return (size_t)((nblk + 1) * 8 + entries * 8 + 256);
}

cudaError_t launch_order(const TileEntry *table, uint64_t entries, const uint64_t *pat_tile0,
                         uint32_t npat, const pm_hit *tmp, pm_hit *hits, uint64_t cap,
                         uint64_t *offsets, const uint32_t *status, void *scratch,
                         cudaStream_t stream)
{
    const uint64_t nblk = (entries + kSeg - 1) / kSeg;
    auto *partial = (unsigned long long *)scratch;
    auto *dest = partial + nblk + 1;
    const unsigned long long *total = partial + nblk;
    launch_dest(table, entries, nullptr, partial, dest, stream);
    k_offsets<<<(npat + 1 + 255) / 256, 256, 0, stream>>>(pat_tile0, npat, entries, dest, total,
                                                          status, offsets);
    launch_gather(table, entries, nullptr, dest, total, status, tmp, hits, cap, stream);
    return cudaGetLastError();
}

cudaError_t launch_order_records(const TileEntry *entries, uint64_t n_max,
                                 const unsigned long long *n_dev,
                                 const unsigned long long *pat_counts, uint32_t npat,
                                 const unsigned long long *hits_found, const pm_hit *tmp,
                                 pm_hit *hits, uint64_t cap, uint64_t *offsets,
                                 const uint32_t *status, void *scratch, cudaStream_t stream)
{
    const uint64_t nblk = (n_max + kSeg - 1) / kSeg;
    auto *partial = (unsigned long long *)scratch;
    auto *dest = partial + nblk + 1;
    launch_dest(entries, n_max, n_dev, partial, dest, stream);
    k_offsets_from_counts<<<1, kOrdThreads, 0, stream>>>(pat_counts, npat, status, offsets);
    launch_gather(entries, n_max, n_dev, dest, hits_found, status, tmp, hits, cap, stream);
    return cudaGetLastError();
}

}  // namespace pm
