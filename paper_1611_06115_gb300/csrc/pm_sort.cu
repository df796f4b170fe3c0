// Sorting of segment records by key (the batched launch's output order).
//
// The batched scan appends one record per (pattern, tile) that has hits, in
// whatever order warps finish.  Records, not hits, are sorted: there are far
// fewer of them, and the hits of one record are already in window order.
// The sort is a least-significant-digit radix sort with 8-bit digits, stable
// within each pass:
//   1. every CTA takes a chunk of 4096 records and counts its digits into a
//      digit-major table hist[digit][cta];
//   2. an exclusive prefix sum over that table gives every (digit, CTA) its
//      first output slot;
//   3. every CTA walks its chunk again in order, 256 records per round, ranks
//      records of equal digit within a warp with __match_any_sync and across
//      the round's warps with per-warp counts, and writes them out.
// The record count lives in device memory; grids are sized for the maximum.
#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr uint64_t kSortChunk = (uint64_t)kSortThreads * kSortRounds;  // records per CTA
constexpr int kScanItems = 16;
constexpr uint64_t kScanSeg = (uint64_t)kSortThreads * kScanItems;

__device__ __forceinline__ uint64_t live_count(uint64_t n_max, const unsigned long long *n_dev)
{
    const uint64_t n = *n_dev;
    return n < n_max ? n : n_max;
}

__device__ __forceinline__ uint32_t block_exclusive_u32(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t sw[kSortThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int q = 0; q < kSortThreads / 32; ++q) {
            const uint32_t t = sw[q];
            sw[q] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    const uint32_t r = sw[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kSortThreads)
    k_rs_hist(const SegRecord *__restrict__ in, uint64_t n_max,
              const unsigned long long *__restrict__ n_dev, int shift, uint32_t *__restrict__ hist,
              uint32_t nblk)
{
    __shared__ uint32_t sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t n = live_count(n_max, n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * kSortChunk;
    for (int r = 0; r < kSortRounds; ++r) {
        const uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&sh[(uint32_t)(in[i].key >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblk + blockIdx.x] = sh[threadIdx.x];
}

// exclusive prefix sum of a u32 array in place (3 steps)
__global__ void __launch_bounds__(kSortThreads)
    k_u32_reduce(const uint32_t *__restrict__ a, uint64_t n, uint32_t *__restrict__ partial)
{
    __shared__ uint32_t stotal;
    const uint64_t base = (uint64_t)blockIdx.x * kScanSeg + (uint64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += a[base + i];
    block_exclusive_u32(s, &stotal);
    if (threadIdx.x == 0) partial[blockIdx.x] = stotal;
}

__global__ void __launch_bounds__(kSortThreads)
    k_u32_scan_partials(uint32_t *__restrict__ partial, uint64_t n)
{
    __shared__ uint32_t stotal;
    uint32_t carry = 0;
    for (uint64_t off = 0; off < n; off += kSortThreads) {
        const uint64_t i = off + threadIdx.x;
        const uint32_t v = i < n ? partial[i] : 0u;
        const uint32_t e = block_exclusive_u32(v, &stotal);
        if (i < n) partial[i] = carry + e;
        carry += stotal;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortThreads)
    k_u32_apply(uint32_t *__restrict__ a, uint64_t n, const uint32_t *__restrict__ partial)
{
    __shared__ uint32_t stotal;
    const uint64_t base = (uint64_t)blockIdx.x * kScanSeg + (uint64_t)threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        c[i] = base + i < n ? a[base + i] : 0u;
        s += c[i];
    }
    uint32_t run = partial[blockIdx.x] + block_exclusive_u32(s, &stotal);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) a[base + i] = run;
        run += c[i];
    }
}

__global__ void __launch_bounds__(kSortThreads)
    k_rs_scatter(const SegRecord *__restrict__ in, uint64_t n_max,
                 const unsigned long long *__restrict__ n_dev, int shift,
                 const uint32_t *__restrict__ hist, uint32_t nblk, SegRecord *__restrict__ out)
{
    constexpr int kW = kSortThreads / 32;
    __shared__ uint32_t sbase[256];
    __shared__ uint32_t swc[kW][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t n = live_count(n_max, n_dev);
    const uint64_t base = (uint64_t)blockIdx.x * kSortChunk;
    sbase[threadIdx.x] = hist[(uint64_t)threadIdx.x * nblk + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
        if (base + (uint64_t)r * kSortThreads >= n) break;  // uniform over the CTA
#pragma unroll
        for (int w = 0; w < kW; ++w) swc[w][threadIdx.x] = 0;
        __syncthreads();
        const uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
        const bool live = i < n;
        SegRecord rec;
        uint32_t d = 256u + (uint32_t)lane;  // dead lanes match nobody
        if (live) {
            rec = in[i];
            d = (uint32_t)(rec.key >> shift) & 0xffu;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (live && rank == 0) swc[warp][d] = __popc(peers);
        __syncthreads();
        if (live) {
            uint32_t off = sbase[d] + rank;
            for (int w = 0; w < warp; ++w) off += swc[w][d];
            out[off] = rec;
        }
        __syncthreads();
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < kW; ++w) add += swc[w][threadIdx.x];
        sbase[threadIdx.x] += add;
        __syncthreads();
    }
}

__global__ void k_rec_to_entries(const SegRecord *__restrict__ recs, uint64_t n_max,
                                 const unsigned long long *__restrict__ n_dev,
                                 TileEntry *__restrict__ entries)
{
    const uint64_t n = live_count(n_max, n_dev);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        entries[i] = TileEntry{recs[i].count, recs[i].src};
}

void scan_u32(uint32_t *a, uint64_t n, uint32_t *partial, cudaStream_t st)
{
    const uint64_t nb = (n + kScanSeg - 1) / kScanSeg;
    if (nb == 0) return;
    k_u32_reduce<<<(unsigned)nb, kSortThreads, 0, st>>>(a, n, partial);
    k_u32_scan_partials<<<1, kSortThreads, 0, st>>>(partial, nb);
    k_u32_apply<<<(unsigned)nb, kSortThreads, 0, st>>>(a, n, partial);
}

}  // namespace

size_t sort_scratch_bytes(uint64_t n_max)
{
    const uint64_t nblk = (n_max + kSortChunk - 1) / kSortChunk;
    const uint64_t hist = 256ull * (nblk ? nblk : 1);
    const uint64_t parts = (hist + kScanSeg - 1) / kScanSeg + 1;
    return (size_t)(n_max * sizeof(SegRecord) + 256 + hist * 4 + 256 + parts * 4 + 256);
}

cudaError_t launch_sort_records(SegRecord *recs, uint64_t n_max, const unsigned long long *n_dev,
                                int key_bits, void *scratch, cudaStream_t stream,
                                SegRecord **sorted)
{
    *sorted = recs;
    if (n_max == 0) return cudaSuccess;
    const uint64_t nblk = (n_max + kSortChunk - 1) / kSortChunk;
    char *p = (char *)scratch;
    SegRecord *alt = (SegRecord *)p;
    p += (n_max * sizeof(SegRecord) + 255) & ~255ull;
    uint32_t *hist = (uint32_t *)p;
    p += (256ull * nblk * 4 + 255) & ~255ull;
    uint32_t *partial = (uint32_t *)p;
    SegRecord *src = recs, *dst = alt;
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_rs_hist<<<(unsigned)nblk, kSortThreads, 0, stream>>>(src, n_max, n_dev, shift, hist,
                                                                (uint32_t)nblk);
        scan_u32(hist, 256ull * nblk, partial, stream);
        k_rs_scatter<<<(unsigned)nblk, kSortThreads, 0, stream>>>(src, n_max, n_dev, shift, hist,
                                                                   (uint32_t)nblk, dst);
        SegRecord *t = src;
        src = dst;
        dst = t;
    }
    *sorted = src;
    return cudaGetLastError();
}

cudaError_t launch_records_to_entries(const SegRecord *recs, uint64_t n_max,
                                      const unsigned long long *n_dev, TileEntry *entries,
                                      cudaStream_t stream)
{
    if (n_max == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n_max + 255) / 256;
    const unsigned grid = (unsigned)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
    k_rec_to_entries<<<grid, 256, 0, stream>>>(recs, n_max, n_dev, entries);
    return cudaGetLastError();
}

}  // namespace pm
