// Device building blocks shared by the per-pattern and the batched scan
// kernels (see pm_scan.cu for the method they implement).
#pragma once

#include "pm_internal.cuh"

namespace pm {
namespace scan {

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

// The exact count of window 32*blk + w (stopping once past `limit`) for a
// text that may hold unknown symbols (unk: one bit per symbol, NULL when the
// text has none).  At an unknown symbol only the class N (every letter)
// matches.  The planes code an unknown symbol as some letter, so the count
// the scan evaluations see there is never above this one: a window they
// drop is past k here too, and the windows they pass are recounted here.
__device__ __forceinline__ uint32_t window_count_exact(const uint2 *__restrict__ planes,
                                                       const uint32_t *__restrict__ unk,
                                                       uint64_t blk, uint32_t w,
                                                       const uint4 *__restrict__ M,
                                                       uint32_t nchunks, uint32_t limit)
{
    if (!unk) return window_count_from(planes, blk, w, M, 0, nchunks, 0u, limit);
    uint32_t count = 0;
    uint2 a = __ldg(planes + blk);
    uint32_t ua = __ldg(unk + blk);
    for (uint32_t c = 0; c < nchunks; ++c) {
        const uint2 b = __ldg(planes + blk + c + 1);
        const uint32_t ub = __ldg(unk + blk + c + 1);
        const uint4 Mc = __ldg(M + c);
        const uint32_t match = class_match(__funnelshift_r(a.x, b.x, w), __funnelshift_r(a.y, b.y, w), Mc);
        const uint32_t u = __funnelshift_r(ua, ub, w);
        const uint32_t is_n = Mc.x & Mc.y & Mc.z & Mc.w;  // also every position past m
        count += __popc(~((match & ~u) | (u & is_n)));
        if (count > limit) break;
        a = b;
        ua = ub;
    }
    return count;
}

// Drop from pass the windows whose exact count (window_count_exact) is past
// k; only texts with unknown symbols need it.
__device__ __forceinline__ uint32_t recount_unknown(uint32_t pass, const uint2 *__restrict__ planes,
                                                   const uint32_t *__restrict__ unk, uint64_t blk,
                                                   const uint4 *__restrict__ M, uint32_t nchunks,
                                                   uint32_t k)
{
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        if (window_count_exact(planes, unk, blk, w, M, nchunks, k) > k) pass &= ~(1u << w);
    }
    return pass;
}

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Pattern-sliced test of the first C chunks (C = 1 or 2) for one lane's 32
// windows; pass mask (window w at bit w) of the windows with at most k
// mismatches in positions 0..32C-1 (k <= 32C-1).  Blocks blk, blk+1 (and
// blk+2 for C = 2) are a, b, c; M0, M1 the masks of chunks 0 and 1.  Step j
// takes windows j, 8 + j, 16 + j, 24 + j, one per byte of a multiply-add
// result that holds matches + k, below 2^(5+C) so bytes never carry: its
// bit 4+C is set exactly when matches + k >= 32C, i.e. when the window has
// at most k mismatches, and moves to bit 8q + j, the window's own bit.
// k4 = k in every byte; one, m8, m16, m24 = 1, 2^8, 2^16, 2^24.
template <int C>
__device__ __forceinline__ uint32_t pass_pattern_sliced(uint2 a, uint2 b, uint2 c, uint4 M0,
                                                        uint4 M1, uint32_t k4, uint32_t one,
                                                        uint32_t m8, uint32_t m16, uint32_t m24)
{
    static_assert(C == 1 || C == 2, "one or two chunks");
    constexpr int kBit = 4 + C;
    uint32_t pass = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int w = 8 * q + j;
            g[q] = __popc(class_match(__funnelshift_r(a.x, b.x, w), __funnelshift_r(a.y, b.y, w), M0));
            if constexpr (C == 2)
                g[q] += __popc(class_match(__funnelshift_r(b.x, c.x, w), __funnelshift_r(b.y, c.y, w), M1));
        }
        uint32_t v = mad_lo(g[3], m24, k4);
        v = mad_lo(g[2], m16, v);
        v = mad_lo(g[1], m8, v);
        v = mad_lo(g[0], one, v);
        // bit kBit of byte q: g[q] + k >= 32C; move bits 8q + kBit to 8q + j = w
        const uint32_t s = j <= kBit ? v >> (kBit - j) : v << (j - kBit);
        pass |= s & (0x01010101u << j);
    }
    return pass;
}

// A position-list entry from shared memory, or from global memory through
// the read-only path (every lane reads the same address: one broadcast).
template <bool kGlobal>
__device__ __forceinline__ uint4 ld_list(const uint4 *p)
{
    if constexpr (kGlobal) return __ldg(p);
    else return *p;
}

// List entries the window-sliced scan tests before it leaves the remaining
// candidates to exact one-by-one counts (checked every four entries).
// Measured on GB300 over a 3.1 Gbp text (m = 32 .. 1024): K = 0 8 entries
// (2-3 % faster than no cut), K = 1..4 4 + 2K (7, 18, 4, 12 % faster); a
// cut one block earlier leaves so many candidates that their serial counts
// cost 1.4-4x the scan.
__host__ __device__ constexpr uint32_t ws_cut(int K) { return K == 0 ? 8u : 4u + 2u * (uint32_t)K; }

// Window-sliced first chunk with a thermometer counter of K+1 levels over the
// listed positions, for all groups of the lane at once.  alive[g] receives
// the windows still at or below K.  After `cut` list entries (checked every
// four) the scan stops if some window is still alive and returns true: the
// few candidates left are cheaper to count one by one (settle_from_regs)
// than to carry the whole tile through the remaining positions.  Returns
// false when every listed position was tested (alive is then exact over the
// first 32 positions) or every window died.
template <int K, bool kGlobal = false>
__device__ __forceinline__ bool alive_window_sliced(const uint2 (&a)[G], const uint2 (&b)[G],
                                                    const uint4 *__restrict__ list,
                                                    uint32_t n_single, uint32_t n_general,
                                                    uint32_t cut, const uint32_t (&valid)[G],
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
        for (int u = 0; u < 4; ++u) q[u] = ld_list<kGlobal>(list + e + u);
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
            return false;
        }
        if (e + 4 >= cut) {
#pragma unroll
            for (int g = 0; g < G; ++g) alive[g] = ~L[g][K];
            return true;
        }
    }
    for (; e < n_single; ++e) {
        const uint4 q = ld_list<kGlobal>(list + e);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t lo = __funnelshift_r(a[g].x, b[g].x, q.x);
            const uint32_t hi = __funnelshift_r(a[g].y, b[g].y, q.x);
            add(g, (lo ^ q.y) | (hi ^ q.z));
        }
    }
    for (uint32_t c = 0; c < n_general; ++c) {
        const uint32_t s = ld_list<kGlobal>(list + n_single + 2 * c).x;
        const uint4 M = ld_list<kGlobal>(list + n_single + 2 * c + 1);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const uint32_t lo = __funnelshift_r(a[g].x, b[g].x, s);
            const uint32_t hi = __funnelshift_r(a[g].y, b[g].y, s);
            add(g, ~class_match(lo, hi, M));
        }
        if ((c & 3) == 3) {
            if (dead_all()) {
#pragma unroll
                for (int g = 0; g < G; ++g) alive[g] = 0u;
                return false;
            }
            if (n_single + c + 1 >= cut) {
#pragma unroll
                for (int g = 0; g < G; ++g) alive[g] = ~L[g][K];
                return true;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) alive[g] = ~L[g][K];
    return false;
}

// One warp tile and its halo, global -> shared, completing on bar.
__device__ __forceinline__ void issue_tile(const uint2 *planes, uint64_t tile, uint2 *dst,
                                           uint64_t *bar)
{
    dev::mbar_arrive_expect_tx(bar, kStageBytes);
    dev::bulk_g2s(dst, planes + tile * (32ull * G), kStageBytes, bar);
}


// Window-valid mask of the 32 windows that start in block blk.
__device__ __forceinline__ uint32_t valid_mask(uint64_t blk, uint64_t nwin)
{
    const uint64_t w0 = blk * 32ull;
    return w0 >= nwin ? 0u : (nwin - w0 >= 32 ? kFull : (1u << (uint32_t)(nwin - w0)) - 1u);
}

// Pattern-sliced evaluation over all chunks for large k (k > 31, where one
// chunk cannot decide a window): 32 per-window counts in registers, one
// chunk after another (chunk c needs blocks blk+c and blk+c+1; blocks 0 and
// 1 are given), until every window of the warp has passed k (the early stop
// of Sec. 2.4) or the pattern ends.  Returns the windows whose full count
// is at most k.
__device__ __forceinline__ uint32_t pass_multi_chunk(const uint2 *__restrict__ planes, uint64_t blk,
                                                     const uint4 *__restrict__ M, uint32_t nchunks,
                                                     uint32_t k, uint32_t valid, uint2 t0, uint2 t1)
{
    uint32_t cnt[32];
#pragma unroll
    for (int w = 0; w < 32; ++w) cnt[w] = 0;
    uint32_t alive = valid;
    for (uint32_t c = 0; c < nchunks; ++c) {
        if (c > 0) {
            t0 = t1;
            t1 = __ldg(planes + blk + c + 1);
        }
        const uint4 Mc = __ldg(M + c);
        uint32_t a2 = 0;
#pragma unroll
        for (int w = 0; w < 32; ++w) {
            cnt[w] += __popc(~class_match(__funnelshift_r(t0.x, t1.x, w), __funnelshift_r(t0.y, t1.y, w), Mc));
            a2 |= (cnt[w] <= k ? 1u : 0u) << w;
        }
        alive &= a2;
        if (!__any_sync(kFull, alive != 0u)) break;
    }
    return alive;
}

// Exact counts of the windows still in `pass` for a pattern longer than 32:
// each lane counts its own remaining windows, chunk by chunk, and drops
// those past k.
__device__ __forceinline__ uint32_t settle_lane(uint32_t pass, uint64_t blk,
                                                const uint4 *__restrict__ M, uint32_t nchunks,
                                                uint32_t k, const uint2 *__restrict__ planes)
{
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        if (window_count_from(planes, blk, w, M, 0, nchunks, 0u, k) > k) pass &= ~(1u << w);
    }
    return pass;
}

// settle_lane for a lane whose blocks blk and blk+1 are in registers (t0, t1)
// and whose block blk+2 is still staged in shared memory (s_next): chunks 0
// and 1 need no load through L1/L2, deeper chunks (rarely reached while k is
// below the expected mismatches of 64 positions) use window_count_from.
__device__ __forceinline__ uint32_t settle_staged(uint32_t pass, uint64_t blk, uint2 t0, uint2 t1,
                                                 const uint2 *s_next, const uint4 *__restrict__ M,
                                                 uint32_t nchunks, uint32_t k,
                                                 const uint2 *__restrict__ planes)
{
    if (!pass) return 0u;
    const uint4 M0 = __ldg(M), M1 = __ldg(M + 1);
    const uint2 t2 = *s_next;
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        uint32_t c = __popc(~class_match(__funnelshift_r(t0.x, t1.x, w), __funnelshift_r(t0.y, t1.y, w), M0));
        if (c <= k)
            c += __popc(~class_match(__funnelshift_r(t1.x, t2.x, w), __funnelshift_r(t1.y, t2.y, w), M1));
        if (c <= k && nchunks > 2) c = window_count_from(planes, blk, w, M, 2, nchunks, c, k);
        if (c > k) pass &= ~(1u << w);
    }
    return pass;
}

// Exact counts of the windows still in `pass`, the first chunk from the
// lane's blocks in registers (t0, t1), the rest through L1/L2 (any m):
// drops those past k.
__device__ __forceinline__ uint32_t settle_from_regs(uint32_t pass, uint64_t blk, uint2 t0, uint2 t1,
                                                    const uint4 *__restrict__ M, uint32_t nchunks,
                                                    uint32_t k, const uint2 *__restrict__ planes)
{
    if (!pass) return 0u;
    const uint4 M0 = __ldg(M);
    uint32_t sv = pass;
    while (sv) {
        const uint32_t w = __ffs(sv) - 1;
        sv &= sv - 1;
        uint32_t c = __popc(~class_match(__funnelshift_r(t0.x, t1.x, w), __funnelshift_r(t0.y, t1.y, w), M0));
        if (c <= k && nchunks > 1) c = window_count_from(planes, blk, w, M, 1, nchunks, c, k);
        if (c > k) pass &= ~(1u << w);
    }
    return pass;
}

// Run-time constants of the pattern-sliced byte test for one k (k <= 63;
// the kernels use it only where k < 32C).
struct PsConst {
    uint32_t one, m8, m16, m24, k4;
};

__device__ __forceinline__ PsConst ps_const(uint32_t two, uint32_t k)
{
    PsConst c;
    c.one = two >> 1;
    c.m8 = c.one << 8;
    c.m16 = c.one << 16;
    c.m24 = c.one << 24;
    c.k4 = (k < 64u ? k : 0u) * (c.m24 | c.m16 | c.m8 | c.one);
    return c;
}

// The windows of one warp tile that hold the pattern with at most k
// mismatches: pass[g] bit w for window 32*blk[g] + w.  VARIANT as in k_scan;
// list (window-sliced only) is the pattern's position list in shared memory;
// stage (pattern-sliced, -1 and -3) is the tile still staged in shared memory.
template <int VARIANT>
__device__ __forceinline__ void tile_pass(const uint2 (&a)[G], const uint2 (&b)[G],
                                          const uint64_t (&blk)[G], const uint32_t (&valid)[G],
                                          const PatDesc &d, const uint4 *__restrict__ M,
                                          uint4 M0, const uint4 *__restrict__ list,
                                          const PsConst &pc, const uint2 *__restrict__ planes,
                                          const uint2 *stage, uint32_t (&pass)[G])
{
    const uint32_t k = (uint32_t)d.k;
    if constexpr (VARIANT >= 0) {
        const bool cut = alive_window_sliced<VARIANT>(a, b, list, d.n_single, d.n_general, ws_cut(VARIANT),
                                                      valid, pass);
        if (cut || d.nchunks > 1) {
#pragma unroll
            for (int g = 0; g < G; ++g)
                pass[g] = settle_from_regs(pass[g], blk[g], a[g], b[g], M, d.nchunks, k, planes);
        }
        return;
    } else if constexpr (VARIANT == -2) {
        // k > 31: one chunk cannot decide; count all chunks (exact, nothing to settle)
#pragma unroll 1
        for (int g = 0; g < G; ++g)
            pass[g] = pass_multi_chunk(planes, blk[g], M, d.nchunks, k, valid[g], a[g], b[g]);
        return;
    } else {
        // -1: one chunk; -3: two chunks (chunk 1 of a pattern with m <= 32
        // reads as all ones: every position past m matches)
        constexpr int C = VARIANT == -3 ? 2 : 1;
        const int lane = threadIdx.x & 31;
        const uint4 M1 = (C == 2 && d.nchunks > 1) ? __ldg(M + 1) : make_uint4(kFull, kFull, kFull, kFull);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            uint32_t t = 0u;
            if (valid[g]) {
                const uint2 c = C == 2 ? stage[32 * g + lane + 2] : make_uint2(0u, 0u);
                t = pass_pattern_sliced<C>(a[g], b[g], c, M0, M1, pc.k4, pc.one, pc.m8, pc.m16,
                                           pc.m24) & valid[g];
            }
            pass[g] = t;
        }
    }
    // Both evaluations are exact for m <= 32.  Longer patterns: count every
    // remaining window exactly and drop those past k.
    if (d.nchunks > 1) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if constexpr (VARIANT == -1 || VARIANT == -3)
                pass[g] = settle_staged(pass[g], blk[g], a[g], b[g], stage + 32 * g + lane + 2, M,
                                        d.nchunks, k, planes);
            else
                pass[g] = settle_lane(pass[g], blk[g], M, d.nchunks, k, planes);
        }
    }
}

// Emit the hits of one warp tile in window order through one
// warp-aggregated atomic on cursor.  Call with the whole warp and only when
// some lane has a pass bit.  Returns (on every lane) the number of hits and
// where they start in tmp.
// kRegs: the lane's blocks a[g], b[g] (registers) and the chunk-0 masks M0
// give the first 32 positions of a hit's count without a memory access
// (deeper chunks, and texts with unknown symbols, count through L1/L2); used
// by the pattern-sliced kernels, whose hits are dense for small m and large
// k.  Otherwise every hit is counted through L1/L2, which keeps a and b out
// of registers during emission.
template <bool kRegs>
__device__ __forceinline__ void emit_tile_hits(uint32_t (&pass)[G], const uint64_t (&blk)[G],
                                               const uint2 (&a)[G], const uint2 (&b)[G], uint4 M0,
                                               const PatDesc &d, const uint4 *__restrict__ M,
                                               const uint2 *__restrict__ planes,
                                               const uint32_t *__restrict__ unk,
                                               pm_hit *__restrict__ tmp, uint64_t cap,
                                               unsigned long long *__restrict__ cursor,
                                               uint32_t &total_out, unsigned long long &base_out)
{
    const int lane = threadIdx.x & 31;
    if (unk) {
#pragma unroll
        for (int g = 0; g < G; ++g)
            pass[g] = recount_unknown(pass[g], planes, unk, blk[g], M, d.nchunks, (uint32_t)d.k);
    }
    uint32_t incl[G], tot[G];
    uint32_t total = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        incl[g] = __popc(pass[g]);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl[g], o);
            if (lane >= o) incl[g] += v;
        }
        tot[g] = __shfl_sync(kFull, incl[g], 31);
        total += tot[g];
    }
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 0);
    total_out = total;
    base_out = base;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        unsigned long long q = base + incl[g] - __popc(pass[g]);
        uint32_t hm = pass[g];
        while (hm) {
            const uint32_t w = __ffs(hm) - 1;
            hm &= hm - 1;
            if (q < cap) {
                uint32_t c;
                if (!kRegs || unk) {
                    c = window_count_exact(planes, unk, blk[g], w, M, d.nchunks, (uint32_t)d.k);
                } else {
                    c = __popc(~class_match(__funnelshift_r(a[g].x, b[g].x, w),
                                            __funnelshift_r(a[g].y, b[g].y, w), M0));
                    if (d.nchunks > 1)
                        c = window_count_from(planes, blk[g], w, M, 1, d.nchunks, c, (uint32_t)d.k);
                }
                tmp[q] = pm_hit{(uint32_t)(blk[g] * 32ull + w), c};
            }
            ++q;
        }
        base += tot[g];
    }
}

}  // namespace scan
}  // namespace pm
