// Text coding (Sec. 2.1, Table 1) and the text handle.
//
// One thread codes one 32-symbol block: it reads 32 ASCII bytes (two 128-bit
// loads when aligned) and produces the block's two bit planes.  Four bytes
// are handled at once as one 32-bit word:
//   code(x)  = ((x >> 1) ^ (x >> 2)) & 3 per byte gives A=0 C=1 G=2 T=3 for
//              upper and lower case (bits 1-3 of the ASCII codes);
//   validity = the byte with bit 5 cleared must equal the letter its code
//              names, looked up with a byte permute; anything else is
//              reported (the first offset wins, by atomicMin);
//   packing  = the four low (high) code bits, one per byte, are gathered
//              into four adjacent plane bits by one multiply, since the
//              partial products of bits 0, 8, 16, 24 with 1 + 2^7 + 2^14 +
//              2^21 land on distinct positions and those of interest are
//              21..24.
#include <cstdarg>
#include <vector>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>

#include "pm_internal.cuh"

namespace pm {

namespace {
thread_local char g_err[512] = "";
constexpr uint64_t kHostChunk = 256ull << 20;  // symbols per staged host piece

__device__ __forceinline__ void code_word(uint32_t x, uint32_t &lo4, uint32_t &hi4, bool &ok)
{
    const uint32_t c = ((x >> 1) ^ (x >> 2)) & 0x03030303u;
    const uint32_t t = c | (c >> 4);
    const uint32_t selector = (t & 0xffu) | ((t >> 8) & 0xff00u);
    const uint32_t canon = __byte_perm(0x54474341u, 0u, selector);  // "ACGT"
    ok = (x & 0xdfdfdfdfu) == canon;
    const uint32_t l = c & 0x01010101u;
    const uint32_t h = (c >> 1) & 0x01010101u;
    lo4 = ((l * 0x00204081u) >> 21) & 0xfu;
    hi4 = ((h * 0x00204081u) >> 21) & 0xfu;
}

// ctl[0]: first offset of a symbol outside ACGT (atomicMin), unless unk is
// given: then such symbols are recorded there (one bit per symbol, the
// planes' block layout) and counted in ctl[4].  ctl[1..3]: how many C, G, T
// the text holds (A: the rest; the padding of the last block codes A, so it
// needs no correction).
__global__ void k_pack(const char *__restrict__ ascii, uint64_t n, uint64_t first,
                       uint2 *__restrict__ planes, uint32_t *__restrict__ unk,
                       unsigned long long *__restrict__ ctl, int aligned)
{
    unsigned long long *bad = ctl;
    uint32_t nc = 0, ng = 0, nt = 0, nu = 0;
    const uint64_t nb = (n + 31) / 32;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride) {
        const uint64_t off = b * 32;
        uint32_t w[8];
        if (aligned && off + 32 <= n) {
            const uint4 *p = reinterpret_cast<const uint4 *>(ascii + off);
            const uint4 u0 = __ldg(p), u1 = __ldg(p + 1);
            w[0] = u0.x; w[1] = u0.y; w[2] = u0.z; w[3] = u0.w;
            w[4] = u1.x; w[5] = u1.y; w[6] = u1.z; w[7] = u1.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint32_t v = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint64_t s = off + 4 * q + i;
                    const uint32_t ch = s < n ? (uint32_t)(uint8_t)ascii[s] : 0x41u;  // pad with A
                    v |= ch << (8 * i);
                }
                w[q] = v;
            }
        }
        uint32_t lo = 0, hi = 0, ub = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t l4, h4;
            bool ok;
            code_word(w[q], l4, h4, ok);
            lo |= l4 << (4 * q);
            hi |= h4 << (4 * q);
            if (!ok) {
                for (int i = 0; i < 4; ++i) {
                    const uint32_t ch = (w[q] >> (8 * i)) & 0xffu;
                    const uint32_t u = ch & 0xdfu;
                    if (u != 'A' && u != 'C' && u != 'G' && u != 'T') {
                        if (unk) {
                            ub |= 1u << (4 * q + i);
                        } else {
                            atomicMin(bad, (unsigned long long)(first + off + 4 * q + i));
                            break;
                        }
                    }
                }
            }
        }
        // Unknown symbols read as A C G T A C G T ... by position in the
        // planes: a pattern rarely matches that periodic text, so the exact
        // recount of candidates (which gives them their true count) stays
        // rare even inside long N runs.
        lo = (lo & ~ub) | (0xaaaaaaaau & ub);
        hi = (hi & ~ub) | (0xccccccccu & ub);
        planes[first / 32 + b] = make_uint2(lo, hi);
        if (unk) unk[first / 32 + b] = ub;
        nc += __popc(lo & ~hi & ~ub);
        ng += __popc(~lo & hi & ~ub);
        nt += __popc(lo & hi & ~ub);
        nu += __popc(ub);
    }
    // letter counts: one atomic per warp and letter (at most 32 * 32 per
    // thread-block row, far below 2^32 per warp over a grid-stride loop of
    // n < 2^32 symbols)
    nc = __reduce_add_sync(0xffffffffu, nc);
    ng = __reduce_add_sync(0xffffffffu, ng);
    nt = __reduce_add_sync(0xffffffffu, nt);
    nu = __reduce_add_sync(0xffffffffu, nu);
    if ((threadIdx.x & 31) == 0) {
        if (nc) atomicAdd(ctl + 1, (unsigned long long)nc);
        if (ng) atomicAdd(ctl + 2, (unsigned long long)ng);
        if (nt) atomicAdd(ctl + 3, (unsigned long long)nt);
        if (nu) atomicAdd(ctl + 4, (unsigned long long)nu);
    }
}

}  // namespace

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

pm_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PM_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PM_E_NOMEM : PM_E_CUDA;
}

bool is_device_pointer(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (mapped into the device's
// address space by unified addressing), or NULL for any other pointer.
const char *pinned_device_view(const char *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? (const char *)a.devicePointer : nullptr;
}

cudaError_t launch_pack(const char *ascii, uint64_t n_chunk, uint64_t first_symbol, uint2 *planes,
                        uint32_t *unk, unsigned long long *bad, cudaStream_t stream)
{
    if (n_chunk == 0) return cudaSuccess;
    const uint64_t nb = (n_chunk + 31) / 32;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (nb + 255) / 256;
    const uint64_t cap = (uint64_t)sms * 16;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    const int aligned = ((uintptr_t)ascii % 16) == 0;
    k_pack<<<grid, 256, 0, stream>>>(ascii, n_chunk, first_symbol, planes, unk, bad, aligned);
    return cudaGetLastError();
}

}  // namespace pm

using namespace pm;

extern "C" {

const char *pm_last_error(void) { return g_err; }

const char *pm_status_string(pm_status s)
{
    switch (s) {
    case PM_OK: return "ok";
    case PM_E_ARG: return "invalid argument";
    case PM_E_SYMBOL: return "text symbol outside A C G T";
    case PM_E_NOMEM: return "out of memory";
    case PM_E_OVERFLOW: return "more hits than capacity";
    case PM_E_TOO_LARGE: return "size beyond the limits of this build";
    case PM_E_TIMEOUT: return "a bounded device wait timed out";
    case PM_E_CUDA: return "CUDA runtime error";
    default: return "unknown status";
    }
}

pm_status pm_encode_text(const char *ascii, uint64_t n, void *stream, pm_text **out)
{
    return pm_encode_text_ex(ascii, n, 0u, stream, out);
}

pm_status pm_encode_text_ex(const char *ascii, uint64_t n, uint32_t flags, void *stream, pm_text **out)
{
    TraceRange trace("pm_encode_text");
    if (!out || (!ascii && n > 0) || (flags & ~PM_TEXT_UNKNOWN_AS_N)) {
        set_error("pm_encode_text: NULL argument or unknown flags 0x%x", flags);
        return PM_E_ARG;
    }
    const bool allow_unknown = (flags & PM_TEXT_UNKNOWN_AS_N) != 0;
    *out = nullptr;
    if (n >= (1ull << 32)) {
        set_error("pm_encode_text: n = %llu >= 2^32", (unsigned long long)n);
        return PM_E_TOO_LARGE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    pm_text *t = new (std::nothrow) pm_text{};
    if (!t) return PM_E_NOMEM;
    cudaGetDevice(&t->device);
    t->n = n;
    t->nblocks = (n + 31) / 32 + kPadBlocks;
    pm_status rc = cuda_status(cudaMalloc(&t->planes, t->nblocks * sizeof(uint2)), "cudaMalloc planes");
    if (rc) { delete t; return rc; }
    if (allow_unknown) {
        rc = cuda_status(cudaMalloc(&t->unk, t->nblocks * sizeof(uint32_t)), "cudaMalloc unknown bits");
        if (rc) { cudaFree(t->planes); delete t; return rc; }
    }

    unsigned long long *bad = nullptr;  // [0] first bad offset, [1..3] C, G, T, [4] unknown counts
    char *staging = nullptr;
    const bool on_device = is_device_pointer(ascii);
    // page-locked host input is read by the coding kernel in place (over the
    // host link, no staging copy); other host memory is staged in pieces
    const char *pinned = on_device ? nullptr : pinned_device_view(ascii);
    const uint64_t body = (n + 31) / 32;
    rc = cuda_status(cudaMemsetAsync(t->planes + body, 0, (t->nblocks - body) * sizeof(uint2), st),
                     "memset padding");
    if (!rc && t->unk)
        rc = cuda_status(cudaMemsetAsync(t->unk + body, 0, (t->nblocks - body) * sizeof(uint32_t), st),
                         "memset padding");
    if (!rc) rc = cuda_status(cudaMallocAsync((void **)&bad, 5 * sizeof *bad, st), "cudaMallocAsync");
    if (!rc) rc = cuda_status(cudaMemsetAsync(bad, 0xff, sizeof *bad, st), "memset");
    if (!rc) rc = cuda_status(cudaMemsetAsync(bad + 1, 0, 4 * sizeof *bad, st), "memset");
    if (!rc && (on_device || pinned)) {
        rc = cuda_status(launch_pack(on_device ? ascii : pinned, n, 0, t->planes, t->unk, bad, st),
                         "pack kernel");
    } else if (!rc && n > 0) {
        const uint64_t chunk = n < kHostChunk ? n : kHostChunk;
        rc = cuda_status(cudaMallocAsync((void **)&staging, (chunk + 15) & ~15ull, st),
                         "cudaMallocAsync staging");
        for (uint64_t off = 0; !rc && off < n; off += kHostChunk) {
            const uint64_t len = n - off < kHostChunk ? n - off : kHostChunk;
            rc = cuda_status(cudaMemcpyAsync(staging, ascii + off, len, cudaMemcpyHostToDevice, st),
                             "copy text to device");
            if (!rc) rc = cuda_status(launch_pack(staging, len, off, t->planes, t->unk, bad, st), "pack kernel");
        }
    }
    unsigned long long h_ctl[5] = {~0ull, 0, 0, 0, 0};
    if (!rc) rc = cuda_status(cudaMemcpyAsync(h_ctl, bad, sizeof h_ctl, cudaMemcpyDeviceToHost, st),
                              "copy status");
    const unsigned long long h_bad = h_ctl[0];
    if (staging) cudaFreeAsync(staging, st);
    if (bad) cudaFreeAsync(bad, st);
    const cudaError_t se = cudaStreamSynchronize(st);
    if (!rc) rc = cuda_status(se, "stream synchronize");
    if (!rc && h_bad != ~0ull) {
        set_error("pm_encode_text: symbol at offset %llu is not A, C, G or T", h_bad);
        rc = PM_E_SYMBOL;
    }
    if (rc) {
        cudaFree(t->planes);
        if (t->unk) cudaFree(t->unk);
        delete t;
        return rc;
    }
    t->n_unknown = h_ctl[4];
    if (t->unk && t->n_unknown == 0) {  // nothing unknown: the searches skip the recount
        cudaFree(t->unk);
        t->unk = nullptr;
    }
    t->count[1] = h_ctl[1];
    t->count[2] = h_ctl[2];
    t->count[3] = h_ctl[3];
    t->count[0] = n - h_ctl[1] - h_ctl[2] - h_ctl[3] - h_ctl[4];
    *out = t;
    return PM_OK;
}

uint64_t pm_text_length(const pm_text *text) { return text ? text->n : 0; }

uint64_t pm_text_unknown(const pm_text *text) { return text ? text->n_unknown : 0; }

pm_status pm_text_letter_counts(const pm_text *text, uint64_t counts[4])
{
    if (!text || !counts) {
        set_error("pm_text_letter_counts: NULL argument");
        return PM_E_ARG;
    }
    for (int i = 0; i < 4; ++i) counts[i] = text->count[i];
    return PM_OK;
}

pm_status pm_text_device_planes(const pm_text *text, const void **planes, uint64_t *bytes)
{
    if (!text) return PM_E_ARG;
    if (planes) *planes = text->planes;
    if (bytes) *bytes = text->nblocks * sizeof(uint2);
    return PM_OK;
}

// ---- coded-text files ----
//
// Layout (little-endian u64 fields): magic "PMTEXT1\0", n, nblocks,
// n_unknown, count[4], has_unknown_bits, checksum; then the planes (nblocks
// x 8 bytes) and, when has_unknown_bits, the unknown bits (nblocks x 4
// bytes).  The checksum is FNV-1a over 64-bit words (offset basis and prime
// of the 64-bit FNV) of the header fields before it and of the data.

namespace {
constexpr char kMagic[8] = {'P', 'M', 'T', 'E', 'X', 'T', '1', '\0'};
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull, kFnvPrime = 0x100000001b3ull;

uint64_t fnv_words(uint64_t h, const void *p, size_t bytes)
{
    const unsigned char *c = (const unsigned char *)p;
    size_t i = 0;
    for (; i + 8 <= bytes; i += 8) {
        uint64_t w;
        std::memcpy(&w, c + i, 8);
        h = (h ^ w) * kFnvPrime;
    }
    for (; i < bytes; ++i) h = (h ^ c[i]) * kFnvPrime;
    return h;
}

struct TextHeader {
    char magic[8];
    uint64_t n, nblocks, n_unknown, count[4], has_unk, checksum;
};
}  // namespace

pm_status pm_text_save(const pm_text *text, const char *path)
{
    if (!text || !path) {
        set_error("pm_text_save: NULL argument");
        return PM_E_ARG;
    }
    TextHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.n = text->n;
    h.nblocks = text->nblocks;
    h.n_unknown = text->n_unknown;
    for (int i = 0; i < 4; ++i) h.count[i] = text->count[i];
    h.has_unk = text->unk ? 1u : 0u;
    std::vector<uint2> planes;
    std::vector<uint32_t> unk;
    try {
        planes.resize(text->nblocks);
        if (text->unk) unk.resize(text->nblocks);
    } catch (...) {
        set_error("pm_text_save: no host memory for %llu blocks", (unsigned long long)text->nblocks);
        return PM_E_NOMEM;
    }
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != text->device) cudaSetDevice(text->device);
    pm_status rc = cuda_status(cudaMemcpy(planes.data(), text->planes, text->nblocks * sizeof(uint2),
                                          cudaMemcpyDeviceToHost), "copy planes");
    if (!rc && text->unk)
        rc = cuda_status(cudaMemcpy(unk.data(), text->unk, text->nblocks * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost), "copy unknown bits");
    if (cur != text->device) cudaSetDevice(cur);
    if (rc) return rc;
    uint64_t c = fnv_words(kFnvBasis, &h, offsetof(TextHeader, checksum));
    c = fnv_words(c, planes.data(), planes.size() * sizeof(uint2));
    if (text->unk) c = fnv_words(c, unk.data(), unk.size() * sizeof(uint32_t));
    h.checksum = c;
    FILE *f = std::fopen(path, "wb");
    if (!f) {
        set_error("pm_text_save: cannot open %s", path);
        return PM_E_ARG;
    }
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
              std::fwrite(planes.data(), sizeof(uint2), planes.size(), f) == planes.size() &&
              (!text->unk || std::fwrite(unk.data(), sizeof(uint32_t), unk.size(), f) == unk.size());
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) {
        set_error("pm_text_save: write to %s failed", path);
        return PM_E_ARG;
    }
    return PM_OK;
}

pm_status pm_text_load(const char *path, void *stream, pm_text **out)
{
    TraceRange trace("pm_text_load");
    if (!path || !out) {
        set_error("pm_text_load: NULL argument");
        return PM_E_ARG;
    }
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) {
        set_error("pm_text_load: cannot open %s", path);
        return PM_E_ARG;
    }
    TextHeader h{};
    auto fail = [&](pm_status rc, const char *why) {
        std::fclose(f);
        set_error("pm_text_load: %s: %s", path, why);
        return rc;
    };
    if (std::fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0)
        return fail(PM_E_ARG, "not a coded-text file");
    if (h.n >= (1ull << 32) || h.nblocks != (h.n + 31) / 32 + kPadBlocks || h.has_unk > 1)
        return fail(PM_E_ARG, "inconsistent header");
    std::vector<uint2> planes;
    std::vector<uint32_t> unk;
    try {
        planes.resize(h.nblocks);
        if (h.has_unk) unk.resize(h.nblocks);
    } catch (...) {
        return fail(PM_E_NOMEM, "no host memory");
    }
    if (std::fread(planes.data(), sizeof(uint2), planes.size(), f) != planes.size() ||
        (h.has_unk && std::fread(unk.data(), sizeof(uint32_t), unk.size(), f) != unk.size()))
        return fail(PM_E_ARG, "file is short");
    std::fclose(f);
    uint64_t c = fnv_words(kFnvBasis, &h, offsetof(TextHeader, checksum));
    c = fnv_words(c, planes.data(), planes.size() * sizeof(uint2));
    if (h.has_unk) c = fnv_words(c, unk.data(), unk.size() * sizeof(uint32_t));
    if (c != h.checksum) {
        set_error("pm_text_load: %s: checksum mismatch", path);
        return PM_E_ARG;
    }
    pm_text *t = new (std::nothrow) pm_text{};
    if (!t) return PM_E_NOMEM;
    cudaGetDevice(&t->device);
    t->n = h.n;
    t->nblocks = h.nblocks;
    t->n_unknown = h.n_unknown;
    for (int i = 0; i < 4; ++i) t->count[i] = h.count[i];
    cudaStream_t st = (cudaStream_t)stream;
    pm_status rc = cuda_status(cudaMalloc(&t->planes, t->nblocks * sizeof(uint2)), "cudaMalloc planes");
    if (!rc && h.has_unk)
        rc = cuda_status(cudaMalloc(&t->unk, t->nblocks * sizeof(uint32_t)), "cudaMalloc unknown bits");
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(t->planes, planes.data(), t->nblocks * sizeof(uint2),
                                         cudaMemcpyHostToDevice, st), "upload planes");
    if (!rc && h.has_unk)
        rc = cuda_status(cudaMemcpyAsync(t->unk, unk.data(), t->nblocks * sizeof(uint32_t),
                                         cudaMemcpyHostToDevice, st), "upload unknown bits");
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st), "stream synchronize");
    if (rc) {
        if (t->planes) cudaFree(t->planes);
        if (t->unk) cudaFree(t->unk);
        delete t;
        return rc;
    }
    *out = t;
    return PM_OK;
}

void pm_text_free(pm_text *text)
{
    if (!text) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != text->device) cudaSetDevice(text->device);
    cudaFree(text->planes);
    if (text->unk) cudaFree(text->unk);
    if (cur != text->device) cudaSetDevice(cur);
    delete text;
}

}  // extern "C"
