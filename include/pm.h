/*
 * pm.h -- C ABI of libpm: k-mismatch matching of IUPAC character-class
 * patterns against a 2-bit DNA text, on one GB300 GPU (sm_103a).
 *
 * Method: "Fast low-level pattern matching algorithm" (Soldo, Krzic, Sersic,
 * arXiv 1611.06115).  Location i of text t holds pattern p with at most k
 * mismatches when  sum_{j=1..m} L[(p[j] << 2) OR t[i+j-1]] <= k  (Eq. 4),
 * where t is coded by Table 1, p by Table 2, and L is the 64-entry
 * match/mismatch dictionary of Table 3 that the paper derives from the
 * prime-residue test of Sec. 1.3 (Eq. 1 and Eq. 3).
 *
 * Conventions shared by every entry point
 *   - Locations are 0-based (the paper's location i is ours + 1).  A text
 *     of n symbols has n-m+1 windows; no window is partial; m > n gives none.
 *   - k is inclusive (Eq. 4 reads "<= k"); k >= m reports every window.
 *   - Errors are returned as pm_status, never thrown.  pm_status_string()
 *     names a status; pm_last_error() gives the calling thread's last
 *     detailed message (for example the offset of a bad text symbol).
 *   - "stream" is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream.  Work is ordered on that stream.
 *   - Pointers documented as "host or device" are classified with
 *     cudaPointerGetAttributes: device (and managed) memory is used in
 *     place, anything else is treated as host memory.
 *   - Handles (pm_text, pm_pattern, pm_batch) are owned by the library and
 *     released with the matching *_free call.  Buffers passed in are owned
 *     by the caller.
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pm_status;

#define PM_OK 0
#define PM_E_ARG (-1)       /* an argument is invalid (NULL, m == 0, k < 0, ...) */
#define PM_E_SYMBOL (-2)    /* a text symbol is not one of A C G T (either case) */
#define PM_E_NOMEM (-3)     /* a device or host allocation failed */
#define PM_E_OVERFLOW (-4)  /* more hits than the caller's capacity */
#define PM_E_TOO_LARGE (-5) /* n >= 2^32, or a size limit of this build */
#define PM_E_TIMEOUT (-6)   /* a bounded wait inside a kernel gave up */
#define PM_E_CUDA (-7)      /* a CUDA runtime call failed */

/* One reported window: 0-based location and its exact mismatch count. */
typedef struct pm_hit {
    uint32_t location;
    uint32_t mismatches;
} pm_hit;

typedef struct pm_text pm_text;       /* device-resident 2-bit text */
typedef struct pm_pattern pm_pattern; /* compiled pattern (host data) */
typedef struct pm_batch pm_batch;     /* patterns + k + scratch, resident on the device */

/* Value of offsets[npat] that signals a device-side failure (a timed-out
 * wait) to callers that did not ask for a synchronous status. */
#define PM_TOTAL_ERROR UINT64_MAX

/* ------------------------------------------------------------------ text */

/*
 * pm_encode_text -- text coding of Sec. 2.1 (Table 1: A=00 C=01 G=10 T=11).
 *
 * ascii   n bytes, host or device.  A C G T in either case; any other byte
 *         is an error (PM_E_SYMBOL; pm_last_error() names its offset).
 * n       number of symbols, 0 <= n < 2^32 (larger: PM_E_TOO_LARGE).
 * stream  the copy (for host input) and the coding kernel run on it.
 * out     receives a new handle.  The coded text lives in device memory on
 *         the current device: two bit planes (low and high code bit), 32
 *         symbols per 32-bit word, 2 bits per symbol in total.
 *
 * The call returns after the coding has finished (it synchronises the
 * stream to check the symbols).  Page-locked host input (cudaHostAlloc,
 * torch pin_memory) is read by the coding kernel in place over the host
 * link; other host input is copied in pieces through a device staging
 * buffer.  Either way the ASCII text never has to fit on the device.
 */
pm_status pm_encode_text(const char *ascii, uint64_t n, void *stream, pm_text **out);

/*
 * pm_encode_text_ex -- pm_encode_text with flags.  flags = 0 is
 * pm_encode_text.  PM_TEXT_UNKNOWN_AS_N accepts bytes outside Table 1 (for
 * example N runs in genome files) instead of failing with PM_E_SYMBOL: each
 * becomes an "unknown" symbol, which the pair test matches with the class N
 * only (every other class, and "-", mismatch it).  The paper's text
 * alphabet has the four letters only; this is an extension.  An unknown
 * symbol costs one more bit of device memory per symbol (about 0.39 GB per
 * 3.1 Gbp) for as long as the text holds one; searches of such a text
 * recount the candidate windows exactly, so their results stay exact.
 * Other flags: PM_E_ARG.
 */
#define PM_TEXT_UNKNOWN_AS_N 1u
pm_status pm_encode_text_ex(const char *ascii, uint64_t n, uint32_t flags, void *stream,
                            pm_text **out);

/* Number of unknown symbols of an encoded text (0 unless it was coded with
 * PM_TEXT_UNKNOWN_AS_N). */
uint64_t pm_text_unknown(const pm_text *text);

/* Number of symbols of an encoded text. */
uint64_t pm_text_length(const pm_text *text);
/* How many A, C, G, T (counts[0..3], Table 1 order) the text holds; with
 * pm_text_unknown they sum to its length.  Counted while coding (pm_encode_text); the search uses
 * them to order the positions it tests first (fewest matches first), which
 * changes no result.  PM_E_ARG for NULL arguments. */
pm_status pm_text_letter_counts(const pm_text *text, uint64_t counts[4]);

/*
 * pm_text_save / pm_text_load -- keep a coded text in a file so that a later
 * process skips the coding (0.78 GB per 3.1 Gbp instead of the 3.1 GB ASCII
 * text).  The paper has no counterpart.  The file holds the length, the
 * letter counts, the planes and (if any) the unknown-symbol bits, with a
 * 64-bit checksum (FNV-1a over 64-bit words).  pm_text_load places the text
 * on the current device (copies queued on `stream`, waited for).
 * Errors: PM_E_ARG for NULL arguments, a file that cannot be opened, written
 * or read in full, is not such a file, or fails its checksum (nothing is
 * allocated); PM_E_NOMEM; PM_E_CUDA.
 */
pm_status pm_text_save(const pm_text *text, const char *path);
pm_status pm_text_load(const char *path, void *stream, pm_text **out);

/* Device address and size in bytes of the coded planes (read-only view for
 * callers that want to inspect the layout); either out pointer may be NULL. */
pm_status pm_text_device_planes(const pm_text *text, const void **planes, uint64_t *bytes);

void pm_text_free(pm_text *text);

/* --------------------------------------------------------------- pattern */

/*
 * pm_compile_pattern -- pattern coding of Sec. 2.2 (Table 2).
 *
 * iupac   m bytes (host) over the IUPAC letters A C G T M R W S Y K V H D B N
 *         and "-", either case.  Any other byte is coded 1111 ("-", which
 *         mismatches every letter), as Sec. 2.2 prescribes; the number of
 *         such bytes is reported by pm_pattern_unknown().
 * m       pattern length, 1 <= m <= PM_MAX_PATTERN.
 * out     receives a new handle (host memory only).
 *
 * Each class becomes a 4-bit membership mask obtained from the residue test
 * of Sec. 1.3 (letter a is in class S iff e_a * n_S = 0 mod M, Eq. 1 and
 * Eq. 3), i.e. exactly the rows of Table 3.
 */
#define PM_MAX_PATTERN (1u << 24)
pm_status pm_compile_pattern(const char *iupac, uint32_t m, pm_pattern **out);

uint32_t pm_pattern_length(const pm_pattern *pattern);
uint32_t pm_pattern_unknown(const pm_pattern *pattern);

/* Copy the compiled membership masks to host memory: for chunk c (pattern
 * positions 32c .. 32c+31), out[4c+0..3] are the A, C, G, T words; bit b of
 * the A word is 1 iff A belongs to the class at position 32c+b (Table 3
 * entry 0).  Positions past m read as members of every class.  words must be
 * at least 4*ceil(m/32).  Host only; no device work. */
pm_status pm_pattern_masks(const pm_pattern *pattern, uint32_t *out, uint64_t words);

void pm_pattern_free(pm_pattern *pattern);

/* ---------------------------------------------------------------- search */

/*
 * pm_search -- Eq. 4 for every window of the text and every pattern
 * (Sec. 2.4), the sum stopping once it exceeds k (Sec. 2.4-2.5), the text
 * split into tiles with an m-1 overlap (Sec. 2.6).  One kernel launch per
 * pattern.
 *
 * text      encoded text.
 * patterns  host array of npat compiled patterns (the same handle may
 *           appear several times, e.g. with different k).
 * npat      number of patterns, 0 <= npat <= PM_MAX_BATCH.
 * k         host array of npat values, each >= 0.
 * hits      output, capacity records, host or device.
 * capacity  number of records hits can hold, at most 2^32 - 1.
 * offsets   output, npat+1 values, host or device (same kind as hits).
 *           Pattern p's hits are hits[offsets[p] .. offsets[p+1]), sorted
 *           by location; offsets[npat] is the total.
 * needed    optional host pointer.  When given, the call waits for the
 *           result, stores the total number of hits there and returns
 *           PM_E_OVERFLOW if it exceeds capacity.
 * stream    all device work is ordered on it.
 *
 * With device buffers and needed == NULL the call is asynchronous: it
 * returns once the work is queued, and the caller reads offsets[npat] after
 * the stream to learn the total.  With host buffers the call waits.
 *
 * If the total exceeds capacity, offsets still hold every pattern's count
 * and no hit record is written.  A device-side failure makes offsets[npat]
 * equal PM_TOTAL_ERROR (and the synchronous forms return PM_E_TIMEOUT); the
 * present search kernels have no bounded wait that could raise it, and
 * callers still check for it.
 * Scratch memory is taken from the stream-ordered pool of the current
 * device (cudaMallocAsync) and released on the stream before returning.
 */
#define PM_MAX_BATCH (1u << 16)
pm_status pm_search(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                    const int32_t *k, pm_hit *hits, uint64_t capacity, uint64_t *offsets,
                    uint64_t *needed, void *stream);

/*
 * pm_search_ex -- pm_search with tuning and measurement options.  Results
 * are identical for every choice of options.
 *
 * variant   how Eq. 4 is evaluated with its early stop (Sec. 2.4-2.5):
 *           PM_VARIANT_PATTERN_SLICED    one window per word: positions
 *                                        0..31 by __popc, then the windows
 *                                        still at or below k one by one
 *                                        (k <= 31; larger k run
 *                                        PM_VARIANT_ALL_CHUNKS);
 *           PM_VARIANT_PATTERN_SLICED_2  the same over positions 0..63
 *                                        (k <= 63, else ALL_CHUNKS);
 *           PM_VARIANT_WINDOW_SLICED     32 windows per word, bit-sliced
 *                                        counter position by position
 *                                        (k <= 8; larger k run
 *                                        PM_VARIANT_PATTERN_SLICED's rule);
 *           PM_VARIANT_ALL_CHUNKS        one window per word, running
 *                                        counts 32 positions at a time until
 *                                        every window of a warp is past k;
 *           PM_VARIANT_AUTO              per pattern from k, by the current
 *                                        device's table (pm_set_auto_variants).
 *           Any other value: PM_E_ARG.
 * grid      CTAs per scan launch; 0 means as many as the device keeps
 *           resident at once.
 * events    NULL, or 2*npat cudaEvent_t handles (created by the caller on
 *           the current device); events[2p] and events[2p+1] are recorded on
 *           the stream just before and just after pattern p's scan kernel.
 * batch     NULL: one scan launch per pattern (variant and grid as above).
 *           Otherwise all pairs run in ONE persistent launch as in
 *           pm_batch_create / pm_batch_run with these batch options, the
 *           scratch (about 56 bytes per unit of capacity) taken from the
 *           stream-ordered pool and released on the stream: nothing waits
 *           unless `needed` or host outputs ask for it.  variant, grid and
 *           events are then ignored, except that events must be NULL
 *           (PM_E_ARG).
 */
#define PM_VARIANT_AUTO 0
#define PM_VARIANT_PATTERN_SLICED 1
#define PM_VARIANT_WINDOW_SLICED 2
#define PM_VARIANT_PATTERN_SLICED_2 3
#define PM_VARIANT_ALL_CHUNKS 4
struct pm_batch_options;
typedef struct pm_options {
    int32_t variant;
    int32_t grid;
    void *const *events;
    const struct pm_batch_options *batch;
} pm_options;

pm_status pm_search_ex(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                       const int32_t *k, pm_hit *hits, uint64_t capacity, uint64_t *offsets,
                       uint64_t *needed, const pm_options *options, void *stream);

/*
 * pm_set_auto_variants -- the variant PM_VARIANT_AUTO runs for k = 0 ..
 * nk-1 on the current device (an autotuner measures the candidates and
 * installs the winners).  The paper has no counterpart: it is a choice
 * among equivalent evaluations of Eq. 4, results are identical for every
 * table.
 *
 * variant_for_k  nk PM_VARIANT_* values other than AUTO, each valid for its
 *                k (WINDOW_SLICED needs k <= 8, PATTERN_SLICED k <= 31,
 *                PATTERN_SLICED_2 k <= 63); read during the call only.
 * nk             0..64; 0 restores the built-in table.  k >= nk uses the
 *                built-in choice (k >= 64 always runs ALL_CHUNKS).  A
 *                pattern of m <= 32 given PATTERN_SLICED_2 with k <= 31 runs
 *                PATTERN_SLICED, which decides it exactly in half the work.
 * Returns PM_E_ARG (table unchanged) for nk > 64, a NULL table with nk > 0,
 * or an entry that is AUTO, unknown or not valid for its k; PM_E_CUDA if
 * there is no current device.  Thread-safe; searches already queued keep
 * the variants they were given.
 *
 * pm_get_auto_variants -- the variants PM_VARIANT_AUTO runs on the current
 * device for k = 0 .. nk-1 (nk <= 64; PM_E_ARG otherwise), written to out.
 */
pm_status pm_set_auto_variants(const int32_t *variant_for_k, uint32_t nk);
pm_status pm_get_auto_variants(int32_t *out, uint32_t nk);

/* ----------------------------------------------------------------- batch */

/*
 * Batched search: many (pattern, k) pairs of uneven m and k in ONE
 * persistent kernel launch over the resident text (Eq. 4 with the early
 * stop of Sec. 2.4-2.5, tiles with m-1 overlap as in Sec. 2.6).  Each text
 * tile is staged once for every pattern of a work item's row, so the text is
 * read from device memory once per row (by default one row per kind of
 * evaluation).  Results are identical to pm_search's for the same pairs.
 *
 * pm_batch_create  copies the patterns' compiled data and k to the device
 *                  and allocates all scratch for up to `capacity` hits
 *                  (cudaMalloc; about 56 bytes per unit of capacity).  The
 *                  pattern handles may be freed afterwards; the text must
 *                  outlive the batch.  Waits for its uploads.
 * options          NULL for defaults, or (0 in any field: its default):
 *                    group      accepted for compatibility and not used
 *                               (a work item row is one group of 8 pairs);
 *                    grid       CTAs of each persistent launch (default: as
 *                               many as the device keeps resident);
 *                    tiles      warp tiles per work item, 1..64 (default 16;
 *                               a tile is 8192 windows for window-sliced
 *                               pairs, 4096 for the others);
 *                    ws_below   pairs with k < ws_below are evaluated
 *                               window-sliced, 1..9 (default 9; -1: none);
 *                    ps1_below  other pairs with k < ps1_below are evaluated
 *                               pattern-sliced over positions 0..31, their
 *                               survivors then counted exactly, 1..32
 *                               (default 18; -1: none);
 *                    ps2_below  other pairs with k < ps2_below over
 *                               positions 0..63, 1..64 (default 41; -1:
 *                               none); the remaining pairs count every
 *                               chunk until a warp's windows are past k.
 *                  Out-of-range values: PM_E_ARG.  Results are identical for
 *                  every choice of options; an autotuner picks them.
 * pm_batch_run     runs the batch into device buffers: hits (capacity
 *                  records) and offsets (npat+1; pattern p's hits are
 *                  hits[offsets[p] .. offsets[p+1]), sorted by location;
 *                  offsets[npat] is the total, PM_TOTAL_ERROR after a
 *                  device-side failure).  If the total exceeds capacity no
 *                  hit is written.  It allocates nothing and does not wait:
 *                  all work is queued on `stream`, so the call may be
 *                  captured in a CUDA graph and replayed.  Runs of one batch
 *                  must not overlap on the GPU (they share its scratch).
 */
typedef struct pm_batch_options {
    int32_t group;
    int32_t grid;
    int32_t tiles;
    int32_t ws_below;
    int32_t ps1_below;
    int32_t ps2_below;
} pm_batch_options;

pm_status pm_batch_create(const pm_text *text, const pm_pattern *const *patterns, uint32_t npat,
                          const int32_t *k, uint64_t capacity, const pm_batch_options *options,
                          void *stream, pm_batch **out);
pm_status pm_batch_run(pm_batch *batch, pm_hit *hits, uint64_t *offsets, void *stream);
uint64_t pm_batch_capacity(const pm_batch *batch);
void pm_batch_free(pm_batch *batch);

/*
 * pm_search_noalloc -- pm_search for callers that must not allocate memory.
 * The paper has no counterpart: this is a deployment concern, not part of
 * the method.
 *
 * Who needs it: code that runs where calling the CUDA allocator is not
 * allowed or not wanted, for example a real-time loop that may not take the
 * allocator's locks or its implicit synchronisation, or an application that
 * has already handed all of its device memory to its own allocator.
 * pm_search draws its scratch from the stream-ordered pool and a pinned host
 * ring; this entry point draws it from one fixed array (about 64 MiB) that
 * the library declares in device global memory.  Every GPU that loads the
 * library holds that array until the process exits.  The call performs no
 * cudaMalloc, cudaMallocAsync, cudaHostAlloc or free of any kind.  It does
 * issue copies, memsets and kernel launches, and waits for the stream when
 * `needed` is given, so it cannot run where CUDA may not be called at all,
 * such as inside a host callback (cudaLaunchHostFunc).
 *
 * Arguments are those of pm_search, except that hits and offsets must be
 * device memory (PM_E_ARG otherwise).  Results are identical to pm_search's.
 *
 * Limits (PM_E_TOO_LARGE beyond them, nothing queued): at most 64 (pattern,
 * k) pairs, at most 4096 32-position chunks over the distinct patterns
 * (e.g. m up to 131072 for one pattern), at most 2^21 warp tiles over all
 * pairs (a tile is 8192 windows for a window-sliced pair, k <= 8, else
 * 4096; e.g. 8.6e9 windows for one pattern with k > 8), capacity at most
 * 2^22 hits.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture.  The address is kept for the life of the
 * process, so do not use this entry point on a device after resetting it
 * (cudaDeviceReset).  All calls share the array and it keeps the
 * previous call's contents (the call clears what has to start at zero):
 * calls whose work overlaps on the GPU, such as calls on two streams or from
 * two threads, race with each other.  Issue them on one stream.
 */
pm_status pm_search_noalloc(const pm_text *text, const pm_pattern *const *patterns,
                            uint32_t npat, const int32_t *k, pm_hit *hits, uint64_t capacity,
                            uint64_t *offsets, uint64_t *needed, void *stream);

/* ----------------------------------------------------------- measurement */

/*
 * pm_check_bounded_wait -- failure detection, checked without a fault.  The
 * paper has no counterpart.  The search kernels hold no spin wait: their
 * copies are per-lane cp.async, completed by cp.async.wait_group.  Any
 * kernel of this library that waits on a shared-memory barrier (an mbarrier
 * completed by a bulk copy) must use the bounded form, which gives up after
 * a time limit, sets the device status bit that turns offsets[npat] into
 * PM_TOTAL_ERROR, and returns, so a lost copy ends as PM_E_TIMEOUT instead
 * of a hung GPU.  This entry point runs that bounded wait once, in a
 * one-warp kernel, on a barrier that receives its arrival only if `arrive`
 * is nonzero, with the given limit (1 ns .. 10 s; PM_E_ARG otherwise), and
 * reports through *timed_out whether the wait gave up (1) or completed (0).
 * Nothing is left pending on the device either way.
 */
pm_status pm_check_bounded_wait(uint64_t limit_ns, int32_t arrive, uint32_t *timed_out);

/*
 * pm_measure_int_pipe -- throughput of one integer instruction kind on the
 * current device, for the ALU roofline of the scan kernels.  The paper has
 * no counterpart (its timings are of a CPU program).
 *
 * op        0 LOP3 (three-input logic), 1 SHF (funnel shift), 2 POPC,
 *           3 IMAD (integer multiply-add); the integer tensor-core forms of
 *           sm_103a: 4 mma.sync m16n8k32 s8 x s8 -> s32, 5 mma.sync
 *           m16n8k256 b1 AND-popcount -> s32, 6 the same with k = 128 (the
 *           1-bit form counts set bits of row AND column: with one-hot text
 *           rows and class-mask columns, Eq. 4's matches over K/4 positions).
 * iters     loop trips per thread (each trip issues 8 instructions of the kind).
 * Outputs   instructions per second over the whole GPU (for ops 4..6:
 *           operations, 2 x M x N x K per warp-wide MMA); the SM clock during
 *           the run in MHz (cycle counter against the global timer); and the
 *           same per clock per SM (per-thread instructions: 32 per warp
 *           instruction).  Allocates a small buffer; synchronises.
 */
pm_status pm_measure_int_pipe(int32_t op, uint32_t iters, double *ops_per_s, double *sm_mhz,
                              double *ops_per_clk_per_sm);

/* ---------------------------------------------------------------- status */

const char *pm_status_string(pm_status status);
const char *pm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PM_H */
