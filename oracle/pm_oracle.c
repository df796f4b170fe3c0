/*
 * Oracle for k-mismatch pattern matching with character classes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the package entry point's smoke check and
 * the CPU-baseline leg of the benchmark use it.  It shares no code, header
 * or table with the CUDA path.
 *
 * It is the plain, slow statement of the method of "Fast low-level pattern
 * matching algorithm" (Soldo, Krzic, Sersic, arXiv 1611.06115), evaluated in
 * the paper's own order and notation:
 *
 *   Table 1  text symbol -> 2-bit code           (Sec. 2.1)
 *   Table 2  pattern class -> 4-bit code         (Sec. 2.2)
 *   Table 3  dictionary L[64]: 0 match, 1 miss   (Sec. 2.3)
 *   index    l = (p[j] << 2) OR t[i+j-1]         (Sec. 2.3, steps 1-3)
 *   Eq. 4    location i is reported iff
 *            sum_{j=1..m} L[(p[j] << 2) OR t[i+j-1]] <= k
 *            (Sec. 2.4); the sum may stop as soon as it exceeds k
 *            (Sec. 2.4 for k = 0, Sec. 2.5 for general k).
 *   Sec. 2.6 the text is cut into one piece per thread, consecutive pieces
 *            overlapping by m-1 symbols, each piece searched on its own.
 *
 * Conventions (readings of the paper that it leaves open):
 *   - Locations are 0-based here; the paper's location i is ours + 1.
 *   - There are n-m+1 windows; none is partial.  m > n gives no window.
 *   - k is inclusive ("<= k" in Eq. 4); k >= m reports every window.
 *   - Lower-case letters are read as upper case.  A pattern symbol not in
 *     Table 2 takes the code 1111 ("-"), as Sec. 2.2 prescribes.  A text
 *     symbol outside Table 1 is an error (the paper's text alphabet has
 *     four letters only).
 *
 * Parity pins (checked by tests, not by this file): the worked examples of
 * Sec. 1.1 and Sec. 2.5 / Table 4, Table 3 against the class column of
 * Table 2 and against the prime-product test of Sec. 1.3 (Eq. 1-3), brute
 * force on tiny inputs, and invariants (monotone in k, chunk-split
 * invariance of Sec. 2.6, all-N and all-"-" patterns).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_ARG (-1)
#define ORACLE_E_SYMBOL (-2)
#define ORACLE_E_OVERFLOW (-3)
#define ORACLE_E_NOMEM (-4)

/* Table 1: A=00, C=01, G=10, T=11.  Returns -1 for any other symbol. */
int oracle_text_code(int ch)
{
    switch (ch) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

/* Table 2: the fifteen IUPAC classes and "-", in the table's order.
 * Unknown or erroneous symbols are coded 1111 (Sec. 2.2). */
int oracle_pattern_code(int ch)
{
    static const char order[16] = {'A', 'C', 'G', 'T', 'M', 'R', 'W', 'S',
                                   'Y', 'K', 'V', 'H', 'D', 'B', 'N', '-'};
    if (ch >= 'a' && ch <= 'z') ch = ch - 'a' + 'A';
    for (int c = 0; c < 16; ++c)
        if (order[c] == ch) return c;
    return 15;
}

/* Table 3: the pair dictionary L, row = pattern code (Table 2 order),
 * column = text code (Table 1 order), entry (row << 2 | column). */
static const uint8_t L[64] = {
    /* A */ 0, 1, 1, 1,
    /* C */ 1, 0, 1, 1,
    /* G */ 1, 1, 0, 1,
    /* T */ 1, 1, 1, 0,
    /* M */ 0, 0, 1, 1,
    /* R */ 0, 1, 0, 1,
    /* W */ 0, 1, 1, 0,
    /* S */ 1, 0, 0, 1,
    /* Y */ 1, 0, 1, 0,
    /* K */ 1, 1, 0, 0,
    /* V */ 0, 0, 0, 1,
    /* H */ 0, 0, 1, 0,
    /* D */ 0, 1, 0, 0,
    /* B */ 1, 0, 0, 0,
    /* N */ 0, 0, 0, 0,
    /* - */ 1, 1, 1, 1,
};

const uint8_t *oracle_table3(void) { return L; }

/* Sec. 2.3, steps 1-2: r[j] = p[j] << 2, then l = r[j] OR t[i]. */
int oracle_lindex(int pcode, int tcode) { return (pcode << 2) | tcode; }

/* Steps 1 and 2 of Sec. 2.5: code a text piece with Table 1.
 * Returns the offset of the first symbol outside Table 1, or -1. */
static int64_t code_text(const char *t, uint64_t len, uint8_t *out)
{
    for (uint64_t i = 0; i < len; ++i) {
        int c = oracle_text_code((unsigned char)t[i]);
        if (c < 0) return (int64_t)i;
        out[i] = (uint8_t)c;
    }
    return -1;
}

/* Step 2 and 3 of Sec. 2.5: code the pattern with Table 2 and shift it:
 * r[j] = p[j] << 2.  Returns how many symbols were not in Table 2. */
static uint32_t code_pattern_shifted(const char *p, uint32_t m, uint8_t *r)
{
    static const char known[] = "ACGTMRWSYKVHDBN-acgtmrwsykvhdbn";
    uint32_t unknown = 0;
    for (uint32_t j = 0; j < m; ++j) {
        int ch = (unsigned char)p[j];
        if (ch == 0 || strchr(known, ch) == NULL) ++unknown;
        r[j] = (uint8_t)(oracle_pattern_code(ch) << 2);
    }
    return unknown;
}

/* Eq. 4 for one window: sum of L[r[j] OR t[i+j]] over the pattern.
 * With early_exit the sum stops once it exceeds k; the value returned is
 * then some number > k (not the full count). */
static uint64_t window_sum(const uint8_t *r, uint32_t m, const uint8_t *tc,
                           int64_t k, int early_exit)
{
    uint64_t s = 0;
    for (uint32_t j = 0; j < m; ++j) {
        s += L[r[j] | tc[j]];
        if (early_exit && (int64_t)s > k) break;
    }
    return s;
}

/* The steps of Sec. 2.5 (step 4) for one window, recorded: the indices l
 * looked up, in order, until the end of the pattern or, with early_exit,
 * until the running sum exceeds k.  Returns how many were looked up, or a
 * negative error.  l_out and v_out must hold m entries. */
int oracle_window_trace(const char *t, uint64_t n, const char *p, uint32_t m,
                        uint64_t i, int64_t k, int early_exit,
                        int32_t *l_out, int32_t *v_out)
{
    if (m == 0 || i + m > n) return ORACLE_E_ARG;
    uint8_t *r = (uint8_t *)malloc(m);
    uint8_t *tc = (uint8_t *)malloc(m);
    if (!r || !tc) { free(r); free(tc); return ORACLE_E_NOMEM; }
    code_pattern_shifted(p, m, r);
    if (code_text(t + i, m, tc) >= 0) { free(r); free(tc); return ORACLE_E_SYMBOL; }
    int64_t s = 0;
    int cnt = 0;
    for (uint32_t j = 0; j < m; ++j) {
        int l = r[j] | tc[j];
        l_out[cnt] = l;
        v_out[cnt] = L[l];
        ++cnt;
        s += L[l];
        if (early_exit && s > k) break;
    }
    free(r); free(tc);
    return cnt;
}

int oracle_count_unknown(const char *p, uint32_t m)
{
    uint8_t *r = (uint8_t *)malloc(m ? m : 1);
    if (!r) return ORACLE_E_NOMEM;
    uint32_t u = code_pattern_shifted(p, m, r);
    free(r);
    return (int)u;
}

/* Full mismatch counts (no early exit) for windows 0..n-m.
 * out must hold n-m+1 entries.  For small inputs. */
int oracle_counts(const char *t, uint64_t n, const char *p, uint32_t m,
                  uint32_t *out, int64_t *bad_pos)
{
    if (m == 0) return ORACLE_E_ARG;
    if (bad_pos) *bad_pos = -1;
    uint8_t *tc = (uint8_t *)malloc(n ? n : 1);
    uint8_t *r = (uint8_t *)malloc(m);
    if (!tc || !r) { free(tc); free(r); return ORACLE_E_NOMEM; }
    int64_t bad = code_text(t, n, tc);
    if (bad >= 0) {
        if (bad_pos) *bad_pos = bad;
        free(tc); free(r);
        return ORACLE_E_SYMBOL;
    }
    code_pattern_shifted(p, m, r);
    if (m <= n)
        for (uint64_t i = 0; i + m <= n; ++i)
            out[i] = (uint32_t)window_sum(r, m, tc + i, 0, 0);
    free(tc); free(r);
    return ORACLE_OK;
}

/* Full counts at chosen window locations (for sampled checks on large
 * texts).  Each location must satisfy loc + m <= n. */
int oracle_counts_at(const char *t, uint64_t n, const char *p, uint32_t m,
                     const uint64_t *locs, uint64_t nlocs, uint32_t *out)
{
    if (m == 0) return ORACLE_E_ARG;
    uint8_t *r = (uint8_t *)malloc(m);
    uint8_t *tc = (uint8_t *)malloc(m);
    if (!r || !tc) { free(r); free(tc); return ORACLE_E_NOMEM; }
    code_pattern_shifted(p, m, r);
    for (uint64_t q = 0; q < nlocs; ++q) {
        uint64_t i = locs[q];
        if (i + m > n || code_text(t + i, m, tc) >= 0) {
            free(r); free(tc);
            return ORACLE_E_ARG;
        }
        out[q] = (uint32_t)window_sum(r, m, tc, 0, 0);
    }
    free(r); free(tc);
    return ORACLE_OK;
}

/* ---- Sec. 2.6: one piece per thread, pieces overlapping by m-1 ---- */

typedef struct {
    const char *t;
    const uint8_t *r;
    uint32_t m;
    int64_t k;
    int early_exit;
    uint64_t w0, w1;   /* windows [w0, w1) of this piece */
    uint32_t *loc;     /* hits found, grown on demand */
    uint32_t *mm;
    uint64_t nhits, cap;
    int64_t bad;       /* absolute offset of a bad text symbol, or -1 */
    int err;
} piece_t;

static int piece_push(piece_t *pc, uint64_t i, uint64_t s)
{
    if (pc->nhits == pc->cap) {
        uint64_t nc = pc->cap ? pc->cap * 2 : 1024;
        uint32_t *a = (uint32_t *)realloc(pc->loc, nc * sizeof(uint32_t));
        if (!a) return ORACLE_E_NOMEM;
        pc->loc = a;
        uint32_t *b = (uint32_t *)realloc(pc->mm, nc * sizeof(uint32_t));
        if (!b) return ORACLE_E_NOMEM;
        pc->mm = b;
        pc->cap = nc;
    }
    pc->loc[pc->nhits] = (uint32_t)i;
    pc->mm[pc->nhits] = (uint32_t)s;
    pc->nhits++;
    return ORACLE_OK;
}

static void *piece_run(void *arg)
{
    piece_t *pc = (piece_t *)arg;
    pc->bad = -1;
    pc->err = ORACLE_OK;
    if (pc->w1 <= pc->w0) return NULL;
    /* the piece of text this thread reads: its windows plus m-1 symbols */
    uint64_t len = (pc->w1 - pc->w0) + pc->m - 1;
    uint8_t *tc = (uint8_t *)malloc(len);
    if (!tc) { pc->err = ORACLE_E_NOMEM; return NULL; }
    int64_t bad = code_text(pc->t + pc->w0, len, tc);
    if (bad >= 0) {
        pc->bad = (int64_t)pc->w0 + bad;
        pc->err = ORACLE_E_SYMBOL;
        free(tc);
        return NULL;
    }
    for (uint64_t i = pc->w0; i < pc->w1; ++i) {
        uint64_t s = window_sum(pc->r, pc->m, tc + (i - pc->w0), pc->k,
                                pc->early_exit);
        if ((int64_t)s <= pc->k) {
            int e = piece_push(pc, i, s);
            if (e) { pc->err = e; break; }
        }
    }
    free(tc);
    return NULL;
}

/*
 * Reports every 0-based location i (i + m <= n) whose Eq. 4 sum is <= k,
 * in increasing order, with its exact mismatch count.  The window range
 * is split into nthreads pieces (Sec. 2.6).  split_at, if non-NULL, gives
 * nthreads-1 explicit piece boundaries (window indices, increasing) so
 * that tests can cut the text at any point.
 *
 * Returns ORACLE_OK, ORACLE_E_OVERFLOW (more than cap hits; *nhits is
 * the number needed and nothing else is valid), ORACLE_E_SYMBOL (*bad_pos
 * is the first bad text offset found), ORACLE_E_ARG or ORACLE_E_NOMEM.
 */
int oracle_search(const char *t, uint64_t n, const char *p, uint32_t m,
                  int64_t k, int early_exit, int nthreads,
                  const uint64_t *split_at, uint32_t *loc, uint32_t *mm,
                  uint64_t cap, uint64_t *nhits, int64_t *bad_pos)
{
    if (m == 0 || k < 0 || nthreads <= 0 || nhits == NULL) return ORACLE_E_ARG;
    *nhits = 0;
    if (bad_pos) *bad_pos = -1;
    /* a bad symbol anywhere in the text is an error, even where no window
     * covers it (m > n); check the part no piece reads */
    if (m > n) {
        uint8_t tmp;
        for (uint64_t i = 0; i < n; ++i)
            if (code_text(t + i, 1, &tmp) >= 0) {
                if (bad_pos) *bad_pos = (int64_t)i;
                return ORACLE_E_SYMBOL;
            }
        return ORACLE_OK;
    }
    uint64_t nwin = n - m + 1;
    uint8_t *r = (uint8_t *)malloc(m);
    piece_t *pcs = (piece_t *)calloc((size_t)nthreads, sizeof(piece_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!r || !pcs || !th) { free(r); free(pcs); free(th); return ORACLE_E_NOMEM; }
    code_pattern_shifted(p, m, r);

    for (int q = 0; q < nthreads; ++q) {
        uint64_t a, b;
        if (split_at) {
            a = q == 0 ? 0 : split_at[q - 1];
            b = q == nthreads - 1 ? nwin : split_at[q];
            if (a > nwin) a = nwin;
            if (b > nwin) b = nwin;
        } else {
            a = nwin * (uint64_t)q / (uint64_t)nthreads;
            b = nwin * (uint64_t)(q + 1) / (uint64_t)nthreads;
        }
        pcs[q].t = t; pcs[q].r = r; pcs[q].m = m; pcs[q].k = k;
        pcs[q].early_exit = early_exit;
        pcs[q].w0 = a; pcs[q].w1 = b;
    }
    int started = 0;
    for (int q = 1; q < nthreads; ++q) {
        if (pthread_create(&th[q], NULL, piece_run, &pcs[q]) != 0) break;
        started = q;
    }
    piece_run(&pcs[0]);
    /* any piece whose thread did not start runs here */
    for (int q = started + 1; q < nthreads; ++q) piece_run(&pcs[q]);
    for (int q = 1; q <= started; ++q) pthread_join(th[q], NULL);

    /* the pieces' text ranges cover [0, n) together */
    int rc = ORACLE_OK;
    int64_t first_bad = -1;
    for (int q = 0; q < nthreads; ++q) {
        if (pcs[q].err == ORACLE_E_SYMBOL &&
            (first_bad < 0 || pcs[q].bad < first_bad))
            first_bad = pcs[q].bad;
        else if (pcs[q].err && rc == ORACLE_OK)
            rc = pcs[q].err;
    }
    if (first_bad >= 0) {
        if (bad_pos) *bad_pos = first_bad;
        rc = ORACLE_E_SYMBOL;
    }
    uint64_t total = 0;
    for (int q = 0; q < nthreads; ++q) total += pcs[q].nhits;
    if (rc == ORACLE_OK) {
        *nhits = total;
        if (total > cap) {
            rc = ORACLE_E_OVERFLOW;
        } else {
            uint64_t o = 0;
            for (int q = 0; q < nthreads; ++q) {
                if (pcs[q].nhits) {
                    memcpy(loc + o, pcs[q].loc, pcs[q].nhits * sizeof(uint32_t));
                    memcpy(mm + o, pcs[q].mm, pcs[q].nhits * sizeof(uint32_t));
                }
                o += pcs[q].nhits;
            }
        }
    }
    for (int q = 0; q < nthreads; ++q) { free(pcs[q].loc); free(pcs[q].mm); }
    free(r); free(pcs); free(th);
    return rc;
}

/* ---- Text symbols outside Table 1 --------------------------------------
 * An extension the paper does not cover: its text alphabet has the four
 * letters of Table 1, while genome files also carry N (and other letters)
 * for bases that are not known.  Reading taken: such a text symbol is
 * "unknown" (code 4 here); the pair test of an unknown text symbol with a
 * pattern class is a match only for N, the class that holds every letter,
 * and a mismatch for every other class and for "-".  Known symbols use
 * Table 3 as before. */
#define TEXT_UNKNOWN 4

static uint8_t code_text_u(int ch)
{
    int c = oracle_text_code(ch);
    return (uint8_t)(c < 0 ? TEXT_UNKNOWN : c);
}

/* r = p << 2 as in Sec. 2.3; N is code 14 of Table 2 */
static uint32_t pair_u(uint8_t r, uint8_t tc)
{
    if (tc == TEXT_UNKNOWN) return (r >> 2) == 14 ? 0u : 1u;
    return L[r | tc];
}

/* Full counts for windows 0..n-m of a text that may hold unknown symbols.
 * out must hold n-m+1 entries.  For small inputs. */
int oracle_counts_unknown_text(const char *t, uint64_t n, const char *p, uint32_t m,
                               uint32_t *out)
{
    if (m == 0) return ORACLE_E_ARG;
    uint8_t *tc = (uint8_t *)malloc(n ? n : 1);
    uint8_t *r = (uint8_t *)malloc(m);
    if (!tc || !r) { free(tc); free(r); return ORACLE_E_NOMEM; }
    for (uint64_t i = 0; i < n; ++i) tc[i] = code_text_u((unsigned char)t[i]);
    code_pattern_shifted(p, m, r);
    if (m <= n)
        for (uint64_t i = 0; i + m <= n; ++i) {
            uint32_t s = 0;
            for (uint32_t j = 0; j < m; ++j) s += pair_u(r[j], tc[i + j]);
            out[i] = s;
        }
    free(tc); free(r);
    return ORACLE_OK;
}

/* Eq. 4 with the early stop over a text that may hold unknown symbols: the
 * 0-based locations whose sum is <= k, in order, with their sums (one
 * thread).  Returns ORACLE_E_OVERFLOW with *nhits = the number needed when
 * it exceeds cap. */
int oracle_search_unknown_text(const char *t, uint64_t n, const char *p, uint32_t m, int64_t k,
                               uint32_t *loc, uint32_t *mm, uint64_t cap, uint64_t *nhits)
{
    if (m == 0 || k < 0 || nhits == NULL) return ORACLE_E_ARG;
    *nhits = 0;
    if (m > n) return ORACLE_OK;
    uint8_t *tc = (uint8_t *)malloc(n);
    uint8_t *r = (uint8_t *)malloc(m);
    if (!tc || !r) { free(tc); free(r); return ORACLE_E_NOMEM; }
    for (uint64_t i = 0; i < n; ++i) tc[i] = code_text_u((unsigned char)t[i]);
    code_pattern_shifted(p, m, r);
    uint64_t h = 0;
    for (uint64_t i = 0; i + m <= n; ++i) {
        int64_t s = 0;
        uint32_t j = 0;
        for (; j < m; ++j) {
            s += pair_u(r[j], tc[i + j]);
            if (s > k) break;
        }
        if (s <= k) {
            if (h < cap) { loc[h] = (uint32_t)i; mm[h] = (uint32_t)s; }
            ++h;
        }
    }
    free(tc); free(r);
    *nhits = h;
    return h > cap ? ORACLE_E_OVERFLOW : ORACLE_OK;
}
