/*
 * bsort oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the bsort method
 * (Guzman, "bsort: a theoretically efficient non-comparison-based sorting
 * algorithm for integer and floating-point numbers"), written from the
 * paper's text.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library; the product (the CUDA library)
 * neither links nor calls it, and shares no code with it.
 *
 * Keys are passed as uint64_t words holding the raw w-bit pattern of each
 * element in the low w bits (upper bits zero), so one implementation covers
 * every word size, including the 3-, 4- and 6-bit examples of the paper.
 *
 * Readings of the paper where it is silent, ambiguous or at odds with itself:
 *   R1 (Alg. 1 bounds)   ranges are half-open [ps, pe), 0 <= ps <= pe <= n.
 *   R2 (Alg. 4 vs text)  the negative half is sorted in the inverted
 *                        direction on its exponent and mantissa bits, as the
 *                        three-pass rule of Sec. III-B, Thm. 3 and Fig. 4
 *                        require; `literal_alg4` keeps the printed form
 *                        (same direction on both halves) as a negative test.
 *   R3 (Alg. 2 base)     a partition of at most one element returns at once.
 *   R4 (mask shifts)     masks are unsigned w-bit words, all shifts logical.
 *   R5 (Alg. 5 split)    the exponent/mantissa switch is kept literally.
 *   R6 (NaN, -0, subnormals) raw-bit handling, no canonicalisation.
 *
 * The definition side (`orc_cmp_total`) restates the order the method must
 * reach -- numeric order, -0 < +0, NaNs at the two ends ordered by their
 * mantissa field -- without using the bit partition, so the two can pin
 * each other.
 *
 * Key-value sorting (not in the paper) is defined here by its plain meaning:
 * `orc_stable_argsort` orders the input positions by the definition order of
 * their keys, equal keys (bit-identical) in input order -- a stable sort, so
 * the permutation is unique and values carried along it are fixed.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Mutation points: the pin tests rebuild the oracle with ORC_PLANT set to one
 * of the numbers below and check that some pin catches each planted mistake.
 * The default build (ORC_PLANT == 0) contains none of them. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

enum { ORC_UNSIGNED = 0, ORC_SIGNED = 1, ORC_FLOAT = 2 };
enum { ORC_LITERAL = 0, ORC_STABLE = 1 };

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,   /* bad width / kind / field sizes */
    ORC_ERR_BITS = 2,  /* a key has bits set above bit w-1 */
    ORC_ERR_MEM = 3
};

typedef struct {
    int mode;             /* ORC_LITERAL: the swap loop of Alg. 1; ORC_STABLE: order-keeping split */
    int check;            /* verify invariants (i)/(ii) after every partition */
    int max_levels;       /* stop after this many bit levels (<= 0: all) */
    int literal_alg4;     /* Alg. 4 exactly as printed (negative test of R2) */
    int mant_bits;        /* f: mantissa width, used by Alg. 5 */
    uint64_t violations;  /* out: invariant violations seen */
    uint64_t partitions;  /* out: partition calls made */
    uint64_t *tmp;        /* scratch for the stable split */
} orc_ctx;

/* Alg. 1 (singlePassBSort): one partition of a[ps, pe) on the single-bit mask
 * m.  Elements whose masked bit is 0 (asc) or 1 (desc) go to the front; the
 * returned k separates the two sides, which then satisfy invariants (i)/(ii)
 * of Sec. II for mask m. */
static size_t single_pass(orc_ctx *c, uint64_t *a, uint64_t m, size_t ps, size_t pe, int asc)
{
    size_t k = ps;
    c->partitions++;
    if (c->mode == ORC_LITERAL) {
        for (size_t i = ps; i < pe; i++) {
            int bit = (a[i] & m) != 0;
            if ((asc && !bit) || (!asc && bit)) {
                uint64_t t = a[i];
                a[i] = a[k];
                a[k] = t;
                k++;
            }
        }
    } else {
        /* Same split, but both sides keep their input order (the rows printed
         * in Figs. 1, 2 and 4 follow this order). */
        size_t t = 0;
        for (size_t i = ps; i < pe; i++) {
            int bit = (a[i] & m) != 0;
            if ((asc && !bit) || (!asc && bit)) c->tmp[t++] = a[i];
        }
        k = ps + t;
#if ORC_PLANT == 7
        for (size_t i = pe; i-- > ps;) {
#else
        for (size_t i = ps; i < pe; i++) {
#endif
            int bit = (a[i] & m) != 0;
            if (!((asc && !bit) || (!asc && bit))) c->tmp[t++] = a[i];
        }
        memcpy(a + ps, c->tmp, (pe - ps) * sizeof(uint64_t));
    }
    if (c->check) {
        /* front side: bit == 0 (asc) / bit == 1 (desc); back side: the other */
        for (size_t i = ps; i < k; i++) {
            int bit = (a[i] & m) != 0;
            if (bit != !asc) c->violations++;
        }
        for (size_t j = k; j < pe; j++) {
            int bit = (a[j] & m) != 0;
            if (bit != asc) c->violations++;
        }
    }
    return k;
}

static int level_done(const orc_ctx *c, int level)
{
    return c->max_levels > 0 && level >= c->max_levels;
}

/* Alg. 2 (binaryQuickSort): partition on m, then recurse on both sides with
 * the next lower bit until the mask is exhausted.  `level` counts the bit
 * levels processed so far including this one. */
static void binary_quicksort(orc_ctx *c, uint64_t *a, uint64_t m, size_t ps, size_t pe, int asc, int level)
{
    if (pe - ps <= 1) return; /* R3 */
    size_t k = single_pass(c, a, m, ps, pe, asc);
    uint64_t m2 = m >> 1; /* R4: logical shift */
    if (m2 == 0 || level_done(c, level)) return;
    binary_quicksort(c, a, m2, ps, k, asc, level + 1);
#if ORC_PLANT == 2
    binary_quicksort(c, a, m2 >> 1, k, pe, asc, level + 1);
#else
    binary_quicksort(c, a, m2, k, pe, asc, level + 1);
#endif
}

/* Alg. 5 (bsortF): one partition per exponent bit; once the mask reaches the
 * lowest exponent bit (m == 1 << f), the mantissa is sorted by Alg. 2. */
static void bsort_f(orc_ctx *c, uint64_t *a, uint64_t m, size_t ps, size_t pe, int asc, int level)
{
    if (pe - ps <= 1) return; /* R3 */
    size_t k = single_pass(c, a, m, ps, pe, asc);
    if (level_done(c, level)) return;
    uint64_t m2 = m >> 1;
    if (m == ((uint64_t)1 << c->mant_bits)) {
        if (m2 == 0) return; /* no mantissa bits */
        binary_quicksort(c, a, m2, ps, k, asc, level + 1);
        binary_quicksort(c, a, m2, k, pe, asc, level + 1);
        return;
    }
    bsort_f(c, a, m2, ps, k, asc, level + 1);
    bsort_f(c, a, m2, k, pe, asc, level + 1);
}

/* Unsigned keys: Alg. 2 from the most significant bit. */
static void bsort_unsigned(orc_ctx *c, uint64_t *a, size_t n, int w, int asc)
{
    binary_quicksort(c, a, (uint64_t)1 << (w - 1), 0, n, asc, 1);
}

/* Alg. 3 (bsortSigned): the sign-bit pass runs in the inverted direction,
 * then both halves are sorted on the remaining bits in the requested one. */
static void bsort_signed(orc_ctx *c, uint64_t *a, size_t n, int w, int asc)
{
    if (n <= 1) return;
    uint64_t m = (uint64_t)1 << (w - 1);
#if ORC_PLANT == 1
    size_t k = single_pass(c, a, m, 0, n, asc);
#else
    size_t k = single_pass(c, a, m, 0, n, !asc);
#endif
    uint64_t m2 = m >> 1;
    if (m2 == 0 || level_done(c, 1)) return;
    binary_quicksort(c, a, m2, 0, k, asc, 2);
    binary_quicksort(c, a, m2, k, n, asc, 2);
}

/* Alg. 4 (bsortFloat) with reading R2: sign pass in the inverted direction;
 * the negative half then runs Alg. 5 with the inverted direction and the
 * non-negative half with the requested one.  The sign pass puts negatives
 * first for an ascending sort and last for a descending one. */
static void bsort_float(orc_ctx *c, uint64_t *a, size_t n, int w, int asc)
{
    if (n <= 1) return;
    uint64_t m = (uint64_t)1 << (w - 1);
    size_t k = single_pass(c, a, m, 0, n, !asc);
    uint64_t m2 = m >> 1;
    if (m2 == 0 || level_done(c, 1)) return;
    int neg_dir = c->literal_alg4 ? asc : !asc;
    if (asc) {
        bsort_f(c, a, m2, 0, k, neg_dir, 2);  /* negatives */
        bsort_f(c, a, m2, k, n, asc, 2);      /* non-negatives */
    } else {
        bsort_f(c, a, m2, 0, k, asc, 2);      /* non-negatives */
        bsort_f(c, a, m2, k, n, neg_dir, 2);  /* negatives */
    }
}

static int check_format(int w, int kind, int e_bits, int f_bits)
{
    if (w < 1 || w > 64) return ORC_ERR_ARG;
    if (kind == ORC_FLOAT) {
        if (e_bits < 1 || f_bits < 0 || e_bits + f_bits + 1 != w) return ORC_ERR_ARG;
        if (e_bits > 11 || f_bits > 52) return ORC_ERR_ARG; /* value() is exact in double only up to binary64 */
    } else if (kind != ORC_UNSIGNED && kind != ORC_SIGNED) {
        return ORC_ERR_ARG;
    }
    return ORC_OK;
}

static int check_bits(const uint64_t *a, size_t n, int w)
{
    if (w == 64) return ORC_OK;
    uint64_t hi = ~(((uint64_t)1 << w) - 1);
    for (size_t i = 0; i < n; i++)
        if (a[i] & hi) return ORC_ERR_BITS;
    return ORC_OK;
}

/* Sorts a[0, n) in place with the method of Algs. 1-5.
 *   w, kind, e_bits, f_bits  word size, key kind and (floats) field widths
 *   asc                      1 ascending, 0 descending
 *   mode                     ORC_LITERAL or ORC_STABLE partition
 *   max_levels               stop after this many bit levels (<= 0: all);
 *                            the state then equals the row printed after that
 *                            many masks in the paper's traces (stable mode)
 *   literal_alg4, check      see orc_ctx
 *   stats_out (may be NULL)  [0] invariant violations, [1] partition calls
 */
int orc_bsort(uint64_t *a, size_t n, int w, int kind, int e_bits, int f_bits, int asc,
              int mode, int max_levels, int literal_alg4, int check, uint64_t *stats_out)
{
    int st = check_format(w, kind, e_bits, f_bits);
    if (st != ORC_OK) return st;
    st = check_bits(a, n, w);
    if (st != ORC_OK) return st;
    orc_ctx c;
    memset(&c, 0, sizeof c);
    c.mode = mode == ORC_STABLE ? ORC_STABLE : ORC_LITERAL;
    c.check = check;
    c.max_levels = max_levels;
    c.literal_alg4 = literal_alg4;
    c.mant_bits = f_bits;
    if (c.mode == ORC_STABLE && n > 0) {
        c.tmp = (uint64_t *)malloc(n * sizeof(uint64_t));
        if (!c.tmp) return ORC_ERR_MEM;
    }
    asc = asc ? 1 : 0;
    if (kind == ORC_UNSIGNED) bsort_unsigned(&c, a, n, w, asc);
    else if (kind == ORC_SIGNED) bsort_signed(&c, a, n, w, asc);
    else bsort_float(&c, a, n, w, asc);
    free(c.tmp);
    if (stats_out) {
        stats_out[0] = c.violations;
        stats_out[1] = c.partitions;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Definition side: the order the sort must produce, written from its meaning
 * rather than from the bit partition.
 *   unsigned: numeric value of the w-bit word;
 *   signed:   numeric value of the w-bit two's-complement word;
 *   float:    numeric value (Sec. III-C layout: sign, biased exponent,
 *             mantissa with implicit leading one for normal numbers);
 *             -0 < +0; -inf / +inf below / above every number; NaNs at the
 *             two ends -- negative NaNs below -inf, positive NaNs above +inf --
 *             ordered by their mantissa field, farther from the middle as the
 *             field grows (Sec. III-C, special values).
 * ------------------------------------------------------------------------- */

typedef struct {
    int w, kind, e_bits, f_bits;
} orc_fmt;

static int64_t signed_value(uint64_t x, int w)
{
    if (w == 64) return (int64_t)x;
    uint64_t sb = (uint64_t)1 << (w - 1);
    if (x & sb) return (int64_t)(x | ~(((uint64_t)1 << w) - 1));
    return (int64_t)x;
}

/* exact value of a finite float pattern (|value| only; sign separate) */
static double float_magnitude(uint64_t x, const orc_fmt *f)
{
    uint64_t mant = x & (((uint64_t)1 << f->f_bits) - 1);
    uint64_t ex = (x >> f->f_bits) & (((uint64_t)1 << f->e_bits) - 1);
    int bias = (1 << (f->e_bits - 1)) - 1;
#if ORC_PLANT == 6
    if (ex == 0) return ldexp((double)mant, -bias - f->f_bits);
#else
    if (ex == 0) return ldexp((double)mant, 1 - bias - f->f_bits); /* subnormal or zero */
#endif
    return ldexp((double)(((uint64_t)1 << f->f_bits) | mant), (int)ex - bias - f->f_bits);
}

/* -1 if x before y in ascending order, 0 if same position (identical), +1 after */
int orc_cmp_total(uint64_t x, uint64_t y, int w, int kind, int e_bits, int f_bits)
{
    if (kind == ORC_UNSIGNED) return x < y ? -1 : (x > y ? 1 : 0);
    if (kind == ORC_SIGNED) {
        int64_t a = signed_value(x, w), b = signed_value(y, w);
        return a < b ? -1 : (a > b ? 1 : 0);
    }
    orc_fmt f = {w, kind, e_bits, f_bits};
    uint64_t emask = ((uint64_t)1 << e_bits) - 1;
    uint64_t fmask = ((uint64_t)1 << f_bits) - 1;
    int sx = (int)((x >> (w - 1)) & 1), sy = (int)((y >> (w - 1)) & 1);
    uint64_t ex = (x >> f_bits) & emask, ey = (y >> f_bits) & emask;
    uint64_t mx = x & fmask, my = y & fmask;
    int nan_x = ex == emask && mx != 0, nan_y = ey == emask && my != 0;
    if (nan_x || nan_y) {
        /* class rank: -NaN (0) < every non-NaN (1) < +NaN (2) */
        int cx = nan_x ? (sx ? 0 : 2) : 1;
        int cy = nan_y ? (sy ? 0 : 2) : 1;
        if (cx != cy) return cx < cy ? -1 : 1;
        /* both NaN of the same sign */
        if (mx == my) return 0;
        if (cx == 2) return mx < my ? -1 : 1; /* +NaN: larger field farther up */
#if ORC_PLANT == 5
        return mx < my ? -1 : 1;
#else
        return mx > my ? -1 : 1;              /* -NaN: larger field farther down */
#endif
    }
    int inf_x = ex == emask, inf_y = ey == emask; /* mantissa zero here */
    double vx, vy;
    if (inf_x) vx = sx ? -INFINITY : INFINITY;
    else vx = sx ? -float_magnitude(x, &f) : float_magnitude(x, &f);
    if (inf_y) vy = sy ? -INFINITY : INFINITY;
    else vy = sy ? -float_magnitude(y, &f) : float_magnitude(y, &f);
    if (vx < vy) return -1;
    if (vx > vy) return 1;
    /* numerically equal: only -0 vs +0 (or identical patterns) remain */
#if ORC_PLANT == 4
    if (sx != sy) return sx ? 1 : -1;
#else
    if (sx != sy) return sx ? -1 : 1;
#endif
    return 0;
}

/* numeric value of a finite float pattern, for tests that pin float_magnitude */
double orc_float_value(uint64_t x, int w, int e_bits, int f_bits)
{
    orc_fmt f = {w, ORC_FLOAT, e_bits, f_bits};
    double m = float_magnitude(x, &f);
    return ((x >> (w - 1)) & 1) ? -m : m;
}

static orc_fmt g_qsort_fmt;
static int g_qsort_asc;

static int qsort_cmp(const void *pa, const void *pb)
{
    uint64_t x = *(const uint64_t *)pa, y = *(const uint64_t *)pb;
    int r = orc_cmp_total(x, y, g_qsort_fmt.w, g_qsort_fmt.kind, g_qsort_fmt.e_bits, g_qsort_fmt.f_bits);
    return g_qsort_asc ? r : -r;
}

/* Sorts a[0, n) by the definition order using the C library's qsort (not
 * thread-safe: uses file-scope comparator state). */
int orc_sort_by_definition(uint64_t *a, size_t n, int w, int kind, int e_bits, int f_bits, int asc)
{
    int st = check_format(w, kind, e_bits, f_bits);
    if (st != ORC_OK) return st;
    st = check_bits(a, n, w);
    if (st != ORC_OK) return st;
    g_qsort_fmt.w = w;
    g_qsort_fmt.kind = kind;
    g_qsort_fmt.e_bits = e_bits;
    g_qsort_fmt.f_bits = f_bits;
    g_qsort_asc = asc ? 1 : 0;
    qsort(a, n, sizeof(uint64_t), qsort_cmp);
    return ORC_OK;
}

/* First index i with a[i] after a[i+1] in the requested direction, or -1 if
 * the array is monotone under the definition order. */
int64_t orc_first_unsorted(const uint64_t *a, size_t n, int w, int kind, int e_bits, int f_bits, int asc)
{
#if ORC_PLANT == 9
    for (size_t i = 0; i + 2 < n; i++) { /* planted: the last pair is never checked */
#else
    for (size_t i = 0; i + 1 < n; i++) {
#endif
        int r = orc_cmp_total(a[i], a[i + 1], w, kind, e_bits, f_bits);
#if ORC_PLANT == 12
        if (asc ? r >= 0 : r <= 0) return (int64_t)i; /* planted: equal neighbours flagged */
#else
        if (asc ? r > 0 : r < 0) return (int64_t)i;
#endif
    }
    return -1;
}

/* How many elements of a[0, n) come strictly before x, and how many are
 * bit-identical to x, in the requested direction.  The element at output
 * position p of a correct sort is the x with less <= p < less + equal. */
void orc_rank(const uint64_t *a, size_t n, uint64_t x, int w, int kind, int e_bits, int f_bits,
              int asc, uint64_t *less_out, uint64_t *equal_out)
{
    uint64_t less = 0, equal = 0;
    for (size_t i = 0; i < n; i++) {
#if ORC_PLANT == 10
        if (a[i] == x) { less++; continue; } /* planted: identical keys counted as before */
#else
        if (a[i] == x) { equal++; continue; }
#endif
        int r = orc_cmp_total(a[i], x, w, kind, e_bits, f_bits);
        if (asc ? r < 0 : r > 0) less++;
    }
    *less_out = less;
    *equal_out = equal;
}

/* Order-independent digest of a multiset of words: two sums and a xor of
 * differently mixed copies of every element, plus the count.  Equal
 * multisets give equal digests; used where an element-by-element oracle
 * comparison would take too long. */
static uint64_t mix_a(uint64_t z)
{
    z ^= z >> 33; z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33; z *= 0xc4ceb9fe1a85ec53ULL;
    return z ^ (z >> 33);
}

void orc_multiset_digest(const uint64_t *a, size_t n, uint64_t *out4)
{
    uint64_t s1 = 0, s2 = 0, x3 = 0;
#if ORC_PLANT == 11
    for (size_t i = 1; i < n; i++) { /* planted: the first element is ignored */
#else
    for (size_t i = 0; i < n; i++) {
#endif
#if ORC_PLANT == 13
        const uint64_t v = a[i] & 0xffffffffULL; /* planted: high half of a word ignored */
#else
        const uint64_t v = a[i];
#endif
        uint64_t h = mix_a(v);
        s1 += h;
        s2 += mix_a(h ^ 0x5851f42d4c957f2dULL) * (v | 1);
        x3 ^= mix_a(v + 0x9e3779b97f4a7c15ULL);
    }
    out4[0] = s1; out4[1] = s2; out4[2] = x3; out4[3] = (uint64_t)n;
}

/* Stable argsort by the definition order: perm[k] = input position of the
 * k-th element of the ordered sequence, elements that compare equal in
 * input order.  A bottom-up merge sort of the positions (stable because a
 * merge takes from the left run on ties). */
int orc_stable_argsort(const uint64_t *a, size_t n, int w, int kind, int e_bits, int f_bits, int asc,
                       uint64_t *perm)
{
    int st = check_format(w, kind, e_bits, f_bits);
    if (st != ORC_OK) return st;
    st = check_bits(a, n, w);
    if (st != ORC_OK) return st;
    uint64_t *tmp = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!tmp) return ORC_ERR_MEM;
    for (size_t i = 0; i < n; i++) perm[i] = i;
    uint64_t *src = perm, *dst = tmp;
    for (size_t width = 1; width < n; width *= 2) {
        for (size_t lo = 0; lo < n; lo += 2 * width) {
            size_t mid = lo + width < n ? lo + width : n;
            size_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            size_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) {
                int r = orc_cmp_total(a[src[i]], a[src[j]], w, kind, e_bits, f_bits);
                if (!asc) r = -r;
#if ORC_PLANT == 8
                int take_left = r < 0; /* planted: ties go right first */
#else
                int take_left = r <= 0;
#endif
                dst[k++] = take_left ? src[i++] : src[j++];
            }
            while (i < mid) dst[k++] = src[i++];
            while (j < hi) dst[k++] = src[j++];
        }
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != perm) memcpy(perm, src, n * sizeof(uint64_t));
    free(tmp);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Keys wider than one word: unsigned and signed integers of w bits, 64 < w
 * <= 128 (any 1 <= w <= 128 is accepted), each key a (hi, lo) pair of words,
 * the pattern's bits 64.. in hi and 0..63 in lo.  The same Algs. 1-3 as
 * above -- the partition on one bit, the MSB-first recursion, the signed
 * key's inverted sign pass -- with the mask given as a bit position, since a
 * 128-bit mask no longer fits one word (Sec. III-C: the method applies to any
 * word size).  The definition side compares the words as one integer.
 * ------------------------------------------------------------------------- */

typedef struct {
    int mode, check, max_levels;
    uint64_t violations, partitions;
    uint64_t *thi, *tlo; /* scratch for the stable split */
} orc_ctx2;

static int bit_of(const uint64_t *hi, const uint64_t *lo, size_t i, int b)
{
    return b >= 64 ? (int)((hi[i] >> (b - 64)) & 1) : (int)((lo[i] >> b) & 1);
}

/* Alg. 1 on the bit at position b of two-word keys. */
static size_t single_pass2(orc_ctx2 *c, uint64_t *hi, uint64_t *lo, int b, size_t ps, size_t pe, int asc)
{
    size_t k = ps;
    c->partitions++;
    if (c->mode == ORC_LITERAL) {
        for (size_t i = ps; i < pe; i++) {
            int bit = bit_of(hi, lo, i, b);
            if ((asc && !bit) || (!asc && bit)) {
                uint64_t th = hi[i], tl = lo[i];
                hi[i] = hi[k]; lo[i] = lo[k];
                hi[k] = th; lo[k] = tl;
                k++;
            }
        }
    } else {
        size_t t = 0;
        for (size_t i = ps; i < pe; i++) {
            int bit = bit_of(hi, lo, i, b);
            if ((asc && !bit) || (!asc && bit)) { c->thi[t] = hi[i]; c->tlo[t] = lo[i]; t++; }
        }
        k = ps + t;
        for (size_t i = ps; i < pe; i++) {
            int bit = bit_of(hi, lo, i, b);
            if (!((asc && !bit) || (!asc && bit))) { c->thi[t] = hi[i]; c->tlo[t] = lo[i]; t++; }
        }
        memcpy(hi + ps, c->thi, (pe - ps) * sizeof(uint64_t));
        memcpy(lo + ps, c->tlo, (pe - ps) * sizeof(uint64_t));
    }
    if (c->check) {
        for (size_t i = ps; i < k; i++)
            if (bit_of(hi, lo, i, b) != !asc) c->violations++;
        for (size_t j = k; j < pe; j++)
            if (bit_of(hi, lo, j, b) != asc) c->violations++;
    }
    return k;
}

/* Alg. 2 from bit position b down to bit 0. */
static void binary_quicksort2(orc_ctx2 *c, uint64_t *hi, uint64_t *lo, int b, size_t ps, size_t pe, int asc,
                              int level)
{
    if (pe - ps <= 1) return; /* R3 */
    size_t k = single_pass2(c, hi, lo, b, ps, pe, asc);
    if (b == 0 || (c->max_levels > 0 && level >= c->max_levels)) return;
#if ORC_PLANT == 14
    binary_quicksort2(c, hi, lo, b - 1, ps, k, !asc, level + 1); /* planted: lower side in the wrong direction */
#else
    binary_quicksort2(c, hi, lo, b - 1, ps, k, asc, level + 1);
#endif
    binary_quicksort2(c, hi, lo, b - 1, k, pe, asc, level + 1);
}

/* Sorts the two-word keys (hi[i], lo[i]), i < n, of w bits (1..128):
 * kind ORC_UNSIGNED (Alg. 2) or ORC_SIGNED (Alg. 3: sign pass inverted).
 * Arguments as orc_bsort; bits at or above w must be zero. */
int orc_bsort2(uint64_t *hi, uint64_t *lo, size_t n, int w, int kind, int asc, int mode, int max_levels, int check,
               uint64_t *stats_out)
{
    if (w < 1 || w > 128 || (kind != ORC_UNSIGNED && kind != ORC_SIGNED)) return ORC_ERR_ARG;
    for (size_t i = 0; i < n; i++) {
        if (w <= 64 && (hi[i] || (w < 64 && (lo[i] >> w)))) return ORC_ERR_BITS;
        if (w > 64 && w < 128 && (hi[i] >> (w - 64))) return ORC_ERR_BITS;
    }
    orc_ctx2 c;
    memset(&c, 0, sizeof c);
    c.mode = mode == ORC_STABLE ? ORC_STABLE : ORC_LITERAL;
    c.check = check;
    c.max_levels = max_levels;
    if (c.mode == ORC_STABLE && n > 0) {
        c.thi = (uint64_t *)malloc(n * sizeof(uint64_t));
        c.tlo = (uint64_t *)malloc(n * sizeof(uint64_t));
        if (!c.thi || !c.tlo) { free(c.thi); free(c.tlo); return ORC_ERR_MEM; }
    }
    asc = asc ? 1 : 0;
    if (kind == ORC_UNSIGNED) {
        binary_quicksort2(&c, hi, lo, w - 1, 0, n, asc, 1);
    } else if (n > 1) {
        size_t k = single_pass2(&c, hi, lo, w - 1, 0, n, !asc);
        if (w > 1 && !(max_levels > 0 && 1 >= max_levels)) {
            binary_quicksort2(&c, hi, lo, w - 2, 0, k, asc, 2);
            binary_quicksort2(&c, hi, lo, w - 2, k, n, asc, 2);
        }
    }
    free(c.thi);
    free(c.tlo);
    if (stats_out) { stats_out[0] = c.violations; stats_out[1] = c.partitions; }
    return ORC_OK;
}

/* Definition side for two-word keys: numeric order of the w-bit pattern as
 * an unsigned or a two's-complement integer.  -1, 0, +1. */
int orc_cmp2(uint64_t xh, uint64_t xl, uint64_t yh, uint64_t yl, int w, int kind)
{
    if (kind == ORC_SIGNED) {
        /* the sign bit decides first: a set sign bit is the smaller number */
        int sx = w > 64 ? (int)((xh >> (w - 65)) & 1) : (int)((xl >> (w - 1)) & 1);
        int sy = w > 64 ? (int)((yh >> (w - 65)) & 1) : (int)((yl >> (w - 1)) & 1);
        if (sx != sy) return sx ? -1 : 1;
    }
    if (xh != yh) return xh < yh ? -1 : 1;
    if (xl != yl) return xl < yl ? -1 : 1;
    return 0;
}
