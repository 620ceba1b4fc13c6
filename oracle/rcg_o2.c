/*
 * rcg_o2.c -- word-level, multi-threaded CPU implementation of the cyclic-group
 * RAID-6 code (the "O2" reference), for checking full-size GPU results byte
 * for byte and for a CPU throughput figure.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite and the benchmark's CPU legs
 * load this file.  It shares no code, table or helper with the CUDA path or
 * with rcg_oracle.c; the tests check it against rcg_oracle.c (the bit-level
 * definition).
 *
 * What it computes.  The same code as rcg_oracle.c (Corollary 3.2.4 with data
 * strip k weighted by x^k, and 1 + x^(k-p+1) for k >= p per equation (qext) of
 * Section 3.3; recovery by the four cases of Lemma 3.1.2), on the same
 * bit-sliced stripes.  Where rcg_oracle.c gathers one codeword at a time, this
 * file works on 64 codewords at once: a 64-bit word of row r holds the x^r
 * coefficients of 64 codewords, so multiplying by x^k is moving whole words
 * between rows.  Elements are held lifted to F2[x]/(x^p - 1) (p rows, row
 * p-1 starting at zero); multiplication by x^k is the cyclic row shift
 * (Lemma 3.4.1's (powers): S_p^k acts on the lift as a rotation), and the
 * residue modulo f = 1 + ... + x^(p-1) is row r XOR row p-1.  Inverses are
 * found by Gaussian elimination over GF(2) on the (p-1) x (p-1) matrix of
 * multiplication by the element (a third method: the library uses Frobenius
 * powers, rcg_oracle.c the extended Euclidean algorithm).
 *
 * Layout: stripe s at buf + s*stripe_stride, strip k at + k*strip_stride, row
 * r at + r*row_stride, C bytes per row (C a multiple of 8 here: every row is
 * processed as C/8 words).  Stripes are split across threads.  Stripes in the
 * horizontal representation of Section 4.5 (o2_h_*) are turned into this form
 * 64 elements at a time and back.  Z_257 (o2_h257_*, at the end) has 256-bit
 * elements and its own word-level code on them.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;

#define O2_MAXP 61
#define O2_MAXN 121

/* ------------------------------------------------------ ring elements */

/* Element of R as a bit mask (bit m = coefficient of x^m, m < p-1). */
static u64 weight(unsigned p, unsigned k)
{
    unsigned e = k < p ? k : k - p + 1;
    u64 lifted = (k < p ? 0 : 1u) ^ (1ull << e);   /* x^e (+ 1), exponents < p */
    if (lifted >> (p - 1) & 1)                     /* x^(p-1) = 1 + ... + x^(p-2) */
        lifted ^= (1ull << p) - 1;
    return lifted;
}

/* Product a*b in R by the multiplication matrix's columns: column c of the
 * matrix of "multiply by a" is a * x^c. */
static u64 mul_xc(unsigned p, u64 a, unsigned c)
{
    /* rotate the lifted p-bit vector by c, then reduce */
    u64 full = (1ull << p) - 1;
    u64 r = ((a << c) | (a >> (p - c))) & full;
    if (c == 0)
        r = a;
    if (r >> (p - 1) & 1)
        r ^= full;
    return r;
}

/* Inverse of a in R by Gaussian elimination on [M | I], M the matrix of
 * multiplication by a (columns a * x^c).  Returns 0 when a is singular. */
static u64 inverse(unsigned p, u64 a)
{
    unsigned n = p - 1;
    u64 rows[O2_MAXP];     /* row i of M, bit c = entry (i, c) */
    u64 aug[O2_MAXP];      /* row i of the identity being transformed */
    for (unsigned i = 0; i < n; i++) {
        rows[i] = 0;
        aug[i] = 1ull << i;
    }
    for (unsigned c = 0; c < n; c++) {
        u64 col = mul_xc(p, a, c);
        for (unsigned i = 0; i < n; i++)
            if (col >> i & 1)
                rows[i] |= 1ull << c;
    }
    for (unsigned c = 0; c < n; c++) {
        unsigned piv = n;
        for (unsigned i = c; i < n; i++)
            if (rows[i] >> c & 1) {
                piv = i;
                break;
            }
        if (piv == n)
            return 0;
        u64 t = rows[c]; rows[c] = rows[piv]; rows[piv] = t;
        t = aug[c]; aug[c] = aug[piv]; aug[piv] = t;
        for (unsigned i = 0; i < n; i++)
            if (i != c && (rows[i] >> c & 1)) {
                rows[i] ^= rows[c];
                aug[i] ^= aug[c];
            }
    }
    /* M^(-1) = the transformed identity; the inverse element is M^(-1) e_0,
     * i.e. column 0 of M^(-1): bit i of it is bit 0 of row i */
    u64 inv = 0;
    for (unsigned i = 0; i < n; i++)
        if (aug[i] & 1)
            inv |= 1ull << i;
    return inv;
}

/* ------------------------------------------------------------ word rows */

typedef struct {
    uint8_t *buf;
    unsigned p, N;
    u64 C, rs, ss, st;
} geo_t;

static u64 *rowp(const geo_t *g, u64 s, unsigned k, unsigned r)
{
    return (u64 *)(g->buf + s * g->st + (u64)k * g->ss + (u64)r * g->rs);
}

/* acc (lifted, p words) += x^e * v (p-1 words; the lifted row p-1 of v is 0) */
static void add_rot(unsigned p, u64 *acc, const u64 *v, unsigned e)
{
    for (unsigned r = 0; r + 1 < p; r++)
        acc[(r + e) % p] ^= v[r];
}

/* acc += w * v, w a mask in R (bits < p-1), v lifted (p words) */
static void add_mul(unsigned p, u64 *acc, const u64 *v, u64 w)
{
    for (unsigned m = 0; m + 1 < p; m++)
        if (w >> m & 1)
            for (unsigned r = 0; r < p; r++)
                acc[(r + m) % p] ^= v[r];
}

/* ---------------------------------------------------- one stripe, one word */

/* Encode or recover word column w of stripe s.  (i, j) = (N, N+1) encodes. */
static void stripe_word(const geo_t *g, u64 s, u64 w, unsigned i, unsigned j, const u64 *inv_w,
                        const u64 (*inv_pair)[O2_MAXN])
{
    unsigned p = g->p, N = g->N;
    u64 dP[O2_MAXP] = {0}, dQ[O2_MAXP] = {0}, d[O2_MAXP];
    for (unsigned k = 0; k < N + 2; k++) {
        if (k == i || k == j)
            continue;
        for (unsigned r = 0; r + 1 < p; r++)
            d[r] = rowp(g, s, k, r)[w];
        if (k < N) {
            for (unsigned r = 0; r + 1 < p; r++)
                dP[r] ^= d[r];
            if (k < p) {
                add_rot(p, dQ, d, k);
            } else {
                add_rot(p, dQ, d, 0);
                add_rot(p, dQ, d, k - p + 1);
            }
        } else if (k == N) {
            for (unsigned r = 0; r + 1 < p; r++)
                dP[r] ^= d[r];
        } else {
            add_rot(p, dQ, d, 0);
        }
    }
    u64 out[O2_MAXP] = {0}, t[O2_MAXP] = {0};
    if (i == N) {                                  /* P and Q */
        for (unsigned r = 0; r + 1 < p; r++) {
            rowp(g, s, N, r)[w] = dP[r];
            rowp(g, s, N + 1, r)[w] = dQ[r] ^ dQ[p - 1];
        }
        return;
    }
    if (j == N + 1) {                              /* data i and Q: RAID-5, then Q */
        add_mul(p, dQ, dP, weight(p, i));          /* dP's lifted row p-1 is 0 */
        for (unsigned r = 0; r + 1 < p; r++) {
            rowp(g, s, i, r)[w] = dP[r];
            rowp(g, s, N + 1, r)[w] = dQ[r] ^ dQ[p - 1];
        }
        return;
    }
    if (j == N) {                                  /* data i and P: w_i D_i = dQ */
        add_mul(p, out, dQ, inv_w[i]);
        for (unsigned r = 0; r + 1 < p; r++) {
            u64 di = out[r] ^ out[p - 1];
            rowp(g, s, i, r)[w] = di;
            rowp(g, s, N, r)[w] = dP[r] ^ di;
        }
        return;
    }
    /* two data strips: (w_i + w_j) D_j = w_i dP + dQ, D_i = D_j + dP */
    memcpy(t, dQ, sizeof(u64) * p);
    add_mul(p, t, dP, weight(p, i));
    add_mul(p, out, t, inv_pair[i][j]);
    for (unsigned r = 0; r + 1 < p; r++) {
        u64 dj = out[r] ^ out[p - 1];
        rowp(g, s, j, r)[w] = dj;
        rowp(g, s, i, r)[w] = dj ^ dP[r];
    }
}

/* ------------------------------------------------------------- threads */

typedef struct {
    const geo_t *g;
    u64 s0, s1;
    unsigned i, j;
    const uint8_t *pairs;
    const u64 *inv_w;
    const u64 (*inv_pair)[O2_MAXN];
    int bad;
} work_t;

static void *worker(void *arg)
{
    work_t *wk = (work_t *)arg;
    const geo_t *g = wk->g;
    for (u64 s = wk->s0; s < wk->s1; s++) {
        unsigned i = wk->pairs ? wk->pairs[2 * s] : wk->i;
        unsigned j = wk->pairs ? wk->pairs[2 * s + 1] : wk->j;
        if (!(i < j && j <= g->N + 1)) {
            wk->bad = 1;
            continue;
        }
        for (u64 w = 0; w < g->C / 8; w++)
            stripe_word(g, s, w, i, j, wk->inv_w, wk->inv_pair);
    }
    return NULL;
}

static int run(unsigned p, unsigned N, u64 C, uint8_t *buf, u64 n_stripes, u64 rs, u64 ss, u64 st,
               unsigned i, unsigned j, const uint8_t *pairs, int threads)
{
    if (p < 3 || p > O2_MAXP || N < 1 || N > 2 * p - 1 || N > O2_MAXN || C == 0 || C % 8)
        return -1;
    for (unsigned t = 2; t * t <= p; t++)
        if (p % t == 0)
            return -1;
    static u64 inv_w[O2_MAXN];
    static u64 inv_pair[O2_MAXN][O2_MAXN];
    for (unsigned a = 0; a < N; a++) {
        inv_w[a] = inverse(p, weight(p, a));
        for (unsigned b = a + 1; b < N; b++) {
            inv_pair[a][b] = inverse(p, weight(p, a) ^ weight(p, b));
            if (inv_pair[a][b] == 0)
                return -3;   /* the weights are not a cone for this p and N */
        }
    }
    geo_t g = {buf, p, N, C, rs, ss, st};
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    pthread_t tid[256];
    work_t wk[256];
    for (int t = 0; t < threads; t++) {
        wk[t].g = &g;
        wk[t].s0 = n_stripes * t / threads;
        wk[t].s1 = n_stripes * (t + 1) / threads;
        wk[t].i = i;
        wk[t].j = j;
        wk[t].pairs = pairs;
        wk[t].inv_w = inv_w;
        wk[t].inv_pair = (const u64 (*)[O2_MAXN])inv_pair;
        wk[t].bad = 0;
        pthread_create(&tid[t], NULL, worker, &wk[t]);
    }
    int bad = 0;
    for (int t = 0; t < threads; t++) {
        pthread_join(tid[t], NULL);
        bad |= wk[t].bad;
    }
    return bad ? -2 : 0;
}

int o2_encode(unsigned p, unsigned N, u64 C, uint8_t *buf, u64 n_stripes, u64 rs, u64 ss, u64 st, int threads)
{
    return run(p, N, C, buf, n_stripes, rs, ss, st, N, N + 1, NULL, threads);
}

/* Recover pair (i, j), or per-stripe pairs (two bytes per stripe) when pairs != NULL. */
int o2_recover(unsigned p, unsigned N, u64 C, uint8_t *buf, u64 n_stripes, u64 rs, u64 ss, u64 st,
               unsigned i, unsigned j, const uint8_t *pairs, int threads)
{
    return run(p, N, C, buf, n_stripes, rs, ss, st, i, j, pairs, threads);
}

/* ---------------------------------------------------- horizontal strips */

/* Stripes in the horizontal representation of Section 4.5: element e of a
 * strip is bits [e(p-1), (e+1)(p-1)) of the strip (bit b = bit b%8 of byte
 * b/8), one ring element each.  Blocks of 64 elements are turned into the
 * bit-sliced form this file already computes on -- p-1 words, bit t of word r
 * = coefficient of x^r of element t -- run through stripe_word, and the
 * strips it wrote are turned back. */

typedef struct {
    uint8_t *buf;
    unsigned p, N;
    u64 strip_bytes, ss, st;
} hgeo_t;

/* Bits [e(p-1), (e+1)(p-1)) of a strip (p-1 <= 60): the bytes that hold
 * them, assembled little-endian (only those bytes are touched), or bit by
 * bit when they span nine bytes. */
static u64 h_get(const uint8_t *strip, unsigned rows, u64 e)
{
    u64 b = e * rows, a = 0;
    unsigned sh = (unsigned)(b & 7), nb = (sh + rows + 7) >> 3;
    if (nb <= 8) {
        for (unsigned q = 0; q < nb; q++)
            a |= (u64)strip[(b >> 3) + q] << (8 * q);
        return (a >> sh) & ((1ull << rows) - 1);
    }
    for (unsigned r = 0; r < rows; r++, b++)
        a |= (u64)((strip[b >> 3] >> (b & 7)) & 1u) << r;
    return a;
}

static void h_put(uint8_t *strip, unsigned rows, u64 e, u64 a)
{
    u64 b = e * rows;
    unsigned sh = (unsigned)(b & 7), nb = (sh + rows + 7) >> 3;
    if (nb <= 8) {
        u64 v = 0, m = ((1ull << rows) - 1) << sh;
        for (unsigned q = 0; q < nb; q++)
            v |= (u64)strip[(b >> 3) + q] << (8 * q);
        v = (v & ~m) | (a << sh);
        for (unsigned q = 0; q < nb; q++)
            strip[(b >> 3) + q] = (uint8_t)(v >> (8 * q));
        return;
    }
    for (unsigned r = 0; r < rows; r++, b++) {
        uint8_t m = (uint8_t)(1u << (b & 7));
        if (a >> r & 1)
            strip[b >> 3] |= m;
        else
            strip[b >> 3] &= (uint8_t)~m;
    }
}

/* Elements [e0, e0 + n) (n <= 64) of stripe s: (i, j) = (N, N+1) encodes. */
static void h_block(const hgeo_t *h, u64 s, u64 e0, unsigned n, unsigned i, unsigned j, const u64 *inv_w,
                    const u64 (*inv_pair)[O2_MAXN])
{
    unsigned p = h->p, N = h->N, rows = p - 1;
    u64 words[(O2_MAXN + 2) * (O2_MAXP - 1)];   /* strip k, row r at k*rows + r */
    memset(words, 0, sizeof(u64) * (N + 2) * rows);
    for (unsigned k = 0; k < N + 2; k++) {
        if (k == i || k == j)
            continue;
        const uint8_t *strip = h->buf + s * h->st + (u64)k * h->ss;
        for (unsigned t = 0; t < n; t++) {
            u64 a = h_get(strip, rows, e0 + t);
            for (unsigned r = 0; r < rows; r++)
                words[k * rows + r] |= (a >> r & 1) << t;
        }
    }
    /* one word per row, rows 8 bytes apart, strips rows*8 bytes apart */
    geo_t g = {(uint8_t *)words, p, N, 8, 8, (u64)rows * 8, (u64)(N + 2) * rows * 8};
    stripe_word(&g, 0, 0, i, j, inv_w, inv_pair);
    for (unsigned q = 0; q < 2; q++) {
        unsigned k = q ? j : i;
        uint8_t *strip = h->buf + s * h->st + (u64)k * h->ss;
        for (unsigned t = 0; t < n; t++) {
            u64 a = 0;
            for (unsigned r = 0; r < rows; r++)
                a |= (words[k * rows + r] >> t & 1) << r;
            h_put(strip, rows, e0 + t, a);
        }
    }
}

typedef struct {
    const hgeo_t *h;
    u64 s0, s1;
    unsigned i, j;
    const uint8_t *pairs;
    const u64 *inv_w;
    const u64 (*inv_pair)[O2_MAXN];
    int bad;
} hwork_t;

static void *h_worker(void *arg)
{
    hwork_t *wk = (hwork_t *)arg;
    const hgeo_t *h = wk->h;
    u64 n_el = h->strip_bytes * 8 / (h->p - 1);
    for (u64 s = wk->s0; s < wk->s1; s++) {
        unsigned i = wk->pairs ? wk->pairs[2 * s] : wk->i;
        unsigned j = wk->pairs ? wk->pairs[2 * s + 1] : wk->j;
        if (!(i < j && j <= h->N + 1)) {
            wk->bad = 1;
            continue;
        }
        for (u64 e0 = 0; e0 < n_el; e0 += 64)
            h_block(h, s, e0, (unsigned)(n_el - e0 < 64 ? n_el - e0 : 64), i, j, wk->inv_w, wk->inv_pair);
    }
    return NULL;
}

static int h_run(unsigned p, unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes, u64 ss, u64 st,
                 unsigned i, unsigned j, const uint8_t *pairs, int threads)
{
    if (p < 3 || p > O2_MAXP || N < 1 || N > 2 * p - 1 || N > O2_MAXN || strip_bytes == 0 ||
        (strip_bytes * 8) % (p - 1))
        return -1;
    for (unsigned t = 2; t * t <= p; t++)
        if (p % t == 0)
            return -1;
    static u64 inv_w[O2_MAXN];
    static u64 inv_pair[O2_MAXN][O2_MAXN];
    for (unsigned a = 0; a < N; a++) {
        inv_w[a] = inverse(p, weight(p, a));
        for (unsigned b = a + 1; b < N; b++) {
            inv_pair[a][b] = inverse(p, weight(p, a) ^ weight(p, b));
            if (inv_pair[a][b] == 0)
                return -3;
        }
    }
    hgeo_t h = {buf, p, N, strip_bytes, ss, st};
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    pthread_t tid[256];
    hwork_t wk[256];
    for (int t = 0; t < threads; t++) {
        wk[t].h = &h;
        wk[t].s0 = n_stripes * t / threads;
        wk[t].s1 = n_stripes * (t + 1) / threads;
        wk[t].i = i;
        wk[t].j = j;
        wk[t].pairs = pairs;
        wk[t].inv_w = inv_w;
        wk[t].inv_pair = (const u64 (*)[O2_MAXN])inv_pair;
        wk[t].bad = 0;
        pthread_create(&tid[t], NULL, h_worker, &wk[t]);
    }
    int bad = 0;
    for (int t = 0; t < threads; t++) {
        pthread_join(tid[t], NULL);
        bad |= wk[t].bad;
    }
    return bad ? -2 : 0;
}

int o2_h_encode(unsigned p, unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes, u64 ss, u64 st, int threads)
{
    return h_run(p, N, strip_bytes, buf, n_stripes, ss, st, N, N + 1, NULL, threads);
}

/* Recover pair (i, j), or per-stripe pairs (two bytes per stripe) when pairs != NULL. */
int o2_h_recover(unsigned p, unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes, u64 ss, u64 st,
                 unsigned i, unsigned j, const uint8_t *pairs, int threads)
{
    return h_run(p, N, strip_bytes, buf, n_stripes, ss, st, i, j, pairs, threads);
}

/* The inverse of a in R (bit mask), 0 when singular -- exposed for the tests. */
u64 o2_inverse(unsigned p, u64 a)
{
    return inverse(p, a);
}

/* ======================================= Z_257: 256-bit elements, word level
 *
 * p = 257 (Section 3.4's Z_257): an element is 256 bits, too wide for the
 * bit masks above, and in the horizontal representation it is exactly 32
 * bytes (four 64-bit words, little-endian).  Elements are held lifted to
 * F2[x]/(x^257 - 1) in five words (bit 256 = bit 0 of word 4, the imaginary
 * row); x^k is a cyclic rotation of the 257 bits, and the residue modulo f
 * flips bits 0..255 when bit 256 is set.  Inverses are solved by Gaussian
 * elimination on the 256 x 256 matrix of multiplication by the element, one
 * per stripe (per erasure pair).  Base code only: N <= 257. */

#define Z_P 257u
#define Z_BITS 256u

typedef struct {
    u64 w[5];
} l257;

static void l257_load(const uint8_t *src, l257 *a)
{
    for (unsigned q = 0; q < 4; q++) {
        u64 v = 0;
        for (unsigned b = 0; b < 8; b++)
            v |= (u64)src[8 * q + b] << (8 * b);
        a->w[q] = v;
    }
    a->w[4] = 0;
}

static void l257_store(uint8_t *dst, const l257 *a)
{
    for (unsigned q = 0; q < 4; q++)
        for (unsigned b = 0; b < 8; b++)
            dst[8 * q + b] = (uint8_t)(a->w[q] >> (8 * b));
}

static void l257_xor(l257 *a, const l257 *b)
{
    for (unsigned q = 0; q < 5; q++)
        a->w[q] ^= b->w[q];
}

/* x^k a in the lift, 0 <= k < 257: bit t moves to bit (t + k) mod 257. */
static void l257_rot(const l257 *a, unsigned k, l257 *out)
{
    if (k == 0) {
        *out = *a;
        return;
    }
    l257 hi = {{0}}, lo = {{0}};
    const unsigned qk = k / 64, rk = k % 64;
    for (int t = 4; t >= 0; t--) {          /* hi = a << k */
        const int s0 = t - (int)qk, s1 = s0 - 1;
        u64 v = s0 >= 0 ? a->w[s0] << rk : 0;
        if (rk && s1 >= 0)
            v |= a->w[s1] >> (64 - rk);
        hi.w[t] = v;
    }
    hi.w[4] &= 1;                            /* keep 257 bits */
    const unsigned m = Z_P - k, qm = m / 64, rm = m % 64;
    for (unsigned t = 0; t < 5; t++) {       /* lo = a >> (257 - k) */
        const unsigned s0 = t + qm, s1 = s0 + 1;
        u64 v = s0 <= 4 ? a->w[s0] >> rm : 0;
        if (rm && s1 <= 4)
            v |= a->w[s1] << (64 - rm);
        lo.w[t] = v;
    }
    for (unsigned q = 0; q < 5; q++)
        out->w[q] = hi.w[q] | lo.w[q];
}

/* residue modulo f = 1 + ... + x^256 */
static void l257_reduce(l257 *a)
{
    if (a->w[4] & 1)
        for (unsigned q = 0; q < 4; q++)
            a->w[q] = ~a->w[q];
    a->w[4] = 0;
}

/* c * t in R, c reduced (256 bits): sum over the set bits m of c of x^m t. */
static void l257_mul(const l257 *c, const l257 *t, l257 *out)
{
    l257 acc = {{0}}, r;
    for (unsigned m = 0; m < Z_BITS; m++)
        if (c->w[m / 64] >> (m % 64) & 1) {
            l257_rot(t, m, &r);
            l257_xor(&acc, &r);
        }
    l257_reduce(&acc);
    *out = acc;
}

/* The inverse of u (reduced) by Gauss-Jordan elimination on [M | e_0], M the
 * matrix of multiplication by u (column c = u x^c): the solution v of
 * u v = 1.  Returns 0 when u is singular. */
static int l257_inverse(const l257 *u, l257 *out)
{
    static __thread u64 row[Z_BITS][5];      /* words 0..3: M's row, bit 0 of word 4: the right side */
    memset(row, 0, sizeof(row));
    for (unsigned c = 0; c < Z_BITS; c++) {
        l257 col;
        l257_rot(u, c, &col);
        l257_reduce(&col);
        for (unsigned i = 0; i < Z_BITS; i++)
            if (col.w[i / 64] >> (i % 64) & 1)
                row[i][c / 64] |= 1ull << (c % 64);
    }
    row[0][4] = 1;
    for (unsigned c = 0; c < Z_BITS; c++) {
        unsigned piv = c;
        while (piv < Z_BITS && !(row[piv][c / 64] >> (c % 64) & 1))
            piv++;
        if (piv == Z_BITS)
            return 0;
        if (piv != c)
            for (unsigned q = 0; q < 5; q++) {
                u64 t = row[c][q];
                row[c][q] = row[piv][q];
                row[piv][q] = t;
            }
        for (unsigned i = 0; i < Z_BITS; i++)
            if (i != c && (row[i][c / 64] >> (c % 64) & 1))
                for (unsigned q = 0; q < 5; q++)
                    row[i][q] ^= row[c][q];
    }
    memset(out, 0, sizeof(*out));
    for (unsigned i = 0; i < Z_BITS; i++)
        if (row[i][4] & 1)
            out->w[i / 64] |= 1ull << (i % 64);
    return 1;
}

static void l257_xpow(unsigned k, l257 *out)
{
    l257 one = {{1, 0, 0, 0, 0}};
    l257_rot(&one, k % Z_P, out);
    l257_reduce(out);
}

typedef struct {
    uint8_t *buf;
    unsigned N;
    u64 n_el, ss, st;
    u64 s0, s1;
    unsigned i, j;
    const uint16_t *pairs;
    int bad;
} zwork_t;

/* Every element of stripe s, lost pair a < b ((N, N+1) encodes), by the four
 * cases of Lemma 3.1.2 on the lifted elements. */
static int z_stripe(const zwork_t *z, u64 s, unsigned a, unsigned b)
{
    const unsigned N = z->N;
    l257 inv = {{0}};
    if (b <= N && a < N) {
        l257 u, t;
        l257_xpow(a, &u);                         /* g_a (data + P) */
        if (b < N) {                              /* g_a + g_b (two data) */
            l257_xpow(b, &t);
            l257_xor(&u, &t);
        }
        if (!l257_inverse(&u, &inv))
            return -3;
    }
    const int read_p = a != N && b != N, read_q = a != N + 1 && b != N + 1;
    uint8_t *const stripe = z->buf + s * z->st;
    for (u64 e = 0; e < z->n_el; e++) {
        uint8_t *const el = stripe + e * 32;
        l257 dP = {{0}}, dQ = {{0}}, d, r;
        if (read_p)
            l257_load(el + (u64)N * z->ss, &dP);
        if (read_q)
            l257_load(el + (u64)(N + 1) * z->ss, &dQ);
        for (unsigned k = 0; k < N; k++) {
            if (k == a || k == b)
                continue;
            l257_load(el + (u64)k * z->ss, &d);
            l257_xor(&dP, &d);
            l257_rot(&d, k, &r);
            l257_xor(&dQ, &r);
        }
        if (a == N) {                             /* P and Q */
            l257_reduce(&dQ);
            l257_store(el + (u64)N * z->ss, &dP);
            l257_store(el + (u64)(N + 1) * z->ss, &dQ);
        } else if (b == N + 1) {                  /* d_a = dP, then Q */
            l257_rot(&dP, a, &r);
            l257_xor(&dQ, &r);
            l257_reduce(&dQ);
            l257_store(el + (u64)a * z->ss, &dP);
            l257_store(el + (u64)(N + 1) * z->ss, &dQ);
        } else if (b == N) {                      /* g_a d_a = dQ, then P */
            l257 da;
            l257_reduce(&dQ);
            l257_mul(&inv, &dQ, &da);
            l257_store(el + (u64)a * z->ss, &da);
            l257_xor(&dP, &da);
            l257_store(el + (u64)N * z->ss, &dP);
        } else {                                  /* (g_a + g_b) d_b = g_a dP + dQ */
            l257 t, db;
            l257_rot(&dP, a, &t);
            l257_xor(&t, &dQ);
            l257_reduce(&t);
            l257_mul(&inv, &t, &db);
            l257_store(el + (u64)b * z->ss, &db);
            l257_xor(&dP, &db);
            l257_store(el + (u64)a * z->ss, &dP);
        }
    }
    return 0;
}

static void *z_worker(void *arg)
{
    zwork_t *wk = (zwork_t *)arg;
    for (u64 s = wk->s0; s < wk->s1; s++) {
        const unsigned a = wk->pairs ? wk->pairs[2 * s] : wk->i;
        const unsigned b = wk->pairs ? wk->pairs[2 * s + 1] : wk->j;
        if (!(a < b && b <= wk->N + 1) || z_stripe(wk, s, a, b))
            wk->bad = 1;
    }
    return NULL;
}

static int z_run(unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes, u64 ss, u64 st, unsigned i,
                 unsigned j, const uint16_t *pairs, int threads)
{
    if (N < 1 || N > Z_P || strip_bytes == 0 || strip_bytes % 32)
        return -1;
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    pthread_t tid[256];
    zwork_t wk[256];
    for (int t = 0; t < threads; t++) {
        zwork_t w = {buf, N, strip_bytes / 32, ss, st, n_stripes * t / threads, n_stripes * (t + 1) / threads,
                     i, j, pairs, 0};
        wk[t] = w;
        pthread_create(&tid[t], NULL, z_worker, &wk[t]);
    }
    int bad = 0;
    for (int t = 0; t < threads; t++) {
        pthread_join(tid[t], NULL);
        bad |= wk[t].bad;
    }
    return bad ? -2 : 0;
}

/* Z_257 stripes in the horizontal representation: strips of strip_bytes (a
 * multiple of 32), element e = bytes [32e, 32e + 32) little-endian. */
int o2_h257_encode(unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes, u64 ss, u64 st, int threads)
{
    return z_run(N, strip_bytes, buf, n_stripes, ss, st, N, N + 1, NULL, threads);
}

/* Recover pair (i, j), or per-stripe pairs (two 16-bit numbers per stripe:
 * strip indices reach 258) when pairs != NULL. */
int o2_h257_recover(unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes, u64 ss, u64 st, unsigned i,
                    unsigned j, const uint16_t *pairs, int threads)
{
    return z_run(N, strip_bytes, buf, n_stripes, ss, st, i, j, pairs, threads);
}

/* The inverse in R (p = 257) of the 32-byte element a, for the tests;
 * returns 0 when a is singular. */
int o2_h257_inverse(const uint8_t *a, uint8_t *out)
{
    l257 u, v;
    l257_load(a, &u);
    if (!l257_inverse(&u, &v))
        return 0;
    l257_store(out, &v);
    return 1;
}
