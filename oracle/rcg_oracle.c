/*
 * rcg_oracle.c -- bit-level CPU oracle for the cyclic-group RAID-6 code of
 * Jackson, Rumynin and Zaboronski, "An approach to RAID-6 based on cyclic
 * groups" (arXiv cs/0611109).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The product library never
 * links, includes or calls it, and it shares no code, table or helper with the
 * CUDA path.
 *
 * What it computes.  A strip is an element of the ring
 *     R = F2[x] / (f),   f = 1 + x + ... + x^(p-1),   p an odd prime,
 * i.e. a polynomial of degree <= p-2 (Lemma 3.4.1: the Sylvester matrix S_p is
 * the companion matrix of f, so multiplying by S_p is multiplying by x in R).
 * The code is the one of Corollary 3.2.4, equation (znparity), with generator
 * g = S_p and 0-based data indices as in Section 4.1 (data strip k is weighted
 * by g^k):
 *     P = sum_k d_k,            Q = sum_k x^k d_k   (mod f).
 * For p < N <= 2p-1 data strips the Q weights continue with the extension
 * (qext) of Section 3.3: strip k >= p is weighted by 1 + x^(k-p+1).  That
 * code is MDS exactly when p satisfies the conditions of Theorem 3.3.3; this
 * file checks condition (3) of that theorem (oracle_cone_extends) and accepts
 * N > p only for such p.
 *
 * Storage (bit slicing).  A strip is p-1 rows of C bytes.  Bit b of the row
 * region (byte b/8, bit b%8) of row r holds the coefficient of x^r of the b-th
 * independent codeword of the strip.  So a strip of C-byte rows carries 8*C
 * ring elements, one per bit position, and every function below works one bit
 * position at a time: gather the polynomial, do the ring arithmetic with a
 * generic carry-less multiply and a long-division remainder, scatter it back.
 *
 * Ring arithmetic is deliberately generic: multiplication is schoolbook
 * carry-less multiplication followed by polynomial long division by f, and
 * inverses come from the extended Euclidean algorithm against f.  None of the
 * rotate-and-fold shortcuts or the closed-form inverse of Section 4.6 appear
 * here; the tests check those closed forms against this file.
 *
 * Stripe layout: stripe s starts at buf + s*stripe_stride; strip k (data
 * 0..N-1, then P = strip N and Q = strip N+1) at + k*strip_stride; row r at
 * + r*row_stride; the row is C bytes.
 *
 * Horizontal storage (the oracle_h_* functions).  Section 4.5 keeps one ring
 * element per machine word instead: for p = 17 a 16-bit word holds y_0..y_15,
 * the coefficients of x^0..x^15.  In general element e of a strip is the
 * little-endian bit string at bits [e(p-1), (e+1)(p-1)) of the strip (bit t is
 * bit t%8 of byte t/8), bit r of it the coefficient of x^r; for p = 17 that is
 * the 16-bit little-endian word e.  The arithmetic is the same; only gather
 * and scatter differ.
 *
 * Large primes (the oracle_big_* and oracle_hbig_* functions, at the end):
 * Section 3.4 names Z_257 beside Z_17, whose elements (256 bits) do not fit
 * the 128-bit polynomials above.  That part holds polynomials as arrays of
 * coefficients and works for any odd prime p <= 257 (base code, N <= p), in
 * the horizontal representation; it shares nothing with the 128-bit code, and
 * the tests require both to agree on every prime both accept.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

/* ---------------------------------------------------------------- F2[x] */

static int poly_degree(u128 a)
{
    int d = -1;
    while (a) {
        a >>= 1;
        d++;
    }
    return d;
}

/* Carry-less (F2[x]) product.  The caller keeps deg(a)+deg(b) < 128. */
static u128 poly_mul(u128 a, u128 b)
{
    u128 r = 0;
    int sh = 0;
    while (b) {
        if (b & 1)
            r ^= a << sh;
        b >>= 1;
        sh++;
    }
    return r;
}

/* Quotient and remainder of polynomial long division a = q*m + r. */
static void poly_divmod(u128 a, u128 m, u128 *q, u128 *r)
{
    int dm = poly_degree(m);
    u128 quo = 0;
    int da = poly_degree(a);
    while (da >= dm) {
        quo ^= (u128)1 << (da - dm);
        a ^= m << (da - dm);
        da = poly_degree(a);
    }
    if (q)
        *q = quo;
    if (r)
        *r = a;
}

/* f = 1 + x + ... + x^(p-1): the characteristic (and minimal) polynomial of
 * the Sylvester matrix S_p, Lemma 3.4.1(ii). */
static u128 poly_f(unsigned p)
{
    return (((u128)1) << p) - 1;
}

/* ------------------------------------------------------------------ R */

/* Product in R = F2[x]/(f).  Operands are reduced (degree <= p-2). */
u64 oracle_ring_mul(unsigned p, u64 a, u64 b)
{
    u128 r;
    poly_divmod(poly_mul(a, b), poly_f(p), NULL, &r);
    return (u64)r;
}

/* x^k in R, for 0 <= k < 128. */
u64 oracle_ring_xpow(unsigned p, unsigned k)
{
    u128 r;
    poly_divmod(((u128)1) << k, poly_f(p), NULL, &r);
    return (u64)r;
}

/* Inverse in R by the extended Euclidean algorithm against f.  Returns 0 when
 * gcd(a, f) != 1 (a not invertible). */
u64 oracle_ring_inv(unsigned p, u64 a)
{
    u128 f = poly_f(p);
    u128 r0 = f, r1, s0 = 0, s1 = 1;
    poly_divmod(a, f, NULL, &r1);
    if (r1 == 0)
        return 0;
    while (r1 != 0) {
        u128 q, rem, s2;
        poly_divmod(r0, r1, &q, &rem);
        s2 = s0 ^ poly_mul(q, s1);
        r0 = r1;
        r1 = rem;
        s0 = s1;
        s1 = s2;
    }
    if (r0 != 1)
        return 0;
    poly_divmod(s0, f, NULL, &r1);
    return (u64)r1;
}

/* Weight of data strip k in Q.  k < p: g^k (Corollary 3.2.4, with g = x);
 * p <= k <= 2p-2: Id + g^(k-p+1), equation (qext) of Section 3.3. */
u64 oracle_weight(unsigned p, unsigned k)
{
    if (k < p)
        return oracle_ring_xpow(p, k);
    return 1u ^ oracle_ring_xpow(p, k - p + 1);
}

/* Lemma 3.3.1: the order d of 2 modulo the prime p (R is a field exactly
 * when d = p - 1). */
unsigned oracle_ord2(unsigned p)
{
    unsigned d = 1, v = 2 % p;
    while (v != 1) {
        v = (2 * v) % p;
        d++;
    }
    return d;
}

/* Greatest common divisor in F2[x] by Euclid's algorithm. */
static u128 poly_gcd(u128 a, u128 b)
{
    while (b != 0) {
        u128 r;
        poly_divmod(a, b, NULL, &r);
        a = b;
        b = r;
    }
    return a;
}

/* Condition (3) of Theorem 3.3.3 for the prime p (3 <= p <= 127): for every
 * 0 < m < p the polynomials X^p + 1 and X^m + X + 1 are coprime.  Returns 1
 * when it holds, i.e. when the cone {g^k} + {Id + g^m} extends the code to
 * 2p - 1 data strips. */
int oracle_cone_extends(unsigned p)
{
    u128 xp1 = (((u128)1) << p) | 1u;
    for (unsigned m = 1; m < p; m++) {
        u128 t = (((u128)1) << m) ^ 2u ^ 1u;
        if (poly_gcd(xp1, t) != 1)
            return 0;
    }
    return 1;
}

/* out[t] = x^k * in[t] in R, for n elements. */
void oracle_mul_xpow_array(unsigned p, unsigned k, const u64 *in, u64 *out, size_t n)
{
    u64 g = oracle_ring_xpow(p, k);
    for (size_t t = 0; t < n; t++)
        out[t] = oracle_ring_mul(p, g, in[t]);
}

/* ------------------------------------------------------ bit slicing */

typedef struct {
    uint8_t *base;
    u64 row_stride, strip_stride, stripe_stride;
    unsigned rows;       /* p - 1 */
    int horizontal;      /* 1: element e is bits [e*rows, (e+1)*rows) of the strip */
} layout_t;

static uint8_t *row_ptr(const layout_t *L, u64 s, unsigned k, unsigned r)
{
    return L->base + s * L->stripe_stride + (u64)k * L->strip_stride + (u64)r * L->row_stride;
}

/* Polynomial of codeword b (a bit position, or an element of a horizontal
 * strip) of strip k of stripe s. */
static u64 gather(const layout_t *L, u64 s, unsigned k, u64 b)
{
    u64 a = 0;
    if (L->horizontal) {
        const uint8_t *strip = L->base + s * L->stripe_stride + (u64)k * L->strip_stride;
        for (unsigned r = 0; r < L->rows; r++) {
            u64 t = b * L->rows + r;
            a |= (u64)((strip[t >> 3] >> (t & 7)) & 1u) << r;
        }
        return a;
    }
    for (unsigned r = 0; r < L->rows; r++) {
        const uint8_t *row = row_ptr(L, s, k, r);
        a |= (u64)((row[b >> 3] >> (b & 7)) & 1u) << r;
    }
    return a;
}

static void scatter(const layout_t *L, u64 s, unsigned k, u64 b, u64 a)
{
    if (L->horizontal) {
        uint8_t *strip = L->base + s * L->stripe_stride + (u64)k * L->strip_stride;
        for (unsigned r = 0; r < L->rows; r++) {
            u64 t = b * L->rows + r;
            uint8_t m = (uint8_t)(1u << (t & 7));
            if ((a >> r) & 1u)
                strip[t >> 3] |= m;
            else
                strip[t >> 3] &= (uint8_t)~m;
        }
        return;
    }
    for (unsigned r = 0; r < L->rows; r++) {
        uint8_t *row = row_ptr(L, s, k, r);
        uint8_t m = (uint8_t)(1u << (b & 7));
        if ((a >> r) & 1u)
            row[b >> 3] |= m;
        else
            row[b >> 3] &= (uint8_t)~m;
    }
}

static int check_args(unsigned p, unsigned N)
{
    if (p < 3 || p > 61 || (p % 2) == 0)
        return -1;
    for (unsigned t = 3; t * t <= p; t += 2)
        if (p % t == 0)
            return -1;
    if (N < 1 || N > 2 * p - 1)
        return -1;
    if (N > p && !oracle_cone_extends(p))
        return -1;
    return 0;
}

/* ------------------------------------------------------------- encode */

/* Equation (znparity) of Corollary 3.2.4 with g = S_p and g_k = g^k, extended
 * by (qext) for k >= p: P = sum_k d_k, Q = sum_k g_k d_k.  Writes strips N
 * and N+1. */
static void encode_layout(const layout_t *Lp, unsigned p, unsigned N, u64 n_codewords, u64 n_stripes)
{
    const layout_t L = *Lp;
    u64 g[128];
    for (unsigned k = 0; k < N; k++)
        g[k] = oracle_weight(p, k);
    for (u64 s = 0; s < n_stripes; s++) {
        for (u64 b = 0; b < n_codewords; b++) {
            u64 P = 0, Q = 0;
            for (unsigned k = 0; k < N; k++) {
                u64 d = gather(&L, s, k, b);
                P ^= d;
                Q ^= oracle_ring_mul(p, g[k], d);
            }
            scatter(&L, s, N, b, P);
            scatter(&L, s, N + 1, b, Q);
        }
    }
}

int oracle_encode(unsigned p, unsigned N, u64 C, uint8_t *buf, u64 n_stripes,
                  u64 row_stride, u64 strip_stride, u64 stripe_stride)
{
    if (check_args(p, N))
        return -1;
    layout_t L = {buf, row_stride, strip_stride, stripe_stride, p - 1, 0};
    encode_layout(&L, p, N, 8 * C, n_stripes);
    return 0;
}

/* ------------------------------------------------------------ recover */

/* Solve the parity equations (cone) of Lemma 3.1.2 for the pair of lost
 * strips i < j (0-based; strip N is P = d_{N+1} of the lemma and strip N+1
 * is Q = d_{N+2}), following the four cases of its proof:
 *   (P, Q):          recompute both parities;
 *   (d_i, P):        d_i = g_i^{-1} (Q + sum_{k != i} g_k d_k), then P;
 *   (d_i, Q):        d_i = P + sum_{k != i} d_k (RAID-5), then Q;
 *   (d_i, d_j):      d_j = (g_i + g_j)^{-1} (g_i P + Q + sum_{k != i,j} (g_k + g_i) d_k),
 *                    then d_i = P + sum_{k != i} d_k.
 * Inverses come from the extended Euclidean algorithm.  The erased strips'
 * contents are never read. */
static int recover_one(const layout_t *L, unsigned p, unsigned N, u64 s, u64 b,
                       unsigned i, unsigned j, const u64 *g)
{
    u64 d[128];
    if (i == N && j == N + 1) {
        u64 P = 0, Q = 0;
        for (unsigned k = 0; k < N; k++) {
            d[k] = gather(L, s, k, b);
            P ^= d[k];
            Q ^= oracle_ring_mul(p, g[k], d[k]);
        }
        scatter(L, s, N, b, P);
        scatter(L, s, N + 1, b, Q);
        return 0;
    }
    if (j == N) { /* d_i and P lost */
        u64 Q = gather(L, s, N + 1, b);
        u64 acc = Q;
        for (unsigned k = 0; k < N; k++) {
            if (k == i)
                continue;
            d[k] = gather(L, s, k, b);
            acc ^= oracle_ring_mul(p, g[k], d[k]);
        }
        u64 gi_inv = oracle_ring_inv(p, g[i]);
        if (gi_inv == 0)
            return -3;
        d[i] = oracle_ring_mul(p, gi_inv, acc);
        u64 P = 0;
        for (unsigned k = 0; k < N; k++)
            P ^= d[k];
        scatter(L, s, i, b, d[i]);
        scatter(L, s, N, b, P);
        return 0;
    }
    if (j == N + 1) { /* d_i and Q lost */
        u64 P = gather(L, s, N, b);
        u64 acc = P;
        for (unsigned k = 0; k < N; k++) {
            if (k == i)
                continue;
            d[k] = gather(L, s, k, b);
            acc ^= d[k];
        }
        d[i] = acc;
        u64 Q = 0;
        for (unsigned k = 0; k < N; k++)
            Q ^= oracle_ring_mul(p, g[k], d[k]);
        scatter(L, s, i, b, d[i]);
        scatter(L, s, N + 1, b, Q);
        return 0;
    }
    /* two data strips lost */
    u64 P = gather(L, s, N, b);
    u64 Q = gather(L, s, N + 1, b);
    u64 rhs = oracle_ring_mul(p, g[i], P) ^ Q;
    for (unsigned k = 0; k < N; k++) {
        if (k == i || k == j)
            continue;
        d[k] = gather(L, s, k, b);
        rhs ^= oracle_ring_mul(p, g[k] ^ g[i], d[k]);
    }
    u64 sum_inv = oracle_ring_inv(p, g[i] ^ g[j]);
    if (sum_inv == 0) /* the pair is not in a cone: Theorem 3.3.3 fails for p */
        return -3;
    d[j] = oracle_ring_mul(p, sum_inv, rhs);
    u64 di = P ^ d[j];
    for (unsigned k = 0; k < N; k++)
        if (k != i && k != j)
            di ^= d[k];
    scatter(L, s, i, b, di);
    scatter(L, s, j, b, d[j]);
    return 0;
}

/* Recover strips i < j of stripes [0, n_stripes) in place.  pairs, when not
 * NULL, gives a per-stripe (i, j) as two bytes per stripe and overrides i, j. */
static int recover_layout(const layout_t *L, unsigned p, unsigned N, u64 n_codewords, u64 n_stripes,
                          unsigned i, unsigned j, const uint8_t *pairs)
{
    u64 g[128];
    for (unsigned k = 0; k < N; k++)
        g[k] = oracle_weight(p, k);
    for (u64 s = 0; s < n_stripes; s++) {
        unsigned a = pairs ? pairs[2 * s] : i;
        unsigned c = pairs ? pairs[2 * s + 1] : j;
        if (!(a < c && c < N + 2))
            return -2;
        for (u64 b = 0; b < n_codewords; b++)
            if (recover_one(L, p, N, s, b, a, c, g))
                return -3;
    }
    return 0;
}

int oracle_recover(unsigned p, unsigned N, u64 C, uint8_t *buf, u64 n_stripes,
                   u64 row_stride, u64 strip_stride, u64 stripe_stride,
                   unsigned i, unsigned j, const uint8_t *pairs)
{
    if (check_args(p, N))
        return -1;
    layout_t L = {buf, row_stride, strip_stride, stripe_stride, p - 1, 0};
    return recover_layout(&L, p, N, 8 * C, n_stripes, i, j, pairs);
}

/* ---------------------------------------------------- horizontal strips */

/* Encode and recovery of stripes in the horizontal representation of Section
 * 4.5 (see the header): strips of strip_bytes bytes, strip_bytes*8 a multiple
 * of p-1, so a strip holds strip_bytes*8/(p-1) ring elements; strip k of
 * stripe s at buf + s*stripe_stride + k*strip_stride.  Same code, same
 * Lemma 3.1.2 case analysis as the bit-sliced functions. */
int oracle_h_encode(unsigned p, unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes,
                    u64 strip_stride, u64 stripe_stride)
{
    if (check_args(p, N) || (strip_bytes * 8) % (p - 1))
        return -1;
    layout_t L = {buf, 0, strip_stride, stripe_stride, p - 1, 1};
    encode_layout(&L, p, N, strip_bytes * 8 / (p - 1), n_stripes);
    return 0;
}

int oracle_h_recover(unsigned p, unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes,
                     u64 strip_stride, u64 stripe_stride, unsigned i, unsigned j, const uint8_t *pairs)
{
    if (check_args(p, N) || (strip_bytes * 8) % (p - 1))
        return -1;
    layout_t L = {buf, 0, strip_stride, stripe_stride, p - 1, 1};
    return recover_layout(&L, p, N, strip_bytes * 8 / (p - 1), n_stripes, i, j, pairs);
}

/* ------------------------------------------------------------- update */

/* Small write: replace data strip i of stripe `stripe` with new_strip (p-1
 * rows of C bytes, rows new_row_stride apart) and bring P and Q back to the
 * values equation (znparity) gives for the new data.  The oracle does this by
 * its definition -- store the new strip, re-encode the stripe -- rather than
 * by the incremental rule P += delta, Q += g^i delta. */
int oracle_update(unsigned p, unsigned N, u64 C, uint8_t *buf, u64 stripe,
                  u64 row_stride, u64 strip_stride, u64 stripe_stride,
                  unsigned i, const uint8_t *new_strip, u64 new_row_stride)
{
    if (check_args(p, N) || i >= N)
        return -1;
    layout_t L = {buf, row_stride, strip_stride, stripe_stride, p - 1, 0};
    for (unsigned r = 0; r < p - 1; r++)
        memmove(row_ptr(&L, stripe, i, r), new_strip + (u64)r * new_row_stride, C);
    return oracle_encode(p, N, C, buf + stripe * stripe_stride, 1, row_stride, strip_stride,
                         stripe_stride);
}

/* -------------------------------------------------------- degraded read */

/* Read strip j of stripe `stripe` as if it were lost, rebuilding it from the
 * other strips with the equation that does not involve the other parity:
 * a data strip or P from the first equation of (znparity) (the RAID-5 rule),
 * Q from the second.  The result goes to out (p-1 rows, out_row_stride apart);
 * strip j itself is not read. */
int oracle_degraded_read(unsigned p, unsigned N, u64 C, const uint8_t *buf, u64 stripe,
                         u64 row_stride, u64 strip_stride, u64 stripe_stride, unsigned j,
                         uint8_t *out, u64 out_row_stride)
{
    if (check_args(p, N) || j >= N + 2)
        return -1;
    layout_t L = {(uint8_t *)buf, row_stride, strip_stride, stripe_stride, p - 1, 0};
    layout_t O = {out, out_row_stride, 0, 0, p - 1, 0};
    for (u64 b = 0; b < 8 * C; b++) {
        u64 v = 0;
        if (j == N + 1) {
            for (unsigned k = 0; k < N; k++)
                v ^= oracle_ring_mul(p, oracle_weight(p, k), gather(&L, stripe, k, b));
        } else {
            for (unsigned k = 0; k <= N; k++)
                if (k != j)
                    v ^= gather(&L, stripe, k, b);
        }
        scatter(&O, 0, 0, b, v);
    }
    return 0;
}

/* ============================================== large primes (p <= 257)
 *
 * The same definitions for primes whose strips do not fit a machine word --
 * Section 3.4 names Z_257 (256-bit elements) beside Z_17 -- on polynomials
 * held as arrays of coefficients, one byte per coefficient (0 or 1), and
 * stripes in the horizontal representation.  Nothing here is shared with the
 * 128-bit code above: multiplication is schoolbook, reduction is long
 * division by f, inverses come from the extended Euclidean algorithm.  The
 * tests run both on the primes both accept and require equal results. */

#define BP_MAXP 257
#define BP_CAP (2 * BP_MAXP + 2) /* room for a product of two residues */

typedef struct {
    int deg;               /* -1 for the zero polynomial */
    uint8_t c[BP_CAP];     /* c[t] = coefficient of x^t */
} bpoly;

static void bp_zero(bpoly *a)
{
    memset(a->c, 0, sizeof(a->c));
    a->deg = -1;
}

static void bp_fix_deg(bpoly *a)
{
    int d = BP_CAP - 1;
    while (d >= 0 && a->c[d] == 0)
        d--;
    a->deg = d;
}

static void bp_add(const bpoly *a, const bpoly *b, bpoly *out)
{
    for (int t = 0; t < BP_CAP; t++)
        out->c[t] = a->c[t] ^ b->c[t];
    bp_fix_deg(out);
}

/* Carry-less product; deg(a) + deg(b) < BP_CAP. */
static void bp_mul(const bpoly *a, const bpoly *b, bpoly *out)
{
    bpoly r;
    bp_zero(&r);
    for (int i = 0; i <= a->deg; i++) {
        if (!a->c[i])
            continue;
        for (int j = 0; j <= b->deg; j++)
            r.c[i + j] ^= b->c[j];
    }
    bp_fix_deg(&r);
    *out = r;
}

/* Long division a = q*m + r, m nonzero.  q may be NULL. */
static void bp_divmod(const bpoly *a, const bpoly *m, bpoly *q, bpoly *r)
{
    bpoly rem = *a, quo;
    bp_zero(&quo);
    while (rem.deg >= m->deg) {
        const int shift = rem.deg - m->deg;
        quo.c[shift] ^= 1;
        for (int t = 0; t <= m->deg; t++)
            rem.c[t + shift] ^= m->c[t];
        bp_fix_deg(&rem);
    }
    bp_fix_deg(&quo);
    if (q)
        *q = quo;
    *r = rem;
}

/* f = 1 + x + ... + x^(p-1) */
static void bp_f(unsigned p, bpoly *f)
{
    bp_zero(f);
    for (unsigned t = 0; t < p; t++)
        f->c[t] = 1;
    f->deg = (int)p - 1;
}

static void bp_ring_mul(unsigned p, const bpoly *a, const bpoly *b, bpoly *out)
{
    bpoly f, prod;
    bp_f(p, &f);
    bp_mul(a, b, &prod);
    bp_divmod(&prod, &f, NULL, out);
}

/* x^k reduced modulo f, k < BP_CAP. */
static void bp_xpow(unsigned p, unsigned k, bpoly *out)
{
    bpoly f, m;
    bp_f(p, &f);
    bp_zero(&m);
    m.c[k] = 1;
    m.deg = (int)k;
    bp_divmod(&m, &f, NULL, out);
}

/* Inverse in R by the extended Euclidean algorithm; returns 0 (and leaves
 * out zero) when gcd(a, f) != 1. */
static int bp_ring_inv(unsigned p, const bpoly *a, bpoly *out)
{
    bpoly f, r0, r1, s0, s1;
    bp_f(p, &f);
    bp_divmod(a, &f, NULL, &r1);
    bp_zero(out);
    if (r1.deg < 0)
        return 0;
    r0 = f;
    bp_zero(&s0);
    bp_zero(&s1);
    s1.c[0] = 1;
    s1.deg = 0;
    while (r1.deg >= 0) {
        bpoly q, rem, qs, s2;
        bp_divmod(&r0, &r1, &q, &rem);
        bp_mul(&q, &s1, &qs);
        bp_add(&s0, &qs, &s2);
        r0 = r1;
        r1 = rem;
        s0 = s1;
        s1 = s2;
    }
    if (r0.deg != 0)
        return 0;
    bp_divmod(&s0, &f, NULL, out);
    return 1;
}

/* Weight of data strip k < p in Q: x^k (Corollary 3.2.4). */
static void bp_weight(unsigned p, unsigned k, bpoly *out)
{
    bp_xpow(p, k, out);
}

/* Residues to and from packed bit strings: bit t (bit t%8 of byte t/8) is
 * the coefficient of x^t, t < p-1. */
static void bp_from_bits(unsigned p, const uint8_t *bits, bpoly *a)
{
    bp_zero(a);
    for (unsigned t = 0; t + 1 < p; t++)
        a->c[t] = (bits[t >> 3] >> (t & 7)) & 1u;
    bp_fix_deg(a);
}

static void bp_to_bits(unsigned p, const bpoly *a, uint8_t *bits)
{
    memset(bits, 0, (p - 1 + 7) / 8);
    for (unsigned t = 0; t + 1 < p; t++)
        bits[t >> 3] |= (uint8_t)(a->c[t] << (t & 7));
}

static int bp_check_prime(unsigned p)
{
    if (p < 3 || p > BP_MAXP || (p % 2) == 0)
        return -1;
    for (unsigned t = 3; t * t <= p; t += 2)
        if (p % t == 0)
            return -1;
    return 0;
}

/* Ring operations on packed residues (bits of (p-1+7)/8 bytes), for the tests. */
int oracle_big_ring_mul(unsigned p, const uint8_t *a, const uint8_t *b, uint8_t *out)
{
    bpoly x, y, z;
    if (bp_check_prime(p))
        return -1;
    bp_from_bits(p, a, &x);
    bp_from_bits(p, b, &y);
    bp_ring_mul(p, &x, &y, &z);
    bp_to_bits(p, &z, out);
    return 0;
}

int oracle_big_ring_xpow(unsigned p, unsigned k, uint8_t *out)
{
    bpoly z;
    if (bp_check_prime(p) || k >= BP_CAP)
        return -1;
    bp_xpow(p, k, &z);
    bp_to_bits(p, &z, out);
    return 0;
}

/* Returns 1 and the inverse when a is a unit, 0 otherwise. */
int oracle_big_ring_inv(unsigned p, const uint8_t *a, uint8_t *out)
{
    bpoly x, z;
    if (bp_check_prime(p))
        return -1;
    bp_from_bits(p, a, &x);
    const int ok = bp_ring_inv(p, &x, &z);
    bp_to_bits(p, &z, out);
    return ok;
}

/* Element e of strip k of stripe s of a horizontal layout: bits
 * [e(p-1), (e+1)(p-1)) of the strip, little-endian. */
static void bp_gather(unsigned p, const uint8_t *buf, u64 ss, u64 st, u64 s, unsigned k, u64 e, bpoly *a)
{
    const uint8_t *strip = buf + s * st + (u64)k * ss;
    bp_zero(a);
    for (unsigned r = 0; r + 1 < p; r++) {
        const u64 t = e * (p - 1) + r;
        a->c[r] = (strip[t >> 3] >> (t & 7)) & 1u;
    }
    bp_fix_deg(a);
}

static void bp_scatter(unsigned p, uint8_t *buf, u64 ss, u64 st, u64 s, unsigned k, u64 e, const bpoly *a)
{
    uint8_t *strip = buf + s * st + (u64)k * ss;
    for (unsigned r = 0; r + 1 < p; r++) {
        const u64 t = e * (p - 1) + r;
        const uint8_t m = (uint8_t)(1u << (t & 7));
        if (a->c[r])
            strip[t >> 3] |= m;
        else
            strip[t >> 3] &= (uint8_t)~m;
    }
}

static int bp_check_args(unsigned p, unsigned N, u64 strip_bytes)
{
    if (bp_check_prime(p) || N < 1 || N > p || (strip_bytes * 8) % (p - 1))
        return -1;
    return 0;
}

/* Equation (znparity): P = sum d_k, Q = sum x^k d_k, on horizontal stripes of
 * any odd prime p <= 257 (base code, N <= p). */
int oracle_hbig_encode(unsigned p, unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes,
                       u64 strip_stride, u64 stripe_stride)
{
    if (bp_check_args(p, N, strip_bytes))
        return -1;
    static bpoly g[BP_MAXP];
    for (unsigned k = 0; k < N; k++)
        bp_weight(p, k, &g[k]);
    const u64 n_el = strip_bytes * 8 / (p - 1);
    for (u64 s = 0; s < n_stripes; s++)
        for (u64 e = 0; e < n_el; e++) {
            bpoly P, Q, d, t;
            bp_zero(&P);
            bp_zero(&Q);
            for (unsigned k = 0; k < N; k++) {
                bp_gather(p, buf, strip_stride, stripe_stride, s, k, e, &d);
                bp_add(&P, &d, &P);
                bp_ring_mul(p, &g[k], &d, &t);
                bp_add(&Q, &t, &Q);
            }
            bp_scatter(p, buf, strip_stride, stripe_stride, s, N, e, &P);
            bp_scatter(p, buf, strip_stride, stripe_stride, s, N + 1, e, &Q);
        }
    return 0;
}

/* Lemma 3.1.2's four cases for the lost pair i < j (strip N = P, N+1 = Q),
 * with inverses by the extended Euclidean algorithm, on horizontal stripes of
 * any odd prime p <= 257.  pairs, when not NULL, gives (i, j) per stripe as
 * two 16-bit numbers (strip indices reach 258 at p = 257). */
int oracle_hbig_recover(unsigned p, unsigned N, u64 strip_bytes, uint8_t *buf, u64 n_stripes,
                        u64 strip_stride, u64 stripe_stride, unsigned i, unsigned j, const uint16_t *pairs)
{
    if (bp_check_args(p, N, strip_bytes))
        return -1;
    static bpoly g[BP_MAXP];
    for (unsigned k = 0; k < N; k++)
        bp_weight(p, k, &g[k]);
    const u64 n_el = strip_bytes * 8 / (p - 1);
    const u64 ss = strip_stride, st = stripe_stride;
    for (u64 s = 0; s < n_stripes; s++) {
        const unsigned a = pairs ? pairs[2 * s] : i;
        const unsigned b = pairs ? pairs[2 * s + 1] : j;
        if (!(a < b && b < N + 2))
            return -2;
        /* the inverse this pair needs: of g_a (data + P), of g_a + g_b (two data) */
        bpoly inv;
        bp_zero(&inv);
        if (b == N) {
            if (!bp_ring_inv(p, &g[a], &inv))
                return -3;
        } else if (b < N) {
            bpoly sum;
            bp_add(&g[a], &g[b], &sum);
            if (!bp_ring_inv(p, &sum, &inv))
                return -3;
        }
        for (u64 e = 0; e < n_el; e++) {
            bpoly d, t, acc, P, Q;
            if (a == N) { /* P and Q: encode */
                bp_zero(&P);
                bp_zero(&Q);
                for (unsigned k = 0; k < N; k++) {
                    bp_gather(p, buf, ss, st, s, k, e, &d);
                    bp_add(&P, &d, &P);
                    bp_ring_mul(p, &g[k], &d, &t);
                    bp_add(&Q, &t, &Q);
                }
                bp_scatter(p, buf, ss, st, s, N, e, &P);
                bp_scatter(p, buf, ss, st, s, N + 1, e, &Q);
            } else if (b == N) { /* d_a and P: d_a = g_a^{-1}(Q + sum_{k != a} g_k d_k), then P */
                bpoly da;
                bp_gather(p, buf, ss, st, s, N + 1, e, &acc);
                for (unsigned k = 0; k < N; k++) {
                    if (k == a)
                        continue;
                    bp_gather(p, buf, ss, st, s, k, e, &d);
                    bp_ring_mul(p, &g[k], &d, &t);
                    bp_add(&acc, &t, &acc);
                }
                bp_ring_mul(p, &inv, &acc, &da);
                P = da;
                for (unsigned k = 0; k < N; k++) {
                    if (k == a)
                        continue;
                    bp_gather(p, buf, ss, st, s, k, e, &d);
                    bp_add(&P, &d, &P);
                }
                bp_scatter(p, buf, ss, st, s, a, e, &da);
                bp_scatter(p, buf, ss, st, s, N, e, &P);
            } else if (b == N + 1) { /* d_a and Q: RAID-5, then Q */
                bpoly da;
                bp_gather(p, buf, ss, st, s, N, e, &da);
                for (unsigned k = 0; k < N; k++) {
                    if (k == a)
                        continue;
                    bp_gather(p, buf, ss, st, s, k, e, &d);
                    bp_add(&da, &d, &da);
                }
                bp_zero(&Q);
                for (unsigned k = 0; k < N; k++) {
                    if (k == a)
                        d = da;
                    else
                        bp_gather(p, buf, ss, st, s, k, e, &d);
                    bp_ring_mul(p, &g[k], &d, &t);
                    bp_add(&Q, &t, &Q);
                }
                bp_scatter(p, buf, ss, st, s, a, e, &da);
                bp_scatter(p, buf, ss, st, s, N + 1, e, &Q);
            } else { /* two data: d_b = (g_a + g_b)^{-1}(g_a P + Q + sum_{k != a,b} (g_k + g_a) d_k) */
                bpoly db, da, w;
                bp_gather(p, buf, ss, st, s, N, e, &P);
                bp_gather(p, buf, ss, st, s, N + 1, e, &Q);
                bp_ring_mul(p, &g[a], &P, &acc);
                bp_add(&acc, &Q, &acc);
                da = P;
                for (unsigned k = 0; k < N; k++) {
                    if (k == a || k == b)
                        continue;
                    bp_gather(p, buf, ss, st, s, k, e, &d);
                    bp_add(&g[k], &g[a], &w);
                    bp_ring_mul(p, &w, &d, &t);
                    bp_add(&acc, &t, &acc);
                    bp_add(&da, &d, &da);
                }
                bp_ring_mul(p, &inv, &acc, &db);
                bp_add(&da, &db, &da);
                bp_scatter(p, buf, ss, st, s, a, e, &da);
                bp_scatter(p, buf, ss, st, s, b, e, &db);
            }
        }
    }
    return 0;
}
