// rcg_ring.cu -- host-side arithmetic in R = F2[x]/(1 + x + ... + x^(p-1))
// for the tables the engine reads: inverses of the trinomials that the
// extended Q-parity of Section 3.3 (equation qext) needs, and the test of
// Theorem 3.3.3 that decides whether a prime allows that extension.
//
// Elements are bit masks of p bits over the lift F2[x]/(x^p - 1) (bit m =
// coefficient of x^m); reduce() maps a lifted element to its residue modulo
// f, which has no x^(p-1) term.  Since x^p - 1 = (x - 1) f with coprime
// factors, the lift is F2 x R and every operation here acts on R through the
// projection.
//
// Inverses.  By Lemma 3.3.1, R is a product of copies of GF(2^d), d the order
// of 2 modulo p, so every unit u of R satisfies u^(2^d - 1) = 1 and
// u^(-1) = u^(2^d - 2) = prod_{t=1}^{d-1} u^(2^t).  Squaring in the lift is
// the Frobenius map u(x) -> u(x^2), a permutation of exponents m -> 2m mod p,
// so the inverse costs d - 1 products of p-bit masks.  The candidate is
// accepted only when u * u^(-1) = 1 in R; otherwise u is not a unit.
#include <stdint.h>

#include <mutex>

#include "rcg_internal.h"

namespace rcg {

namespace {

uint64_t all_ones(uint32_t p) { return (p == 64) ? ~0ull : ((1ull << p) - 1); }

// x^s * a in the lift: a cyclic rotation of p bits.
uint64_t rotate(uint32_t p, uint64_t a, uint32_t s) {
    s %= p;
    if (s == 0) return a;
    return ((a << s) | (a >> (p - s))) & all_ones(p);
}

uint64_t mul_lift(uint32_t p, uint64_t a, uint64_t b) {
    uint64_t c = 0;
    for (uint32_t m = 0; m < p; ++m)
        if ((a >> m) & 1) c ^= rotate(p, b, m);
    return c;
}

// a(x^2) in the lift (the Frobenius map).
uint64_t frobenius(uint32_t p, uint64_t a) {
    uint64_t c = 0;
    for (uint32_t m = 0; m < p; ++m)
        if ((a >> m) & 1) c |= 1ull << ((2 * m) % p);
    return c;
}

}  // namespace

uint64_t ring_reduce(uint32_t p, uint64_t a) {
    // x^(p-1) = 1 + x + ... + x^(p-2) modulo f
    if ((a >> (p - 1)) & 1) a ^= all_ones(p);
    return a;
}

uint32_t order_of_two(uint32_t p) {
    uint32_t d = 1, v = 2 % p;
    while (v != 1) {
        v = (2 * v) % p;
        ++d;
    }
    return d;
}

uint64_t ring_inverse(uint32_t p, uint64_t u) {
    const uint32_t d = order_of_two(p);
    uint64_t f = u, inv = 1;
    for (uint32_t t = 1; t < d; ++t) {
        f = frobenius(p, f);
        inv = mul_lift(p, inv, f);
    }
    inv = ring_reduce(p, inv);
    return ring_reduce(p, mul_lift(p, u, inv)) == 1 ? inv : 0;
}

void trinomial_inverses(uint32_t p, uint64_t *masks) {
    for (uint32_t u = 0; u < p; ++u)
        for (uint32_t v = 0; v < p; ++v)
            masks[u * p + v] = ring_inverse(p, 1ull ^ (1ull << u) ^ (1ull << v));
}

bool cone_extends(uint32_t p) {
    // Theorem 3.3.3: {x^k} together with {1 + x^m} is a cone exactly when
    // every 1 + x^u + x^v, 0 < u < v < p, is a unit of R.
    static std::mutex lock;
    static int8_t memo[kMaxP + 1] = {};
    if (p < 3 || p > static_cast<uint32_t>(kMaxP)) return false;
    std::lock_guard<std::mutex> g(lock);
    if (memo[p] == 0) {
        bool ok = true;
        for (uint32_t u = 1; u < p && ok; ++u)
            for (uint32_t v = u + 1; v < p && ok; ++v)
                ok = ring_inverse(p, 1ull ^ (1ull << u) ^ (1ull << v)) != 0;
        memo[p] = ok ? 1 : -1;
    }
    return memo[p] > 0;
}

}  // namespace rcg
