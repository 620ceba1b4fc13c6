"""Pins for the oracle's large-prime path (coefficient-array polynomials,
any odd prime p <= 257), used for Z_257 -- the 256-bit-element instance that
Section 3.4 names beside Z_17 -- in the horizontal representation of Section
4.5 (element e of a strip = bytes [32e, 32e + 32), little-endian).

Independent models:
  * the 128-bit oracle code (already pinned) on every prime both accept:
    same products, inverses, encodes and recoveries;
  * at p = 257, facts the paper and the algebra fix: x^p = 1 and x has order
    p (Lemma 3.4.1), x^(p-1) = 1 + ... + x^(p-2) (the last column of S_p),
    sum x^k = 0 (Lemma 3.2.2), the word formula of Section 4.6 for x^k y on a
    256-bit word, R a product of fields GF(2^16) (Lemma 3.3.1, ord_257(2) =
    16, so a^(2^16) = a), the closed-form inverse (1 + x^z)^(-1) =
    sum_{t <= (p-1)/2} x^(2tz) of Section 4.6, EVENODD's diagonal parity
    (Section 3.4 says the construction is EVENODD), and the two-data
    reconstruction of Section 4.6 evaluated with its own Horner forms.
"""
import random

import numpy as np
import pytest

from test_oracle_pins import all_pairs

P = 257
W = 256                     # bits of an element
ONES = (1 << W) - 1
POISON = 0xA5


# ---------------------------------------------- the paper's word formulas

def xk_word(y, k):
    """Section 4.6's formula for g^k y on a (p-1)-bit word, p = 257:
    (y << k) ^ (y >> (p - k)) ^ (bit p-1-k of y ? all ones : 0), 0 <= k <= 256,
    shifts logical and kept to 256 bits."""
    k %= P
    if k == 0:
        return y
    r = ((y << k) & ONES) ^ (y >> (P - k))
    if (y >> (P - 1 - k)) & 1:
        r ^= ONES
    return r


def mul_word(a, y):
    """a * y as the sum over the set bits m of a of g^m y."""
    acc = 0
    m = 0
    while a:
        if a & 1:
            acc ^= xk_word(y, m)
        a >>= 1
        m += 1
    return acc


def closed_inverse(z):
    """Section 4.6: (1 + g^z)^(-1) = sum_{t=0}^{(p-1)/2} g^(2tz), as a word."""
    return mul_word_sum([(2 * t * z) % P for t in range((P - 1) // 2 + 1)])


def mul_word_sum(exps):
    acc = 0
    for e in exps:
        acc ^= xk_word(1, e)
    return acc


def elements(strip):
    return [int.from_bytes(bytes(strip[32 * e:32 * e + 32]), "little") for e in range(len(strip) // 32)]


def h_random(seed, N, B, S):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(S, N + 2, B), dtype=np.uint8)


# ------------------------------------- the same answers as the 128-bit code

@pytest.mark.parametrize("p", [3, 5, 7, 11, 13, 17, 29, 59, 61])
def test_big_ring_equals_word_ring_on_small_primes(oracle, p):
    rnd = random.Random(p)
    for k in range(0, 127):
        assert oracle.big_ring_xpow(p, k) == oracle.ring_xpow(p, k)
    for _ in range(60):
        a, b = rnd.getrandbits(p - 1), rnd.getrandbits(p - 1)
        assert oracle.big_ring_mul(p, a, b) == oracle.ring_mul(p, a, b)
        assert oracle.big_ring_inv(p, a) == oracle.ring_inv(p, a)


@pytest.mark.parametrize("p,N,B,S", [(3, 3, 16, 2), (5, 4, 16, 2), (5, 5, 32, 2), (13, 12, 24, 2),
                                     (17, 16, 64, 2), (17, 1, 32, 1), (29, 20, 56, 1)])
def test_hbig_equals_h_on_small_primes(oracle, p, N, B, S):
    h = h_random(p + N, N, B, S)
    a, b = h.copy(), h.copy()
    oracle.h_encode(p, N, B, a, S)
    oracle.hbig_encode(p, N, B, b, S)
    assert np.array_equal(a, b)
    pairs = all_pairs(N)
    rng = np.random.default_rng(p)
    for t in rng.choice(len(pairs), min(12, len(pairs)), replace=False):
        i, j = pairs[t]
        x, y = a.copy(), a.copy()
        for z in (x, y):
            z[:, i] = POISON
            z[:, j] = POISON ^ 0x3C
        oracle.h_recover(p, N, B, x, S, i, j)
        oracle.hbig_recover(p, N, B, y, S, i, j)
        assert np.array_equal(x, y), (i, j)
        assert np.array_equal(y, a), (i, j)


# ---------------------------------------------------------- Z_257 algebra

def test_x_has_order_p(oracle):
    # Lemma 3.4.1(i): S_p^p = Id and no smaller power is
    assert oracle.big_ring_xpow(P, P) == 1
    assert oracle.big_ring_xpow(P, 0) == 1
    for k in range(1, P):
        assert oracle.big_ring_xpow(P, k) != 1


def test_last_column_of_the_sylvester_matrix(oracle):
    # x * x^(p-2) = x^(p-1) = 1 + x + ... + x^(p-2): the all-ones column
    assert oracle.big_ring_xpow(P, P - 1) == ONES
    for k in range(P - 1):
        assert oracle.big_ring_xpow(P, k) == 1 << k


def test_sum_of_the_powers_is_zero(oracle):
    # Lemma 3.2.2
    acc = 0
    for k in range(P):
        acc ^= oracle.big_ring_xpow(P, k)
    assert acc == 0


def test_products_match_the_word_formula(oracle):
    rnd = random.Random(257)
    for k in list(range(0, 9)) + [15, 16, 17, 100, 128, 200, 255, 256]:
        for _ in range(6):
            y = rnd.getrandbits(W)
            assert oracle.big_ring_mul(P, oracle.big_ring_xpow(P, k), y) == xk_word(y, k), k
    for _ in range(10):
        a, y = rnd.getrandbits(W), rnd.getrandbits(W)
        assert oracle.big_ring_mul(P, a, y) == mul_word(a, y)
        assert oracle.big_ring_mul(P, a, y) == oracle.big_ring_mul(P, y, a)


def test_frobenius_order_sixteen(oracle):
    # Lemma 3.3.1: ord_257(2) = 16, R = GF(2^16)^16, so squaring 16 times is
    # the identity and squaring is additive
    assert oracle.ord2(17) == 8  # the helper itself, on a prime the paper discusses
    d, v = 1, 2
    while v != 1:
        v = 2 * v % P
        d += 1
    assert d == 16
    rnd = random.Random(16)
    for _ in range(4):
        a, b = rnd.getrandbits(W), rnd.getrandbits(W)
        sq = lambda u: oracle.big_ring_mul(P, u, u)
        assert sq(a ^ b) == sq(a) ^ sq(b)
        t = a
        for _ in range(16):
            t = sq(t)
        assert t == a
        t = a
        for _ in range(8):
            t = sq(t)
        assert t != a or a in (0, 1)


def test_closed_form_inverse_every_z(oracle):
    # Section 4.6, and the unit property of 1 + x^z (Lemma 3.2.3)
    for z in range(1, P):
        u = 1 ^ oracle.big_ring_xpow(P, z)
        inv = oracle.big_ring_inv(P, u)
        assert inv == closed_inverse(z), z
        assert oracle.big_ring_mul(P, u, inv) == 1


def test_inverse_as_a_product_of_frobenius_images(oracle):
    # (1 + x^z)^(2^8) = 1 + x^(256 z) = 1 + x^(-z), so (1 + x^z)^(-1) =
    # x^z * prod_{k=1}^{7} (1 + x^(z 2^k)): seven binomials instead of 129 terms
    for z in range(1, P):
        acc = oracle.big_ring_xpow(P, z)
        for k in range(1, 8):
            acc = oracle.big_ring_mul(P, acc, 1 ^ oracle.big_ring_xpow(P, z * (1 << k) % P))
        assert acc == oracle.big_ring_inv(P, 1 ^ oracle.big_ring_xpow(P, z)), z


def test_random_units_invert(oracle):
    rnd = random.Random(3)
    for _ in range(20):
        a = rnd.getrandbits(W)
        inv = oracle.big_ring_inv(P, a)
        if inv:
            assert oracle.big_ring_mul(P, a, inv) == 1
        else:  # a shares a factor with f: then a^(2^16 - 1) is not 1
            t, e = a, 1
            for _ in range(15):
                t = oracle.big_ring_mul(P, t, t)
                e = oracle.big_ring_mul(P, e, t)
            assert oracle.big_ring_mul(P, a, e) != 1


# ---------------------------------------------------------- Z_257 encode

@pytest.mark.parametrize("N,B", [(1, 32), (2, 64), (5, 96), (16, 64), (257, 32)])
def test_z257_encode(oracle, N, B):
    h = h_random(700 + N, N, B, 1)
    oracle.hbig_encode(P, N, B, h, 1)
    d = [elements(h[0, k]) for k in range(N)]
    P_el, Q_el = elements(h[0, N]), elements(h[0, N + 1])
    for e in range(B // 32):
        p_want = 0
        q_want = 0
        for k in range(N):
            p_want ^= d[k][e]
            q_want ^= xk_word(d[k][e], k)  # Q = sum g^k d_k, word formula
        assert P_el[e] == p_want
        assert Q_el[e] == q_want
    if N == 1:
        assert np.array_equal(h[0, 1], h[0, 0]) and np.array_equal(h[0, 2], h[0, 0])


@pytest.mark.parametrize("N", [3, 257])
def test_z257_q_is_evenodd_diagonal_parity(oracle, N):
    # EVENODD with the imaginary row p-1 = 0 and strips t >= N zero: a_{r,t}
    # is coefficient r of data strip t; S = sum_{t=1}^{p-1} a_{p-1-t, t};
    # Q_r = S + sum_t a_{<r-t>, t}
    h = h_random(800 + N, N, 32, 1)
    oracle.hbig_encode(P, N, 32, h, 1)
    d = [elements(h[0, k])[0] for k in range(N)]
    coef = lambda r, t: (d[t] >> r) & 1 if (t < N and r < P - 1) else 0
    S = 0
    for t in range(1, P):
        S ^= coef(P - 1 - t, t)
    q = 0
    for r in range(P - 1):
        bit = S
        for t in range(N):
            bit ^= coef((r - t) % P, t)
        q |= bit << r
    assert elements(h[0, N + 1])[0] == q


# -------------------------------------------------------- Z_257 recovery

def test_z257_every_pair_round_trips(oracle):
    N, B = 6, 64
    h = h_random(900, N, B, 1)
    oracle.hbig_encode(P, N, B, h, 1)
    for (i, j) in all_pairs(N):
        lost = h.copy()
        lost[0, i] = POISON
        lost[0, j] = POISON ^ 0xFF
        oracle.hbig_recover(P, N, B, lost, 1, i, j)
        assert np.array_equal(lost, h), (i, j)


def test_z257_wide_array_sampled_pairs(oracle):
    N, B = 257, 32
    h = h_random(901, N, B, 2)
    oracle.hbig_encode(P, N, B, h, 2)
    rnd = random.Random(901)
    pairs = np.array([[256, 258], sorted(rnd.sample(range(N + 2), 2))], dtype=np.uint16)
    for extra in [(0, 256), (255, 256), (256, 257), (257, 258), (3, 258)]:
        lost = h.copy()
        lost[:, extra[0]] = POISON
        lost[:, extra[1]] = POISON
        oracle.hbig_recover(P, N, B, lost, 2, *extra)
        assert np.array_equal(lost, h), extra
    lost = h.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON
        lost[s, j] = POISON
    oracle.hbig_recover(P, N, B, lost, 2, pairs=pairs)
    assert np.array_equal(lost, h)


def test_z257_two_data_by_the_section_4_6_horner_forms(oracle):
    # D_y = A dP + g^(-x) A dQ with A = (1 + g^z)^(-1) = sum_t g^(2tz): the
    # Horner forms (delP), (delQ) -- A v = v + g^(2z)(v + g^(2z)(... v)) with
    # (p+1)/2 terms -- on words; D_x = D_y + dP
    N, B = 9, 64
    h = h_random(950, N, B, 1)
    oracle.hbig_encode(P, N, B, h, 1)
    d = [elements(h[0, k]) for k in range(N + 2)]
    for (x, y) in [(0, 1), (2, 7), (0, 8), (3, 4)]:
        z = y - x
        lost = h.copy()
        lost[0, x] = POISON
        lost[0, y] = POISON
        oracle.hbig_recover(P, N, B, lost, 1, x, y)
        got = [elements(lost[0, k]) for k in (x, y)]
        for e in range(B // 32):
            dP, dQ = d[N][e], d[N + 1][e]
            for k in range(N):
                if k not in (x, y):
                    dP ^= d[k][e]
                    dQ ^= xk_word(d[k][e], k)

            def horner(v):
                acc = v
                for _ in range((P + 1) // 2 - 1):
                    acc = v ^ xk_word(acc, 2 * z)
                return acc

            Dy = horner(dP) ^ xk_word(horner(dQ), P - x)
            Dx = Dy ^ dP
            assert (got[0][e], got[1][e]) == (Dx, Dy), (x, y, e)
            assert (Dx, Dy) == (d[x][e], d[y][e])


def test_z257_rejects_out_of_range(oracle):
    h = h_random(1, 3, 32, 1)
    with pytest.raises(ValueError):
        oracle.hbig_encode(P, 258, 32, np.zeros((1, 260, 32), np.uint8), 1)  # N > p: base code only
    with pytest.raises(ValueError):
        oracle.hbig_encode(P, 3, 48, np.zeros((1, 5, 48), np.uint8), 1)  # not whole elements
    with pytest.raises(ValueError):
        oracle.hbig_encode(259, 3, 32, h, 1)  # p out of range
    with pytest.raises(ValueError):
        oracle.hbig_recover(P, 3, 32, h, 1, 2, 2)
