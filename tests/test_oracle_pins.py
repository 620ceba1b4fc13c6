"""Pins for the CPU oracle: every oracle function checked against something other
than itself -- values the paper prints (tests/golden/), the paper's own matrix
description of the generator, closed forms, invariants, the EVENODD definition
and brute force over all candidates.

The independent model used here is plain GF(2) linear algebra on the Sylvester
matrix S_p exactly as Lemma 3.4.1 draws it (ones on the sub-diagonal, last
column all ones); it shares nothing with the oracle's polynomial arithmetic.
"""
import itertools
import os
import re

import numpy as np
import pytest

from paper_cs_0611109_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PRIMES = [3, 5, 7, 11, 13, 17, 29, 59, 61]


# ----------------------------------------------------------- GF(2) model

def sylvester(p):
    """S_p of Lemma 3.4.1: (p-1)x(p-1), ones below the diagonal, last column ones."""
    n = p - 1
    S = np.zeros((n, n), dtype=np.int64)
    for r in range(1, n):
        S[r, r - 1] = 1
    S[:, n - 1] = 1
    return S


def mm(A, B):
    return (A @ B) % 2


def mpow(S, k):
    R = np.eye(S.shape[0], dtype=np.int64)
    for _ in range(k):
        R = mm(R, S)
    return R


def vec(a, n):
    return np.array([(a >> r) & 1 for r in range(n)], dtype=np.int64)


def unvec(v):
    return int(sum(int(b) << r for r, b in enumerate(v)))


def gf2_rank(M):
    M = M.copy() % 2
    rank = 0
    rows, cols = M.shape
    for c in range(cols):
        piv = [r for r in range(rank, rows) if M[r, c]]
        if not piv:
            continue
        M[[rank, piv[0]]] = M[[piv[0], rank]]
        for r in range(rows):
            if r != rank and M[r, c]:
                M[r] ^= M[rank]
        rank += 1
    return rank


def bits_of(stripes):
    """uint8 (..., rows, C) -> int64 (..., rows, 8C): coefficient planes, one column per codeword."""
    return np.unpackbits(stripes, axis=-1, bitorder="little").astype(np.int64)


def model_encode_bits(p, N, dbits):
    """P and Q coefficient planes from data planes dbits [N, p-1, 8C] by the parity
    equations (znparity) with g = S_p, g_k = g^k."""
    S = sylvester(p)
    P = np.zeros_like(dbits[0])
    Q = np.zeros_like(dbits[0])
    G = np.eye(p - 1, dtype=np.int64)
    for k in range(N):
        P ^= dbits[k]
        Q ^= mm(G, dbits[k])
        G = mm(G, S)
    return P, Q


def read_matrix(name):
    rows = [l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]
    return np.array([[int(x) for x in r] for r in rows], dtype=np.int64)


def random_stripes(seed, p, N, C, S):
    return np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, S))


# ------------------------------------------------------------- generator

def test_sylvester_matches_printed_matrices():
    # Section 4.5 prints S_17 in full; Section 2.1 (hg) prints G = S_3.
    assert np.array_equal(sylvester(17), read_matrix("sylvester_s17.txt"))
    assert np.array_equal(sylvester(3), read_matrix("matrix_g_p3.txt"))


@pytest.mark.parametrize("p", PRIMES)
def test_mul_by_x_is_the_sylvester_matrix(oracle, p):
    # Lemma 3.4.1(ii): S_p is the companion matrix of 1+...+x^(p-1), i.e. the
    # matrix of multiplication by x.  Column c of S_p = x * x^c.
    S = sylvester(p)
    for c in range(p - 1):
        assert np.array_equal(vec(oracle.ring_mul(p, 2, 1 << c), p - 1), S[:, c])
        assert oracle.ring_mul(p, 1 << c, 2) == oracle.ring_mul(p, 2, 1 << c)


@pytest.mark.parametrize("p", PRIMES)
def test_ring_mul_is_matrix_polynomial(oracle, p):
    # b(S_p) a == a*b: the ring product agrees with evaluating b at the matrix.
    rng = np.random.default_rng(p)
    S = sylvester(p)
    powers = [mpow(S, t) for t in range(p - 1)]
    for _ in range(12):
        a = int(rng.integers(0, 1 << (p - 1)))
        b = int(rng.integers(0, 1 << (p - 1)))
        M = np.zeros((p - 1, p - 1), dtype=np.int64)
        for t in range(p - 1):
            if (b >> t) & 1:
                M ^= powers[t]
        assert unvec(mm(M, vec(a, p - 1))) == oracle.ring_mul(p, a, b)


@pytest.mark.parametrize("p", PRIMES)
def test_order_is_p(oracle, p):
    # Lemma 3.4.1(i): S_p has order p; x^p = 1 and x^k != 1 for 0 < k < p.
    assert oracle.ring_xpow(p, p) == 1
    assert oracle.ring_xpow(p, 0) == 1
    for k in range(1, p):
        assert oracle.ring_xpow(p, k) != 1
    assert np.array_equal(mpow(sylvester(p), p), np.eye(p - 1, dtype=np.int64))
    # x^k for k < p-1 is the monomial; x^(p-1) is all ones (= 1+x+...+x^(p-2)).
    for k in range(p - 1):
        assert oracle.ring_xpow(p, k) == 1 << k
    assert oracle.ring_xpow(p, p - 1) == (1 << (p - 1)) - 1


@pytest.mark.parametrize("p", PRIMES)
def test_roots_of_unity_sum_to_zero(oracle, p):
    # Lemma 3.2.2: sum_{k<p} g^k = 0.
    acc = 0
    for k in range(p):
        acc ^= oracle.ring_xpow(p, k)
    assert acc == 0


@pytest.mark.parametrize("n", range(3, 22))
def test_id_plus_sylvester_invertible_iff_odd(n):
    # Lemma 3.4.1(ii) for the (n-1)x(n-1) companion matrix of 1+...+x^(n-1).
    M = (sylvester(n) + np.eye(n - 1, dtype=np.int64)) % 2
    assert (gf2_rank(M) == n - 1) == (n % 2 == 1)


def powers_closed_form(N, k, a):
    """Equation (powers) of Lemma 3.4.1, written with the paper's labels: the
    vector (x_{N-1}, ..., x_1) top to bottom, i.e. x_j is coefficient N-1-j, and
    output position t is x_k + x_{(k-1-t) mod N} with x_j = 0 unless 1 <= j <= N-1."""
    def lab(j):
        return (a >> (N - 1 - j)) & 1 if 1 <= j <= N - 1 else 0
    out = 0
    for t in range(N - 1):
        out |= (lab(k) ^ lab((k - 1 - t) % N)) << t
    return out


@pytest.mark.parametrize("p", [3, 5, 7, 13, 17, 29, 59])
def test_powers_closed_form(oracle, p):
    rng = np.random.default_rng(1000 + p)
    a = rng.integers(0, 1 << (p - 1), size=40, dtype=np.uint64)
    for k in range(1, p + 1):
        got = oracle.mul_xpow_array(p, k, a)
        want = [powers_closed_form(p, k, int(v)) for v in a]
        assert [int(v) for v in got] == want


def test_z17_word_formulas(oracle):
    # Sections 4.5 and 4.6 store one Z_17 element per 16-bit lane (bit r =
    # coefficient of x^r).  x^k is: shift left by k, shift right (logically) by
    # 17-k, and flip all 16 bits when bit 16-k was set (it lands on the
    # imaginary 17th coefficient).  For k=1 this is the doubling-with-sign-mask
    # form of Section 4.5.
    x = np.arange(1 << 16, dtype=np.uint64)
    for k in range(1, 17):
        y = ((x << np.uint64(k)) & np.uint64(0xFFFF)) ^ (x >> np.uint64(17 - k))
        y ^= np.where((x >> np.uint64(16 - k)) & np.uint64(1), np.uint64(0xFFFF), np.uint64(0))
        assert np.array_equal(oracle.mul_xpow_array(17, k, x), y), k
    double = ((x + x) & np.uint64(0xFFFF)) ^ np.where(x & np.uint64(0x8000), np.uint64(0xFFFF), np.uint64(0))
    assert np.array_equal(oracle.mul_xpow_array(17, 1, x), double)


@pytest.mark.parametrize("p", PRIMES)
def test_inverse_closed_form(oracle, p):
    # Section 4.6: (1+g^z)^{-1} = sum_{j=0}^{(p-1)/2} g^{2jz} and g^{-k} = g^{p-k};
    # checked against the oracle's extended-Euclid inverse.
    for z in range(1, p):
        closed = 0
        for j in range((p - 1) // 2 + 1):
            closed ^= oracle.ring_xpow(p, (2 * j * z) % p)
        one_plus = 1 ^ oracle.ring_xpow(p, z)
        assert oracle.ring_inv(p, one_plus) == closed
        assert oracle.ring_mul(p, one_plus, closed) == 1
    for k in range(1, p):
        assert oracle.ring_inv(p, oracle.ring_xpow(p, k)) == oracle.ring_xpow(p, p - k)
    assert oracle.ring_inv(p, 0) == 0


def test_gf4_ring_for_p3(oracle):
    # Section 2.2: {0, 1, G, G^2} is closed under + and x and is the field GF(4).
    G = read_matrix("matrix_g_p3.txt")
    assert np.array_equal(mm(G, G), (G + np.eye(2, dtype=np.int64)) % 2)  # G^2 = Id + G
    assert oracle.ring_xpow(3, 2) == 0b11
    for a in range(1, 4):
        inv = oracle.ring_inv(3, a)
        assert inv in (1, 2, 3) and oracle.ring_mul(3, a, inv) == 1
        for b in range(4):
            assert oracle.ring_mul(3, a, b) in range(4)


# ---------------------------------------------------------------- encode

def parse_equations(name):
    eqs = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = [s.strip() for s in line.split("=")]
        eqs.append((lhs, [t.strip() for t in rhs.split("+")]))
    return eqs


def test_hordiag_worked_example(oracle):
    # Section 2.1: the four-disk code (p = 3, N = 2) over all 16 data dibit pairs.
    # Codeword b (bit position b of the rows) carries d11,d12,d21,d22 = bits 0..3 of b.
    p, N, C = 3, 2, 2
    buf = np.zeros((1, N + 2, p - 1, C), dtype=np.uint8)
    val = {}
    for name, k, r, bit in (("d11", 0, 0, 0), ("d12", 0, 1, 1), ("d21", 1, 0, 2), ("d22", 1, 1, 3)):
        plane = np.array([(b >> bit) & 1 for b in range(16)], dtype=np.uint8)
        val[name] = plane
        buf[0, k, r] = np.packbits(plane, bitorder="little")
    oracle.encode(p, N, C, buf, 1)
    got = bits_of(buf)[0]
    eqs = parse_equations("hordiag_p3.txt")
    where = {"pi11": (2, 0), "pi12": (2, 1), "pi21": (3, 0), "pi22": (3, 1)}
    for lhs, terms in eqs[:4]:
        want = np.bitwise_xor.reduce([val[t] for t in terms])
        assert np.array_equal(got[where[lhs]], want), lhs
        val[lhs] = want
    # the printed recovery formulas give back the data from the parities
    for lhs, terms in eqs[4:]:
        assert np.array_equal(np.bitwise_xor.reduce([val[t] for t in terms]), val[lhs]), lhs
    # and the oracle rebuilds both data strips from P and Q
    lost = buf.copy()
    lost[0, 0:2] = 0xA5
    oracle.recover(p, N, C, lost, 1, 0, 1)
    assert np.array_equal(lost, buf)


@pytest.mark.parametrize("p,N,C", [(3, 3, 16), (5, 4, 32), (7, 5, 16), (13, 12, 16), (17, 17, 16), (29, 7, 16), (59, 58, 16), (61, 3, 16)])
def test_encode_matches_matrix_model(oracle, p, N, C):
    buf = random_stripes(7, p, N, C, 2)
    oracle.encode(p, N, C, buf, 2)
    b = bits_of(buf)
    for s in range(2):
        P, Q = model_encode_bits(p, N, b[s, :N])
        assert np.array_equal(b[s, N], P)
        assert np.array_equal(b[s, N + 1], Q)


def test_p52_five_disk_code(oracle):
    # Section 2.2, equations (gf4)/(p52): pi2 = d1 + G d2 + G^2 d3 with G from (hg).
    p, N, C = 3, 3, 16
    G = read_matrix("matrix_g_p3.txt")
    buf = random_stripes(11, p, N, C, 1)
    oracle.encode(p, N, C, buf, 1)
    b = bits_of(buf)[0]
    assert np.array_equal(b[N + 1], (b[0] + mm(G, b[1]) + mm(mm(G, G), b[2])) % 2)
    assert np.array_equal(b[N], (b[0] + b[1] + b[2]) % 2)


def evenodd_diagonal_parity(p, rows):
    """EVENODD diagonal parity (Blaum, Brady, Bruck, Menon 1995) of a data array
    rows[t][i] = row i of data column t, t < p, i < p-1 (uint8 [p, p-1, C]).
    The imaginary row p-1 is zero; S is the XOR of the diagonal that ends in
    it, and row i of the parity is S plus the XOR of a_{<i-t>, t} over t."""
    def a(i, t):
        return rows[t, i] if i < p - 1 else np.zeros_like(rows[0, 0])
    S = np.zeros_like(rows[0, 0])
    for t in range(1, p):
        S ^= a(p - 1 - t, t)
    out = np.empty_like(rows[0])
    for i in range(p - 1):
        acc = S.copy()
        for t in range(p):
            acc ^= a((i - t) % p, t)
        out[i] = acc
    return out


@pytest.mark.parametrize("p,N", [(3, 3), (5, 5), (5, 2), (7, 7), (13, 12), (17, 17), (17, 9), (29, 29), (59, 58)])
def test_q_equals_evenodd(oracle, p, N):
    # Section 3.4: the code with g = S_p is EVENODD; columns beyond N are zero.
    C = 16
    buf = random_stripes(13, p, N, C, 2)
    oracle.encode(p, N, C, buf, 2)
    for s in range(2):
        cols = np.zeros((p, p - 1, C), dtype=np.uint8)
        cols[:N] = buf[s, :N]
        assert np.array_equal(buf[s, N + 1], evenodd_diagonal_parity(p, cols))


@pytest.mark.parametrize("p,N", [(5, 4), (13, 12), (59, 58), (7, 1)])
def test_p_is_xor_of_data(oracle, p, N):
    C = 48
    buf = random_stripes(17, p, N, C, 3)
    oracle.encode(p, N, C, buf, 3)
    assert np.array_equal(buf[:, N], np.bitwise_xor.reduce(buf[:, :N], axis=1))


def test_special_cases(oracle):
    # N = 1: x^0 = 1, so P = Q = d_0.
    for p in (3, 5, 13, 59):
        buf = random_stripes(19, p, 1, 32, 2)
        oracle.encode(p, 1, 32, buf, 2)
        assert np.array_equal(buf[:, 1], buf[:, 0]) and np.array_equal(buf[:, 2], buf[:, 0])
    # all-zero data: zero parity.
    buf = np.full((2, 6, 4, 16), 0xFF, dtype=np.uint8)
    buf[:, :4] = 0
    oracle.encode(5, 4, 16, buf, 2)
    assert not buf.any()
    # one-hot: data strip k holding the monomial x^r gives Q = x^(r+k).
    p, N = 7, 5
    for k in range(N):
        for r in range(p - 1):
            buf = np.zeros((1, N + 2, p - 1, 16), dtype=np.uint8)
            buf[0, k, r] = 0xFF
            oracle.encode(p, N, 16, buf, 1)
            want = oracle.ring_xpow(p, r + k)
            q = [(want >> t) & 1 for t in range(p - 1)]
            assert [int(buf[0, N + 1, t, 0] == 0xFF) for t in range(p - 1)] == q
            assert all(buf[0, N + 1, t, 0] in (0, 0xFF) for t in range(p - 1))


def test_explicit_strides(oracle):
    # The same stripes in a padded, non-packed layout give the same bytes.
    p, N, C = 7, 4, 32
    packed = random_stripes(23, p, N, C, 3)
    oracle.encode(p, N, C, packed, 3)
    rs, ss, st = 48, 48 * (p - 1) + 16, (48 * (p - 1) + 16) * (N + 2) + 32
    padded = np.zeros(st * 3, dtype=np.uint8)
    for s in range(3):
        for k in range(N):
            for r in range(p - 1):
                o = s * st + k * ss + r * rs
                padded[o:o + C] = packed[s, k, r]
    oracle.encode(p, N, C, padded, 3, rs, ss, st)
    for s in range(3):
        for k in (N, N + 1):
            for r in range(p - 1):
                o = s * st + k * ss + r * rs
                assert np.array_equal(padded[o:o + C], packed[s, k, r])


# --------------------------------------------------------------- recovery

def all_pairs(N):
    return [(i, j) for i in range(N + 2) for j in range(i + 1, N + 2)]


@pytest.mark.parametrize("p,N", [(5, 4), (13, 12)])
def test_bruteforce_every_pair(oracle, p, N):
    # Lemma 3.1.2 by exhaustion: for every erasure pair, enumerate all 2^(p-1)
    # candidates for the unknown data strip, keep those that satisfy both
    # parity equations (znparity) written with the matrix S_p, and require
    # exactly one -- the original -- which the oracle must also return.
    C = 4
    n = p - 1
    buf = random_stripes(29, p, N, C, 1)
    oracle.encode(p, N, C, buf, 1)
    b = bits_of(buf)[0]  # [N+2, n, 8C]
    S = sylvester(p)
    g = [mpow(S, k) for k in range(N)]
    cand = np.array([vec(c, n) for c in range(1 << n)], dtype=np.int64)  # [2^n, n]
    weights = (1 << np.arange(n)).astype(np.int64)

    def rows(M):  # [count, n] candidate vectors -> ints
        return (M * weights[None, :]).sum(axis=1)

    def cols(M):  # [n, 8C] coefficient planes -> one int per codeword
        return (M * weights[:, None]).sum(axis=0)

    for (i, j) in all_pairs(N):
        if i < N and j < N:
            dP = b[N].copy()
            dQ = b[N + 1].copy()
            for k in range(N):
                if k not in (i, j):
                    dP ^= b[k]
                    dQ ^= mm(g[k], b[k])
            # d_i = dP + c, d_j = c must satisfy g_i d_i + g_j d_j = dQ
            images = rows(mm(cand, ((g[i] + g[j]) % 2).T))
            rhs = cols((dQ + mm(g[i], dP)) % 2)
            truth = cols(b[j])
        elif i < N and j == N:
            dQ = b[N + 1].copy()
            for k in range(N):
                if k != i:
                    dQ ^= mm(g[k], b[k])
            images = rows(mm(cand, g[i].T))
            rhs = cols(dQ)
            truth = cols(b[i])
        elif i < N and j == N + 1:
            dP = b[N].copy()
            for k in range(N):
                if k != i:
                    dP ^= b[k]
            images = rows(cand)
            rhs = cols(dP)
            truth = cols(b[i])
        else:
            images = None
        if images is not None:
            counts = (images[:, None] == rhs[None, :]).sum(axis=0)
            assert np.all(counts == 1), (i, j)
            sol = np.array([int(np.nonzero(images == r)[0][0]) for r in rhs])
            assert np.array_equal(sol, truth), (i, j)
        lost = buf.copy()
        lost[0, i] = 0xA5
        lost[0, j] = 0x5A
        oracle.recover(p, N, C, lost, 1, i, j)
        assert np.array_equal(lost, buf), (i, j)


@pytest.mark.parametrize("p,N,C,S", [(5, 4, 64, 6), (7, 5, 48, 3), (13, 12, 16, 2), (29, 20, 16, 1), (59, 58, 16, 1), (3, 2, 16, 4), (17, 17, 16, 1)])
def test_roundtrip_all_pairs(oracle, p, N, C, S):
    # encode -> poison two strips -> recover gives back the original stripe
    buf = random_stripes(31, p, N, C, S)
    oracle.encode(p, N, C, buf, S)
    pairs = all_pairs(N)
    if len(pairs) > 60:
        rng = np.random.default_rng(p)
        pairs = [pairs[t] for t in rng.choice(len(pairs), 60, replace=False)]
    for (i, j) in pairs:
        lost = buf.copy()
        lost[:, i] = 0xA5
        lost[:, j] = 0x3C
        oracle.recover(p, N, C, lost, S, i, j)
        assert np.array_equal(lost, buf), (i, j)


def test_per_stripe_pairs(oracle):
    p, N, C, S = 13, 12, 32, 8
    buf = random_stripes(37, p, N, C, S)
    oracle.encode(p, N, C, buf, S)
    pairs = inputs.random_pairs(5, N, S, "any")
    lost = buf.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = 0xA5
        lost[s, j] = 0xA5
    oracle.recover(p, N, C, lost, S, pairs=pairs)
    assert np.array_equal(lost, buf)


def test_update_and_degraded_read(oracle):
    p, N, C, S = 13, 6, 48, 3
    buf = random_stripes(41, p, N, C, S)
    oracle.encode(p, N, C, buf, S)
    new = inputs.random_bytes(43, (p - 1) * C).reshape(p - 1, C)
    before = buf.copy()
    oracle.update(p, N, C, buf, 1, 2, new)
    assert np.array_equal(buf[1, 2], new)
    # P changes by old + new (first equation of znparity is linear)
    assert np.array_equal(buf[1, N], before[1, N] ^ before[1, 2] ^ new)
    # Q is again the EVENODD diagonal parity of the new data
    cols = np.zeros((p, p - 1, C), dtype=np.uint8)
    cols[:N] = buf[1, :N]
    assert np.array_equal(buf[1, N + 1], evenodd_diagonal_parity(p, cols))
    assert np.array_equal(np.delete(buf, 1, axis=0), np.delete(before, 1, axis=0))
    for j in range(N + 2):
        lost = buf.copy()
        lost[2, j] = 0xA5
        assert np.array_equal(oracle.degraded_read(p, N, C, lost, 2, j), buf[2, j]), j


def test_invalid_arguments_rejected(oracle):
    buf = np.zeros((1, 6, 4, 16), dtype=np.uint8)
    for p, N in ((9, 4), (2, 1), (63, 4), (5, 0), (5, 10), (7, 8), (15, 4)):
        with pytest.raises(ValueError):
            oracle.encode(p, N, 16, buf, 1)
    with pytest.raises(ValueError):
        oracle.recover(5, 4, 16, buf, 1, 2, 2)
    with pytest.raises(ValueError):
        oracle.recover(5, 4, 16, buf, 1, 3, 6)
