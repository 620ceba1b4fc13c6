"""Pins for the oracle's extended code (equation qext of Section 3.3) and its
prime checks (Lemma 3.3.1, Theorem 3.3.3).

The independent models are the paper's printed prime lists
(tests/golden/cone_primes.txt), GF(2) linear algebra on the Sylvester matrix
S_p (Theorem 3.3.3 condition (1) read as matrices: every pairwise sum of cone
elements non-singular), the qext parity equations written with S_p, and brute
force over all candidates for every erasure pair.
"""
import os

import numpy as np
import pytest

from paper_cs_0611109_gb300 import inputs

from test_oracle_pins import (all_pairs, bits_of, gf2_rank, mm, mpow, random_stripes, sylvester,
                              vec)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_lists():
    out = {}
    for line in open(os.path.join(GOLDEN, "cone_primes.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split(":", 1)
            out[k.strip()] = [int(x) for x in v.split()]
    return out


def primes(lo, hi):
    return [n for n in range(lo, hi) if n > 1 and all(n % d for d in range(2, int(n ** 0.5) + 1))]


def weight_matrix(p, k):
    """S_p^k for k < p, Id + S_p^(k-p+1) for p <= k <= 2p-2 (equation qext)."""
    S = sylvester(p)
    if k < p:
        return mpow(S, k)
    return (np.eye(p - 1, dtype=np.int64) + mpow(S, k - p + 1)) % 2


# ------------------------------------------------------------- prime checks

def test_primitive_two_list(oracle):
    want = golden_lists()["primitive_two"]
    assert [p for p in primes(3, 100) if oracle.ord2(p) == p - 1] == want


def test_order_of_two(oracle):
    g = golden_lists()
    assert oracle.ord2(g["first_non_mersenne_failure"][0]) == g["order_of_two_mod_73"][0]
    # ord divides p - 1 and 2^ord = 1 (mod p), by direct powering
    for p in primes(3, 128):
        d = oracle.ord2(p)
        assert (p - 1) % d == 0 and pow(2, d, p) == 1
        assert all(pow(2, e, p) != 1 for e in range(1, d))


def test_failing_primes_below_128(oracle):
    g = golden_lists()
    failing = [p for p in primes(3, 128) if not oracle.cone_extends(p)]
    assert failing == sorted(g["mersenne"] + g["first_non_mersenne_failure"])
    assert all(oracle.cone_extends(p) for p in g["fermat"])


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13, 17, 19, 31])
def test_cone_condition_1_with_sylvester_matrix(oracle, p):
    # Theorem 3.3.3 (1) for g = S_p: the 2p-1 matrices Id, g, ..., g^(p-1),
    # Id + g, ..., Id + g^(p-1) form a cone (every pairwise sum non-singular).
    n = p - 1
    cone = [weight_matrix(p, k) for k in range(2 * p - 1)]
    ok = all(gf2_rank((cone[a] + cone[b]) % 2) == n
             for a in range(len(cone)) for b in range(a + 1, len(cone)))
    assert all(gf2_rank(M) == n for M in cone)
    assert ok == oracle.cone_extends(p)


def test_weights_are_the_matrix_weights(oracle):
    for p in (5, 7, 13):
        for k in range(2 * p - 1):
            M = weight_matrix(p, k)
            w = oracle.weight(p, k)
            assert np.array_equal(M[:, 0], vec(w, p - 1)), (p, k)  # image of the unit 1


# ------------------------------------------------------------ extended code

@pytest.mark.parametrize("p,N", [(5, 6), (5, 9), (13, 25), (11, 21), (17, 33), (29, 40), (59, 117)])
def test_qext_encode_matches_matrix_model(oracle, p, N):
    C = 16
    buf = random_stripes(71, p, N, C, 2)
    oracle.encode(p, N, C, buf, 2)
    b = bits_of(buf)
    W = [weight_matrix(p, k) for k in range(N)]
    for s in range(2):
        P = np.bitwise_xor.reduce(b[s, :N], axis=0)
        Q = np.zeros_like(P)
        for k in range(N):
            Q ^= mm(W[k], b[s, k])
        assert np.array_equal(b[s, N], P)
        assert np.array_equal(b[s, N + 1], Q)


def test_qext_reduces_to_base_code(oracle):
    # the first p strips of an extended stripe have the base code's weights:
    # zero strips k >= p change nothing
    p, C = 13, 32
    base = random_stripes(73, p, p, C, 1)
    oracle.encode(p, p, C, base, 1)
    ext = np.zeros((1, 2 * p - 1 + 2, p - 1, C), dtype=np.uint8)
    ext[0, :p] = base[0, :p]
    oracle.encode(p, 2 * p - 1, C, ext, 1)
    assert np.array_equal(ext[0, 2 * p - 1:], base[0, p:])


def solutions(p, N, b, i, j):
    """Brute force: the number of candidates for the unknown strip(s) of the
    pair (i, j) consistent with both parity equations, per codeword, and the
    candidate found; b are the coefficient planes [N+2, p-1, 8C]."""
    n = p - 1
    W = [weight_matrix(p, k) for k in range(N)]
    cand = np.array([vec(c, n) for c in range(1 << n)], dtype=np.int64)
    wts = (1 << np.arange(n)).astype(np.int64)
    rows = lambda M: (M * wts[None, :]).sum(axis=1)
    cols = lambda M: (M * wts[:, None]).sum(axis=0)
    if j < N:
        dP, dQ = b[N].copy(), b[N + 1].copy()
        for k in range(N):
            if k not in (i, j):
                dP ^= b[k]
                dQ ^= mm(W[k], b[k])
        images = rows(mm(cand, ((W[i] + W[j]) % 2).T))
        rhs = cols((dQ + mm(W[i], dP)) % 2)
        truth = cols(b[j])
    elif j == N:
        dQ = b[N + 1].copy()
        for k in range(N):
            if k != i:
                dQ ^= mm(W[k], b[k])
        images, rhs, truth = rows(mm(cand, W[i].T)), cols(dQ), cols(b[i])
    else:
        dP = b[N].copy()
        for k in range(N):
            if k != i:
                dP ^= b[k]
        images, rhs, truth = rows(cand), cols(dP), cols(b[i])
    counts = (images[:, None] == rhs[None, :]).sum(axis=0)
    return counts, images, rhs, truth


@pytest.mark.parametrize("p,N,n_pairs", [(5, 9, None), (13, 25, 80)])
def test_qext_bruteforce_pairs(oracle, p, N, n_pairs):
    # Lemma 3.1.2 for the extended cone: every erasure pair has exactly one
    # solution, the original, and the oracle returns it.
    C = 4
    buf = random_stripes(79, p, N, C, 1)
    oracle.encode(p, N, C, buf, 1)
    b = bits_of(buf)[0]
    pairs = [pq for pq in all_pairs(N) if pq != (N, N + 1)]
    if n_pairs:
        rng = np.random.default_rng(p)
        pick = rng.choice(len(pairs), n_pairs, replace=False)
        # keep every mixed pair class: base+extended, extended+extended, with P, with Q
        must = [(0, p), (p - 1, 2 * p - 2), (p, 2 * p - 2), (1, N), (p + 2, N), (p + 3, N + 1), (2 * p - 2, N + 1)]
        pairs = sorted(set([pairs[t] for t in pick] + must))
    for (i, j) in pairs:
        counts, images, rhs, truth = solutions(p, N, b, i, j)
        assert np.all(counts == 1), (i, j)
        sol = np.array([int(np.nonzero(images == r)[0][0]) for r in rhs])
        assert np.array_equal(sol, truth), (i, j)
        lost = buf.copy()
        lost[0, i] = 0xA5
        lost[0, j] = 0x5A
        oracle.recover(p, N, C, lost, 1, i, j)
        assert np.array_equal(lost, buf), (i, j)


def test_failing_prime_has_an_unsolvable_pair(oracle):
    # p = 7 (Mersenne) fails Theorem 3.3.3: 1 + x + x^3 divides x^7 - 1, so
    # the extended pair (data 1, data p-1+3) -- weights x and 1 + x^3 -- has
    # several solutions, and the oracle refuses N > p for this prime.
    p, N, C = 7, 13, 4
    buf = random_stripes(83, p, p, C, 1)
    ext = np.zeros((1, N + 2, p - 1, C), dtype=np.uint8)
    ext[0, :p] = buf[0, :p]
    with pytest.raises(ValueError):
        oracle.encode(p, N, C, ext, 1)
    # build the extended parities from the matrix model and count solutions
    b = np.zeros((N + 2, p - 1, 8 * C), dtype=np.int64)
    rnd = bits_of(random_stripes(89, p, N, C, 1))[0]
    b[:N] = rnd[:N]
    b[N] = np.bitwise_xor.reduce(b[:N], axis=0)
    for k in range(N):
        b[N + 1] ^= mm(weight_matrix(p, k), b[k])
    counts, _, _, _ = solutions(p, N, b, 1, p - 1 + 3)
    # the kernel of x + 1 + x^3 on R is the component F2[x]/(1 + x + x^3) of
    # Lemma 3.3.1, of dimension ord_7(2) = 3: 2^3 candidates per codeword
    assert np.all(counts == 2 ** oracle.ord2(p))
    counts, _, _, _ = solutions(p, N, b, 0, p)  # x^0 + (1 + x) = x: fine
    assert np.all(counts == 1)


@pytest.mark.parametrize("p,N,C,S", [(5, 9, 32, 3), (13, 25, 16, 2), (29, 57, 16, 1), (59, 117, 16, 1), (17, 33, 16, 1), (11, 20, 16, 2)])
def test_qext_roundtrip(oracle, p, N, C, S):
    buf = random_stripes(97, p, N, C, S)
    oracle.encode(p, N, C, buf, S)
    pairs = all_pairs(N)
    rng = np.random.default_rng(p + N)
    pairs = [pairs[t] for t in rng.choice(len(pairs), min(40, len(pairs)), replace=False)]
    for (i, j) in pairs:
        lost = buf.copy()
        lost[:, i] = 0xA5
        lost[:, j] = 0x3C
        oracle.recover(p, N, C, lost, S, i, j)
        assert np.array_equal(lost, buf), (i, j)


def test_qext_update_and_degraded_read(oracle):
    p, N, C, S = 13, 22, 32, 2
    buf = random_stripes(101, p, N, C, S)
    oracle.encode(p, N, C, buf, S)
    before = buf.copy()
    for i in (3, p + 4):
        new = inputs.random_bytes(103 + i, (p - 1) * C).reshape(p - 1, C)
        old = buf[1, i].copy()
        oracle.update(p, N, C, buf, 1, i, new)
        # Q changes by the weight of strip i times (old + new), by the matrix model
        delta = bits_of((old ^ new)[None])[0]
        want_q = bits_of(before[1, N + 1][None])[0] ^ mm(weight_matrix(p, i), delta)
        assert np.array_equal(bits_of(buf[1, N + 1][None])[0], want_q)
        before = buf.copy()
    for j in list(range(0, N + 2, 3)) + [N, N + 1]:
        lost = buf.copy()
        lost[0, j] = 0xA5
        assert np.array_equal(oracle.degraded_read(p, N, C, lost, 0, j), buf[0, j]), j


def test_qext_invalid_arguments(oracle):
    buf = np.zeros((1, 40, 12, 16), dtype=np.uint8)
    for p, N in ((13, 26), (7, 8), (3, 4), (31, 32)):
        with pytest.raises(ValueError):
            oracle.encode(p, N, 16, buf, 1)
