"""Pins for O2 (oracle/rcg_o2.c), the word-level multi-threaded CPU
implementation used to check full-size GPU results byte for byte: it must
equal the bit-level oracle (itself pinned to the paper) on every operation,
erasure class, extended layout and stride, and its Gaussian-elimination
inverse must equal the oracle's extended-Euclid inverse."""
import numpy as np
import pytest

from paper_cs_0611109_gb300 import inputs

POISON_I, POISON_J = 0xA5, 0x5A


@pytest.fixture(scope="module")
def o2(oracle):
    oracle.build_o2()
    return oracle


def stripes(seed, p, N, C, S):
    return np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, S))


CASES = [(3, 1, 8, 3), (3, 3, 16, 2), (5, 4, 1024, 4), (5, 9, 40, 3), (7, 7, 64, 2), (13, 12, 4096, 2),
         (13, 25, 24, 2), (17, 33, 16, 1), (29, 57, 8, 1), (59, 58, 64, 2), (59, 117, 8, 1), (61, 121, 8, 1),
         (61, 61, 16, 1)]


@pytest.mark.parametrize("p,N,C,S", CASES)
def test_o2_encode_equals_oracle(o2, p, N, C, S):
    h = stripes(6000 + p + N, p, N, C, S)
    a, b = h.copy(), h.copy()
    o2.encode(p, N, C, a, S)
    o2.o2_encode(p, N, C, b, S, threads=3)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("p,N,C,S", CASES)
@pytest.mark.parametrize("kind", ["dd", "dp", "dq", "pq", "any"])
def test_o2_recover_equals_oracle(o2, p, N, C, S, kind):
    if kind == "dd" and N < 2:
        pytest.skip("two-data erasures need N >= 2")
    h = stripes(6100 + p + N, p, N, C, S)
    o2.encode(p, N, C, h, S)
    pairs = inputs.random_pairs(6101 + N, N, S, kind)
    lost = h.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    a, b = lost.copy(), lost.copy()
    o2.recover(p, N, C, a, S, pairs=pairs)
    o2.o2_recover(p, N, C, b, S, pairs=pairs, threads=2)
    assert np.array_equal(a, b)
    assert np.array_equal(b, h)


@pytest.mark.parametrize("p,N", [(5, 4), (5, 9), (13, 14)])
def test_o2_every_pair(o2, p, N):
    C, S = 16, 2
    h = stripes(6200 + p + N, p, N, C, S)
    o2.encode(p, N, C, h, S)
    for i in range(N + 2):
        for j in range(i + 1, N + 2):
            lost = h.copy()
            lost[:, i] = POISON_I
            lost[:, j] = POISON_J
            o2.o2_recover(p, N, C, lost, S, i, j)
            assert np.array_equal(lost, h), (i, j)


def test_o2_strides(o2):
    p, N, C, S = 13, 5, 48, 3
    rs, ss = 64, 64 * (p - 1) + 32
    st = ss * (N + 2) + 16
    flat = inputs.random_bytes(6300, st * S)
    a, b = flat.copy(), flat.copy()
    o2.encode(p, N, C, a, S, rs, ss, st)
    o2.o2_encode(p, N, C, b, S, rs, ss, st, threads=2)
    assert np.array_equal(a, b)  # padding between rows, strips and stripes untouched too


@pytest.mark.parametrize("p", [3, 5, 7, 13, 17, 29, 31, 59, 61])
def test_o2_inverse_equals_euclid(o2, p):
    rng = np.random.default_rng(p)
    for a in [int(rng.integers(1, 1 << (p - 1))) for _ in range(60)] + [1, 2, (1 << (p - 1)) - 1]:
        assert o2.o2_inverse(p, a) == o2.ring_inv(p, a), (p, a)


def test_o2_invalid_arguments(o2):
    h = np.zeros((1, 10, 4, 16), dtype=np.uint8)
    with pytest.raises(ValueError):
        o2.o2_encode(5, 4, 12, h, 1)      # C not a multiple of 8
    with pytest.raises(ValueError):
        o2.o2_encode(9, 4, 16, h, 1)      # not a prime
    with pytest.raises(ValueError):
        o2.o2_encode(7, 8, 16, np.zeros((1, 10, 6, 16), dtype=np.uint8), 1)  # 7 fails Theorem 3.3.3


# ------------------------------------------------ horizontal representation

H_CASES = [(3, 1, 16, 3), (3, 3, 48, 2), (5, 4, 64, 3), (5, 9, 32, 2), (17, 16, 256, 2), (17, 33, 64, 1),
           (17, 5, 16 * 9, 2)]


def h_stripes(seed, N, B, S):
    return np.ascontiguousarray(inputs.random_bytes(seed, S * (N + 2) * B).reshape(S, N + 2, B))


@pytest.mark.parametrize("p,N,B,S", H_CASES)
def test_o2_h_encode_equals_oracle(o2, p, N, B, S):
    h = h_stripes(6400 + p + N, N, B, S)
    a, b = h.copy(), h.copy()
    o2.h_encode(p, N, B, a, S)
    o2.o2_h_encode(p, N, B, b, S, threads=2)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("p,N,B,S", H_CASES)
@pytest.mark.parametrize("kind", ["dd", "dp", "dq", "pq", "any"])
def test_o2_h_recover_equals_oracle(o2, p, N, B, S, kind):
    if kind == "dd" and N < 2:
        pytest.skip("two-data erasures need N >= 2")
    h = h_stripes(6500 + p + N, N, B, S)
    o2.h_encode(p, N, B, h, S)
    pairs = inputs.random_pairs(6501 + N, N, S, kind)
    lost = h.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    a, b = lost.copy(), lost.copy()
    o2.h_recover(p, N, B, a, S, pairs=pairs)
    o2.o2_h_recover(p, N, B, b, S, pairs=pairs, threads=3)
    assert np.array_equal(a, b)
    assert np.array_equal(b, h)


def test_o2_h_every_pair_and_strides(o2):
    p, N, B, S = 17, 6, 48, 3
    ss, st = B + 16, (N + 2) * (B + 16) + 32
    flat = inputs.random_bytes(6600, st * S)
    a, b = flat.copy(), flat.copy()
    o2.h_encode(p, N, B, a, S, ss, st)
    o2.o2_h_encode(p, N, B, b, S, ss, st, threads=2)
    assert np.array_equal(a, b)  # padding between strips and stripes untouched too
    for i in range(N + 2):
        for j in range(i + 1, N + 2):
            lost = b.copy()
            for s in range(S):
                lost[s * st + i * ss: s * st + i * ss + B] = POISON_I
                lost[s * st + j * ss: s * st + j * ss + B] = POISON_J
            o2.o2_h_recover(p, N, B, lost, S, i, j, strip_stride=ss, stripe_stride=st)
            assert np.array_equal(lost, b), (i, j)


def test_o2_h_invalid_arguments(o2):
    h = np.zeros((1, 6, 64), dtype=np.uint8)
    with pytest.raises(ValueError):
        o2.o2_h_encode(9, 4, 64, h, 1)      # not a prime
    with pytest.raises(ValueError):
        o2.o2_h_encode(7, 4, 64, h, 1)      # p - 1 = 6 does not divide the 512 bits of a strip
    with pytest.raises(ValueError):
        o2.o2_h_recover(5, 4, 64, h, 1, 2, 2)


# ------------------------------------------------- Z_257 (256-bit elements)

def test_o2_h257_inverse_equals_the_oracle(oracle):
    import random
    rnd = random.Random(257)
    for z in list(range(1, 12)) + [128, 255, 256]:
        u = 1 ^ oracle.big_ring_xpow(257, z)
        assert oracle.o2_h257_inverse(u) == oracle.big_ring_inv(257, u)
    for _ in range(6):
        a = rnd.getrandbits(256)
        assert oracle.o2_h257_inverse(a) == oracle.big_ring_inv(257, a)


@pytest.mark.parametrize("N,B,S", [(1, 32, 2), (4, 64, 3), (17, 96, 2), (257, 32, 2)])
def test_o2_h257_equals_the_oracle(oracle, N, B, S):
    rng = np.random.default_rng(2570 + N)
    h = rng.integers(0, 256, size=(S, N + 2, B), dtype=np.uint8)
    a, b = h.copy(), h.copy()
    oracle.hbig_encode(257, N, B, a, S)
    oracle.o2_h257_encode(N, B, b, S, threads=3)
    assert np.array_equal(a, b)
    pairs = [(i, j) for i in range(N + 2) for j in range(i + 1, N + 2)]
    picks = list(rng.choice(len(pairs), min(10, len(pairs)), replace=False))
    if N == 257:
        picks += [pairs.index((256, 258)), pairs.index((3, 257))]
    for t in picks:
        i, j = pairs[t]
        x, y = a.copy(), a.copy()
        for z in (x, y):
            z[:, i] = 0xA5
            z[:, j] = 0x5A
        oracle.hbig_recover(257, N, B, x, S, i, j)
        oracle.o2_h257_recover(N, B, y, S, i, j, threads=2)
        assert np.array_equal(x, y), (i, j)
        assert np.array_equal(y, a), (i, j)


def test_o2_h257_per_stripe_pairs_and_strides(oracle):
    N, B, S = 9, 64, 5
    ss, st = 96, 96 * (N + 2) + 32
    rng = np.random.default_rng(2571)
    flat = rng.integers(0, 256, size=st * S, dtype=np.uint8)
    a, b = flat.copy(), flat.copy()
    oracle.hbig_encode(257, N, B, a, S, ss, st)
    oracle.o2_h257_encode(N, B, b, S, ss, st)
    assert np.array_equal(a, b)
    pairs = np.array([[0, 1], [3, N], [2, N + 1], [N, N + 1], [4, 8]], dtype=np.uint16)
    x, y = a.copy(), a.copy()
    oracle.hbig_recover(257, N, B, x, S, pairs=pairs, strip_stride=ss, stripe_stride=st)
    oracle.o2_h257_recover(N, B, y, S, pairs=pairs, strip_stride=ss, stripe_stride=st)
    assert np.array_equal(x, y)
    assert np.array_equal(y, a)
