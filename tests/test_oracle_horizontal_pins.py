"""Pins for the oracle's horizontal representation (Section 4.5): one ring
element per (p-1)-bit field of a strip, little-endian -- for p = 17 one 16-bit
word holding y_0..y_15, the coefficients of x^0..x^15.

The independent models are (1) the bit-sliced oracle, already pinned, applied
to the transposed stripe (row r of the bit-sliced strip holds bit r of every
element), (2) the Z_17 word formulas the paper prints: Q by the Horner form
Q = d + g Q of Section 4.2 with g x = (x + x) ^ (x < 0 ? 0xffff : 0) of
Section 4.5, and the two-data reconstruction of Section 4.6 evaluated with its
own Horner forms (delP), (delQ) and the word formula for g^k x.
"""
import numpy as np
import pytest

from test_oracle_pins import all_pairs

POISON = 0xA5


def h_random(seed, p, N, strip_bytes, S):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(S, N + 2, strip_bytes), dtype=np.uint8)


def to_bitsliced(h, p):
    """[S, strips, strip_bytes] horizontal -> [S, strips, p-1, L/8] bit-sliced,
    L = strip_bytes * 8 / (p-1) elements per strip (L a multiple of 8)."""
    S, K, B = h.shape
    L = B * 8 // (p - 1)
    bits = np.unpackbits(h, axis=-1, bitorder="little").reshape(S, K, L, p - 1)
    return np.ascontiguousarray(np.packbits(bits.transpose(0, 1, 3, 2), axis=-1, bitorder="little"))


def from_bitsliced(b, p):
    S, K, R, C = b.shape
    bits = np.unpackbits(b, axis=-1, bitorder="little")  # [S, K, p-1, L]
    return np.ascontiguousarray(np.packbits(bits.transpose(0, 1, 3, 2).reshape(S, K, -1), axis=-1,
                                            bitorder="little"))


CASES = [(3, 2, 16, 3), (3, 3, 32, 2), (5, 4, 16, 3), (5, 5, 64, 2), (5, 9, 32, 2), (7, 6, 48, 2),
         (13, 12, 24, 2), (17, 16, 64, 3), (17, 1, 32, 2), (17, 33, 32, 1), (29, 20, 56, 1)]


@pytest.mark.parametrize("p,N,B,S", CASES)
def test_h_encode_is_the_transposed_bitsliced_code(oracle, p, N, B, S):
    h = h_random(10 + p + N, p, N, B, S)
    b = to_bitsliced(h, p)
    assert np.array_equal(from_bitsliced(b, p), h)  # the transposition is a bijection
    C = b.shape[-1]
    oracle.encode(p, N, C, b, S)
    oracle.h_encode(p, N, B, h, S)
    assert np.array_equal(h, from_bitsliced(b, p))


@pytest.mark.parametrize("p,N,B", [(5, 4, 16), (3, 3, 16), (17, 16, 32), (5, 9, 16), (13, 25, 24)])
def test_h_recover_is_the_transposed_bitsliced_code(oracle, p, N, B):
    h = h_random(20 + p, p, N, B, 1)
    oracle.h_encode(p, N, B, h, 1)
    pairs = all_pairs(N)
    if len(pairs) > 60:
        rng = np.random.default_rng(p)
        pairs = [pairs[t] for t in rng.choice(len(pairs), 60, replace=False)]
    for (i, j) in pairs:
        lost = h.copy()
        lost[0, i] = POISON
        lost[0, j] = POISON ^ 0xFF
        b = to_bitsliced(lost, p)
        oracle.recover(p, N, b.shape[-1], b, 1, i, j)
        oracle.h_recover(p, N, B, lost, 1, i, j)
        assert np.array_equal(lost, from_bitsliced(b, p)), (i, j)
        assert np.array_equal(lost, h), (i, j)


def g_word(x):
    """Section 4.5: y = g x on int16 words, y = (x + x) ^ ((x < 0) ? 0xffff : 0)."""
    x = x.astype(np.int16)
    return ((x.astype(np.int32) * 2).astype(np.int16) ^ np.where(x < 0, np.int16(-1), np.int16(0))).astype(np.uint16)


def gk_word(x, k):
    """Section 4.6: y = g^k x = (x << k) ^ (x >> (17 - k)) ^ (((x << (k-1)) < 0) ? 0xffff : 0),
    1 <= k <= 16, the right shift logical (psrlw)."""
    x = x.astype(np.uint16).astype(np.uint32)
    y = ((x << k) & 0xFFFF) ^ (x >> (17 - k))
    sign = ((x << (k - 1)) & 0x8000) != 0
    return (y ^ np.where(sign, 0xFFFF, 0)).astype(np.uint16)


@pytest.mark.parametrize("N", [1, 2, 5, 16, 17])
def test_h17_encode_by_the_papers_horner_form(oracle, N):
    # Section 4.2: P = D + P, Q = D + g Q over the disks from the last to the first
    S, B = 2, 64
    h = h_random(30 + N, 17, N, B, S)
    w = h.view(np.uint16)  # [S, N+2, 32] little-endian words
    P = np.zeros_like(w[:, 0])
    Q = np.zeros_like(w[:, 0])
    for k in range(N - 1, -1, -1):
        P ^= w[:, k]
        Q = g_word(Q) ^ w[:, k]
    oracle.h_encode(17, N, B, h, S)
    assert np.array_equal(w[:, N], P)
    assert np.array_equal(w[:, N + 1], Q)


@pytest.mark.parametrize("x,y", [(0, 1), (2, 9), (3, 15), (0, 15), (7, 8), (14, 15)])
def test_h17_two_data_reconstruction_by_section_4_6(oracle, x, y):
    # D_y = (1 + g^z)^-1 dP + g^(17-x) (1 + g^z)^-1 dQ, each by the Horner form
    # with (p+1)/2 = 9 terms; D_x = D_y + dP.  (delP) is read as
    # dP + g^2z (dP + g^2z (... )), the sum of the even powers of g^z.
    N, B = 16, 64
    h = h_random(40 + x + y, 17, N, B, 1)
    oracle.h_encode(17, N, B, h, 1)
    w = h.view(np.uint16)[0]
    dP = w[N].copy()
    dQ = w[N + 1].copy()
    for k in range(N):
        if k in (x, y):
            continue
        dP ^= w[k]
        dQ ^= gk_word(w[k], k) if k else w[k]
    z = y - x

    def horner(v):
        acc = v.copy()
        for _ in range(8):
            acc = gk_word(acc, (2 * z) % 17) ^ v if (2 * z) % 17 else acc ^ v
        return acc

    Dy = horner(dP) ^ gk_word(horner(dQ), 17 - x) if x else horner(dP) ^ horner(dQ)
    Dx = Dy ^ dP
    lost = h.copy()
    lost[0, x] = POISON
    lost[0, y] = POISON
    oracle.h_recover(17, N, B, lost, 1, x, y)
    lw = lost.view(np.uint16)[0]
    assert np.array_equal(lw[y], Dy) and np.array_equal(lw[x], Dx)
    assert np.array_equal(lw[y], w[y]) and np.array_equal(lw[x], w[x])


@pytest.mark.parametrize("p,B", [(3, 8), (5, 8), (17, 16)])
def test_h_element_boundaries(oracle, p, B):
    # a single set bit in element e of data strip 1: P and Q change only in
    # element e, and there Q = x * (that element) of the ring
    N = 3
    L = B * 8 // (p - 1)
    for e in (0, 1, L - 1):
        for r in (0, p - 2):
            h = np.zeros((1, N + 2, B), dtype=np.uint8)
            t = e * (p - 1) + r
            h[0, 1, t // 8] |= 1 << (t % 8)
            oracle.h_encode(p, N, B, h, 1)
            bits = np.unpackbits(h[0], axis=-1, bitorder="little").reshape(N + 2, L, p - 1)
            for k in (N, N + 1):
                others = np.delete(bits[k], e, axis=0)
                assert not others.any(), (p, e, r, k)
            assert bits[N, e].tolist() == [int(q == r) for q in range(p - 1)]
            want = oracle.ring_xpow(p, 1 + r)  # x * x^r in R
            got = sum(int(v) << q for q, v in enumerate(bits[N + 1, e]))
            assert got == want, (p, e, r)


def test_h_invalid_arguments(oracle):
    h = np.zeros((1, 10, 16), dtype=np.uint8)
    with pytest.raises(ValueError):
        oracle.h_encode(13, 4, 4, h, 1)  # 32 bits is not a whole number of 12-bit elements
    with pytest.raises(ValueError):
        oracle.h_encode(7, 8, 16, h, 1)  # N > p where Theorem 3.3.3 fails
    oracle.h_encode(13, 4, 3, h, 1)      # 24 bits: two elements
