"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the RAID-6 method: it only makes random
bytes and random erasure choices.  The CUDA library carries a twin of the byte
generator (``rcg_fill_random``) so that full-size buffers can be generated on
the device; a test checks that the two agree byte for byte.

Byte generator.  Word w (8 bytes, little-endian) of stream ``seed`` is the
(w+1)-th output of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the public
64-bit version by Vigna) started from state ``seed * 2**40``:

    z  = seed * 2**40 + (w + 1) * 0x9E3779B97F4A7C15      (mod 2**64)
    z ^= z >> 30;  z *= 0xBF58476D1CE4E5B9
    z ^= z >> 27;  z *= 0x94D049BB133111EB
    z ^= z >> 31

A buffer of n bytes is the byte string of words 0, 1, 2, ... truncated to n.
Byte offset o (a multiple of 8) of the buffer starts at word o / 8, so any
stripe of a packed stripe array can be regenerated on its own.
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
SEED_SHIFT = 40


def splitmix_words(seed: int, first_word: int, n_words: int) -> np.ndarray:
    """Words [first_word, first_word + n_words) of stream ``seed`` as uint64."""
    w = np.arange(first_word, first_word + n_words, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (w + np.uint64(1)) * np.uint64(GAMMA) + np.uint64((seed << SEED_SHIFT) & (2**64 - 1))
        z ^= z >> np.uint64(30)
        z *= np.uint64(M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(M2)
        z ^= z >> np.uint64(31)
    return z


def random_bytes(seed: int, nbytes: int, byte_offset: int = 0) -> np.ndarray:
    """Bytes [byte_offset, byte_offset + nbytes) of stream ``seed`` (uint8)."""
    if byte_offset % 8:
        raise ValueError("byte_offset must be a multiple of 8")
    n_words = (nbytes + 7) // 8
    w = splitmix_words(seed, byte_offset // 8, n_words)
    return w.astype("<u8").view(np.uint8)[:nbytes].copy()


def stripe_bytes(p: int, n_data: int, C: int) -> int:
    """Bytes of one packed stripe: N data strips + P + Q, each p-1 rows of C bytes."""
    return (n_data + 2) * (p - 1) * C


def random_stripes(seed: int, p: int, n_data: int, C: int, n_stripes: int,
                   first_stripe: int = 0) -> np.ndarray:
    """Packed stripes [first_stripe, first_stripe + n_stripes) of a random array,
    shape (n_stripes, N+2, p-1, C).  Parity strips hold random bytes too; an
    encode overwrites them."""
    sb = stripe_bytes(p, n_data, C)
    flat = random_bytes(seed, sb * n_stripes, sb * first_stripe)
    return flat.reshape(n_stripes, n_data + 2, p - 1, C)


def random_pairs(seed: int, n_data: int, n: int, kind: str = "any", dtype=np.uint8) -> np.ndarray:
    """n erasure pairs (i < j) as [n, 2] of `dtype` (uint8, or uint16 where
    strip indices pass 255), drawn uniformly within a class.

    kind: "any" (i < j among all N+2 strips), "dd" (two data strips),
    "dp" (data + P), "dq" (data + Q), "pq" (both parities)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = n_data
    if N + 1 > np.iinfo(dtype).max:
        raise ValueError("strip indices up to %d do not fit %s" % (N + 1, np.dtype(dtype).name))
    out = np.empty((n, 2), dtype=dtype)
    if kind == "any":
        a = rng.integers(0, N + 2, size=n)
        b = rng.integers(0, N + 1, size=n)
        b = np.where(b >= a, b + 1, b)
        out[:, 0] = np.minimum(a, b)
        out[:, 1] = np.maximum(a, b)
    elif kind == "dd":
        if N < 2:
            raise ValueError("two-data erasures need N >= 2")
        a = rng.integers(0, N, size=n)
        b = rng.integers(0, N - 1, size=n)
        b = np.where(b >= a, b + 1, b)
        out[:, 0] = np.minimum(a, b)
        out[:, 1] = np.maximum(a, b)
    elif kind in ("dp", "dq"):
        out[:, 0] = rng.integers(0, N, size=n)
        out[:, 1] = N if kind == "dp" else N + 1
    elif kind == "pq":
        out[:, 0] = N
        out[:, 1] = N + 1
    else:
        raise ValueError(kind)
    return out


BATCH_PRIMES = (5, 13, 29, 59)


def batched_jobs(seed: int, n: int, c_min: int = 512, c_max: int = 65536, encode_share: float = 0.6):
    """Stripe descriptors of the uneven batched workload: p uniform over
    {5, 13, 29, 59}, N uniform in [3, p-1], row bytes log-uniform in
    [c_min, c_max] rounded down to a multiple of 16, and an operation --
    encode with probability encode_share, else the recovery of an erasure
    pair i < j drawn uniformly among the N+2 strips.  One stripe per
    descriptor; returns a list of dicts (p, n, c, op, i, j)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.choice(BATCH_PRIMES, size=n)
    out = []
    logc = rng.uniform(np.log(c_min), np.log(c_max), size=n)
    u = rng.uniform(size=n)
    for k in range(n):
        pk = int(p[k])
        nk = int(rng.integers(3, pk))           # [3, p-1]
        ck = max(16, (int(np.exp(logc[k])) // 16) * 16)
        if u[k] < encode_share:
            out.append(dict(p=pk, n=nk, c=ck, op="encode", i=0, j=0))
        else:
            a = int(rng.integers(0, nk + 2))
            b = int(rng.integers(0, nk + 1))
            b = b + 1 if b >= a else b
            out.append(dict(p=pk, n=nk, c=ck, op="recover", i=min(a, b), j=max(a, b)))
    return out
