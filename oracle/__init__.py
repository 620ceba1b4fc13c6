"""CPU oracle for the cyclic-group RAID-6 code (arXiv cs/0611109).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product package never imports this
module and this module never imports the product package.

This file is a thin ctypes binding over ``rcg_oracle.c`` (compiled with gcc into
``oracle/_build/``).  All arithmetic lives in the C file: bit-level polynomial
arithmetic in R = F2[x]/(1 + x + ... + x^(p-1)), one codeword per bit position,
following Corollary 3.2.4 (encode, extended to 2p - 1 data strips by equation
qext of Section 3.3 when Theorem 3.3.3 allows it) and Lemma 3.1.2 (the four
erasure-pair cases).  Buffers are numpy uint8 arrays in the stripe layout
``[stripe][strip 0..N+1][row 0..p-2][C bytes]`` (strip N = P, strip N+1 = Q),
with optional explicit byte strides.

Parity pins: every function here is checked against facts the paper and the
mathematics fix (tests/test_oracle_pins.py); no function is unpinned.

``rcg_o2.c`` ("O2") is a second, word-level and multi-threaded CPU
implementation of the same code (64 codewords per machine word, inverses by
Gaussian elimination), bound below as ``o2_encode`` / ``o2_recover``.  It is
fast enough to check full-size GPU results byte for byte; it is pinned to the
bit-level functions above (tests/test_oracle_o2.py) and shares no code with
them or with the product.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librcg_oracle.so")

_u64 = ctypes.c_uint64
_uint = ctypes.c_uint
_vp = ctypes.c_void_p


def build(src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle with gcc (portable C, no target-specific flags)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def load(path: str | None = None) -> ctypes.CDLL:
    lib = ctypes.CDLL(path or build())
    lib.oracle_ring_mul.restype = _u64
    lib.oracle_ring_mul.argtypes = [_uint, _u64, _u64]
    lib.oracle_ring_xpow.restype = _u64
    lib.oracle_ring_xpow.argtypes = [_uint, _uint]
    lib.oracle_ring_inv.restype = _u64
    lib.oracle_ring_inv.argtypes = [_uint, _u64]
    lib.oracle_weight.restype = _u64
    lib.oracle_weight.argtypes = [_uint, _uint]
    lib.oracle_ord2.restype = _uint
    lib.oracle_ord2.argtypes = [_uint]
    lib.oracle_cone_extends.restype = ctypes.c_int
    lib.oracle_cone_extends.argtypes = [_uint]
    lib.oracle_mul_xpow_array.restype = None
    lib.oracle_mul_xpow_array.argtypes = [_uint, _uint, _vp, _vp, ctypes.c_size_t]
    lib.oracle_encode.restype = ctypes.c_int
    lib.oracle_encode.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _u64]
    lib.oracle_recover.restype = ctypes.c_int
    lib.oracle_recover.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _u64, _uint, _uint, _vp]
    lib.oracle_update.restype = ctypes.c_int
    lib.oracle_update.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _u64, _uint, _vp, _u64]
    lib.oracle_degraded_read.restype = ctypes.c_int
    lib.oracle_degraded_read.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _u64, _uint, _vp, _u64]
    lib.oracle_h_encode.restype = ctypes.c_int
    lib.oracle_h_encode.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64]
    lib.oracle_h_recover.restype = ctypes.c_int
    lib.oracle_h_recover.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _uint, _uint, _vp]
    for name in ("oracle_big_ring_mul",):
        getattr(lib, name).restype = ctypes.c_int
        getattr(lib, name).argtypes = [_uint, _vp, _vp, _vp]
    lib.oracle_big_ring_xpow.restype = ctypes.c_int
    lib.oracle_big_ring_xpow.argtypes = [_uint, _uint, _vp]
    lib.oracle_big_ring_inv.restype = ctypes.c_int
    lib.oracle_big_ring_inv.argtypes = [_uint, _vp, _vp]
    lib.oracle_hbig_encode.restype = ctypes.c_int
    lib.oracle_hbig_encode.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64]
    lib.oracle_hbig_recover.restype = ctypes.c_int
    lib.oracle_hbig_recover.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _uint, _uint, _vp]
    return lib


_lib: ctypes.CDLL | None = None


def lib() -> ctypes.CDLL:
    """The loaded oracle.  RCG_ORACLE_LIB, when set, names another build of
    rcg_oracle.c to load instead (the mutation tests use it)."""
    global _lib
    if _lib is None:
        _lib = load(os.environ.get("RCG_ORACLE_LIB") or None)
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _strides(p, N, C, row_stride, strip_stride, stripe_stride):
    row_stride = C if row_stride is None else row_stride
    strip_stride = (p - 1) * row_stride if strip_stride is None else strip_stride
    stripe_stride = (N + 2) * strip_stride if stripe_stride is None else stripe_stride
    return row_stride, strip_stride, stripe_stride


def _check_buf(buf: np.ndarray):
    if buf.dtype != np.uint8 or not buf.flags["C_CONTIGUOUS"] or not buf.flags["WRITEABLE"]:
        raise ValueError("oracle buffers must be writeable C-contiguous uint8 arrays")


# ------------------------------------------------------------------ ring ops

def ring_mul(p: int, a: int, b: int) -> int:
    """Product in R = F2[x]/(1+...+x^(p-1)); bit r of an int = coefficient of x^r."""
    return int(lib().oracle_ring_mul(p, a, b))


def ring_xpow(p: int, k: int) -> int:
    """x^k in R (0 <= k < 128)."""
    return int(lib().oracle_ring_xpow(p, k))


def ring_inv(p: int, a: int) -> int:
    """Inverse in R by extended Euclid; 0 if a is not invertible."""
    return int(lib().oracle_ring_inv(p, a))


def weight(p: int, k: int) -> int:
    """Q weight of data strip k: x^k for k < p, 1 + x^(k-p+1) for p <= k <= 2p-2
    (equation qext of Section 3.3)."""
    return int(lib().oracle_weight(p, k))


def ord2(p: int) -> int:
    """Order of 2 modulo the prime p (Lemma 3.3.1)."""
    return int(lib().oracle_ord2(p))


def cone_extends(p: int) -> bool:
    """Condition (3) of Theorem 3.3.3 for the prime p (3 <= p <= 127): the
    code extends to 2p - 1 data strips."""
    return bool(lib().oracle_cone_extends(p))


def mul_xpow_array(p: int, k: int, a: np.ndarray) -> np.ndarray:
    """x^k * a[t] in R for every element of a uint64 array."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.empty_like(a)
    lib().oracle_mul_xpow_array(p, k, _ptr(a), _ptr(out), a.size)
    return out


# ------------------------------------------------------------- stripe ops

def encode(p, N, C, buf, n_stripes, row_stride=None, strip_stride=None, stripe_stride=None):
    """Write P and Q of every stripe (Corollary 3.2.4, equation znparity)."""
    _check_buf(buf)
    rs, ss, st = _strides(p, N, C, row_stride, strip_stride, stripe_stride)
    rc = lib().oracle_encode(p, N, C, _ptr(buf), n_stripes, rs, ss, st)
    if rc:
        raise ValueError("oracle_encode: invalid arguments")


def recover(p, N, C, buf, n_stripes, i=0, j=1, pairs=None, row_stride=None,
            strip_stride=None, stripe_stride=None):
    """Rebuild strips i < j (or per-stripe pairs, uint8 [n_stripes, 2]) in place
    by the case analysis of Lemma 3.1.2."""
    _check_buf(buf)
    rs, ss, st = _strides(p, N, C, row_stride, strip_stride, stripe_stride)
    pp = None
    if pairs is not None:
        pairs = np.ascontiguousarray(pairs, dtype=np.uint8)
        pp = _ptr(pairs)
    rc = lib().oracle_recover(p, N, C, _ptr(buf), n_stripes, rs, ss, st, i, j, pp)
    if rc:
        raise ValueError("oracle_recover: invalid arguments (rc=%d)" % rc)


def update(p, N, C, buf, stripe, i, new_strip, row_stride=None, strip_stride=None,
           stripe_stride=None):
    """Store new_strip ((p-1) x C uint8) as data strip i of one stripe and
    re-encode that stripe."""
    _check_buf(buf)
    rs, ss, st = _strides(p, N, C, row_stride, strip_stride, stripe_stride)
    new_strip = np.ascontiguousarray(new_strip, dtype=np.uint8).reshape(p - 1, -1)
    rc = lib().oracle_update(p, N, C, _ptr(buf), stripe, rs, ss, st, i, _ptr(new_strip),
                             new_strip.shape[1])
    if rc:
        raise ValueError("oracle_update: invalid arguments")


def degraded_read(p, N, C, buf, stripe, j, row_stride=None, strip_stride=None,
                  stripe_stride=None) -> np.ndarray:
    """Strip j of one stripe rebuilt from the others, as a (p-1) x C array."""
    _check_buf(buf)
    rs, ss, st = _strides(p, N, C, row_stride, strip_stride, stripe_stride)
    out = np.zeros((p - 1, C), dtype=np.uint8)
    rc = lib().oracle_degraded_read(p, N, C, _ptr(buf), stripe, rs, ss, st, j, _ptr(out), C)
    if rc:
        raise ValueError("oracle_degraded_read: invalid arguments")
    return out


# --------------------------------------------------------- horizontal strips

def _h_strides(N, strip_bytes, strip_stride, stripe_stride):
    strip_stride = strip_bytes if strip_stride is None else strip_stride
    stripe_stride = (N + 2) * strip_stride if stripe_stride is None else stripe_stride
    return strip_stride, stripe_stride


def h_encode(p, N, strip_bytes, buf, n_stripes, strip_stride=None, stripe_stride=None):
    """Encode stripes in the horizontal representation of Section 4.5: element
    e of a strip is bits [e(p-1), (e+1)(p-1)) of the strip, little-endian (for
    p = 17 the 16-bit word e)."""
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    rc = lib().oracle_h_encode(p, N, strip_bytes, _ptr(buf), n_stripes, ss, st)
    if rc:
        raise ValueError("oracle_h_encode: invalid arguments")


def h_recover(p, N, strip_bytes, buf, n_stripes, i=0, j=1, pairs=None, strip_stride=None,
              stripe_stride=None):
    """Rebuild strips i < j (or per-stripe pairs) of horizontal stripes in place
    (Lemma 3.1.2)."""
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    pp = None
    if pairs is not None:
        pairs = np.ascontiguousarray(pairs, dtype=np.uint8)
        pp = _ptr(pairs)
    rc = lib().oracle_h_recover(p, N, strip_bytes, _ptr(buf), n_stripes, ss, st, i, j, pp)
    if rc:
        raise ValueError("oracle_h_recover: invalid arguments (rc=%d)" % rc)


# ------------------------------------------- large primes (p up to 257)

def _big_bytes(p: int) -> int:
    return (p - 1 + 7) // 8


def _to_bits(p: int, a: int) -> np.ndarray:
    return np.frombuffer(int(a).to_bytes(_big_bytes(p), "little"), dtype=np.uint8).copy()


def _from_bits(b: np.ndarray) -> int:
    return int.from_bytes(bytes(b), "little")


def big_ring_mul(p: int, a: int, b: int) -> int:
    """a * b in R for any odd prime p <= 257 (bit m = coefficient of x^m):
    coefficient arrays, schoolbook product, long division by f."""
    x, y, out = _to_bits(p, a), _to_bits(p, b), np.zeros(_big_bytes(p), np.uint8)
    if lib().oracle_big_ring_mul(p, _ptr(x), _ptr(y), _ptr(out)):
        raise ValueError("oracle_big_ring_mul: invalid p")
    return _from_bits(out)


def big_ring_xpow(p: int, k: int) -> int:
    out = np.zeros(_big_bytes(p), np.uint8)
    if lib().oracle_big_ring_xpow(p, k, _ptr(out)):
        raise ValueError("oracle_big_ring_xpow: invalid arguments")
    return _from_bits(out)


def big_ring_inv(p: int, a: int) -> int:
    """Inverse in R by the extended Euclidean algorithm; 0 when a is not a unit."""
    x, out = _to_bits(p, a), np.zeros(_big_bytes(p), np.uint8)
    rc = lib().oracle_big_ring_inv(p, _ptr(x), _ptr(out))
    if rc < 0:
        raise ValueError("oracle_big_ring_inv: invalid p")
    return _from_bits(out) if rc else 0


def hbig_encode(p, N, strip_bytes, buf, n_stripes, strip_stride=None, stripe_stride=None):
    """Encode horizontal stripes (element e = bits [e(p-1), (e+1)(p-1)) of a
    strip) for any odd prime p <= 257, N <= p: the coefficient-array code."""
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    if lib().oracle_hbig_encode(p, N, strip_bytes, _ptr(buf), n_stripes, ss, st):
        raise ValueError("oracle_hbig_encode: invalid arguments")


def hbig_recover(p, N, strip_bytes, buf, n_stripes, i=0, j=1, pairs=None, strip_stride=None,
                 stripe_stride=None):
    """Rebuild strips i < j (or per-stripe pairs, [n_stripes, 2] of 16-bit
    numbers) of horizontal stripes of any odd prime p <= 257 in place
    (Lemma 3.1.2, inverses by Euclid)."""
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    pp = None
    if pairs is not None:
        pairs = np.ascontiguousarray(pairs, dtype=np.uint16)
        pp = _ptr(pairs)
    rc = lib().oracle_hbig_recover(p, N, strip_bytes, _ptr(buf), n_stripes, ss, st, i, j, pp)
    if rc:
        raise ValueError("oracle_hbig_recover: invalid arguments (rc=%d)" % rc)


# ------------------------------------------------------- O2 (word-level)

_O2_SRC = os.path.join(_HERE, "rcg_o2.c")
_O2_LIB = os.path.join(_HERE, "_build", "librcg_o2.so")
_o2: ctypes.CDLL | None = None


def build_o2(src: str = _O2_SRC, out: str = _O2_LIB) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def o2() -> ctypes.CDLL:
    global _o2
    if _o2 is None:
        L = ctypes.CDLL(build_o2())
        L.o2_encode.restype = ctypes.c_int
        L.o2_encode.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _u64, ctypes.c_int]
        L.o2_recover.restype = ctypes.c_int
        L.o2_recover.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _u64, _uint, _uint, _vp, ctypes.c_int]
        L.o2_inverse.restype = _u64
        L.o2_inverse.argtypes = [_uint, _u64]
        L.o2_h_encode.restype = ctypes.c_int
        L.o2_h_encode.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, ctypes.c_int]
        L.o2_h_recover.restype = ctypes.c_int
        L.o2_h_recover.argtypes = [_uint, _uint, _u64, _vp, _u64, _u64, _u64, _uint, _uint, _vp, ctypes.c_int]
        L.o2_h257_encode.restype = ctypes.c_int
        L.o2_h257_encode.argtypes = [_uint, _u64, _vp, _u64, _u64, _u64, ctypes.c_int]
        L.o2_h257_recover.restype = ctypes.c_int
        L.o2_h257_recover.argtypes = [_uint, _u64, _vp, _u64, _u64, _u64, _uint, _uint, _vp, ctypes.c_int]
        L.o2_h257_inverse.restype = ctypes.c_int
        L.o2_h257_inverse.argtypes = [_vp, _vp]
        _o2 = L
    return _o2


def _threads(threads):
    return threads or os.cpu_count() or 1


def o2_encode(p, N, C, buf, n_stripes, row_stride=None, strip_stride=None, stripe_stride=None, threads=None):
    """Word-level encode (Corollary 3.2.4 / qext) of n_stripes stripes in place; C % 8 == 0."""
    _check_buf(buf)
    rs, ss, st = _strides(p, N, C, row_stride, strip_stride, stripe_stride)
    rc = o2().o2_encode(p, N, C, _ptr(buf), n_stripes, rs, ss, st, _threads(threads))
    if rc:
        raise ValueError("o2_encode: invalid arguments (rc=%d)" % rc)


def o2_recover(p, N, C, buf, n_stripes, i=0, j=1, pairs=None, row_stride=None, strip_stride=None,
               stripe_stride=None, threads=None):
    """Word-level recovery (Lemma 3.1.2) of pair (i, j) or per-stripe pairs, in place."""
    _check_buf(buf)
    rs, ss, st = _strides(p, N, C, row_stride, strip_stride, stripe_stride)
    pp = None
    if pairs is not None:
        pairs = np.ascontiguousarray(pairs, dtype=np.uint8)
        pp = _ptr(pairs)
    rc = o2().o2_recover(p, N, C, _ptr(buf), n_stripes, rs, ss, st, i, j, pp, _threads(threads))
    if rc:
        raise ValueError("o2_recover: invalid arguments (rc=%d)" % rc)


def o2_h_encode(p, N, strip_bytes, buf, n_stripes, strip_stride=None, stripe_stride=None, threads=None):
    """Word-level encode of stripes in the horizontal representation of Section 4.5, in place."""
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    rc = o2().o2_h_encode(p, N, strip_bytes, _ptr(buf), n_stripes, ss, st, _threads(threads))
    if rc:
        raise ValueError("o2_h_encode: invalid arguments (rc=%d)" % rc)


def o2_h_recover(p, N, strip_bytes, buf, n_stripes, i=0, j=1, pairs=None, strip_stride=None,
                 stripe_stride=None, threads=None):
    """Word-level recovery (Lemma 3.1.2) of horizontal stripes, pair (i, j) or per-stripe pairs, in place."""
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    pp = None
    if pairs is not None:
        pairs = np.ascontiguousarray(pairs, dtype=np.uint8)
        pp = _ptr(pairs)
    rc = o2().o2_h_recover(p, N, strip_bytes, _ptr(buf), n_stripes, ss, st, i, j, pp, _threads(threads))
    if rc:
        raise ValueError("o2_h_recover: invalid arguments (rc=%d)" % rc)


def o2_h257_encode(N, strip_bytes, buf, n_stripes, strip_stride=None, stripe_stride=None, threads=None):
    """Word-level encode of Z_257 stripes in the horizontal representation
    (element e = bytes [32e, 32e + 32)), N <= 257."""
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    rc = o2().o2_h257_encode(N, strip_bytes, _ptr(buf), n_stripes, ss, st, _threads(threads))
    if rc:
        raise ValueError("o2_h257_encode: invalid arguments (rc=%d)" % rc)


def o2_h257_recover(N, strip_bytes, buf, n_stripes, i=0, j=1, pairs=None, strip_stride=None,
                    stripe_stride=None, threads=None):
    _check_buf(buf)
    ss, st = _h_strides(N, strip_bytes, strip_stride, stripe_stride)
    pp = None
    if pairs is not None:
        pairs = np.ascontiguousarray(pairs, dtype=np.uint16)  # strip indices reach 258
        pp = _ptr(pairs)
    rc = o2().o2_h257_recover(N, strip_bytes, _ptr(buf), n_stripes, ss, st, i, j, pp, _threads(threads))
    if rc:
        raise ValueError("o2_h257_recover: invalid arguments (rc=%d)" % rc)


def o2_h257_inverse(a: int) -> int:
    """Inverse in R (p = 257) by Gaussian elimination; 0 when singular."""
    x = np.frombuffer(int(a).to_bytes(32, "little"), dtype=np.uint8).copy()
    out = np.zeros(32, np.uint8)
    return int.from_bytes(bytes(out), "little") if o2().o2_h257_inverse(_ptr(x), _ptr(out)) else 0


def o2_inverse(p: int, a: int) -> int:
    return int(o2().o2_inverse(p, a))
