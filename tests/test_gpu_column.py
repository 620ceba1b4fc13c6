"""Parity of the column kernel (bit-sliced stripes of p <= 7 held in
registers, Q by Horner's rule) with the CPU oracle and with the tile engine
on the same inputs.  Bit-exact everywhere."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_cs_0611109_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

POISON_I, POISON_J = 0xA5, 0x5A


@pytest.fixture(scope="module")
def rcg():
    from paper_cs_0611109_gb300 import build
    build.build()
    from paper_cs_0611109_gb300 import rcg as R
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return R


@pytest.fixture(scope="module")
def ctxs(rcg):
    col = rcg.Context(0)           # default: column kernel for p <= 7
    eng = rcg.Context(0)
    eng.set_column_kernel(rcg.RCG_COLUMN_OFF)
    yield col, eng
    col.close()
    eng.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def stripes(seed, p, N, C, S):
    return np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, S))


CASES = [(3, 1, 16, 4), (3, 3, 1040, 3), (5, 4, 1024, 5), (5, 5, 48, 3), (5, 7, 2048 + 16, 2), (5, 9, 256, 3),
         (7, 1, 32, 2), (7, 6, 4096, 2), (7, 7, 1040, 2)]


@pytest.mark.parametrize("p,N,C,S", CASES)
def test_column_encode_matches_oracle_and_engine(rcg, ctxs, oracle, p, N, C, S):
    col, eng = ctxs
    host = stripes(4000 + p + N, p, N, C, S)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    for c in (col, eng):
        buf = dev(host)
        c.encode(rcg.make_layout(buf, p, N, C), 0, S)
        assert c.last_device_status() == 0
        assert np.array_equal(buf.cpu().numpy(), want)


@pytest.mark.parametrize("p,N,C,S", CASES)
@pytest.mark.parametrize("kind", ["dd", "dp", "dq", "pq", "any"])
def test_column_recover_many_matches_oracle(rcg, ctxs, oracle, p, N, C, S, kind):
    if kind == "dd" and N < 2:
        pytest.skip("two-data erasures need N >= 2")
    col, _ = ctxs
    host = stripes(4100 + p + N, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    pairs = inputs.random_pairs(4101 + N, N, S, kind)
    lost = host.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    want = lost.copy()
    oracle.recover(p, N, C, want, S, pairs=pairs)
    buf = dev(lost)
    col.recover_many(rcg.make_layout(buf, p, N, C), 0, S, dev(pairs))
    assert col.last_device_status() == 0
    assert np.array_equal(buf.cpu().numpy(), want)
    assert np.array_equal(want, host)


@pytest.mark.parametrize("p,N", [(5, 9), (5, 4), (3, 3), (7, 7)])
def test_column_recover_every_pair(rcg, ctxs, oracle, p, N):
    col, _ = ctxs
    C, S = 64, 2
    host = stripes(4200 + p + N, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    for i in range(N + 2):
        for j in range(i + 1, N + 2):
            lost = host.copy()
            lost[:, i] = POISON_I
            lost[:, j] = POISON_J
            buf = dev(lost)
            L = rcg.make_layout(buf, p, N, C)
            for s in range(S):
                col.recover(L, s, i, j)
            assert np.array_equal(buf.cpu().numpy(), host), (i, j)
    assert col.last_device_status() == 0


def test_column_strides_and_subrange(rcg, ctxs, oracle):
    col, _ = ctxs
    p, N, C, S = 5, 4, 96, 6
    rs, ss = 128, 128 * (p - 1) + 32
    st = ss * (N + 2) + 64
    flat = inputs.random_bytes(4300, st * S)
    buf = dev(flat)
    L = rcg.make_layout(buf, p, N, C, rs, ss, st)
    col.encode(L, 2, 3)
    assert col.last_device_status() == 0
    want = flat.copy()
    oracle.encode(p, N, C, want[2 * st:], 3, rs, ss, st)
    assert np.array_equal(buf.cpu().numpy(), want)
    # recover a pair in place on the strided layout
    v = buf.cpu().numpy().copy()
    s0 = 3 * st
    for k in (1, N + 1):
        for r in range(p - 1):
            v[s0 + k * ss + r * rs: s0 + k * ss + r * rs + C] = POISON_I
    buf2 = dev(v)
    col.recover(rcg.make_layout(buf2, p, N, C, rs, ss, st), 3, 1, N + 1)
    assert col.last_device_status() == 0
    assert np.array_equal(buf2.cpu().numpy(), want)


def test_column_rejects_bad_pairs_on_device(rcg, ctxs, oracle):
    col, _ = ctxs
    p, N, C, S = 5, 4, 64, 4
    host = stripes(4400, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    pairs = np.array([[0, 1], [2, 2], [3, 7], [4, 5]], dtype=np.uint8)
    lost = host.copy()
    lost[0, 0:2] = POISON_I
    lost[3, 4:6] = POISON_I
    buf = dev(lost)
    col.recover_many(rcg.make_layout(buf, p, N, C), 0, S, dev(pairs))
    torch.cuda.synchronize()
    assert col.last_device_status() == rcg.RCG_DEV_BADPAIR
    got = buf.cpu().numpy()
    assert np.array_equal(got[[0, 3]], host[[0, 3]])
    assert np.array_equal(got[[1, 2]], lost[[1, 2]])


def test_column_kernel_setting_is_validated(rcg, ctxs):
    col, _ = ctxs
    with pytest.raises(rcg.RcgError):
        col.set_column_kernel(7)
