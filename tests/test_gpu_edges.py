"""Edge cases on every kernel, bit-exact against the oracles: one data strip
(P = Q = d_0), all-zero and all-ones stripes, rows of 1 MiB, empty launches
and stripe subranges."""
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
    col = rcg.Context(0)            # column kernel for p <= 7
    eng = rcg.Context(0)            # tile engine everywhere
    eng.set_column_kernel(rcg.RCG_COLUMN_OFF)
    yield {"column": col, "engine": eng}
    col.close()
    eng.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def stripes(seed, p, N, C, S):
    return np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, S))


@pytest.mark.parametrize("path", ["column", "engine"])
@pytest.mark.parametrize("p", [3, 5, 7, 13, 59])
def test_one_data_strip_every_pair(rcg, ctxs, oracle, path, p):
    # N = 1: x^0 = 1, so P = Q = d_0; every pair among d_0, P, Q
    c = ctxs[path]
    N, C, S = 1, 1040, 2
    host = stripes(7000 + p, p, N, C, S)
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    c.encode(L, 0, S)
    enc = buf.cpu().numpy()
    assert np.array_equal(enc[:, 1], enc[:, 0]) and np.array_equal(enc[:, 2], enc[:, 0])
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        lost = enc.copy()
        lost[:, i] = POISON_I
        lost[:, j] = POISON_J
        b = dev(lost)
        Lb = rcg.make_layout(b, p, N, C)
        for s in range(S):
            c.recover(Lb, s, i, j)
        assert np.array_equal(b.cpu().numpy(), enc), (i, j)
    assert c.last_device_status() == 0


def test_horizontal_one_data_strip(rcg, ctxs, oracle):
    c = ctxs["column"]
    for p in (3, 5, 17):
        N, B, S = 1, 64, 2
        h = np.ascontiguousarray(inputs.random_bytes(7100 + p, S * 3 * B).reshape(S, 3, B))
        buf = dev(h)
        L = rcg.make_hlayout(buf, p, N, B)
        c.h_encode(L, 0, S)
        enc = buf.cpu().numpy()
        assert np.array_equal(enc[:, 1], enc[:, 0]) and np.array_equal(enc[:, 2], enc[:, 0])
        for (i, j) in ((0, 1), (0, 2), (1, 2)):
            lost = enc.copy()
            lost[:, i] = POISON_I
            lost[:, j] = POISON_J
            b = dev(lost)
            for s in range(S):
                c.h_recover(rcg.make_hlayout(b, p, N, B), s, i, j)
            assert np.array_equal(b.cpu().numpy(), enc), (p, i, j)
    assert c.last_device_status() == 0


@pytest.mark.parametrize("path", ["column", "engine"])
@pytest.mark.parametrize("p,N", [(5, 4), (13, 12), (59, 58), (13, 25)])
@pytest.mark.parametrize("fill", [0x00, 0xFF])
def test_constant_stripes(rcg, ctxs, oracle, path, p, N, fill):
    # all-zero data gives zero parity; all-ones data gives the oracle's parity
    c = ctxs[path]
    C, S = 256, 2
    host = np.full((S, N + 2, p - 1, C), fill, dtype=np.uint8)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    if fill == 0:
        assert not want.any()
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    c.encode(L, 0, S)
    assert np.array_equal(buf.cpu().numpy(), want)
    pairs = np.array([[0, N - 1], [1, N + 1]], dtype=np.uint8)
    lost = want.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    b = dev(lost)
    c.recover_many(rcg.make_layout(b, p, N, C), 0, S, dev(pairs))
    assert np.array_equal(b.cpu().numpy(), want)
    assert c.last_device_status() == 0


@pytest.mark.parametrize("path,p,N", [("engine", 13, 3), ("column", 5, 4), ("engine", 5, 4), ("engine", 59, 2)])
def test_one_mebibyte_rows(rcg, ctxs, oracle, path, p, N):
    # rows of 1 MiB + 16 bytes: hundreds of column tiles per stripe and a
    # ragged last tile; every byte against O2
    c = ctxs[path]
    C, S = (1 << 20) + 16, 2
    host = stripes(7200 + p, p, N, C, S)
    want = host.copy()
    oracle.o2_encode(p, N, C, want, S)
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    c.encode(L, 0, S)
    assert np.array_equal(buf.cpu().numpy(), want)
    pairs = inputs.random_pairs(7201, N, S, "any")
    lost = want.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    b = dev(lost)
    c.recover_many(rcg.make_layout(b, p, N, C), 0, S, dev(pairs))
    assert np.array_equal(b.cpu().numpy(), want)
    assert c.last_device_status() == 0


def test_empty_launches_are_noops(rcg, ctxs):
    c = ctxs["column"]
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    pairs = torch.zeros(16, dtype=torch.uint8, device="cuda")
    for p, N in ((5, 4), (13, 12)):
        L = rcg.make_layout(buf, p, N, 16)
        c.encode(L, 0, 0)
        c.recover_many(L, 0, 0, pairs)
    c.h_encode(rcg.make_hlayout(buf, 17, 4, 64), 0, 0)
    c.h_recover_many(rcg.make_hlayout(buf, 17, 4, 64), 0, 0, pairs)
    assert c.batch_submit([]) == 0
    torch.cuda.synchronize()
    assert c.last_device_status() == 0
    assert not buf.any()


@pytest.mark.parametrize("path,p,N", [("column", 5, 4), ("engine", 13, 12), ("engine", 29, 40)])
def test_recover_many_subrange(rcg, ctxs, oracle, path, p, N):
    # first_stripe > 0: only stripes [2, 5) are touched, the others stay poisoned
    c = ctxs[path]
    C, S = 528, 7
    host = stripes(7300 + p, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    lost = host.copy()
    lost[:, 0] = POISON_I
    lost[:, N] = POISON_J
    buf = dev(lost)
    pairs = np.tile(np.array([[0, N]], dtype=np.uint8), (3, 1))
    c.recover_many(rcg.make_layout(buf, p, N, C), 2, 3, dev(pairs))
    got = buf.cpu().numpy()
    assert np.array_equal(got[2:5], host[2:5])
    assert np.array_equal(got[:2], lost[:2]) and np.array_equal(got[5:], lost[5:])
    assert c.last_device_status() == 0


@pytest.mark.parametrize("shape", ["wide", "pair"])
@pytest.mark.parametrize("p,N,C", [(5, 4, 1040), (13, 12, 2064), (59, 58, 528), (13, 25, 2064)])
def test_degraded_read_and_update_in_both_shapes(rcg, oracle, shape, p, N, C):
    # every kind of ring slot -- P and Q together, P alone, Q alone, the small
    # write's copied strip -- in both engine shapes, against the oracle
    S = 3
    host = stripes(7400 + p + N, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    with rcg.Context(0) as c:
        c.set_column_kernel(rcg.RCG_COLUMN_OFF)
        c.set_engine_shape(rcg.RCG_SHAPE_WIDE if shape == "wide" else rcg.RCG_SHAPE_PAIR)
        for j in sorted({0, N // 2, N - 1, N, N + 1}):
            lost = host.copy()
            lost[:, j] = POISON_I  # the strip served is never read
            buf = dev(lost)
            L = rcg.make_layout(buf, p, N, C)
            out = torch.zeros((S, p - 1, C), dtype=torch.uint8, device="cuda")
            assert c.batch_wait(c.batch_submit([rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, j, out)]))
            assert c.last_device_status() == 0
            assert np.array_equal(out.cpu().numpy(), host[:, j]), j
            one = torch.zeros((p - 1, C), dtype=torch.uint8, device="cuda")
            c.degraded_read(L, 1, j, one)
            torch.cuda.synchronize()
            assert np.array_equal(one.cpu().numpy(), host[1, j]), j
            assert np.array_equal(buf.cpu().numpy(), lost)  # the stripes are not written
        want = host.copy()
        buf = dev(host)
        L = rcg.make_layout(buf, p, N, C)
        for s, i in ((0, 0), (1, N - 1), (2, N // 2)):
            new = inputs.random_bytes(7500 + 7 * s + i, (p - 1) * C).reshape(p - 1, C)
            c.update(L, s, i, dev(new))
            oracle.update(p, N, C, want, s, i, new)
        torch.cuda.synchronize()
        assert c.last_device_status() == 0
        assert np.array_equal(buf.cpu().numpy(), want)
