"""Parity of the horizontal-representation kernel (Section 4.5: one ring
element per (p-1)-bit lane, for p = 17 one 16-bit word) with the CPU oracle.

Bit-exact everywhere.  Expected bytes are the oracle's oracle.h_encode /
oracle.h_recover (themselves pinned to the bit-sliced oracle and to the
paper's Z_17 word formulas) and, for recoveries, the encoded stripe itself.
"""
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
def ctx(rcg):
    c = rcg.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def raw(seed, N, B, S):
    """Seeded horizontal stripes [S, N+2, B] from the shared generator."""
    return np.ascontiguousarray(inputs.random_bytes(seed, S * (N + 2) * B).reshape(S, N + 2, B))


def h_encoded(oracle, seed, p, N, B, S):
    h = raw(seed, N, B, S)
    oracle.h_encode(p, N, B, h, S)
    return h


def clean(ctx):
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0


ENCODE_CASES = [(3, 1, 16, 3), (3, 3, 48, 2), (5, 4, 1024, 3), (5, 9, 1040, 2), (5, 2, 16, 1),
                (17, 1, 64, 2), (17, 16, 4096, 3), (17, 16, 65536 + 16, 1), (17, 33, 2048, 2), (17, 20, 16, 4)]


@pytest.mark.parametrize("p,N,B,S", ENCODE_CASES)
def test_h_encode_matches_oracle(rcg, ctx, oracle, p, N, B, S):
    h = raw(3000 + p + N, N, B, S)
    buf = dev(h)
    ctx.h_encode(rcg.make_hlayout(buf, p, N, B), 0, S)
    clean(ctx)
    oracle.h_encode(p, N, B, h, S)
    assert np.array_equal(buf.cpu().numpy(), h)


def test_h_encode_strides_and_subrange(rcg, ctx, oracle):
    p, N, B, S = 17, 6, 96, 5
    ss, st = 128, 128 * (N + 2) + 48
    flat = inputs.random_bytes(3100, st * S)
    buf = dev(flat)
    ctx.h_encode(rcg.make_hlayout(buf, p, N, B, ss, st), 1, 3)
    clean(ctx)
    want = flat.copy()
    oracle.h_encode(p, N, B, want[st:], 3, ss, st)
    assert np.array_equal(buf.cpu().numpy(), want)


@pytest.mark.parametrize("p,N,B,S", [(3, 3, 16, 2), (5, 4, 64, 2), (5, 9, 48, 1), (17, 16, 256, 1),
                                     (17, 33, 64, 1)])
def test_h_recover_every_pair(rcg, ctx, oracle, p, N, B, S):
    h = h_encoded(oracle, 3200 + p + N, p, N, B, S)
    pairs = [(i, j) for i in range(N + 2) for j in range(i + 1, N + 2)]
    if len(pairs) > 200:
        rng = np.random.default_rng(N)
        pairs = [pairs[t] for t in sorted(rng.choice(len(pairs), 200, replace=False))]
    for (i, j) in pairs:
        lost = h.copy()
        lost[:, i] = POISON_I
        lost[:, j] = POISON_J
        buf = dev(lost)
        L = rcg.make_hlayout(buf, p, N, B)
        for s in range(S):
            ctx.h_recover(L, s, i, j)
        want = lost.copy()
        oracle.h_recover(p, N, B, want, S, i, j)
        got = buf.cpu().numpy()
        assert np.array_equal(got, want), (i, j)
        assert np.array_equal(got, h), (i, j)
    clean(ctx)


@pytest.mark.parametrize("p,N,B", [(17, 16, 4096), (17, 33, 4096 + 16), (5, 9, 1024), (3, 3, 512)])
@pytest.mark.parametrize("kind", ["dd", "dp", "dq", "pq", "any"])
def test_h_recover_many_per_stripe_pairs(rcg, ctx, oracle, p, N, B, kind):
    S = 12
    h = h_encoded(oracle, 3300 + p + N, p, N, B, S)
    pairs = inputs.random_pairs(3301 + len(kind), N, S, kind)
    lost = h.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    buf = dev(lost)
    ctx.h_recover_many(rcg.make_hlayout(buf, p, N, B), 0, S, dev(pairs))
    clean(ctx)
    want = lost.copy()
    oracle.h_recover(p, N, B, want, S, pairs=pairs)
    assert np.array_equal(want, h)
    assert np.array_equal(buf.cpu().numpy(), want)


def test_h_recover_many_rejects_bad_pairs(rcg, ctx, oracle):
    p, N, B, S = 17, 4, 64, 4
    h = h_encoded(oracle, 3400, p, N, B, S)
    pairs = np.array([[0, 1], [3, 3], [2, 9], [4, 5]], dtype=np.uint8)
    lost = h.copy()
    lost[0, 0:2] = POISON_I
    lost[3, 4:6] = POISON_I
    buf = dev(lost)
    ctx.h_recover_many(rcg.make_hlayout(buf, p, N, B), 0, S, dev(pairs))
    torch.cuda.synchronize()
    assert ctx.last_device_status() == rcg.RCG_DEV_BADPAIR
    got = buf.cpu().numpy()
    assert np.array_equal(got[[0, 3]], h[[0, 3]])
    assert np.array_equal(got[[1, 2]], lost[[1, 2]])


def test_h_validation(rcg, ctx):
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    bad = [(13, 4, 64), (7, 4, 64), (5, 10, 64), (3, 4, 64), (17, 34, 64), (17, 4, 24), (17, 4, 0)]
    for p, N, B in bad:
        with pytest.raises(rcg.RcgError):
            ctx.h_encode(rcg.make_hlayout(buf, p, N, B), 0, 1)
    with pytest.raises(rcg.RcgError):
        ctx.h_encode(rcg.make_hlayout(buf[1:], 17, 4, 64), 0, 1)  # misaligned base
    with pytest.raises(rcg.RcgError):
        ctx.h_recover(rcg.make_hlayout(buf, 17, 4, 64), 0, 2, 2)
    with pytest.raises(rcg.RcgError):
        ctx.h_recover(rcg.make_hlayout(buf, 17, 4, 64), 0, 1, 6)
    clean(ctx)


@pytest.mark.slow
def test_h17_full_size(rcg, ctx, oracle):
    # the horizontal bench geometry: p = 17, N = 16, 64 KiB strips, 4096 stripes, seed 5;
    # encode checked on every byte by O2, sampled stripes by the bit-level oracle, and every
    # recovery against the encoded stripes (the solution is unique, Lemma 3.1.2)
    p, N, B, S, seed = 17, 16, 65536, 4096, 5
    buf = torch.empty((S, N + 2, B), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(buf, buf.numel(), seed)
    want = buf.cpu().numpy()
    L = rcg.make_hlayout(buf, p, N, B)
    ctx.h_encode(L, 0, S)
    clean(ctx)
    # every byte against the word-level O2 (itself pinned to the bit-level oracle)
    oracle.o2_h_encode(p, N, B, want, S)
    assert np.array_equal(buf.cpu().numpy(), want)
    del want
    sb = (N + 2) * B
    for s in (0, S - 1):
        h = np.ascontiguousarray(inputs.random_bytes(seed, sb, s * sb).reshape(1, N + 2, B))
        oracle.h_encode(p, N, B, h, 1)
        assert np.array_equal(buf[s].cpu().numpy(), h[0]), s
    x = buf[:, 0].clone()
    for k in range(1, N):
        x ^= buf[:, k]
    assert torch.equal(x, buf[:, N])
    del x
    enc = buf.clone()
    idx = torch.arange(S, device="cuda")
    for n, kind in enumerate(("dd", "dp", "dq", "pq")):
        pairs = inputs.random_pairs(3500 + n, N, S, kind)
        pd = dev(pairs)
        buf[idx, pd[:, 0].long()] = POISON_I
        buf[idx, pd[:, 1].long()] = POISON_J
        ctx.h_recover_many(L, 0, S, pd)
        clean(ctx)
        assert torch.equal(buf, enc), kind
        s = 1000 + 77 * n
        lost = enc[s:s + 1].cpu().numpy()
        lost[0, pairs[s, 0]] = POISON_I
        lost[0, pairs[s, 1]] = POISON_J
        oracle.h_recover(p, N, B, lost, 1, int(pairs[s, 0]), int(pairs[s, 1]))
        assert np.array_equal(lost[0], buf[s].cpu().numpy()), (kind, s)
