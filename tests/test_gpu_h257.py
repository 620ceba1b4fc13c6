"""GPU parity of Z_257 (p = 257, 256-bit elements, horizontal representation)
with the CPU oracles: the coefficient-array bit-level oracle on small stripes
(every pair at N = 6, sampled pairs up to N = 257) and the word-level O2 on
the full-size geometry, byte for byte."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

P = 257
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


def h_random(seed, N, B, S):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(S, N + 2, B), dtype=np.uint8)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev16(pairs):
    """16-bit pairs on the device (as int16: the same bytes)."""
    return dev(np.ascontiguousarray(pairs, dtype=np.uint16).view(np.int16))


# (N, strip bytes, stripes): one element, ragged blocks (257 elements: a block
# of 256 and one of 1), the widest array
ENC = [(1, 32, 3), (2, 64, 2), (5, 8224, 2), (16, 1024, 3), (256, 64, 2), (257, 32, 2)]


@pytest.mark.parametrize("N,B,S", ENC)
def test_h257_encode_matches_oracle(rcg, ctx, oracle, N, B, S):
    h = h_random(5700 + N, N, B, S)
    want = h.copy()
    oracle.hbig_encode(P, N, B, want, S)
    buf = dev(h)
    ctx.h_encode(rcg.make_hlayout(buf, P, N, B), 0, S)
    assert ctx.last_device_status() == 0
    assert np.array_equal(buf.cpu().numpy(), want)


def test_h257_every_pair_matches_oracle(rcg, ctx, oracle):
    N, B, S = 6, 64, 2
    h = h_random(5800, N, B, S)
    oracle.hbig_encode(P, N, B, h, S)
    for i in range(N + 2):
        for j in range(i + 1, N + 2):
            lost = h.copy()
            lost[:, i] = POISON_I
            lost[:, j] = POISON_J
            want = lost.copy()
            oracle.hbig_recover(P, N, B, want, S, i, j)
            buf = dev(lost)
            L = rcg.make_hlayout(buf, P, N, B)
            for s in range(S):
                ctx.h_recover(L, s, i, j)
            assert np.array_equal(buf.cpu().numpy(), want), (i, j)
            assert np.array_equal(want, h), (i, j)
    assert ctx.last_device_status() == 0


@pytest.mark.parametrize("N", [17, 257])
def test_h257_wide_pairs_match_oracle(rcg, ctx, oracle, N):
    B, S = 64, 1
    h = h_random(5900 + N, N, B, S)
    oracle.hbig_encode(P, N, B, h, S)
    rng = np.random.default_rng(N)
    pairs = [(0, 1), (0, N - 1), (N - 2, N - 1), (1, N), (N - 1, N + 1), (N, N + 1)]
    pairs += [tuple(sorted(rng.choice(N + 2, 2, replace=False).tolist())) for _ in range(4)]
    for i, j in pairs:
        lost = h.copy()
        lost[:, i] = POISON_I
        lost[:, j] = POISON_J
        buf = dev(lost)
        ctx.h_recover(rcg.make_hlayout(buf, P, N, B), 0, i, j)
        assert np.array_equal(buf.cpu().numpy(), h), (i, j)
    assert ctx.last_device_status() == 0


def test_h257_recover_many_16bit_pairs_and_strides(rcg, ctx, oracle):
    N, B, S = 257, 96, 5
    ss, st = 128, 128 * (N + 2) + 64
    rng = np.random.default_rng(6000)
    flat = rng.integers(0, 256, size=st * S, dtype=np.uint8)
    oracle.o2_h257_encode(N, B, flat, S, ss, st)
    pairs = np.array([[256, 258], [3, 257], [0, 256], [257, 258], [10, 200]], dtype=np.uint16)
    lost = flat.copy()
    for s, (i, j) in enumerate(pairs.tolist()):
        for k in (i, j):
            lost[s * st + k * ss: s * st + k * ss + B] = POISON_I
    want = lost.copy()
    oracle.hbig_recover(P, N, B, want, S, pairs=pairs, strip_stride=ss, stripe_stride=st)
    assert np.array_equal(want, flat)
    buf = dev(lost)
    ctx.h_recover_many(rcg.make_hlayout(buf, P, N, B, ss, st), 0, S, dev16(pairs))
    assert ctx.last_device_status() == 0
    assert np.array_equal(buf.cpu().numpy(), want)  # the padding is untouched too


def test_h257_bad_pairs_and_arguments(rcg, ctx, oracle):
    N, B, S = 4, 32, 3
    h = h_random(6100, N, B, S)
    oracle.hbig_encode(P, N, B, h, S)
    buf = dev(h)
    L = rcg.make_hlayout(buf, P, N, B)
    ctx.h_recover_many(L, 0, S, dev16([[1, 1], [0, 9], [0, 1]]))
    torch.cuda.synchronize()
    assert ctx.last_device_status() == rcg.RCG_DEV_BADPAIR
    assert np.array_equal(buf.cpu().numpy(), h)  # every stripe intact (the valid pair rebuilt itself)
    for bad in [rcg.make_hlayout(buf, P, N, 48),        # not whole elements
                rcg.make_hlayout(buf, P, 258, B),       # beyond the base code
                rcg.make_hlayout(buf, P, N, B, 48)]:    # stride not a multiple of 32
        with pytest.raises(rcg.RcgError):
            ctx.h_encode(bad, 0, 1)
    with pytest.raises(rcg.RcgError):
        ctx.h_recover(L, 0, 2, 2)
    pairs = torch.zeros(2 * S + 1, dtype=torch.int16, device="cuda")
    with pytest.raises(rcg.RcgError):  # 16-bit pairs must be 4-byte aligned
        ctx.h_recover_many(L, 0, S, pairs[1:].data_ptr())


H257_FULL = (256, 65536, 256)  # N, strip bytes, stripes: the bench geometry (4.3 GB of data)


def test_h257_full_size_matches_o2(rcg, ctx, oracle):
    from paper_cs_0611109_gb300 import inputs
    N, B, S = H257_FULL
    buf = torch.empty((S, N + 2, B), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(buf, buf.numel(), 7)
    host = buf.cpu().numpy()
    ctx.h_encode(rcg.make_hlayout(buf, P, N, B), 0, S)
    oracle.o2_h257_encode(N, B, host, S)
    assert ctx.last_device_status() == 0
    assert np.array_equal(buf.cpu().numpy(), host)
    # per-stripe pairs of every class, drawn from a seed
    rng = np.random.default_rng(7)
    pairs = np.array([sorted(rng.choice(N + 2, 2, replace=False).tolist()) for _ in range(S)], dtype=np.uint16)
    lost = host.copy()
    for s, (i, j) in enumerate(pairs.tolist()):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    buf.copy_(dev(lost))
    ctx.h_recover_many(rcg.make_hlayout(buf, P, N, B), 0, S, dev16(pairs))
    oracle.o2_h257_recover(N, B, lost, S, pairs=pairs)
    assert ctx.last_device_status() == 0
    got = buf.cpu().numpy()
    assert np.array_equal(got, lost)
    assert np.array_equal(got, host)
    # and one stripe against the bit-level oracle, for one element of each strip
    s = 3
    one = np.ascontiguousarray(inputs.random_bytes(7, (N + 2) * B, s * (N + 2) * B).reshape(N + 2, B)[:, :32][None])
    oracle.hbig_encode(P, N, 32, one, 1)
    assert np.array_equal(got[s, :, :32], one[0])
