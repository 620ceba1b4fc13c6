"""Parity of the CUDA path with the CPU oracle for the extended Q-parity of
Section 3.3 (equation qext): up to 2p - 1 data strips, strip k >= p weighted
in Q by 1 + x^(k-p+1), for primes that satisfy Theorem 3.3.3.

Every comparison is bit-exact.  A recovery's expected bytes are the oracle's
(recomputed where cheap) and, by the uniqueness of Lemma 3.1.2 (which holds
here because the weights form a cone, Theorem 3.3.3), the encoded stripe
itself.
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


_ENCODED = {}


def encoded(oracle, seed, p, N, C, S):
    """Seeded stripes encoded by the oracle (computed once per shape; a copy)."""
    key = (seed, p, N, C, S)
    if key not in _ENCODED:
        host = np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, S))
        oracle.encode(p, N, C, host, S)
        _ENCODED[key] = host
    return _ENCODED[key].copy()


def class_pairs(p, N):
    """One erasure pair of every recovery class the extended code has: two
    regular data strips, a regular and an extended one (including the
    degenerate i = 0 and i = j - p + 1, where the trinomial is a monomial),
    two extended ones, regular/extended data + P, data + Q, and P + Q."""
    e0, e1, eN = p, p + 1, N - 1
    pairs = [(1, p - 1), (0, eN), (1, e0), (2, e1 + 1), (3, eN), (e0, eN), (e0, e1), (1, N), (eN, N),
             (p - 1, N + 1), (eN, N + 1), (e0, N + 1), (N, N + 1), (0, 1)]
    return np.array(sorted(set(pairs)), dtype=np.uint8)


def poison(host, pairs):
    lost = host.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    return lost


# ------------------------------------------------------------------- encode

ENCODE_CASES = [
    (5, 6, 1024, 3), (5, 9, 1040, 2), (11, 21, 160, 2), (13, 14, 4096 + 16, 2), (13, 25, 2048, 2),
    (17, 33, 272, 2), (29, 57, 784, 2), (59, 59, 528, 1), (59, 117, 1040, 1), (61, 121, 96, 1),
]


@pytest.mark.parametrize("p,N,C,S", ENCODE_CASES)
def test_qext_encode_matches_oracle(rcg, ctx, oracle, p, N, C, S):
    host = np.ascontiguousarray(inputs.random_stripes(2000 + p + N, p, N, C, S))
    buf = dev(host)
    ctx.encode(rcg.make_layout(buf, p, N, C), 0, S)
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    assert np.array_equal(buf.cpu().numpy(), want)


def test_qext_layouts_beyond_the_limit_are_rejected(rcg, ctx):
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    for p, N in ((5, 10), (7, 8), (3, 4), (31, 32), (13, 26)):
        assert rcg.rcg_prime_info(p)["max_data"] < N
        with pytest.raises(rcg.RcgError):
            ctx.encode(rcg.make_layout(buf, p, N, 16), 0, 1)
    for p, N in ((5, 9), (7, 7), (13, 25)):
        ctx.encode(rcg.make_layout(buf, p, N, 16), 0, 1)
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0


# ------------------------------------------------------------------ recovery

@pytest.mark.parametrize("p,N,C,S", [(5, 9, 1024, 2), (5, 7, 48, 1), (13, 25, 272, 1), (11, 16, 96, 1)])
def test_qext_recover_every_pair(rcg, ctx, oracle, p, N, C, S):
    host = encoded(oracle, 2100 + p + N, p, N, C, S)
    L = None
    for i in range(N + 2):
        for j in range(i + 1, N + 2):
            lost = host.copy()
            lost[:, i] = POISON_I
            lost[:, j] = POISON_J
            buf = dev(lost)
            L = rcg.make_layout(buf, p, N, C)
            for s in range(S):
                ctx.recover(L, s, i, j)
            want = lost.copy()
            oracle.recover(p, N, C, want, S, i, j)
            got = buf.cpu().numpy()
            assert np.array_equal(got, want), (i, j)
            assert np.array_equal(got, host), (i, j)
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0


@pytest.mark.parametrize("p,N,C", [(29, 57, 784), (59, 117, 272), (13, 25, 4096 + 48), (61, 100, 96)])
def test_qext_recover_many_every_class(rcg, ctx, oracle, p, N, C):
    pairs = class_pairs(p, N)
    S = len(pairs)
    host = encoded(oracle, 2200 + p, p, N, C, S)
    lost = poison(host, pairs)
    want = lost.copy()
    oracle.recover(p, N, C, want, S, pairs=pairs)
    assert np.array_equal(want, host)
    buf = dev(lost)
    ctx.recover_many(rcg.make_layout(buf, p, N, C), 0, S, dev(pairs))
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0
    assert np.array_equal(buf.cpu().numpy(), want)


@pytest.mark.parametrize("solve", ["chain", "table"])
@pytest.mark.parametrize("shape", ["wide", "pair"])
@pytest.mark.parametrize("copy", ["tensor", "rows"])
@pytest.mark.parametrize("p,N,C", [(59, 117, 528), (13, 25, 2064)])
def test_qext_recover_every_configuration(rcg, oracle, solve, shape, copy, p, N, C):
    # both two-data solves, both engine shapes and both copy paths give the
    # encoded (= unique, Lemma 3.1.2) stripes back, for every class
    pairs = np.concatenate([class_pairs(p, N), inputs.random_pairs(31, N, 8, "any")])
    S = len(pairs)
    host = encoded(oracle, 2300 + p, p, N, C, S)
    lost = poison(host, pairs)
    with rcg.Context(0) as c:
        c.set_dd_solve(rcg.RCG_SOLVE_CHAIN if solve == "chain" else rcg.RCG_SOLVE_TABLE)
        c.set_engine_shape(rcg.RCG_SHAPE_WIDE if shape == "wide" else rcg.RCG_SHAPE_PAIR)
        c.set_copy_mode(rcg.RCG_COPY_AUTO if copy == "tensor" else rcg.RCG_COPY_ROWS)
        buf = dev(lost)
        L = rcg.make_layout(buf, p, N, C)
        c.recover_many(L, 0, S, dev(pairs))
        assert c.last_device_status() == 0
        assert np.array_equal(buf.cpu().numpy(), host)
        # encode in the same configuration
        buf2 = dev(lost)
        c.encode(rcg.make_layout(buf2, p, N, C), 0, S)
        assert c.last_device_status() == 0
        got = buf2.cpu().numpy()
        assert np.array_equal(got[:, :N], lost[:, :N])
        data_ok = np.array([not (pairs[s] < N).any() for s in range(S)])
        assert np.array_equal(got[data_ok], host[data_ok])


# ------------------------------------------------------ small write, degraded read

@pytest.mark.parametrize("p,N,C", [(5, 9, 1024), (13, 25, 4096), (59, 117, 528)])
def test_qext_update_matches_oracle(rcg, ctx, oracle, p, N, C):
    S = 2
    host = encoded(oracle, 2400 + p, p, N, C, S)
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    want = host.copy()
    for s, i in ((0, p), (1, N - 1), (0, p - 1), (1, 0), (0, N - 1)):
        new = inputs.random_bytes(2500 + s * 131 + i, (p - 1) * C).reshape(p - 1, C)
        ctx.update(L, s, i, dev(new))
        oracle.update(p, N, C, want, s, i, new)
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0
    assert np.array_equal(buf.cpu().numpy(), want)


@pytest.mark.parametrize("p,N,C", [(5, 9, 1024), (29, 57, 784), (59, 117, 528)])
def test_qext_degraded_read_matches_oracle(rcg, ctx, oracle, p, N, C):
    host = encoded(oracle, 2600 + p, p, N, C, 2)
    for j in (0, p - 1, p, N - 1, N, N + 1):
        lost = host.copy()
        lost[1, j] = POISON_I
        buf = dev(lost)
        out = torch.zeros((p - 1, C), dtype=torch.uint8, device="cuda")
        ctx.degraded_read(rcg.make_layout(buf, p, N, C), 1, j, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.degraded_read(p, N, C, lost, 1, j)), j
        assert np.array_equal(out.cpu().numpy(), host[1, j]), j
    assert ctx.last_device_status() == 0


# ------------------------------------------------------------------ batches

def test_qext_batch_mixed_with_regular_jobs(rcg, ctx, oracle):
    # one persistent launch over extended and regular stripes of several p
    specs = [(5, 9, 1024, 3), (13, 25, 2048, 2), (13, 12, 4096, 2), (59, 117, 272, 1), (29, 20, 784, 2)]
    bufs, hosts, jobs, wants = [], [], [], []
    for n, (p, N, C, S) in enumerate(specs):
        host = encoded(oracle, 2700 + n, p, N, C, S)
        raw = np.ascontiguousarray(inputs.random_stripes(2700 + n, p, N, C, S))
        if n % 2 == 0:  # encode job
            buf = dev(raw)
            jobs.append(rcg.make_job(rcg.make_layout(buf, p, N, C), 0, S, rcg.RCG_OP_ENCODE))
        else:           # recover a pair with an extended strip where there is one
            i, j = (0, N - 1)
            lost = host.copy()
            lost[:, i] = POISON_I
            lost[:, j] = POISON_J
            buf = dev(lost)
            jobs.append(rcg.make_job(rcg.make_layout(buf, p, N, C), 0, S, rcg.RCG_OP_RECOVER, i, j))
        bufs.append(buf)
        wants.append(host)
    t = ctx.batch_submit(jobs)
    assert ctx.batch_wait(t)
    assert ctx.last_device_status() == 0
    for buf, want in zip(bufs, wants):
        assert np.array_equal(buf.cpu().numpy(), want)


# ------------------------------------------------------- full-size workload

def class_draw(rng, p, N, S, lo_i, hi_i, lo_j, hi_j):
    out = np.empty((S, 2), dtype=np.uint8)
    for s in range(S):
        while True:
            i, j = int(rng.integers(lo_i, hi_i)), int(rng.integers(lo_j, hi_j))
            if i < j:
                break
        out[s] = (i, j)
    return out


@pytest.mark.slow
def test_qext_full_size_every_class(rcg, ctx, oracle):
    # the extended bench geometry: p=59, N=117, 2 KiB rows, 512 stripes
    # (7.1 GB of user data), seed 6; one launch per class over all stripes
    p, N, C, S, seed = 59, 117, 2048, 512, 6
    sb = inputs.stripe_bytes(p, N, C)
    buf = torch.empty((S, N + 2, p - 1, C), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(buf, S * sb, seed)
    L = rcg.make_layout(buf, p, N, C)
    full = buf.cpu().numpy()
    ctx.encode(L, 0, S)
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0
    oracle.o2_encode(p, N, C, full, S)  # every byte against O2 (word-level CPU)
    assert np.array_equal(buf.cpu().numpy(), full)
    del full
    for s in (0, S - 1):
        host = np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, 1, first_stripe=s))
        oracle.encode(p, N, C, host, 1)
        assert np.array_equal(buf[s].cpu().numpy(), host[0]), s
    x = buf[:, 0].clone()  # property at full size: P is the XOR of the data strips
    for k in range(1, N):
        x ^= buf[:, k]
    assert torch.equal(x, buf[:, N])
    del x
    enc = buf.clone()
    rng = np.random.Generator(np.random.PCG64(62))
    classes = {"dd_regular": (0, p, 0, p), "dd_mixed": (0, p, p, N), "dd_extended": (p, N, p, N),
               "dp_extended": (p, N, N, N + 1), "dq_extended": (p, N, N + 1, N + 2)}
    idx = torch.arange(S, device="cuda")
    for n, (kind, box) in enumerate(classes.items()):
        pairs = class_draw(rng, p, N, S, *box)
        pd = dev(pairs)
        buf[idx, pd[:, 0].long()] = POISON_I
        buf[idx, pd[:, 1].long()] = POISON_J
        lost_all = buf.cpu().numpy()
        ctx.recover_many(L, 0, S, pd)
        torch.cuda.synchronize()
        assert ctx.last_device_status() == 0
        assert torch.equal(buf, enc), kind
        oracle.o2_recover(p, N, C, lost_all, S, pairs=pairs)
        assert np.array_equal(buf.cpu().numpy(), lost_all), kind
        del lost_all
        s = (97 * n + 13) % S
        lost = enc[s:s + 1].cpu().numpy()
        lost[0, pairs[s, 0]] = POISON_I
        lost[0, pairs[s, 1]] = POISON_J
        oracle.recover(p, N, C, lost, 1, int(pairs[s, 0]), int(pairs[s, 1]))
        assert np.array_equal(lost[0], buf[s].cpu().numpy()), (kind, s)


def test_qext_host_memory_calls(rcg, oracle):
    # stripes in pinned host memory, streamed through device staging
    p, N, C, S = 13, 25, 2048, 9
    want = encoded(oracle, 2800, p, N, C, S)
    host = np.ascontiguousarray(inputs.random_stripes(2800, p, N, C, S))
    pinned = torch.from_numpy(host).pin_memory()
    L = rcg.make_layout(pinned, p, N, C)
    with rcg.Context(0) as c:
        c.set_host_chunk(3 * inputs.stripe_bytes(p, N, C))
        c.encode_host(L, 0, S)
        torch.cuda.synchronize()
        assert np.array_equal(pinned.numpy(), want)
        pairs = class_pairs(p, N)[:S]
        for s, (i, j) in enumerate(pairs):
            pinned[s, int(i)] = POISON_I
            pinned[s, int(j)] = POISON_J
        c.recover_many_host(L, 0, S, pairs)
        torch.cuda.synchronize()
        assert c.last_device_status() == 0
        assert np.array_equal(pinned.numpy(), want)
