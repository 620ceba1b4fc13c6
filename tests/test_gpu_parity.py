"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is bit-exact: the code is XOR over GF(2), so there is no
floating-point tolerance, and Lemma 3.1.2 makes every recovery unique.
Small cases compare whole buffers with the oracle; the full-size workloads
compare oracle-sampled stripes plus properties that hold at any size.
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


def host_stripes(seed, p, N, C, S):
    return np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, S))


def check_clean(ctx):
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0


# ------------------------------------------------------------ generator twin

@pytest.mark.parametrize("nbytes,offset", [(16, 0), (1000, 0), (4096 + 7, 8), (1 << 20, 1 << 16), (33, 24)])
def test_fill_random_matches_host_generator(rcg, nbytes, offset):
    buf = torch.zeros(nbytes + 32, dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(buf, nbytes, 3, offset)
    torch.cuda.synchronize()
    got = buf.cpu().numpy()
    assert np.array_equal(got[:nbytes], inputs.random_bytes(3, nbytes, offset))
    assert not got[nbytes:].any()


# ------------------------------------------------------------------- encode

ENCODE_CASES = [
    (3, 1, 16, 3), (3, 2, 48, 5), (3, 3, 16, 2), (5, 4, 1024, 9), (5, 5, 32, 4), (7, 6, 1040, 3),
    (11, 10, 160, 3), (13, 12, 4096, 3), (13, 1, 64, 2), (17, 17, 2048 + 16, 2), (29, 28, 512, 2),
    (29, 5, 3008, 2), (59, 58, 2048, 1), (59, 2, 272, 2), (61, 61, 96, 1), (61, 60, 1024, 1),
]


@pytest.mark.parametrize("p,N,C,S", ENCODE_CASES)
def test_encode_matches_oracle(rcg, ctx, oracle, p, N, C, S):
    host = host_stripes(100 + p, p, N, C, S)
    buf = dev(host)
    ctx.encode(rcg.make_layout(buf, p, N, C), 0, S)
    check_clean(ctx)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    assert np.array_equal(buf.cpu().numpy(), want)


def test_encode_subrange_and_strides(rcg, ctx, oracle):
    # non-packed layout, first_stripe offset: untouched stripes and padding stay as they were
    p, N, C, S = 7, 5, 96, 6
    rs, ss = 128, 128 * (p - 1) + 32
    st = ss * (N + 2) + 64
    flat = inputs.random_bytes(5, st * S)
    buf = dev(flat)
    ctx.encode(rcg.make_layout(buf, p, N, C, rs, ss, st), 2, 3)
    check_clean(ctx)
    want = flat.copy()
    oracle.encode(p, N, C, want[2 * st:], 3, rs, ss, st)
    assert np.array_equal(buf.cpu().numpy(), want)


def test_zero_stripes_is_noop(rcg, ctx):
    buf = torch.zeros(6 * 4 * 16, dtype=torch.uint8, device="cuda")
    ctx.encode(rcg.make_layout(buf, 5, 4, 16), 0, 0)
    check_clean(ctx)
    assert not buf.any()


# ------------------------------------------------------------------ recovery

def all_pairs(N):
    return [(i, j) for i in range(N + 2) for j in range(i + 1, N + 2)]


@pytest.mark.parametrize("p,N,C,S", [(5, 4, 1024, 6), (7, 5, 48, 3), (3, 3, 16, 2), (13, 12, 1040, 1), (17, 16, 256, 1)])
def test_recover_every_pair_matches_oracle(rcg, ctx, oracle, p, N, C, S):
    host = host_stripes(200 + p, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    for (i, j) in all_pairs(N):
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
    check_clean(ctx)


@pytest.mark.parametrize("kind", ["dd", "dp", "dq", "pq", "any"])
@pytest.mark.parametrize("p,N,C,S", [(13, 12, 4096, 8), (59, 58, 2048, 2), (29, 20, 784, 5)])
def test_recover_many_per_stripe_pairs(rcg, ctx, oracle, kind, p, N, C, S):
    host = host_stripes(300 + p, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    pairs = inputs.random_pairs(7, N, S, kind)
    lost = host.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    buf = dev(lost)
    ctx.recover_many(rcg.make_layout(buf, p, N, C), 0, S, dev(pairs))
    check_clean(ctx)
    want = lost.copy()
    oracle.recover(p, N, C, want, S, pairs=pairs)
    got = buf.cpu().numpy()
    assert np.array_equal(got, want)
    assert np.array_equal(got, host)


@pytest.mark.parametrize("p,N,C,S", [(13, 12, 4096, 4), (59, 58, 528, 2), (3, 3, 16, 2), (61, 61, 96, 2), (5, 4, 1024, 3)])
def test_two_data_solves_agree(rcg, oracle, p, N, C, S):
    # the chain solve and the Section 4.6 table solve give the oracle's bytes
    host = host_stripes(330 + p, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    pairs = inputs.random_pairs(8, N, S, "dd")
    lost = host.copy()
    for s, (i, j) in enumerate(pairs):
        lost[s, i] = POISON_I
        lost[s, j] = POISON_J
    want = lost.copy()
    oracle.recover(p, N, C, want, S, pairs=pairs)
    assert np.array_equal(want, host)
    for solve in (rcg.RCG_SOLVE_CHAIN, rcg.RCG_SOLVE_TABLE):
        with rcg.Context(0) as c:
            c.set_dd_solve(solve)
            buf = dev(lost)
            c.recover_many(rcg.make_layout(buf, p, N, C), 0, S, dev(pairs))
            assert c.last_device_status() == 0
            assert np.array_equal(buf.cpu().numpy(), want), solve


def test_recover_many_rejects_bad_pairs_on_device(rcg, ctx, oracle):
    p, N, C, S = 5, 4, 64, 4
    host = host_stripes(9, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    pairs = np.array([[0, 1], [2, 2], [3, 7], [4, 5]], dtype=np.uint8)  # stripes 1, 2 invalid
    lost = host.copy()
    lost[0, 0:2] = POISON_I
    lost[3, 4:6] = POISON_I
    buf = dev(lost)
    ctx.recover_many(rcg.make_layout(buf, p, N, C), 0, S, dev(pairs))
    torch.cuda.synchronize()
    assert ctx.last_device_status() == rcg.RCG_DEV_BADPAIR
    got = buf.cpu().numpy()
    assert np.array_equal(got[[0, 3]], host[[0, 3]])
    assert np.array_equal(got[[1, 2]], lost[[1, 2]])  # invalid stripes untouched


def test_host_validation(rcg, ctx):
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(rcg.RcgError):
        ctx.encode(rcg.make_layout(buf, 9, 4, 16), 0, 1)  # 9 is not prime
    with pytest.raises(rcg.RcgError):
        ctx.encode(rcg.make_layout(buf, 7, 8, 16), 0, 1)  # N > p, and 7 fails Theorem 3.3.3
    with pytest.raises(rcg.RcgError):
        ctx.encode(rcg.make_layout(buf, 5, 4, 24), 0, 1)  # C not a multiple of 16
    with pytest.raises(rcg.RcgError):
        ctx.encode(rcg.make_layout(buf[1:], 5, 4, 16), 0, 1)  # misaligned base
    with pytest.raises(rcg.RcgError):
        ctx.recover(rcg.make_layout(buf, 5, 4, 16), 0, 3, 3)
    with pytest.raises(rcg.RcgError):
        ctx.recover(rcg.make_layout(buf, 5, 4, 16), 0, 2, 6)
    check_clean(ctx)


# ------------------------------------------------------ small write, degraded read

@pytest.mark.parametrize("p,N,C", [(5, 4, 1024), (13, 12, 4096), (59, 58, 528), (3, 1, 16)])
def test_update_matches_oracle(rcg, ctx, oracle, p, N, C):
    S = 3
    host = host_stripes(400 + p, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    want = host.copy()
    for s, i in ((0, 0), (1, N - 1), (2, N // 2), (1, 0)):
        new = inputs.random_bytes(500 + s * 7 + i, (p - 1) * C).reshape(p - 1, C)
        ctx.update(L, s, i, dev(new))
        oracle.update(p, N, C, want, s, i, new)
    check_clean(ctx)
    assert np.array_equal(buf.cpu().numpy(), want)


@pytest.mark.parametrize("p,N,C", [(5, 4, 1024), (13, 12, 4096), (59, 58, 528)])
def test_degraded_read_matches_oracle(rcg, ctx, oracle, p, N, C):
    S = 2
    host = host_stripes(600 + p, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    lostall = host.copy()
    for j in list(range(0, N, max(1, N // 4))) + [N, N + 1]:
        lost = host.copy()
        lost[1, j] = POISON_I
        buf = dev(lost)
        out = torch.zeros((p - 1, C), dtype=torch.uint8, device="cuda")
        ctx.degraded_read(rcg.make_layout(buf, p, N, C), 1, j, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.degraded_read(p, N, C, lost, 1, j)), j
        assert np.array_equal(out.cpu().numpy(), host[1, j]), j
        assert np.array_equal(buf.cpu().numpy(), lost)  # the stripe is not modified
    check_clean(ctx)


@pytest.mark.parametrize("p,N,C,S", [(59, 58, 528, 2), (13, 12, 4096 + 48, 2), (5, 4, 1024, 3)])
def test_row_copy_path_matches_oracle(rcg, oracle, p, N, C, S):
    # the per-row bulk-copy path (used where the driver refuses a tensor map)
    host = host_stripes(950 + p, p, N, C, S)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    with rcg.Context(0) as c:
        c.set_copy_mode(rcg.RCG_COPY_ROWS)
        buf = dev(host)
        L = rcg.make_layout(buf, p, N, C)
        c.encode(L, 0, S)
        torch.cuda.synchronize()
        assert np.array_equal(buf.cpu().numpy(), want)
        pairs = inputs.random_pairs(3, N, S, "any")
        buf[0, pairs[0, 0]] = POISON_I
        c.recover_many(L, 0, S, dev(pairs))
        new = inputs.random_bytes(77, (p - 1) * C).reshape(p - 1, C)
        c.update(L, S - 1, N - 1, dev(new))
        oracle.update(p, N, C, want, S - 1, N - 1, new)
        assert c.last_device_status() == 0
        assert np.array_equal(buf.cpu().numpy(), want)


# ------------------------------------------------------- host-memory stripes

@pytest.mark.parametrize("p,N,C,S,chunk", [(13, 12, 4096, 70, 1 << 28), (13, 12, 4096, 70, 3 << 20),
                                              (5, 4, 1024, 33, 50000), (59, 58, 528, 5, 4096)])
def test_host_memory_calls_match_oracle(rcg, oracle, p, N, C, S, chunk):
    # chunk sizes that give one chunk, several chunks over three streams, and one stripe per chunk
    host = host_stripes(1100 + p, p, N, C, S)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    pinned = torch.from_numpy(host.copy()).pin_memory()
    L = rcg.make_layout(pinned, p, N, C)
    ctx = rcg.Context(0)
    ctx.set_host_chunk(chunk)
    ctx.encode_host(L, 0, S)
    torch.cuda.synchronize()
    assert np.array_equal(pinned.numpy(), want)
    pairs = inputs.random_pairs(9, N, S, "any")
    for s, (i, j) in enumerate(pairs):
        pinned[s, int(i)] = POISON_I
        pinned[s, int(j)] = POISON_J
    ctx.recover_many_host(L, 0, S, pairs)
    torch.cuda.synchronize()
    assert ctx.last_device_status() == 0
    assert np.array_equal(pinned.numpy(), want)
    ctx.close()


def test_host_memory_calls_need_pinned_memory(rcg, ctx):
    pageable = torch.zeros((2, 6, 4, 16), dtype=torch.uint8)
    with pytest.raises(rcg.RcgError):
        ctx.encode_host(rcg.make_layout(pageable, 5, 4, 16), 0, 2)


# ------------------------------------------------------- failure detection

def test_bounded_wait_runs_out_and_reports(rcg, oracle):
    # a wait that nothing completes: the kernel gives up after 20 ms, records
    # RCG_DEV_TIMEOUT and returns; the context keeps working afterwards
    import time
    with rcg.Context(0) as c:
        t0 = time.perf_counter()
        rcg.rcg_selftest_wait_timeout(c.handle, 20 * 10 ** 6)
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        assert c.last_device_status() == rcg.RCG_DEV_TIMEOUT
        assert 0.015 < elapsed < 5.0
        assert c.last_device_status() == 0  # reading cleared it
        host = host_stripes(77, 5, 4, 64, 2)
        want = host.copy()
        oracle.encode(5, 4, 64, want, 2)
        buf = dev(host)
        c.encode(rcg.make_layout(buf, 5, 4, 64), 0, 2)
        assert c.last_device_status() == 0
        assert np.array_equal(buf.cpu().numpy(), want)


def test_batch_wait_times_out_on_the_host(rcg):
    # the host-side wait is bounded too: a zero-ish limit on a running batch
    # returns RCG_ETIMEOUT (False) while the batch keeps going
    p, N, C, S = 59, 58, 2048, 64
    buf = torch.empty((S, N + 2, p - 1, C), dtype=torch.uint8, device="cuda")
    with rcg.Context(0) as c:
        L = rcg.make_layout(buf, p, N, C)
        rcg.rcg_selftest_wait_timeout(c.handle, 50 * 10 ** 6)  # keeps the stream busy ~50 ms
        t = c.batch_submit([rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE)])
        assert c.batch_wait(t, 1000) is False
        assert c.batch_wait(t, 10 ** 10) is True
        assert c.last_device_status() == rcg.RCG_DEV_TIMEOUT  # from the probe only


# ------------------------------------------------------------------ batches

def test_batch_mixed_jobs_alone_and_in_the_mix(rcg, ctx, oracle):
    # every job of a mixed batch gives the same bytes as the oracle (and as
    # the single-op calls) -- alone vs in the mix, tolerance 0
    specs = [(5, 4, 1024, 3, "enc"), (13, 12, 4096, 2, "rec"), (29, 7, 528, 2, "deg"),
             (59, 58, 2048, 1, "rec"), (3, 2, 16, 4, "enc"), (13, 6, 1040, 2, "upd"),
             (61, 60, 64, 1, "rec")]
    bufs, jobs, wants, outs = [], [], [], []
    for n, (p, N, C, S, kind) in enumerate(specs):
        host = host_stripes(700 + n, p, N, C, S)
        if kind != "enc":
            oracle.encode(p, N, C, host, S)
        want = host.copy()
        buf = dev(host)
        L = rcg.make_layout(buf, p, N, C)
        if kind == "enc":
            oracle.encode(p, N, C, want, S)
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE))
        elif kind == "rec":
            i, j = (1, N - 1) if N > 2 else (0, N)
            buf[:, i] = POISON_I
            buf[:, j] = POISON_J
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_RECOVER, i, j))
        elif kind == "deg":
            out = torch.zeros((S, p - 1, C), dtype=torch.uint8, device="cuda")
            outs.append((out, host[:, 3].copy()))
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, 3, out))
        elif kind == "upd":
            new = inputs.random_bytes(800, S * (p - 1) * C).reshape(S, p - 1, C)
            newd = dev(new)
            outs.append((newd, None))
            for s in range(S):
                oracle.update(p, N, C, want, s, 2, new[s])
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_UPDATE, 2, 0, newd))
        bufs.append(buf)
        wants.append(want)
    ticket = ctx.batch_submit(jobs)
    assert ctx.batch_wait(ticket)
    check_clean(ctx)
    for buf, want in zip(bufs, wants):
        assert np.array_equal(buf.cpu().numpy(), want)
    for out, want in outs:
        if want is not None:
            assert np.array_equal(out.cpu().numpy(), want)


def test_batched_uneven_jobs_alone_and_in_the_mix(rcg, ctx, oracle):
    # the uneven batched workload's distributions (row bytes capped so the test
    # stays small): every stripe of the one-launch batch equals the same stripe
    # run alone (one launch per stripe), and sampled stripes equal the oracle
    jobs = inputs.batched_jobs(17, 400, c_min=512, c_max=4096)
    sizes = [inputs.stripe_bytes(j["p"], j["n"], j["c"]) for j in jobs]
    offs = np.cumsum([0] + [(b + 255) // 256 * 256 for b in sizes])
    arena = torch.empty(int(offs[-1]), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(arena, arena.numel(), 21)
    lays = [rcg.make_layout(arena.data_ptr() + int(o), j["p"], j["n"], j["c"]) for o, j in zip(offs, jobs)]
    # recover jobs run on encoded stripes
    t = ctx.batch_submit([rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE) for L, j in zip(lays, jobs) if j["op"] == "recover"])
    assert ctx.batch_wait(t)
    start = arena.clone()
    mix = [rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE) if j["op"] == "encode" else
           rcg.make_job(L, 0, 1, rcg.RCG_OP_RECOVER, j["i"], j["j"]) for L, j in zip(lays, jobs)]
    for L, j in zip(lays, jobs):   # poison the erased strips of the recover jobs
        if j["op"] == "recover":
            sb = (j["p"] - 1) * j["c"]
            for k in (j["i"], j["j"]):
                arena[L.base - arena.data_ptr() + k * sb: L.base - arena.data_ptr() + (k + 1) * sb] = POISON_I
    poisoned = arena.clone()
    t = ctx.batch_submit(mix)
    assert ctx.batch_wait(t)
    check_clean(ctx)
    in_mix = arena.clone()
    arena.copy_(poisoned)
    for L, j in zip(lays, jobs):   # alone: one launch per stripe
        if j["op"] == "encode":
            ctx.encode(L, 0, 1)
        else:
            ctx.recover(L, 0, j["i"], j["j"])
    check_clean(ctx)
    assert torch.equal(arena, in_mix)
    got = in_mix.cpu().numpy()
    ref = start.cpu().numpy()
    for k in list(range(0, len(jobs), 37)):
        j, o, b = jobs[k], int(offs[k]), sizes[k]
        want = ref[o:o + b].copy()
        if j["op"] == "encode":
            want = np.ascontiguousarray(poisoned[o:o + b].cpu().numpy())
            oracle.encode(j["p"], j["n"], j["c"], want, 1)
        assert np.array_equal(got[o:o + b], want), k


def test_prepared_batch_launches_repeatedly(rcg, ctx, oracle):
    p, N, C, S = 13, 12, 1024, 6
    host = host_stripes(950, p, N, C, S)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    b = ctx.batch_prepare([rcg.make_job(L, s, 1, rcg.RCG_OP_ENCODE) for s in range(S)])
    for _ in range(3):
        buf.copy_(dev(host))
        assert ctx.batch_wait(ctx.batch_launch(b))
        assert np.array_equal(buf.cpu().numpy(), want)
    rcg.rcg_batch_free(b)
    check_clean(ctx)


def test_batch_many_small_jobs_replays_graph(rcg, ctx, oracle):
    p, N, C, S = 13, 5, 64, 40
    host = host_stripes(900, p, N, C, S)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    for rep in range(3):  # reuse of the captured graph with different table sizes
        buf = dev(host)
        L = rcg.make_layout(buf, p, N, C)
        jobs = [rcg.make_job(L, s, 1, rcg.RCG_OP_ENCODE) for s in range(S - rep * 7)]
        t = ctx.batch_submit(jobs)
        assert ctx.batch_wait(t)
        got = buf.cpu().numpy()
        n = S - rep * 7
        assert np.array_equal(got[:n], want[:n])
        assert np.array_equal(got[n:], host[n:])
    check_clean(ctx)


# ---------------------------------------------------------- full-size workloads

def sample_check(oracle, buf, p, N, C, seed, stripes, pairs=None):
    """Compare sampled stripes of a device buffer with the oracle run on the
    regenerated input of those stripes."""
    for s in stripes:
        host = np.ascontiguousarray(inputs.random_stripes(seed, p, N, C, 1, first_stripe=s))
        oracle.encode(p, N, C, host, 1)
        got = buf[s].cpu().numpy()
        assert np.array_equal(got, host[0]), s


@pytest.mark.slow
def test_p5n4_full_encode_and_every_pair(rcg, ctx, oracle):
    # p=5, N=4, 1 KiB rows, 1024 stripes, seed 0; all 15 erasure pairs
    p, N, C, S = 5, 4, 1024, 1024
    host = host_stripes(0, p, N, C, S)
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    ctx.encode(L, 0, S)
    check_clean(ctx)
    assert np.array_equal(buf.cpu().numpy(), want)
    enc = buf.clone()
    sub = 64  # the oracle's own recovery on the first 64 stripes of every pair
    for (i, j) in all_pairs(N):
        buf.copy_(enc)
        buf[:, i] = POISON_I
        buf[:, j] = POISON_J
        lost = buf[:sub].cpu().numpy()
        pairs = torch.tensor([[i, j]] * S, dtype=torch.uint8, device="cuda")
        ctx.recover_many(L, 0, S, pairs)
        check_clean(ctx)
        got = buf.cpu().numpy()
        assert np.array_equal(got, want), (i, j)
        oracle.recover(p, N, C, lost, sub, i, j)
        assert np.array_equal(got[:sub], lost), (i, j)


@pytest.mark.slow
def test_p13n12_full_size(rcg, ctx, oracle):
    # p=13, N=12, 4 KiB rows, 8192 stripes (~4.5 GiB user data), seed 1
    p, N, C, S, seed = 13, 12, 4096, 8192, 1
    sb = inputs.stripe_bytes(p, N, C)
    buf = torch.empty((S, N + 2, p - 1, C), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(buf, S * sb, seed)
    L = rcg.make_layout(buf, p, N, C)
    full = buf.cpu().numpy()  # every byte, checked below against O2 (word-level CPU)
    ctx.encode(L, 0, S)
    check_clean(ctx)
    samples = [0, 1, 4095, 5000, S - 1]
    sample_check(oracle, buf, p, N, C, seed, samples)
    oracle.o2_encode(p, N, C, full, S)
    assert np.array_equal(buf.cpu().numpy(), full)
    # property at full size: P is the XOR of the data strips
    x = buf[:, 0].clone()
    for k in range(1, N):
        x ^= buf[:, k]
    assert torch.equal(x, buf[:, N])
    del x
    enc = buf.clone()
    for kind in ("dd", "dp", "dq", "pq"):
        pairs = inputs.random_pairs(11, N, S, kind)
        pd = dev(pairs)
        idx = torch.arange(S, device="cuda")
        buf[idx, pd[:, 0].long()] = POISON_I
        buf[idx, pd[:, 1].long()] = POISON_J
        lost_all = buf.cpu().numpy()
        ctx.recover_many(L, 0, S, pd)
        check_clean(ctx)
        assert torch.equal(buf, enc), kind
        oracle.o2_recover(p, N, C, lost_all, S, pairs=pairs)  # every byte, on the same input
        assert np.array_equal(buf.cpu().numpy(), lost_all), kind
        del lost_all
        for s in samples[:3]:
            lost = enc[s:s + 1].cpu().numpy()
            lost[0, pairs[s, 0]] = POISON_I
            lost[0, pairs[s, 1]] = POISON_J
            oracle.recover(p, N, C, lost, 1, int(pairs[s, 0]), int(pairs[s, 1]))
            assert np.array_equal(lost[0], buf[s].cpu().numpy()), (kind, s)


@pytest.mark.slow
def test_p59n58_full_size_double_data(rcg, ctx, oracle):
    # p=59, N=58, 2 KiB rows, 1024 stripes (~7 GiB), uniformly random data pairs
    p, N, C, S, seed = 59, 58, 2048, 1024, 2
    sb = inputs.stripe_bytes(p, N, C)
    buf = torch.empty((S, N + 2, p - 1, C), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(buf, S * sb, seed)
    L = rcg.make_layout(buf, p, N, C)
    full = buf.cpu().numpy()
    ctx.encode(L, 0, S)
    check_clean(ctx)
    sample_check(oracle, buf, p, N, C, seed, [0, S - 1])
    oracle.o2_encode(p, N, C, full, S)  # every byte against O2
    assert np.array_equal(buf.cpu().numpy(), full)
    del full
    enc = buf.clone()
    pairs = inputs.random_pairs(12, N, S, "dd")
    pd = dev(pairs)
    idx = torch.arange(S, device="cuda")
    buf[idx, pd[:, 0].long()] = POISON_I
    buf[idx, pd[:, 1].long()] = POISON_J
    lost_all = buf.cpu().numpy()
    ctx.recover_many(L, 0, S, pd)
    check_clean(ctx)
    assert torch.equal(buf, enc)
    oracle.o2_recover(p, N, C, lost_all, S, pairs=pairs)
    assert np.array_equal(buf.cpu().numpy(), lost_all)
    del lost_all
    s = 517
    lost = enc[s:s + 1].cpu().numpy()
    lost[0, pairs[s, 0]] = POISON_I
    lost[0, pairs[s, 1]] = POISON_J
    oracle.recover(p, N, C, lost, 1, int(pairs[s, 0]), int(pairs[s, 1]))
    assert np.array_equal(lost[0], buf[s].cpu().numpy())


@pytest.mark.slow
def test_p13n12_degraded_read_and_small_write(rcg, ctx, oracle):
    # the launches bench.py --workload p13n12_ops times: one batch job over 8192
    # stripes each; every rebuilt byte is checked, sampled stripes by the oracle
    p, N, C, S, seed = 13, 12, 4096, 8192, 1
    buf = torch.empty((S, N + 2, p - 1, C), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(buf, buf.numel(), seed)
    L = rcg.make_layout(buf, p, N, C)
    ctx.encode(L, 0, S)
    aux = torch.zeros((S, p - 1, C), dtype=torch.uint8, device="cuda")
    for j in (3, N, N + 1):
        assert ctx.batch_wait(ctx.batch_submit([rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, j, aux)]))
        check_clean(ctx)
        assert torch.equal(aux, buf[:, j]), j
    new = torch.empty_like(aux)
    rcg.rcg_fill_random(new, new.numel(), seed + 7)
    before = buf[[0, S - 1]].cpu().numpy()
    assert ctx.batch_wait(ctx.batch_submit([rcg.make_job(L, 0, S, rcg.RCG_OP_UPDATE, 5, 0, new)]))
    check_clean(ctx)
    assert torch.equal(buf[:, 5], new)
    x = buf[:, 0].clone()
    for k in range(1, N):
        x ^= buf[:, k]
    assert torch.equal(x, buf[:, N])  # P is the XOR of the (new) data everywhere
    del x
    for n, s in enumerate((0, S - 1)):
        want = np.ascontiguousarray(before[n:n + 1])
        oracle.update(p, N, C, want, 0, 5, new[s].cpu().numpy())
        assert np.array_equal(buf[s].cpu().numpy(), want[0]), s
    # every byte: P and Q after the small write equal O2's encode of the new data
    host = buf.cpu().numpy()
    full = host.copy()
    oracle.o2_encode(p, N, C, full, S)
    assert np.array_equal(host, full)
