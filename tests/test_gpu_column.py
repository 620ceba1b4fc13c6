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


# ------------------------------------------------ degraded read, small write

@pytest.mark.parametrize("p,N,C,S", [(3, 3, 48, 2), (5, 4, 1024, 2), (5, 9, 256, 2), (7, 6, 1040, 2)])
def test_column_degraded_read_every_strip(rcg, ctxs, oracle, p, N, C, S):
    col, eng = ctxs
    host = stripes(4500 + p + N, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    for j in range(N + 2):
        for s in range(S):
            want = oracle.degraded_read(p, N, C, host, s, j)
            assert np.array_equal(want, host[s, j])  # a codeword: the strip itself
            for c in (col, eng):
                out = torch.zeros((p - 1, C), dtype=torch.uint8, device="cuda")
                c.degraded_read(L, s, j, out)
                assert c.last_device_status() == 0
                assert np.array_equal(out.cpu().numpy(), want), (j, s)
    assert np.array_equal(buf.cpu().numpy(), host)  # the stripe is not touched


@pytest.mark.parametrize("p,N,C", [(3, 2, 32), (5, 4, 1024), (5, 9, 64), (7, 7, 528)])
def test_column_small_write_matches_oracle(rcg, ctxs, oracle, p, N, C):
    col, _ = ctxs
    S = 3
    host = stripes(4600 + p + N, p, N, C, S)
    oracle.encode(p, N, C, host, S)
    want = host.copy()
    buf = dev(host)
    L = rcg.make_layout(buf, p, N, C)
    for s, i in enumerate([0, N - 1, N // 2]):
        new = inputs.random_bytes(4601 + s, (p - 1) * C).reshape(p - 1, C)
        oracle.update(p, N, C, want, s, i, new)
        col.update(L, s, i, dev(new))
    assert col.last_device_status() == 0
    assert np.array_equal(buf.cpu().numpy(), want)


# ------------------------------------------------------------ batches

def mixed_batch(rcg, oracle, seed, specs):
    """Jobs of every op on separate buffers (codewords for all but encode);
    returns (device buffers, jobs, outputs, expected buffers, expected outputs)."""
    bufs, jobs, outs, want_bufs, want_outs = [], [], [], [], []
    for n, (p, N, C, S, kind) in enumerate(specs):
        host = stripes(seed + n, p, N, C, S)
        if kind != "enc":
            oracle.encode(p, N, C, host, S)
        want = host.copy()
        aux = None
        if kind == "enc":
            oracle.encode(p, N, C, want, S)
            job = lambda L: rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE)
        elif kind.startswith("rec"):
            i, j = {"rec_dd": (0, N - 1), "rec_dp": (N - 1, N), "rec_dq": (0, N + 1), "rec_pq": (N, N + 1)}[kind]
            host[:, i] = POISON_I
            host[:, j] = POISON_J
            job = lambda L, i=i, j=j: rcg.make_job(L, 0, S, rcg.RCG_OP_RECOVER, i, j)
        elif kind.startswith("deg"):
            jj = {"deg_d": N // 2, "deg_p": N, "deg_q": N + 1}[kind]
            aux = torch.zeros((S, p - 1, C), dtype=torch.uint8, device="cuda")
            want_outs.append(np.stack([oracle.degraded_read(p, N, C, want, s, jj) for s in range(S)]))
            job = lambda L, jj=jj, aux=aux: rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, jj, aux)
        else:  # small write of strip N - 1
            new = inputs.random_bytes(seed + 500 + n, S * (p - 1) * C).reshape(S, p - 1, C)
            for s in range(S):
                oracle.update(p, N, C, want, s, N - 1, new[s])
            aux = dev(new)
            want_outs.append(new)
            job = lambda L, aux=aux: rcg.make_job(L, 0, S, rcg.RCG_OP_UPDATE, N - 1, 0, aux)
        buf = dev(host)
        jobs.append(job(rcg.make_layout(buf, p, N, C)))
        bufs.append(buf)
        if aux is not None:
            outs.append(aux)
        want_bufs.append(want)
    return bufs, jobs, outs, want_bufs, want_outs


SMALL = [(3, 2, 32, 3, "enc"), (3, 3, 1040, 2, "rec_dd"), (5, 4, 1024, 40, "enc"), (5, 4, 1024, 7, "rec_dd"),
         (5, 4, 512, 3, "rec_dp"), (5, 3, 2048, 2, "rec_dq"), (5, 4, 64, 5, "rec_pq"), (5, 9, 256, 3, "rec_dd"),
         (5, 8, 96, 2, "deg_d"), (5, 4, 1040, 2, "deg_q"), (7, 6, 4096, 2, "deg_p"), (7, 7, 528, 3, "upd"),
         (5, 4, 16, 9, "upd"), (7, 5, 1024, 3, "enc")]
LARGE = [(13, 12, 1024, 3, "enc"), (29, 8, 512, 2, "rec_dd"), (59, 20, 2048, 1, "deg_d"), (13, 6, 4096, 2, "upd")]


TABLES = ["params", "device"]


def set_tables(rcg, c, tables):
    c.set_batch_tables(rcg.RCG_TABLES_AUTO if tables == "params" else rcg.RCG_TABLES_DEVICE)


@pytest.mark.parametrize("tables", TABLES)
@pytest.mark.parametrize("mix", ["small", "large", "both"])
def test_batch_with_column_jobs_matches_oracle(rcg, ctxs, oracle, mix, tables):
    # p <= 7 jobs run in the column kernels of the batch, the others in the
    # tile engine; the same slot is launched with only one kind, then both.
    # These tables are small: "params" passes them in the kernels' parameter
    # blocks, "device" copies them to a device buffer in the batch graph.
    col, eng = ctxs
    specs = SMALL if mix == "small" else LARGE if mix == "large" else SMALL + LARGE
    for c in (col, eng):  # column kernels in the batch, and the tile engine alone
        set_tables(rcg, c, tables)
        for rep in range(2):
            bufs, jobs, outs, want_bufs, want_outs = mixed_batch(rcg, oracle, 4700 + 10 * rep, specs)
            assert c.batch_wait(c.batch_submit(jobs))
            assert c.last_device_status() == 0
            for k, (b, w) in enumerate(zip(bufs, want_bufs)):
                assert np.array_equal(b.cpu().numpy(), w), (specs[k], rep)
            for o, w in zip(outs, want_outs):
                assert np.array_equal(o.cpu().numpy(), w)
        set_tables(rcg, c, "params")


# (column jobs, engine jobs): tables of about 2.2 KB, 15 KB and 39 KB -- the
# parameter block's small and large classes, and one over its 31 744 bytes
# that goes to a device buffer even when parameter tables are allowed
SIZE_CLASSES = [(4, 4), (60, 20), (300, 4)]


@pytest.mark.parametrize("n_col,n_eng", SIZE_CLASSES)
def test_batch_table_size_classes(rcg, oracle, n_col, n_eng):
    kinds = ["enc", "rec_dd", "rec_dp", "rec_dq", "rec_pq", "deg_d", "deg_q", "upd"]
    specs = [(5, 4, 64 + 16 * (k % 5), 1 + k % 2, kinds[k % len(kinds)]) for k in range(n_col)]
    specs += [(13, 6, 512, 1, kinds[k % len(kinds)]) for k in range(n_eng)]
    results = []
    with rcg.Context(0) as c:
        for tables in TABLES:
            set_tables(rcg, c, tables)
            bufs, jobs, outs, want_bufs, want_outs = mixed_batch(rcg, oracle, 5200, specs)
            assert c.batch_wait(c.batch_submit(jobs))
            assert c.last_device_status() == 0
            for k, (b, w) in enumerate(zip(bufs, want_bufs)):
                assert np.array_equal(b.cpu().numpy(), w), (tables, specs[k])
            for o, w in zip(outs, want_outs):
                assert np.array_equal(o.cpu().numpy(), w), tables
            results.append([b.cpu().numpy() for b in bufs])
    for a, b in zip(*results):
        assert np.array_equal(a, b)


def test_batch_tables_setting_is_validated(rcg):
    with rcg.Context(0) as c:
        with pytest.raises(rcg.RcgError):
            c.set_batch_tables(2)
        c.set_batch_tables(rcg.RCG_TABLES_DEVICE)
        c.set_batch_tables(rcg.RCG_TABLES_AUTO)


def test_p5n4_sixteen_operations_in_one_batch(rcg, oracle):
    # the p = 5, N = 4, 1 KiB-row geometry (1024 stripes): encode and the 15
    # erasure pairs, each on a copy of its own, as ONE batch (384 MB) -- the
    # form in which this small geometry can fill HBM; every byte against O2,
    # sampled stripes against the bit-level oracle
    p, N, C, S = 5, 4, 1024, 1024
    host = stripes(0, p, N, C, S)
    enc = host.copy()
    oracle.o2_encode(p, N, C, enc, S)
    pairs = [(i, j) for i in range(N + 2) for j in range(i + 1, N + 2)]
    copies = torch.empty((16, S, N + 2, p - 1, C), dtype=torch.uint8, device="cuda")
    copies[0] = dev(host)
    for k, (i, j) in enumerate(pairs, 1):
        lost = enc.copy()
        lost[:, i] = POISON_I
        lost[:, j] = POISON_J
        copies[k] = dev(lost)
    jobs = [rcg.make_job(rcg.make_layout(copies[0], p, N, C), 0, S, rcg.RCG_OP_ENCODE)]
    for k, (i, j) in enumerate(pairs, 1):
        jobs.append(rcg.make_job(rcg.make_layout(copies[k], p, N, C), 0, S, rcg.RCG_OP_RECOVER, i, j))
    with rcg.Context(0) as c:
        assert c.batch_wait(c.batch_submit(jobs))
        assert c.last_device_status() == 0
    got = copies.cpu().numpy()
    for k in range(16):
        assert np.array_equal(got[k], enc), k
    sample = stripes(0, p, N, C, S)[:8].copy()
    oracle.encode(p, N, C, sample, 8)
    assert np.array_equal(got[0, :8], sample)


@pytest.mark.parametrize("tables", TABLES + ["alternating"])
def test_back_to_back_batches_switching_kernels(rcg, oracle, tables):
    # batches launched without waiting, alternating column-kernel-only, tile-
    # engine-only and mixed tables, so each replayed graph switches its kernel
    # nodes on and off while the previous batches still run (and, alternating,
    # parameter-block and device tables follow each other on the stream):
    # every batch must run on its own table
    kinds = ["p5", "p13", "mix", "p5", "p5"] * 60
    bufs = []
    for k, kind in enumerate(kinds):
        geos = {"p5": [(5, 4, 544)], "p13": [(13, 6, 512)], "mix": [(13, 6, 512), (5, 4, 544)]}[kind]
        entry = []
        for g, (p, N, C) in enumerate(geos):
            host = stripes(7000 + 2 * k + g, p, N, C, 1)
            entry.append((p, N, C, host, dev(host)))
        bufs.append(entry)
    with rcg.Context(0) as c:
        for k, entry in enumerate(bufs):
            set_tables(rcg, c, TABLES[k % 2] if tables == "alternating" else tables)
            c.batch_submit([rcg.make_job(rcg.make_layout(d, p, N, C), 0, 1, rcg.RCG_OP_ENCODE)
                            for p, N, C, _, d in entry])
        torch.cuda.synchronize()
        assert c.last_device_status() == 0
    for k, entry in enumerate(bufs):
        for p, N, C, host, d in entry:
            want = host.copy()
            oracle.encode(p, N, C, want, 1)
            assert np.array_equal(d.cpu().numpy(), want), (k, kinds[k], p)
