"""rcg_batch_submit_noalloc: the batch entry point for callers that may not
allocate device memory (a framework whose allocator owns the whole GPU, or a
submit path that cannot take cudaMalloc's implicit synchronisation).

It must give exactly the bytes rcg_batch_submit gives for the same jobs, and
the bytes of the CPU oracle -- the code is XOR over GF(2), so the tolerance is
zero -- on two calls in a row, the second reusing the scratch the first one
left behind.  Recoveries, degraded reads and small writes run on stripes the
oracle encoded (codewords), so the bytes they check are the code's.  This file is
collected last so that a failure here does not hide the rest of the suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_cs_0611109_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rcg():
    from paper_cs_0611109_gb300 import build
    build.build()
    from paper_cs_0611109_gb300 import rcg as R
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return R


def make_batch(rcg, oracle, seed, specs):
    """Device buffers and jobs for a mixed batch, and the oracle's expected
    bytes.  Recoveries, degraded reads and small writes run on stripes the
    oracle encoded first (codewords); a recovery's erased strips are poisoned.
    Returns (buffers, jobs, outs, expected buffers, expected outs)."""
    bufs, jobs, outs, want_bufs, want_outs = [], [], [], [], []
    for n, (p, N, C, S, kind) in enumerate(specs):
        host = np.ascontiguousarray(inputs.random_stripes(seed + n, p, N, C, S))
        if kind != "enc":
            oracle.encode(p, N, C, host, S)
        want = host.copy()
        if kind == "enc":
            oracle.encode(p, N, C, want, S)
        elif kind == "rec":
            i, j = 1, min(3, N + 1)
            host[:, i] = 0xA5
            host[:, j] = 0x5A
        buf = torch.from_numpy(host).cuda()
        L = rcg.make_layout(buf, p, N, C)
        if kind == "enc":
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE))
        elif kind == "rec":
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_RECOVER, i, j))
        elif kind == "deg":
            out = torch.zeros((S, p - 1, C), dtype=torch.uint8, device="cuda")
            outs.append(out)
            want_outs.append(np.stack([oracle.degraded_read(p, N, C, want, s, 0) for s in range(S)]))
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, 0, out))
        elif kind == "upd":
            new = inputs.random_bytes(seed + 99, S * (p - 1) * C).reshape(S, p - 1, C)
            for s in range(S):
                oracle.update(p, N, C, want, s, N - 1, new[s])
            new_dev = torch.from_numpy(np.ascontiguousarray(new)).cuda()
            outs.append(new_dev)
            want_outs.append(new)
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_UPDATE, N - 1, 0, new_dev))
        bufs.append(buf)
        want_bufs.append(want)
    return bufs, jobs, outs, want_bufs, want_outs


def run_both(rcg, oracle, seed, specs, with_status=True):
    # reference: the existing context-based batch entry point
    ref_bufs, ref_jobs, ref_outs, _, _ = make_batch(rcg, oracle, seed, specs)
    with rcg.Context(0) as ctx:
        t = ctx.batch_submit(ref_jobs)
        assert ctx.batch_wait(t)
        assert ctx.last_device_status() == 0
    # the same jobs through the no-allocation entry point
    bufs, jobs, outs, want_bufs, want_outs = make_batch(rcg, oracle, seed, specs)
    status = torch.zeros(1, dtype=torch.int32, device="cuda") if with_status else None
    rcg.rcg_batch_submit_noalloc(jobs, status)
    torch.cuda.synchronize()
    if with_status:
        assert int(status.item()) == 0
    for a, b, w in zip(ref_bufs, bufs, want_bufs):
        assert torch.equal(a, b)
        assert np.array_equal(b.cpu().numpy(), w)  # and the oracle's bytes
    for a, b, w in zip(ref_outs, outs, want_outs):
        assert torch.equal(a, b)
        assert np.array_equal(b.cpu().numpy(), w)


FIRST = [(13, 12, 4096, 6, "enc"), (5, 4, 1024, 9, "rec"), (59, 58, 528, 2, "rec"),
         (29, 7, 1040, 3, "deg"), (13, 6, 256, 4, "upd"), (3, 2, 16, 5, "enc")]
SECOND = [(59, 58, 2048, 3, "enc"), (13, 12, 1024, 40, "rec"), (61, 60, 64, 2, "deg"),
          (5, 4, 64, 17, "upd")]


def test_noalloc_matches_batch_submit_twice_in_a_row(rcg, oracle):
    run_both(rcg, oracle, 1000, FIRST)
    run_both(rcg, oracle, 2000, SECOND)


# 120 engine jobs (their tensor-map entries and work items: about 46 KB of
# table) and 40 column jobs: over the 31 744 bytes a kernel parameter block
# holds, so this table goes through the scratch; FIRST and SECOND are small
# and travel in the kernels' parameter blocks
KINDS = ["enc", "rec", "deg", "upd"]
LARGE_TABLE = [(13, 6, 256, 1, KINDS[k % 4]) for k in range(120)] + \
              [(5, 4, 64, 1 + k % 3, KINDS[k % 4]) for k in range(40)]


def test_noalloc_large_table_between_small_ones(rcg, oracle):
    run_both(rcg, oracle, 4000, LARGE_TABLE)
    run_both(rcg, oracle, 5000, FIRST)
    run_both(rcg, oracle, 6000, LARGE_TABLE)


def test_noalloc_without_a_status_word(rcg, oracle):
    # with status_dev = NULL device-side errors go unreported, but a valid
    # batch still gives the oracle's bytes
    run_both(rcg, oracle, 3000, SECOND, with_status=False)


def test_noalloc_rejects_too_many_jobs(rcg):
    n = rcg.RCG_NOALLOC_MAX_JOBS + 1
    buf = torch.zeros((n, 6, 4, 16), dtype=torch.uint8, device="cuda")
    L = rcg.make_layout(buf, 5, 4, 16)
    jobs = [rcg.make_job(L, s, 1, rcg.RCG_OP_ENCODE) for s in range(n)]  # one stripe each
    with pytest.raises(rcg.RcgError) as e:
        rcg.rcg_batch_submit_noalloc(jobs)
    assert e.value.status == rcg.RCG_EINVAL
    # the limit itself is accepted
    rcg.rcg_batch_submit_noalloc(jobs[:rcg.RCG_NOALLOC_MAX_JOBS])
    torch.cuda.synchronize()
