"""rcg_batch_submit_noalloc: the batch entry point for callers that may not
allocate device memory (a framework whose allocator owns the whole GPU, or a
submit path that cannot take cudaMalloc's implicit synchronisation).

It must give exactly the bytes rcg_batch_submit gives for the same jobs --
the code is XOR over GF(2), so the tolerance is zero -- on two calls in a row,
the second reusing the scratch the first one left behind.  This file is
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


def make_batch(rcg, seed, specs):
    """Device buffers and jobs for a mixed batch; returns (buffers, jobs, outs)."""
    bufs, jobs, outs = [], [], []
    for n, (p, N, C, S, kind) in enumerate(specs):
        host = np.ascontiguousarray(inputs.random_stripes(seed + n, p, N, C, S))
        buf = torch.from_numpy(host).cuda()
        L = rcg.make_layout(buf, p, N, C)
        if kind == "enc":
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE))
        elif kind == "rec":
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_RECOVER, 1, min(3, N + 1)))
        elif kind == "deg":
            out = torch.zeros((S, p - 1, C), dtype=torch.uint8, device="cuda")
            outs.append(out)
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, 0, out))
        elif kind == "upd":
            new = torch.from_numpy(inputs.random_bytes(seed + 99, S * (p - 1) * C).reshape(S, p - 1, C)).cuda()
            outs.append(new)
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_UPDATE, N - 1, 0, new))
        bufs.append(buf)
    return bufs, jobs, outs


def run_both(rcg, seed, specs):
    # reference: the existing context-based batch entry point
    ref_bufs, ref_jobs, ref_outs = make_batch(rcg, seed, specs)
    with rcg.Context(0) as ctx:
        t = ctx.batch_submit(ref_jobs)
        assert ctx.batch_wait(t)
        assert ctx.last_device_status() == 0
    # the same jobs through the no-allocation entry point
    bufs, jobs, outs = make_batch(rcg, seed, specs)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rcg.rcg_batch_submit_noalloc(jobs, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for a, b in zip(ref_bufs, bufs):
        assert torch.equal(a, b)
    for a, b in zip(ref_outs, outs):
        assert torch.equal(a, b)


def test_noalloc_matches_batch_submit_twice_in_a_row(rcg):
    first = [(13, 12, 4096, 6, "enc"), (5, 4, 1024, 9, "rec"), (59, 58, 528, 2, "rec"),
             (29, 7, 1040, 3, "deg"), (13, 6, 256, 4, "upd"), (3, 2, 16, 5, "enc")]
    second = [(59, 58, 2048, 3, "enc"), (13, 12, 1024, 40, "rec"), (61, 60, 64, 2, "deg"),
              (5, 4, 64, 17, "upd")]
    run_both(rcg, 1000, first)
    run_both(rcg, 2000, second)


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
