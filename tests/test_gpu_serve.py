"""The serving loop: continuous batching over a Poisson request stream.

Every request's result must be the same alone and in the mix (tolerance 0:
the code is XOR over GF(2)): the served run is compared with the same
requests run one at a time through the single-operation calls, and sampled
stripes with the CPU oracle.
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


def make_stream(rcg, seed, n, rate_per_s):
    """n requests on n distinct stripes (c4-like geometry, rows <= 4 KiB):
    70 % encode, 20 % degraded read, 10 % two-erasure rebuild; Poisson
    arrivals at rate_per_s.  Returns device state and the request list."""
    rng = np.random.Generator(np.random.PCG64(seed))
    geo = inputs.batched_jobs(seed, n, c_min=512, c_max=4096)
    sizes = [inputs.stripe_bytes(g["p"], g["n"], g["c"]) for g in geo]
    offs = np.cumsum([0] + [(b + 255) // 256 * 256 for b in sizes])
    arena = torch.empty(int(offs[-1]), dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(arena, arena.numel(), seed)
    kinds = rng.choice(["encode", "degraded", "rebuild"], size=n, p=[0.7, 0.2, 0.1])
    out_sizes = [(g["p"] - 1) * g["c"] for g in geo]
    out_offs = np.cumsum([0] + [(b + 255) // 256 * 256 for b in out_sizes])
    outs = torch.zeros(int(out_offs[-1]), dtype=torch.uint8, device="cuda")
    arrivals = np.cumsum(rng.exponential(1e9 / rate_per_s, size=n)).astype(np.int64)
    reqs = []
    for k, g in enumerate(geo):
        L = rcg.make_layout(arena.data_ptr() + int(offs[k]), g["p"], g["n"], g["c"])
        if kinds[k] == "encode":
            job = rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE)
        elif kinds[k] == "degraded":
            j = int(rng.integers(0, g["n"] + 2))
            job = rcg.make_job(L, 0, 1, rcg.RCG_OP_DEGRADED_READ, 0, j, outs.data_ptr() + int(out_offs[k]))
        else:
            a, b = sorted(rng.choice(g["n"] + 2, size=2, replace=False).tolist())
            job = rcg.make_job(L, 0, 1, rcg.RCG_OP_RECOVER, a, b)
        reqs.append((kinds[k], g, int(offs[k]), job))
    return arena, outs, reqs, arrivals, offs


def prepare_state(rcg, arena, reqs):
    """Encode the stripes that degraded reads and rebuilds work on, then
    poison the erased strips of the rebuilds."""
    with rcg.Context(0) as c:
        pre = [job for kind, g, o, job in reqs if kind != "encode"]
        for job in pre:
            c.encode(job.layout, 0, 1)
        torch.cuda.synchronize()
    for kind, g, o, job in reqs:
        if kind == "rebuild":
            sb = (g["p"] - 1) * g["c"]
            for k in (job.i, job.j):
                arena[o + k * sb: o + (k + 1) * sb] = 0xA5


# batched with the default of up to eight batches in flight, batched with two,
# and one launch per request
@pytest.mark.parametrize("per_job,batches", [(False, 0), (False, 2), (True, 0)])
def test_served_results_equal_alone(rcg, oracle, per_job, batches):
    arena, outs, reqs, arrivals, offs = make_stream(rcg, 31, 600, rate_per_s=200000)
    prepare_state(rcg, arena, reqs)
    initial = arena.clone()
    with rcg.Context(0) as c:
        srv = rcg.rcg_serve_create(c.handle, max_inflight_jobs=256, max_batch_jobs=128,
                                   per_job_launches=per_job, max_inflight_batches=batches)
        rcg.rcg_serve_submit(srv, [r[3] for r in reqs], arrivals)
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 60 * 10 ** 9)
        res = rcg.rcg_serve_results(srv, len(reqs))
        stats = rcg.rcg_serve_get_stats(srv)
        rcg.rcg_serve_destroy(srv)
        assert c.last_device_status() == 0
    served, served_outs = arena.clone(), outs.clone()
    assert all(r["status"] == 0 for r in res)
    for r in res:
        assert r["arrival_ns"] <= r["admit_ns"] <= r["launch_ns"] <= r["complete_ns"], r
    assert stats["completed"] == len(reqs)
    if per_job:
        # one kernel launch per request, each with its own launch number
        assert stats["kernel_launches"] == len(reqs)
        assert len({r["batch"] for r in res}) == len(reqs)
    else:
        assert max(r["batch"] for r in res) < len(reqs)  # requests were batched together
        assert stats["kernel_launches"] == len({r["batch"] for r in res})
        assert stats["max_inflight_launches"] <= (batches or 8)
    # alone: the same requests one at a time on the initial state
    arena.copy_(initial)
    outs.zero_()
    with rcg.Context(0) as c:
        for kind, g, o, job in reqs:
            if kind == "encode":
                c.encode(job.layout, 0, 1)
            elif kind == "degraded":
                c.degraded_read(job.layout, 0, job.j, job.aux)
            else:
                c.recover(job.layout, 0, job.i, job.j)
        torch.cuda.synchronize()
    assert torch.equal(arena, served)
    assert torch.equal(outs, served_outs)
    # and every sampled request agrees with the oracle: encodes and rebuilds by
    # the stripe's bytes, degraded reads by the strip they returned
    got = served.cpu().numpy()
    got_outs = served_outs.cpu().numpy()
    start = initial.cpu().numpy()
    out_offs = np.cumsum([0] + [((g["p"] - 1) * g["c"] + 255) // 256 * 256 for _, g, _, _ in reqs])
    checked = {"encode": 0, "degraded": 0, "rebuild": 0}
    for k in range(len(reqs)):
        kind, g, o, job = reqs[k]
        if checked[kind] >= 25:
            continue
        checked[kind] += 1
        b = inputs.stripe_bytes(g["p"], g["n"], g["c"])
        want = np.ascontiguousarray(start[o:o + b])
        if kind == "encode":
            oracle.encode(g["p"], g["n"], g["c"], want, 1)
        elif kind == "rebuild":
            oracle.recover(g["p"], g["n"], g["c"], want, 1, job.i, job.j)
        else:
            strip = oracle.degraded_read(g["p"], g["n"], g["c"], want, 0, job.j)
            n_out = (g["p"] - 1) * g["c"]
            assert np.array_equal(got_outs[out_offs[k]:out_offs[k] + n_out].reshape(g["p"] - 1, g["c"]), strip), k
        assert np.array_equal(got[o:o + b], want), k
    assert min(checked.values()) > 0


def test_batched_mode_keeps_several_batches_in_flight(rcg):
    # every request arrives at once, one request per batch: batches go out on
    # the server's streams without waiting for one another, up to the limit
    arena, outs, reqs, arrivals, offs = make_stream(rcg, 34, 200, rate_per_s=10 ** 9)
    prepare_state(rcg, arena, reqs)
    with rcg.Context(0) as c:
        with pytest.raises(rcg.RcgError):
            rcg.rcg_serve_create(c.handle, max_inflight_batches=9)
        srv = rcg.rcg_serve_create(c.handle, max_inflight_jobs=512, max_batch_jobs=1)
        rcg.rcg_serve_submit(srv, [r[3] for r in reqs], np.zeros(len(reqs), np.int64))
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 60 * 10 ** 9)
        res = rcg.rcg_serve_results(srv, len(reqs))
        stats = rcg.rcg_serve_get_stats(srv)
        rcg.rcg_serve_destroy(srv)
        assert c.last_device_status() == 0
    assert all(r["status"] == 0 for r in res)
    assert stats["kernel_launches"] == len(reqs)
    assert 2 < stats["max_inflight_launches"] <= 8


def test_per_job_mode_keeps_many_launches_in_flight(rcg):
    # every request arrives at once: per-job mode must not gate single
    # launches behind one another in rounds
    arena, outs, reqs, arrivals, offs = make_stream(rcg, 33, 400, rate_per_s=10 ** 9)
    prepare_state(rcg, arena, reqs)
    with rcg.Context(0) as c:
        srv = rcg.rcg_serve_create(c.handle, max_inflight_jobs=512, per_job_launches=True)
        rcg.rcg_serve_submit(srv, [r[3] for r in reqs], np.zeros(len(reqs), np.int64))
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 60 * 10 ** 9)
        stats = rcg.rcg_serve_get_stats(srv)
        rcg.rcg_serve_destroy(srv)
        assert c.last_device_status() == 0
    assert stats["kernel_launches"] == len(reqs)
    assert stats["max_inflight_launches"] > 2


def default_footprint(g, kind):
    """The default HBM footprint of a request (rcg.h): (N + 2) strips of the
    stripe, plus the output strip of a degraded read."""
    fp = (g["n"] + 2) * (g["p"] - 1) * g["c"]
    if kind == "degraded":
        fp += (g["p"] - 1) * g["c"]
    return fp


@pytest.mark.parametrize("explicit", [True, False])
def test_admission_respects_the_hbm_budget(rcg, explicit):
    arena, outs, reqs, arrivals, offs = make_stream(rcg, 32, 200, rate_per_s=10 ** 7)
    prepare_state(rcg, arena, reqs)
    if explicit:  # caller-declared footprints
        fps = [inputs.stripe_bytes(g["p"], g["n"], g["c"]) + (g["p"] - 1) * g["c"] for _, g, _, _ in reqs]
    else:         # the server's default footprint of each job
        fps = [default_footprint(g, kind) for kind, g, _, _ in reqs]
    budget = 3 * max(fps)
    with rcg.Context(0) as c:
        srv = rcg.rcg_serve_create(c.handle, hbm_budget_bytes=budget, max_batch_jobs=64)
        rcg.rcg_serve_submit(srv, [r[3] for r in reqs], arrivals, footprints=fps if explicit else None)
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 60 * 10 ** 9)
        res = rcg.rcg_serve_results(srv, len(reqs))
        rcg.rcg_serve_destroy(srv)
    # at any admission instant the admitted-but-not-completed footprint fits the budget
    events = sorted([(r["admit_ns"], fps[r["id"]]) for r in res] + [(r["complete_ns"], -fps[r["id"]]) for r in res],
                    key=lambda e: (e[0], e[1]))
    used = peak = 0
    for t, d in events:
        used += d
        peak = max(peak, used)
        assert used <= budget
    assert peak > max(fps)  # the budget, not a one-at-a-time rule, was what limited admission


def test_requests_on_overlapping_stripes_run_in_order(rcg, oracle):
    # a 4-stripe encode, a degraded read of a strip of its third stripe and an
    # encode of its second stripe arrive together: they touch the same bytes,
    # so both must wait for the 4-stripe encode (never share its launch).  The
    # degraded read rebuilds data strip 1 from P, which is only right once the
    # encode has written P.
    p, N, C, S = 13, 6, 512, 4
    host = np.ascontiguousarray(inputs.random_stripes(41, p, N, C, S))  # P, Q hold random bytes
    want = host.copy()
    oracle.encode(p, N, C, want, S)
    buf = torch.from_numpy(host.copy()).cuda()
    out = torch.zeros((p - 1, C), dtype=torch.uint8, device="cuda")
    L = rcg.make_layout(buf, p, N, C)
    jobs = [rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE),
            rcg.make_job(L, 2, 1, rcg.RCG_OP_DEGRADED_READ, 0, 1, out),
            rcg.make_job(L, 1, 1, rcg.RCG_OP_ENCODE)]
    with rcg.Context(0) as c:
        srv = rcg.rcg_serve_create(c.handle)
        rcg.rcg_serve_submit(srv, jobs, [0, 0, 0])
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 60 * 10 ** 9)
        res = rcg.rcg_serve_results(srv, len(jobs))
        stats = rcg.rcg_serve_get_stats(srv)
        rcg.rcg_serve_destroy(srv)
        assert c.last_device_status() == 0
    assert res[0]["batch"] < res[1]["batch"] and res[0]["batch"] < res[2]["batch"]
    assert res[1]["admit_ns"] >= res[0]["complete_ns"] and res[2]["admit_ns"] >= res[0]["complete_ns"]
    assert stats["conflict_waits"] >= 2
    assert np.array_equal(out.cpu().numpy(), host[2, 1])
    assert np.array_equal(buf.cpu().numpy(), want)


def test_submit_is_all_or_nothing(rcg):
    buf = torch.zeros((4, 6, 4, 64), dtype=torch.uint8, device="cuda")
    L = rcg.make_layout(buf, 5, 4, 64)
    good = rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE)
    bad = rcg.make_job(L, 0, 2, rcg.RCG_OP_RECOVER, 0, 1)  # recovery of two stripes: refused
    with rcg.Context(0) as c:
        srv = rcg.rcg_serve_create(c.handle)
        with pytest.raises(rcg.RcgError) as e:
            rcg.rcg_serve_submit(srv, [good, good, bad], [0, 0, 0])
        assert e.value.status == rcg.RCG_EINVAL
        assert rcg.rcg_serve_submit(srv, [good], [0]) == 0  # nothing of the refused call was queued
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 10 ** 10)
        assert len(rcg.rcg_serve_results(srv, 10)) == 1
        rcg.rcg_serve_destroy(srv)
