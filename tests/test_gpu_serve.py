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


@pytest.mark.parametrize("per_job", [False, True])
def test_served_results_equal_alone(rcg, oracle, per_job):
    arena, outs, reqs, arrivals, offs = make_stream(rcg, 31, 600, rate_per_s=200000)
    prepare_state(rcg, arena, reqs)
    initial = arena.clone()
    with rcg.Context(0) as c:
        srv = rcg.rcg_serve_create(c.handle, max_inflight_jobs=256, max_batch_jobs=128,
                                   per_job_launches=per_job)
        rcg.rcg_serve_submit(srv, [r[3] for r in reqs], arrivals)
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 60 * 10 ** 9)
        res = rcg.rcg_serve_results(srv, len(reqs))
        rcg.rcg_serve_destroy(srv)
        assert c.last_device_status() == 0
    served, served_outs = arena.clone(), outs.clone()
    assert all(r["status"] == 0 for r in res)
    for r in res:
        assert r["arrival_ns"] <= r["admit_ns"] <= r["launch_ns"] <= r["complete_ns"], r
    if not per_job:
        assert max(r["batch"] for r in res) < len(reqs)  # requests were batched together
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
    # and sampled stripes agree with the oracle
    got = served.cpu().numpy()
    start = initial.cpu().numpy()
    for k in range(0, len(reqs), 53):
        kind, g, o, job = reqs[k]
        b = inputs.stripe_bytes(g["p"], g["n"], g["c"])
        want = np.ascontiguousarray(start[o:o + b])
        if kind == "encode":
            oracle.encode(g["p"], g["n"], g["c"], want, 1)
        elif kind == "rebuild":
            oracle.recover(g["p"], g["n"], g["c"], want, 1, job.i, job.j)
        assert np.array_equal(got[o:o + b], want), k


def test_admission_respects_the_hbm_budget(rcg):
    arena, outs, reqs, arrivals, offs = make_stream(rcg, 32, 200, rate_per_s=10 ** 7)
    prepare_state(rcg, arena, reqs)
    fps = [inputs.stripe_bytes(g["p"], g["n"], g["c"]) + (g["p"] - 1) * g["c"] for _, g, _, _ in reqs]
    budget = 3 * max(fps)
    with rcg.Context(0) as c:
        srv = rcg.rcg_serve_create(c.handle, hbm_budget_bytes=budget, max_batch_jobs=64)
        rcg.rcg_serve_submit(srv, [r[3] for r in reqs], arrivals, footprints=fps)
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 60 * 10 ** 9)
        res = rcg.rcg_serve_results(srv, len(reqs))
        rcg.rcg_serve_destroy(srv)
    # at any admission instant the admitted-but-not-completed footprint fits the budget
    events = sorted([(r["admit_ns"], fps[r["id"]]) for r in res] + [(r["complete_ns"], -fps[r["id"]]) for r in res],
                    key=lambda e: (e[0], e[1]))
    used = 0
    for t, d in events:
        used += d
        assert used <= budget
