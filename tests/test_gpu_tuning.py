"""The batch autotuner: it times the real batch under candidate layouts, which
is only sound because every batch operation is idempotent on non-overlapping
jobs -- so after autotuning (about 30 runs) every job's bytes must equal the
oracle's single run.  Every tuning knob must give identical results, and a
tuning round-trips through the JSON cache keyed by GPU model and SM count."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SPECS = [(5, 4, 1024, 3, "enc"), (13, 12, 4096, 2, "rec"), (29, 7, 528, 2, "deg"),
         (59, 58, 2048, 1, "rec"), (3, 2, 16, 4, "enc"), (13, 6, 1040, 2, "upd"),
         (61, 60, 64, 1, "rec"), (13, 25, 2048, 2, "rec"), (5, 9, 4096 + 16, 3, "enc")]
_ORACLE = {}


def oracle_arrays(oracle, seed, n, p, N, C, S, kind):
    """(input stripes, expected stripes) for one job; the oracle runs once per key."""
    key = (seed, n)
    if key not in _ORACLE:
        host = np.ascontiguousarray(inputs.random_stripes(seed + n, p, N, C, S))
        if kind != "enc":
            oracle.encode(p, N, C, host, S)
        want = host.copy()
        if kind == "enc":
            oracle.encode(p, N, C, want, S)
        elif kind == "upd":
            new = inputs.random_bytes(seed + 99, S * (p - 1) * C).reshape(S, p - 1, C)
            for s in range(S):
                oracle.update(p, N, C, want, s, 2, new[s])
        _ORACLE[key] = (host, want)
    host, want = _ORACLE[key]
    return host.copy(), want


def mixed_batch(rcg, oracle, seed):
    """Jobs of every operation over several geometries, with the oracle's
    expected bytes: (jobs, [(device tensor, expected array)])."""
    jobs, checks = [], []
    for n, (p, N, C, S, kind) in enumerate(SPECS):
        host, want = oracle_arrays(oracle, seed, n, p, N, C, S, kind)
        buf = dev(host)
        L = rcg.make_layout(buf, p, N, C)
        if kind == "enc":
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE))
        elif kind == "rec":
            i, j = (1, N - 1) if N > 2 else (0, N)
            buf[:, i] = POISON_I
            buf[:, j] = POISON_J
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_RECOVER, i, j))
        elif kind == "deg":
            out = torch.zeros((S, p - 1, C), dtype=torch.uint8, device="cuda")
            checks.append((out, host[:, 3].copy()))
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, 3, out))
        elif kind == "upd":
            new = inputs.random_bytes(seed + 99, S * (p - 1) * C).reshape(S, p - 1, C)
            newd = dev(new)
            checks.append((newd, new.copy()))  # the new strips are read, never written
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_UPDATE, 2, 0, newd))
        checks.append((buf, want))
    return jobs, checks


def assert_all(checks):
    for t, want in checks:
        assert np.array_equal(t.cpu().numpy(), want)


def test_autotune_leaves_one_runs_results(rcg, oracle):
    jobs, checks = mixed_batch(rcg, oracle, 5000)
    with rcg.Context(0) as c:
        t = c.batch_autotune(jobs)
        assert c.last_device_status() == 0
        assert t["shape"] in (rcg.RCG_SHAPE_AUTO, rcg.RCG_SHAPE_WIDE, rcg.RCG_SHAPE_PAIR)
        assert t["schedule"] in (rcg.RCG_SCHED_STATIC, rcg.RCG_SCHED_DYNAMIC)
        assert t["tile_div"] in (1, 2, 4) and t["ring"] in (rcg.RCG_RING_FIXED, rcg.RCG_RING_BYTES)
        assert t["ms"] > 0
        assert_all(checks)
        # the tuning stays on the context: a fresh batch under it is exact too
        jobs2, checks2 = mixed_batch(rcg, oracle, 5100)
        assert c.batch_wait(c.batch_submit(jobs2))
        assert c.last_device_status() == 0
        assert_all(checks2)


@pytest.mark.parametrize("shape", ["wide", "pair"])
@pytest.mark.parametrize("tile_div", [1, 2, 4])
@pytest.mark.parametrize("item_bytes", [0, 64 << 10, 4 << 20])
@pytest.mark.parametrize("schedule", ["static", "dynamic"])
@pytest.mark.parametrize("ring", ["fixed", "bytes"])
def test_every_tuning_gives_identical_results(rcg, oracle, shape, tile_div, item_bytes, schedule, ring):
    jobs, checks = mixed_batch(rcg, oracle, 5200)
    tuning = {"shape": rcg.RCG_SHAPE_WIDE if shape == "wide" else rcg.RCG_SHAPE_PAIR,
              "schedule": rcg.RCG_SCHED_STATIC if schedule == "static" else rcg.RCG_SCHED_DYNAMIC,
              "item_bytes": item_bytes, "tile_div": tile_div,
              "ring": rcg.RCG_RING_FIXED if ring == "fixed" else rcg.RCG_RING_BYTES}
    with rcg.Context(0) as c:
        c.set_batch_tuning(tuning)
        assert c.batch_wait(c.batch_submit(jobs))
        assert c.last_device_status() == 0
        assert_all(checks)


def test_tuning_validation_and_cache(rcg, tmp_path):
    with rcg.Context(0) as c:
        good = {"shape": rcg.RCG_SHAPE_WIDE, "schedule": rcg.RCG_SCHED_DYNAMIC, "item_bytes": 0, "tile_div": 2}
        c.set_batch_tuning(good)
        for bad in ({**good, "shape": 9}, {**good, "schedule": 5}, {**good, "item_bytes": 1000},
                    {**good, "tile_div": 0}, {**good, "tile_div": 9}, {**good, "ring": 4}):
            with pytest.raises(rcg.RcgError):
                c.set_batch_tuning(bad)
        c.set_batch_tuning(None)
    path = str(tmp_path / "tuning.json")
    assert rcg.load_tuning(path) is None
    rcg.save_tuning(path, {**good, "ms": 1.5})
    back = rcg.load_tuning(path)
    assert back["tile_div"] == 2 and back["shape"] == rcg.RCG_SHAPE_WIDE
    assert rcg.tuning_key() in open(path).read()
