"""CPU tests of the serving engine's admission bookkeeping (rcg_admission.h).

The class decides which submitted requests start: requests whose device byte
extents overlap must run one after the other, in submission order, and the
in-flight count and HBM budget bound what runs at once.  It uses exact-extent
hashes and merged interval maps to find conflicts quickly; these tests drive it
through seeded random scripts (through a small C++ driver compiled here) and
check every decision against a brute-force model that compares extents pair by
pair, plus the safety properties themselves.
"""
import collections
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_cs_0611109_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("adm") / "serve_admission_driver")
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(ROOT, "tests", "serve_admission_driver.cpp"), "-o", exe], check=True)
    return exe


class Driver:
    def __init__(self, exe, budget, max_inflight):
        self.p = subprocess.Popen([exe], stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True, bufsize=1)
        self.cmd(f"I {budget} {max_inflight}")

    def cmd(self, line):
        self.p.stdin.write(line + "\n")
        self.p.stdin.flush()
        out = self.p.stdout.readline().split()
        assert out and out[0] == "ok", (line, out)
        return [int(v) for v in out[1:]]

    def add(self, arrival, footprint, ext):
        flat = " ".join(f"{lo} {hi}" for lo, hi in ext)
        return self.cmd(f"R {arrival} {footprint} {len(ext)} {flat}")[0]

    def admit(self, now):
        return self.cmd(f"A {now}")

    def retire(self, i):
        self.cmd(f"X {i}")

    def stats(self):
        return self.cmd("S")

    def close(self):
        self.p.stdin.write("Q\n")
        self.p.stdin.close()
        assert self.p.wait(timeout=10) == 0


def overlap(a, b):
    return a[0] < b[1] and b[0] < a[1]


def any_overlap(ea, eb):
    return any(overlap(a, b) for a in ea for b in eb)


class Model:
    """The admission policy with conflicts found by comparing every pair of
    extents: requests are examined in submission order; one that has not
    arrived, or would pass the in-flight limit or the budget, ends the pass;
    one overlapping an in-flight request or an earlier waiting one waits; a
    waiting request is looked at again only after some request has retired."""

    def __init__(self, budget, max_inflight):
        self.budget, self.max_inflight = budget, max_inflight
        self.items = []
        self.pending = collections.deque()
        self.blocked = []
        self.busy = {}
        self.used = 0
        self.freed = False
        self.waits = 0

    def add(self, arrival, footprint, ext):
        self.items.append((arrival, footprint, [e for e in ext if e[1] > e[0]]))
        self.pending.append(len(self.items) - 1)
        return len(self.items) - 1

    def retire(self, i):
        self.used -= self.items[i][1]
        del self.busy[i]
        self.freed = True

    def admit(self, now):
        if self.freed and self.blocked:
            self.pending = collections.deque(self.blocked + list(self.pending))
            self.blocked = []
        self.freed = False
        out = []
        while self.pending:
            i = self.pending[0]
            arrival, footprint, ext = self.items[i]
            if arrival > now or len(self.busy) >= self.max_inflight or self.used + footprint > self.budget:
                break
            self.pending.popleft()
            if any(any_overlap(ext, self.items[j][2]) for j in list(self.busy) + self.blocked):
                self.blocked.append(i)
                self.waits += 1
                continue
            self.busy[i] = True
            self.used += footprint
            out.append(i)
        return out


def random_extent(rng, pool):
    """Mostly whole stripes from a small pool (exact repeats, the common case
    in serving), sometimes an arbitrary range that straddles several."""
    if rng.random() < 0.7:
        return pool[rng.integers(len(pool))]
    lo = int(rng.integers(0, pool[-1][1]))
    return (lo, lo + int(rng.integers(1, 3 * (pool[0][1] - pool[0][0]))))


def run_script(exe, seed, n_req, budget, max_inflight, n_stripes, stripe=4096, gap=0):
    rng = np.random.default_rng(seed)
    pool = [(k * (stripe + gap), k * (stripe + gap) + stripe) for k in range(n_stripes)]
    d = Driver(exe, budget, max_inflight)
    m = Model(budget, max_inflight)
    reqs = []
    t = 0
    for _ in range(n_req):
        t += int(rng.integers(0, 3))
        ext = [random_extent(rng, pool)]
        if rng.random() < 0.3:
            ext.append(random_extent(rng, pool))
        fp = int(rng.integers(1, budget // 3 + 2))
        reqs.append((t, fp, ext))
        assert d.add(t, fp, ext) == m.add(t, fp, ext)

    # ext as the class stores it: the two extents merged when they overlap or touch
    def norm(ext):
        ext = [e for e in ext if e[1] > e[0]]
        if len(ext) == 2 and ext[1][0] <= ext[0][1] and ext[0][0] <= ext[1][1]:
            ext = [(min(ext[0][0], ext[1][0]), max(ext[0][1], ext[1][1]))]
        return ext

    admitted_at, retired_at = {}, {}
    inflight = []
    now, step = 0, 0
    while len(retired_at) < n_req:
        step += 1
        assert step < 50 * n_req + 1000, "no progress"
        got = d.admit(now)
        assert got == m.admit(now), (seed, now)
        for i in got:
            assert reqs[i][0] <= now
            admitted_at[i] = step
            inflight.append(i)
        # safety: in-flight requests are disjoint, within the limits
        assert len(inflight) <= max_inflight
        assert sum(reqs[i][1] for i in inflight) <= budget
        for a in range(len(inflight)):
            for b in range(a + 1, len(inflight)):
                assert not any_overlap(reqs[inflight[a]][2], reqs[inflight[b]][2])
        st = d.stats()
        assert st[0] == len(inflight) and st[1] == sum(reqs[i][1] for i in inflight) and st[2] == m.waits
        # retire a random subset of what runs; time moves on
        for i in list(inflight):
            if rng.random() < 0.4:
                inflight.remove(i)
                d.retire(i)
                m.retire(i)
                retired_at[i] = step
        if not got or rng.random() < 0.5:
            now += int(rng.integers(1, 4))
    d.close()
    # order: of two overlapping requests the earlier one finished before the
    # later one started
    for j in range(n_req):
        for i in range(j):
            if any_overlap(norm(reqs[i][2]), norm(reqs[j][2])):
                assert retired_at[i] <= admitted_at[j], (seed, i, j)
    return m.waits


@pytest.mark.parametrize("seed", range(6))
def test_admission_matches_model_contended(driver, seed):
    # few stripes: most requests wait on another
    waits = run_script(driver, seed, n_req=300, budget=10 ** 6, max_inflight=8, n_stripes=6)
    assert waits > 0


@pytest.mark.parametrize("seed", range(4))
def test_admission_matches_model_limits(driver, seed):
    # many stripes, tight budget and in-flight limits
    run_script(driver, 100 + seed, n_req=300, budget=40, max_inflight=3, n_stripes=64, gap=512)


@pytest.mark.parametrize("seed", range(3))
def test_admission_touching_stripes(driver, seed):
    # stripes back to back: touching extents merge in the waiting map but must
    # not count as overlapping
    run_script(driver, 200 + seed, n_req=250, budget=10 ** 6, max_inflight=16, n_stripes=12, stripe=64)


def test_admission_independent_requests_all_start(driver):
    # disjoint requests within the limits all start at once, in order
    d = Driver(driver, 10 ** 9, 1000)
    for k in range(100):
        d.add(0, 10, [(k * 100, k * 100 + 50)])
    assert d.admit(0) == list(range(100))
    d.close()


def test_admission_same_stripe_in_order(driver):
    # every request on one stripe: one at a time, in submission order, and a
    # later request on other bytes is not held up by them
    d = Driver(driver, 10 ** 9, 1000)
    for _ in range(5):
        d.add(0, 1, [(0, 4096)])
    d.add(0, 1, [(8192, 8192 + 4096)])
    assert d.admit(0) == [0, 5]
    for k in range(4):
        assert d.admit(0) == []
        d.retire(k)
        assert d.admit(0) == [k + 1]
    d.close()


def test_admission_two_extents_and_arrival(driver):
    # a request whose second extent overlaps a running one waits; requests
    # that have not arrived do not start
    d = Driver(driver, 10 ** 9, 1000)
    d.add(0, 1, [(0, 100)])
    d.add(0, 1, [(1000, 1100), (50, 60)])
    d.add(5, 1, [(2000, 2100)])
    assert d.admit(0) == [0]
    assert d.admit(4) == []
    assert d.admit(5) == [2]
    d.retire(0)
    assert d.admit(5) == [1]
    d.close()


def test_admission_budget_stops_the_pass(driver):
    # the first request that would pass the budget stops admission
    d = Driver(driver, 100, 1000)
    d.add(0, 60, [(0, 10)])
    d.add(0, 60, [(100, 110)])
    d.add(0, 10, [(200, 210)])
    assert d.admit(0) == [0]
    d.retire(0)
    assert d.admit(0) == [1, 2]
    d.close()
