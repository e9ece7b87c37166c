"""The serving loop's scheduler on the CPU, against a stand-in backend whose
contact angle relaxes exponentially and whose clock advances with the work
done (no GPU)."""
import math

import pytest

from paper_2605_30878_gb300 import serve


class SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """theta(s) = theta_set + amp * exp(-s / decay) after s steps; a step of a
    batch costs its nodes / rate seconds of simulated time."""

    def __init__(self, clock, rate=1e9, amp=10.0, decay=500.0, bytes_per_node=100):
        self.clock, self.rate, self.amp, self.decay = clock, rate, amp, decay
        self.bytes_per_node = bytes_per_node
        self.opened, self.closed, self.batches_made = [], [], []
        self.live_bytes = 0
        self.max_live_bytes = 0

    def prepare(self, req):
        nodes = req.L ** (2 if req.lattice == 9 else 3)
        return dict(bytes=nodes * self.bytes_per_node, fluid_nodes=nodes)

    def open(self, req, case):
        self.opened.append(req.rid)
        self.live_bytes += case["bytes"]
        self.max_live_bytes = max(self.max_live_bytes, self.live_bytes)
        return dict(req=req, steps=0, nodes=case["fluid_nodes"], bytes=case["bytes"])

    def batch(self, lattice, handles):
        assert all(h["req"].lattice == lattice for h in handles)
        self.batches_made.append((lattice, [h["req"].rid for h in handles]))
        return list(handles)

    def close_batch(self, b):
        pass

    def launch(self, batches, n):
        work = 0
        for b in batches:
            for h in b:
                h["steps"] += n
                work += h["nodes"] * n
        self.done_at = self.clock.t + work / self.rate

    def wait(self, batches):
        self.clock.t = max(self.clock.t, self.done_at)

    def angle_deg(self, h):
        return h["req"].theta_deg + self.amp * math.exp(-h["steps"] / self.decay)

    def close(self, h):
        self.closed.append(h["req"].rid)
        self.live_bytes -= h["bytes"]


def _run(reqs, **kw):
    clk = SimClock()
    be = FakeBackend(clk, **{k: kw.pop(k) for k in list(kw) if k in ("rate", "amp", "decay")})
    srv = serve.Server(be, clock=clk, sleep=clk.sleep, **kw)
    res, summ = srv.run(reqs)
    return be, res, summ


def test_poisson_requests_recipe():
    reqs = serve.poisson_requests()
    assert len(reqs) == 200
    assert sum(q.lattice == 9 for q in reqs) == 100
    gaps = [b.arrival - a.arrival for a, b in zip(reqs, reqs[1:])]
    assert all(g > 0 for g in gaps)
    assert abs(reqs[-1].arrival / 200 - 1 / 20.0) < 0.02          # mean inter-arrival 1/lambda
    for q in reqs:
        lo, hi = (128, 1024) if q.lattice == 9 else (64, 192)
        assert lo <= q.L <= hi and 20 <= q.theta_deg <= 160 and 1 <= q.rho_ratio <= 1000
    assert serve.poisson_requests()[7] == reqs[7]                    # seeded


def test_convergence_step_matches_the_criterion():
    """amp e^{-s/500} changes by less than 0.1 deg between checks 1000 apart
    first at s = 3000 (10 (e^-4 - e^-6) = 0.158, 10 (e^-6 - e^-8) = 0.0214)."""
    reqs = [serve.Request(0, 0.0, 9, 64, 60.0, 1.0)]
    be, res, summ = _run(reqs, memory_budget=10 ** 9)
    r = res[0]
    assert r.converged and r.steps == 4000
    assert abs(r.theta_measured - (60 + 10 * math.exp(-8))) < 1e-12
    assert summ["converged"] == 1 and be.closed == [0]


def test_not_converged_at_the_step_cap():
    reqs = [serve.Request(0, 0.0, 19, 16, 60.0, 1.0)]
    be, res, summ = _run(reqs, memory_budget=10 ** 9, amp=1000.0, decay=1e5, max_steps=5000)
    assert not res[0].converged and res[0].steps == 5000


def test_fifo_admission_under_the_memory_budget():
    """Budget for two 64^2 cases at a time: the third waits for a retirement,
    and admissions follow arrival order."""
    reqs = [serve.Request(i, 0.01 * i, 9, 64, 30.0 + 10 * i, 1.0) for i in range(5)]
    budget = 2 * 64 * 64 * 100
    be, res, summ = _run(reqs, memory_budget=budget)
    assert be.opened == [0, 1, 2, 3, 4]
    assert be.max_live_bytes <= budget
    assert summ["peak_active"] == 2
    for a, b in zip(res, res[1:]):
        assert a.admitted <= b.admitted
    assert res[2].admitted >= min(res[0].finished, res[1].finished)
    assert all(r.converged for r in res)


def test_max_active_and_continuous_batching():
    """Cases join and leave a running batch; each membership change rebuilds
    only its own lattice's batch."""
    reqs = [serve.Request(i, 0.0, 9 if i % 2 else 19, 32, 90.0, 1.0) for i in range(6)]
    be, res, summ = _run(reqs, memory_budget=10 ** 12, max_active=3)
    assert summ["peak_active"] == 3
    for lat, members in be.batches_made:
        assert len(members) <= 3 and all(reqs[m].lattice == lat for m in members)
    assert sorted(be.closed) == list(range(6))


def test_latency_and_throughput_bookkeeping():
    """One case alone: latency = its steps x nodes / rate (+ no queueing),
    MLUPS = rate / 1e6."""
    reqs = [serve.Request(0, 0.5, 9, 100, 45.0, 1.0)]
    be, res, summ = _run(reqs, memory_budget=10 ** 12, rate=2e8)
    r = res[0]
    assert abs(r.latency - r.steps * 100 * 100 / 2e8) < 1e-5       # + the idle loop's sleep quantum
    assert summ["mlups"] == pytest.approx(200.0, rel=0.01)
    assert abs(summ["node_steps"] - r.steps * 100 * 100) == 0
    assert r.admitted == pytest.approx(0.5, abs=0.06)


def test_request_larger_than_the_budget_is_an_error():
    reqs = [serve.Request(0, 0.0, 19, 64, 45.0, 1.0)]
    with pytest.raises(ValueError):
        _run(reqs, memory_budget=1000)


def test_request_case_geometry():
    """The drop of a request meets the solid at the requested angle: for the
    two circles, (R^2 + r^2 - d^2) / (2 R r) = cos(theta), the law of cosines
    in the triangle of the two centres and a contact point."""
    q = serve.Request(0, 0.0, 9, 200, 120.0, 1000.0)
    c = serve.request_case(q)
    R, r = c["R"], c["R0"]
    d = math.dist(c["drop_center"][:2], c["solid_center"][:2])
    assert abs((R * R + r * r - d * d) / (2 * R * r) - math.cos(math.radians(120.0))) < 1e-12
    P = c["params"]
    assert P["rho_l"] == 1000.0 and P["mu_l"] / P["mu_g"] == 100.0
    assert P["mu_l"] / P["rho_l"] >= 0.01 - 1e-15
    assert c["fluid_nodes"] == int((c["solid"] == 0).sum())


def test_failed_and_unmeasurable_cases():
    """A non-finite state retires the case as failed at its next check; an
    angle that cannot be measured (NaN) neither converges nor fails it."""
    class Odd(FakeBackend):
        def angle_deg(self, h):
            if h["req"].rid == 0:
                return None
            if h["req"].rid == 1:
                return float("nan")
            return super().angle_deg(h)
    clk = SimClock()
    be = Odd(clk)
    reqs = [serve.Request(i, 0.0, 9, 32, 60.0, 1.0) for i in range(3)]
    res, summ = serve.Server(be, 10 ** 9, max_steps=5000, clock=clk, sleep=clk.sleep).run(reqs)
    assert res[0].failed and not res[0].converged and res[0].steps == 1000
    assert not res[1].failed and not res[1].converged and res[1].steps == 5000
    assert res[2].converged
    assert summ["failed"] == 1 and summ["converged"] == 1


def test_batches_never_hold_more_slots_than_the_table():
    """Rebuilding one lattice's batch while the other's old batch is still
    open could ask for more slots than exist; all dirty batches close first."""
    class Slots(FakeBackend):
        live = 0
        peak = 0

        def batch(self, lattice, handles):
            Slots.live += len(handles)
            Slots.peak = max(Slots.peak, Slots.live)
            return super().batch(lattice, handles)

        def close_batch(self, b):
            Slots.live -= len(b)
    clk = SimClock()
    be = Slots(clk)
    reqs = [serve.Request(i, 0.001 * i, 9 if i % 3 else 19, 24 + (i % 7), 60.0, 1.0) for i in range(40)]
    serve.Server(be, 10 ** 12, max_active=8, clock=clk, sleep=clk.sleep).run(reqs)
    assert Slots.peak <= 8 and Slots.live == 0


class OomError(RuntimeError):
    """Stands in for lbm.LbmError(LBM_ERR_OOM) from lbm_create_domain."""


def test_allocation_failure_mid_stream_retires_only_that_request():
    """Request 3's domain creation fails with an out-of-memory error while
    others are running: it is retired as failed at once, the rest converge,
    and the budget bookkeeping stays balanced (nothing was charged for it)."""
    class FailingOpen(FakeBackend):
        def open(self, req, case):
            if req.rid == 3:
                raise OomError("LBM_ERR_OOM: cudaMalloc of %d bytes failed" % case["bytes"])
            return super().open(req, case)
    clk = SimClock()
    be = FailingOpen(clk)
    reqs = [serve.Request(i, 0.002 * i, 9 if i % 2 else 19, 32 + i, 40.0 + 5 * i, 1.0) for i in range(7)]
    res, summ = serve.Server(be, 10 ** 12, max_active=4, clock=clk, sleep=clk.sleep).run(reqs)
    bad = res[3]
    assert bad.failed and not bad.converged and bad.steps == 0
    assert "OomError" in bad.error and "LBM_ERR_OOM" in bad.error
    assert bad.finished >= bad.arrival and math.isnan(bad.admitted)
    assert all(r.converged and not r.failed for k, r in enumerate(res) if k != 3)
    assert summ["failed"] == 1 and summ["converged"] == 6
    assert 3 not in be.opened and sorted(be.closed) == [0, 1, 2, 4, 5, 6]
    assert be.live_bytes == 0
    for lat, members in be.batches_made:
        assert 3 not in members


def test_device_failure_in_a_chunk_retires_that_case():
    """The backend's wait reports one case's device state as failed (as the GPU
    backend does for LBM_ERR_UNSTABLE or LBM_ERR_TIMEOUT): that case retires as
    failed after the chunk, its batch is rebuilt without it, the others go on."""
    class FailingDevice(FakeBackend):
        def wait(self, batches):
            super().wait(batches)
            return [h for b in batches for h in b if h["req"].rid == 1 and h["steps"] >= 600]
    clk = SimClock()
    be = FailingDevice(clk)
    reqs = [serve.Request(i, 0.0, 9, 40, 60.0, 1.0) for i in range(4)]
    res, summ = serve.Server(be, 10 ** 12, clock=clk, sleep=clk.sleep).run(reqs)
    assert res[1].failed and res[1].steps == 600 and res[1].error == "device state failed"
    assert all(r.converged for k, r in enumerate(res) if k != 1)
    assert sorted(be.closed) == [0, 1, 2, 3] and be.live_bytes == 0
    later = [m for lat, m in be.batches_made[1:]]
    assert later and all(1 not in m for m in later)


def test_prepare_failure_is_a_failed_request():
    class FailingPrepare(FakeBackend):
        def prepare(self, req):
            if req.rid == 0:
                raise ValueError("bad geometry")
            return super().prepare(req)
    clk = SimClock()
    be = FailingPrepare(clk)
    reqs = [serve.Request(i, 0.0, 19, 24, 60.0, 1.0) for i in range(2)]
    res, summ = serve.Server(be, 10 ** 12, clock=clk, sleep=clk.sleep).run(reqs)
    assert res[0].failed and "bad geometry" in res[0].error and res[1].converged
    assert be.opened == [1]
