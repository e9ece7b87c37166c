"""Serving loop: wetting cases arrive over time and are advanced in continuous
batches until their contact angle has converged.

A request is a drop on a cylinder (D2Q9) or on a sphere (D3Q19), placed at
the spherical-cap shape that meets the solid at the requested angle (the
paper starts its cases at the analytic equilibrium shape, Sec. III).  The
server

  * admits requests first come, first served while the device footprint of
    every admitted case (lbm_domain_bytes) fits a memory budget and the batch
    table has room,
  * advances every admitted case of a lattice in one batch (one launch per
    phase for all of them), the two lattices' batches on their own streams,
  * rebuilds a batch whenever a case joins or leaves it (continuous
    batching: a case never waits for the others of its batch),
  * measures each case's contact angle every `check_every` of its steps and
    retires it once the angle moved less than `tol_deg` since the previous
    check (converged), or at `max_steps` (not converged).

Time to converged is the wall time from a request's arrival to the chunk
boundary at which its convergence was seen.  The scheduler talks to the
simulation through a small backend interface, so its logic runs on the CPU
against a stand-in backend in tests.
"""
import collections
import dataclasses
import math
import time

import numpy as np

from . import workloads as wl


# ---------------------------------------------------------------- requests

@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    lattice: int            # 9 (drop on a cylinder) or 19 (drop on a sphere)
    L: int                  # box edge: L x L (2D) or L x L x L (3D)
    theta_deg: float
    rho_ratio: float


def poisson_requests(n=200, rate=20.0, seed=3, L2=(128, 1024), L3=(64, 192), ratio=(1.0, 1000.0),
                     theta=(20.0, 160.0)):
    """n requests with exponential inter-arrival times of mean 1/rate, half
    D2Q9 with L ~ U(L2) and half D3Q19 with L ~ U(L3) (in random order),
    theta ~ U(theta) degrees, density ratio log-uniform on `ratio`."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    kinds = rng.permutation(np.arange(n) % 2)
    out = []
    for i in range(n):
        lat = 9 if kinds[i] == 0 else 19
        lo, hi = L2 if lat == 9 else L3
        L = int(rng.integers(lo, hi + 1))
        th = float(rng.uniform(*theta))
        r = float(math.exp(rng.uniform(math.log(ratio[0]), math.log(ratio[1]))))
        out.append(Request(i, float(t[i]), lat, L, th, r))
    return out


def request_case(req, precision=1, sigma=0.01, W=4.0, M_phi=0.02, solid_frac=0.10, drop_frac=0.16):
    """Parameters, geometry and initial drop of a request.

    Cylinder / sphere of radius solid_frac*L at the box centre, drop of radius
    drop_frac*L centred on the +y (2D) or +z (3D) axis at the distance where
    the two circles / spheres meet at theta; all periodic.  These fractions
    keep the drop's apex at most 0.42 L from the box centre at theta = 160 deg
    (clear of its periodic image) and its cap at least 0.13 L high at
    theta = 20 deg.  rho_g = 1,
    mu_g = 0.1; mu_l/mu_g = clip(rho_ratio/10, 1, 100), which keeps the liquid
    kinematic viscosity >= 0.01 (tau >= 0.53) over the whole ratio range and
    gives the paper's mu ratio 100 at density ratio 1000."""
    L = req.L
    R, r = solid_frac * L, drop_frac * L
    if req.lattice == 9:
        shape, center, axis = (1, L, L), (L / 2.0, L / 2.0, 0.0), 1
    else:
        shape, center, axis = (L, L, L), (L / 2.0, L / 2.0, L / 2.0), 2
    solid, ghosts = wl.sphere_domain(req.lattice, shape, center, R)
    mu_g = 0.1
    mu_l = mu_g * min(max(req.rho_ratio / 10.0, 1.0), 100.0)
    params = dict(lattice=req.lattice, nx=L, ny=L, nz=1 if req.lattice == 9 else L, periodic=7,
                  precision=precision, rho_l=req.rho_ratio, rho_g=1.0, mu_l=mu_l, mu_g=mu_g, sigma=sigma,
                  W=W, M_phi=M_phi, theta=math.radians(req.theta_deg), g=(0, 0, 0))
    drop = wl.droplet_on_sphere_center(center, R, r, math.radians(req.theta_deg), axis=axis)
    normal = [0.0, 0.0, 0.0]
    normal[axis] = 1.0
    cap = math.dist(drop, center) + r - R                     # apex height above the solid surface
    return dict(params=params, solid=solid, ghosts=ghosts, drop_center=tuple(drop), R0=r, solid_center=center,
                R=R, normal=tuple(normal), cap_height=cap, fluid_nodes=int((solid == 0).sum()))


# ---------------------------------------------------------------- backend on the GPU

class GpuBackend:
    """Cases are lbm.Domain objects; each lattice's cases share one CUDA stream
    and one lbm.Batch (batched=True), or are stepped one after the other by
    their own launches (batched=False, the per-case baseline)."""

    def __init__(self, precision=1, exclude=6.0, keep_final=False, batched=True):
        """exclude: interface points nearer the solid than min(exclude, half
        the drop's initial cap height) are left out of the contact-angle fit."""
        import torch
        from . import lbm
        self.lbm, self.torch = lbm, torch
        self.batched = batched
        self.precision = precision
        self.exclude = exclude
        self.keep_final = keep_final                     # keep each case's final color field (tests)
        self.final = {}
        self.streams = {9: torch.cuda.Stream(), 19: torch.cuda.Stream()}
        self._handles = {}                               # id(domain) -> handle

    def prepare(self, req):
        case = request_case(req, precision=self.precision)
        case["bytes"] = self.lbm.domain_bytes(case["params"], len(case["ghosts"][0]))
        return case

    def open(self, req, case):
        # the workspace is allocated on the stream that will use it, so the
        # caching allocator orders its reuse after that stream's work
        with self.torch.cuda.stream(self.streams[req.lattice]):
            d = self.lbm.Domain(case["params"], case["solid"], case["ghosts"], stream=self.streams[req.lattice])
        d.init_droplet(case["drop_center"], case["R0"])
        probe = self.lbm.make_probe(1, case["solid_center"], case["R"], case["normal"],
                                    min(self.exclude, 0.5 * case["cap_height"]))
        case["solid"] = case["ghosts"] = None           # host copies are no longer needed
        h = dict(domain=d, probe=probe, rid=req.rid)
        self._handles[id(d)] = h
        return h

    def batch(self, lattice, handles):
        if not self.batched:
            return [h["domain"] for h in handles]
        return self.lbm.Batch([h["domain"] for h in handles], stream=self.streams[lattice])

    def close_batch(self, b):
        if self.batched:
            b.close()

    def launch(self, batches, n):
        for b in batches:                                # asynchronous; the lattices overlap
            if self.batched:
                b.step(n)
            else:
                for d in b:
                    d.step(n)

    def wait(self, batches):
        """Wait for the chunk; returns the handles of the cases whose device
        state failed in it (a non-finite value, LBM_ERR_UNSTABLE, or a halo
        copy that timed out, LBM_ERR_TIMEOUT).  The other cases go on."""
        lbm = self.lbm
        bad = []
        for b in batches:
            doms = b.domains if self.batched else b
            try:
                if self.batched:
                    b.sync()
                else:
                    for d in doms:
                        d.sync()
                continue
            except lbm.LbmError as e:
                if e.status not in (lbm.LBM_ERR_UNSTABLE, lbm.LBM_ERR_TIMEOUT):
                    raise
            for d in doms:                               # the batch names only its first failure
                try:
                    d.sync()
                except lbm.LbmError as e:
                    if e.status not in (lbm.LBM_ERR_UNSTABLE, lbm.LBM_ERR_TIMEOUT):
                        raise
                    bad.append(self._handles[id(d)])
        return bad

    def angle_deg(self, h):
        """Contact angle in degrees; NaN when no interface could be fitted, None
        when the state went non-finite."""
        dg = h["domain"].diagnostics(h["probe"])
        if dg["nan_flag"]:
            return None
        return math.degrees(dg["contact_angle"])

    def close(self, h):
        if self.keep_final:
            self.final[h["rid"]] = {f: h["domain"].read(f) for f in ("N", "B", "phi", "u", "p")}
        self._handles.pop(id(h["domain"]), None)
        h["domain"].close()


# ---------------------------------------------------------------- scheduler

@dataclasses.dataclass
class Result:
    rid: int
    lattice: int
    L: int
    arrival: float
    admitted: float = float("nan")
    finished: float = float("nan")
    steps: int = 0
    converged: bool = False
    failed: bool = False
    theta_set: float = float("nan")
    theta_measured: float = float("nan")
    fluid_nodes: int = 0
    error: str = ""

    @property
    def latency(self):
        return self.finished - self.arrival


class Server:
    def __init__(self, backend, memory_budget, chunk=200, check_every=1000, tol_deg=0.1, max_steps=20000,
                 max_active=96, clock=time.perf_counter, sleep=time.sleep):
        if check_every % chunk:
            raise ValueError("check_every must be a multiple of chunk")
        self.backend = backend
        self.memory_budget = memory_budget
        self.chunk, self.check_every = chunk, check_every
        self.tol_deg, self.max_steps, self.max_active = tol_deg, max_steps, max_active
        self.clock, self.sleep = clock, sleep

    def run(self, requests):
        """Serve every request; returns (results in request order, summary dict)."""
        be = self.backend
        t0 = self.clock()
        now = lambda: self.clock() - t0                          # noqa: E731
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
        waiting = collections.deque()                            # arrived, not admitted: (req, case)
        active = {9: [], 19: []}                                 # lattice -> list of entries
        batches = {}
        dirty = set()
        used_bytes = 0
        results = {q.rid: Result(q.rid, q.lattice, q.L, q.arrival, theta_set=q.theta_deg) for q in requests}
        node_steps = 0
        n_rebuilds = 0
        peak_active = 0
        phase = collections.Counter()                            # host seconds per phase of the loop

        def timed(name, fn, *a):
            t1 = self.clock()
            out = fn(*a)
            phase[name] += self.clock() - t1
            return out

        def give_up(q, exc):
            """A request whose set-up failed is retired as failed; the others go on."""
            r = results[q.rid]
            r.failed, r.finished, r.error = True, now(), "%s: %s" % (type(exc).__name__, exc)

        def arrivals():
            t = now()
            while pending and pending[0].arrival <= t:
                q = pending.popleft()
                try:
                    waiting.append((q, timed("prepare", be.prepare, q)))
                except Exception as exc:                     # noqa: BLE001 -- reported in the result
                    give_up(q, exc)

        while pending or waiting or active[9] or active[19]:
            arrivals()
            # first come, first served while the head fits
            while waiting:
                q, case = waiting[0]
                n_act = len(active[9]) + len(active[19])
                if case["bytes"] > self.memory_budget:
                    raise ValueError("request %d needs %d bytes, more than the whole budget" % (q.rid, case["bytes"]))
                if used_bytes + case["bytes"] > self.memory_budget or n_act >= self.max_active:
                    break
                waiting.popleft()
                try:
                    h = timed("open", be.open, q, case)
                except Exception as exc:                     # noqa: BLE001 -- e.g. LBM_ERR_OOM
                    give_up(q, exc)
                    continue
                used_bytes += case["bytes"]
                active[q.lattice].append(dict(req=q, h=h, bytes=case["bytes"], steps=0, prev=None,
                                              fluid=case["fluid_nodes"]))
                results[q.rid].admitted = now()
                results[q.rid].fluid_nodes = case["fluid_nodes"]
                dirty.add(q.lattice)
            peak_active = max(peak_active, len(active[9]) + len(active[19]))
            if not (active[9] or active[19]):
                if pending:
                    timed("idle", self.sleep, max(0.0, min(pending[0].arrival - now(), 0.05)))
                continue
            for lat in dirty:                                     # close first: their slots are reused
                if lat in batches:
                    timed("rebuild", be.close_batch, batches.pop(lat))
            for lat in dirty:
                if active[lat]:
                    batches[lat] = timed("rebuild", be.batch, lat, [e["h"] for e in active[lat]])
                    n_rebuilds += 1
            dirty.clear()
            running = [batches[lat] for lat in (9, 19) if lat in batches]
            timed("launch", be.launch, running, self.chunk)
            arrivals()                                    # host-side set-up overlaps the chunk
            broken = {id(h) for h in (timed("wait", be.wait, running) or ())}
            for lat in (9, 19):
                keep = []
                for e in active[lat]:
                    e["steps"] += self.chunk
                    node_steps += e["fluid"] * self.chunk
                    done = False
                    if id(e["h"]) in broken:                   # device state failed in this chunk
                        r = results[e["req"].rid]
                        done, r.failed, r.error = True, True, "device state failed"
                    elif e["steps"] % self.check_every == 0:
                        th = timed("check", be.angle_deg, e["h"])
                        r = results[e["req"].rid]
                        if th is None:                           # non-finite state: the case failed
                            done, r.failed = True, True
                        else:
                            r.theta_measured = th
                            if math.isfinite(th) and e["prev"] is not None and abs(th - e["prev"]) < self.tol_deg:
                                done, r.converged = True, True
                            e["prev"] = th if math.isfinite(th) else None
                    if not done and e["steps"] >= self.max_steps:
                        done = True
                    if done:
                        r = results[e["req"].rid]
                        r.finished, r.steps = now(), e["steps"]
                        timed("retire", be.close, e["h"])
                        used_bytes -= e["bytes"]
                        dirty.add(lat)
                    else:
                        keep.append(e)
                active[lat] = keep
            for lat in list(dirty):
                if not active[lat] and lat in batches:
                    be.close_batch(batches.pop(lat))
        for b in batches.values():
            be.close_batch(b)
        res = [results[q.rid] for q in requests]
        # the served span: first arrival to last completion
        wall = max(r.finished for r in res) - min(r.arrival for r in res) if res else 0.0
        lat = np.array([r.latency for r in res]) if res else np.zeros(1)
        summary = dict(requests=len(res), converged=int(sum(r.converged for r in res)),
                       failed=int(sum(r.failed for r in res)), wall_s=wall,
                       p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                       mean_s=float(lat.mean()), mlups=node_steps / wall / 1e6 if wall > 0 else 0.0,
                       node_steps=int(node_steps), batch_rebuilds=n_rebuilds, peak_active=peak_active,
                       steps_mean=float(np.mean([r.steps for r in res])) if res else 0.0,
                       host_seconds={k: round(v, 3) for k, v in sorted(phase.items())})
        return res, summary
