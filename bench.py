#!/usr/bin/env python
"""Throughput of the fused color-gradient wetting step on GB300.

Workload: D3Q19 192^3, solid sphere R = 32 at the box centre, drop R0 = 24 on
its +z pole placed at the contact angle (60 deg by default), density ratio 1000,
viscosity ratio 100, sigma = 0.005, FP32, all axes periodic.  One step = one
full time step of the hot path (ghost update, fused collide/segregate/stream
kernel, color kernel) over the whole grid.  MLUPS counts every node of the grid
(solid included), as the paper's Eq. (MLUPSDefinition).

Further objects of the same JSON line (rank 0, one GPU): the same case over
its five contact angles, FP32 against FP64 after 400 steps and FP32 on to 20000
(`theta_sweep`); the other population storage on the same case; the 64
batched cases; the paper's Table I grids; the 256^3 sphere-packing
imbibition, FP32 and FP16 storage against an FP64 reference (`packing`); the
served Poisson request stream (`serving`).

With torchrun (N > 1) every rank runs an independent case (the next contact
angle of the sweep 30..150 deg) -- replicas with no collective on the data path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline at <=0.5 deg contact-angle error; served p50/p99 latency"
THETA_SWEEP = [60.0, 30.0, 90.0, 120.0, 150.0]
N_GRID, R_SPHERE, R_DROP = 192, 32.0, 24.0
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_step_d3q19_traffic.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--theta", type=float, default=None)
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-case batched measurement")
    ap.add_argument("--batch-steps", type=int, default=5000, help="timed steps of the 64-case batch (each arm)")
    ap.add_argument("--batch-cases", type=int, default=64,
                    help="the 64-case batch over its first this many cases (64: all; fewer for profiling a small batch)")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests of the served workload (Poisson arrivals at 20/s); 0 skips it")
    ap.add_argument("--serve-plain", action="store_true",
                    help="also serve the same stream with per-case launches instead of batches")
    ap.add_argument("--no-table", action="store_true", help="skip the paper's Table I grids")
    ap.add_argument("--no-other-storage", action="store_true",
                    help="skip the run of the same case with the other population storage (fp16 / fp32)")
    ap.add_argument("--table-steps", type=int, default=2000)
    ap.add_argument("--sweep-steps", type=int, default=20000,
                    help="contact-angle sweep 30..150 deg of the bench case for this many FP32 steps (0 skips it)")
    ap.add_argument("--sweep-fp64-steps", type=int, default=400,
                    help="steps of the FP32-vs-FP64 comparison within the sweep (and of the bench line's "
                         "contact-angle check)")
    ap.add_argument("--packing-steps", type=int, default=5000,
                    help="run the 256^3 sphere-packing imbibition for this many steps with FP32 and FP16 "
                         "storage (0 skips it)")
    ap.add_argument("--packing-fp64-steps", type=int, default=200,
                    help="steps of the FP64 reference run of the packing")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16"],
                    help="population storage: fp32 (the bench default) or fp16 (shifted, scaled)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

_T0 = time.perf_counter()


def note(phase):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print("[bench %7.1f s] %s" % (time.perf_counter() - _T0, phase), file=sys.stderr, flush=True)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        """Rows sampled since start()."""
        if self.proc is None:
            return []
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.file.read())) if len(r) >= 9]
        self.file.close()
        os.unlink(self.file.name)
        self.proc = None
        return rows

    @staticmethod
    def summary(rows, window):
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "window": window}


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            v = json.load(f).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in ("lbm_kernels.cuh", "lbm_kernels_pair.cuh", "lbm_lattice.cuh", "lbm_launch.cuh",
                 "lbm_launch_impl.cuh"):
        with open(os.path.join(ROOT, "paper_2605_30878_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(fluid_nodes, fp16=False):
    """DRAM bytes per k_step launch from the committed ncu summary (FP32, or
    FP16 population storage), scaled to this launch's fluid nodes; None if the
    kernel source changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_hash") != kernel_source_hash():
        return None
    if fp16:
        rec = rec.get("k_step_fp16_storage")
        if rec is None:
            return None
    return rec["dram_bytes_per_fluid_node"] * fluid_nodes


def k_step_bytes_per_fluid_node(Q, D, s, contrast, moving=None, rest=None):
    """Algorithmic bytes of one k_step launch per fluid node (float arithmetic):
    pull the Q - 1 moving populations of N (moving bytes each: s, or 2 with FP16
    storage) -- the deviation form takes the pressure and every moment from
    them, so the rest population is not read, and the collision needs B only
    through phi, which k_phi computed --, write N* and B* (rest + (Q - 1)
    moving bytes each; the rest plane is float), read phi (s), read the previous
    u (D s, only with a density contrast), write u (D s) and p (s), read the
    4-byte bounce-back mask."""
    moving = s if moving is None else moving
    rest = s if rest is None else rest
    pop = rest + (Q - 1) * moving
    return (Q - 1) * moving + 2 * pop + s + (D * s if contrast else 0) + D * s + s + 4


def workload(theta, precision, n=N_GRID):
    from paper_2605_30878_gb300 import workloads as wl
    scale = n / float(N_GRID)
    return wl.sphere_config(n=n, R=R_SPHERE * scale, R0=R_DROP * scale, theta_deg=theta, rho_ratio=1000.0,
                            mu_ratio=100.0, sigma=0.005, precision=precision)


def max_over_ranks(value, dist=None, device="cuda"):
    """The largest `value` over all ranks (the slowest rank's time); value itself
    without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, steps, world, ms_max):
    """Whole-job throughput of `world` replicas, each advancing nodes_per_rank
    nodes `steps` steps, timed by the slowest rank."""
    return nodes_per_rank * steps * world / (ms_max * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ CPU oracle

def time_oracle(cfg, min_seconds, max_steps, warmup=1):
    import oracle
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    o.step(warmup)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        o.step(1)
        steps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    nn = cfg["solid"].size
    return nn * steps / dt / 1e6, steps, dt


def cores_used():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


# device state per grid node of the bench case (populations, fields, tables):
# 349 B with FP32 storage, 205 B with FP16 storage at 192^3
STATE_BYTES_PER_NODE = {"fp32": 349.2, "fp16": 205.2}


def arm_config(n, theta, storage, world):
    """The bench line's `config`, the same in both arms."""
    return {"workload": "D3Q19 %d^3 drop on sphere: sphere R=%g at the centre, drop R0=%g on the +z pole "
                        "at theta=%g deg, rho_l/rho_g=1000, mu_l/mu_g=100, sigma=0.005, %s, periodic"
                        % (n, R_SPHERE * n / N_GRID, R_DROP * n / N_GRID, theta,
                           "FP32" if storage == "fp32" else "FP32 arithmetic, FP16 populations"),
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (%.2f GB state vs 129 MB L2)" % (n ** 3 * STATE_BYTES_PER_NODE[storage] / 1e9)}


def run_reference(args):
    """The oracle, as it stands, on the host cores: each timed step is one full
    oracle time step of a scaled replica of the workload (same geometry ratios
    and physics), sized so warm-up + timed steps take about two minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    theta = args.theta if args.theta is not None else THETA_SWEEP[0]
    probe_cfg = workload(theta, 1, n=32)
    rate32, _, _ = time_oracle(probe_cfg, 0.5, 3)
    budget_s = 120.0
    n_ref = int((budget_s * rate32 * 1e6 / max(1, args.steps + args.warmup)) ** (1.0 / 3.0))
    n_ref = max(24, min(N_GRID, n_ref - n_ref % 8))
    cfg = workload(theta, 1, n=n_ref)
    import oracle
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    nn = n_ref ** 3
    value = nn * args.steps / dt / 1e6
    sample = ("D3Q19 %d^3 replica of the 192^3 drop-on-sphere workload (sphere R=%.1f, drop R0=%.1f, theta=%g deg, "
              "density ratio 1000), %d oracle steps after %d warm-up" % (n_ref, R_SPHERE * n_ref / N_GRID,
                                                                          R_DROP * n_ref / N_GRID, theta,
                                                                          args.steps, args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args.n, theta, args.storage, 1),
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched cases

DIAG = tuple(1.0 / math.sqrt(3.0) for _ in range(3))


def drop_radius_fitting(n, R, theta_deg, want, margin=3.0):
    """The largest drop radius <= want for a cap on a sphere of radius R at the
    centre of an n^3 periodic box, meeting it at theta with its centre on the
    box diagonal (d^2 = R^2 + r^2 - 2 R r cos(theta) from the sphere centre),
    whose extent along every axis, d / sqrt(3) + r, stays `margin` inside half
    the box: each interface point then lies within half a box of the sphere
    centre, the image the contact-angle fit takes."""
    c = math.cos(math.radians(theta_deg))
    extent = lambda r: math.sqrt(R * R + r * r - 2.0 * R * r * c) / math.sqrt(3.0) + r     # noqa: E731
    limit = 0.5 * n - margin
    if extent(want) <= limit:
        return want
    lo, hi = 0.0, want
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if extent(mid) <= limit else (lo, mid)
    return lo


def batch_cases(seed=2, count=64):
    """64 independent D3Q19 drop-on-sphere cases: grid n ~ U{48..128}, sphere
    R = U(0.2, 0.3) n at the centre, theta ~ U(20, 160) deg, density ratio in
    {1, 10, 1000} (viscosity ratio 100 at 1000, else 1), FP32.  The drop sits
    on the sphere along the box diagonal (the direction with the most room
    before its periodic image), radius 0.75 R or less where a cap that large
    would leave half the box along some axis (high angles, small boxes)."""
    from paper_2605_30878_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(48, 129))
        R = float(rng.uniform(0.2, 0.3) * n)
        theta = float(rng.uniform(20.0, 160.0))
        ratio = float(rng.choice([1.0, 10.0, 1000.0]))
        r0 = drop_radius_fitting(n, R, theta, 0.75 * R)
        cfg = wl.sphere_config(n=n, R=R, R0=r0, theta_deg=theta, rho_ratio=ratio,
                               mu_ratio=100.0 if ratio == 1000.0 else 1.0, precision=1)
        d = math.sqrt(R * R + r0 * r0 - 2.0 * R * r0 * math.cos(math.radians(theta)))
        cfg["drop_center"] = tuple(cfg["solid_center"][a] + d * DIAG[a] for a in range(3))
        cfg["axis"] = DIAG
        out.append(cfg)
    return out


def run_batch_bench(lbm, steps, count=64):
    """The 64-case batch: aggregate MLUPS of the 64 cases advanced in one batch (one
    launch per phase, tile shape autotuned) against a second copy of the same
    cases each stepped by its own launches, for the same number of steps; then
    the contact angle of every case from both copies."""
    import torch
    cfgs = batch_cases()[:count]

    def make():
        out = []
        for c in cfgs:
            d = lbm.Domain(c["params"], c["solid"], c["ghosts"])
            d.init_droplet(c["drop_center"], c["R0"])
            out.append(d)
        return out
    plain, batched = make(), make()
    nodes = sum(int((c["solid"] == 0).sum()) for c in cfgs)      # fluid nodes, as the main metric
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    b = lbm.Batch(batched)
    chosen, trial_ms = b.tune(steps_per_trial=10)                 # advances every case
    lead = lbm.BATCH_TILE_SHAPES * 11
    for d in plain:
        d.step(lead)                                              # the same steps, untimed
    torch.cuda.synchronize()
    ev[0].record(stream)
    for d in plain:
        d.step(steps)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t_plain = ev[0].elapsed_time(ev[1]) * 1e-3
    ev[2].record(stream)
    b.step(steps)
    ev[3].record(stream)
    torch.cuda.synchronize()
    t_batch = ev[2].elapsed_time(ev[3]) * 1e-3
    b.sync()
    # contact angle of every case from both copies, with the serving loop's
    # estimator: interface points nearer the sphere than min(1.5 W, half the
    # drop's initial cap height) are left out of the fit
    dtheta, err_set, per_case = [], [], []
    n_unmeasured = 0
    for c, dp, db in zip(cfgs, plain, batched):
        cap = math.dist(c["drop_center"], c["solid_center"]) + c["R0"] - c["R"]
        probe = lbm.make_probe(1, c["solid_center"], c["R"], c["axis"], min(6.0, 0.5 * cap))
        gp, gb = dp.diagnostics(probe), db.diagnostics(probe)
        tp, tb = math.degrees(gp["contact_angle"]), math.degrees(gb["contact_angle"])
        th_set = math.degrees(c["params"]["theta"])
        per_case.append({"n": c["params"]["nx"], "theta_set": round(th_set, 3),
                         "rho_ratio": c["params"]["rho_l"] / c["params"]["rho_g"],
                         "theta_batched": None if math.isnan(tb) else round(tb, 4),
                         "theta_plain": None if math.isnan(tp) else round(tp, 4),
                         "n_fit": int(gb["n_fit"]), "nan_flag": int(gb["nan_flag"])})
        if math.isnan(tp) or math.isnan(tb):
            n_unmeasured += 1                                     # reported, never counted as agreement
            continue
        dtheta.append(abs(tb - tp))
        err_set.append(abs(tb - th_set))
    res = {"cases": len(cfgs), "nodes": nodes, "steps": steps, "steps_before_timing": lead,
           "mlups_batched": nodes * steps / t_batch / 1e6, "mlups_plain": nodes * steps / t_plain / 1e6,
           "speedup": t_plain / t_batch, "tile_shape_chosen": int(chosen),
           "tune_ms_per_step": [round(float(x), 4) for x in trial_ms],
           "launches_per_step_batched": b.launches_per_step(),
           "launches_per_step_plain": sum(d.launches_per_step() for d in plain),
           "contact_angle_batched_vs_plain_max_deg": max(dtheta) if dtheta else None,
           "contact_angle_measured_cases": len(dtheta), "contact_angle_unmeasured_cases": n_unmeasured,
           "contact_angle_vs_set_deg": {"median": float(np.median(err_set)) if err_set else None,
                                        "max": float(np.max(err_set)) if err_set else None,
                                        "measured": len(err_set)},
           "per_case": per_case}
    b.close()
    for d in plain + batched:
        d.close()
    torch.cuda.empty_cache()
    return res


def time_domain(dom, steps, warmup=20):
    """Seconds per step of dom.step over `steps` steps (CUDA events on its stream)."""
    import torch
    dom.step(warmup)
    dom.sync()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    dom.step(steps)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / steps


def run_other_storage(lbm, args, cfg, probe, n_angle, fp64_deg):
    """The bench case with the other population storage: ms per step (CUDA
    events, same K and W), its k_step against its own algorithmic bytes, and
    its contact angle after n_angle steps against FP64's."""
    import torch
    prec = lbm.FP32 if args.storage == "fp16" else lbm.FP16
    key = "fp32" if prec == lbm.FP32 else "fp16"
    P = dict(cfg["params"], precision=prec)
    d = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
    fluid = d.fluid_nodes()
    d.init_droplet(cfg["drop_center"], cfg["R0"])
    sec = time_domain(d, args.steps, warmup=args.warmup)
    kms = d.profile_steps(max(3, min(args.steps, 60)))
    t_step = kms[1] / max(3, min(args.steps, 60)) * 1e-3
    kb = k_step_bytes_per_fluid_node(19, 3, 4, True, 2 if prec == lbm.FP16 else 4) * fluid
    peak, peak_kind = hbm_peak()
    d.close()
    da = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
    da.init_droplet(cfg["drop_center"], cfg["R0"])
    da.step(n_angle)
    deg = math.degrees(da.diagnostics(probe)["contact_angle"])
    da.close()
    torch.cuda.empty_cache()
    n = cfg["params"]["nx"]
    return {"storage": key, "value": n ** 3 / sec / 1e6, "unit": "MLUPS", "ms_per_step": sec * 1e3,
            "k_step": {"avg_launch_ms": t_step * 1e3, "bytes_per_fluid_node": kb / fluid,
                       "traffic": recorded_traffic(fluid, fp16=prec == lbm.FP16),
                       "achieved_gbs": kb / t_step / 1e9, "frac": kb / t_step / 1e9 / peak, "peak_kind": peak_kind},
            "contact_angle_deg": deg, "vs_fp64_deg": abs(deg - fp64_deg) if fp64_deg is not None else None}


def run_theta_sweep(lbm, n, steps, fp64_steps, storage="fp32"):
    """The contact-angle sweep: the bench case (density ratio 1000) at theta =
    30, 60, 90, 120, 150 deg.  Per angle: the line's storage and FP64 from the
    same initial state for `fp64_steps` steps, their contact angles compared
    (the metric's <= 0.5 deg reading: same discretisation, the two
    precisions); then the line's storage on to `steps` steps: measured angle
    against the set one, max |u| (the spurious current), MLUPS."""
    import torch
    prec = lbm.FP16 if storage == "fp16" else lbm.FP32
    out = {"steps": steps, "fp64_steps": fp64_steps, "storage": storage, "angles": []}
    for theta in (30.0, 60.0, 90.0, 120.0, 150.0):
        cfg = workload(theta, prec, n=n)
        probe = lbm.make_probe(1, (n / 2.0, n / 2.0, n / 2.0), R_SPHERE * n / N_GRID, (0, 0, 1), 6.0)
        row = {"theta_set_deg": theta}
        deg = {}
        for p_, key in ((prec, storage), (lbm.FP64, "fp64")):
            d = lbm.Domain(dict(cfg["params"], precision=p_), cfg["solid"], cfg["ghosts"])
            d.init_droplet(cfg["drop_center"], cfg["R0"])
            d.step(fp64_steps)
            dg = d.diagnostics(probe)
            deg[key] = math.degrees(dg["contact_angle"])
            row["n_fit_%s_at_fp64_steps" % key] = int(dg["n_fit"])
            if p_ == prec and steps > fp64_steps:
                sec = time_domain(d, steps - fp64_steps, warmup=0)
                dg = d.diagnostics(probe)
                row.update(theta_deg=math.degrees(dg["contact_angle"]), max_u=dg["max_u"],
                           n_fit=int(dg["n_fit"]), mlups=n ** 3 / sec / 1e6, nan_flag=dg["nan_flag"])
                row["vs_set_deg"] = abs(row["theta_deg"] - theta)
            d.close()
            torch.cuda.empty_cache()
        row["%s_deg_at_fp64_steps" % storage] = deg[storage]
        row["fp64_deg_at_fp64_steps"] = deg["fp64"]
        row["%s_vs_fp64_deg" % storage] = abs(deg[storage] - deg["fp64"])
        out["angles"].append(row)
        print("sweep", row, file=sys.stderr, flush=True)
    diffs = [r["%s_vs_fp64_deg" % storage] for r in out["angles"]]
    out["max_%s_vs_fp64_deg" % storage] = max(diffs)
    out["within_0p5_deg"] = bool(all(d <= 0.5 for d in diffs))
    return out


def run_paper_table(lbm, steps):
    """The paper's Table I grids of its two static wetting benchmarks (drop on
    a flat plate: walls at y = 0 and y = ny-1, periodic x, drop area 1e4 at
    500 x 300 scaled with the grid; drop on a cylinder: R = 0.2 L at the box
    centre, drop on its top, all periodic), density ratio 1000, viscosity ratio
    100, FP32 and FP64, MLUPS on every grid node as the paper counts them.  The
    smaller grids fit in the 129 MB L2."""
    from paper_2605_30878_gb300 import workloads as wl
    out = {}
    for name, nx, ny in (("plate", 500, 300), ("plate", 1000, 600), ("plate", 1500, 900),
                         ("cylinder", 201, 201), ("cylinder", 401, 401), ("cylinder", 601, 601)):
        shape = (1, ny, nx)
        if name == "plate":
            solid, ghosts = wl.wall_domain(9, shape, 1, 1)
            periodic = 1
            scale = nx / 500.0
            r = math.sqrt(1e4 / math.pi) * scale
            center = (nx / 2.0, 1.0 + 0.6 * r, 0.0)
        else:
            R = 0.2 * nx
            solid, ghosts = wl.sphere_domain(9, shape, (nx / 2.0, ny / 2.0, 0.0), R)
            periodic = 7
            r = 0.5 * R
            center = (nx / 2.0, ny / 2.0 + R + 0.5 * r, 0.0)
        row = {}
        for prec, key in ((lbm.FP32, "fp32"), (lbm.FP64, "fp64")):
            P = dict(lattice=9, nx=nx, ny=ny, nz=1, periodic=periodic, precision=prec, rho_l=1000.0, rho_g=1.0,
                     mu_l=10.0, mu_g=0.1, sigma=0.01, W=4.0, M_phi=0.02, theta=math.radians(60.0))
            d = lbm.Domain(P, solid, ghosts)
            d.init_droplet(center, r)
            sec = time_domain(d, steps)
            row[key + "_mlups"] = round(nx * ny / sec / 1e6, 1)
            d.close()
        out["%s %dx%d" % (name, nx, ny)] = row
    return out


def run_packing_bench(lbm, steps, checkpoints=10, fp64_steps=200):
    """The 256^3 sphere packing (radii U(8, 16), porosity 0.45 in x >= 24,
    seed 1): liquid slab 0 <= x < 16 (tanh, periodic image included) in the
    sphere-free reservoir, theta = 45 deg, density and viscosity ratio 1,
    sigma = 0.01, all periodic.  FP32 and FP16 population storage run `steps`
    steps; FP64 (about 45x slower on this GPU, whose FP64 units are few) runs
    the first `fp64_steps` as the reference.  Reported: the liquid saturation
    of the packing region (sum of phi over its fluid nodes / their count) at
    each checkpoint, its deviation from FP64 and from FP32, the phase-mass
    drift and MLUPS (every node of the grid)."""
    import torch
    from paper_2605_30878_gb300 import workloads as wl
    n = 256
    c, rad = wl.sphere_packing(n=n)
    solid, ghosts = wl.packing_domain(c, rad, n=n)
    fluid = solid.reshape(-1) == 0
    x = np.tile(np.arange(n), n * n)
    region = fluid & (x >= 24)
    d_slab = np.minimum(np.abs(x - 7.5), n - np.abs(x - 7.5))        # periodic distance to the slab centre
    phi0 = wl.tanh_field(8.0 - d_slab, 4.0)
    ref_marks = [fp64_steps // 2, fp64_steps]
    marks = sorted(set(ref_marks + [steps * (k + 1) // checkpoints for k in range(checkpoints)]))
    out = {"porosity_packing_region": float(1.0 - solid[:, :, 24:].mean()), "spheres": int(len(rad)),
           "ghost_nodes": int(len(ghosts[0])), "steps": steps, "checkpoints": marks}
    sat = {}
    for prec, key, last in ((lbm.FP32, "fp32", steps), (lbm.FP16, "fp16", steps), (lbm.FP64, "fp64", fp64_steps)):
        P = dict(lattice=19, nx=n, ny=n, nz=n, periodic=7, precision=prec, rho_l=1.0, rho_g=1.0, mu_l=0.1,
                 mu_g=0.1, sigma=0.01, W=4.0, M_phi=0.02, theta=math.radians(45.0))
        d = lbm.Domain(P, solid, ghosts)
        d.init_phi(phi0)
        m0 = d.diagnostics()["phi_sum"]
        sat[key] = []
        gpu_s, done = 0.0, 0
        for mk in marks:
            if mk > last:
                break
            gpu_s += time_domain(d, mk - done, warmup=0) * (mk - done)
            done = mk
            sat[key].append(float(d.read("phi")[region].mean()))
        dg = d.diagnostics()
        out[key] = {"steps": done, "mlups": round(n ** 3 * done / gpu_s / 1e6, 1),
                    "phi_sum_drift_rel": (dg["phi_sum"] - m0) / m0, "max_u": dg["max_u"], "nan_flag": dg["nan_flag"]}
        print("packing", key, out[key], file=sys.stderr, flush=True)
        d.close()
        torch.cuda.empty_cache()
    out["saturation"] = sat
    k64 = len(sat["fp64"])
    for key in ("fp32", "fp16"):
        out[key]["saturation_max_abs_dev_vs_fp64"] = float(np.max(np.abs(np.array(sat[key][:k64]) -
                                                                       np.array(sat["fp64"]))))
        out[key]["saturation_final"] = sat[key][-1]
    out["fp16"]["saturation_max_abs_dev_vs_fp32"] = float(np.max(np.abs(np.array(sat["fp16"]) -
                                                                        np.array(sat["fp32"]))))
    return out


def run_serve_bench(n_requests, batched=True):
    """The served workload: Poisson arrivals at 20/s (seed 3), half D2Q9 drops
    on cylinders (L ~ U{128..1024}^2), half D3Q19 drops on spheres
    (L ~ U{64..192}^3), theta ~ U(20, 160) deg, density ratio log-uniform on
    [1, 1000], FP32; each case runs until its contact angle moves less than
    0.1 deg per 1000 steps (cap 20000 steps).  Memory budget: 60% of the free
    device memory."""
    import torch
    from paper_2605_30878_gb300 import serve
    reqs = serve.poisson_requests(n=n_requests)
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(serve.GpuBackend(batched=batched), memory_budget=int(0.6 * free))
    res, summ = srv.run(reqs)
    errs = [abs(r.theta_measured - r.theta_set) for r in res if r.converged]
    out = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in summ.items()}
    out.update({"unit_latency": "s from arrival to converged", "mlups_unit": "fluid-node MLUPS over the served span",
                "theta_err_vs_set_deg": {"median": float(np.median(errs)) if errs else None,
                                         "max": float(np.max(errs)) if errs else None},
                "memory_budget_gb": round(srv.memory_budget / 1e9, 1)})
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch

    from paper_2605_30878_gb300 import build as lib_build
    from paper_2605_30878_gb300 import lbm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    lib_build.build()
    theta = args.theta if args.theta is not None else THETA_SWEEP[rank % len(THETA_SWEEP)]
    prec = lbm.FP16 if args.storage == "fp16" else lbm.FP32
    cfg = workload(theta, prec, n=args.n)
    P = cfg["params"]
    n = args.n
    nn = n ** 3
    probe = lbm.make_probe(1, (n / 2.0, n / 2.0, n / 2.0), R_SPHERE * n / N_GRID, (0, 0, 1), 6.0)
    ng = len(cfg["ghosts"][0])

    dom = lbm.Domain(P, cfg["solid"], cfg["ghosts"])
    fluid = dom.fluid_nodes()
    dom.init_droplet(cfg["drop_center"], cfg["R0"])
    dom.step(args.warmup)
    dom.sync()
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    start.record(stream)
    dom.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    rows = clocks.stop()
    ms = start.elapsed_time(end)
    dom.sync()
    ms = max_over_ranks(ms, dist)
    value = whole_job_mlups(nn, args.steps, world, ms)
    diag32 = dom.diagnostics(probe)
    window = "timed region"
    if len(rows) < 3:
        # A short timed region (20 steps take ~8 ms) holds no 200 ms sample:
        # sample the same steps again for about a second right after it, untimed.
        n_load = max(1, int(1000.0 / max(ms / args.steps, 1e-3)))
        clocks.start()
        dom.step(n_load)
        torch.cuda.synchronize()
        rows += clocks.stop()
        window = "timed region + %d untimed steps of the same case right after it (%.2f s)" % (
            n_load, n_load * ms / args.steps / 1e3)
    clk = ClockSampler.summary(rows, window)

    # dominant kernel timed kernel by kernel with CUDA events on the same stream
    prof_steps = max(3, min(args.steps, 60))
    kms = dom.profile_steps(prof_steps)
    t_step = kms[1] / prof_steps * 1e-3
    s, Q, D = 4, 19, 3
    sp = 2 if prec == lbm.FP16 else 4
    kb = k_step_bytes_per_fluid_node(Q, D, s, True, sp) * fluid
    achieved = kb / t_step / 1e9
    peak, peak_kind = hbm_peak()
    traffic = recorded_traffic(fluid, fp16=prec == lbm.FP16)
    share = kms / kms.sum()
    launches = dom.launches_per_step()
    bytes_step = dom.bytes_per_fluid_node()
    dom.close()
    del dom
    torch.cuda.empty_cache()

    line = None
    if rank == 0:
        # the contact-angle sweep over its five angles (FP32 vs FP64 at a fixed step count,
        # then the line's storage on); the bench case's own angle comes from it
        note("theta sweep")
        sweep = None
        n_angle = max(400, args.sweep_fp64_steps)
        if world == 1 and args.sweep_steps > 0 and not args.no_fp64_check:
            try:
                sweep = run_theta_sweep(lbm, n, max(args.sweep_steps, n_angle), n_angle, args.storage)
            except Exception as exc:
                sweep = {"error": repr(exc)}
        row = next((r for r in (sweep or {}).get("angles", []) if r["theta_set_deg"] == theta), None)
        angle = {"set_deg": theta, "after_steps": n_angle, "max_u_after_timed_run": diag32["max_u"]}
        if row is not None:
            angle[args.storage + "_deg"] = row["%s_deg_at_fp64_steps" % args.storage]
            angle["fp64_deg"] = row["fp64_deg_at_fp64_steps"]
        else:
            # the contact angle after the same number of steps in the line's storage and FP64
            for name, aprec in ((args.storage + "_deg", prec), ("fp64_deg", lbm.FP64)):
                if aprec == lbm.FP64 and args.no_fp64_check:
                    continue
                da = lbm.Domain(dict(P, precision=aprec), cfg["solid"], cfg["ghosts"])
                da.init_droplet(cfg["drop_center"], cfg["R0"])
                da.step(n_angle)
                angle[name] = math.degrees(da.diagnostics(probe)["contact_angle"])
                da.close()
                del da
                torch.cuda.empty_cache()
        if "fp64_deg" in angle:
            angle[args.storage + "_vs_fp64_deg"] = abs(angle[args.storage + "_deg"] - angle["fp64_deg"])
        angle[args.storage + "_deg_after_timed_run"] = math.degrees(diag32["contact_angle"])

        # end to end through the C ABI from host buffers: create (host mask and ghost
        # list -> device), init, K steps, diagnostics (device -> host), destroy;
        # after one untimed round of the same calls (1 step), as the steps have
        # their warm-up: a serving process creates domains of this size again
        # and again, and the library's workspace pool then holds one
        dw = lbm.Domain(P, cfg["solid"], cfg["ghosts"], workspace="library")
        dw.init_droplet(cfg["drop_center"], cfg["R0"])
        dw.step(1)
        dw.diagnostics(probe)
        dw.close()
        del dw
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        de = lbm.Domain(P, cfg["solid"], cfg["ghosts"], workspace="library")
        t_create = time.perf_counter()
        de.init_droplet(cfg["drop_center"], cfg["R0"])
        de.sync()
        t_init = time.perf_counter()
        de.step(args.steps)
        de.sync()
        t_steps = time.perf_counter()
        de.diagnostics(probe)
        t_read = time.perf_counter()
        de.close()
        t_end = time.perf_counter()
        e2e_s = t_end - t0
        e2e_parts = {"create_s": t_create - t0, "init_s": t_init - t_create, "steps_s": t_steps - t_init,
                     "per_step_ms": 1e3 * (t_steps - t_init) / args.steps, "diagnostics_d2h_s": t_read - t_steps,
                     "destroy_s": t_end - t_read}
        h2d = nn + ng * (4 + 8 * 4 + 8 * s)
        d2h = 32 * 8 + 4

        # the other storage precision on the same case (FP16 storage when the line is FP32 and back)
        other = None
        if world == 1 and not args.no_other_storage:
            try:
                other = run_other_storage(lbm, args, cfg, probe, n_angle, angle.get("fp64_deg"))
            except Exception as exc:
                other = {"error": repr(exc)}

        note("cpu")
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, st, dt = time_oracle(cfg, 10.0, 20)
            cpu = {"value": rate, "unit": "MLUPS", "cores": cores_used(), "kind": "oracle",
                   "sample": "%d FP64 oracle steps of the %d^3 workload after 1 warm-up step (%.1f s)" % (st, n, dt)}

        note("batched")
        batched = None
        if world == 1 and not args.no_batch:
            try:
                batched = run_batch_bench(lbm, args.batch_steps, args.batch_cases)
            except Exception as exc:                       # reported in the line, not fatal to it
                batched = {"error": repr(exc)}
        note("table")
        table = None
        if world == 1 and not args.no_table:
            try:
                table = run_paper_table(lbm, args.table_steps)
            except Exception as exc:
                table = {"error": repr(exc)}
        note("packing")
        packing = None
        if world == 1 and args.packing_steps > 0:
            try:
                packing = run_packing_bench(lbm, args.packing_steps,
                                            fp64_steps=min(args.packing_fp64_steps, args.packing_steps))
            except Exception as exc:
                packing = {"error": repr(exc)}
        note("serving")
        serving = None
        if world == 1 and args.serve_requests > 0:
            try:
                serving = run_serve_bench(args.serve_requests)
                if args.serve_plain:
                    serving["per_case_launches"] = run_serve_bench(args.serve_requests, batched=False)
            except Exception as exc:
                serving = {"error": repr(exc)}

        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if sp == 4 else "f32 (f16 population storage)", "data": "synthetic",
            "config": arm_config(n, theta, args.storage, world),
            "nodes": {"grid": nn, "fluid": fluid, "ghost": ng, "state_bytes": lbm.domain_bytes(P, ng)},
            "roofline": {"bound": "hbm", "kernel": "k_step_pair<19,%s,contrast>" % ("half" if sp == 2 else "float"),
                         "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "bytes_per_fluid_node": k_step_bytes_per_fluid_node(Q, D, s, True, sp),
                         "avg_launch_ms": t_step * 1e3,
                         "kernel_share": {"ghost": share[0], "step": share[1], "phi": share[2]}},
            "step_bytes_per_fluid_node": bytes_step,
            "step_effective_gbs": bytes_step * fluid * args.steps * world / (ms * 1e-3) / 1e9 / world,
            "mlups_fluid_nodes": fluid * args.steps * world / (ms * 1e-3) / 1e6,
            "cpu_baseline": cpu,
            "e2e": {"value": nn * args.steps / e2e_s / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps, "seconds": e2e_s, "parts": e2e_parts,
                    "steps_only_mlups": nn * args.steps / e2e_parts["steps_s"] / 1e6},
            "gpu_launches": launches * args.steps,
            "clocks": clk,
            "contact_angle": angle,
            "other_storage": other,
            "batched": batched,
            "serving": serving,
            "paper_table1": table,
            "packing": packing,
            "theta_sweep": sweep,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
