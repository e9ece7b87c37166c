"""Batched launches (many uneven domains, one launch per phase, one block per
tile): every domain of a mixed batch against the FP64 oracle stepped alone,
and against the same domains stepped one by one on the GPU (identical to the
bit), for every tile shape the autotuner can pick, for both lattices and every
storage precision."""
import gc
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import lbm
from paper_2605_30878_gb300 import workloads as wl

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_30878_gb300 import build
    build.build()
    lbm.load()


def _cases(precision, seed=4, count=5):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(20, 44))
        R = float(rng.uniform(0.2, 0.3) * n)
        theta = float(rng.uniform(20, 160))
        ratio = [1.0, 10.0, 1000.0][k % 3]
        cfg = wl.sphere_config(n=n, R=R, R0=0.6 * R, theta_deg=theta, rho_ratio=ratio,
                               mu_ratio=(100.0 if ratio > 1 else 1.0), precision=precision)
        cfg["params"]["ghost_rule"] = k % 2
        out.append(cfg)
    return out


def _make(cfgs):
    doms = []
    for c in cfgs:
        d = lbm.Domain(c["params"], c["solid"], c["ghosts"])
        d.init_droplet(c["drop_center"], c["R0"])
        doms.append(d)
    return doms


def _mixed_2d(precision, seed=13, count=5):
    """D2Q9 drops on cylinders of different sizes, density ratios 1, 10, 1000
    (viscosity ratio 100 at 1000, else 1) and both ghost rules."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx, ny = int(rng.integers(40, 120)), int(rng.integers(30, 80))
        R = float(rng.uniform(0.1, 0.2) * min(nx, ny))
        cfg = wl.cylinder_config(nx=nx, ny=ny, R=R, R0=0.8 * R, theta_deg=float(rng.uniform(20, 160)))
        ratio = [1.0, 10.0, 1000.0][k % 3]
        cfg["params"].update(precision=precision, ghost_rule=k % 2, rho_l=ratio, rho_g=1.0,
                             mu_l=0.1 * (100.0 if ratio == 1000.0 else 1.0), mu_g=0.1)
        out.append(cfg)
    return out


@pytest.mark.parametrize("Q", [9, 19])
@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_mixed_batch_matches_the_oracle(precision, Q):
    """Every domain of a mixed batch -- sizes, density ratios 1/10/1000, both
    ghost rules, domains joining at both step parities -- against the FP64
    oracle stepped alone from the same initial state, after each of three legs
    (tile shape 0 for 1 step and shape 5 for 4 -- both two nodes per thread
    in float --, shape 2 for 5; TMA halos on interior tiles, element copies at
    the y and z ends), within the parity bounds of every precision."""
    cfgs = _cases(precision, seed=13) if Q == 19 else _mixed_2d(precision)
    doms = _make(cfgs)
    orcs = []
    for c in cfgs:
        o = oracle.Oracle(c["params"], c["solid"], c["ghosts"])
        o.init_droplet(c["drop_center"], c["R0"])
        orcs.append(o)
    early = (1, 3)                                   # these join the batch one step ahead (odd parity)
    for k in early:
        doms[k].step(1)
        orcs[k].step(1)
    b = lbm.Batch(doms)
    taken = [int(k in early) for k in range(len(cfgs))]
    for variant, n in ((0, 1), (5, 4), (2, 5)):
        b.set_variant(variant)
        b.step(n)
        b.sync()
        for k, (d, o, c) in enumerate(zip(doms, orcs, cfgs)):
            o.step(n)
            fluid = c["solid"].reshape(-1) == 0
            taken[k] += n
            steps = taken[k]
            pu.check(pu.read_gpu(d), pu.read_oracle(o), c["params"], precision, fluid, steps,
                     "batch Q=%d domain %d (ratio %g, rule %d) after %d steps" %
                     (Q, k, c["params"]["rho_l"], c["params"].get("ghost_rule", 0), steps))
    # the batched step map itself: each oracle takes its domain's GPU state,
    # the batch and the oracles advance one step from identical inputs
    fresh = []
    for d, c in zip(doms, cfgs):
        o = oracle.Oracle(c["params"], c["solid"], c["ghosts"])
        for f in ("N", "B", "phi", "u", "p"):
            o.set(f, d.read(f))
        fresh.append(o)
    b.step(1)
    b.sync()
    for k, (d, o, c) in enumerate(zip(doms, fresh, cfgs)):
        o.step(1)
        pu.check(pu.read_gpu(d), pu.read_oracle(o), c["params"], precision, c["solid"].reshape(-1) == 0, 1,
                 "batch Q=%d domain %d, one step from its GPU state" % (Q, k))
    b.close()


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_batch_equals_individual_steps(precision):
    cfgs = _cases(precision)
    alone = _make(cfgs)
    for d in alone:
        d.step(16)                        # 5 + 4 + 3 + 2 + 1 + 1 batched steps
    mixed = _make(cfgs)
    mixed[1].step(1)                      # domains may enter the batch at different parities
    b = lbm.Batch(mixed)
    for v, n in ((1, 5), (2, 4), (0, 3), (3, 2), (4, 1), (5, 1)):
        b.set_variant(v)
        b.step(n)
    b.sync()
    alone[1].step(1)                      # the extra step domain 1 took before joining
    for k, (a, m) in enumerate(zip(alone, mixed)):
        for f in ("N", "B", "phi", "u", "p"):
            assert np.array_equal(a.read(f), m.read(f)), (k, f)

@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16])
def test_velocity_and_pressure_stay_zero_at_solid_nodes(precision):
    """The stencils read the previous velocity at solid nodes as 0, so no step
    kernel may leave anything else there: neither the two-node kernel's lane
    for a solid partner node nor the zeros it writes around the fluid to fill
    whole 32-byte sectors (FP32 storage).  Ragged small boxes, stepped alone
    and batched with every tile shape."""
    cfgs = _cases(precision)
    alone, mixed = _make(cfgs), _make(cfgs)
    for d in alone:
        d.step(3)
    b = lbm.Batch(mixed)
    for v in range(lbm.BATCH_TILE_SHAPES):
        b.set_variant(v)
        b.step(1)
    b.sync()
    b.close()
    for c, a, m in zip(cfgs, alone, mixed):
        solid = c["solid"].reshape(-1) != 0
        assert solid.any()
        for d in (a, m):
            u, p = d.read("u"), d.read("p")
            assert not np.any(u[:, solid]) and not np.any(p[solid])
            assert np.any(u[:, ~solid])


def test_batch_rejects_outside_steps_and_mixed_precision():
    cfgs = _cases(lbm.FP32, count=2)
    doms = _make(cfgs)
    with lbm.Batch(doms) as b:
        doms[0].step(1)
        with pytest.raises(lbm.LbmError) as e:
            b.step(1)
        assert e.value.status == lbm.LBM_ERR_ARG
    other = _make(_cases(lbm.FP64, count=1))
    with pytest.raises(lbm.LbmError):
        lbm.Batch([doms[1], other[0]])


def test_autotuner_picks_a_shape_and_keeps_results():
    cfgs = _cases(lbm.FP32, seed=9, count=4)
    a, m = _make(cfgs), _make(cfgs)
    b = lbm.Batch(m)
    chosen, ms = b.tune(steps_per_trial=3)
    assert chosen in range(lbm.BATCH_TILE_SHAPES) and len(ms) == lbm.BATCH_TILE_SHAPES and (ms > 0).all()
    assert b.variant == chosen
    for d in a:
        d.step(4 * lbm.BATCH_TILE_SHAPES)   # tuning advanced every domain shapes x (3 + 1) steps
    b.sync()
    for x, y in zip(a, m):
        assert np.array_equal(x.read("B"), y.read("B"))


def _cases_2d(precision, seed=7, count=4):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nx, ny = int(rng.integers(40, 150)), int(rng.integers(30, 90))
        R = float(rng.uniform(0.1, 0.2) * min(nx, ny))
        cfg = wl.cylinder_config(nx=nx, ny=ny, R=R, R0=0.8 * R, theta_deg=float(rng.uniform(20, 160)))
        P = cfg["params"]
        P["precision"] = precision
        P["ghost_rule"] = k % 2
        if k % 2:                               # density and viscosity contrast on every other case
            P.update(rho_l=100.0, rho_g=1.0, mu_l=1.0, mu_g=0.1)
        out.append(cfg)
    return out


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32, lbm.FP16])
def test_batch_equals_individual_steps_d2q9(precision):
    cfgs = _cases_2d(precision)
    alone, mixed = _make(cfgs), _make(cfgs)
    for d in alone:
        d.step(15)
    b = lbm.Batch(mixed)
    assert b.launches_per_step() == 4            # ghosts, contrast step, plain step, color
    for v, n in ((2, 3), (1, 3), (0, 4), (3, 2), (4, 2), (5, 1)):
        b.set_variant(v)
        b.step(n)
    b.sync()
    for k, (a, m) in enumerate(zip(alone, mixed)):
        for f in ("N", "B", "phi", "u", "p"):
            assert np.array_equal(a.read(f), m.read(f)), (k, f)


def test_two_live_batches_and_slot_reuse():
    """Batches alive at the same time hold separate slots of the constant
    parameter table; a closed batch's slots go to the next one."""
    cfgs = _cases(lbm.FP32, seed=11, count=4)
    alone, mixed = _make(cfgs), _make(cfgs)
    b1, b2 = lbm.Batch(mixed[:2]), lbm.Batch(mixed[2:])
    b1.step(3)
    b2.step(5)
    b1.close()
    b3 = lbm.Batch(mixed[:1])                    # reuses a slot b1 held
    b3.step(2)
    b3.sync()
    b2.sync()
    for d, n in zip(alone, (5, 3, 5, 5)):
        d.step(n)
    for k, (a, m) in enumerate(zip(alone, mixed)):
        assert np.array_equal(a.read("N"), m.read("N")), k
        assert np.array_equal(a.read("phi"), m.read("phi")), k


def test_batch_size_limit():
    """At most 96 domains per batch (the constant table's slots per precision)."""
    cfg = wl.sphere_config(n=12, R=3.0, R0=2.5, theta_deg=90.0, rho_ratio=1.0, mu_ratio=1.0, precision=lbm.FP32)
    gc.collect()                                 # batches of earlier tests give their slots back
    doms = _make([cfg] * 97)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Batch(doms)
    assert e.value.status == lbm.LBM_ERR_ARG and "96" in str(e.value)
    with lbm.Batch(doms[:96]) as b:
        b.step(2)
        b.sync()
    a = _make([cfg])[0]
    a.step(2)
    assert np.array_equal(a.read("N"), doms[95].read("N"))
    # slots need not be contiguous: free slot 0 and slot 95 around a live batch
    b1, b2 = lbm.Batch(doms[0:1]), lbm.Batch(doms[1:95])
    b1.close()
    with lbm.Batch(doms[95:97]) as b3:
        b3.step(3)
        b3.sync()
    b2.close()
    a.step(3)
    assert np.array_equal(a.read("N"), doms[95].read("N"))
    a2 = _make([cfg])[0]
    a2.step(3)
    assert np.array_equal(a2.read("N"), doms[96].read("N"))


@pytest.mark.parametrize("precision", [lbm.FP32, lbm.FP16])
@pytest.mark.parametrize("Q", [9, 19])
def test_tma_halo_equals_element_copies(precision, Q, monkeypatch):
    """Large enough for tiles whose halo needs no periodic image in y, z: the
    single-domain step kernel copies their halo with tiled TMA loads from
    kernel-parameter maps, the batched kernel with every tile shape from maps
    in global memory; a domain created with LBM_HALO_COPY=elements copies
    every halo element by element.  All states must agree to the bit."""
    if Q == 19:
        cfg = wl.sphere_config(n=96, R=20.0, R0=14.0, theta_deg=70.0, rho_ratio=1000.0, precision=precision)
    else:
        cfg = wl.cylinder_config(nx=160, ny=128, R=20.0, R0=16.0, theta_deg=110.0)
        cfg["params"].update(precision=precision, rho_l=1000.0, rho_g=1.0, mu_l=10.0, mu_g=0.1)
    monkeypatch.setenv("LBM_HALO_COPY", "elements")
    copied = _make([cfg])
    monkeypatch.delenv("LBM_HALO_COPY")
    alone = _make([cfg])
    for d in copied + alone:
        d.step(9)
    want = {f: copied[0].read(f) for f in ("N", "B", "phi", "u", "p")}
    for f in want:
        assert np.array_equal(alone[0].read(f), want[f]), ("single domain, TMA", f)
    for variant in range(lbm.BATCH_TILE_SHAPES):
        doms = _make([cfg])
        with lbm.Batch(doms) as b:
            b.set_variant(variant)
            b.step(9)
            b.sync()
        for f in want:
            assert np.array_equal(doms[0].read(f), want[f]), ("batched TMA, tile shape %d" % variant, f)
