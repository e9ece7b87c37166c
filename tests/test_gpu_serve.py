"""The serving loop on the GPU: short streams of mixed D2Q9 / D3Q19 requests
served in continuous batches.  Every request's final state against the FP64
oracle stepped alone for the same number of steps (within the parity bounds),
and against the same request run alone on the GPU (identical to the bit)."""
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2605_30878_gb300 import lbm, serve

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


def test_served_cases_equal_cases_run_alone():
    reqs = serve.poisson_requests(n=8, rate=200.0, seed=5, L2=(48, 96), L3=(32, 48))
    be = serve.GpuBackend(keep_final=True)
    srv = serve.Server(be, memory_budget=2 << 30, chunk=100, check_every=500, max_steps=2500)
    res, summ = srv.run(reqs)
    assert summ["requests"] == 8 and summ["failed"] == 0
    assert summ["batch_rebuilds"] >= 2 and summ["peak_active"] >= 2
    for q, r in zip(reqs, res):
        assert r.steps > 0 and math.isfinite(r.finished)
        assert r.converged or r.steps == 2500
        c = serve.request_case(q)
        d = lbm.Domain(c["params"], c["solid"], c["ghosts"])
        d.init_droplet(c["drop_center"], c["R0"])
        d.step(r.steps)
        for f in ("N", "B", "phi", "u", "p"):
            assert np.array_equal(d.read(f), be.final[q.rid][f]), (q.rid, f)
        d.close()


@pytest.mark.parametrize("precision", [lbm.FP64, lbm.FP32])
def test_served_mix_matches_the_oracle(precision):
    """Requests arriving over ~20 ms join and leave both lattices' batches in
    chunks of 5 steps (odd, so cases join at either step parity); each retires
    after 30 steps (its second angle check; 45 if no angle can be measured).
    Each final state against the oracle stepped alone as many steps."""
    reqs = serve.poisson_requests(n=8, rate=400.0, seed=6, L2=(40, 72), L3=(24, 36))
    be = serve.GpuBackend(precision=precision, keep_final=True)
    srv = serve.Server(be, memory_budget=2 << 30, chunk=5, check_every=15, tol_deg=1e9, max_steps=45)
    res, summ = srv.run(reqs)
    assert summ["requests"] == 8 and summ["failed"] == 0 and summ["batch_rebuilds"] >= 2
    for q, r in zip(reqs, res):
        c = serve.request_case(q, precision=precision)
        o = oracle.Oracle(c["params"], c["solid"], c["ghosts"])
        o.init_droplet(c["drop_center"], c["R0"])
        o.step(r.steps)
        fluid = c["solid"].reshape(-1) == 0
        pu.check(be.final[q.rid], pu.read_oracle(o), c["params"], precision, fluid, r.steps,
                 "served request %d (Q=%d, L=%d, ratio %.1f) after %d steps" % (q.rid, q.lattice, q.L,
                                                                              q.rho_ratio, r.steps))
