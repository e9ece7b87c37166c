"""The serving loop on the GPU: a short stream of mixed D2Q9 / D3Q19 requests
served in continuous batches, then every request run alone for the same
number of steps -- the final color fields must be identical to the bit."""
import math

import numpy as np
import pytest

from paper_2605_30878_gb300 import lbm, serve

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
        assert np.array_equal(d.read("phi"), be.final[q.rid]), q.rid
        d.close()
