"""Device-side failure reporting without a GPU fault.

The step kernel's one device wait -- a block waiting for its TMA halo copy on
a shared-memory mbarrier -- is bounded by a time limit and a poll count; when
it gives up, the kernel sets the domain's timeout bit and returns.  A copy
that never lands cannot be made safely, so lbm_debug_expire_halo_wait arms an
mbarrier for bytes no copy delivers (issuing no copy at all) and waits on it
with the step kernel's own wait function and a short limit.  Nothing is in
flight when the wait ends, so the GPU context stays usable."""
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


def _case(precision=lbm.FP32):
    return wl.sphere_config(n=32, R=6.0, R0=5.0, theta_deg=70.0, rho_ratio=10.0, precision=precision)


def _domain(cfg):
    d = lbm.Domain(cfg["params"], cfg["solid"], cfg["ghosts"])
    d.init_droplet(cfg["drop_center"], cfg["R0"])
    return d


def test_expired_halo_wait_is_reported_and_poisons_the_domain():
    cfg = _case()
    d = _domain(cfg)
    d.step(3)
    d.sync()
    limit = 20_000_000                                     # 20 ms
    waited = d.debug_expire_halo_wait(limit, measure=True)
    # the time bound ended the wait (the poll cap is far longer than 20 ms)
    assert limit <= waited < limit + 200_000_000, waited
    with pytest.raises(lbm.LbmError) as e:
        d.sync()
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    # poisoned: every call that would advance or change the state is refused
    for call in (lambda: d.step(1), lambda: d.init_droplet(cfg["drop_center"], cfg["R0"]),
                 lambda: d.write("phi", np.zeros(cfg["solid"].size)), lambda: d.profile_steps(1),
                 lambda: lbm.Batch([d]), lambda: d.debug_expire_halo_wait(limit)):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.status == lbm.LBM_ERR_TIMEOUT
    with pytest.raises(lbm.LbmError) as e:
        d.sync()
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    d.close()


def test_expired_wait_in_a_batch_is_reported_by_the_batch():
    cfgs = [_case(), wl.sphere_config(n=28, R=5.0, R0=4.0, theta_deg=110.0, rho_ratio=1.0, precision=lbm.FP32)]
    doms = [_domain(c) for c in cfgs]
    b = lbm.Batch(doms)
    b.step(2)
    doms[1].debug_expire_halo_wait(5_000_000)              # asynchronous, on the batch's stream
    b.step(1)
    with pytest.raises(lbm.LbmError) as e:
        b.sync()
    assert e.value.status == lbm.LBM_ERR_TIMEOUT and "domain 1" in str(e.value)
    with pytest.raises(lbm.LbmError) as e:
        b.step(1)
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    doms[0].sync()                                         # the other domain is unaffected
    b.close()


def test_context_stays_usable_after_an_expired_wait():
    """After the expired wait a new domain steps normally and matches the FP64
    oracle to the parity bound."""
    bad = _domain(_case())
    bad.debug_expire_halo_wait(1_000_000)
    with pytest.raises(lbm.LbmError):
        bad.sync()
    cfg = _case(lbm.FP64)
    g = _domain(cfg)
    o = oracle.Oracle(cfg["params"], cfg["solid"], cfg["ghosts"])
    o.init_droplet(cfg["drop_center"], cfg["R0"])
    g.step(5)
    o.step(5)
    g.sync()
    pu.check(pu.read_gpu(g), pu.read_oracle(o), cfg["params"], lbm.FP64, cfg["solid"].reshape(-1) == 0, 5,
             "after an expired wait")


def test_debug_wait_arguments():
    d = _domain(_case())
    for bad in (0, 999, 2_000_000_000):
        with pytest.raises(lbm.LbmError) as e:
            d.debug_expire_halo_wait(bad)
        assert e.value.status == lbm.LBM_ERR_ARG
    d.sync()                                               # nothing was launched
    assert not math.isnan(d.diagnostics()["phi_sum"])
