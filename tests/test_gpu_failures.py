"""Failure paths of the library, made on the host or by a bounded wait.

No test here faults, traps or hangs the GPU.  Plan creation is made to fail
by the library's test-only host fault injection (NRSENSE_FAULT: the first
device allocation, cuFFT plan or upload reports failure), and every failure
must come back as its status code with all resources released, after which
a normal plan works in the same process.  The TMA halo wait of the k-space
interpolation is given a limit of zero polls (NRSENSE_TMA_POLL_LIMIT=0):
every TMA-staged CTA records ERR_TIMEOUT, waits (bounded) for its own copy
to land and returns; the status word reports it and the context stays
usable.
"""

import numpy as np
import pytest

import synth
from helpers import TOL_FP32, make_plan, rel_l2, to_dev
from oracle import operators as O

pytestmark = pytest.mark.gpu

SHAPE = (16, 16, 24)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def case():
    return synth.small_case(SHAPE, 4, 2, [2500, 1800], seed=141)


def _healthy(case):
    # a plan made after the failure computes the operator correctly
    plan = make_plan(case, SHAPE)
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    y = plan.forward(to_dev(case["x"])).cpu().numpy()
    ref = np.concatenate(O.stacked_forward(geo, case["x"], d64, case["smaps"], case["coords"]))
    assert rel_l2(y, ref) < TOL_FP32
    assert plan.device_status() == 0
    plan.close()


@pytest.mark.parametrize("fault,code", [("alloc", -2), ("cufft", -3), ("upload", -4)])
def test_injected_plan_failure_reports_status_and_releases(case, monkeypatch, fault, code):
    import torch
    from paper_2501_16713_gb300 import NrsenseError
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("NRSENSE_FAULT", fault)
    with pytest.raises(NrsenseError) as ex:
        make_plan(case, SHAPE)
    assert ex.value.code == code
    monkeypatch.delenv("NRSENSE_FAULT")
    torch.cuda.synchronize()
    # the failed creation released what it had allocated (free memory back
    # within 64 MB: the caching allocator and the driver move a little)
    assert torch.cuda.mem_get_info()[0] > before - (64 << 20)
    _healthy(case)


def test_tma_wait_limit_expires_with_timeout_status(case, monkeypatch):
    import ctypes
    from paper_2501_16713_gb300.nrsense import Tuning
    monkeypatch.setenv("NRSENSE_TMA_POLL_LIMIT", "0")
    plan = make_plan(case, SHAPE)
    monkeypatch.delenv("NRSENSE_TMA_POLL_LIMIT")
    assert plan.device_status() == 0
    t = Tuning()
    # grid 32 x 32 x 48, 8^3 tiles: interior tiles take the TMA-staged halo
    t.spread_variant, t.interp_coils, t.interp_tma = 3, 4, 1
    st = plan.lib.nrsense_plan_set_tuning(plan._h, ctypes.byref(t))
    assert st == 0
    plan.forward(to_dev(case["x"]))
    assert plan.device_status() == -7        # ERR_TIMEOUT, latched and cleared
    assert plan.device_status() == 0
    plan.close()
    _healthy(case)
