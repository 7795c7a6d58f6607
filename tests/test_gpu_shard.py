"""Phase-sharded operator and CG through the library's reduction hook, on one GPU.

Two host threads stand in for two ranks: each owns a plan of half the
motion states (phase_partition) and registers a reduction hook that sums the
two ranks' images on the host (stream synchronised, copy to the host, a
barrier with a timeout, the sum in rank order, copy back).  Only the host
waits; no kernel waits on another.  The sharded normal operator must match
the plan of all states, and CG run concurrently on both ranks must match the
unsharded solve, with both ranks holding bitwise the same iterates.
"""

import threading

import numpy as np
import pytest

import synth
from helpers import make_plan, rel_l2, to_dev

pytestmark = pytest.mark.gpu

SHAPE = (16, 16, 24)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


class HostAllReduce:
    """In-process stand-in for an all-reduce over `world` threads."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.slots = [None] * world
        self.calls = [0] * world

    def hook(self, rank):
        def fn(buf, stream):
            stream.synchronize()
            self.slots[rank] = buf.cpu()
            self.bar.wait()
            total = self.slots[0].clone()
            for r in range(1, self.world):
                total += self.slots[r]
            self.bar.wait()  # every rank has read the slots
            buf.copy_(total.to(buf.device))
            self.calls[rank] += 1
        return fn


def _run_ranks(fns):
    out, errs = [None] * len(fns), []

    def body(r):
        import torch
        try:
            # a new host thread: make the device (its primary context) current
            # before the first library call, as every rank process does
            torch.cuda.set_device(0)
            out[r] = fns[r]()
        except Exception as e:  # noqa: BLE001
            errs.append(e)

    ts = [threading.Thread(target=body, args=(r,)) for r in range(len(fns))]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=600)
    assert not errs, errs
    return out


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2501_16713_gb300.shard import ShardedPlan
    case = synth.small_case(SHAPE, 4, 4, [2600, 1900, 2300, 1500], seed=161)
    full = make_plan(case, SHAPE)
    disp = to_dev(np.stack(case["disp"]))
    coords = [to_dev(c) for c in case["coords"]]
    smaps = to_dev(case["smaps"])
    ar = HostAllReduce(2)
    ranks = [ShardedPlan(SHAPE, disp, coords, smaps, r, 2, reduce=ar.hook(r)) for r in range(2)]
    yield case, full, ranks, ar
    for p in ranks:
        p.close()
    full.close()
    torch.cuda.synchronize()


def test_shards_hold_disjoint_states(setup):
    _, _, ranks, _ = setup
    assert ranks[0].phases + ranks[1].phases == [0, 1, 2, 3]
    assert ranks[0].phases and ranks[1].phases


def test_sharded_normal_matches_all_states(setup):
    import torch
    case, full, ranks, ar = setup
    x = to_dev(case["x"])
    lam = 0.3
    ref = full.normal(x, lam)
    outs = _run_ranks([lambda p=p: p.normal(x, lam) for p in ranks])
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    assert rel_l2(outs[0].cpu().numpy(), ref.cpu().numpy()) < 1e-6
    assert ar.calls[0] >= 1 and ar.calls[1] >= 1


def test_sharded_cg_matches_unsharded(setup):
    import torch
    case, full, ranks, _ = setup
    x = to_dev(case["x"])
    y_all = full.forward(x)
    lam = 1e-2 * float(torch.linalg.norm(full.normal(x)) / torch.linalg.norm(x))
    xf, itf, _, trf, _ = full.solve_cg(y_all, lam, tol=1e-5, maxit=200)
    res = _run_ranks([lambda p=p: p.solve_cg(p.local_data(y_all), lam, tol=1e-5, maxit=200)
                      for p in ranks])
    torch.cuda.synchronize()
    (x0, it0, _, tr0, _), (x1, it1, _, tr1, _) = res
    assert torch.equal(x0, x1) and it0 == it1
    assert abs(it0 - itf) <= 1
    assert tr0 < 2e-5
    assert rel_l2(x0.cpu().numpy(), xf.cpu().numpy()) < 1e-4
