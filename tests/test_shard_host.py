"""Phase sharding on CPU: the partition of the motion states and the sum of
per-rank partial operators over gloo ranks (world size 2).

Each rank applies the FP64 oracle to its own states only, the partial images
are all-reduced, and lambda x is added once -- the composition the library
performs through its reduction hook.  The all-reduced operator must equal the
oracle's normal operator of all states, and conjugate gradients run on every
rank with the sharded operator (replicated vectors, local inner products)
must reproduce the unsharded iterates.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2501_16713_gb300.shard import local_rows, phase_partition, sharded_normal

SHAPE = (8, 8, 10)
LAM_CG = 750.0  # about 1e-2 of lambda_max (7.6e4) of the case below


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("counts,world", [
    ([1500, 1500, 1500, 1500], 2), ([600000, 900000, 1200000, 1500000, 1900000, 2400000], 4),
    ([5, 0, 7, 3, 9], 3), ([10, 20, 30], 3), ([4, 4], 5), ([100], 1),
    ([3, 1, 4, 1, 5, 9, 2, 6], 8)])
def test_partition_covers_every_state_once_in_contiguous_balanced_blocks(counts, world):
    blocks = phase_partition(counts, world)
    assert len(blocks) == world
    flat = [j for b in blocks for j in b]
    assert flat == list(range(len(counts)))            # each once, in order (contiguous)
    if len(counts) >= world:
        assert all(blocks)                             # every rank works
        loads = [sum(counts[j] for j in b) for b in blocks]
        # a greedy cut overshoots its target by less than one state
        assert max(loads) <= sum(counts) / world + max(counts)
    else:
        assert [len(b) for b in blocks] == [1] * len(counts) + [0] * (world - len(counts))


def test_local_rows_select_each_states_samples():
    counts = [3, 0, 5, 2]
    assert local_rows(counts, [0, 2]) == [(0, 3), (3, 8)]
    assert local_rows(counts, [1, 3]) == [(3, 3), (8, 10)]


def _case():
    import synth
    return synth.small_case(SHAPE, 2, 4, [300, 250, 350, 200], seed=151, max_disp=1.5)


def _full_normal(case, x, lam):
    from oracle import operators as O
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    return O.normal(geo, x, d64, case["smaps"], case["coords"], lam)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from oracle import operators as O
    from oracle import solvers
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    case = _case()
    geo = O.Geometry(SHAPE)
    counts = [c.shape[0] for c in case["coords"]]
    mine = phase_partition(counts, world)[rank]
    d64 = [case["disp"][j].astype(np.float64) for j in mine]
    om = [case["coords"][j] for j in mine]

    def all_reduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        tr = torch.view_as_real(t).clone()
        dist.all_reduce(tr)
        return torch.view_as_complex(tr).numpy()

    local = lambda v: O.normal(geo, v, d64, case["smaps"], om, 0.0)  # noqa: E731
    rng = np.random.default_rng(152)
    x = rng.standard_normal(SHAPE) + 1j * rng.standard_normal(SHAPE)
    lam = 0.05
    Ex = sharded_normal(x, local, all_reduce, lam)
    # right-hand side: each rank's adjoint of its own data, all-reduced
    ys = O.stacked_forward(geo, case["x"], d64, case["smaps"], om)
    b = all_reduce(O.stacked_adjoint(geo, ys, d64, case["smaps"], om))
    xs, it, hist = solvers.cg(lambda v: sharded_normal(v, local, all_reduce, LAM_CG), b,
                              tol=1e-12, maxit=8)
    out[rank] = (mine, Ex, b, xs, it, hist)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_operator_and_cg_match_the_whole_gloo():
    from oracle import operators as O
    from oracle import solvers
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    case = _case()
    rng = np.random.default_rng(152)
    x = rng.standard_normal(SHAPE) + 1j * rng.standard_normal(SHAPE)
    lam = 0.05
    full = _full_normal(case, x, lam)
    geo = O.Geometry(SHAPE)
    d64 = [d.astype(np.float64) for d in case["disp"]]
    ys = O.stacked_forward(geo, case["x"], d64, case["smaps"], case["coords"])
    b = O.stacked_adjoint(geo, ys, d64, case["smaps"], case["coords"])
    # eight iterations of a moderately conditioned solve (lambda ~ 1e-2
    # lambda_max): the two summation orders' FP64 rounding differences (1e-16)
    # grow through the iterations (to about 1e-7 by the twelfth); a missing or
    # doubled state, or lambda added per rank, would differ at O(1)
    xf, itf, histf = solvers.cg(lambda v: _full_normal(case, v, LAM_CG), b, tol=1e-12, maxit=8)
    assert sorted(res[0][0] + res[1][0]) == [0, 1, 2, 3] and res[0][0] and res[1][0]
    for r in range(world):
        mine, Ex, br, xs, it, hist = res[r]
        scale = np.linalg.norm(full)
        assert np.linalg.norm(Ex - full) <= 1e-12 * scale
        assert np.linalg.norm(br - b) <= 1e-12 * np.linalg.norm(b)
        assert it == itf
        assert np.allclose(hist, histf, rtol=1e-8, atol=0)
        assert np.linalg.norm(xs - xf) <= 1e-8 * np.linalg.norm(xf)
    # both ranks hold the same iterates (replicated vectors)
    assert np.array_equal(res[0][3], res[1][3])
