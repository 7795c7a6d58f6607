"""Training of the learned CG preconditioner (host orchestration only).

The network (nrsense_cnn_*) is trained on pairs that the plain CG solver
generates: for a right-hand side b = sum_j A_j^H y_j, every CG iterate x_k
gives the residual r_k and the error e_k = x* - x_k, and E e_k = r_k, so e_k
is what an exact preconditioner E^{-1} returns for r_k.  The default loss is
the energy loss 1 - c|c| / (<z, E z> <e_k, r_k>), c = Re<z, r_k>, z = M(r_k):
the error energy left after a line search along z (flexible CG ignores the
scale of the search direction); it costs one normal-operator application per
pair.  Without a plan the cosine distance between z and e_k is used.  Every
forward, backward and Adam step runs in the library's kernels; this module
only picks pairs and calls the C ABI.
"""

from __future__ import annotations

import math

import numpy as np

from .nrsense import CNN_CHANNELS, Cnn, Plan


def laplacian_params(c, stencil="central"):
    """Parameters of the symmetric form (z = u0 + N4^T (I + W5^T W5) N4 u0)
    that make it z = u0 + c D^T D u0 = u0 - c L u0 with D the zero-padded
    difference along each axis (first layer: +-sqrt(c) D along each axis of
    each of Re, Im; hidden layers: identity on those 12 channels; W5 = 0).
    stencil "central": D u[i] = (u[i+1] - u[i-1]) / 2 (L has a null at the
    Nyquist frequency); "forward": D u[i] = u[i+1] - u[i] (L is the 7-point
    Laplacian).  For fixed masks the ReLU pairs cancel, so the map is linear,
    symmetric and positive definite: a local approximation of the inverse of
    a normal operator whose k-space weight grows as |k|^-2."""
    params = [(np.zeros((co, ci, 3, 3, 3), np.float32), np.zeros(co, np.float32))
              for ci, co in zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:])]
    w1 = params[0][0]
    if stencil == "central":
        a, taps = 0.5 * math.sqrt(c), (2, 0)
    elif stencil == "forward":
        a, taps = math.sqrt(c), (2, 1)
    else:
        raise ValueError(stencil)
    for ax in range(3):
        for comp in range(2):
            ch = 4 * ax + 2 * comp
            ip, im = [1, 1, 1], [1, 1, 1]
            ip[ax], im[ax] = taps
            w1[ch, comp][tuple(ip)], w1[ch, comp][tuple(im)] = a, -a
            w1[ch + 1, comp][tuple(ip)], w1[ch + 1, comp][tuple(im)] = -a, a
    for l in (1, 2, 3):
        for ch in range(12):
            params[l][0][ch, ch, 1, 1, 1] = 1.0
    return params


def generate_pairs(plan: Plan, ys, lam, tol=1e-5, maxit=200, per_run=None, keep_last=None):
    """Record (r_k, e_k) pairs from one plain-CG solve per right-hand side.

    ys: iterable of k-space data tensors (layout of Plan.forward's output).
    per_run: recorded iterates per solve (default: all of them).
    keep_last: keep only the last `keep_last` recorded pairs of each solve.
    Returns (r, e) as two complex64 CUDA tensors (K, *shape) and per-solve
    iteration counts."""
    import torch
    rs, es, iters = [], [], []
    for y in ys:
        cap = maxit if per_run is None else int(per_run)
        _, it, _, _, _, r, e = plan.solve_cg_record(y, lam, cap, tol=tol, maxit=maxit)
        if keep_last is not None:
            r, e = r[-keep_last:], e[-keep_last:]
        rs.append(r.clone())
        es.append(e.clone())
        iters.append(it)
    return torch.cat(rs), torch.cat(es), iters


def train(net: Cnn, r, e, steps, lr=2e-3, lr_final=2e-4, batch=4, seed=0, log_every=0,
          plan: Plan | None = None, lam=0.0, freeze_bias=False):
    """Adam on the energy loss (plan given) or the cosine loss over (r, e)
    pairs: `steps` updates of `batch` pairs each (gradients accumulated on
    the device), learning rate decayed
    from lr to lr_final along a cosine.  Returns the mean loss of each step
    (NaN where not read back: only every log_every-th step synchronises, and
    every step when log_every is 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = r.shape[0]
    order = rng.permutation(n)
    pos = 0
    losses = []
    for step in range(int(steps)):
        want = log_every == 0 or step % log_every == 0 or step == steps - 1
        tot = 0.0
        for b in range(batch):
            if pos == n:
                order = rng.permutation(n)
                pos = 0
            i = int(order[pos])
            pos += 1
            L = net.gradients(r[i], e[i], accumulate=b > 0, want_loss=want, plan=plan, lam=lam)
            if want:
                tot += L
        frac = step / max(1, steps - 1)
        cur = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * frac))
        net.adam_step(cur, grad_scale=1.0 / batch, freeze_bias=freeze_bias)
        losses.append(tot / batch if want else float("nan"))
    return losses


def mean_loss(net: Cnn, r, e, plan: Plan | None = None, lam=0.0):
    """Mean loss of the network over pairs (gradients overwritten, no update)."""
    tot = 0.0
    for i in range(r.shape[0]):
        tot += net.gradients(r[i], e[i], plan=plan, lam=lam)
    return tot / max(1, r.shape[0])


def fcg_iterations(plan: Plan, y, lam, net, tol=1e-4, maxit=500):
    """Flexible-CG iterations to tol on one problem (a validation score)."""
    _, it, _, _, code, _ = plan.solve_fcg(y, lam, net, tol=tol, maxit=maxit)
    return it if code == 0 else maxit + 1


def train_select(net: Cnn, r, e, blocks, score, seed=0, log=None):
    """Train in blocks [(steps, lr, lr_final), ...] and keep the parameters
    with the lowest score(net) (e.g. fcg_iterations on held-out data),
    including the starting point.  Returns [(block, loss, score), ...]."""
    best_score = score(net)
    best = net.get_params()
    hist = [(-1, float("nan"), best_score)]
    for k, (steps, lr, lr_final) in enumerate(blocks):
        losses = train(net, r, e, steps, lr=lr, lr_final=lr_final, seed=seed + k,
                       log_every=max(1, steps // 4))
        sc = score(net)
        hist.append((k, losses[-1], sc))
        if log:
            log(f"block {k}: loss {losses[-1]:.4f}, score {sc}")
        if sc < best_score:
            best_score, best = sc, net.get_params()
    net.set_params(best)
    return hist
