"""FP64 oracle of the learned preconditioner network (test infrastructure).

The build target adds a learned preconditioner for the Tikhonov CG solve of
the reconstruction problem: a small 3D convolutional network M that maps a
residual r to a search direction z ~ E^{-1} r, used inside flexible CG.  The
paper itself has no learned component; this module fixes the network's
definition so the CUDA kernels can be checked against it.

Definition (all arrays channel-first here, (C, D, H, W)):
  s  = sqrt(mean |r|^2)                       (input scale, not trained)
  u0 = [Re r, Im r] / s                       (2 channels)
  h_l = relu(conv_l(h_{l-1}))  for l = 1..4   (16 channels each)
  o  = conv_5(h_4)                            (2 channels)
  z  = (u0 + o)  read back as a complex image (residual connection)
conv_l is a 3x3x3 cross-correlation with zero padding and a bias:
  conv(x)[o, d, h, w] = b[o] + sum_{c, tz, ty, tx} W[o, c, tz, ty, tx] x[c, d+tz-1, h+ty-1, w+tx-1].
Flexible CG is invariant to the scale of M's output, so the training losses
are scale invariant.  For the target e = E^{-1} r (so E e = r):
  cosine loss  L = 1 - Re<z, e> / (||z|| ||e||);
  energy loss  L = 1 - c |c| / (<z, E z> <e, r>),  c = Re<z, r>:
the fraction of the error energy ||e||_E^2 = <e, r> left after an exact line
search from the current iterate along z (Re<z, E e> = c); a direction with
c < 0 points uphill and scores above 1.  The energy loss weights errors by E,
as CG's convergence does.
"""

from __future__ import annotations

import numpy as np

CHANNELS = (2, 16, 16, 16, 16, 2)


def init_params(seed: int, channels=CHANNELS):
    """He-style random initialisation (weights (Cout, Cin, 3, 3, 3), biases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        std = np.sqrt(2.0 / (27 * cin))
        params.append((rng.standard_normal((cout, cin, 3, 3, 3)) * std,
                       np.zeros(cout)))
    # start close to the identity map: small last layer
    w, b = params[-1]
    params[-1] = (w * 0.1, b)
    return params


def conv3d(x, w, b):
    """3x3x3 cross-correlation with zero padding; x (Cin, D, H, W)."""
    cin, D, H, W = x.shape
    xp = np.zeros((cin, D + 2, H + 2, W + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((w.shape[0], D, H, W)) + b[:, None, None, None]
    for tz in range(3):
        for ty in range(3):
            for tx in range(3):
                out += np.einsum("oc,cdhw->odhw", w[:, :, tz, ty, tx],
                                 xp[:, tz:tz + D, ty:ty + H, tx:tx + W])
    return out


def conv3d_backward(x, w, dy):
    """Gradients of sum(dy * conv3d(x, w, b)) w.r.t. x, w and b."""
    cin, D, H, W = x.shape
    xp = np.zeros((cin, D + 2, H + 2, W + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for tz in range(3):
        for ty in range(3):
            for tx in range(3):
                sl = (slice(None), slice(tz, tz + D), slice(ty, ty + H), slice(tx, tx + W))
                dw[:, :, tz, ty, tx] = np.einsum("odhw,cdhw->oc", dy, xp[sl])
                dxp[sl] += np.einsum("oc,odhw->cdhw", w[:, :, tz, ty, tx], dy)
    db = dy.sum(axis=(1, 2, 3))
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, db


def conv3d_transpose(y, w):
    """Adjoint of conv3d(., w, 0) with respect to its input: x = W^T y."""
    cout, D, H, W = y.shape
    yp = np.zeros((cout, D + 2, H + 2, W + 2))
    yp[:, 1:-1, 1:-1, 1:-1] = y
    x = np.zeros((w.shape[1], D, H, W))
    # x[c, p] = sum_{o, t} w[o, c, t] y[o, p - t + 1]: correlation with flipped taps
    for tz in range(3):
        for ty in range(3):
            for tx in range(3):
                x += np.einsum("oc,odhw->cdhw", w[:, :, tz, ty, tx],
                               yp[:, 2 - tz:2 - tz + D, 2 - ty:2 - ty + H, 2 - tx:2 - tx + W])
    return x


def input_scale(r):
    return float(np.sqrt(np.mean(np.abs(r) ** 2)))


def _identity(a):
    return a


def forward(params, r, rnd=_identity):
    """z = M(r) and the activations needed by backward.

    rnd is applied to the network input and to every hidden activation (the
    values a reduced-precision implementation stores between layers, e.g.
    bf16_round); the identity gives the exact definition.  The residual path
    u0 and the last layer's output are not rounded."""
    s = input_scale(r)
    u0 = np.stack([r.real, r.imag]) / s
    h = rnd(u0)
    acts = [h]
    for l, (w, b) in enumerate(params):
        h = conv3d(h, w, b)
        if l < len(params) - 1:
            h = rnd(np.maximum(h, 0.0))
        acts.append(h)
    zc = u0 + acts[-1]
    return zc[0] + 1j * zc[1], acts


def loss(z, e):
    """1 - Re<z, e> / (||z|| ||e||)."""
    nz, ne = np.linalg.norm(z), np.linalg.norm(e)
    return 1.0 - np.real(np.vdot(z, e)) / (nz * ne)


def loss_grad_z(z, e):
    """dL/dz as a complex array (derivative w.r.t. Re z + i d/d Im z)."""
    nz, ne = np.linalg.norm(z), np.linalg.norm(e)
    c = np.real(np.vdot(z, e))
    return -(e / (nz * ne) - c * z / (nz ** 3 * ne))


def loss_energy(z, r, e, Ez):
    """1 - c|c| / (<z, E z> <e, r>), c = Re<z, r>; Ez = E z."""
    c = np.real(np.vdot(z, r))
    zEz = np.real(np.vdot(z, Ez))
    er = np.real(np.vdot(e, r))
    return 1.0 - c * abs(c) / (zEz * er)


def loss_energy_grad_z(z, r, e, Ez):
    """dL/dz of the energy loss (E Hermitian: d<z, E z>/dz = 2 E z)."""
    c = np.real(np.vdot(z, r))
    zEz = np.real(np.vdot(z, Ez))
    er = np.real(np.vdot(e, r))
    return -2.0 * abs(c) * r / (zEz * er) + 2.0 * c * abs(c) * Ez / (zEz ** 2 * er)


def backward(params, acts, dz, rnd=_identity):
    """Parameter gradients given dL/dz (the residual path has no parameters).

    rnd is applied to dL/do and to every back-propagated activation gradient
    after its ReLU mask (identity: the exact definition)."""
    grads = [None] * len(params)
    g = rnd(np.stack([dz.real, dz.imag]))
    for l in range(len(params) - 1, -1, -1):
        w, b = params[l]
        if l < len(params) - 1:
            g = rnd(g * (acts[l + 1] > 0))
        gx, gw, gb = conv3d_backward(acts[l], w, g)
        grads[l] = (gw, gb)
        g = gx
    return grads


def loss_and_grads(params, r, e, rnd=_identity):
    z, acts = forward(params, r, rnd)
    L = loss(z, e)
    grads = backward(params, acts, loss_grad_z(z, e), rnd)
    return L, grads


def loss_and_grads_energy(params, r, e, E, rnd=_identity):
    """Energy loss and parameter gradients; E is a callable applying the
    (Hermitian positive definite) system operator to an image."""
    z, acts = forward(params, r, rnd)
    Ez = E(z)
    L = loss_energy(z, r, e, Ez)
    grads = backward(params, acts, loss_energy_grad_z(z, r, e, Ez), rnd)
    return L, grads


# ---------------------------------------------------------------------------
# Symmetric form.  The same five layers (biases unused): N4 = D_4 W_4 D_3 W_3
# D_2 W_2 D_1 W_1 maps u0 to the 16-channel h_4 (ReLU masks D_l set by the
# forward pass) and W_5 maps h_4 to 2 channels.  The network returns
#   z = u0 + N4^T (I + W_5^T W_5) N4 u0,
# i.e. z = (I + A^T A) u0 with A = [N4; W_5 N4] for fixed masks: a symmetric
# positive definite map, as CG-type methods expect of a preconditioner.
# (With W_5 = 0 and first-layer +-finite differences it is I - c Laplacian.)

def forward_spd(params, r, rnd=_identity):
    """z of the symmetric form and the intermediates backward_spd needs."""
    s = input_scale(r)
    u0 = np.stack([r.real, r.imag]) / s
    L = len(params)
    h = [rnd(u0)]
    for l in range(L - 1):
        w = params[l][0]
        h.append(rnd(np.maximum(conv3d(h[-1], w, np.zeros(w.shape[0])), 0.0)))
    w5 = params[L - 1][0]
    t5 = rnd(conv3d(h[L - 1], w5, np.zeros(w5.shape[0])))
    # middle: m = h_4 + W_5^T t5, masked by D_4 (h_4 is zero where D_4 is)
    u = [None] * L
    u[L - 1] = rnd(h[L - 1] + conv3d_transpose(t5, w5) * (h[L - 1] > 0))
    # transposed chain: u_l = D_l W_{l+1}^T u_{l+1}, o = W_1^T u_1
    for l in range(L - 2, 0, -1):
        u[l] = rnd(conv3d_transpose(u[l + 1], params[l][0]) * (h[l] > 0))
    o = conv3d_transpose(u[1], params[0][0])
    zc = u0 + o
    return zc[0] + 1j * zc[1], (h, u, t5)


def backward_spd(params, inter, dz, rnd=_identity):
    """Weight gradients of the symmetric form given dL/dz (biases: zero)."""
    h, u, t5 = inter
    L = len(params)
    gw = [np.zeros_like(w) for w, _ in params]
    zero = lambda w: np.zeros(w.shape[0])
    # adjoint of the transposed chain o = W_1^T u_1, u_l = D_l W_{l+1}^T u_{l+1}
    g = rnd(np.stack([dz.real, dz.imag]))
    for l in range(L - 1):
        w = params[l][0]
        gw[l] += conv3d_backward(g, w, u[l + 1])[1]
        g = rnd(conv3d(g, w, zero(w)) * (h[l + 1] > 0))
    # g = dL/dm (masked).  m = h_4 + W_5^T W_5 h_4:
    w5 = params[L - 1][0]
    q = rnd(conv3d(g, w5, zero(w5)))
    gw[L - 1] += conv3d_backward(h[L - 1], w5, q)[1] + conv3d_backward(g, w5, t5)[1]
    g = rnd(g + conv3d_transpose(q, w5) * (h[L - 1] > 0))   # D_4 dL/dh_4
    # back through the forward chain h_l = D_l W_l h_{l-1}, l = 4 .. 1
    for l in range(L - 2, -1, -1):
        if l < L - 2:
            g = rnd(g * (h[l + 1] > 0))
        gx, dw, _ = conv3d_backward(h[l], params[l][0], g)
        gw[l] += dw
        g = gx
    return [(w, np.zeros(b.shape)) for w, (_, b) in zip(gw, params)]


def loss_and_grads_spd(params, r, e, E=None, rnd=_identity):
    """Loss and gradients of the symmetric form: cosine loss (E None) or the
    energy loss with the operator callable E."""
    z, inter = forward_spd(params, r, rnd)
    if E is None:
        L, dz = loss(z, e), loss_grad_z(z, e)
    else:
        Ez = E(z)
        L, dz = loss_energy(z, r, e, Ez), loss_energy_grad_z(z, r, e, Ez)
    return L, backward_spd(params, inter, dz, rnd)


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); state = (t, m, v) lists."""
    t, m, v = state
    t += 1
    new = []
    for i, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        out = []
        for k, (p, gp) in enumerate(((w, gw), (b, gb))):
            m[i][k] = beta1 * m[i][k] + (1 - beta1) * gp
            v[i][k] = beta2 * v[i][k] + (1 - beta2) * gp * gp
            mh = m[i][k] / (1 - beta1 ** t)
            vh = v[i][k] / (1 - beta2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new, (t, m, v)


def adam_init(params):
    z = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]
    z2 = [[np.zeros_like(w), np.zeros_like(b)] for w, b in params]
    return (0, z, z2)


def bf16_round(a):
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
