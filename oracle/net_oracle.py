"""FP64 numpy oracle of the warm-start network (encoder-decoder that proposes the initial
gap state; it replaces the uniform random initial gap angles of Algorithm 2, whose MCMC
then runs unchanged).  The network is this project's own addition, not part of the
paper: its definition (layers, input encoding, loss, parameter layout) is the one the
library's mpr_net.h states, and this file writes that definition out plainly.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and nothing in the library).  It
shares no code with the CUDA path.

Precisions:
  * ``bf16_storage=False``: everything in float64 (pinned by finite differences and by
    scipy's correlate2d in the CPU tests);
  * ``bf16_storage=True``: the same arithmetic in float64, with values rounded to bf16
    (round to nearest even) where the library stores them in bf16: network input, conv
    weights, layer outputs, pooled maps and the ReLU-gated gradients.
The GPU tests apply the building blocks below (conv3x3, conv3x3_grad, pool, upsample and
their adjoints, circ_loss) to the kernels' own inputs of each step, layer by layer.

Arrays are NHWC: x[b, y, x, c].  Conv weights w[t, ci, co] with tap t = 3 dy + dx,
(dy, dx) in {0, 1, 2}^2 addressing input pixel (y + dy - 1, x + dx - 1), zero padding.
"""
from __future__ import annotations

import math

import numpy as np

LEVEL = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
CIN = [32, 32, 32, 64, 64, 128, 128, 256, 128 + 256, 128, 64 + 128, 64, 32 + 64, 32]
COUT = [32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32]
N_IN = 32
HEAD_C = 32
EPS_NORM = 1e-12            # added to u^2 + v^2 in the loss


# ------------------------------------------------------------------ precision
def bf16(x):
    """Round to the nearest bf16 value (ties to even), returned as float64.  The value is
    first rounded to float32 (the library rounds float32 results)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def to_bf16_bits(x):
    """bf16 bit patterns (uint16) of bf16(x)."""
    return (np.ascontiguousarray(bf16(x).astype(np.float32)).view(np.uint32) >> 16).astype(np.uint16)


def from_bf16_bits(b):
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ parameter layout
def layout():
    """Offsets of (W, b) per convolution and of the head in the parameter vector."""
    off = 0
    conv = []
    for l in range(14):
        ow = off
        off += 9 * CIN[l] * COUT[l]
        ob = off
        off += COUT[l]
        conv.append((ow, ob))
    owh = off
    off += 2 * HEAD_C
    obh = off
    off += 2
    return conv, owh, obh, off


def unpack(theta):
    conv, owh, obh, n = layout()
    assert theta.size == n
    Ws = [theta[ow:ow + 9 * CIN[l] * COUT[l]].reshape(9, CIN[l], COUT[l]).astype(np.float64)
          for l, (ow, ob) in enumerate(conv)]
    bs = [theta[ob:ob + COUT[l]].astype(np.float64) for l, (ow, ob) in enumerate(conv)]
    wh = theta[owh:owh + 2 * HEAD_C].reshape(HEAD_C, 2).astype(np.float64)
    bh = theta[obh:obh + 2].astype(np.float64)
    return Ws, bs, wh, bh


def pack(dWs, dbs, dwh, dbh):
    conv, owh, obh, n = layout()
    g = np.zeros(n, np.float64)
    for l, (ow, ob) in enumerate(conv):
        g[ow:ow + dWs[l].size] = dWs[l].ravel()
        g[ob:ob + dbs[l].size] = dbs[l]
    g[owh:owh + 2 * HEAD_C] = dwh.ravel()
    g[obh:obh + 2] = dbh
    return g


# ------------------------------------------------------------------ building blocks
def conv3x3(x, w, b=None):
    """out[b, y, x, co] = sum over taps and ci of x[b, y + dy - 1, x + dx - 1, ci] w[3 dy + dx, ci, co]
    (+ b[co]); pixels outside the image are zero.  Float64."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0))).astype(np.float64)
    wa = w.astype(np.float64)
    out = np.zeros((B, H, W, w.shape[2]))
    for t in range(9):
        dy, dx = divmod(t, 3)
        out += xp[:, dy:dy + H, dx:dx + W, :] @ wa[t]
    if b is not None:
        out += b.astype(np.float64)
    return out


def conv3x3_grad(x, w, g):
    """Gradients of sum(g * conv3x3(x, w)) w.r.t. x and w (the adjoint, tap by tap).  Float64."""
    B, H, W, Cin = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0))).astype(np.float64)
    dxp = np.zeros_like(xp)
    dw = np.zeros(w.shape)
    wa, ga = w.astype(np.float64), g.astype(np.float64)
    g2 = ga.reshape(-1, g.shape[3])
    for t in range(9):
        dy, dx = divmod(t, 3)
        dw[t] = xp[:, dy:dy + H, dx:dx + W, :].reshape(-1, Cin).T @ g2
        dxp[:, dy:dy + H, dx:dx + W, :] += ga @ wa[t].T
    return dxp[:, 1:H + 1, 1:W + 1, :], dw


def pool(x):
    """2 x 2 average pooling."""
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 0::2] + x[:, 1::2, 1::2])


def pool_adjoint(g):
    return 0.25 * np.repeat(np.repeat(g, 2, axis=1), 2, axis=2)


def upsample(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample_adjoint(g):
    return g[:, 0::2, 0::2] + g[:, 0::2, 1::2] + g[:, 1::2, 0::2] + g[:, 1::2, 1::2]


def net_input(z, mask, zmin, zmax, stride=1):
    """(cos theta, sin theta, 1) at sample sites, zeros at gap sites, padded to 32 channels;
    theta = q phi, q = 1/2, phi = 2 pi (z - zmin) / (zmax - zmin) (Eq. 1).  At stride S the
    frame pixel (Y, X) holds the mean of these over the S x S block of sites it stands for."""
    B, H, W = z.shape
    x = np.zeros((B, H, W, N_IN))
    for b in range(B):
        th = math.pi * (z[b].astype(np.float64) - zmin[b]) / (zmax[b] - zmin[b])
        s = mask[b] != 0
        x[b, :, :, 0] = np.where(s, np.cos(th), 0.0)
        x[b, :, :, 1] = np.where(s, np.sin(th), 0.0)
        x[b, :, :, 2] = np.where(s, 1.0, 0.0)
    if stride > 1:
        S = stride
        x = x.reshape(B, H // S, S, W // S, S, N_IN).mean(axis=(2, 4))
    return x


def circ_loss(uv, phi_t, mask, stride=1):
    """Mean over gap sites of 1 - cos(theta - theta_t), theta the direction of (u, v),
    theta_t = phi_t / 2; returns (loss, dL/duv).  At stride S every gap site of a frame
    pixel's S x S block takes that pixel's (u, v): the block's terms add up to
    n_g - (u Tc + v Ts) / |(u, v)|, (Tc, Ts) the sum of its gaps' (cos, sin) theta_t."""
    u, v = uv[..., 0], uv[..., 1]
    gap = (mask == 0).astype(np.float64)
    c = np.cos(0.5 * phi_t.astype(np.float64)) * gap
    s = np.sin(0.5 * phi_t.astype(np.float64)) * gap
    n_gap = int(gap.sum())
    if n_gap == 0:
        return 0.0, np.zeros_like(uv)
    if stride > 1:
        S = stride
        B, H, W = gap.shape
        blk = lambda a: a.reshape(B, H // S, S, W // S, S).sum(axis=(2, 4))
        c, s, gap = blk(c), blk(s), blk(gap)
    n = np.sqrt(u * u + v * v + EPS_NORM)
    dot = u * c + v * s
    loss = float(np.sum(gap - dot / n) / n_gap)
    du = (dot * u / n ** 3 - c / n) / n_gap
    dv = (dot * v / n ** 3 - s / n) / n_gap
    return loss, np.stack([du, dv], axis=-1)


# ------------------------------------------------------------------ the network
def _layer_input(l, x0, acts, pools):
    if l == 0:
        return x0
    if l in (2, 4, 6):
        return pools[l // 2 - 1]
    if l in (8, 10, 12):
        skip = {8: 5, 10: 3, 12: 1}[l]
        return np.concatenate([acts[skip], upsample(acts[l - 1])], axis=3)
    return acts[l - 1]


def forward(theta, z, mask, zmin, zmax, bf16_storage=False, stride=1):
    """Network output (u, v) per frame pixel (per site at stride 1), and the cache for backward."""
    r = bf16 if bf16_storage else (lambda a: a)
    Ws, bs, wh, bh = unpack(theta)
    Wr = [r(w) for w in Ws]
    x0 = r(net_input(z, mask, zmin, zmax, stride))
    acts, pools, ins = [None] * 14, [None] * 3, [None] * 14
    for l in range(14):
        xin = _layer_input(l, x0, acts, pools)
        ins[l] = xin
        acts[l] = r(np.maximum(conv3x3(xin, Wr[l], bs[l]), 0.0))
        if l in (1, 3, 5):
            pools[l // 2] = r(pool(acts[l]))
    uv = acts[13] @ wh + bh
    return uv, dict(Wr=Wr, wh=wh, acts=acts, ins=ins)


def loss_and_grad(theta, z, mask, phi_t, zmin, zmax, bf16_storage=False, stride=1):
    """Loss and gradient (same layout as theta) for one batch."""
    r = bf16 if bf16_storage else (lambda a: a)
    uv, cache = forward(theta, z, mask, zmin, zmax, bf16_storage, stride)
    loss, duv = circ_loss(uv, phi_t, mask, stride)
    acts, ins, Wr, wh = cache["acts"], cache["ins"], cache["Wr"], cache["wh"]
    dact = [None] * 14
    dact[13] = duv @ wh.T
    dwh = acts[13].reshape(-1, HEAD_C).T @ duv.reshape(-1, 2)
    dbh = duv.reshape(-1, 2).sum(axis=0)
    dWs, dbs = [None] * 14, [None] * 14

    def add(i, g):
        dact[i] = g if dact[i] is None else dact[i] + g

    for l in range(13, -1, -1):
        gl = r(np.where(acts[l] > 0, dact[l], 0.0))
        dbs[l] = gl.reshape(-1, COUT[l]).sum(axis=0)
        dx, dWs[l] = conv3x3_grad(ins[l], Wr[l], gl)
        if l == 0:
            continue
        if l in (2, 4, 6):
            add(l - 1, pool_adjoint(dx))
        elif l in (8, 10, 12):
            skip = {8: 5, 10: 3, 12: 1}[l]
            cs = COUT[skip]
            add(skip, dx[..., :cs])
            add(l - 1, upsample_adjoint(dx[..., cs:]))
        else:
            add(l - 1, dx)
    return loss, pack(dWs, dbs, dwh, dbh)


def warm_phi(uv):
    """Initial gap angle phi_0 = 2 theta_0, theta_0 the direction of (u, max(v, 0)) (the
    library keeps theta_0 < pi by taking v >= 1e-6 |u|)."""
    u, v = uv[..., 0], np.maximum(uv[..., 1], 1e-6 * np.abs(uv[..., 0]))
    return 2.0 * np.arctan2(v, u)


def init_params(seed=0, scale=1.0):
    """Random parameters with He-like scales (for tests; the library draws its own)."""
    rng = np.random.default_rng(seed)
    conv, owh, obh, n = layout()
    th = np.zeros(n)
    for l, (ow, ob) in enumerate(conv):
        fan = 9 * (3 if l == 0 else CIN[l])
        w = rng.normal(0, scale * math.sqrt(2.0 / fan), (9, CIN[l], COUT[l]))
        if l == 0:
            w[:, 3:, :] = 0.0
        th[ow:ow + w.size] = w.ravel()
        th[ob:ob + COUT[l]] = rng.normal(0, 0.05, COUT[l])
    th[owh:owh + 2 * HEAD_C] = rng.normal(0, math.sqrt(1.0 / HEAD_C), 2 * HEAD_C)
    th[obh:obh + 2] = rng.normal(0, 0.05, 2)
    return th
