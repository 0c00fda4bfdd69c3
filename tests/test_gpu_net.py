"""Warm-start network on the GPU against the FP64 oracle (oracle/net_oracle.py): single
convolutions (forward, data and weight gradients), every layer of the whole network's
forward and backward pass, the Adam step, training progress and the warm-start write into
a context.

Tolerances.  The kernels multiply bf16 values exactly and accumulate in fp32; the oracle
uses the same bf16 values and accumulates in fp64.  A value the kernels store in bf16 can
therefore differ from the exact one by half a bf16 unit (round to nearest) plus the fp32
accumulation error, and an fp32 value by the accumulation error alone.  The whole network
is checked step by step: each layer's output, pooled map, gradient and weight gradient is
compared element by element with the oracle applied to the kernels' own inputs of that step
(read back with mpr_net_tensor), so rounding differences never accumulate across layers and
every element is held to the single-step bound.
"""
import math

import numpy as np
import pytest

import oracle.net_oracle as no
from paper_1811_01604_gb300 import mpr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda().contiguous()


def _bits(x):
    return _dev(no.to_bf16_bits(x).view(np.int16))


def _from_bits(t):
    return no.from_bf16_bits(t.cpu().numpy().view(np.uint16))


CONV_CASES = [  # B, H, W, Cin, Cout: ragged tile edges, every N tile width, both tile kinds
    (2, 20, 13, 32, 32),     # halo tile (N <= 64, weights resident), one channel block
    (2, 18, 20, 96, 32),     # halo tile, two channel blocks (the second half zero-padded)
    (1, 16, 24, 64, 64),     # halo tile, N = 64
    (1, 12, 20, 192, 64),    # halo tile, weights streamed per channel block (N = 64)
    (2, 10, 16, 192, 32),    # halo tile, weights streamed per channel block (N = 32)
    (1, 9, 30, 96, 64),      # general tile
    (2, 16, 16, 64, 96),     # general tile, N = 96
    (1, 7, 5, 32, 256),      # general tile, N = 256
    (1, 6, 34, 128, 128),    # general tile, two channel blocks
    (3, 1, 1, 32, 32),       # tiles mostly outside the image
]


@pytest.mark.parametrize("B,H,W,Cin,Cout", CONV_CASES)
def test_conv3x3_forward_matches_oracle(B, H, W, Cin, Cout):
    rng = np.random.default_rng(B * 1000 + Cin + Cout)
    x = no.bf16(rng.normal(size=(B, H, W, Cin)))
    w = no.bf16(rng.normal(0, 1 / math.sqrt(9 * Cin), size=(9, Cin, Cout)))
    b = rng.normal(0, 0.1, Cout).astype(np.float32)
    for relu in (0, 1):
        out = torch.zeros((B, H, W, Cout), dtype=torch.int16, device="cuda")
        mpr.mpr_net_conv3x3(_bits(x), B, H, W, Cin, _bits(w), _dev(b), Cout, relu, out)
        torch.cuda.synchronize()
        got = _from_bits(out)
        acc = no.conv3x3(x, w, b.astype(np.float64))
        ref = no.bf16(np.maximum(acc, 0) if relu else acc)
        # one bf16 unit of the result is at most 2^-7 of its magnitude
        tol = 2.0 ** -7 * np.abs(ref) + 1e-6 * np.abs(acc).max()
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (int(bad.sum()), got[bad][:4], ref[bad][:4], acc[bad][:4])
        assert np.mean(got == ref) > 0.99


@pytest.mark.parametrize("B,H,W,Cin,Cout", CONV_CASES)
def test_conv3x3_backward_matches_oracle(B, H, W, Cin, Cout):
    rng = np.random.default_rng(B * 77 + Cin * 3 + Cout)
    x = no.bf16(rng.normal(size=(B, H, W, Cin)))
    w = no.bf16(rng.normal(0, 1 / math.sqrt(9 * Cin), size=(9, Cin, Cout)))
    g = no.bf16(rng.normal(size=(B, H, W, Cout)))
    din = torch.full((B, H, W, Cin), 7.0, dtype=torch.float32, device="cuda")   # overwritten
    dw0 = rng.normal(size=(9, Cin, Cout)).astype(np.float32)                   # added to
    dw = _dev(dw0)
    scratch = torch.zeros((9, Cin, Cout), dtype=torch.int16, device="cuda")
    mpr.mpr_net_conv3x3_bwd(_bits(x), _bits(g), B, H, W, Cin, _bits(w), Cout, din, dw, scratch)
    torch.cuda.synchronize()
    rdx, rdw = no.conv3x3_grad(x, w, g)
    gx = din.cpu().numpy().astype(np.float64)
    gw = dw.cpu().numpy().astype(np.float64) - dw0
    ex = np.abs(gx - rdx) - (1e-4 * np.abs(rdx) + 1e-5 * np.abs(rdx).max())
    ew = np.abs(gw - rdw) - (1e-4 * np.abs(rdw) + 1e-5 * np.abs(rdw).max() + 1e-6)
    assert ex.max() <= 0, (float(ex.max()), float(np.abs(rdx).max()))
    assert ew.max() <= 0, (float(ew.max()), float(np.abs(rdw).max()))


def _batch(seed, B, H, W, p=0.4):
    rng = np.random.default_rng(seed)
    z = rng.normal(50, 10, (B, H, W)).astype(np.float32)
    m = (rng.random((B, H, W)) > p).astype(np.uint8)
    phi = rng.uniform(0, 2 * math.pi, (B, H, W)).astype(np.float32)
    zmin = np.array([z[b][m[b] == 1].min() for b in range(B)], np.float64)
    zmax = np.array([z[b][m[b] == 1].max() for b in range(B)], np.float64)
    return z, m, phi, zmin, zmax


def _blocks():
    conv, owh, obh, n = no.layout()
    out = []
    for l, (ow, ob) in enumerate(conv):
        out.append((f"W{l}", ow, ob))
        out.append((f"b{l}", ob, ob + no.COUT[l]))
    out.append(("Wh", owh, obh))
    out.append(("bh", obh, n))
    return out


# Element-wise check of one tensor.  got: the kernels' values; exact: the value the oracle
# computes in FP64 from the kernels' own inputs of that step; absum: the sum of the absolute
# values of the terms behind each element.  A kernel value may differ from the exact one by
# its FP32 accumulation error (at most REL_ACC of absum: products of bf16 values are exact in
# FP32, and the sums of a few thousand terms carry a relative rounding error far below 2^-16)
# plus, for values stored in bf16, half a bf16 unit of the larger of the two (round to
# nearest).  Returns the number of elements outside that bound.
REL_ACC = 2.0 ** -16


def _half_ulp_bf16(a):
    e = np.floor(np.log2(np.maximum(np.abs(a), 1e-300)))
    return np.where(a == 0, 0.0, 2.0 ** (e - 8))


def _outside(got, exact, absum, bf16_out):
    got = np.asarray(got, np.float64)
    allowed = REL_ACC * absum + 1e-30
    if bf16_out:
        allowed = allowed + _half_ulp_bf16(np.maximum(np.abs(got), np.abs(exact)))
    return int((np.abs(got - exact) > allowed).sum())


def _loss_grad_terms(uv, phi, mask, S):
    """Magnitudes of the two terms of dL/du and dL/dv (circ_loss), |dot u| / n^3 + |Tc| / n
    and |dot v| / n^3 + |Ts| / n over the gap count: the FP32 kernel forms their
    difference, so its rounding error scales with them, not with the (cancelling) result."""
    B, H, W = mask.shape
    gap = (mask == 0).astype(np.float64)
    c = np.cos(0.5 * phi.astype(np.float64)) * gap
    sn = np.sin(0.5 * phi.astype(np.float64)) * gap
    blk = lambda a: a.reshape(B, H // S, S, W // S, S).sum(axis=(2, 4))
    c, sn = blk(c), blk(sn)
    u, v = uv[..., 0], uv[..., 1]
    n = np.sqrt(u * u + v * v + no.EPS_NORM)
    dot = np.abs(u * c + v * sn)
    ng = max(1.0, gap.sum())
    return np.stack([(dot * np.abs(u) / n ** 3 + np.abs(c) / n) / ng,
                     (dot * np.abs(v) / n ** 3 + np.abs(sn) / n) / ng], axis=-1)


def _gpu_tensors(net, B, Hf, Wf):
    """The network's internal tensors after mpr_net_loss_grad, as float64 arrays."""
    def bf(kind, i, shape):
        t = np.zeros(shape, np.uint16)
        mpr.mpr_net_tensor(net, kind, i, t)
        return no.from_bf16_bits(t)

    def f32(kind, i, shape):
        t = np.zeros(shape, np.float32)
        mpr.mpr_net_tensor(net, kind, i, t)
        return t.astype(np.float64)

    lv = lambda l: (B, Hf >> no.LEVEL[l], Wf >> no.LEVEL[l], no.COUT[l])
    x0 = bf(mpr.MPR_NET_T_INPUT, 0, (B, Hf, Wf, no.N_IN))
    acts = [bf(mpr.MPR_NET_T_ACT, l, lv(l)) for l in range(14)]
    pools = [bf(mpr.MPR_NET_T_POOL, i, (B, Hf >> (i + 1), Wf >> (i + 1), no.COUT[2 * i + 1])) for i in range(3)]
    dacts = [f32(mpr.MPR_NET_T_DACT, l, lv(l)) for l in range(14)]
    uv = f32(mpr.MPR_NET_T_OUT, 0, (B, Hf, Wf, 2))
    return x0, acts, pools, dacts, uv


@pytest.mark.parametrize("B,H,W,S", [(2, 16, 24, 1), (1, 32, 32, 1), (2, 32, 48, 2), (1, 64, 32, 2),
                                     (2, 64, 32, 4), (1, 64, 64, 8)])
def test_network_layer_by_layer_matches_oracle(B, H, W, S):
    # Every step of the forward and backward pass is checked element by element against the
    # FP64 oracle applied to the kernels' own inputs of that step (their stored bf16
    # activations, pooled maps and FP32 gradients), so one step's rounding never becomes the
    # next step's reference: each tensor is held to the bound of a single step (_outside)
    # and no element may fall outside it.
    z, m, phi, zmin, zmax = _batch(B * H + W, B, H, W)
    th = no.init_params(11).astype(np.float32)
    Hf, Wf = H // S, W // S
    net = mpr.mpr_net_create(0, stride=S)
    try:
        assert mpr.mpr_net_stride(net) == S
        assert mpr.mpr_net_num_params(net) == th.size
        mpr.mpr_net_set_params(net, th)
        back = np.zeros_like(th)
        mpr.mpr_net_get_params(net, back)
        assert np.array_equal(back, th)
        mpr.mpr_net_zero_grads(net)
        loss = mpr.mpr_net_loss_grad(net, _dev(z), _dev(m), _dev(phi), zmin, zmax, B, H, W)
        g = np.zeros_like(th)
        mpr.mpr_net_get_grads(net, g)
        x0, acts, pools, dacts, uv = _gpu_tensors(net, B, Hf, Wf)
    finally:
        mpr.mpr_net_free(net)
    Ws, bs, wh, bh = no.unpack(th.astype(np.float64))
    Wr = [no.bf16(w) for w in Ws]
    bad = {}

    # input encoding: cos, sin of the Eq. 1 half angle and the sample indicator, block means
    # at stride S, in bf16 (the kernel evaluates them in FP32: slack 1e-6 of the value)
    ref = no.net_input(z, m, zmin, zmax, S)
    bad["input"] = _outside(x0, ref, 1e-6 / REL_ACC * np.abs(ref) + 1e-6 / REL_ACC, True)

    def layer_in(l):
        if l == 0:
            return x0
        if l in (2, 4, 6):
            return pools[l // 2 - 1]
        if l in (8, 10, 12):
            skip = {8: 5, 10: 3, 12: 1}[l]
            return np.concatenate([acts[skip], no.upsample(acts[l - 1])], axis=3)
        return acts[l - 1]

    # forward: each convolution (+ bias, ReLU) and each pooled map from the stored inputs
    for l in range(14):
        xin = layer_in(l)
        exact = np.maximum(no.conv3x3(xin, Wr[l], bs[l]), 0.0)
        absum = no.conv3x3(np.abs(xin), np.abs(Wr[l]), np.abs(bs[l]))
        bad[f"act{l}"] = _outside(acts[l], exact, absum, True)
    for i in range(3):
        a = acts[2 * i + 1]
        bad[f"pool{i}"] = _outside(pools[i], no.pool(a), no.pool(np.abs(a)), True)
    # head (FP32) and loss
    bad["head"] = _outside(uv, acts[13] @ wh + bh, np.abs(acts[13]) @ np.abs(wh) + np.abs(bh), False)
    rloss, duv = no.circ_loss(uv, phi, m, S)
    assert loss == pytest.approx(rloss, rel=1e-5, abs=1e-9)

    # backward: the head's gradients and the gradient w.r.t. the last activation; the loss
    # gradient is a difference of two terms in FP32 (relative rounding 1e-5 of their size,
    # with the FP32 sine and cosine of the targets)
    conv, owh, obh, _ = no.layout()
    dterm = 1e-5 / REL_ACC * _loss_grad_terms(uv, phi, m, S)
    bad["dact13"] = _outside(dacts[13], duv @ wh.T, dterm @ np.abs(wh.T), False)
    bad["dWh"] = _outside(g[owh:obh].reshape(no.HEAD_C, 2),
                          acts[13].reshape(-1, no.HEAD_C).T @ duv.reshape(-1, 2),
                          np.abs(acts[13]).reshape(-1, no.HEAD_C).T @ dterm.reshape(-1, 2), False)
    bad["dbh"] = _outside(g[obh:obh + 2], duv.reshape(-1, 2).sum(0), dterm.reshape(-1, 2).sum(0), False)
    # every convolution: weight and bias gradients from the stored gated gradient, and the
    # data gradient it sends to the layers below (added up where a tensor feeds two layers)
    dx_to = [np.zeros_like(a) for a in acts]
    dx_abs = [np.zeros_like(a) for a in acts]
    for l in range(13, -1, -1):
        gl = no.bf16(np.where(acts[l] > 0, dacts[l], 0.0))        # the kernels' gated bf16 gradient
        xin = layer_in(l)
        dx, dW = no.conv3x3_grad(xin, Wr[l], gl)
        ax, aW = no.conv3x3_grad(np.abs(xin), np.abs(Wr[l]), np.abs(gl))
        ow, ob = conv[l]
        bad[f"dW{l}"] = _outside(g[ow:ob].reshape(dW.shape), dW, aW, False)
        bad[f"db{l}"] = _outside(g[ob:ob + no.COUT[l]], gl.reshape(-1, no.COUT[l]).sum(0),
                                 np.abs(gl).reshape(-1, no.COUT[l]).sum(0), False)
        if l == 0:
            continue
        if l in (2, 4, 6):
            dx_to[l - 1] += no.pool_adjoint(dx)
            dx_abs[l - 1] += no.pool_adjoint(ax)
        elif l in (8, 10, 12):
            skip = {8: 5, 10: 3, 12: 1}[l]
            cs = no.COUT[skip]
            dx_to[skip] += dx[..., :cs]
            dx_abs[skip] += ax[..., :cs]
            dx_to[l - 1] += no.upsample_adjoint(dx[..., cs:])
            dx_abs[l - 1] += no.upsample_adjoint(ax[..., cs:])
        else:
            dx_to[l - 1] += dx
            dx_abs[l - 1] += ax
    for l in range(13):
        bad[f"dact{l}"] = _outside(dacts[l], dx_to[l], dx_abs[l], False)
    assert not any(bad.values()), {k: v for k, v in bad.items() if v}


def test_adam_first_step_closed_form():
    B, H, W = 2, 16, 16
    z, m, phi, zmin, zmax = _batch(3, B, H, W)
    net = mpr.mpr_net_create(5)
    try:
        w0 = np.zeros(mpr.mpr_net_num_params(net), np.float32)
        mpr.mpr_net_get_params(net, w0)
        mpr.mpr_net_zero_grads(net)
        mpr.mpr_net_loss_grad(net, _dev(z), _dev(m), _dev(phi), zmin, zmax, B, H, W)
        g = np.zeros_like(w0)
        mpr.mpr_net_get_grads(net, g)
        lr = 1e-3
        mpr.mpr_net_adam_step(net, lr)
        w1 = np.zeros_like(w0)
        mpr.mpr_net_get_params(net, w1)
        g2 = np.zeros_like(w0)
        mpr.mpr_net_get_grads(net, g2)
    finally:
        mpr.mpr_net_free(net)
    # t = 1: bias-corrected moments are g and g^2, so the step is lr g / (|g| + eps)
    g64 = g.astype(np.float64)
    expect = w0 - lr * g64 / (np.abs(g64) + 1e-8)
    assert np.allclose(w1, expect, rtol=1e-5, atol=1e-7)
    assert np.all(g2 == 0)


def test_training_fits_the_truth_of_a_fixed_batch():
    """Targets: the Eq. 1 angles of the hidden truth at the gaps; the loss must fall."""
    from paper_1811_01604_gb300 import synth
    B, H, W = 4, 32, 32
    zs = torch.stack([synth.wm_field_gpu(H, W, 0.5, 4.0, 40 + b) for b in range(B)]).contiguous()
    ms = torch.stack([synth.mask_uniform_gpu(H, W, 0.33, 80 + b) for b in range(B)]).contiguous()
    zmin = np.array([float(zs[b][ms[b] == 1].min()) for b in range(B)])
    zmax = np.array([float(zs[b][ms[b] == 1].max()) for b in range(B)])
    phi = torch.stack([2 * math.pi * (zs[b].double() - zmin[b]) / (zmax[b] - zmin[b]) for b in range(B)])
    phi = phi.clamp(0, 2 * math.pi).float().contiguous()
    net = mpr.mpr_net_create(1)
    try:
        losses = [mpr.mpr_net_train_step(net, zs, ms, phi, zmin, zmax, B, H, W, 2e-3) for _ in range(150)]
    finally:
        mpr.mpr_net_free(net)
    assert all(np.isfinite(losses))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:5])


def _ctx_grid(H, W, seed):
    from paper_1811_01604_gb300 import synth
    z = synth.wm_field_gpu(H, W, 0.5, 8.0, seed)
    m = synth.mask_uniform_gpu(H, W, 0.4, seed + 1)
    return z, m


@pytest.mark.parametrize("shapes,S", [([(64, 64)], 1), ([(61, 45)], 1),
                                      ([(64, 64), (64, 64), (40, 48), (33, 70)], 1),
                                      ([(61, 45)], 2), ([(64, 64), (40, 48), (33, 70)], 2),
                                      ([(61, 45), (64, 64)], 4), ([(61, 45), (64, 70)], 8)])
def test_warmstart_writes_the_network_state_into_gap_sites(shapes, S):
    grids = [_ctx_grid(H, W, 7 + i) for i, (H, W) in enumerate(shapes)]
    net = mpr.mpr_net_create(3, stride=S)
    ctx = mpr.mpr_init_batch([g[0] for g in grids], [g[1] for g in grids], mpr.mpr_default_params(seed=1))
    try:
        before = []
        for i, (H, W) in enumerate(shapes):
            phi = torch.zeros((H, W), dtype=torch.float32, device="cuda")
            mpr.mpr_get_state_batch(ctx, i, phi)
            before.append(phi.cpu().numpy())
        mpr.mpr_warmstart_init(ctx, net)
        for i, (H, W) in enumerate(shapes):
            info = mpr.mpr_batch_info(ctx, i)
            phi = torch.zeros((H, W), dtype=torch.float32, device="cuda")
            mpr.mpr_get_state_batch(ctx, i, phi)
            phi = phi.cpu().numpy()
            # the network frame: ceil(side / S) rounded up to a multiple of 8, S sites per pixel
            Hp, Wp = ((H + S - 1) // S + 7) // 8 * 8 * S, ((W + S - 1) // S + 7) // 8 * 8 * S
            zp = torch.zeros((1, Hp, Wp), dtype=torch.float32, device="cuda")
            mp = torch.zeros((1, Hp, Wp), dtype=torch.uint8, device="cuda")
            zp[0, :H, :W] = grids[i][0]
            mp[0, :H, :W] = grids[i][1]
            uv = torch.zeros((1, Hp // S, Wp // S, 2), dtype=torch.float32, device="cuda")
            mpr.mpr_net_forward(net, zp, mp, [info["zmin"]], [info["zmax"]], 1, Hp, Wp, uv)
            up = uv.cpu().numpy()[0].repeat(S, axis=0).repeat(S, axis=1)      # nearest upsampling
            want = no.warm_phi(up[:H, :W].astype(np.float64))
            gap = grids[i][1].cpu().numpy() == 0
            d = np.abs(phi[gap] - want[gap])
            assert d.max() < 1e-5
            assert np.array_equal(phi[~gap], before[i][~gap])        # samples untouched
            assert np.all(phi[gap] >= 0) and np.all(phi[gap] < 2 * math.pi)
        # the MCMC runs on from the warm state
        mpr.mpr_estimate_T(ctx)
        mpr.mpr_equilibrate(ctx)
    finally:
        mpr.mpr_free(ctx)
        mpr.mpr_net_free(net)


def test_rejects_bad_shapes():
    net = mpr.mpr_net_create(0)
    try:
        z = torch.zeros((1, 12, 16), device="cuda")
        m = torch.zeros((1, 12, 16), dtype=torch.uint8, device="cuda")
        uv = torch.zeros((1, 12, 16, 2), device="cuda")
        with pytest.raises(mpr.MprError):
            mpr.mpr_net_forward(net, z, m, [0.0], [1.0], 1, 12, 16, uv)
    finally:
        mpr.mpr_net_free(net)
