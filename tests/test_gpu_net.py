"""Warm-start network on the GPU against the FP64 oracle (oracle/net_oracle.py): single
convolutions (forward, data and weight gradients), the whole network's output, loss and
gradient, the Adam step, training progress and the warm-start write into a context.

Tolerances.  The kernels multiply bf16 values exactly and accumulate in fp32; the oracle
uses the same bf16 values and accumulates in fp64, rounding to bf16 where the kernels
store bf16.  A stored bf16 value can therefore differ by one bf16 unit (at most 2^-7 of
its magnitude) where the fp32 sum lies within its rounding error of a bf16 rounding
boundary; everything else differs by fp32 accumulation error (about 1e-6 relative).  In
a single convolution that bounds the error directly.  Through the whole network such
flips cascade (deep layers end up with a large share of values one unit apart), so the
whole-network tolerance is measured, not assumed: the oracle is re-run with fp32
accumulation, and the GPU must be within 4x that run's distance to the fp64-accumulated
reference (plus a small floor).
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


@pytest.mark.parametrize("B,H,W,S", [(2, 16, 24, 1), (1, 32, 32, 1), (2, 32, 48, 2), (1, 64, 32, 2)])
def test_network_output_loss_and_gradient_match_oracle(B, H, W, S):
    z, m, phi, zmin, zmax = _batch(B * H + W, B, H, W)
    th = no.init_params(11).astype(np.float32)
    net = mpr.mpr_net_create(0, stride=S)
    try:
        assert mpr.mpr_net_stride(net) == S
        assert mpr.mpr_net_num_params(net) == th.size
        mpr.mpr_net_set_params(net, th)
        back = np.zeros_like(th)
        mpr.mpr_net_get_params(net, back)
        assert np.array_equal(back, th)
        uv = torch.zeros((B, H // S, W // S, 2), dtype=torch.float32, device="cuda")
        mpr.mpr_net_forward(net, _dev(z), _dev(m), zmin, zmax, B, H, W, uv)
        mpr.mpr_net_zero_grads(net)
        loss = mpr.mpr_net_loss_grad(net, _dev(z), _dev(m), _dev(phi), zmin, zmax, B, H, W)
        g = np.zeros_like(th)
        mpr.mpr_net_get_grads(net, g)
    finally:
        mpr.mpr_net_free(net)
    th64 = th.astype(np.float64)
    ruv, _ = no.forward(th64, z, m, zmin, zmax, bf16_storage=True, stride=S)
    rloss, rg = no.loss_and_grad(th64, z, m, phi, zmin, zmax, bf16_storage=True, stride=S)
    # the same bf16 reference accumulated in fp32: its distance to rg is the sensitivity
    # of this network's gradient to one-unit bf16 rounding flips
    # ... in two tap orders and with truncated sums (the tensor cores' adders truncate, so
    # flips land elsewhere); the largest distance is the sensitivity
    runs = ((False, False), (True, False), (False, True))
    euvs = [no.forward(th64, z, m, zmin, zmax, bf16_storage=True, acc32=True, stride=S, rev=rv, chop=ch)[0]
            for rv, ch in runs]
    egs = [no.loss_and_grad(th64, z, m, phi, zmin, zmax, bf16_storage=True, acc32=True, stride=S, rev=rv,
                            chop=ch)[1] for rv, ch in runs]
    guv = uv.cpu().numpy().astype(np.float64)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(guv, ruv) <= 4 * max(rel(e, ruv) for e in euvs) + 1e-3
    assert loss == pytest.approx(rloss, rel=2e-3)
    for name, a, b in _blocks():
        ref, got = rg[a:b], g[a:b].astype(np.float64)
        nr = np.linalg.norm(ref)
        if nr == 0:
            assert np.linalg.norm(got) <= 1e-6
            continue
        err, sens = rel(got, ref), max(rel(e[a:b], ref) for e in egs)
        cos = float(got @ ref) / (np.linalg.norm(got) * nr)
        assert err <= 4 * sens + 2e-3 and cos > 0.995, (name, err, sens, cos)
    assert rel(g, rg) <= 4 * max(rel(e, rg) for e in egs) + 1e-3


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
                                      ([(61, 45)], 2), ([(64, 64), (40, 48), (33, 70)], 2)])
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
