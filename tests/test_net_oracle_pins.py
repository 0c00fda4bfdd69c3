"""Pins of the FP64 warm-start network oracle against things other than itself: scipy's
correlate2d, torch's bf16 rounding, adjoint identities, closed forms of the loss and
finite differences of the whole network."""
import math

import numpy as np
import pytest
from scipy.signal import correlate2d

import oracle.net_oracle as no


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e4, 1000),
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, -0.0]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(no.bf16(x), ref)
    assert no.bf16(1 + 2 ** -8) == 1.0                 # halfway: to the even neighbour (1.0)
    assert no.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6     # halfway: to the even neighbour
    assert np.array_equal(no.from_bf16_bits(no.to_bf16_bits(x)), no.bf16(x))


def test_conv_single_channel_is_scipy_correlate2d():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(7, 9))
    k = rng.normal(size=(3, 3))
    w = k.reshape(9, 1, 1)
    got = no.conv3x3(x[None, :, :, None], w)[0, :, :, 0]
    ref = correlate2d(x, k, mode="same", boundary="fill", fillvalue=0.0)
    assert np.allclose(got, ref, atol=1e-12)


def test_conv_channels_sum_and_bias():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 5, 6, 3))
    w = rng.normal(size=(9, 3, 2))
    b = rng.normal(size=2)
    got = no.conv3x3(x, w, b)
    for bb in range(2):
        for co in range(2):
            ref = sum(correlate2d(x[bb, :, :, ci], w[:, ci, co].reshape(3, 3), mode="same") for ci in range(3))
            assert np.allclose(got[bb, :, :, co], ref + b[co], atol=1e-12)


def test_conv_grad_is_the_adjoint():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 5, 4, 3))
    w = rng.normal(size=(9, 3, 2))
    g = rng.normal(size=(2, 5, 4, 2))
    dx, dw = no.conv3x3_grad(x, w, g)
    # <g, conv(x, w)> is bilinear: its derivative along (ex, ew) is <dx, ex> + <dw, ew>
    ex, ew = rng.normal(size=x.shape), rng.normal(size=w.shape)
    f = lambda t: float(np.sum(g * no.conv3x3(x + t * ex, w + t * ew)))
    eps = 1e-4
    fd = (f(eps) - f(-eps)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(dx * ex) + np.sum(dw * ew)), rel=1e-9)
    # the data gradient alone equals the convolution with the point-reflected kernel
    wf = w[::-1].transpose(0, 2, 1)
    assert np.allclose(dx, no.conv3x3(g, wf), atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 8, 6, 3))
    y = rng.normal(size=(2, 4, 3, 3))
    assert np.sum(no.pool(x) * y) == pytest.approx(np.sum(x * no.pool_adjoint(y)), rel=1e-12)
    assert np.sum(no.upsample(y) * x) == pytest.approx(np.sum(y * no.upsample_adjoint(x)), rel=1e-12)
    assert np.allclose(no.pool(np.ones_like(x)), 1.0)
    assert np.allclose(no.pool(no.upsample(y)), y)


def test_input_encoding_follows_eq1_half_angle():
    z = np.array([[[0.0, 10.0, 5.0, 7.0]]], np.float32)        # B=1, H=1, W=4
    m = np.array([[[1, 1, 1, 0]]], np.uint8)
    x = no.net_input(z, m, [0.0], [10.0])
    assert x.shape == (1, 1, 4, 32)
    assert np.allclose(x[0, 0, 0, :3], [1, 0, 1])              # zmin: theta 0
    assert np.allclose(x[0, 0, 1, :3], [-1, 0, 1], atol=1e-15)  # zmax: theta pi
    assert np.allclose(x[0, 0, 2, :3], [0, 1, 1], atol=1e-15)   # midpoint: theta pi/2
    assert np.all(x[0, 0, 3] == 0) and np.all(x[..., 3:] == 0)


def test_circular_loss_closed_forms_and_gradient():
    phi_t = np.array([[[1.0, 2.0, 4.0, 0.5]]])
    m = np.array([[[0, 0, 0, 1]]], np.uint8)                    # last site is a sample: ignored
    th = 0.5 * phi_t
    aligned = np.stack([3 * np.cos(th), 3 * np.sin(th)], -1)
    assert no.circ_loss(aligned, phi_t, m)[0] == pytest.approx(0.0, abs=1e-12)
    assert no.circ_loss(-aligned, phi_t, m)[0] == pytest.approx(2.0, abs=1e-12)
    ortho = np.stack([-np.sin(th), np.cos(th)], -1)
    assert no.circ_loss(ortho, phi_t, m)[0] == pytest.approx(1.0, abs=1e-12)
    rng = np.random.default_rng(5)
    uv = rng.normal(size=(1, 1, 4, 2))
    L, d = no.circ_loss(uv, phi_t, m)
    e = rng.normal(size=uv.shape)
    eps = 1e-6
    fd = (no.circ_loss(uv + eps * e, phi_t, m)[0] - no.circ_loss(uv - eps * e, phi_t, m)[0]) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(d * e)), rel=1e-7)
    assert np.all(d[0, 0, 3] == 0)
    assert no.circ_loss(uv, phi_t, np.ones_like(m))[0] == 0.0


def _batch(seed, B, H, W):
    rng = np.random.default_rng(seed)
    z = rng.normal(50, 10, (B, H, W)).astype(np.float32)
    m = (rng.random((B, H, W)) > 0.4).astype(np.uint8)
    phi = rng.uniform(0, 2 * math.pi, (B, H, W)).astype(np.float32)
    zmin = np.array([z[b][m[b] == 1].min() for b in range(B)], np.float64)
    zmax = np.array([z[b][m[b] == 1].max() for b in range(B)], np.float64)
    return z, m, phi, zmin, zmax


def test_layout_size():
    conv, owh, obh, n = no.layout()
    expect = sum(9 * a * b + b for a, b in zip(no.CIN, no.COUT)) + 2 * 32 + 2
    assert n == expect and obh == n - 2 and owh == n - 66


def test_network_gradient_matches_finite_differences():
    z, m, phi, zmin, zmax = _batch(6, 2, 8, 16)
    th = no.init_params(7)
    L, g = no.loss_and_grad(th, z, m, phi, zmin, zmax)
    rng = np.random.default_rng(8)
    for _ in range(2):
        d = rng.normal(size=th.size)
        eps = 1e-6
        Lp = no.loss_and_grad(th + eps * d, z, m, phi, zmin, zmax)[0]
        Lm = no.loss_and_grad(th - eps * d, z, m, phi, zmin, zmax)[0]
        fd = (Lp - Lm) / (2 * eps)
        assert fd == pytest.approx(float(g @ d), rel=1e-5, abs=1e-9)
    # single coordinates of the first layer, a decoder layer and the head
    conv, owh, obh, n = no.layout()
    for idx in (conv[0][0] + 5, conv[0][1] + 1, conv[8][0] + 1234, conv[13][1] + 3, owh + 7, obh + 1):
        e = np.zeros(n)
        e[idx] = 1.0
        eps = 1e-6
        fd = (no.loss_and_grad(th + eps * e, z, m, phi, zmin, zmax)[0] -
              no.loss_and_grad(th - eps * e, z, m, phi, zmin, zmax)[0]) / (2 * eps)
        assert fd == pytest.approx(g[idx], rel=1e-4, abs=1e-8)


def test_bf16_storage_is_a_small_perturbation_of_fp64():
    z, m, phi, zmin, zmax = _batch(9, 1, 16, 8)
    th = no.init_params(10)
    L64, g64 = no.loss_and_grad(th, z, m, phi, zmin, zmax)
    Lb, gb = no.loss_and_grad(th, z, m, phi, zmin, zmax, bf16_storage=True)
    assert abs(Lb - L64) < 2e-2 * abs(L64)
    assert np.linalg.norm(gb - g64) < 0.1 * np.linalg.norm(g64)


def test_warm_phi_range():
    uv = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [-1.0, -5.0], [2.0, -1.0]])
    phi = no.warm_phi(uv)
    assert phi[0] == pytest.approx(2e-6, rel=1e-6) and phi[1] == pytest.approx(math.pi)
    assert np.all(phi < 2 * math.pi) and np.all(phi >= 0)
    assert phi[2] == pytest.approx(2 * math.pi, abs=1e-5)


# ---------------------------------------------------------------- stride 2 (coarse frame)
def test_stride2_loss_is_the_site_loss_of_the_upsampled_prediction():
    # every gap site of a 2 x 2 block takes its frame pixel's (u, v): the block-sum form
    # must equal the per-site definition on the nearest-upsampled prediction, and its
    # gradient the block sum of the per-site gradient (chain rule of the upsampling)
    rng = np.random.default_rng(21)
    B, H, W = 2, 8, 12
    m = (rng.random((B, H, W)) > 0.45).astype(np.uint8)
    phi = rng.uniform(0, 2 * math.pi, (B, H, W))
    uv = rng.normal(size=(B, H // 2, W // 2, 2))
    L2, g2 = no.circ_loss(uv, phi, m, stride=2)
    up = uv.repeat(2, axis=1).repeat(2, axis=2)
    L1, g1 = no.circ_loss(up, phi, m, stride=1)
    assert L2 == pytest.approx(L1, rel=1e-13)
    assert np.allclose(g2, g1.reshape(B, H // 2, 2, W // 2, 2, 2).sum(axis=(2, 4)), rtol=0, atol=1e-14)
    # direct: mean over gaps of 1 - cos(theta(pixel) - phi/2)
    th = np.arctan2(up[..., 1], up[..., 0])
    direct = np.mean((1.0 - np.cos(th - 0.5 * phi))[m == 0])
    assert L2 == pytest.approx(direct, rel=1e-6)


def test_stride2_input_is_block_mean_of_site_input():
    z, m, phi, zmin, zmax = _batch(22, 2, 8, 16)
    x1 = no.net_input(z, m, zmin, zmax)
    x2 = no.net_input(z, m, zmin, zmax, stride=2)
    assert x2.shape == (2, 4, 8, no.N_IN)
    blk = x1[:, 0:2, 2:4, :3]                          # the 2 x 2 block of frame pixel (0, 1)
    assert np.allclose(x2[:, 0, 1, :3], blk.mean(axis=(1, 2)), rtol=0, atol=1e-15)
    assert np.all((x2[..., 2] >= 0) & (x2[..., 2] <= 1)) and np.all(x2[..., 3:] == 0)


def test_stride2_network_gradient_matches_finite_differences():
    z, m, phi, zmin, zmax = _batch(23, 2, 16, 16)
    th = no.init_params(24)
    L, g = no.loss_and_grad(th, z, m, phi, zmin, zmax, stride=2)
    rng = np.random.default_rng(25)
    for _ in range(2):
        d = rng.normal(size=th.size)
        eps = 1e-6
        Lp = no.loss_and_grad(th + eps * d, z, m, phi, zmin, zmax, stride=2)[0]
        Lm = no.loss_and_grad(th - eps * d, z, m, phi, zmin, zmax, stride=2)[0]
        assert (Lp - Lm) / (2 * eps) == pytest.approx(float(g @ d), rel=1e-5, abs=1e-9)
