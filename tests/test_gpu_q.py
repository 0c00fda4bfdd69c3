"""Couplings q < 1/2 (Eq. 2 bounds q by 1/2; the paper fixes q = 1/2 and leaves fitting q
to data open): the list kernels keep theta = q phi on the arc [0, 2 pi q), reflect only
inside it and turn proposals that leave it by -+2 pi q (the modulo 2 pi of phi).

  * FP64 (MPR_PREC_F64): trajectories equal to the FP64 oracle's over 200 sweeps
    (1e-9 rad; rounding alone separates them), and a whole fill at q = 0.3 equal to the
    oracle's (e_s, T-hat, relaxation length, final state, zhat to float rounding);
  * FP32: per sweep from the same state, |d phi| <= 1e-5 rad where decisions agree and
    at most 1e-6 of the decisions flipped (+1), as for q = 1/2; the tracked energy equals
    Eq. 2 recomputed.
"""
import math

import numpy as np
import pytest

import oracle.oracle as orc
from paper_1811_01604_gb300 import mpr, synth

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


def _circ(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


@pytest.mark.parametrize("q", [0.3, 0.2])
@pytest.mark.parametrize("or_mode", [mpr.MPR_OR_CONSERVING, mpr.MPR_OR_NONE])
def test_q_trajectory_f64_matches_oracle(q, or_mode):
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    H, W = z.shape
    gap = mask == 0
    seed, T = 13, 0.3 * (q / 0.5) ** 2
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=seed, q=q, or_mode=or_mode,
                                                             precision=mpr.MPR_PREC_F64))
    try:
        mpr.mpr_set_T(ctx, T)
        got = np.zeros((H, W), np.float64)
        sw0 = mpr.mpr_get_state64(ctx, got)
        phi, _, _, _ = orc.map_angles(z, mask)
        orc.init_gaps(phi, mask, seed)
        assert _circ(got, phi).max() < 1e-13
        for s in range(200):
            a = 1.0 + s / 3.0 if s < 30 else 1.0
            orc.sweep(phi, mask, a, T, q=q, seed=seed, sweep_index=sw0 + s, or_mode=or_mode)
            mpr.mpr_sweep(ctx, 1, a)
            if s % 20 == 19:
                mpr.mpr_get_state64(ctx, got)
                d = _circ(got[gap], phi[gap])
                assert d.max() < 1e-9, (s, float(d.max()), int((d > 1e-6).sum()))
        info = mpr.mpr_get_info(ctx)
    finally:
        mpr.mpr_free(ctx)
    # gap angles stay in [0, 2 pi): the arc of theta = q phi is never left (samples lie in
    # [0, 2 pi], the maximum mapping to 2 pi by Eq. 1)
    assert (got[gap] >= 0).all() and (got[gap] < TWO_PI).all()
    assert (got >= 0).all() and (got <= TWO_PI + 1e-12).all()
    e_orc = orc.energy(phi, q=q)
    assert abs(info["H_exact"] / e_orc - 1) < 1e-12
    assert abs(info["H_tracked"] / e_orc - 1) < 1e-11


@pytest.mark.parametrize("q", [0.3, 0.15])
def test_q_single_sweep_f32_parity_and_energy(q):
    z = synth.wm_field(96, 0.5, 6.0, seed=21, W=83)
    mask = synth.mask_uniform(96, 83, 0.5, seed=22)
    H, W = z.shape
    gap = mask == 0
    seed, T = 19, 0.2 * (q / 0.5) ** 2
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=seed, q=q))
    flips = n = 0
    worst = 0.0
    try:
        mpr.mpr_set_T(ctx, T)
        phi = np.zeros((H, W), np.float32)
        for it in range(60):
            a = (1.0, 3.0, 12.0)[it % 3]
            sw = mpr.mpr_get_state(ctx, phi)
            assert (phi >= 0).all() and (phi <= TWO_PI + 1e-5).all()
            ref = phi.astype(np.float64)
            orc.sweep(ref, mask, a=a, T=T, q=q, seed=seed, sweep_index=sw)
            mpr.mpr_sweep(ctx, 1, a)
            got = np.zeros_like(phi)
            mpr.mpr_get_state(ctx, got)
            d = _circ(got[gap], ref[gap])
            bad = d > 1e-5
            flips += int(bad.sum())
            n += int(gap.sum())
            if (~bad).any():
                worst = max(worst, float(d[~bad].max()))
        info = mpr.mpr_get_info(ctx)
    finally:
        mpr.mpr_free(ctx)
    assert flips <= 1e-6 * n + 1, (flips, n)
    assert worst < 1e-5
    assert abs(info["H_tracked"] / info["H_exact"] - 1) < 1e-6


def test_q_fill_f64_matches_oracle_end_to_end():
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    H, W = z.shape
    q, seed = 0.3, 8
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=seed, q=q, precision=mpr.MPR_PREC_F64))
    zhat = np.zeros((H, W), np.float32)
    try:
        st = mpr.mpr_fill(ctx, zhat)
        info = mpr.mpr_get_info(ctx)
        got = np.zeros((H, W), np.float64)
        mpr.mpr_get_state64(ctx, got)
    finally:
        mpr.mpr_free(ctx)
    ref_z, ref_phi, out = orc.fill(z, mask, orc.params(seed=seed, q=q, T_W=W, T_H=H))
    assert abs(info["e_s"] / out.e_s - 1) < 1e-12
    assert abs(info["T"] / out.T_hat - 1) < 1e-9
    assert st.sweeps == out.eq.sweeps and st.a == out.eq.a
    gap = mask == 0
    assert _circ(got[gap], ref_phi[gap]).max() < 1e-8
    tol = 2 * np.spacing(np.abs(ref_z).astype(np.float32)).astype(np.float64) + 1e-9 * (out.zmax - out.zmin)
    assert (np.abs(zhat.astype(np.float64) - ref_z) <= tol).all()


def test_q_fill_f32_runs_and_tile_path_refused():
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    H, W = z.shape
    with pytest.raises(mpr.MprError) as e:
        mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(q=0.3, exec_mode=mpr.MPR_EXEC_TILE))
    assert e.value.status == mpr.MPR_EINVAL
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=2, q=0.3))
    zhat = np.zeros((H, W), np.float32)
    try:
        mpr.mpr_fill(ctx, zhat)
        info = mpr.mpr_get_info(ctx)
    finally:
        mpr.mpr_free(ctx)
    assert abs(info["H_tracked"] / info["H_exact"] - 1) < 1e-6
    assert (zhat >= info["zmin"]).all() and (zhat <= info["zmax"]).all()
    assert (zhat[mask == 1] == z[mask == 1]).all()
