"""The FP64 path (MPR_PREC_F64) against the FP64 oracle, trajectory by trajectory.

With every step of Algorithm 1 in double on both sides, the GPU (unit vectors, CUDA's
double sin/cos/exp) and the oracle (angles, libm) differ by rounding alone, ~1e-15 rad
per update.  Under the energy-conserving reflection and without over-relaxation such
differences do not grow: two oracle runs whose start differs by 1e-15 rad stay within
1e-13 rad over 300 sweeps at T = 0.05 to 1 on the 64 x 64 grid (2e-11 on an all-free
lattice at T = 1).  So no Metropolis decision flips and the chains coincide: the whole
fill -- Eq. 4, the e(T, L) table, T-hat, the relaxation with its window and slope test,
the M averaged sweeps -- must agree to rounding.  The printed reflection (Eq. 6 as
printed, q = 1) amplifies rounding (the same 1e-15 start separates completely within 50
sweeps on an all-free lattice at T = 0.3, and with the 64 x 64 grid's samples grows to
1e-7 rad in 300 sweeps at T = 0.3, completely at T = 1), so its trajectory is compared
over a short run at low T only.
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


def _gpu_state(ctx, H, W):
    phi = np.zeros((H, W), np.float64)
    sw = mpr.mpr_get_state64(ctx, phi)
    return phi, sw


@pytest.mark.parametrize("or_mode,T,n_sweeps,tol", [
    (mpr.MPR_OR_CONSERVING, 0.3, 200, 1e-9),
    (mpr.MPR_OR_NONE, 0.3, 200, 1e-9),
    (mpr.MPR_OR_LITERAL, 0.05, 40, 1e-8),
])
def test_f64_trajectory_matches_oracle(or_mode, T, n_sweeps, tol):
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    H, W = z.shape
    gap = mask == 0
    seed = 11
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=seed, or_mode=or_mode,
                                                             precision=mpr.MPR_PREC_F64))
    try:
        mpr.mpr_set_T(ctx, T)
        ref, sw0 = _gpu_state(ctx, H, W)
        # the oracle starts from its own map and initial draw (Algorithm 2 steps 2.2, 3)
        phi, zmin, zmax, _ = orc.map_angles(z, mask)
        orc.init_gaps(phi, mask, seed)
        assert _circ(ref, phi).max() < 1e-14
        worst = 0.0
        for s in range(n_sweeps):
            a = 1.0 + s / 3.0 if s < 30 else 1.0
            orc.sweep(phi, mask, a, T, seed=seed, sweep_index=sw0 + s, or_mode=or_mode)
            mpr.mpr_sweep(ctx, 1, a)
            if s % 10 == 9 or s == n_sweeps - 1:
                got, sw = _gpu_state(ctx, H, W)
                assert sw == sw0 + s + 1
                d = _circ(got[gap], phi[gap])
                worst = max(worst, float(d.max()))
                assert d.max() < tol, (s, float(d.max()), int((d > 1e-6).sum()))
        info = mpr.mpr_get_info(ctx)
    finally:
        mpr.mpr_free(ctx)
    e_orc = orc.energy(phi)
    assert abs(info["H_exact"] / e_orc - 1) < 1e-12
    assert abs(info["H_tracked"] / e_orc - 1) < 1e-11
    print(f"or_mode {or_mode}: max |d phi| over {n_sweeps} sweeps {worst:.2e} rad")


@pytest.mark.parametrize("case", ["grid64", "ragged"])
def test_f64_fill_matches_oracle_end_to_end(case):
    if case == "grid64":
        c = synth.config("grid64")
        z, mask = c["z"], c["mask"]
    else:
        z = synth.wm_field(150, 1.5, 8.0, seed=41, W=97)
        mask = synth.mask_disks(150, 97, 0.5, seed=42)
    H, W = z.shape
    seed = 5
    prm = mpr.mpr_default_params(seed=seed, precision=mpr.MPR_PREC_F64)
    ctx = mpr.mpr_init(z, mask, W, H, prm)
    zhat = np.zeros((H, W), np.float32)
    try:
        st = mpr.mpr_fill(ctx, zhat)
        info = mpr.mpr_get_info(ctx)
        got, _ = _gpu_state(ctx, H, W)
    finally:
        mpr.mpr_free(ctx)
    ref_z, ref_phi, out = orc.fill(z, mask, orc.params(seed=seed, T_W=W, T_H=H))
    assert abs(info["e_s"] / out.e_s - 1) < 1e-12                       # Eq. 4
    assert abs(info["T"] / out.T_hat - 1) < 1e-9                        # table + Eq. 5 inversion
    assert st.sweeps == out.eq.sweeps and st.a == out.eq.a              # same relaxation
    assert abs(st.e_last - out.eq.e_last) < 1e-10
    gap = mask == 0
    assert _circ(got[gap], ref_phi[gap]).max() < 1e-8                   # same final state
    # zhat leaves as float: within two float32 spacings of the oracle's double value
    tol = 2 * np.spacing(np.abs(ref_z).astype(np.float32)).astype(np.float64) + 1e-9 * (out.zmax - out.zmin)
    assert (np.abs(zhat.astype(np.float64) - ref_z) <= tol).all()
    assert (zhat[mask == 1] == z[mask == 1]).all()
    print(f"{case}: T-hat {info['T']:.6g}, {st.sweeps} relaxation sweeps, "
          f"max |d zhat| {np.abs(zhat - ref_z).max():.2e}")


def test_f64_refuses_tile_and_fast_modes_and_chains():
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    H, W = z.shape
    for bad in (dict(exec_mode=mpr.MPR_EXEC_TILE), dict(trig_mode=mpr.MPR_TRIG_FAST)):
        with pytest.raises(mpr.MprError) as e:
            mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(precision=mpr.MPR_PREC_F64, **bad))
        assert e.value.status == mpr.MPR_EINVAL
    with pytest.raises(mpr.MprError) as e:
        mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(precision=7))
    assert e.value.status == mpr.MPR_EINVAL
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(precision=mpr.MPR_PREC_F64))
    try:
        mpr.mpr_set_T(ctx, 0.2)
        out = np.zeros((H, W), np.float32)
        with pytest.raises(mpr.MprError) as e:
            mpr.mpr_predict_chains(ctx, 2, 5, out)
        assert e.value.status == mpr.MPR_EINVAL
    finally:
        mpr.mpr_free(ctx)


def test_f64_state_roundtrip_and_f32_widening():
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    H, W = z.shape
    rng = np.random.default_rng(3)
    phi = rng.uniform(0, TWO_PI, (H, W)).astype(np.float32)
    for prec in (mpr.MPR_PREC_F64, mpr.MPR_PREC_F32):
        ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(precision=prec))
        try:
            mpr.mpr_set_state(ctx, phi, 9)
            got64, sw = _gpu_state(ctx, H, W)
            got32 = np.zeros((H, W), np.float32)
            mpr.mpr_get_state(ctx, got32)
        finally:
            mpr.mpr_free(ctx)
        gap = mask == 0
        assert sw == 9
        d = _circ(got64[gap], phi[gap].astype(np.float64)).max()
        # FP64: sincos and atan2 in double; FP32: the float vector's own rounding (~1e-7)
        assert d < (1e-14 if prec == mpr.MPR_PREC_F64 else 1e-6)
        assert _circ(got32[gap], got64[gap]).max() < 1e-6
