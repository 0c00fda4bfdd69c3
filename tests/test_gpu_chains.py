"""Independent-chain realizations (mpr_predict_chains) against the single chain and the
FP64 oracle's fork (reading R-CH: the equilibrated state forked into K chains with Philox
chain words chain + k 2^24, all from the same sweep counter, every realization averaged).

  * K = 1 without burn-in is exactly mpr_predict (bitwise), and the grid's own state is left
    unchanged;
  * one averaged sweep per chain (after 0 or 2 burn-in sweeps) from a state set on both
    sides: the mean angle of the K chains at every gap site within 1e-5 rad of the
    oracle's, except at most 1e-6 of the decisions (plus one per chain) whose accept /
    reflect / wrap outcome flipped in rounding, and their neighbours in later sweeps;
  * whole fills (relaxation, then K chains x M_per_chain sweeps) as estimators: MAE and
    RMSE averaged over independent seeds within 1 % of the oracle's.
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle.oracle as orc
from paper_1811_01604_gb300 import mpr, synth

pytestmark = pytest.mark.gpu
TWO_PI = 2 * math.pi


def _ctx(z, mask, **kw):
    H, W = z.shape
    return mpr.mpr_init(np.ascontiguousarray(z, np.float32), np.ascontiguousarray(mask, np.uint8), W, H,
                        mpr.mpr_default_params(**kw))


def test_one_chain_is_predict_and_state_is_kept():
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    H, W = z.shape
    ctx = _ctx(z, mask, seed=5)
    try:
        mpr.mpr_set_T(ctx, 0.2)
        mpr.mpr_sweep(ctx, 30, 2.0)
        phi0 = np.zeros((H, W), np.float32)
        sw0 = mpr.mpr_get_state(ctx, phi0)
        zc = np.zeros_like(z)
        mpr.mpr_predict_chains(ctx, 1, 12, zc)
        phi1 = np.zeros_like(phi0)
        assert mpr.mpr_get_state(ctx, phi1) == sw0 and np.array_equal(phi0, phi1)
        zp = np.zeros_like(z)
        mpr.mpr_predict(ctx, 12, zp)
    finally:
        mpr.mpr_free(ctx)
    assert np.array_equal(zc, zp)


@pytest.mark.parametrize("K,burn", [(2, 0), (5, 0), (3, 2)])
def test_chains_match_oracle_fork_from_same_state(K, burn):
    L = 128
    z = synth.wm_field(L, 1.0, 8.0, seed=61)
    mask = synth.mask_uniform(L, L, 0.4, seed=1_000_061)
    phi, zmin, zmax, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, seed=8)
    T, sw = 0.1, 40
    ctx = _ctx(z, mask, seed=8)
    try:
        mpr.mpr_set_T(ctx, T)
        mpr.mpr_set_state(ctx, phi.astype(np.float32), sw)
        st = np.zeros((L, L), np.float32)
        mpr.mpr_get_state(ctx, st)                       # the GPU's FP32 state, used by both
        zg = np.zeros_like(z)
        mpr.mpr_predict_chains(ctx, K, 1, zg, burn_in=burn)
    finally:
        mpr.mpr_free(ctx)
    prm = orc.params(seed=8)
    zo = orc.predict_chains(st.astype(np.float64), mask, z, T, prm, zmin, zmax, K=K, M_per_chain=1,
                            sweep_index=sw, burn_in=burn)
    g = mask == 0
    to_phi = TWO_PI / (zmax - zmin)
    d = np.abs(zg[g].astype(np.float64) - zo[g]) * to_phi
    d = np.minimum(d, TWO_PI / K - d) if K > 1 else np.minimum(d, TWO_PI - d)
    bad = int((d > 1e-5).sum())
    # a flipped decision in a burn-in sweep also moves its neighbours in the later sweeps
    assert bad <= (1e-6 * K * (1 + burn) * g.sum() + K) * (1 + 4 * burn), bad
    assert np.array_equal(zg[~g], z[~g])


def test_chain_fills_match_oracle_statistics():
    # 256^2, 33 % gaps, fixed T, 200 relaxation sweeps (slope test off), then 4 chains x 25
    L, K, m, T = 256, 4, 25, 0.12
    z = synth.wm_field(L, 0.5, 5.0, seed=41)
    mask = synth.mask_uniform(L, L, 0.33, seed=1_000_041)
    seeds = (3, 4, 5, 6, 7, 8)
    g = mask == 0

    def errors(zh):
        e = zh[g].astype(np.float64) - z[g]
        return np.abs(e).mean(), np.sqrt((e ** 2).mean())

    def oracle_run(seed):
        prm = orc.params(seed=seed, i_max=199, n_fit=10**6, M=m)
        phi, zmin, zmax, _ = orc.map_angles(z, mask)
        orc.init_gaps(phi, mask, seed=seed)
        out, sw, _ = orc.equilibrate(phi, mask, T, prm)
        assert out.sweeps == 200
        return errors(orc.predict_chains(phi, mask, z, T, prm, zmin, zmax, K=K, M_per_chain=m,
                                         sweep_index=sw))

    with ThreadPoolExecutor(max_workers=min(len(seeds), os.cpu_count() or 1)) as ex:
        oracle = list(ex.map(oracle_run, seeds))
    gpu = []
    for seed in seeds:
        ctx = _ctx(z, mask, seed=seed, i_max=199, n_fit=10**6, M=m)
        try:
            mpr.mpr_set_T(ctx, T)
            st = mpr.mpr_equilibrate(ctx)
            assert st.sweeps == 200
            zg = np.zeros_like(z)
            mpr.mpr_predict_chains(ctx, K, m, zg)
        finally:
            mpr.mpr_free(ctx)
        assert np.array_equal(zg[~g], z[~g])
        gpu.append(errors(zg))
    mae_o, rmse_o = np.mean(oracle, axis=0)
    mae_g, rmse_g = np.mean(gpu, axis=0)
    assert abs(mae_g / mae_o - 1) < 0.01, (mae_g, mae_o)
    assert abs(rmse_g / rmse_o - 1) < 0.01, (rmse_g, rmse_o)


def test_chain_arguments_are_checked():
    c = synth.config("grid64")
    ctx = _ctx(c["z"], c["mask"], seed=1)
    try:
        zh = np.zeros_like(c["z"])
        with pytest.raises(mpr.MprError):
            mpr.mpr_predict_chains(ctx, 2, 5, zh)            # temperature not set yet
        mpr.mpr_set_T(ctx, 0.2)
        for K, m in ((0, 5), (129, 5), (2, 0)):
            with pytest.raises(mpr.MprError) as e:
                mpr.mpr_predict_chains(ctx, K, m, zh)
            assert e.value.status == mpr.MPR_EINVAL
    finally:
        mpr.mpr_free(ctx)
