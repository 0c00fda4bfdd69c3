"""Precision study: FP32 sweep kernels with accurate vs fast transcendentals against the
FP64 oracle, on a 512 x 512 crop of the 4096^2 workload (nu = 1, correlation length 32,
half of the sites missing as disks plus random sites).

Run with -s to print the table; the bounds asserted here are the ones the design notes
derive (|d phi| <= 1e-5 rad where decisions agree; flipped decisions <= 1e-6 of all in the
accurate mode; MAE/RMSE within 1 % of the oracle's for both modes).

Whole runs of the two sides diverge after the first flipped decision, so they are compared
as estimators: one run's MAE on this crop moves by about +-1 % from seed to seed (on both
sides), so the 1 % bound applies to the mean over SEEDS independent chains of each side.
"""
import json
import math
import os
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle.oracle as orc
from paper_1811_01604_gb300 import mpr

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TWO_PI = 2 * math.pi


@pytest.fixture(scope="module")
def crop():
    sys.path.insert(0, ROOT)
    import bench
    z, m = bench.make_inputs(0)
    return np.ascontiguousarray(z[:512, :512]), np.ascontiguousarray(m[:512, :512])


def _circ(a, b):
    d = np.abs(a.astype(np.float64) - b.astype(np.float64)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


def _single_sweeps(z, m, T, trig, sweeps=24):
    H, W = z.shape
    ctx = mpr.mpr_init(z, m, W, H, mpr.mpr_default_params(seed=2, trig_mode=trig))
    gap = m == 0
    flips = n = 0
    errs = []
    try:
        mpr.mpr_set_T(ctx, T)
        phi = np.zeros((H, W), np.float32)
        for it in range(sweeps):
            a = (1.0, 4.0, 16.0, 64.0)[it % 4]
            sw = mpr.mpr_get_state(ctx, phi)
            ref = phi.astype(np.float64)
            orc.sweep(ref, m, a=a, T=T, seed=2, chain=0, sweep_index=sw)
            mpr.mpr_sweep(ctx, 1, a)
            got = np.zeros_like(phi)
            mpr.mpr_get_state(ctx, got)
            d = _circ(got[gap], ref[gap])
            bad = d > 1e-5
            flips += int(bad.sum())
            n += int(gap.sum())
            errs.append(d[~bad])
    finally:
        mpr.mpr_free(ctx)
    e = np.concatenate(errs)
    return dict(flips=flips, decisions=n, max_err=float(e.max()), mean_err=float(e.mean()),
                p99_err=float(np.quantile(e, 0.99)))


SEEDS = (6, 7, 8, 9, 10, 11, 12, 13)


def _errors(zh, z, m):
    g = m == 0
    err = zh[g].astype(np.float64) - z[g]
    return float(np.abs(err).mean()), float(np.sqrt((err ** 2).mean()))


def _oracle_runs(z, m, T):
    """(MAE, RMSE) of the oracle's fill per seed; the C oracle runs outside the GIL, so
    the seeds run on parallel threads."""
    def one(seed):
        prm = orc.params(seed=seed, i_max=199, n_fit=10**6, M=100)
        zo, _, _ = orc.fill(z, m, prm, T_fixed=T)
        return _errors(zo, z, m)
    with ThreadPoolExecutor(max_workers=min(len(SEEDS), os.cpu_count() or 1)) as ex:
        return list(ex.map(one, SEEDS))


def _run(z, m, T, trig, seed):
    H, W = z.shape
    ctx = mpr.mpr_init(z, m, W, H, mpr.mpr_default_params(seed=seed, trig_mode=trig, i_max=199,
                                                          n_fit=10**6, M=100))
    try:
        mpr.mpr_set_T(ctx, T)
        mpr.mpr_equilibrate(ctx)
        zh = np.zeros_like(z)
        mpr.mpr_predict(ctx, 100, zh)
        info = mpr.mpr_get_info(ctx)
    finally:
        mpr.mpr_free(ctx)
    mae, rmse = _errors(zh, z, m)
    return dict(mae=mae, rmse=rmse, energy_drift=abs(info["H_tracked"] / info["H_exact"] - 1))


def test_precision_accurate_vs_fast_against_oracle(crop):
    z, m = crop
    H, W = z.shape
    ctx = mpr.mpr_init(z, m, W, H, mpr.mpr_default_params(seed=2, T_cap=256))
    try:
        T, _ = mpr.mpr_estimate_T(ctx)
    finally:
        mpr.mpr_free(ctx)
    oracle_runs = np.array(_oracle_runs(z, m, T))
    ref = dict(mae=float(oracle_runs[:, 0].mean()), rmse=float(oracle_runs[:, 1].mean()),
               mae_per_seed=oracle_runs[:, 0].tolist())
    report = {"T_hat": T, "seeds": list(SEEDS), "oracle": ref}
    for name, trig in (("accurate", mpr.MPR_TRIG_ACCURATE), ("fast", mpr.MPR_TRIG_FAST)):
        one = _single_sweeps(z, m, T, trig)
        runs = [_run(z, m, T, trig, s) for s in SEEDS]
        run = dict(mae=float(np.mean([r["mae"] for r in runs])),
                   rmse=float(np.mean([r["rmse"] for r in runs])),
                   mae_per_seed=[r["mae"] for r in runs],
                   energy_drift=max(r["energy_drift"] for r in runs))
        run["mae_rel_to_oracle"] = run["mae"] / ref["mae"] - 1
        run["rmse_rel_to_oracle"] = run["rmse"] / ref["rmse"] - 1
        report[name] = dict(single_sweep=one, run=run)
        assert one["max_err"] <= 1e-5
        assert abs(run["mae_rel_to_oracle"]) < 0.01 and abs(run["rmse_rel_to_oracle"]) < 0.01, run
        assert run["energy_drift"] < 1e-6
    acc = report["accurate"]["single_sweep"]
    assert acc["flips"] <= 1e-6 * acc["decisions"] + 1
    print("PRECISION_REPORT " + json.dumps(report))
