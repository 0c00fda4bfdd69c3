"""The 1024 x 1024 workloads against the FP64 oracle, and the e(T, L) table's lattice cap.

* 1024^2 grids (Whittle-Matern nu = 0.5 and 2.5, correlation length 16, Gaussian and
  lognormal, 33 % and 66 % of the sites removed at random), each at its T-hat, with a
  fixed run: 100 relaxation sweeps of Algorithm 2 step 5 (slope test disabled) and M = 100
  averaged sweeps.  Whole runs of the two sides diverge after the first flipped decision,
  so the fills are compared as estimators: MAE and RMSE against the hidden field, averaged
  over independent chains of each side, within 1 % of the oracle's.  The C oracle runs
  outside the GIL, all chains of all grids on parallel threads.
* Eq. 5 defines e(T, L) on the grid's own lattice; the library builds it on a lattice whose
  sides are capped (T_cap = 1024 by default).  On a 2048^2 grid the T-hat of the capped
  table must lie within 0.5 % of the T-hat of the full-size table (finite-size corrections
  of e(T, L) are of order 1 / L; measured difference 0.11 %).
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle.oracle as orc
from paper_1811_01604_gb300 import mpr, synth

pytestmark = pytest.mark.gpu

L = 1024
RELAX, M = 100, 100
SEEDS = (11, 12, 13)
VARIANTS = [(nu, kind, p) for nu in (0.5, 2.5) for kind in ("gauss", "lognormal") for p in (0.33, 0.66)]


def _grid(nu, kind, p):
    seed = 1 if nu == 0.5 else 2
    z = synth.wm_field(L, nu, 16.0, seed=seed)
    if kind == "lognormal":
        z = synth.lognormal(z).astype(np.float32)
    mask = synth.mask_uniform(L, L, p, seed=1_000_000 + seed + int(100 * p))
    return np.ascontiguousarray(z, np.float32), np.ascontiguousarray(mask, np.uint8)


def _errors(zh, z, gap):
    e = zh[gap].astype(np.float64) - z[gap]
    return np.abs(e).mean(), np.sqrt((e ** 2).mean())


@pytest.fixture(scope="module")
def runs():
    grids = {v: _grid(*v) for v in VARIANTS}
    T = {}
    for v, (z, mask) in grids.items():
        ctx = mpr.mpr_init(z, mask, L, L, mpr.mpr_default_params(seed=1))
        try:
            T[v] = mpr.mpr_estimate_T(ctx)[0]
        finally:
            mpr.mpr_free(ctx)

    def oracle_run(job):
        v, seed = job
        z, mask = grids[v]
        prm = orc.params(seed=seed, i_max=RELAX - 1, n_fit=10**6, M=M)
        zo, _, fo = orc.fill(z, mask, prm, T_fixed=T[v])
        assert fo.eq.sweeps == RELAX
        return _errors(zo, z, mask == 0)

    jobs = [(v, s) for v in VARIANTS for s in SEEDS]
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        oracle = dict(zip(jobs, ex.map(oracle_run, jobs)))
    gpu = {}
    for v, s in jobs:
        z, mask = grids[v]
        ctx = mpr.mpr_init(z, mask, L, L, mpr.mpr_default_params(seed=s, i_max=RELAX - 1, n_fit=10**6, M=M))
        try:
            mpr.mpr_set_T(ctx, T[v])
            st = mpr.mpr_equilibrate(ctx)
            assert st.sweeps == RELAX
            zg = np.zeros_like(z)
            mpr.mpr_predict(ctx, M, zg)
        finally:
            mpr.mpr_free(ctx)
        gap = mask == 0
        assert np.array_equal(zg[~gap], z[~gap])
        gpu[(v, s)] = _errors(zg, z, gap)
    return oracle, gpu


@pytest.mark.parametrize("nu,kind,p", VARIANTS)
def test_1024_fill_matches_oracle_statistics(runs, nu, kind, p):
    oracle, gpu = runs
    v = (nu, kind, p)
    mae_o, rmse_o = np.mean([oracle[(v, s)] for s in SEEDS], axis=0)
    mae_g, rmse_g = np.mean([gpu[(v, s)] for s in SEEDS], axis=0)
    assert abs(mae_g / mae_o - 1) < 0.01, (mae_g, mae_o)
    assert abs(rmse_g / rmse_o - 1) < 0.01, (rmse_g, rmse_o)


def test_capped_table_temperature_matches_full_size_table():
    z = synth.wm_field_gpu(2048, 2048, 1.0, 32.0, 5)
    mask = synth.mask_uniform_gpu(2048, 2048, 0.5, 1_000_005)
    T = {}
    for cap in (1024, 0):                       # 0: the table on the grid's own 2048^2 lattice
        ctx = mpr.mpr_init(z, mask, 2048, 2048, mpr.mpr_default_params(seed=1, T_cap=cap))
        try:
            T[cap] = mpr.mpr_estimate_T(ctx)[0]
        finally:
            mpr.mpr_free(ctx)
    assert abs(T[1024] / T[0] - 1) < 0.005, T
