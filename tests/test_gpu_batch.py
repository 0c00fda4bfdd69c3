"""GPU tests of the batched form: many grids of their own sizes in one context."""
import numpy as np
import pytest

from paper_1811_01604_gb300 import mpr, synth

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64), (37, 101), (130, 90), (16, 300)]


def _grids():
    out = []
    for i, (H, W) in enumerate(SHAPES):
        z = synth.wm_field(H, 0.5 + i % 2, 6.0, seed=50 + i, W=W)
        m = synth.mask_uniform(H, W, 0.3 + 0.1 * i, seed=60 + i)
        out.append((z, m))
    return out


def _single(z, m, chain, T, sweeps, M, with_info=False, **kw):
    H, W = z.shape
    ctx = mpr.mpr_init(z, m, W, H, mpr.mpr_default_params(seed=5, chain=chain, **kw))
    try:
        info = mpr.mpr_batch_info(ctx, 0)
        mpr.mpr_set_T(ctx, T)
        mpr.mpr_sweep(ctx, sweeps, 3.0)
        zh = np.zeros_like(z)
        mpr.mpr_predict(ctx, M, zh)
        return (zh, info) if with_info else zh
    finally:
        mpr.mpr_free(ctx)


@pytest.mark.parametrize("exec_mode,prec", [(mpr.MPR_EXEC_TILE, mpr.MPR_PREC_F32), (mpr.MPR_EXEC_LIST, mpr.MPR_PREC_F32),
                                            (mpr.MPR_EXEC_LIST, mpr.MPR_PREC_F64)])
def test_batch_reproduces_separate_runs_bitwise(exec_mode, prec):
    # the batch's set-up runs each step once for all grids (Eq. 1 extremes, pack, gap
    # lists, Eq. 4 partials, Eq. 2 energies), a single grid's set-up one grid at a time:
    # the same e_s, extremes and estimates bit for bit, in FP32 and FP64 lattices
    g = _grids()
    T, sweeps, M = 0.09, 11, 7
    ctx = mpr.mpr_init_batch([z for z, _ in g], [m for _, m in g],
                             mpr.mpr_default_params(seed=5, chain=0, exec_mode=exec_mode, precision=prec))
    try:
        assert mpr.mpr_batch_size(ctx) == len(g)
        info = mpr.mpr_batch_info_all(ctx)
        mpr.mpr_set_T(ctx, T)
        mpr.mpr_sweep(ctx, sweeps, 3.0)
        outs = [np.zeros_like(z) for z, _ in g]
        mpr.mpr_predict_batch(ctx, M, outs)
    finally:
        mpr.mpr_free(ctx)
    for i, (z, m) in enumerate(g):
        ref, ref_info = _single(z, m, i, T, sweeps, M, with_info=True, exec_mode=exec_mode, precision=prec)
        assert np.array_equal(outs[i].view(np.uint32), ref.view(np.uint32)), i
        for k in ("e_s", "zmin", "zmax"):
            assert info[i][k] == ref_info[k], (i, k)


def test_batch_relaxation_stops_per_grid_like_separate_runs():
    g = _grids()
    ctx = mpr.mpr_init_batch([z for z, _ in g], [m for _, m in g], mpr.mpr_default_params(seed=8))
    try:
        mpr.mpr_set_T(ctx, 0.1)
        mpr.mpr_equilibrate(ctx)
        info = [mpr.mpr_batch_info(ctx, i) for i in range(len(g))]
    finally:
        mpr.mpr_free(ctx)
    for i, (z, m) in enumerate(g):
        H, W = z.shape
        c1 = mpr.mpr_init(z, m, W, H, mpr.mpr_default_params(seed=8, chain=i))
        try:
            mpr.mpr_set_T(c1, 0.1)
            st = mpr.mpr_equilibrate(c1)
        finally:
            mpr.mpr_free(c1)
        assert info[i]["sweeps"] == st.sweeps and info[i]["converged"] == st.converged


def test_autotune_leaves_the_chain_unchanged():
    g = _grids()
    res = []
    for tune in (False, True):
        ctx = mpr.mpr_init_batch([z for z, _ in g], [m for _, m in g], mpr.mpr_default_params(seed=3))
        try:
            mpr.mpr_set_T(ctx, 0.1)
            if tune:
                t = mpr.mpr_autotune(ctx)
                assert 0 <= t["tile_cfg"] < 3 and 4 <= t["graph_sweeps"] <= 64 and t["ms_per_sweep"] > 0
            mpr.mpr_sweep(ctx, 5, 2.0)
            outs = [np.zeros_like(z) for z, _ in g]
            mpr.mpr_predict_batch(ctx, 4, outs)
            res.append(outs)
        finally:
            mpr.mpr_free(ctx)
    for a, b in zip(*res):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_every_tile_configuration_gives_the_same_lattice(cfg):
    z, m = _grids()[2]
    ref = _single(z, m, 0, 0.1, 6, 3, tile_cfg=0)
    got = _single(z, m, 0, 0.1, 6, 3, tile_cfg=cfg)
    assert np.array_equal(ref.view(np.uint32), got.view(np.uint32))


def test_batch_fill_quality_and_per_grid_temperatures():
    shapes = [(96, 96), (128, 160), (200, 200)]
    zs, ms = [], []
    for i, (H, W) in enumerate(shapes):
        zs.append(synth.wm_field(H, 0.5, 5.0, seed=70 + i, W=W))
        ms.append(synth.mask_uniform(H, W, 0.33, seed=80 + i))
    ctx = mpr.mpr_init_batch(zs, ms, mpr.mpr_default_params(seed=11, M=50))
    try:
        outs = [np.zeros_like(z) for z in zs]
        mpr.mpr_fill_batch(ctx, outs)
        info = [mpr.mpr_batch_info(ctx, i) for i in range(len(zs))]
        assert mpr.mpr_batch_info_all(ctx) == info          # one read of every grid's state
    finally:
        mpr.mpr_free(ctx)
    for z, m, o, inf in zip(zs, ms, outs, info):
        gap = m == 0
        assert np.array_equal(o[~gap], z[~gap])
        mae = np.abs(o[gap].astype(np.float64) - z[gap]).mean()
        assert 2.5 < mae < 4.5                    # the paper's data model: MAAE about 3.4 at 33 %
        assert 0.02 < inf["T"] < 0.5 and inf["sweeps"] >= 1
