"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (written here, derived in the design notes):
  * Philox: bitwise.
  * Eq. 1 angles: FP32 rounding of an FP64 value, |d phi| <= 1e-6 rad.
  * Eq. 4 / Eq. 2 energies: relative 1e-6 (FP32 cosines summed in FP64).
  * one sweep from an identical state: |d phi| <= 1e-5 rad (circular) at every site
    whose decisions agree; sites beyond that are counted as flipped decisions and must be
    at most 1e-6 of all decisions (plus one, for sample sizes below 10^6).
  * whole runs (chains diverge after the first flip): MAE and RMSE, averaged over
    independent chains of each side, within 1% relative of the oracle's at 256^2, and
    within 6% of the paper's Table 2-3 values at L = 1024.
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


def circ(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


def make_ctx(z, mask, **kw):
    H, W = z.shape
    p = mpr.mpr_default_params(**kw)
    return mpr.mpr_init(np.ascontiguousarray(z, np.float32), np.ascontiguousarray(mask, np.uint8),
                        W, H, p)


def test_philox_bitwise_against_oracle():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(100_000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:10] = 0
    ctr[10:20] = 0xFFFFFFFF
    for seed in (0, 0x0123456789ABCDEF, 2**64 - 1):
        out = np.zeros_like(ctr)
        mpr.mpr_philox(ctr, seed, out)
        assert np.array_equal(out, orc.philox_batch(ctr, seed))


@pytest.mark.parametrize("name", ["grid64", "odd"])
def test_map_sample_energy_and_energy(name):
    if name == "grid64":
        c = synth.config("grid64"); z, mask = c["z"], c["mask"]
    else:                                             # ragged odd sizes, two tiles plus a tail
        z = synth.wm_field(37, 0.5, 3.0, seed=5, W=601)
        mask = synth.mask_uniform(37, 601, 0.4, seed=6)
    ctx = make_ctx(z, mask)
    try:
        info = mpr.mpr_get_info(ctx)
        phi_o, zmin, zmax, _ = orc.map_angles(z, mask)
        assert info["zmin"] == zmin and info["zmax"] == zmax
        e_s, _ = orc.sample_energy(phi_o, mask)
        assert abs(info["e_s"] / e_s - 1) < 1e-6
        phi = np.zeros(z.shape, np.float32)
        assert mpr.mpr_get_state(ctx, phi) == 0
        s = mask == 1
        assert circ(phi[s], phi_o[s]).max() <= 1e-6
        assert np.all((phi >= 0) & (phi <= TWO_PI + 1e-6))
        H_ref = orc.energy(phi.astype(np.float64))
        assert abs(info["H_exact"] / H_ref - 1) < 1e-6
    finally:
        mpr.mpr_free(ctx)


EXEC = [mpr.MPR_EXEC_TILE, mpr.MPR_EXEC_LIST]


def _sweep_parity(z, mask, T, a_list, sweeps, trig=mpr.MPR_TRIG_ACCURATE, seed=11,
                  exec_mode=mpr.MPR_EXEC_TILE):
    ctx = make_ctx(z, mask, seed=seed, trig_mode=trig, exec_mode=exec_mode)
    flips = decisions = 0
    worst = 0.0
    try:
        mpr.mpr_set_T(ctx, T)
        phi = np.zeros(z.shape, np.float32)
        gap = mask == 0
        for it in range(sweeps):
            a = a_list[it % len(a_list)]
            sw = mpr.mpr_get_state(ctx, phi)
            ref = phi.astype(np.float64)
            orc.sweep(ref, mask, a=a, T=T, seed=seed, chain=0, sweep_index=sw)
            mpr.mpr_sweep(ctx, 1, a)
            got = np.zeros_like(phi)
            assert mpr.mpr_get_state(ctx, got) == sw + 1
            d = circ(got[gap], ref[gap])
            bad = d > 1e-5
            flips += int(bad.sum())
            decisions += int(gap.sum())
            if (~bad).any():
                worst = max(worst, float(d[~bad].max()))
            assert np.array_equal(got[~gap], phi[~gap])      # samples frozen, bitwise
    finally:
        mpr.mpr_free(ctx)
    return flips, decisions, worst


@pytest.mark.parametrize("exec_mode", EXEC)
def test_single_sweep_parity_grid64(exec_mode):
    c = synth.config("grid64")
    flips, n, worst = _sweep_parity(c["z"], c["mask"], T=0.12, a_list=[1.0, 2.5, 6.0, 20.0],
                                    sweeps=120, exec_mode=exec_mode)
    assert worst <= 1e-5
    assert flips <= 1e-6 * n + 1, (flips, n)


@pytest.mark.parametrize("exec_mode", EXEC)
def test_single_sweep_parity_256_ragged_gaps(exec_mode):
    z = synth.wm_field(256, 0.5, 5.0, seed=21, W=250)
    mask = synth.mask_uniform(256, 250, 0.5, seed=22)
    flips, n, worst = _sweep_parity(z, mask, T=0.1, a_list=[1.0, 4.0, 9.0], sweeps=40,
                                    exec_mode=exec_mode)
    assert n > 1_000_000
    assert worst <= 1e-5
    assert flips <= 1e-6 * n + 1, (flips, n)


@pytest.mark.parametrize("cfg", [0, 1, 2])
@pytest.mark.parametrize("shape", [(64, 64), (37, 601), (200, 130), (1, 9), (3, 1), (2, 3), (5, 2),
                                   (6, 7), (33, 127), (17, 262)])
def test_tile_and_list_paths_are_bitwise_identical(shape, cfg):
    # same arithmetic and the same Philox counters: the fused tile sweep (with its
    # duplicated ring updates and its pairs of sites sharing a Philox block, also where a
    # row ends inside a quad of columns) must reproduce the two half-sweep launches bit for
    # bit, in every tile shape
    H, W = shape
    z = synth.wm_field(H, 0.5, 4.0, seed=13, W=W) if H > 1 and W > 1 else \
        np.arange(H * W, dtype=np.float32).reshape(H, W)
    mask = synth.mask_uniform(H, W, 0.45, seed=14)
    mask.flat[0] = 1; mask.flat[-1] = 1
    states = []
    for mode in (mpr.MPR_EXEC_LIST, mpr.MPR_EXEC_TILE):
        ctx = make_ctx(z, mask, seed=17, exec_mode=mode, tile_cfg=cfg)
        try:
            mpr.mpr_set_T(ctx, 0.08)
            for a in (1.0, 3.0, 7.5, 1.0, 12.0):
                mpr.mpr_sweep(ctx, 3, a)
            mpr.mpr_sweep(ctx, 9, 2.0)                  # one graph of 8 plus one direct sweep
            phi = np.zeros((H, W), np.float32)
            sw = mpr.mpr_get_state(ctx, phi)
            states.append((phi, sw, mpr.mpr_get_info(ctx)))
        finally:
            mpr.mpr_free(ctx)
    (p0, s0, i0), (p1, s1, i1) = states
    assert s0 == s1 == 24
    assert np.array_equal(p0.view(np.uint32), p1.view(np.uint32))
    assert i0["H_exact"] == i1["H_exact"]
    assert i0["H_tracked"] == i1["H_tracked"]            # exact integer totals of both paths


@pytest.mark.parametrize("shape", [(2, 3), (5, 2), (6, 7), (9, 13), (33, 127)])
def test_small_and_ragged_grids_sweep_like_the_oracle(shape):
    # the quad counters at the right edge of rows whose width is not a multiple of 4, and
    # grids narrower than a quad, against the FP64 oracle sweep by sweep
    H, W = shape
    z = synth.wm_field(H, 0.5, 3.0, seed=23, W=W)
    mask = synth.mask_uniform(H, W, 0.5, seed=24)
    mask.flat[0] = 1; mask.flat[-1] = 1
    flips, n, worst = _sweep_parity(z, mask, T=0.2, a_list=[1.0, 3.0, 8.0], sweeps=30)
    assert n > 0
    assert worst <= 1e-5
    assert flips <= 1e-6 * n + 1, (flips, n)


def test_tracked_energy_matches_exact_energy():
    c = synth.config("grid64")
    ctx = make_ctx(c["z"], c["mask"])
    try:
        mpr.mpr_set_T(ctx, 0.1)
        st = mpr.mpr_sweep(ctx, 300, 5.0)
        info = mpr.mpr_get_info(ctx)
        assert abs(info["H_tracked"] / info["H_exact"] - 1) < 1e-6
        assert abs(st.e - info["H_exact"] / orc.n_gp(64, 64)) < 1e-6
    finally:
        mpr.mpr_free(ctx)


def test_fixed_length_run_matches_oracle_statistics():
    # 256^2, 33% gaps, fixed T, 200 relaxation sweeps (slope test disabled) then M = 100.
    # Whole runs of the two sides diverge after the first flipped decision, so the fills
    # are compared as estimators: MAE/RMSE averaged over independent chains (seeds) of
    # each side within 1 %.  The C oracle runs outside the GIL, on parallel threads.
    L = 256
    z = synth.wm_field(L, 0.5, 5.0, seed=41)
    mask = synth.mask_uniform(L, L, 0.33, seed=1_000_041)
    T = 0.12
    seeds = (3, 4, 5, 6, 7, 8)
    g = mask == 0

    def errors(zh):
        e = zh[g].astype(np.float64) - z[g]
        return np.abs(e).mean(), np.sqrt((e ** 2).mean())

    def oracle_run(seed):
        prm = orc.params(seed=seed, i_max=199, n_fit=10**6, M=100)
        zo, _, fo = orc.fill(z, mask, prm, T_fixed=T)
        return errors(zo), fo.eq.sweeps, fo.eq.a

    with ThreadPoolExecutor(max_workers=min(len(seeds), os.cpu_count() or 1)) as ex:
        oracle = list(ex.map(oracle_run, seeds))
    gpu = []
    for seed, (_, o_sweeps, o_a) in zip(seeds, oracle):
        ctx = make_ctx(z, mask, seed=seed, i_max=199, n_fit=10**6, M=100)
        try:
            mpr.mpr_set_T(ctx, T)
            st = mpr.mpr_equilibrate(ctx)
            assert st.sweeps == 200 and o_sweeps == 200
            assert st.a >= 1.0 and abs(st.a / o_a - 1) < 0.5
            zg = np.zeros_like(z)
            mpr.mpr_predict(ctx, 100, zg)
        finally:
            mpr.mpr_free(ctx)
        assert np.array_equal(zg[~g], z[~g])
        gpu.append(errors(zg))
    mae_o, rmse_o = np.mean([o[0] for o in oracle], axis=0)
    mae_g, rmse_g = np.mean(gpu, axis=0)
    assert abs(mae_g / mae_o - 1) < 0.01, (mae_g, mae_o)
    assert abs(rmse_g / rmse_o - 1) < 0.01, (rmse_g, rmse_o)


def test_temperature_estimate_matches_oracle():
    c = synth.config("grid64")
    kw = dict(KT=8, T_min=1e-3, T_max=2.0, M_T=60, i_max=1500, seed=5)
    ctx = make_ctx(c["z"], c["mask"], T_cap=32, **kw)
    try:
        T_g, e_s_g = mpr.mpr_estimate_T(ctx)
    finally:
        mpr.mpr_free(ctx)
    prm = orc.params(T_W=32, T_H=32, **kw)
    Tk, ek, _ = orc.e_table(prm)
    phi, _, _, _ = orc.map_angles(c["z"], c["mask"])
    e_s, _ = orc.sample_energy(phi, c["mask"])
    T_o = orc.invert_T(Tk, ek, e_s)
    assert abs(e_s_g / e_s - 1) < 1e-6
    assert abs(T_g / T_o - 1) < 0.05, (T_g, T_o)


@pytest.mark.parametrize("p", [0.33, 0.66])
def test_paper_table_2_3_at_L1024(p):
    # Whole method on the paper's setting (nu = 0.5, kappa = 0.2, L = 1024): MAAE and MRASE
    # of Tables 2-3 (3.38/4.24 at 33%, 3.83/4.82 at 66%) within 6%.
    paper = {0.33: (3.380, 4.244), 0.66: (3.827, 4.821)}[p]
    z = synth.wm_field(1024, 0.5, 5.0, seed=7)
    mask = synth.mask_uniform(1024, 1024, p, seed=1_000_007)
    ctx = make_ctx(z, mask, seed=7)
    try:
        zh = np.zeros_like(z)
        st = mpr.mpr_fill(ctx, zh)
        info = mpr.mpr_get_info(ctx)
    finally:
        mpr.mpr_free(ctx)
    g = mask == 0
    err = zh[g].astype(np.float64) - z[g]
    assert abs(np.abs(err).mean() / paper[0] - 1) < 0.06
    assert abs(np.sqrt((err ** 2).mean()) / paper[1] - 1) < 0.06
    assert 0.01 < info["T"] < 0.5 and st.sweeps >= 1
    assert zh[g].min() >= info["zmin"] and zh[g].max() <= info["zmax"]


def test_degenerate_inputs():
    z = np.full((8, 8), 3.0, np.float32)
    with pytest.raises(mpr.MprError) as e:
        make_ctx(z, np.ones((8, 8), np.uint8))
    assert e.value.status == mpr.MPR_ENODATA
    z = synth.wm_field(8, 0.5, 2.0, seed=1)
    cb = (np.indices((8, 8)).sum(0) % 2).astype(np.uint8)
    ctx = make_ctx(z, cb)
    try:
        with pytest.raises(mpr.MprError) as e:
            mpr.mpr_estimate_T(ctx)
        assert e.value.status == mpr.MPR_ENOPAIRS
    finally:
        mpr.mpr_free(ctx)
    # no gaps at all: the fill returns the data
    ctx = make_ctx(z, np.ones((8, 8), np.uint8))
    try:
        mpr.mpr_set_T(ctx, 0.1)
        zh = np.zeros_like(z)
        mpr.mpr_fill(ctx, zh)
        assert np.array_equal(zh, z)
    finally:
        mpr.mpr_free(ctx)
    # tiny and one-row grids
    for H, W in [(1, 2), (1, 9), (2, 2), (3, 1), (5, 3)]:
        zz = np.arange(H * W, dtype=np.float32).reshape(H, W)
        m = np.zeros((H, W), np.uint8); m.flat[0] = 1; m.flat[-1] = 1
        ctx = make_ctx(zz, m)
        try:
            mpr.mpr_set_T(ctx, 0.2)
            zh = np.zeros_like(zz)
            mpr.mpr_fill(ctx, zh)
            assert np.all(np.isfinite(zh)) and zh.min() >= 0 and zh.max() <= H * W - 1
            assert zh.flat[0] == 0 and zh.flat[-1] == H * W - 1
        finally:
            mpr.mpr_free(ctx)


def test_tile_path_fill_matches_list_path_fill():
    c = synth.config("grid64")
    out = []
    for mode in (mpr.MPR_EXEC_LIST, mpr.MPR_EXEC_TILE):
        ctx = make_ctx(c["z"], c["mask"], seed=9, KT=6, T_cap=32, M_T=30, M=20, exec_mode=mode)
        try:
            zh = np.zeros_like(c["z"])
            st = mpr.mpr_fill(ctx, zh)
            out.append((zh, st.sweeps, mpr.mpr_get_info(ctx)["T"]))
        finally:
            mpr.mpr_free(ctx)
    (z0, n0, T0), (z1, n1, T1) = out
    assert T0 == T1 and n0 == n1
    assert np.abs(z0.astype(np.float64) - z1).max() < 1e-3     # same chain; sums differ in order


def test_runs_are_bitwise_reproducible():
    c = synth.config("grid64")
    outs = []
    for _ in range(2):
        ctx = make_ctx(c["z"], c["mask"], seed=9, KT=6, T_cap=32, M_T=30, M=20)
        try:
            zh = np.zeros_like(c["z"])
            mpr.mpr_fill(ctx, zh)
            outs.append(zh)
        finally:
            mpr.mpr_free(ctx)
    assert np.array_equal(outs[0], outs[1])


def test_pooled_memory_reuse_and_release():
    # contexts take device memory from the library's pool: a context built on memory that
    # a released context left behind, and one built after the pool was handed back to
    # the driver, give bitwise the same states as the first one
    c = synth.config("grid64")
    H, W = c["z"].shape

    def states():
        ctx = make_ctx(c["z"], c["mask"], seed=9)
        try:
            mpr.mpr_set_T(ctx, 0.2)
            mpr.mpr_sweep(ctx, 5, 3.0)
            phi = np.zeros((H, W), np.float32)
            mpr.mpr_get_state(ctx, phi)
        finally:
            mpr.mpr_free(ctx)
        return phi

    first = states()
    assert np.array_equal(states(), first)
    mpr.mpr_release_memory()
    assert np.array_equal(states(), first)
    mpr.mpr_release_memory()


@pytest.mark.parametrize("exec_mode", EXEC)
@pytest.mark.parametrize("i_max", [0, 1, 5, 9])
def test_relaxation_loop_stops_at_i_max(exec_mode, i_max):
    # Algorithm 2 step 5 ends after sweep i = i_max + 1 when the slope test has not passed
    # (n_fit larger than the run: the slope stays at its initial -1); the device-side loop
    # runs chunks of several sweeps, so it must stop within one chunk and leave the counters
    # exactly where the oracle's loop leaves them
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    ctx = make_ctx(z, mask, seed=4, i_max=i_max, n_fit=10**6, exec_mode=exec_mode)
    try:
        mpr.mpr_set_T(ctx, 0.2)
        st = mpr.mpr_equilibrate(ctx)
        phi = np.zeros(z.shape, np.float32)
        sw = mpr.mpr_get_state(ctx, phi)
        mpr.mpr_sweep(ctx, 3, 1.0)                     # the context stays usable
        sw2 = mpr.mpr_get_state(ctx, phi)
    finally:
        mpr.mpr_free(ctx)
    ref = orc.map_angles(z, mask)[0]
    orc.init_gaps(ref, mask, 4)
    out, sw_ref, _ = orc.equilibrate(ref, mask, 0.2, orc.params(seed=4, i_max=i_max, n_fit=10**6))
    assert st.sweeps == out.sweeps == i_max + 1
    assert st.converged == 0
    assert st.a == out.a
    assert sw == sw_ref and sw2 == sw + 3
