"""The persistent multi-sweep kernel (one launch per phase) against the list path, and its
bounded waits.

* A fixed-window phase is one launch in which tiles start their next sweep as soon as they
  and their eight neighbours have finished the previous one; the relaxation is one launch
  in which every sweep waits for the control step of the one before.  Both must leave the
  lattice bitwise equal to the list path's half-sweep launches (same arithmetic, same Philox
  counters), on grids of many tiles, in every compiled tile configuration, with the same
  tracked energies: each site's energy change is rounded to a whole number of 2^-23 where
  it is computed and the totals are integer sums, so no result depends on the kernel, the
  tile shape, the thread count or the order in which tiles finish.  A relaxation with the
  slope test therefore stops at the same sweep with the same lattice in every
  configuration.
* A wait that expires (test support: block 0 waits for a flag that nothing sets, with a
  short limit) must end the launch with MPR_ETIMEOUT, and the GPU and the library must
  still give correct results afterwards.
"""
import numpy as np
import pytest

from paper_1811_01604_gb300 import mpr, synth

pytestmark = pytest.mark.gpu


def _ctx(z, mask, **kw):
    H, W = z.shape
    return mpr.mpr_init(np.ascontiguousarray(z, np.float32), np.ascontiguousarray(mask, np.uint8), W, H,
                        mpr.mpr_default_params(**kw))


def _state(ctx, shape):
    phi = np.zeros(shape, np.float32)
    sw = mpr.mpr_get_state(ctx, phi)
    return phi, sw


def _grid(H, W, seed):
    z = synth.wm_field(H, 1.0, 8.0, seed=seed, W=W)
    mask = synth.mask_disks(H, W, 0.5, seed=seed + 1)
    return z, mask


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_fixed_window_launch_matches_list_path_bitwise(cfg):
    # 40 sweeps in one launch over 9 x 24 .. 18 x 48 tiles: sweeps overlap across the grid
    H, W = 290, 1530
    z, mask = _grid(H, W, 31)
    out = []
    for mode in (mpr.MPR_EXEC_LIST, mpr.MPR_EXEC_TILE):
        ctx = _ctx(z, mask, seed=5, exec_mode=mode, tile_cfg=cfg)
        try:
            mpr.mpr_set_T(ctx, 0.07)
            mpr.mpr_sweep(ctx, 40, 1.0)
            mpr.mpr_sweep(ctx, 13, 6.0)
            phi, sw = _state(ctx, z.shape)
            out.append((phi, sw, mpr.mpr_get_info(ctx)))
        finally:
            mpr.mpr_free(ctx)
    (p0, s0, i0), (p1, s1, i1) = out
    assert s0 == s1 == 53
    assert np.array_equal(p0.view(np.uint32), p1.view(np.uint32))
    assert i0["H_exact"] == i1["H_exact"]
    assert i0["H_tracked"] == i1["H_tracked"]


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_relaxation_launch_matches_list_path(cfg):
    # the whole relaxation in one launch: same stopping sweep, window and lattice
    H, W = 300, 700
    z, mask = _grid(H, W, 41)
    out = []
    for mode in (mpr.MPR_EXEC_LIST, mpr.MPR_EXEC_TILE):
        ctx = _ctx(z, mask, seed=8, exec_mode=mode, tile_cfg=cfg)
        try:
            mpr.mpr_set_T(ctx, 0.05)
            st = mpr.mpr_equilibrate(ctx)
            phi, sw = _state(ctx, z.shape)
            out.append((phi, sw, st))
        finally:
            mpr.mpr_free(ctx)
    (p0, s0, st0), (p1, s1, st1) = out
    assert st0.sweeps == st1.sweeps > 20 and s0 == s1 == st1.sweeps
    assert st0.a == st1.a and st0.converged == st1.converged
    assert np.array_equal(p0.view(np.uint32), p1.view(np.uint32))


def test_relaxation_is_the_same_in_every_configuration_at_1024():
    # the slope test reads the exact energy totals: list path and every tile shape stop at
    # the same sweep with the same window, lattice and tracked energy
    z = synth.wm_field(1024, 0.5, 16.0, seed=91)
    mask = synth.mask_uniform(1024, 1024, 0.33, seed=92)
    runs = []
    for mode, cfg in ((mpr.MPR_EXEC_LIST, 0), (mpr.MPR_EXEC_TILE, 0), (mpr.MPR_EXEC_TILE, 1),
                      (mpr.MPR_EXEC_TILE, 2)):
        ctx = _ctx(z, mask, seed=12, exec_mode=mode, tile_cfg=cfg)
        try:
            mpr.mpr_estimate_T(ctx)
            st = mpr.mpr_equilibrate(ctx)
            phi, sw = _state(ctx, z.shape)
            runs.append((st.sweeps, st.a, mpr.mpr_get_info(ctx)["H_tracked"], phi))
        finally:
            mpr.mpr_free(ctx)
    for r in runs[1:]:
        assert r[:3] == runs[0][:3]
        assert np.array_equal(r[3].view(np.uint32), runs[0][3].view(np.uint32))
    assert runs[0][0] > 20


def test_equilibrium_launch_prediction_matches_list_path():
    # the M accumulating sweeps of the prediction as one launch (per-tile angle sums)
    H, W = 200, 520
    z, mask = _grid(H, W, 51)
    out = []
    for mode in (mpr.MPR_EXEC_LIST, mpr.MPR_EXEC_TILE):
        ctx = _ctx(z, mask, seed=3, exec_mode=mode)
        try:
            mpr.mpr_set_T(ctx, 0.05)
            mpr.mpr_sweep(ctx, 30, 4.0)
            zh = np.zeros_like(z)
            mpr.mpr_predict(ctx, 60, zh)
            out.append(zh)
        finally:
            mpr.mpr_free(ctx)
    gap = mask == 0
    # same chain; the angle sums are added in another order (per tile vs per gap list)
    assert np.abs(out[0].astype(np.float64) - out[1])[gap].max() < 1e-3
    assert np.array_equal(out[0][~gap], out[1][~gap])


def test_batch_of_many_shapes_in_one_relaxation_launch():
    # grids stop at different sweeps inside one launch; each must match its own list run
    shapes = [(40, 50), (128, 300), (17, 900), (256, 256)]
    zs, ms = [], []
    for i, (H, W) in enumerate(shapes):
        zs.append(synth.wm_field(H, 1.0, 8.0, seed=60 + 2 * i, W=W))
        ms.append(synth.mask_uniform(H, W, 0.4, seed=61 + 2 * i))
    res = {}
    for mode in (mpr.MPR_EXEC_LIST, mpr.MPR_EXEC_TILE):
        ctx = mpr.mpr_init_batch(zs, ms, mpr.mpr_default_params(seed=2, exec_mode=mode))
        try:
            mpr.mpr_set_T(ctx, 0.06)
            mpr.mpr_equilibrate(ctx)
            res[mode] = [mpr.mpr_batch_info(ctx, g)["sweeps"] for g in range(len(shapes))]
            phis = []
            for g, (H, W) in enumerate(shapes):
                phi = np.zeros((H, W), np.float32)
                mpr.mpr_get_state_batch(ctx, g, phi)
                phis.append(phi)
            res[(mode, "phi")] = phis
        finally:
            mpr.mpr_free(ctx)
    assert res[mpr.MPR_EXEC_LIST] == res[mpr.MPR_EXEC_TILE]
    assert len(set(res[mpr.MPR_EXEC_TILE])) > 1                     # they stop at different sweeps
    for a, b in zip(res[(mpr.MPR_EXEC_LIST, "phi")], res[(mpr.MPR_EXEC_TILE, "phi")]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("phase", ["fixed", "relax"])
def test_expired_wait_returns_timeout_and_gpu_stays_usable(phase):
    z, mask = _grid(96, 700, 71)
    H, W = z.shape

    def reference():
        ctx = _ctx(z, mask, seed=6)
        try:
            mpr.mpr_set_T(ctx, 0.1)
            mpr.mpr_sweep(ctx, 6, 2.0)
            return _state(ctx, z.shape)[0]
        finally:
            mpr.mpr_free(ctx)

    before = reference()
    mpr.mpr_debug_wait_limit(2_000_000, stall=True)          # 2 ms, and a flag nothing sets
    try:
        ctx = _ctx(z, mask, seed=6)
        try:
            mpr.mpr_set_T(ctx, 0.1)
            with pytest.raises(mpr.MprError) as e:
                if phase == "fixed":
                    mpr.mpr_sweep(ctx, 6, 2.0)
                else:
                    mpr.mpr_equilibrate(ctx)
            assert e.value.status == mpr.MPR_ETIMEOUT
        finally:
            mpr.mpr_free(ctx)
    finally:
        mpr.mpr_debug_wait_limit(0, stall=False)
    # the device and the library are fine: a fresh context gives the same state as before
    after = reference()
    assert np.array_equal(before.view(np.uint32), after.view(np.uint32))


def test_trace_stamps_every_item_and_changes_nothing():
    # the bench's timestamps (mpr_debug_trace): every work item of a fixed-window launch is
    # stamped in order (taken, copy issued, copy landed, updated, written back), every
    # control step has its ticket before its publication, and the lattice is bitwise what
    # the same sweeps give without the trace
    import torch
    z, mask = _grid(290, 1530, 31)
    ntiles = 10 * 12                                   # 32 x 128 tiles
    states = []
    for traced in (False, True):
        ctx = _ctx(z, mask, seed=5, tile_cfg=2)
        try:
            mpr.mpr_set_T(ctx, 0.07)
            buf = torch.zeros(ntiles * 12 * 6 + 8192, dtype=torch.int64, device="cuda")
            if traced:
                mpr.mpr_debug_trace(buf)
            try:
                mpr.mpr_sweep(ctx, 12, 1.0)
                torch.cuda.synchronize()
            finally:
                mpr.mpr_debug_trace(None)
            states.append(_state(ctx, z.shape)[0])
        finally:
            mpr.mpr_free(ctx)
    assert np.array_equal(states[0].view(np.uint32), states[1].view(np.uint32))
    t = buf.cpu().numpy().astype(np.int64)
    it = t[: ntiles * 12 * 6].reshape(-1, 6)
    assert np.all(it[:, :4] > 0)
    assert np.all(np.diff(it[:, :4], axis=1) >= 0)
    done = it[:, 4] > 0
    assert done.sum() >= len(it) - 152 * 8             # all but each block's last item
    assert np.all(it[done, 4] >= it[done, 3])
    blocks = it[:, 5] & 0xFFFFFFFF
    assert blocks.max() < 152 * 8
    ctl = t[ntiles * 12 * 6:].reshape(-1, 2)
    ctl = ctl[ctl[:, 0] > 0]
    assert len(ctl) == 12 and np.all(ctl[:, 1] >= ctl[:, 0])
