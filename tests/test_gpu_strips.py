"""Row strips of one grid on the GPU (paper_1811_01604_gb300.strips with the library's strip
contexts), several strips driven by one process on one GPU, against a single context on
the whole grid.

The strips draw the whole grid's random numbers (Philox site index of the grid) and see
their neighbours' boundary rows after every half-sweep, so with the slope test off (the
relaxation then runs i_max + 1 sweeps, its window driven by exact acceptance counts) the
final lattice and the estimates must equal the single context's bit for bit.  With the
slope test on, the strips' energy totals are added in another order than the single
context's (rounding only), which leaves the relaxation's stopping sweep unchanged except in
a case of measure zero: the whole method (T-hat from the strips' Eq. 4 sums and the table
of the grid's shape, relaxation, M sweeps) must then give the single context's T-hat
(within 1e-12), stopping sweep and estimates.
"""
import numpy as np
import pytest

from paper_1811_01604_gb300 import mpr, strips, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

H, W, M = 301, 257, 24


def _grid():
    z = synth.wm_field(H, 0.5, 6.0, seed=77, W=W)
    mask = synth.mask_uniform(H, W, 0.45, seed=78)
    return torch.from_numpy(z).cuda(), torch.from_numpy(mask).cuda()


def _single(z, mask, T, **kw):
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params(seed=5, exec_mode=mpr.MPR_EXEC_LIST, M=M, **kw))
    try:
        if T is None:
            T, _ = mpr.mpr_estimate_T(ctx)
        else:
            mpr.mpr_set_T(ctx, T)
        st = mpr.mpr_equilibrate(ctx)
        zh = torch.empty_like(z)
        mpr.mpr_predict(ctx, M, zh)
        phi = torch.empty_like(z)
        mpr.mpr_get_state(ctx, phi)
    finally:
        mpr.mpr_free(ctx)
    return zh, phi, st.sweeps, T


def _strips(z, mask, n, T, **kw):
    ss = [strips.GpuStrip(z, mask, y0, y1, H, mpr.mpr_default_params(seed=5, M=M, **kw))
          for y0, y1 in strips.partition(H, n)]
    try:
        est, sweeps = strips.fill(strips.LocalComm(ss), M, T=T)
        T_hat = mpr.mpr_get_info(ss[0].ctx)["T"]
        phi = torch.cat([s.state() for s in ss])
        return torch.cat(est), phi, sweeps, T_hat
    finally:
        for s in ss:
            s.close()


@pytest.mark.parametrize("n", [2, 3, 5])
def test_strips_reproduce_the_single_context_bitwise(n):
    z, mask = _grid()
    kw = dict(i_max=39, n_fit=10**6)
    zh0, phi0, sw0, _ = _single(z, mask, 0.12, **kw)
    zh1, phi1, sw1, _ = _strips(z, mask, n, 0.12, **kw)
    assert sw0 == sw1 == 40
    assert torch.equal(phi0.view(torch.int32), phi1.view(torch.int32))
    assert torch.equal(zh0.view(torch.int32), zh1.view(torch.int32))


def test_strips_run_the_whole_method_like_the_single_context():
    z, mask = _grid()
    zh0, phi0, sw0, T0 = _single(z, mask, None)
    zh1, phi1, sw1, T1 = _strips(z, mask, 3, None)
    assert abs(T1 / T0 - 1) < 1e-12
    assert sw0 == sw1
    assert torch.equal(zh0.view(torch.int32), zh1.view(torch.int32))
    gap = mask == 0
    assert torch.equal(zh1[~gap], z[~gap])


def test_strip_arguments_are_checked():
    z, mask = _grid()
    with pytest.raises(mpr.MprError) as e:                    # odd first row of the block
        mpr.mpr_strip_init(z[1:20].contiguous(), mask[1:20].contiguous(), W, 19, 1, H, 0.0, 1.0)
    assert e.value.status == mpr.MPR_EINVAL
    with pytest.raises(mpr.MprError) as e:                    # the tile kernels carry no row offset
        mpr.mpr_strip_init(z[:20].contiguous(), mask[:20].contiguous(), W, 20, 0, H, 0.0, 1.0,
                           mpr.mpr_default_params(exec_mode=mpr.MPR_EXEC_TILE))
    assert e.value.status == mpr.MPR_EINVAL
    with pytest.raises(mpr.MprError) as e:                    # a block without an own row
        mpr.mpr_strip_init(z[10:12].contiguous(), mask[10:12].contiguous(), W, 2, 10, H, 0.0, 1.0)
    assert e.value.status == mpr.MPR_EINVAL
