"""The allocation-free entry point against the allocating one (collected last on purpose).

mpr_sample_energy_static serves callers that may not allocate device memory; it keeps its
scratch in one fixed device array shared by all calls.  Two calls in a row on different
inputs (and a repeat of the first) must each agree with e_s as mpr_init computes it,
within the relative 1e-6 that the parity tests allow Eq. 4 energies (mpr_init forms the
cosine arguments in FP32, this entry point in FP64).
"""
import numpy as np
import pytest

from paper_1811_01604_gb300 import mpr, synth

pytestmark = pytest.mark.gpu


def _pairs(mask):
    m = mask.astype(bool)
    return int((m[:, 1:] & m[:, :-1]).sum() + (m[1:, :] & m[:-1, :]).sum())


def _allocating_e_s(z, mask):
    H, W = z.shape
    ctx = mpr.mpr_init(z, mask, W, H, mpr.mpr_default_params())
    try:
        return mpr.mpr_get_info(ctx)["e_s"]
    finally:
        mpr.mpr_free(ctx)


def test_static_sample_energy_matches_allocating_path_on_consecutive_calls():
    import torch
    cases = []
    z1 = synth.wm_field(300, 0.5, 5.0, seed=101, W=257)
    m1 = synth.mask_uniform(300, 257, 0.33, seed=102)
    z2 = synth.wm_field(64, 2.5, 16.0, seed=103)
    m2 = synth.mask_uniform(64, 64, 0.66, seed=104)
    for z, m in ((z1, m1), (z2, m2), (z1, m1)):
        H, W = z.shape
        zd = torch.from_numpy(z).cuda()
        md = torch.from_numpy(m).cuda()
        e_s, n_pairs = mpr.mpr_sample_energy_static(zd, md, W, H, 0.5)
        torch.cuda.synchronize()
        cases.append((e_s, n_pairs, _allocating_e_s(z, m), _pairs(m)))
    for e_s, n_pairs, ref, ref_pairs in cases:
        assert n_pairs == ref_pairs
        assert abs(e_s / ref - 1) < 1e-6
    assert cases[0][0] == cases[2][0]            # the shared scratch keeps no state


def test_static_sample_energy_limits_and_errors():
    import torch
    z = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    m = torch.ones((4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(mpr.MprError) as e:
        mpr.mpr_sample_energy_static(z, m, 4, 4)            # constant data: Eq. 1 undefined
    assert e.value.status == mpr.MPR_ENODATA
    zr = torch.arange(16, dtype=torch.float32, device="cuda").reshape(4, 4)
    with pytest.raises(mpr.MprError) as e:
        mpr.mpr_sample_energy_static(zr, m, 4, 4, 0.6)      # q outside (0, 1/2], as mpr_init
    assert e.value.status == mpr.MPR_EINVAL
    big = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(mpr.MprError) as e:
        mpr.mpr_sample_energy_static(big, big, 1, 16385)    # more rows than the scratch holds
    assert e.value.status == mpr.MPR_EINVAL
