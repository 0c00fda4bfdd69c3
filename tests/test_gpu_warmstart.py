"""What the trained warm start gains: a network trained (by the library's own kernels) on
equilibrium states of the MCMC starts the relaxation closer to equilibrium, so Algorithm 2's
slope test stops after fewer sweeps, at the same final error (the MCMC, unchanged, still
decides it).  Evaluated on fresh grids with the 1024 x 1024 workload's statistics
(nu = 0.5, correlation length 16, 33 % uniform gaps) at 256 x 256.

Run with -s to print the numbers.
"""
import json
import math

import numpy as np
import pytest

from paper_1811_01604_gb300 import mpr, synth, warmstart

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def trained():
    groups = warmstart.training_grids(n64=256, n128=512, seed=10_000)
    sets = [warmstart.equilibrium_states(z, m, states_per_grid=4, spacing=20, seed=20_000) for z, m in groups]
    held = [warmstart.equilibrium_states(z[:32], m[:32], states_per_grid=1, seed=30_000)
            for z, m in warmstart.training_grids(n64=32, n128=32, seed=40_000)]
    net = warmstart.WarmStartNet(seed=0)
    loss0 = [warmstart.eval_loss(net, s) for s in held]
    losses = warmstart.train(net, sets, steps=800, batch=32, lr=1e-3, seed=0)
    loss1 = [warmstart.eval_loss(net, s) for s in held]
    yield net, dict(train_first=float(np.mean(losses[:20])), train_last=float(np.mean(losses[-20:])),
                    held_before=loss0, held_after=loss1, n_states=sum(s.n for s in sets))
    net.close()


def _eval_grids(n, L=256, seed=1):
    zs = [synth.wm_field_gpu(L, L, 0.5, 16.0, seed + i) for i in range(n)]
    ms = [synth.mask_uniform_gpu(L, L, 0.33, seed + 1_000_000 + i) for i in range(n)]
    return zs, ms


def _fill(zs, ms, net=None, seed=5):
    ctx = mpr.mpr_init_batch(zs, ms, mpr.mpr_default_params(seed=seed))
    try:
        if net is not None:
            net.warmstart(ctx)
        out = [torch.zeros_like(z) for z in zs]
        mpr.mpr_fill_batch(ctx, out)
        sweeps = [mpr.mpr_batch_info(ctx, g)["sweeps"] for g in range(len(zs))]
    finally:
        mpr.mpr_free(ctx)
    mae = [float((o - z)[m == 0].abs().mean()) for o, z, m in zip(out, zs, ms)]
    return np.array(sweeps), np.array(mae)


def test_trained_network_cuts_relaxation_sweeps_at_equal_error(trained):
    net, tr = trained
    assert tr["train_last"] < 0.7 * tr["train_first"]
    assert all(a < 0.8 * b for a, b in zip(tr["held_after"], tr["held_before"]))
    zs, ms = _eval_grids(6)
    s_rand, e_rand = _fill(zs, ms)
    s_warm, e_warm = _fill(zs, ms, net)
    report = dict(training=tr, sweeps_random=s_rand.tolist(), sweeps_warm=s_warm.tolist(),
                  mae_random=e_rand.tolist(), mae_warm=e_warm.tolist())
    print("WARMSTART_REPORT " + json.dumps(report))
    assert s_warm.mean() < s_rand.mean()
    assert e_warm.mean() <= 1.02 * e_rand.mean()
