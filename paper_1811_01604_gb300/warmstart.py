"""Learned warm start: training data made by the library's own MCMC, and the training loop.

The network (include/mpr_net.h) proposes the initial gap angles that Algorithm 2 otherwise
draws uniformly at random; the conditional hybrid Monte Carlo that follows is unchanged, so
it still decides the final error.  Its training targets are equilibrium states of that
MCMC: grids with the statistics of the 64 x 64 and 1024 x 1024 workloads (fresh seeds),
relaxed by Algorithm 2 at their own estimated temperature, then sampled every few sweeps.

Every numeric step (MCMC, network forward/backward, Adam) runs in libmpr's kernels; this
module only generates seeded inputs, slices batches and calls the C ABI.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import mpr, synth


def _lognormal_t(z):
    g = (z - 50.0) / 10.0
    return 50.0 * (0.5 * g - 0.125).exp()


def _uniform_masks(n, H, W, p, seed, device):
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    r = torch.rand((n, H * W), generator=gen, device=device)
    k = int(round(p * H * W))
    idx = torch.topk(r, k, dim=1).indices            # k distinct sites per grid
    m = torch.ones((n, H * W), dtype=torch.uint8, device=device)
    m.scatter_(1, idx, 0)
    return m.view(n, H, W)


def training_grids(n64: int, n128: int, seed: int = 10_000, device="cuda", n256: int = 0):
    """Input grids for the training set, as shape groups of (z, mask) CUDA tensors:
      * n64 grids 64 x 64: nu = 0.5, correlation length 4, 33 % uniform gaps;
      * n128 crops 128 x 128 of 1024 x 1024 fields: nu in {0.5, 2.5}, correlation
        length 16, Gaussian or lognormal, 33 % or 66 % uniform gaps;
      * n256 crops 256 x 256 of 4096 x 4096 fields with nu = 1, correlation length 32, and
        half of the sites missing as disks of radius 8-64 (a quarter of the crop) plus
        uniform gaps: the statistics of the 4096^2 workload, whose large holes the other
        groups never show.
    Seeds start at `seed` (>= 10^4, disjoint from the evaluation workloads)."""
    import torch
    groups = []
    if n64:
        zs = [synth.wm_field_gpu(64, 64, 0.5, 4.0, seed + i, device=device) for i in range(n64)]
        z = torch.stack(zs)
        m = _uniform_masks(n64, 64, 64, 0.33, seed + 500_000, device)
        groups.append((z.contiguous(), m.contiguous()))
    if n128:
        per = 64                                        # crops per 1024^2 field
        zs, ms = [], []
        f = 0
        while sum(x.shape[0] for x in zs) < n128:
            rng = np.random.Generator(np.random.PCG64(seed + 100_000 + f))
            nu = float(rng.choice([0.5, 2.5]))
            p = float(rng.choice([0.33, 0.66]))
            z = synth.wm_field_gpu(1024, 1024, nu, 16.0, seed + 100_000 + f, device=device)
            if rng.random() < 0.5:
                z = _lognormal_t(z.double()).float()
            c = z.view(8, 128, 8, 128).permute(0, 2, 1, 3).reshape(per, 128, 128)
            zs.append(c)
            ms.append(_uniform_masks(per, 128, 128, p, seed + 200_000 + f, device))
            f += 1
        groups.append((torch.cat(zs)[:n128].contiguous(), torch.cat(ms)[:n128].contiguous()))
    if n256:
        zs, ms = [], []
        f = 0
        while sum(x.shape[0] for x in zs) < n256:
            z = synth.wm_field_gpu(4096, 4096, 1.0, 32.0, seed + 300_000 + f, device=device)
            zs.append(z.view(16, 256, 16, 256).permute(0, 2, 1, 3).reshape(256, 256, 256))
            f += 1
        z = torch.cat(zs)[:n256].contiguous()
        m = np.stack([synth.mask_disks(256, 256, 0.5, seed + 400_000 + i) for i in range(n256)])
        groups.append((z, torch.from_numpy(m).to(device).contiguous()))
    return groups


@dataclass
class StateSet:
    """Equilibrium states of one shape: z, mask, phi [N][H][W] (CUDA), zmin, zmax [N]."""
    z: object
    mask: object
    phi: object
    zmin: np.ndarray
    zmax: np.ndarray

    @property
    def n(self):
        return int(self.z.shape[0])


def equilibrium_states(z, mask, states_per_grid: int = 4, spacing: int = 20, seed: int = 10_000,
                       chunk: int = 1024) -> StateSet:
    """Runs Algorithm 2 (estimate T, relax with the slope test) on every grid of a batch and
    records `states_per_grid` states `spacing` equilibrium sweeps apart."""
    import torch
    N, H, W = z.shape
    zo, mo, po, zmin, zmax = [], [], [], [], []
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        zz = [z[i] for i in range(c0, c1)]
        mm = [mask[i] for i in range(c0, c1)]
        prm = mpr.mpr_default_params(seed=seed + c0, T_cap=256)
        ctx = mpr.mpr_init_batch(zz, mm, prm)
        try:
            mpr.mpr_estimate_T(ctx)
            mpr.mpr_equilibrate(ctx)
            info = [mpr.mpr_batch_info(ctx, g) for g in range(c1 - c0)]
            for k in range(states_per_grid):
                if k:
                    mpr.mpr_sweep(ctx, spacing, prm.a_eq)
                phi = torch.empty((c1 - c0, H, W), dtype=torch.float32, device=z.device)
                for g in range(c1 - c0):
                    mpr.mpr_get_state_batch(ctx, g, phi[g])
                po.append(phi)
                zo.append(z[c0:c1])
                mo.append(mask[c0:c1])
                zmin += [x["zmin"] for x in info]
                zmax += [x["zmax"] for x in info]
        finally:
            mpr.mpr_free(ctx)
    return StateSet(torch.cat(zo).contiguous(), torch.cat(mo).contiguous(), torch.cat(po).contiguous(),
                    np.array(zmin), np.array(zmax))


class WarmStartNet:
    """Owner of an mpr_net handle."""

    def __init__(self, seed: int = 0, stream=None, stride: int = 1):
        self.h = mpr.mpr_net_create(seed, stream, stride=stride)

    def close(self):
        if self.h:
            mpr.mpr_net_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return mpr.mpr_net_num_params(self.h)

    def params(self):
        out = np.zeros(self.num_params, np.float32)
        mpr.mpr_net_get_params(self.h, out)
        return out

    def set_params(self, p):
        mpr.mpr_net_set_params(self.h, np.ascontiguousarray(p, dtype=np.float32))

    def warmstart(self, ctx):
        mpr.mpr_warmstart_init(ctx, self.h)


def train(net: WarmStartNet, sets, steps: int, batch: int = 32, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0, lr_final: float = 0.1):
    """Adam on random batches (drawn per step from one shape group, groups in proportion
    to their number of sites; `batch` grids of 128^2 sites or the same number of sites in
    other shapes); cosine decay of the learning rate to lr * lr_final.  Returns the loss of
    every step."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.array([s.n * s.z.shape[1] * s.z.shape[2] for s in sets], np.float64)
    prob = sizes / sizes.sum()
    losses = []
    for it in range(steps):
        s = sets[int(rng.choice(len(sets), p=prob))]
        # batches of about batch x 128^2 sites whatever the shape
        bs = max(1, min(s.n, int(round(batch * 128 * 128 / (s.z.shape[1] * s.z.shape[2])))))
        idx = np.sort(rng.choice(s.n, size=bs, replace=False))
        ti = torch.as_tensor(idx, device=s.z.device)
        z = s.z.index_select(0, ti).contiguous()
        m = s.mask.index_select(0, ti).contiguous()
        ph = s.phi.index_select(0, ti).contiguous()
        B, H, W = z.shape
        f = lr_final + (1 - lr_final) * 0.5 * (1 + math.cos(math.pi * it / max(1, steps)))
        loss = mpr.mpr_net_train_step(net.h, z, m, ph, s.zmin[idx], s.zmax[idx], B, H, W, lr * f)
        losses.append(loss)
        if log_every and (it % log_every == 0 or it == steps - 1):
            print(f"step {it} loss {loss:.4f}", flush=True)
    return losses


def eval_loss(net: WarmStartNet, s: StateSet, batch: int = 64) -> float:
    """Mean loss over a state set (gradients are computed and then discarded)."""
    tot, n = 0.0, 0
    for b0 in range(0, s.n, batch):
        b1 = min(s.n, b0 + batch)
        B, H, W = b1 - b0, s.z.shape[1], s.z.shape[2]
        lo = mpr.mpr_net_loss_grad(net.h, s.z[b0:b1], s.mask[b0:b1], s.phi[b0:b1], s.zmin[b0:b1],
                                   s.zmax[b0:b1], B, H, W)
        tot += lo * B
        n += B
    mpr.mpr_net_zero_grads(net.h)
    return tot / max(1, n)
