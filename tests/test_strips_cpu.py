"""Row strips of one grid on the CPU: the oracle's strip functions pinned to its whole-grid
functions, and the strip driver (paper_1811_01604_gb300.strips) with oracle strips, in one
process and over two gloo ranks.

The strip decomposition changes nothing in the method: the checkerboard of Sect. 3.3 makes
the sites of one colour independent given the other colour, and the random numbers are
drawn from counters of the whole grid's site indices.  So a run over strips must give the
whole-grid run's lattice and estimates bit for bit, as long as nothing depends on the order
in which floating-point totals are added: the window of Algorithm 2 step 5.2 depends on
integer acceptance counts (exact), and the slope test of step 5.4, which reads the energy
sum, is switched off (n_fit beyond the run), so the relaxation runs i_max + 1 sweeps.
"""
import os
import sys

import numpy as np
import pytest

import oracle.oracle as orc
from paper_1811_01604_gb300 import strips, synth

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
from _strip_oracle import OracleStrip  # noqa: E402

H, W, T, M, I_MAX = 42, 37, 0.15, 12, 29


def _grid(seed=5):
    z = synth.wm_field(H, 0.5, 4.0, seed=seed, W=W)
    mask = synth.mask_uniform(H, W, 0.45, seed=seed + 1)
    return z, mask


def _prm():
    return orc.params(seed=3, i_max=I_MAX, n_fit=10**6, M=M)


def _whole_grid(z, mask):
    prm = _prm()
    phi, zmin, zmax, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, prm.seed, 0)
    phi0 = phi.copy()
    out, sw, _ = orc.equilibrate(phi, mask, T, prm)
    relaxed = phi.copy()
    zhat, _ = orc.predict(phi, mask, z, T, prm, zmin, zmax, M, sweep_index=sw)
    return phi0, relaxed, zhat, out


def test_partition_blocks_start_on_even_rows():
    for Hg in (4, 5, 42, 1001):
        for n in range(1, min(8, Hg // 2) + 1):
            parts = strips.partition(Hg, n)
            assert parts[0][0] == 0 and parts[-1][1] == Hg
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            for y0, y1 in parts:
                row0, Hb = strips.block(y0, y1, Hg)
                assert row0 % 2 == 0 and y1 > y0 and row0 + Hb <= Hg


def test_oracle_strip_sweeps_and_energy_are_the_whole_grid_ones():
    z, mask = _grid()
    phi, _, _, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, 7, 0)
    whole = phi.copy()
    n_whole = orc.sweep(whole, mask, 2.5, T, seed=7, sweep_index=4)
    parts = strips.partition(H, 3)
    blocks = []
    for y0, y1 in parts:
        row0, Hb = strips.block(y0, y1, H)
        frozen = mask[row0:row0 + Hb].copy()
        frozen[:y0 - row0] = 1
        frozen[y1 - row0:] = 1
        blocks.append([phi[row0:row0 + Hb].copy(), frozen, row0, y0 - row0, y1 - row0])
    n = 0
    for color in (0, 1):
        for b in blocks:
            n += orc.sweep_rows(b[0], b[1], b[2], b[3], b[4], color, 2.5, T, seed=7, sweep_index=4)
        for k in range(len(blocks) - 1):                      # boundary rows to the neighbours
            blocks[k + 1][0][0] = blocks[k][0][blocks[k][4] - 1]
            blocks[k][0][-1] = blocks[k + 1][0][blocks[k + 1][3]]
    got = np.concatenate([b[0][b[3]:b[4]] for b in blocks])
    assert n == n_whole
    assert np.array_equal(got, whole)
    E = sum(orc.energy_rows(b[0], b[3], b[4]) for b in blocks)
    assert abs(E - orc.energy(whole)) <= 1e-12 * abs(orc.energy(whole))


def test_relax_steps_reproduce_the_oracle_loop():
    z, mask = _grid(9)
    prm = orc.params(seed=2, i_max=60, n_fit=8, n_f=3)
    phi, _, _, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, prm.seed, 0)
    ref = phi.copy()
    out, _, ehist = orc.equilibrate(ref, mask, T, prm)
    P = int((mask == 0).sum())
    ngp = orc.n_gp(W, H)
    r = orc.Relax(prm, orc.energy(phi) / ngp)
    go, sw = True, 0
    while go:
        nacc = orc.sweep(phi, mask, r.s.a, T, seed=prm.seed, sweep_index=sw)
        sw += 1
        go = r.step(nacc, P, orc.energy(phi) / ngp)
    assert (r.s.i, r.s.a, r.s.k) == (out.sweeps, out.a, out.k)
    assert np.array_equal(r.hist[: r.s.i + 1], ehist)
    assert np.array_equal(phi, ref)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_strip_driver_in_one_process_matches_the_whole_grid(n):
    z, mask = _grid()
    phi0, relaxed, zhat, out = _whole_grid(z, mask)
    ss = [OracleStrip(phi0, z, mask, y0, y1, _prm()) for y0, y1 in strips.partition(H, n)]
    est, sweeps = strips.fill(strips.LocalComm(ss), M, T=T)
    assert sweeps == out.sweeps == I_MAX + 1
    assert np.array_equal(np.concatenate(est), zhat)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(HERE))
    sys.path.insert(0, HERE)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z, mask = _grid()
        phi, _, _, _ = orc.map_angles(z, mask)
        orc.init_gaps(phi, mask, _prm().seed, 0)
        y0, y1 = strips.partition(H, world)[rank]
        s = OracleStrip(phi, z, mask, y0, y1, _prm())
        est, sweeps = strips.fill(strips.DistComm(s, dist), M, T=T)
        q.put((rank, est[0], s.state().copy(), sweeps))
    finally:
        dist.destroy_process_group()


def test_strip_driver_over_two_gloo_ranks_matches_the_whole_grid():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    z, mask = _grid()
    _, _, zhat, out = _whole_grid(z, mask)
    assert all(r[3] == out.sweeps for r in res)
    assert np.array_equal(np.concatenate([r[1] for r in res]), zhat)
