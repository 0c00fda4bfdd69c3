"""Pins of the FP64 oracle to facts fixed by the paper, by mathematics or by a library.

None of these retype the oracle's formulas: each compares it with a closed form,
an exact density by quadrature, an invariant, a library routine (cuRAND's host
Philox4x32-10), or the statistics the paper prints (Tables 2-3).
"""
import ctypes
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle.oracle as orc
from paper_1811_01604_gb300 import synth

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------- Philox (Sect. 3.3)
def _curand_host_blocks(seed, nblocks):
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            lib = ctypes.CDLL(path)
            break
        except OSError:
            continue
    else:
        pytest.skip("libcurand not available")
    g = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(g), 161):   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
    out = np.zeros(4 * nblocks, np.uint32)
    assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    lib.curandDestroyGenerator(g)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 0x0123456789ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host Philox4x32-10 generator emits block b of its stream from the counter
    # {b / 65536, 0, b % 65536, 0} under key (seed lo, seed hi).
    n = 3 * 65536
    ref = _curand_host_blocks(seed, n)
    b = np.arange(n, dtype=np.uint64)
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = (b >> 16).astype(np.uint32)
    ctr[:, 2] = (b & 0xFFFF).astype(np.uint32)
    got = orc.philox_batch(ctr, seed)
    assert np.array_equal(got, ref)


def test_philox_uniformity_of_site_streams():
    # counters {site, sweep, chain, 0}: the 24-bit uniforms must be U(0,1) and x0/x1 uncorrelated
    n = 200_000
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n) % 4096
    ctr[:, 1] = np.arange(n) // 4096
    ctr[:, 2] = 7
    o = orc.philox_batch(ctr, 12345)
    u = (o[:, 0] >> 8) / 2.0**24
    r = (o[:, 1] >> 8) / 2.0**24
    for v in (u, r):
        counts, _ = np.histogram(v, bins=64, range=(0, 1))
        assert stats.chisquare(counts).pvalue > 1e-3
        assert stats.kstest(v, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(u, r)[0, 1]) < 0.01


@pytest.mark.parametrize("start", [0.1, 3.0, 6.2])
def test_proposal_window_and_wrap_use_the_site_stream(start):
    # A lone free site has no neighbours: no reflection, dH = 0, so every proposal is
    # accepted and one sweep moves it by 2pi(u - 1/2)/a (mod 2pi) (Algorithm 1, steps 2-3),
    # with u the top 24 bits of word 0 of the Philox block at counter {site 0, sweep 0,
    # chain, 0}, which is block `chain` of cuRAND's host stream.
    seed = 0xC0FFEE
    blocks = _curand_host_blocks(seed, 96)
    for chain in range(96):
        a = 1.0 + (chain % 6) * 0.75
        phi = np.array([[start]])
        n = orc.sweep(phi, np.zeros((1, 1), np.uint8), a=a, T=1.0, seed=seed, chain=chain,
                      sweep_index=0)
        u = float(blocks[chain, 0] >> 8) / 2.0**24
        expect = math.fmod(start + TWO_PI * (u - 0.5) / a + 2 * TWO_PI, TWO_PI)
        assert n == 1 and abs(phi[0, 0] - expect) < 1e-12


# ---------------------------------------------------------------- Eq. 1 map
def test_map_closed_form_and_inverse():
    z = np.array([[10.0, 12.5, 20.0], [15.0, 99.0, 17.5]], np.float32)
    mask = np.array([[1, 1, 1], [1, 0, 1]], np.uint8)
    phi, zmin, zmax, ns = orc.map_angles(z, mask)
    assert ns == 5 and zmin == 10.0 and zmax == 20.0       # the gap value 99 is ignored
    want = {(0, 0): 0.0, (0, 1): math.pi / 2, (0, 2): TWO_PI, (1, 0): math.pi, (1, 2): 1.5 * math.pi}
    for (y, x), v in want.items():
        assert abs(phi[y, x] - v) < 1e-15
    assert phi[1, 1] == 0.0                                  # gap untouched
    for (y, x) in want:
        assert abs(orc.unmap(phi[y, x], zmin, zmax) - z[y, x]) < 1e-12


def test_map_degenerate_inputs():
    z = np.full((3, 3), 4.0, np.float32)
    mask = np.ones((3, 3), np.uint8)
    _, zmin, zmax, ns = orc.map_angles(z, mask)
    assert ns == 9 and zmin == zmax                          # constant data: no map exists
    mask1 = np.zeros((3, 3), np.uint8); mask1[1, 1] = 1
    _, _, _, ns1 = orc.map_angles(z, mask1)
    assert ns1 == 1
    with pytest.raises(ValueError):
        orc.fill(z, mask, orc.params(M=1), T_fixed=0.1, eq_sweeps=1)


# ---------------------------------------------------------------- Eq. 4 and Eq. 2
def test_sample_energy_constant_ramp_and_pairs():
    W, H = 7, 5
    mask = np.ones((H, W), np.uint8)
    phi = np.full((H, W), 2.0)
    e, nsp = orc.sample_energy(phi, mask)
    assert e == -1.0 and nsp == W * (H - 1) + H * (W - 1)
    beta = 0.3                                               # one-row ramp: every bond differs by beta
    phi1 = (beta * np.arange(W, dtype=np.float64))[None, :]
    e1, n1 = orc.sample_energy(phi1, np.ones((1, W), np.uint8), q=0.5)
    assert n1 == W - 1 and abs(e1 + math.cos(0.5 * beta)) < 1e-15
    cb = (np.indices((H, W)).sum(0) % 2).astype(np.uint8)   # checkerboard samples: no pairs
    assert orc.sample_energy(phi, cb)[1] == 0
    # two isolated pairs by hand
    m2 = np.zeros((3, 3), np.uint8); m2[0, 0] = m2[0, 1] = 1; m2[2, 2] = m2[1, 2] = 1
    p2 = np.zeros((3, 3)); p2[0, 1] = 1.0; p2[2, 2] = 3.0; p2[1, 2] = 0.5
    e2, n2 = orc.sample_energy(p2, m2)
    assert n2 == 2 and abs(e2 + 0.5 * (math.cos(0.5) + math.cos(1.25))) < 1e-15


def test_energy_bond_count_and_uniform_state():
    for W, H in [(1, 1), (1, 5), (4, 3), (16, 16)]:
        brute = sum(1 for y in range(H) for x in range(W) for dx, dy in ((1, 0), (0, 1))
                    if x + dx < W and y + dy < H)
        assert orc.n_gp(W, H) == brute
        assert orc.energy(np.full((H, W), 1.234), 0.5) == pytest.approx(-brute, abs=1e-12)
    # two sites: E = -cos(q dphi)
    assert orc.energy(np.array([[0.0, 2.0]]), 0.5) == pytest.approx(-math.cos(1.0), abs=1e-15)


# ---------------------------------------------------------------- Eq. 6 over-relaxation
def test_over_relaxation_conserves_local_energy_and_is_involution():
    rng = np.random.default_rng(5)
    reflected = 0
    for _ in range(20000):
        nnb = int(rng.integers(1, 5))
        nb = rng.uniform(0, TWO_PI, nnb)
        phi = rng.uniform(0, TWO_PI)
        p1 = orc.over_relax(phi, nb)
        assert 0.0 <= p1 < TWO_PI
        assert abs(orc.local_energy(p1, nb) - orc.local_energy(phi, nb)) <= 1e-12
        if p1 != phi:
            reflected += 1
            assert abs(orc.over_relax(p1, nb) - phi) <= 1e-12
    assert reflected > 5000                                 # the reflection is usually in range


def test_over_relaxation_special_cases():
    # neighbours at pi: local field along q*phi = pi/2, so phi -> 2pi - phi
    assert orc.over_relax(1.0, [math.pi] * 4) == pytest.approx(TWO_PI - 1.0, abs=1e-13)
    # counterexample to the printed (q = 1) formula: neighbours at 0, phi = 1
    lit = orc.over_relax(1.0, [0.0] * 4, mode=orc.OR_LITERAL)
    assert lit == pytest.approx(TWO_PI - 1.0, abs=1e-13)
    e0 = orc.local_energy(1.0, [0.0] * 4)
    assert orc.local_energy(lit, [0.0] * 4) == pytest.approx(-e0, abs=1e-12)   # energy flips sign
    assert orc.over_relax(1.0, [0.0] * 4) == 1.0            # reflection leaves [0,2pi): keep phi
    assert orc.over_relax(1.0, [0.0, TWO_PI], q=1.0) == 1.0  # vanishing field: keep phi
    assert orc.over_relax(2.5, [0.3, 1.0], mode=orc.OR_NONE) == 2.5


# ---------------------------------------------------------------- Algorithm 1 invariants
def test_samples_never_change_and_angles_stay_in_range():
    rng = np.random.default_rng(2)
    H, W = 13, 11
    mask = (rng.random((H, W)) < 0.5).astype(np.uint8)
    phi = rng.uniform(0, TWO_PI, (H, W))
    before = phi.copy()
    for s in range(40):
        orc.sweep(phi, mask, a=1.0 + s / 3.0, T=0.05, seed=9, sweep_index=s)
    assert np.array_equal(phi[mask == 1], before[mask == 1])
    assert np.all((phi >= 0) & (phi < TWO_PI))
    assert not np.array_equal(phi[mask == 0], before[mask == 0])


def _conditional_cdf(nb, T, q=0.5, n=200001):
    x = np.linspace(0.0, TWO_PI, n)
    logp = np.cos(q * (x[:, None] - np.asarray(nb)[None, :])).sum(1) / T
    p = np.exp(logp - logp.max())
    c = integrate.cumulative_trapezoid(p, x, initial=0.0)
    c /= c[-1]
    return lambda v: np.interp(v, x, c)


def _final_states(H, W, mask, phi0, T, a, sweeps, chains, or_mode=orc.OR_CONSERVING, q=0.5):
    out = []
    for ch in range(chains):
        phi = phi0.copy()
        orc.init_gaps(phi, mask, seed=77, chain=ch)
        for s in range(sweeps):
            orc.sweep(phi, mask, a=a, T=T, q=q, seed=77, chain=ch, sweep_index=s, or_mode=or_mode)
        out.append(phi.copy())
    return np.array(out)


@pytest.mark.parametrize("case", ["corner2", "center4", "center4_lowT", "center4_q0.3", "corner2_q0.15",
                                  "center4_q0.3_noOR"])
def test_single_free_site_matches_boltzmann_density(case):
    # Eq. 3 restricted to one free site: p(phi) ~ exp(sum_j cos(q(phi - phi_j)) / T) on [0, 2pi),
    # for the paper's q = 1/2 and for couplings below it (Eq. 2 allows q <= 1/2)
    q, or_mode = 0.5, orc.OR_CONSERVING
    if case.startswith("corner2"):
        H = W = 2; free = (0, 0); nb_idx = [(0, 1), (1, 0)]; T, a, sweeps = 0.4, 1.0, 12
    elif case == "center4_lowT":
        H = W = 3; free = (1, 1); nb_idx = [(0, 1), (2, 1), (1, 0), (1, 2)]; T, a, sweeps = 0.05, 4.0, 30
    else:
        H = W = 3; free = (1, 1); nb_idx = [(0, 1), (2, 1), (1, 0), (1, 2)]; T, a, sweeps = 0.3, 1.0, 12
    if "_q" in case:
        q = float(case.split("_q")[1].split("_")[0])
        T = T * (q / 0.5) ** 2          # same curvature of the energy well
    if case.endswith("noOR"):
        or_mode = orc.OR_NONE
    rng = np.random.default_rng(11)
    phi0 = rng.uniform(0.5, 5.5, (H, W))
    mask = np.ones((H, W), np.uint8); mask[free] = 0
    finals = _final_states(H, W, mask, phi0, T, a, sweeps, chains=2500, or_mode=or_mode, q=q)
    v = finals[:, free[0], free[1]]
    cdf = _conditional_cdf([phi0[i] for i in nb_idx], T, q=q)
    assert stats.kstest(v, cdf).pvalue > 0.01


@pytest.mark.parametrize("q", [0.5, 0.3, 0.15])
def test_infinite_temperature_energy_for_any_coupling(q):
    # T -> infinity: independent uniform angles, E cos(q(phi_i - phi_j)) = |E exp(i q phi)|^2
    # = (sin(pi q) / (pi q))^2 per bond (4 / pi^2 at q = 1/2)
    L, T, n = 16, 1e6, 300
    mask = np.zeros((L, L), np.uint8)
    phi = np.zeros((L, L))
    orc.init_gaps(phi, mask, seed=5)
    ngp = orc.n_gp(L, L)
    e = []
    for s in range(n):
        orc.sweep(phi, mask, a=1.0, T=T, q=q, seed=5, sweep_index=s)
        e.append(orc.energy(phi, q=q) / ngp)
    expect = -(math.sin(math.pi * q) / (math.pi * q)) ** 2
    # one state: per-bond variance <= 1/2 over 480 bonds (correlated through shared sites:
    # sd <= 0.05); n nearly independent states
    assert abs(np.mean(e) - expect) < 4 * 0.05 / math.sqrt(n)


def test_two_free_sites_match_joint_density_marginals():
    # 2 x 2 grid, the two top sites free (adjacent, different colours), bottom row samples
    H = W = 2
    phi0 = np.array([[0.0, 0.0], [1.2, 4.0]])
    mask = np.array([[0, 0], [1, 1]], np.uint8)
    T, q = 0.35, 0.5
    finals = _final_states(H, W, mask, phi0, T, 1.0, 16, chains=2500)
    n = 1201
    x = np.linspace(0, TWO_PI, n)
    A, B = np.meshgrid(x, x, indexing="ij")   # A = phi(0,0), B = phi(0,1)
    E = -(np.cos(q * (A - B)) + np.cos(q * (A - phi0[1, 0])) + np.cos(q * (B - phi0[1, 1])))
    p = np.exp(-(E - E.min()) / T)
    for axis, site in ((1, (0, 0)), (0, (0, 1))):
        marg = integrate.trapezoid(p, x, axis=axis)
        c = integrate.cumulative_trapezoid(marg, x, initial=0.0); c /= c[-1]
        v = finals[:, site[0], site[1]]
        assert stats.kstest(v, lambda t: np.interp(t, x, c)).pvalue > 0.01


def test_high_temperature_energy_expansion():
    # Unconditional chain at large T: e = -4/pi^2 - Var_0(H)/(T N_GP) + O(T^-2) with the
    # infinite-temperature variance of independent uniform angles (q = 1/2):
    #   Var cos = 1/2 - 16/pi^4 per bond, Cov = 2/pi^2 - 16/pi^4 for bonds sharing a site.
    L, T = 16, 50.0
    mask = np.zeros((L, L), np.uint8)
    phi = np.zeros((L, L))
    orc.init_gaps(phi, mask, seed=3)
    ngp = orc.n_gp(L, L)
    deg = np.full((L, L), 4); deg[0, :] -= 1; deg[-1, :] -= 1; deg[:, 0] -= 1; deg[:, -1] -= 1
    pairs = int((deg * (deg - 1) // 2).sum())
    v1 = 0.5 - 16 / math.pi**4
    c2 = 2 / math.pi**2 - 16 / math.pi**4
    expect = -4 / math.pi**2 - (ngp * v1 + 2 * pairs * c2) / (T * ngp)
    es = []
    for s in range(4200):
        orc.sweep(phi, mask, a=1.0, T=T, seed=3, sweep_index=s)
        if s >= 200:
            es.append(orc.energy(phi) / ngp)
    assert abs(np.mean(es) - expect) < 2e-3
    assert abs(expect + 4 / math.pi**2) > 0.01               # the 1/T term is resolved


def test_low_temperature_equipartition():
    # T -> 0: H ~ -N_GP + (q^2/2) sum (dphi)^2, N-1 quadratic modes, so <e> = -1 + (N-1)T/(2 N_GP)
    L, T = 12, 1e-3
    mask = np.zeros((L, L), np.uint8)
    phi = np.full((L, L), math.pi)
    ngp = orc.n_gp(L, L)
    es = []
    for s in range(3300):
        orc.sweep(phi, mask, a=60.0, T=T, seed=4, sweep_index=s)
        if s >= 300:
            es.append(orc.energy(phi) / ngp)
    expect = -1 + (L * L - 1) * T / (2 * ngp)
    assert abs((np.mean(es) + 1) / (expect + 1) - 1) < 0.05


def test_zero_temperature_quench_aligns_full_lattice():
    L = 8
    mask = np.zeros((L, L), np.uint8)
    phi = np.zeros((L, L))
    orc.init_gaps(phi, mask, seed=21)
    prm = orc.params(i_max=3000, n_fit=10**6, seed=21)     # never stops on the slope test
    orc.equilibrate(phi, mask, 1e-9, prm)
    dmax = max(np.abs(np.diff(phi, axis=0)).max(), np.abs(np.diff(phi, axis=1)).max())
    assert dmax < 1e-2
    assert orc.energy(phi) / orc.n_gp(L, L) < -1 + 1e-5


# ---------------------------------------------------------------- Algorithm 2 pieces
def test_sg_slope_closed_forms():
    n = 20
    t = np.arange(n, dtype=np.float64)
    assert orc.sg_slope(3.0 - 0.25 * t) == pytest.approx(-0.25, abs=1e-14)
    assert orc.sg_slope(np.full(n, -0.7)) == 0.0
    assert orc.sg_slope(t * t) == pytest.approx(n - 1, abs=1e-11)   # LS slope of t^2 is 2*tbar


def test_equilibrate_control_invariants():
    c = synth.config("grid64")
    phi, zmin, zmax, _ = orc.map_angles(c["z"], c["mask"])
    orc.init_gaps(phi, c["mask"], seed=0)
    prm = orc.params(i_max=400, n_fit=20, n_f=5)
    out, next_sweep, ehist = orc.equilibrate(phi, c["mask"], 0.1, prm)
    assert next_sweep == out.sweeps and 1 <= out.sweeps <= prm.i_max + 1
    if out.sweeps <= prm.i_max:                               # stopped by the slope test
        last = out.sweeps - 1
        assert out.k >= 0 and last >= prm.n_fit and last % prm.n_f == 0
        assert out.k == pytest.approx(orc.sg_slope(ehist[last + 2 - prm.n_fit: last + 2]), abs=0)
    assert out.a >= 1.0
    # the window factor only ever takes values 1 + i/k_a
    assert out.a == 1.0 or abs((out.a - 1.0) * prm.k_a - round((out.a - 1.0) * prm.k_a)) < 1e-9
    assert ehist[1] > ehist[-1]                               # relaxation lowers the energy


def test_window_factor_follows_step_5_2():
    # at a tiny temperature acceptance stays below A_targ, so a(i+1) = 1 + (i+1)/k_a every sweep
    c = synth.config("grid64")
    phi, _, _, _ = orc.map_angles(c["z"], c["mask"])
    orc.init_gaps(phi, c["mask"], seed=0)
    prm = orc.params(i_max=6, n_fit=1000, k_a=3.0)
    out, _, _ = orc.equilibrate(phi, c["mask"], 1e-7, prm)
    assert out.sweeps == 7 and out.a == pytest.approx(1 + 7 / 3.0, abs=1e-15)


def test_invert_T_interpolation():
    Tk = np.array([0.1, 0.2, 0.4, 0.8])
    ek = np.array([-0.98, -0.96, -0.90, -0.80])
    assert orc.invert_T(Tk, ek, -0.96) == pytest.approx(0.2)
    assert orc.invert_T(Tk, ek, -0.93) == pytest.approx(0.3)
    assert orc.invert_T(Tk, ek, -0.99) == 0.1
    assert orc.invert_T(Tk, ek, -0.5) == 0.8


def test_e_table_monotone_and_bounded():
    prm = orc.params(KT=8, T_W=16, T_H=16, M_T=40, i_max=600, T_min=1e-3, T_max=20.0, seed=8)
    Tk, ek, sw = orc.e_table(prm)
    assert np.all(np.diff(ek) > 0)
    assert ek[0] > -1 and ek[0] < -1 + 1e-3
    assert ek[-1] < -4 / math.pi**2
    assert np.all(sw >= 1)


def test_predict_back_transforms_each_realization():
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    phi, zmin, zmax, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, seed=0)
    prm = orc.params(M=1)
    ref = phi.copy()
    orc.sweep(ref, mask, a=1.0, T=0.1, seed=0, sweep_index=5)
    zhat, nxt = orc.predict(phi, mask, z, 0.1, prm, zmin, zmax, M=1, sweep_index=5)
    assert nxt == 6
    g = mask == 0
    assert np.allclose(zhat[g], zmin + ref[g] * (zmax - zmin) / TWO_PI, rtol=0, atol=1e-12)
    assert np.array_equal(zhat[~g], z[~g].astype(np.float64))
    assert zhat[g].min() >= zmin and zhat[g].max() <= zmax


# ---------------------------------------------------------------- whole method vs Tables 2-3
def _paper_rows():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_table2_3.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, prec, p, maae, mrase = line.split()
                rows.append((t, float(p), float(maae), float(mrase)))
    return rows


@pytest.mark.parametrize("p", [0.33, 0.66])
def test_fill_reproduces_paper_validation_measures(p):
    # Same data model as Tables 2-3 (nu = 0.5, kappa = 0.2, N(50, 10^2)); a 160^2 grid keeps
    # the oracle fast.  The paper averages 100 masks at L = 1024, so allow 6%.
    rows = [r for r in _paper_rows() if r[1] == p]
    maae = np.mean([r[2] for r in rows]); mrase = np.mean([r[3] for r in rows])
    L = 160
    z = synth.wm_field(L, 0.5, 5.0, seed=31)
    mask = synth.mask_uniform(L, L, p, seed=1_000_031)
    prm = orc.params(M=100, KT=16, T_W=32, T_H=32, M_T=50, i_max=2000, seed=31)
    zhat, _, out = orc.fill(z, mask, prm)
    g = mask == 0
    err = zhat[g] - z[g]
    assert abs(np.abs(err).mean() / maae - 1) < 0.06
    assert abs(np.sqrt((err**2).mean()) / mrase - 1) < 0.06
    assert 0.01 < out.T_hat < 0.5


# ---------------------------------------------------------------- independent chains (R-CH)
def test_predict_chains_one_chain_is_predict():
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    phi, zmin, zmax, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, seed=3)
    prm = orc.params(seed=3, M=7)
    zc = orc.predict_chains(phi, mask, z, 0.2, prm, zmin, zmax, K=1, M_per_chain=7, sweep_index=11)
    zp, _ = orc.predict(phi.copy(), mask, z, 0.2, prm, zmin, zmax, M=7, sweep_index=11)
    assert np.array_equal(zc, zp)


def test_predict_chains_is_the_mean_of_forked_chains():
    # fork k continues the state with chain word k * 2^24 from the same sweep counter
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    phi, zmin, zmax, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, seed=4)
    prm = orc.params(seed=4, M=5)
    K, m = 3, 5
    zc = orc.predict_chains(phi, mask, z, 0.15, prm, zmin, zmax, K=K, M_per_chain=m, sweep_index=20)
    forks = [orc.predict(phi.copy(), mask, z, 0.15, prm, zmin, zmax, M=m, chain=k << 24,
                         sweep_index=20)[0] for k in range(K)]
    assert np.allclose(zc, np.mean(forks, axis=0), rtol=0, atol=1e-12)
    assert not np.array_equal(forks[0], forks[1])          # the forks draw different streams


def test_predict_chains_single_free_site_posterior_mean():
    # one free site with four sample neighbours: the mean over K chains x m sweeps of the
    # site's angle converges to the mean of the Eq. 3 density (quadrature)
    H = W = 3
    rng = np.random.default_rng(5)
    phi0 = rng.uniform(1.0, 3.0, (H, W))
    mask = np.ones((H, W), np.uint8); mask[1, 1] = 0
    nb = [phi0[0, 1], phi0[2, 1], phi0[1, 0], phi0[1, 2]]
    T = 0.3
    x = np.linspace(0.0, TWO_PI, 400001)
    p = np.exp(np.cos(0.5 * (x[:, None] - np.array(nb)[None, :])).sum(1) / T)
    mean = integrate.trapezoid(x * p, x) / integrate.trapezoid(p, x)
    sd = np.sqrt(integrate.trapezoid((x - mean) ** 2 * p, x) / integrate.trapezoid(p, x))
    phi0[1, 1] = mean                                       # start at a typical value
    z = phi0.astype(np.float32)                             # map: zmin = 0, zmax = 2 pi
    prm = orc.params(seed=6, a_eq=1.0)
    K, m = 200, 200
    zc = orc.predict_chains(phi0, mask, z, T, prm, 0.0, TWO_PI, K=K, M_per_chain=m)
    # correlation time of the hybrid update here is a few sweeps: 8 standard errors of
    # K * m / 5 effectively independent draws
    assert abs(zc[1, 1] - mean) < 8 * sd / np.sqrt(K * m / 5), (zc[1, 1], mean, sd)


def test_predict_chains_burn_in_is_skipped_sweeps():
    # burn_in b then m averaged sweeps = the mean of each fork's sweeps b+1 .. b+m
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    phi, zmin, zmax, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, seed=9)
    prm = orc.params(seed=9)
    K, b, m = 2, 3, 4
    zc = orc.predict_chains(phi, mask, z, 0.15, prm, zmin, zmax, K=K, M_per_chain=m, sweep_index=7,
                            burn_in=b)
    forks = []
    for k in range(K):
        f = phi.copy()
        for s in range(b):
            orc.sweep(f, mask, a=1.0, T=0.15, seed=9, chain=k << 24, sweep_index=7 + s)
        forks.append(orc.predict(f, mask, z, 0.15, prm, zmin, zmax, M=m, chain=k << 24,
                                 sweep_index=7 + b)[0])
    assert np.allclose(zc, np.mean(forks, axis=0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("or_mode,T,sweeps,bound", [
    (orc.OR_CONSERVING, 0.3, 200, 1e-12),
    (orc.OR_NONE, 0.3, 200, 1e-12),
])
def test_rounding_differences_do_not_grow(or_mode, T, sweeps, bound):
    # Two runs whose gap angles start 1e-15 rad apart (rounding-sized) stay within ~1e-13
    # rad: the reflection about the field and the proposal rotation are isometries, so
    # differences are carried, not amplified.  This is what lets an FP64 implementation
    # of the same steps follow this oracle's trajectory to rounding.
    c = synth.config("grid64")
    z, mask = c["z"], c["mask"]
    gap = mask == 0
    phi, _, _, _ = orc.map_angles(z, mask)
    orc.init_gaps(phi, mask, 13)
    rng = np.random.default_rng(0)
    p2 = phi.copy()
    p2[gap] = (p2[gap] + rng.uniform(-1e-15, 1e-15, int(gap.sum())) * (p2[gap] + 1)) % TWO_PI
    for s in range(sweeps):
        a = 1.0 + s / 3.0 if s < 30 else 1.0
        orc.sweep(phi, mask, a, T, seed=13, sweep_index=s, or_mode=or_mode)
        orc.sweep(p2, mask, a, T, seed=13, sweep_index=s, or_mode=or_mode)
    d = np.abs(phi - p2)[gap] % TWO_PI
    assert np.minimum(d, TWO_PI - d).max() < bound


def test_printed_reflection_amplifies_rounding():
    # Eq. 6 as printed (the q = 1 reflection) is chaotic: on an all-free 64 x 64 lattice at
    # T = 0.3 the same 1e-15 start separates the two runs completely within 100 sweeps
    mask = np.zeros((64, 64), np.uint8)
    phi = np.zeros((64, 64))
    orc.init_gaps(phi, mask, 7)
    rng = np.random.default_rng(0)
    p2 = (phi + rng.uniform(-1e-15, 1e-15, phi.shape) * (phi + 1)) % TWO_PI
    for s in range(100):
        a = 1.0 + s / 3.0 if s < 30 else 1.0
        orc.sweep(phi, mask, a, 0.3, seed=3, sweep_index=s, or_mode=orc.OR_LITERAL)
        orc.sweep(p2, mask, a, 0.3, seed=3, sweep_index=s, or_mode=orc.OR_LITERAL)
    d = np.abs(phi - p2) % TWO_PI
    assert np.minimum(d, TWO_PI - d).max() > 1e-3
