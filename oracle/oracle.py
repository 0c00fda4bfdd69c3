"""ctypes wrapper of the FP64 C oracle (``mpr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.  It shares
no code with the CUDA path.

All functions take numpy arrays laid out row-major ``[H][W]``; ``mask`` is
uint8 with 1 marking a sample site and 0 a gap (prediction) site.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpr_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libmpr_oracle.so")
_lock = threading.Lock()
_lib = None

OR_CONSERVING, OR_LITERAL, OR_NONE = 0, 1, 2
F_REFLECTED, F_WRAPPED, F_ACCEPTED, F_VISITED = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` (Algorithm 2 step 1.1 plus the table readings)."""
    _fields_ = [
        ("seed", ctypes.c_uint64), ("q", ctypes.c_double), ("A_targ", ctypes.c_double),
        ("k_a", ctypes.c_double), ("n_f", ctypes.c_int), ("n_fit", ctypes.c_int),
        ("i_max", ctypes.c_int), ("M", ctypes.c_int), ("or_mode", ctypes.c_int),
        ("a_eq", ctypes.c_double), ("KT", ctypes.c_int), ("T_min", ctypes.c_double),
        ("T_max", ctypes.c_double), ("T_W", ctypes.c_int), ("T_H", ctypes.c_int),
        ("M_T", ctypes.c_int),
    ]


class EquilOut(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("a", ctypes.c_double), ("k", ctypes.c_double),
                ("A_last", ctypes.c_double), ("e_last", ctypes.c_double)]


class RelaxState(ctypes.Structure):
    """Mirror of ``orc_relax``: the Algorithm 2 step 5 loop state (e: history buffer)."""
    _fields_ = [("i", ctypes.c_int), ("k", ctypes.c_double), ("a", ctypes.c_double),
                ("A", ctypes.c_double), ("e", ctypes.c_void_p)]


class FillOut(ctypes.Structure):
    _fields_ = [("zmin", ctypes.c_double), ("zmax", ctypes.c_double), ("e_s", ctypes.c_double),
                ("T_hat", ctypes.c_double), ("n_sp", ctypes.c_longlong), ("n_gap", ctypes.c_long),
                ("eq", EquilOut)]


def params(**kw) -> Params:
    """Default parameters (the readings listed in the oracle's header)."""
    d = dict(seed=0, q=0.5, A_targ=0.3, k_a=3.0, n_f=5, n_fit=20, i_max=10000, M=100,
             or_mode=OR_CONSERVING, a_eq=1.0, KT=16, T_min=1e-4, T_max=1.0, T_W=64, T_H=64,
             M_T=100)
    d.update(kw)
    return Params(**d)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i, u32, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            vp = ctypes.c_void_p
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_philox_batch.argtypes = [vp, u64, vp, ctypes.c_long]
            L.orc_map.argtypes = [vp, vp, i, i, vp, P(d), P(d)]
            L.orc_map.restype = ctypes.c_long
            L.orc_unmap.argtypes = [d, d, d]
            L.orc_unmap.restype = d
            L.orc_sample_energy.argtypes = [vp, vp, i, i, d, P(ctypes.c_longlong)]
            L.orc_sample_energy.restype = d
            L.orc_energy.argtypes = [vp, i, i, d]
            L.orc_energy.restype = d
            L.orc_n_gp.argtypes = [i, i]
            L.orc_n_gp.restype = ctypes.c_long
            L.orc_local_energy.argtypes = [d, vp, i, d]
            L.orc_local_energy.restype = d
            L.orc_over_relax.argtypes = [d, vp, i, d, i]
            L.orc_over_relax.restype = d
            L.orc_sweep.argtypes = [vp, vp, i, i, d, d, d, u64, u32, u32, i, vp, vp]
            L.orc_sweep.restype = ctypes.c_long
            L.orc_sweep_rows.argtypes = [vp, vp, i, i, i, i, i, i, d, d, d, u64, u32, u32, i]
            L.orc_sweep_rows.restype = ctypes.c_long
            L.orc_energy_rows.argtypes = [vp, i, i, i, i, d]
            L.orc_energy_rows.restype = d
            L.orc_relax_step.argtypes = [P(RelaxState), ctypes.c_long, ctypes.c_long, d, P(Params)]
            L.orc_relax_step.restype = i
            L.orc_init_gaps.argtypes = [vp, vp, i, i, u64, u32]
            L.orc_sg_slope.argtypes = [vp, i]
            L.orc_sg_slope.restype = d
            L.orc_equilibrate.argtypes = [vp, vp, i, i, d, P(Params), u32, P(u32), P(EquilOut), vp]
            L.orc_predict.argtypes = [vp, vp, vp, i, i, d, P(Params), u32, P(u32), d, d, i, vp]
            L.orc_predict_chains.argtypes = [vp, vp, vp, i, i, d, P(Params), u32, u32, d, d, i, i, i, vp]
            L.orc_T_grid.argtypes = [P(Params), vp]
            L.orc_e_table.argtypes = [P(Params), vp, vp, vp]
            L.orc_invert_T.argtypes = [vp, vp, i, d]
            L.orc_invert_T.restype = d
            L.orc_fill.argtypes = [vp, vp, i, i, P(Params), d, i, vp, vp, P(FillOut)]
            L.orc_fill.restype = i
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def philox4x32_10(ctr, key):
    ctr = _c(ctr, np.uint32); key = _c(key, np.uint32); out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(ctr), _p(key), _p(out))
    return out


def philox_batch(ctr, seed):
    """ctr: uint32 [n, 4] -> uint32 [n, 4] with key = (seed lo, seed hi)."""
    ctr = _c(ctr, np.uint32).reshape(-1, 4); out = np.zeros_like(ctr)
    lib().orc_philox_batch(_p(ctr), ctypes.c_uint64(seed), _p(out), ctr.shape[0])
    return out


def map_angles(z, mask):
    """Eq. 1.  Returns (phi [H][W] float64 with 0 at gaps, zmin, zmax, n_samples)."""
    z = _c(z, np.float32); mask = _c(mask, np.uint8); H, W = z.shape
    phi = np.zeros((H, W), np.float64); zmin = ctypes.c_double(); zmax = ctypes.c_double()
    ns = lib().orc_map(_p(z), _p(mask), W, H, _p(phi), ctypes.byref(zmin), ctypes.byref(zmax))
    return phi, zmin.value, zmax.value, ns


def unmap(phi, zmin, zmax):
    return lib().orc_unmap(float(phi), float(zmin), float(zmax))


def sweep_rows(phi, mask, row0, y_a, y_b, color, a, T, q=0.5, seed=0, chain=0, sweep_index=0,
               or_mode=OR_CONSERVING):
    """Algorithm 1 on the colour-`color` gap sites of rows [y_a, y_b) of a block holding rows
    [row0, row0 + Hb) of a grid (in place); returns the accepted proposals."""
    assert phi.dtype == np.float64 and phi.flags.c_contiguous
    mask = _c(mask, np.uint8); Hb, W = phi.shape
    return lib().orc_sweep_rows(_p(phi), _p(mask), W, Hb, row0, y_a, y_b, color, a, T, q, seed,
                                chain, sweep_index, or_mode)


def energy_rows(phi, y_a, y_b, q=0.5):
    """Eq. 2 over the bonds whose upper or left end lies in rows [y_a, y_b) of the block."""
    phi = _c(phi, np.float64); Hb, W = phi.shape
    return lib().orc_energy_rows(_p(phi), W, Hb, y_a, y_b, q)


class Relax:
    """The Algorithm 2 step 5 loop driven from outside (one step per sweep)."""

    def __init__(self, prm: Params, e0: float):
        self.prm = prm
        self.hist = np.zeros(prm.i_max + 2, np.float64)
        self.hist[0] = e0
        self.s = RelaxState(i=0, k=-1.0, a=1.0, A=0.0, e=self.hist.ctypes.data)

    def step(self, nacc: int, P: int, e_next: float) -> bool:
        """Steps 5.2-5.5; False once the loop ends."""
        return bool(lib().orc_relax_step(ctypes.byref(self.s), int(nacc), int(P), float(e_next),
                                         ctypes.byref(self.prm)))


def sample_energy(phi, mask, q=0.5):
    """Eq. 4.  Returns (e_s, N_SP)."""
    phi = _c(phi, np.float64); mask = _c(mask, np.uint8); H, W = phi.shape
    nsp = ctypes.c_longlong()
    e = lib().orc_sample_energy(_p(phi), _p(mask), W, H, q, ctypes.byref(nsp))
    return e, nsp.value


def energy(phi, q=0.5):
    phi = _c(phi, np.float64); H, W = phi.shape
    return lib().orc_energy(_p(phi), W, H, q)


def n_gp(W, H):
    return lib().orc_n_gp(W, H)


def local_energy(v, nb, q=0.5):
    nb = _c(nb, np.float64)
    return lib().orc_local_energy(float(v), _p(nb), len(nb), q)


def over_relax(phi, nb, q=0.5, mode=OR_CONSERVING):
    nb = _c(nb, np.float64)
    return lib().orc_over_relax(float(phi), _p(nb), len(nb), q, mode)


def init_gaps(phi, mask, seed, chain=0):
    """Algorithm 2 step 2.2 (in place)."""
    H, W = phi.shape
    assert phi.dtype == np.float64 and phi.flags.c_contiguous
    mask = _c(mask, np.uint8)
    lib().orc_init_gaps(_p(phi), _p(mask), W, H, ctypes.c_uint64(seed), chain)
    return phi


def sweep(phi, mask, a, T, q=0.5, seed=0, chain=0, sweep_index=0, or_mode=OR_CONSERVING,
          record=False):
    """One hybrid sweep in place.  Returns n_accepted, or (n_acc, flags, margins)."""
    H, W = phi.shape
    assert phi.dtype == np.float64 and phi.flags.c_contiguous
    mask = _c(mask, np.uint8)
    flags = np.zeros((H, W), np.uint8) if record else None
    margins = np.zeros((H, W), np.float64) if record else None
    n = lib().orc_sweep(_p(phi), _p(mask), W, H, float(a), float(T), float(q),
                        ctypes.c_uint64(seed), chain, sweep_index, or_mode,
                        _p(flags) if record else None, _p(margins) if record else None)
    return (n, flags, margins) if record else n


def sg_slope(e):
    e = _c(e, np.float64)
    return lib().orc_sg_slope(_p(e), len(e))


def equilibrate(phi, mask, T, prm: Params, chain=0, sweep_index=0):
    """Algorithm 2 step 5 in place.  Returns (EquilOut, next sweep index, e history)."""
    H, W = phi.shape
    mask = _c(mask, np.uint8)
    sw = ctypes.c_uint32(sweep_index); out = EquilOut()
    ehist = np.zeros(prm.i_max + 2, np.float64)
    lib().orc_equilibrate(_p(phi), _p(mask), W, H, float(T), ctypes.byref(prm), chain,
                          ctypes.byref(sw), ctypes.byref(out), _p(ehist))
    return out, sw.value, ehist[: out.sweeps + 1].copy()


def predict(phi, mask, z, T, prm: Params, zmin, zmax, M, chain=0, sweep_index=0):
    """Algorithm 2 steps 6-7 in place.  Returns (zhat float64 [H][W], next sweep index)."""
    H, W = phi.shape
    mask = _c(mask, np.uint8); z = _c(z, np.float32)
    sw = ctypes.c_uint32(sweep_index); zhat = np.zeros((H, W), np.float64)
    lib().orc_predict(_p(phi), _p(mask), _p(z), W, H, float(T), ctypes.byref(prm), chain,
                      ctypes.byref(sw), float(zmin), float(zmax), int(M), _p(zhat))
    return zhat, sw.value


def T_grid(prm: Params):
    Tk = np.zeros(prm.KT, np.float64)
    lib().orc_T_grid(ctypes.byref(prm), _p(Tk))
    return Tk


def e_table(prm: Params):
    """Eq. 5 table: returns (T_k, e_k, relaxation sweeps per temperature)."""
    Tk = np.zeros(prm.KT, np.float64); ek = np.zeros(prm.KT, np.float64)
    sw = np.zeros(prm.KT, np.int32)
    lib().orc_e_table(ctypes.byref(prm), _p(Tk), _p(ek), _p(sw))
    return Tk, ek, sw


def invert_T(Tk, ek, e_s):
    Tk = _c(Tk, np.float64); ek = _c(ek, np.float64)
    return lib().orc_invert_T(_p(Tk), _p(ek), len(Tk), float(e_s))


def predict_chains(phi, mask, z, T, prm: Params, zmin, zmax, K, M_per_chain, chain=0, sweep_index=0,
                   burn_in=0):
    """Independent chains (reading R-CH): phi forked into K chains with chain words
    chain + k 2^24, each from sweep counter sweep_index, burn_in sweeps not averaged, then
    M_per_chain sweeps; returns zhat (float64[H][W]), the mean over all K * M_per_chain
    realizations.  phi is unchanged."""
    phi = _c(phi, np.float64); mask = _c(mask, np.uint8); z = _c(z, np.float32)
    H, W = phi.shape
    zhat = np.zeros((H, W), np.float64)
    lib().orc_predict_chains(_p(phi), _p(mask), _p(z), W, H, float(T), ctypes.byref(prm),
                             chain, sweep_index, float(zmin), float(zmax), int(K), int(burn_in),
                             int(M_per_chain), _p(zhat))
    return zhat


def fill(z, mask, prm: Params, T_fixed=0.0, eq_sweeps=-1):
    """Algorithm 2 end to end.  Returns (zhat, phi, FillOut); raises on status != 0."""
    z = _c(z, np.float32); mask = _c(mask, np.uint8); H, W = z.shape
    zhat = np.zeros((H, W), np.float64); phi = np.zeros((H, W), np.float64); out = FillOut()
    st = lib().orc_fill(_p(z), _p(mask), W, H, ctypes.byref(prm), float(T_fixed), int(eq_sweeps),
                        _p(zhat), _p(phi), ctypes.byref(out))
    if st != 0:
        raise ValueError(f"oracle fill failed with status {st}")
    return zhat, phi, out
