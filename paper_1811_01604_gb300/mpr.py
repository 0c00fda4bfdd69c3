"""Thin Python binding of the C ABI in include/mpr.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays; they are passed as raw pointers and
the library decides host or device from the pointer.  A non-zero status raises
MprError.  There is no fallback: if libmpr.so is missing the import of the
library fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MPR_OK, MPR_EINVAL, MPR_ENOMEM, MPR_ECUDA, MPR_ENODATA, MPR_ENOPAIRS, MPR_ETIMEOUT, \
    MPR_ENOTEQUIL, MPR_ESTATE = range(9)
MPR_OR_CONSERVING, MPR_OR_LITERAL, MPR_OR_NONE = 0, 1, 2
MPR_TRIG_ACCURATE, MPR_TRIG_FAST = 0, 1
MPR_EXEC_AUTO, MPR_EXEC_LIST, MPR_EXEC_TILE = 0, 1, 2
MPR_PREC_F32, MPR_PREC_F64 = 0, 1
MPR_NET_T_INPUT, MPR_NET_T_ACT, MPR_NET_T_POOL, MPR_NET_T_DACT, MPR_NET_T_OUT = 0, 1, 2, 3, 4


class MprError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class mpr_params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("q", ctypes.c_double), ("A_targ", ctypes.c_double),
        ("k_a", ctypes.c_double), ("n_f", ctypes.c_int), ("n_fit", ctypes.c_int),
        ("i_max", ctypes.c_int), ("M", ctypes.c_int), ("or_mode", ctypes.c_int),
        ("trig_mode", ctypes.c_int), ("a_eq", ctypes.c_double), ("KT", ctypes.c_int),
        ("T_min", ctypes.c_double), ("T_max", ctypes.c_double), ("T_cap", ctypes.c_int),
        ("M_T", ctypes.c_int), ("exec_mode", ctypes.c_int), ("chain", ctypes.c_uint32),
        ("tile_cfg", ctypes.c_int), ("precision", ctypes.c_int),
    ]


class mpr_sweep_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("acceptance", ctypes.c_double), ("e", ctypes.c_double)]


class mpr_equil_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("a", ctypes.c_double), ("k", ctypes.c_double),
                ("A_last", ctypes.c_double), ("e_last", ctypes.c_double),
                ("converged", ctypes.c_int)]


_lib = None

# (name, restype, argtypes) of every entry point declared in include/mpr.h
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGS = [
    ("mpr_default_params", None, [ctypes.POINTER(mpr_params)]),
    ("mpr_status_string", ctypes.c_char_p, [_I]),
    ("mpr_init", _I, [ctypes.POINTER(_VP), _VP, _VP, _I, _I, ctypes.POINTER(mpr_params), _VP]),
    ("mpr_estimate_T", _I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("mpr_set_T", _I, [_VP, _D]),
    ("mpr_sweep", _I, [_VP, _I, _D, ctypes.POINTER(mpr_sweep_stats)]),
    ("mpr_equilibrate", _I, [_VP, ctypes.POINTER(mpr_equil_stats)]),
    ("mpr_predict", _I, [_VP, _I, _VP]),
    ("mpr_predict_chains", _I, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]),
    ("mpr_fill", _I, [_VP, _VP, ctypes.POINTER(mpr_equil_stats)]),
    ("mpr_init_batch", _I, [ctypes.POINTER(_VP), _I, _VP, _VP, _VP, _VP, ctypes.POINTER(mpr_params), _VP]),
    ("mpr_batch_size", _I, [_VP]),
    ("mpr_predict_batch", _I, [_VP, _I, _VP]),
    ("mpr_fill_batch", _I, [_VP, _VP]),
    ("mpr_batch_info", _I, [_VP, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I),
                            ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("mpr_batch_info_all", _I, [_VP, _I, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("mpr_autotune", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    ("mpr_free", None, [_VP]),
    ("mpr_last_error", ctypes.c_char_p, [_VP]),
    ("mpr_get_state", _I, [_VP, _VP, ctypes.POINTER(ctypes.c_uint32)]),
    ("mpr_set_state", _I, [_VP, _VP, ctypes.c_uint32]),
    ("mpr_get_info", _I, [_VP] + [ctypes.POINTER(_D)] * 6),
    ("mpr_time_sweeps", _I, [_VP, _I, _D, ctypes.POINTER(_D)]),
    ("mpr_kernel_launches", ctypes.c_uint64, []),
    ("mpr_sweep_timing_start", None, []),
    ("mpr_sweep_timing_read", None, [_I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("mpr_debug_wait_limit", None, [ctypes.c_uint64, _I]),
    ("mpr_debug_trace", None, [_VP, ctypes.c_uint64]),
    ("mpr_release_memory", _I, []),
    ("mpr_sample_energy_static", _I, [_VP, _VP, _I, _I, _D, ctypes.POINTER(_D),
                                      ctypes.POINTER(ctypes.c_longlong), _VP]),
    ("mpr_philox", _I, [_VP, ctypes.c_uint64, _VP, ctypes.c_size_t, _VP]),
    ("mpr_strip_extremes", _I, [_VP, _VP, _I, _I, _I, _I, ctypes.POINTER(_D), _VP]),
    ("mpr_strip_init", _I, [ctypes.POINTER(_VP), _VP, _VP, _I, _I, _I, _I, _D, _D, ctypes.POINTER(mpr_params),
                            _VP]),
    ("mpr_strip_pairs", _I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    ("mpr_strip_temperature", _I, [_VP, _D, ctypes.POINTER(_D)]),
    ("mpr_strip_energy", _I, [_VP, ctypes.POINTER(_D)]),
    ("mpr_strip_gaps", ctypes.c_longlong, [_VP]),
    ("mpr_strip_begin", _I, [_VP, _I, _D, _D]),
    ("mpr_strip_half_sweep", _I, [_VP, _I, _I, _VP]),
    ("mpr_strip_control", _I, [_VP, _VP, _I, ctypes.POINTER(_I)]),
    ("mpr_strip_row_bytes", ctypes.c_size_t, [_VP]),
    ("mpr_strip_row", _I, [_VP, _I, _VP]),
    ("mpr_strip_predict", _I, [_VP, _I, _VP]),
    ("mpr_get_state_batch", _I, [_VP, _I, _VP]),
    ("mpr_get_state64", _I, [_VP, _VP, ctypes.POINTER(ctypes.c_uint32)]),
    # include/mpr_net.h
    ("mpr_net_create", _I, [ctypes.POINTER(_VP), ctypes.c_uint64, _VP]),
    ("mpr_net_create_strided", _I, [ctypes.POINTER(_VP), ctypes.c_uint64, ctypes.c_int, _VP]),
    ("mpr_net_stride", ctypes.c_int, [_VP]),
    ("mpr_net_tensor", _I, [_VP, _I, _I, _VP, ctypes.c_longlong]),
    ("mpr_net_free", None, [_VP]),
    ("mpr_net_last_error", ctypes.c_char_p, [_VP]),
    ("mpr_net_num_params", ctypes.c_longlong, [_VP]),
    ("mpr_net_get_params", _I, [_VP, _VP]),
    ("mpr_net_set_params", _I, [_VP, _VP]),
    ("mpr_net_get_grads", _I, [_VP, _VP]),
    ("mpr_net_zero_grads", _I, [_VP]),
    ("mpr_net_loss_grad", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, ctypes.POINTER(_D)]),
    ("mpr_net_adam_step", _I, [_VP, ctypes.c_float]),
    ("mpr_net_train_step", _I, [_VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, ctypes.c_float,
                                ctypes.POINTER(_D)]),
    ("mpr_net_forward", _I, [_VP, _VP, _VP, _VP, _VP, _I, _I, _I, _VP]),
    ("mpr_warmstart_init", _I, [_VP, _VP]),
    ("mpr_net_conv3x3", _I, [_VP, _I, _I, _I, _I, _VP, _VP, _I, _I, _VP, _VP]),
    ("mpr_net_conv3x3_bwd", _I, [_VP, _VP, _I, _I, _I, _I, _VP, _I, _VP, _VP, _VP, _VP]),
]


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libmpr.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"MPR CUDA library not found at {path}")
        L = ctypes.CDLL(path)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def _check(ctx, st, ok=(MPR_OK,)):
    if st not in ok:
        msg = lib().mpr_last_error(ctx).decode() if ctx else ""
        name = lib().mpr_status_string(st).decode()
        raise MprError(st, f"{name}: {msg}")
    return st


def mpr_default_params(**overrides) -> mpr_params:
    p = mpr_params()
    lib().mpr_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def mpr_init(z, mask, W: int, H: int, params: mpr_params | None = None, stream=None):
    ctx = ctypes.c_void_p()
    st = lib().mpr_init(ctypes.byref(ctx), _ptr(z), _ptr(mask), int(W), int(H),
                        ctypes.byref(params) if params is not None else None, _stream(stream))
    if st != MPR_OK:
        raise MprError(st, lib().mpr_status_string(st).decode())
    return ctx


def mpr_estimate_T(ctx):
    T, es = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().mpr_estimate_T(ctx, ctypes.byref(T), ctypes.byref(es)))
    return T.value, es.value


def mpr_set_T(ctx, T: float):
    _check(ctx, lib().mpr_set_T(ctx, float(T)))


def mpr_sweep(ctx, n: int, a: float) -> mpr_sweep_stats:
    out = mpr_sweep_stats()
    _check(ctx, lib().mpr_sweep(ctx, int(n), float(a), ctypes.byref(out)))
    return out


def mpr_equilibrate(ctx) -> mpr_equil_stats:
    out = mpr_equil_stats()
    _check(ctx, lib().mpr_equilibrate(ctx, ctypes.byref(out)), ok=(MPR_OK, MPR_ENOTEQUIL))
    return out


def mpr_predict(ctx, M: int, zhat):
    _check(ctx, lib().mpr_predict(ctx, int(M), _ptr(zhat)))


def mpr_predict_chains(ctx, K: int, M_per_chain: int, zhat, burn_in: int = 0):
    _check(ctx, lib().mpr_predict_chains(ctx, int(K), int(burn_in), int(M_per_chain), _ptr(zhat)))


def mpr_fill(ctx, zhat) -> mpr_equil_stats:
    out = mpr_equil_stats()
    _check(ctx, lib().mpr_fill(ctx, _ptr(zhat), ctypes.byref(out)), ok=(MPR_OK, MPR_ENOTEQUIL))
    return out


def _ptr_array(bufs):
    arr = (ctypes.c_void_p * len(bufs))()
    for i, b in enumerate(bufs):
        arr[i] = _ptr(b)
    return arr


def mpr_init_batch(zs, masks, params: mpr_params | None = None, stream=None):
    """zs, masks: sequences of [H][W] arrays/tensors (sizes may differ)."""
    n = len(zs)
    W = (ctypes.c_int * n)(*[int(z.shape[1]) for z in zs])
    H = (ctypes.c_int * n)(*[int(z.shape[0]) for z in zs])
    ctx = ctypes.c_void_p()
    st = lib().mpr_init_batch(ctypes.byref(ctx), n, _ptr_array(zs), _ptr_array(masks), W, H,
                              ctypes.byref(params) if params is not None else None, _stream(stream))
    if st != MPR_OK:
        raise MprError(st, lib().mpr_status_string(st).decode())
    return ctx


def mpr_batch_size(ctx) -> int:
    return int(lib().mpr_batch_size(ctx))


def mpr_predict_batch(ctx, M: int, zhats):
    _check(ctx, lib().mpr_predict_batch(ctx, int(M), _ptr_array(zhats)))


def mpr_fill_batch(ctx, zhats) -> int:
    return _check(ctx, lib().mpr_fill_batch(ctx, _ptr_array(zhats)), ok=(MPR_OK, MPR_ENOTEQUIL))


def mpr_batch_info(ctx, g: int) -> dict:
    T, es, zmin, zmax = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    sw, cv = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().mpr_batch_info(ctx, int(g), ctypes.byref(T), ctypes.byref(es), ctypes.byref(sw),
                                     ctypes.byref(cv), ctypes.byref(zmin), ctypes.byref(zmax)))
    return dict(T=T.value, e_s=es.value, sweeps=sw.value, converged=cv.value, zmin=zmin.value,
                zmax=zmax.value)


def mpr_batch_info_all(ctx) -> list:
    """mpr_batch_info of every grid of the batch, in one read of the control state."""
    n = mpr_batch_size(ctx)
    T, es, zmin, zmax = (np.zeros(n, np.float64) for _ in range(4))
    sw, cv = np.zeros(n, np.int32), np.zeros(n, np.int32)
    _check(ctx, lib().mpr_batch_info_all(ctx, n, T.ctypes.data, es.ctypes.data, sw.ctypes.data, cv.ctypes.data,
                                         zmin.ctypes.data, zmax.ctypes.data))
    return [dict(T=float(T[g]), e_s=float(es[g]), sweeps=int(sw[g]), converged=int(cv[g]), zmin=float(zmin[g]),
                 zmax=float(zmax[g])) for g in range(n)]


def mpr_autotune(ctx) -> dict:
    cfg, gs, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(ctx, lib().mpr_autotune(ctx, ctypes.byref(cfg), ctypes.byref(gs), ctypes.byref(ms)))
    return dict(tile_cfg=cfg.value, graph_sweeps=gs.value, ms_per_sweep=ms.value)


def mpr_free(ctx):
    if ctx:
        lib().mpr_free(ctx)


def mpr_last_error(ctx) -> str:
    return lib().mpr_last_error(ctx).decode()


def mpr_get_state(ctx, phi) -> int:
    sw = ctypes.c_uint32()
    _check(ctx, lib().mpr_get_state(ctx, _ptr(phi), ctypes.byref(sw)))
    return sw.value


def mpr_get_state64(ctx, phi) -> int:
    sw = ctypes.c_uint32()
    _check(ctx, lib().mpr_get_state64(ctx, _ptr(phi), ctypes.byref(sw)))
    return sw.value


def mpr_set_state(ctx, phi, sweep: int):
    _check(ctx, lib().mpr_set_state(ctx, _ptr(phi), int(sweep)))


def mpr_get_info(ctx) -> dict:
    v = [ctypes.c_double() for _ in range(6)]
    _check(ctx, lib().mpr_get_info(ctx, *[ctypes.byref(x) for x in v]))
    keys = ("H_exact", "H_tracked", "zmin", "zmax", "T", "e_s")
    return {k: x.value for k, x in zip(keys, v)}


def mpr_time_sweeps(ctx, n: int, a: float) -> float:
    ms = ctypes.c_double()
    _check(ctx, lib().mpr_time_sweeps(ctx, int(n), float(a), ctypes.byref(ms)))
    return ms.value


def mpr_sample_energy_static(z, mask, W: int, H: int, q: float = 0.5, stream=None):
    """Allocation-free e_s (Eq. 4) of device-resident data; returns (e_s, n_pairs)."""
    e = ctypes.c_double()
    n = ctypes.c_longlong()
    st = lib().mpr_sample_energy_static(_ptr(z), _ptr(mask), int(W), int(H), float(q),
                                        ctypes.byref(e), ctypes.byref(n), _stream(stream))
    if st != MPR_OK:
        raise MprError(st, lib().mpr_status_string(st).decode())
    return e.value, n.value


# ---------------------------------------------------------------- row strips of one grid
def mpr_strip_extremes(z, mask, W: int, Hb: int, row0: int, H_global: int, stream=None):
    """(zmin, zmax, n_samples) of the strip's own rows (device buffers)."""
    out = (ctypes.c_double * 3)()
    st = lib().mpr_strip_extremes(_ptr(z), _ptr(mask), int(W), int(Hb), int(row0), int(H_global), out,
                                  _stream(stream))
    if st != MPR_OK:
        raise MprError(st, lib().mpr_status_string(st).decode())
    return out[0], out[1], int(out[2])


def mpr_strip_init(z, mask, W: int, Hb: int, row0: int, H_global: int, zmin: float, zmax: float,
                   params: mpr_params | None = None, stream=None):
    ctx = ctypes.c_void_p()
    st = lib().mpr_strip_init(ctypes.byref(ctx), _ptr(z), _ptr(mask), int(W), int(Hb), int(row0), int(H_global),
                              float(zmin), float(zmax), ctypes.byref(params) if params is not None else None,
                              _stream(stream))
    if st != MPR_OK:
        raise MprError(st, lib().mpr_status_string(st).decode())
    return ctx


def mpr_strip_pairs(ctx):
    s, n = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().mpr_strip_pairs(ctx, ctypes.byref(s), ctypes.byref(n)))
    return s.value, n.value


def mpr_strip_temperature(ctx, e_s: float) -> float:
    T = ctypes.c_double()
    _check(ctx, lib().mpr_strip_temperature(ctx, float(e_s), ctypes.byref(T)))
    return T.value


def mpr_strip_energy(ctx) -> float:
    H = ctypes.c_double()
    _check(ctx, lib().mpr_strip_energy(ctx, ctypes.byref(H)))
    return H.value


def mpr_strip_gaps(ctx) -> int:
    return int(lib().mpr_strip_gaps(ctx))


def mpr_strip_begin(ctx, phase: int, H_total: float = 0.0, P_total: float = 0.0):
    _check(ctx, lib().mpr_strip_begin(ctx, int(phase), float(H_total), float(P_total)))


def mpr_strip_half_sweep(ctx, color: int, phase: int, totals):
    _check(ctx, lib().mpr_strip_half_sweep(ctx, int(color), int(phase), _ptr(totals)))


def mpr_strip_control(ctx, totals, phase: int, want_stop: bool = True):
    stop = ctypes.c_int(0)
    _check(ctx, lib().mpr_strip_control(ctx, _ptr(totals), int(phase), ctypes.byref(stop) if want_stop else None))
    return bool(stop.value)


def mpr_strip_row_bytes(ctx) -> int:
    return int(lib().mpr_strip_row_bytes(ctx))


def mpr_strip_row(ctx, which: int, buf):
    _check(ctx, lib().mpr_strip_row(ctx, int(which), _ptr(buf)))


def mpr_strip_predict(ctx, M: int, zhat):
    _check(ctx, lib().mpr_strip_predict(ctx, int(M), _ptr(zhat)))


def mpr_kernel_launches() -> int:
    return int(lib().mpr_kernel_launches())


def mpr_sweep_timing_start() -> None:
    """Enables (and resets) the library's CUDA-event timing of every sweep-kernel launch."""
    lib().mpr_sweep_timing_start()


def mpr_sweep_timing_read(stop: bool = True) -> dict:
    """The sweep-kernel timing record: total ms, launches, sweeps x sites, sweeps x gap sites."""
    ms, n, ss, gu = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
    lib().mpr_sweep_timing_read(1 if stop else 0, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(ss),
                                ctypes.byref(gu))
    return dict(ms=ms.value, launches=int(n.value), site_sweeps=ss.value, gap_updates=gu.value)


def mpr_debug_trace(buf=None) -> None:
    """Bench support: per-item timestamps of the sweep kernel into a cleared int64 CUDA
    tensor (None stops); the layout is in include/mpr.h."""
    if buf is None:
        lib().mpr_debug_trace(None, 0)
    else:
        lib().mpr_debug_trace(_ptr(buf), int(buf.numel()))


def mpr_debug_wait_limit(ns: int = 0, stall: bool = False) -> None:
    """Test support: limit of the sweep kernel's waits (0 = default) and the expiring wait."""
    lib().mpr_debug_wait_limit(int(ns), 1 if stall else 0)


def mpr_release_memory():
    """Hands the device memory kept by the library's pool (from released contexts) back
    to the driver."""
    _check(None, lib().mpr_release_memory())


def mpr_philox(ctr, seed: int, out, stream=None):
    n = (ctr.numel() if hasattr(ctr, "numel") else ctr.size) // 4
    st = lib().mpr_philox(_ptr(ctr), ctypes.c_uint64(seed), _ptr(out), n, _stream(stream))
    if st != MPR_OK:
        raise MprError(st, lib().mpr_status_string(st).decode())


def mpr_get_state_batch(ctx, g: int, phi):
    _check(ctx, lib().mpr_get_state_batch(ctx, int(g), _ptr(phi)))


# ---------------------------------------------------------------- warm-start network
def _ncheck(net, st):
    if st != MPR_OK:
        msg = lib().mpr_net_last_error(net).decode() if net else ""
        raise MprError(st, f"{lib().mpr_status_string(st).decode()}: {msg}")
    return st


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def mpr_net_create(seed: int = 0, stream=None, stride: int = 1):
    net = ctypes.c_void_p()
    if stride == 1:
        _ncheck(None, lib().mpr_net_create(ctypes.byref(net), ctypes.c_uint64(seed), _stream(stream)))
    else:
        _ncheck(None, lib().mpr_net_create_strided(ctypes.byref(net), ctypes.c_uint64(seed), int(stride),
                                                   _stream(stream)))
    return net


def mpr_net_stride(net) -> int:
    return int(lib().mpr_net_stride(net))


def mpr_net_tensor(net, kind: int, index: int, out) -> None:
    """Copies an internal tensor of the network (MPR_NET_T_*) into out (numpy array or tensor
    with exactly the tensor's element count; bf16 tensors as uint16 / int16 bit patterns)."""
    n = int(out.numel()) if hasattr(out, "numel") else int(out.size)
    _ncheck(net, lib().mpr_net_tensor(net, int(kind), int(index), _ptr(out), n))


def mpr_net_free(net):
    if net:
        lib().mpr_net_free(net)


def mpr_net_num_params(net) -> int:
    return int(lib().mpr_net_num_params(net))


def mpr_net_get_params(net, out):
    _ncheck(net, lib().mpr_net_get_params(net, _ptr(out)))


def mpr_net_set_params(net, params):
    _ncheck(net, lib().mpr_net_set_params(net, _ptr(params)))


def mpr_net_get_grads(net, out):
    _ncheck(net, lib().mpr_net_get_grads(net, _ptr(out)))


def mpr_net_zero_grads(net):
    _ncheck(net, lib().mpr_net_zero_grads(net))


def mpr_net_loss_grad(net, z, mask, phi_t, zmin, zmax, B: int, H: int, W: int, want_loss=True):
    lo = ctypes.c_double()
    zmin, zmax = _f64(zmin), _f64(zmax)
    _ncheck(net, lib().mpr_net_loss_grad(net, _ptr(z), _ptr(mask), _ptr(phi_t), _ptr(zmin), _ptr(zmax),
                                         int(B), int(H), int(W), ctypes.byref(lo) if want_loss else None))
    return lo.value if want_loss else None


def mpr_net_adam_step(net, lr: float):
    _ncheck(net, lib().mpr_net_adam_step(net, float(lr)))


def mpr_net_train_step(net, z, mask, phi_t, zmin, zmax, B: int, H: int, W: int, lr: float,
                       want_loss=True):
    lo = ctypes.c_double()
    zmin, zmax = _f64(zmin), _f64(zmax)
    _ncheck(net, lib().mpr_net_train_step(net, _ptr(z), _ptr(mask), _ptr(phi_t), _ptr(zmin), _ptr(zmax),
                                          int(B), int(H), int(W), float(lr),
                                          ctypes.byref(lo) if want_loss else None))
    return lo.value if want_loss else None


def mpr_net_forward(net, z, mask, zmin, zmax, B: int, H: int, W: int, uv):
    zmin, zmax = _f64(zmin), _f64(zmax)
    _ncheck(net, lib().mpr_net_forward(net, _ptr(z), _ptr(mask), _ptr(zmin), _ptr(zmax), int(B), int(H),
                                       int(W), _ptr(uv)))


def mpr_warmstart_init(ctx, net):
    _check(ctx, lib().mpr_warmstart_init(ctx, net))


def mpr_net_conv3x3(x, B, H, W, Cin, w, bias, Cout, relu, out, stream=None):
    st = lib().mpr_net_conv3x3(_ptr(x), int(B), int(H), int(W), int(Cin), _ptr(w), _ptr(bias), int(Cout),
                               int(relu), _ptr(out), _stream(stream))
    _ncheck(None, st)


def mpr_net_conv3x3_bwd(x, gout, B, H, W, Cin, w, Cout, din, dw, w_scratch, stream=None):
    st = lib().mpr_net_conv3x3_bwd(_ptr(x), _ptr(gout), int(B), int(H), int(W), int(Cin), _ptr(w),
                                   int(Cout), _ptr(din), _ptr(dw), _ptr(w_scratch), _stream(stream))
    _ncheck(None, st)
