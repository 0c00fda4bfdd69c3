"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import glob
import os
import re

from paper_1811_01604_gb300 import build, mpr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(mpr_[A-Za-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mpr_init", "mpr_estimate_T", "mpr_sweep", "mpr_equilibrate", "mpr_predict",
                 "mpr_free"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in mpr._SIGS}
    assert declared_functions() <= bound


def test_default_params_and_status_strings_without_gpu():
    p = mpr.mpr_default_params()
    assert p.q == 0.5 and p.A_targ == 0.3 and p.n_fit == 20 and p.M == 100
    assert mpr.lib().mpr_status_string(mpr.MPR_ENOPAIRS).decode() == "MPR_ENOPAIRS"


def test_init_rejects_bad_arguments_before_touching_the_device():
    import numpy as np
    z = np.zeros((4, 4), np.float32)
    m = np.ones((4, 4), np.uint8)
    for W, H in [(0, 4), (4, 0), (4, 70000), (140000, 2)]:
        ctx = ctypes.c_void_p()
        st = mpr.lib().mpr_init(ctypes.byref(ctx), mpr._ptr(z), mpr._ptr(m), W, H, None, None)
        assert st == mpr.MPR_EINVAL and not ctx.value
    # q outside (0, 1/2]; q < 1/2 with the tile kernels or the printed reflection
    for bad in (mpr.mpr_default_params(q=0.75), mpr.mpr_default_params(q=0.0),
                mpr.mpr_default_params(q=0.25, exec_mode=mpr.MPR_EXEC_TILE),
                mpr.mpr_default_params(q=0.25, or_mode=mpr.MPR_OR_LITERAL),
                mpr.mpr_default_params(precision=mpr.MPR_PREC_F64, exec_mode=mpr.MPR_EXEC_TILE),
                mpr.mpr_default_params(precision=mpr.MPR_PREC_F64, trig_mode=mpr.MPR_TRIG_FAST),
                mpr.mpr_default_params(precision=3)):
        ctx = ctypes.c_void_p()
        st = mpr.lib().mpr_init(ctypes.byref(ctx), mpr._ptr(z), mpr._ptr(m), 4, 4, ctypes.byref(bad), None)
        assert st == mpr.MPR_EINVAL and not ctx.value
