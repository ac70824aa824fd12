"""The C-ABI library loads on a machine without a GPU and exports every declared symbol."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                src = f.read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(qk_\w+)\s*\(", src, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    from paper_2506_03437_b300 import _lib
    names = declared()
    assert len(names) >= 12
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(names) == sorted(_lib.EXPORTS)


def test_calls_without_gpu_fail_cleanly():
    import torch
    from paper_2506_03437_b300 import _lib
    if torch.cuda.is_available():
        return
    c = _lib.QkConfig()
    _lib.lib.qk_config_default(ctypes.byref(c))
    assert c.d == 128 and abs(c.tau_rho - 0.01) < 1e-12 and abs(c.upper_recall - 0.99) < 1e-12
    h = ctypes.c_void_p()
    st = _lib.lib.qk_create(ctypes.byref(c), ctypes.byref(h))
    assert st != _lib.OK and _lib.lib.qk_last_error()
    c.d = 100
    assert _lib.lib.qk_create(ctypes.byref(c), ctypes.byref(h)) == _lib.ERR_ARG
