"""CPU checks of the C ABI: the library builds, loads without a GPU and exports every
entry point that include/fsi.h declares; the Python binding covers the same names."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent


def declared_functions():
    text = (ROOT / "include" / "fsi.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fsi_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fsi_accel_grad", "fsi_step", "fsi_accel", "fsi_grad", "fsi_hhs_interval",
                 "fsi_create", "fsi_destroy", "fsi_sync_status"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2210_02472_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(str(lib_path))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_names_match_header():
    from paper_2210_02472_b300 import build
    build.build()
    from paper_2210_02472_b300 import fsi
    assert sorted(fsi.EXPORTED) == declared_functions()
    for n in fsi.EXPORTED:
        if n not in ("fsi_default_params", "fsi_create", "fsi_destroy", "fsi_set_params",
                     "fsi_last_error"):
            assert hasattr(fsi, n), n


def test_default_params_without_gpu():
    from paper_2210_02472_b300 import build
    build.build()
    from paper_2210_02472_b300 import fsi
    p = fsi.fsi_params()
    fsi._lib.fsi_default_params(ctypes.byref(p))
    assert p.precision == fsi.FSI_FP64 and p.max_level == 40
    assert abs(p.eta_ff - 0.2) < 1e-15 and abs(p.eta_jerk - 0.1) < 1e-15


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2210_02472_b300 import build
    build.build()
    from paper_2210_02472_b300 import fsi
    h = ctypes.c_void_p()
    code = fsi._lib.fsi_create(ctypes.byref(h), None)
    assert code == fsi.FSI_ERR_CUDA and not h.value
    assert b"context creation failed" in fsi._lib.fsi_last_error()
