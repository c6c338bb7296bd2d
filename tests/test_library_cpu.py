"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without a GPU and
exports every entry point that include/msp.h declares; the config defaults are the
Section 5 parameters."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "msp.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|long long|const char\*)\s+(msp_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("msp_setup", "msp_update_values", "msp_solve", "msp_free"):
        assert n in names


def test_library_loads_and_exports_declared_symbols():
    import ctypes
    from paper_2208_08594_gb300 import _native
    L = _native.lib()  # builds with nvcc if stale
    for n in _declared():
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value
    assert set(_native.EXPORTS) == set(_declared())


def test_config_defaults_and_status_strings():
    from paper_2208_08594_gb300 import _native
    cfg = _native.msp_config_default()
    assert (cfg.restart, cfg.max_it, cfg.coarse_max, cfg.npass) == (30, 1000, 10000, 2)
    assert cfg.decoupling == 1 and cfg.precond == 0 and cfg.precision == 0
    assert _native.msp_status_string(0) == "ok"
    assert "pattern" in _native.msp_status_string(-2)


def test_invalid_arguments_rejected_without_gpu_work():
    import ctypes
    from paper_2208_08594_gb300 import _native
    L = _native.lib()
    h = ctypes.c_void_p()
    cfg = _native.msp_config_default()
    assert L.msp_setup(ctypes.byref(h), ctypes.byref(cfg), 0, 4, None, None, None, 0, None) == -1
    cfg.restart = 1000
    assert L.msp_setup(ctypes.byref(h), ctypes.byref(cfg), 10, 4, None, None, None, 10, None) == -1
    assert L.msp_free(None) == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without the compiled library the binding raises instead of
    computing anything (the solver exists only as CUDA kernels)."""
    from paper_2208_08594_gb300 import _native, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing_libmsp.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(ImportError):
        _native.lib(build_if_missing=False)


def test_estimate_grows_with_the_system():
    from paper_2208_08594_gb300 import _native
    small = _native.msp_estimate_device_bytes(1000, 4, 7000)
    big = _native.msp_estimate_device_bytes(100000, 4, 700000)
    wider = _native.msp_estimate_device_bytes(1000, 6, 7000)
    assert 0 < small < big and small < wider
    # at least the values, the ILU factors and the Krylov bases
    n = 100000 * 4
    assert big >= 700000 * 16 * 8 * 2 + n * 8 * 2 * 30
