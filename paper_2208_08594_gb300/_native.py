"""ctypes binding of ``libmsp.so`` (include/msp.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device arrays are passed
as CUDA ``torch.Tensor`` objects (PyTorch provides the device memory and the stream);
nothing here computes any part of the solve.  A missing library raises at import of
the first call: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MSP_OK, MSP_NOT_CONVERGED = 0, 1
MSP_ERR_ARG, MSP_ERR_PATTERN, MSP_ERR_SINGULAR_BLOCK = -1, -2, -3
MSP_ERR_NONFINITE, MSP_ERR_BREAKDOWN, MSP_ERR_NOMEM = -4, -5, -6
MSP_ERR_TIMEOUT, MSP_ERR_CUDA = -7, -8
MSP_PREC_MSP, MSP_PREC_NONE, MSP_PREC_R_ONLY, MSP_PREC_P_ONLY, MSP_PREC_N_ONLY = 0, 1, 2, 3, 4
MSP_PRECISION_FP64, MSP_PRECISION_FP32 = 0, 1
MSP_COLOURING_ALG41, MSP_COLOURING_JP = 0, 1
MSP_SMOOTHER_PGS_MC, MSP_SMOOTHER_PJAC, MSP_SMOOTHER_PGS_NO = 0, 1, 2

# every entry point declared in include/msp.h
EXPORTS = ("msp_config_default", "msp_setup", "msp_update_values", "msp_update_values_host",
           "msp_solve",
           "msp_solve_host", "msp_free", "msp_status_string", "msp_apply_precond", "msp_spmv",
           "msp_num_levels", "msp_level_info", "msp_level_get", "msp_colour0",
           "msp_last_error", "msp_stats_enable", "msp_stats_reset", "msp_stats_launches",
           "msp_stats_count", "msp_stats_get", "msp_vertices_grouping_noalloc",
           "msp_noalloc_error", "msp_wells_setup", "msp_wells_reduced",
           "msp_wells_update_values", "msp_wells_reduce_rhs", "msp_wells_recover",
           "msp_wells_free", "msp_device_bytes", "msp_estimate_device_bytes",
           "msp_server_create", "msp_server_submit", "msp_server_wait", "msp_server_get_stats",
           "msp_server_free", "msp_set_instances", "msp_solve_batch",
           "msp_stage_values_host", "msp_update_values_staged", "msp_fma_rate",
           "msp_wells_setup_scalar", "msp_wells_update_values_scalar", "msp_wells_pack_rhs",
           "msp_wells_unpack", "msp_level_tiles")

# largest n accepted by msp_vertices_grouping_noalloc (size of its fixed scratch)
NOALLOC_MAX_VERTICES = 1 << 16


class MspConfig(C.Structure):
    _fields_ = [("mu", C.c_int), ("restart", C.c_int), ("max_it", C.c_int),
                ("coarse_max", C.c_int), ("npass", C.c_int), ("pre_sweeps", C.c_int),
                ("post_sweeps", C.c_int), ("bgs_sweeps", C.c_int), ("decoupling", C.c_int),
                ("bilu_order", C.c_int), ("precond", C.c_int), ("max_levels", C.c_int),
                ("beta", C.c_double), ("agg_seed", C.c_ulonglong),
                ("coarse_hard_max", C.c_int), ("precision", C.c_int), ("colouring", C.c_int),
                ("smoother", C.c_int), ("loop_limit", C.c_int), ("autotune", C.c_int)]


class MspSolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("setup_performed", C.c_int),
                ("setup_calls", C.c_int), ("levels", C.c_int), ("colours_l0", C.c_int),
                ("rel_residual", C.c_double), ("rel_residual_est", C.c_double),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double)]


MSP_REQ_NEW_PATTERN, MSP_REQ_RELEASE = 1, 2
MSP_EXEC_RUN, MSP_EXEC_RELEASE = 0, 1


class MspRequest(C.Structure):
    _fields_ = [("key", C.c_int64), ("nb", C.c_int32), ("b", C.c_int32), ("nnzb", C.c_int64),
                ("h_row_ptr", C.c_void_p), ("h_col_idx", C.c_void_p), ("h_values", C.c_void_p),
                ("h_rhs", C.c_void_p), ("h_x", C.c_void_p), ("rel_tol", C.c_double),
                ("flags", C.c_int32)]


class MspResult(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("key", C.c_int64), ("status", C.c_int32),
                ("slot", C.c_int32), ("setup", C.c_int32), ("pad", C.c_int32),
                ("info", MspSolveInfo), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("latency_ms", C.c_double), ("device_bytes", C.c_int64)]


class MspServerStats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("submitted", "completed", "queued", "running",
                                         "rejected", "evictions", "resident_systems",
                                         "resident_bytes", "peak_charged_bytes")]


MSP_SERVER_EXEC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int32, C.POINTER(MspRequest), C.c_int32,
                                 C.c_int32, C.POINTER(C.c_int64))


class MspServerConfig(C.Structure):
    _fields_ = [("slots", C.c_int32), ("device", C.c_int32), ("hbm_budget", C.c_int64),
                ("cfg", MspConfig), ("exec", MSP_SERVER_EXEC_FN), ("exec_user", C.c_void_p)]


class MspError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%d)%s" % (where, msp_status_string(status), status,
                                                    _last_error_suffix()))


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libmsp.so (building it first if it is missing or stale and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError("libmsp.so is not built: run paper_2208_08594_gb300.build.build()")
    L = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    L.msp_config_default.argtypes = [C.POINTER(MspConfig)]
    L.msp_setup.argtypes = [C.POINTER(P), C.POINTER(MspConfig), C.c_int32, C.c_int32, P, P, P,
                            C.c_int64, P]
    L.msp_update_values.argtypes = [P, P, P]
    L.msp_update_values_host.argtypes = [P, P, P]
    L.msp_solve.argtypes = [P, P, P, D, C.POINTER(MspSolveInfo), P]
    L.msp_solve_host.argtypes = [P, P, P, D, C.POINTER(MspSolveInfo), P]
    L.msp_free.argtypes = [P]
    L.msp_status_string.argtypes = [I]
    L.msp_status_string.restype = C.c_char_p
    L.msp_apply_precond.argtypes = [P, P, P, P]
    L.msp_spmv.argtypes = [P, P, P, P]
    L.msp_num_levels.argtypes = [P]
    L.msp_level_info.argtypes = [P, I, P, P, P]
    L.msp_level_tiles.argtypes = [P, I, P, P, P]
    L.msp_level_get.argtypes = [P, I, P, P, P, P, P, P]
    L.msp_colour0.argtypes = [P, P]
    L.msp_last_error.argtypes = []
    L.msp_last_error.restype = C.c_char_p
    L.msp_stats_enable.argtypes = [I]
    L.msp_stats_reset.argtypes = []
    L.msp_stats_launches.argtypes = []
    L.msp_stats_launches.restype = C.c_longlong
    L.msp_stats_count.argtypes = []
    L.msp_stats_get.argtypes = [I, C.c_char_p, I, P, P, P, P]
    L.msp_vertices_grouping_noalloc.argtypes = [C.c_int32, P, P, P, C.POINTER(C.c_int32), P]
    L.msp_noalloc_error.argtypes = []
    L.msp_noalloc_error.restype = C.c_char_p
    L.msp_wells_setup.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int32, P, P, P,
                                  C.c_int64, P]
    L.msp_wells_reduced.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                    C.POINTER(P), C.POINTER(P), C.POINTER(P)]
    L.msp_wells_update_values.argtypes = [P, P, P]
    L.msp_wells_reduce_rhs.argtypes = [P, P, P, P]
    L.msp_wells_recover.argtypes = [P, P, P, P, P]
    L.msp_wells_free.argtypes = [P]
    L.msp_wells_setup_scalar.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int32, P, P, P,
                                         C.c_int64, P, P, P, P, P, P]
    L.msp_wells_update_values_scalar.argtypes = [P, P, P, P, P, P]
    L.msp_wells_pack_rhs.argtypes = [P, P, P, P, P]
    L.msp_wells_unpack.argtypes = [P, P, P, P, P]
    L.msp_device_bytes.argtypes = [P, C.POINTER(C.c_int64)]
    L.msp_set_instances.argtypes = [P, C.c_int32, P]
    L.msp_stage_values_host.argtypes = [P, P, P]
    L.msp_update_values_staged.argtypes = [P, P]
    L.msp_fma_rate.argtypes = [I, C.POINTER(D), P]
    L.msp_solve_batch.argtypes = [P, P, P, D, P, P]
    L.msp_estimate_device_bytes.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.POINTER(MspConfig)]
    L.msp_estimate_device_bytes.restype = C.c_int64
    L.msp_server_create.argtypes = [C.POINTER(P), C.POINTER(MspServerConfig)]
    L.msp_server_submit.argtypes = [P, C.POINTER(MspRequest), C.POINTER(C.c_int64)]
    L.msp_server_wait.argtypes = [P, C.c_int64, D, C.POINTER(MspResult)]
    L.msp_server_get_stats.argtypes = [P, C.POINTER(MspServerStats)]
    L.msp_server_free.argtypes = [P]
    for name in EXPORTS:
        if name not in ("msp_status_string", "msp_last_error", "msp_stats_launches",
                        "msp_noalloc_error", "msp_estimate_device_bytes"):
            getattr(L, name).restype = I
    _lib = L
    return L


def _last_error_suffix():
    try:
        e = lib(False).msp_last_error()
        return (": " + e.decode()) if e else ""
    except Exception:
        return ""


def msp_status_string(status: int) -> str:
    return lib().msp_status_string(int(status)).decode()


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check_dev(t, dtype, numel, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA tensor of %s" % (name, dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))


def msp_config_default(**overrides) -> MspConfig:
    cfg = MspConfig()
    lib().msp_config_default(C.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def msp_setup(cfg: MspConfig, nb: int, b: int, row_ptr, col_idx, values, stream=None):
    import torch
    _check_dev(row_ptr, torch.int32, nb + 1, "row_ptr")
    _check_dev(col_idx, torch.int32, None, "col_idx")
    nnzb = col_idx.numel()
    _check_dev(values, torch.float64, nnzb * b * b, "values")
    h = C.c_void_p()
    st = lib().msp_setup(C.byref(h), C.byref(cfg), nb, b, _ptr(row_ptr), _ptr(col_idx),
                         _ptr(values), nnzb, _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_setup")
    return h


def msp_update_values(h, values, stream=None):
    st = lib().msp_update_values(h, _ptr(values), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_update_values")


def msp_update_values_host(h, values: np.ndarray, stream=None):
    assert values.dtype == np.float64 and values.flags.c_contiguous
    st = lib().msp_update_values_host(h, _ptr(values), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_update_values_host")


def _info_dict(info):
    return {f: getattr(info, f) for f, _ in MspSolveInfo._fields_}


def msp_solve(h, b, x, rel_tol=1e-6, stream=None):
    info = MspSolveInfo()
    st = lib().msp_solve(h, _ptr(b), _ptr(x), float(rel_tol), C.byref(info), _stream(stream))
    if st < 0 and st != MSP_ERR_BREAKDOWN:
        raise MspError(st, "msp_solve")
    return _info_dict(info)


def msp_solve_host(h, b: np.ndarray, x: np.ndarray, rel_tol=1e-6, stream=None):
    assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous
    info = MspSolveInfo()
    st = lib().msp_solve_host(h, _ptr(b), _ptr(x), float(rel_tol), C.byref(info),
                              _stream(stream))
    if st < 0 and st != MSP_ERR_BREAKDOWN:
        raise MspError(st, "msp_solve_host")
    return _info_dict(info)


def msp_free(h):
    if h:
        lib().msp_free(h)


def msp_apply_precond(h, g, w, stream=None):
    st = lib().msp_apply_precond(h, _ptr(g), _ptr(w), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_apply_precond")


def msp_spmv(h, x, y, stream=None):
    st = lib().msp_spmv(h, _ptr(x), _ptr(y), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_spmv")


def msp_num_levels(h) -> int:
    return lib().msp_num_levels(h)


def msp_level_info(h, level):
    n, nnz, nc = C.c_int32(), C.c_int32(), C.c_int32()
    st = lib().msp_level_info(h, level, C.byref(n), C.byref(nnz), C.byref(nc))
    if st != MSP_OK:
        raise MspError(st, "msp_level_info")
    return n.value, nnz.value, nc.value


def msp_level_tiles(h, level):
    """(ELL slots per row, sweep lanes per row, restriction lanes per row) of a level."""
    k, g, r = C.c_int32(), C.c_int32(), C.c_int32()
    st = lib().msp_level_tiles(h, level, C.byref(k), C.byref(g), C.byref(r))
    if st != MSP_OK:
        raise MspError(st, "msp_level_tiles")
    return k.value, g.value, r.value


def msp_level_get(h, level):
    n, nnz, ncol = msp_level_info(h, level)
    perm = np.zeros(n, np.int32)
    cptr = np.zeros(max(ncol + 1, 1), np.int32)
    agg = np.zeros(n, np.int32)
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(nnz, np.int32)
    v = np.zeros(nnz)
    st = lib().msp_level_get(h, level, _ptr(perm), _ptr(cptr) if ncol else None, _ptr(agg),
                             _ptr(rp), _ptr(ci), _ptr(v))
    if st != MSP_OK:
        raise MspError(st, "msp_level_get")
    return dict(n=n, nnz=nnz, ncolours=ncol, perm=perm,
                cptr=cptr[:ncol + 1] if ncol else np.zeros(0, np.int32), agg=agg,
                row_ptr=rp, col_idx=ci, values=v)


def msp_colour0(h, nb: int):
    c = np.zeros(nb, np.int32)
    g = lib().msp_colour0(h, _ptr(c))
    if g < 0:
        raise MspError(g, "msp_colour0")
    return c, g


def msp_stats_enable(mode: int):
    st = lib().msp_stats_enable(int(mode))
    if st != MSP_OK:
        raise MspError(st, "msp_stats_enable")


def msp_stats_reset():
    lib().msp_stats_reset()


def msp_stats_launches() -> int:
    return int(lib().msp_stats_launches())


def msp_stats_get():
    """{site: (launches, total_ms, bytes, flops)} of the call sites timed since the last
    reset."""
    L = lib()
    out = {}
    for k in range(L.msp_stats_count()):
        name = C.create_string_buffer(64)
        n, ms, by, fl = C.c_longlong(), C.c_double(), C.c_double(), C.c_double()
        if L.msp_stats_get(k, name, 64, C.byref(n), C.byref(ms), C.byref(by),
                           C.byref(fl)) == MSP_OK and n.value > 0:
            out[name.value.decode()] = (n.value, ms.value, by.value, fl.value)
    return out


def msp_vertices_grouping_noalloc(n: int, row_ptr, col_idx, colour, stream=None) -> int:
    """Colouring of a structurally symmetric block pattern without any device
    allocation (for callers that cannot allocate); returns the number of colours."""
    g = C.c_int32()
    st = lib().msp_vertices_grouping_noalloc(int(n), _ptr(row_ptr), _ptr(col_idx), _ptr(colour),
                                             C.byref(g), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_vertices_grouping_noalloc: " +
                       lib().msp_noalloc_error().decode())
    return g.value


class _DeviceArray:
    """A device array owned by the library, exposed through __cuda_array_interface__ so
    that torch.as_tensor makes a zero-copy view of it."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2}


def msp_wells_setup(nb: int, b: int, nw: int, row_ptr, col_idx, values, stream=None):
    import torch
    _check_dev(row_ptr, torch.int32, nb + 1, "row_ptr")
    _check_dev(col_idx, torch.int32, None, "col_idx")
    nnzb = col_idx.numel()
    _check_dev(values, torch.float64, nnzb * b * b, "values")
    W = C.c_void_p()
    st = lib().msp_wells_setup(C.byref(W), nb, b, nw, _ptr(row_ptr), _ptr(col_idx),
                               _ptr(values), nnzb, _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_setup")
    return W


def msp_wells_setup_scalar(nr: int, b: int, nw: int, row_ptr, col_idx, values, well_ptr,
                           well_cells, arw, awr, aww, stream=None):
    """Wells with one unknown each (see include/msp.h): cell matrix A_RR, the perforations
    of every well, A_RW (b per perforation), A_WR (b per perforation) and A_WW (one per
    well), all CUDA tensors."""
    import torch
    _check_dev(row_ptr, torch.int32, nr + 1, "row_ptr")
    _check_dev(col_idx, torch.int32, None, "col_idx")
    nnzb = col_idx.numel()
    _check_dev(values, torch.float64, nnzb * b * b, "values")
    _check_dev(well_ptr, torch.int32, nw + 1, "well_ptr")
    _check_dev(well_cells, torch.int32, None, "well_cells")
    nperf = well_cells.numel()
    _check_dev(arw, torch.float64, nperf * b, "arw")
    _check_dev(awr, torch.float64, nperf * b, "awr")
    _check_dev(aww, torch.float64, nw, "aww")
    W = C.c_void_p()
    st = lib().msp_wells_setup_scalar(C.byref(W), nr, b, nw, _ptr(row_ptr), _ptr(col_idx),
                                      _ptr(values), nnzb, _ptr(well_ptr), _ptr(well_cells),
                                      _ptr(arw), _ptr(awr), _ptr(aww), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_setup_scalar")
    return W


def msp_wells_update_values_scalar(W, values, arw, awr, aww, stream=None):
    st = lib().msp_wells_update_values_scalar(W, _ptr(values), _ptr(arw), _ptr(awr), _ptr(aww),
                                              _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_update_values_scalar")


def msp_wells_pack_rhs(W, gr, gw, g, stream=None):
    st = lib().msp_wells_pack_rhs(W, _ptr(gr), _ptr(gw), _ptr(g), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_pack_rhs")


def msp_wells_unpack(W, x, xr, xw, stream=None):
    st = lib().msp_wells_unpack(W, _ptr(x), _ptr(xr), _ptr(xw), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_unpack")


def msp_wells_reduced(W, b: int):
    """(nr, row_ptr, col_idx, values) of the reduced matrix as views (torch
    tensors on the current device, not to be written) of the arrays W owns."""
    import torch
    nr, nnzb = C.c_int32(), C.c_int64()
    rp, ci, v = C.c_void_p(), C.c_void_p(), C.c_void_p()
    st = lib().msp_wells_reduced(W, C.byref(nr), C.byref(nnzb), C.byref(rp), C.byref(ci),
                                 C.byref(v))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_reduced")
    view = lambda p, n, t: torch.as_tensor(_DeviceArray(p.value, n, t), device="cuda")
    return (nr.value, view(rp, nr.value + 1, "<i4"), view(ci, nnzb.value, "<i4"),
            view(v, nnzb.value * b * b, "<f8"))


def msp_wells_update_values(W, values, stream=None):
    st = lib().msp_wells_update_values(W, _ptr(values), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_update_values")


def msp_wells_reduce_rhs(W, g, gs, stream=None):
    st = lib().msp_wells_reduce_rhs(W, _ptr(g), _ptr(gs), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_reduce_rhs")


def msp_wells_recover(W, g, xs, x, stream=None):
    st = lib().msp_wells_recover(W, _ptr(g), _ptr(xs), _ptr(x), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_wells_recover")


def msp_wells_free(W):
    if W:
        lib().msp_wells_free(W)


def msp_device_bytes(h) -> int:
    out = C.c_int64()
    st = lib().msp_device_bytes(h, C.byref(out))
    if st != MSP_OK:
        raise MspError(st, "msp_device_bytes")
    return out.value


def msp_estimate_device_bytes(nb: int, b: int, nnzb: int, cfg: MspConfig = None) -> int:
    cfg = cfg if cfg is not None else msp_config_default()
    return lib().msp_estimate_device_bytes(nb, b, nnzb, C.byref(cfg))


def msp_server_create(slots: int, hbm_budget: int, cfg: MspConfig = None, device: int = 0,
                      exec_fn=None):
    """exec_fn: optional MSP_SERVER_EXEC_FN replacing the CUDA solver (keep a reference to it
    for the server's lifetime)."""
    sc = MspServerConfig()
    sc.slots, sc.device, sc.hbm_budget = int(slots), int(device), int(hbm_budget)
    sc.cfg = cfg if cfg is not None else msp_config_default()
    if exec_fn is not None:
        sc.exec = exec_fn
    S = C.c_void_p()
    st = lib().msp_server_create(C.byref(S), C.byref(sc))
    if st != MSP_OK:
        raise MspError(st, "msp_server_create")
    return S


def msp_server_submit(S, req: MspRequest) -> int:
    t = C.c_int64()
    st = lib().msp_server_submit(S, C.byref(req), C.byref(t))
    if st != MSP_OK:
        raise MspError(st, "msp_server_submit")
    return t.value


def msp_server_wait(S, ticket: int, timeout_s: float = -1.0):
    """The result of a ticket as a dict, or None if it has not completed within timeout_s."""
    r = MspResult()
    st = lib().msp_server_wait(S, int(ticket), float(timeout_s), C.byref(r))
    if st == MSP_ERR_TIMEOUT:
        return None
    if st != MSP_OK:
        raise MspError(st, "msp_server_wait")
    out = {f: getattr(r, f) for f, _ in MspResult._fields_ if f not in ("info", "pad")}
    out["info"] = _info_dict(r.info)
    return out


def msp_server_get_stats(S):
    st_ = MspServerStats()
    st = lib().msp_server_get_stats(S, C.byref(st_))
    if st != MSP_OK:
        raise MspError(st, "msp_server_get_stats")
    return {f: getattr(st_, f) for f, _ in MspServerStats._fields_}


def msp_server_free(S):
    if S:
        lib().msp_server_free(S)


def msp_set_instances(h, offsets):
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    st = lib().msp_set_instances(h, int(off.size - 1), _ptr(off))
    if st != MSP_OK:
        raise MspError(st, "msp_set_instances")


def msp_solve_batch(h, count: int, b, x, rel_tol=1e-6, stream=None):
    """Per-instance info dicts; raises on an error status other than breakdown."""
    infos = (MspSolveInfo * int(count))()
    st = lib().msp_solve_batch(h, _ptr(b), _ptr(x), float(rel_tol),
                               C.cast(infos, C.c_void_p), _stream(stream))
    if st < 0 and st != MSP_ERR_BREAKDOWN and not any(i.status for i in infos):
        raise MspError(st, "msp_solve_batch")
    return [_info_dict(i) for i in infos]


def msp_stage_values_host(h, values: np.ndarray, stream=None):
    assert values.dtype == np.float64 and values.flags.c_contiguous
    st = lib().msp_stage_values_host(h, _ptr(values), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_stage_values_host")


def msp_update_values_staged(h, stream=None):
    st = lib().msp_update_values_staged(h, _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_update_values_staged")


def msp_fma_rate(precision: int, stream=None) -> float:
    """Measured FLOP/s (2 x FMAs) of the current device in FP64 or FP32."""
    out = C.c_double()
    st = lib().msp_fma_rate(int(precision), C.byref(out), _stream(stream))
    if st != MSP_OK:
        raise MspError(st, "msp_fma_rate")
    return out.value
