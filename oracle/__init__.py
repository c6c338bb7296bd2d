"""CPU FP64 oracle for the multi-stage preconditioned FGMRES solve (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library; the two meet only through
the seeded inputs of ``synthetic``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build

PREC_MSP, PREC_NONE, PREC_R_ONLY, PREC_P_ONLY, PREC_N_ONLY = 0, 1, 2, 3, 4
ORC_OK, ORC_NOT_CONVERGED = 0, 1


class OrcConfig(C.Structure):
    _fields_ = [("mu", C.c_int), ("restart", C.c_int), ("max_it", C.c_int),
                ("coarse_max", C.c_int), ("npass", C.c_int), ("pre_sweeps", C.c_int),
                ("post_sweeps", C.c_int), ("bgs_sweeps", C.c_int), ("decoupling", C.c_int),
                ("bilu_order", C.c_int), ("precond", C.c_int), ("max_levels", C.c_int),
                ("beta", C.c_double), ("agg_seed", C.c_ulonglong),
                ("coarse_hard_max", C.c_int), ("colouring", C.c_int),
                ("smoother", C.c_int)]


class OrcInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("setup_performed", C.c_int),
                ("setup_calls", C.c_int), ("levels", C.c_int), ("colours_l0", C.c_int),
                ("rel_residual", C.c_double), ("rel_residual_est", C.c_double),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # MSP_ORACLE_LIB: a library built from a modified copy of the oracle's source (the
        # test that plants mistakes in the oracle checks that its pins catch them)
        _lib = C.CDLL(os.environ.get("MSP_ORACLE_LIB") or build())
        P = C.c_void_p
        _lib.orc_create.restype = P
        _lib.orc_create.argtypes = [C.POINTER(OrcConfig), C.c_int, C.c_int, P, P, P,
                                    C.POINTER(C.c_int)]
        for name in ("orc_update_values", "orc_apply_precond", "orc_spmv", "orc_num_levels",
                     "orc_colours_l0", "orc_setup_calls", "orc_level_info", "orc_level_get",
                     "orc_colour0", "orc_bilu_pivots", "orc_solve"):
            getattr(_lib, name).restype = C.c_int
        _lib.orc_free.argtypes = [P]
        _lib.orc_free.restype = None
        _lib.orc_update_values.argtypes = [P, P]
        _lib.orc_solve.argtypes = [P, P, P, C.c_double, C.POINTER(OrcInfo)]
        _lib.orc_apply_precond.argtypes = [P, P, P]
        _lib.orc_spmv.argtypes = [P, P, P]
        _lib.orc_num_levels.argtypes = [P]
        _lib.orc_colours_l0.argtypes = [P]
        _lib.orc_setup_calls.argtypes = [P]
        _lib.orc_level_info.argtypes = [P, C.c_int, P, P, P]
        _lib.orc_level_get.argtypes = [P, C.c_int, P, P, P, P, P, P]
        _lib.orc_colour0.argtypes = [P, P]
        _lib.orc_bilu_pivots.argtypes = [P, P]
        _lib.orc_vertices_grouping.restype = C.c_int
        _lib.orc_vertices_grouping.argtypes = [C.c_int, P, P, P]
        _lib.orc_jp_colouring.restype = C.c_int
        _lib.orc_jp_colouring.argtypes = [C.c_int, P, P, P]
        _lib.orc_wells_create.restype = P
        _lib.orc_wells_create.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P,
                                          C.POINTER(C.c_int)]
        _lib.orc_wells_free.argtypes = [P]
        _lib.orc_wells_nnzb.restype = C.c_int
        _lib.orc_wells_nnzb.argtypes = [P]
        _lib.orc_wells_get.argtypes = [P, P, P, P]
        _lib.orc_wells_update_values.restype = C.c_int
        _lib.orc_wells_update_values.argtypes = [P, P]
        _lib.orc_wells_reduce_rhs.argtypes = [P, P, P]
        _lib.orc_wells_recover.argtypes = [P, P, P, P]
        _lib.orc_jacobi_sweep.restype = None
        _lib.orc_jacobi_sweep.argtypes = [C.c_int, P, P, P, P, P]
        _lib.orc_pgs_no_sweep.restype = None
        _lib.orc_pgs_no_sweep.argtypes = [C.c_int, P, P, P, P, P, C.c_int]
        _lib.orc_pgs_mc.restype = C.c_int
        _lib.orc_pgs_mc.argtypes = [C.c_int, P, P, P, C.c_int, P, P, P, C.c_int]
        _lib.orc_pairwise.restype = C.c_int
        _lib.orc_pairwise.argtypes = [C.c_int, P, P, P, C.c_double, C.c_ulonglong, P]
        _lib.orc_splitmix64.restype = C.c_ulonglong
        _lib.orc_splitmix64.argtypes = [C.c_ulonglong]
        _lib.orc_set_max_it.restype = C.c_int
        _lib.orc_set_max_it.argtypes = [C.c_void_p, C.c_int]
        _lib.orc_config_default.argtypes = [C.POINTER(OrcConfig)]
        _lib.orc_config_default.restype = None
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_config(**kw) -> OrcConfig:
    cfg = OrcConfig()
    lib().orc_config_default(C.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


class OracleError(RuntimeError):
    pass


class Oracle:
    """One oracle solver instance over a BSR matrix (``synthetic.BSRMatrix``-like)."""

    def __init__(self, a, **cfg):
        self.cfg = default_config(**cfg)
        self.nb, self.b = int(a.nb), int(a.b)
        self._rp, self._ci = _i32(a.row_ptr), _i32(a.col_idx)
        v = _f64(a.values)
        st = C.c_int(0)
        self._h = lib().orc_create(C.byref(self.cfg), self.nb, self.b, _p(self._rp),
                                   _p(self._ci), _p(v), C.byref(st))
        if not self._h:
            raise OracleError("orc_create failed with status %d" % st.value)

    def close(self):
        if self._h:
            lib().orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update_values(self, values):
        v = _f64(values)
        st = lib().orc_update_values(self._h, _p(v))
        if st != 0:
            raise OracleError("orc_update_values: %d" % st)

    def solve(self, rhs, tol=1e-6):
        r = _f64(rhs)
        x = np.zeros(self.nb * self.b)
        info = OrcInfo()
        lib().orc_solve(self._h, _p(r), _p(x), tol, C.byref(info))
        return x, {f: getattr(info, f) for f, _ in OrcInfo._fields_}

    def set_max_it(self, max_it):
        if lib().orc_set_max_it(self._h, int(max_it)) != 0:
            raise OracleError("orc_set_max_it")

    def apply_precond(self, g):
        g = _f64(g)
        w = np.zeros_like(g)
        lib().orc_apply_precond(self._h, _p(g), _p(w))
        return w

    def spmv(self, x):
        x = _f64(x)
        y = np.zeros_like(x)
        lib().orc_spmv(self._h, _p(x), _p(y))
        return y

    @property
    def num_levels(self):
        return lib().orc_num_levels(self._h)

    @property
    def setup_calls(self):
        return lib().orc_setup_calls(self._h)

    def colour0(self):
        c = np.zeros(self.nb, dtype=np.int32)
        g = lib().orc_colour0(self._h, _p(c))
        return c, g

    def level(self, l):
        n, nnz, ncol = C.c_int(), C.c_int(), C.c_int()
        if lib().orc_level_info(self._h, l, C.byref(n), C.byref(nnz), C.byref(ncol)) != 0:
            raise IndexError(l)
        n, nnz, ncol = n.value, nnz.value, ncol.value
        perm = np.zeros(n, np.int32)
        cptr = np.zeros(max(ncol + 1, 1), np.int32)
        agg = np.zeros(n, np.int32)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros(nnz)
        lib().orc_level_get(self._h, l, _p(perm), _p(cptr) if ncol else None, _p(agg), _p(rp),
                            _p(ci), _p(v))
        return dict(n=n, nnz=nnz, ncolours=ncol, perm=perm, cptr=cptr[:ncol + 1] if ncol else
                    np.zeros(0, np.int32), agg=agg, row_ptr=rp, col_idx=ci, values=v)

    def bilu_pivots(self):
        out = np.zeros((self.nb, self.b, self.b))
        lib().orc_bilu_pivots(self._h, _p(out))
        return out


def vertices_grouping(n, row_ptr, col_idx):
    """Algorithm 4.2 on a pattern; returns (colour[1..g], g)."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    c = np.zeros(n, np.int32)
    g = lib().orc_vertices_grouping(n, _p(rp), _p(ci), _p(c))
    return c, g


def jp_colouring(n, row_ptr, col_idx):
    """Greedy first-fit colouring of a pattern in Jones-Plassmann priority order (degree
    descending, then the high word of SplitMix64(v ^ seed), then index); returns
    (colour[1..g], g)."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    c = np.zeros(n, np.int32)
    g = lib().orc_jp_colouring(n, _p(rp), _p(ci), _p(c))
    return c, g


class Wells:
    """Elimination of the last ``n_wells`` block rows (the well unknowns of Eq.
    Jacobian-system): the Schur complement on the reservoir rows, the reduced right-hand
    side and the recovery of the well unknowns."""

    def __init__(self, a, n_wells):
        self.nb, self.b, self.nw = int(a.nb), int(a.b), int(n_wells)
        self.nr = self.nb - self.nw
        self._rp, self._ci = _i32(a.row_ptr), _i32(a.col_idx)
        v = _f64(a.values)
        st = C.c_int(0)
        self._h = lib().orc_wells_create(self.nb, self.b, self.nw, _p(self._rp), _p(self._ci),
                                         _p(v), C.byref(st))
        if not self._h:
            raise OracleError("orc_wells_create failed with status %d" % st.value)

    def close(self):
        if self._h:
            lib().orc_wells_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reduced(self):
        """(row_ptr, col_idx, values) of the Schur complement (nr block rows)."""
        nnzb = lib().orc_wells_nnzb(self._h)
        rp = np.zeros(self.nr + 1, np.int32)
        ci = np.zeros(nnzb, np.int32)
        v = np.zeros(nnzb * self.b * self.b)
        lib().orc_wells_get(self._h, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def update_values(self, values):
        v = _f64(values)
        if lib().orc_wells_update_values(self._h, _p(v)) != 0:
            raise OracleError("orc_wells_update_values")

    def reduce_rhs(self, g):
        g = _f64(g)
        gs = np.zeros(self.nr * self.b)
        lib().orc_wells_reduce_rhs(self._h, _p(g), _p(gs))
        return gs

    def recover(self, g, xs):
        g, xs = _f64(g), _f64(xs)
        x = np.zeros(self.nb * self.b)
        lib().orc_wells_recover(self._h, _p(g), _p(xs), _p(x))
        return x


PGS_NO_CHUNK = 16  # rows per chunk of the PGS-NO sweep


def jacobi_sweep(row_ptr, col_idx, values, b, x):
    """One PJAC-NO sweep (natural order) from x; returns the new x."""
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(values)
    bb, xx = _f64(b), _f64(x).copy()
    lib().orc_jacobi_sweep(len(rp) - 1, _p(rp), _p(ci), _p(v), _p(bb), _p(xx))
    return xx


def pgs_no_sweep(row_ptr, col_idx, values, b, x, forward=True):
    """One PGS-NO sweep (chunks of PGS_NO_CHUNK rows, Gauss-Seidel inside a chunk, the
    other chunks at their values from the start of the sweep) from x; returns the new x."""
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(values)
    bb, xx = _f64(b), _f64(x).copy()
    lib().orc_pgs_no_sweep(len(rp) - 1, _p(rp), _p(ci), _p(v), _p(bb), _p(xx), int(forward))
    return xx


def pgs_mc(row_ptr, col_idx, values, cptr, b, x, forward=True):
    """One PGS-MC sweep on a CSR matrix in colour order (class c = cptr[c]..cptr[c+1]-1)."""
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(values)
    cp = _i32(cptr)
    bb = _f64(b)
    xx = _f64(x).copy()
    lib().orc_pgs_mc(len(rp) - 1, _p(rp), _p(ci), _p(v), len(cp) - 1, _p(cp), _p(bb), _p(xx),
                     1 if forward else 0)
    return xx


def pairwise(row_ptr, col_idx, values, beta=0.25, seed=0):
    rp, ci, v = _i32(row_ptr), _i32(col_idx), _f64(values)
    agg = np.zeros(len(rp) - 1, np.int32)
    nc = lib().orc_pairwise(len(rp) - 1, _p(rp), _p(ci), _p(v), beta, seed, _p(agg))
    return agg, nc


def splitmix64(x):
    return lib().orc_splitmix64(x)
